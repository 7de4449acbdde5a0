/*
 * gbh.h -- C ABI of the GB300 (sm_103a) hierarchization library, libgbh.so.
 *
 * The library changes the basis of anisotropic full "combination grids" of the
 * sparse grid combination technique between the nodal basis and the
 * piecewise-linear hierarchical basis (P. Hupp, "Hierarchization for the
 * Sparse Grid Combination Technique", arXiv 1309.0392, Sec. 2-3).
 *
 * Grid layout (all entry points).  A grid of level vector l[0..d-1] has
 * n_k = 2^{l_k} + 1 points in dimension k, boundary included, and is stored
 * densely in "standard row major order" (Sec. 3) with dimension 0 contiguous:
 * element (i_0, ..., i_{d-1}) sits at offset i_0 + n_0 (i_1 + n_1 (i_2 + ...)).
 * levels[0] therefore belongs to the contiguous dimension.  The paper numbers
 * dimensions 1..d with x_1 fastest; this is the same order, 0-based.
 *
 * Memory and ownership.  Every pointer to grid data is a DEVICE pointer owned
 * by the caller; transforms work in place.  `levels` and other small arrays
 * are HOST pointers read during the call only.  Element alignment (4 bytes for
 * GBH_F32, 8 for GBH_F64) is required; nothing else.  The single-grid entry
 * points allocate no device memory.
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream).  Calls are stream-ordered and asynchronous: the return code
 * reports argument errors and launch errors; kernels may still be running when
 * the call returns.
 *
 * Errors.  Every entry point returns a gbh_status (0 = success).  On an
 * argument error nothing is launched and the data is untouched.
 */
#ifndef GBH_H
#define GBH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { GBH_F32 = 0, GBH_F64 = 1 } gbh_dtype;

typedef enum {
    GBH_OK = 0,
    GBH_EINVAL = -1,    /* null pointer, d out of [1, 16], bad op/path value   */
    GBH_EDTYPE = -2,    /* dtype not GBH_F32 / GBH_F64                          */
    GBH_EALIGN = -3,    /* data pointer not aligned to the element size         */
    GBH_ERANGE = -4,    /* a level outside [0, 30], or the point count or the
                           byte size overflows int64                            */
    GBH_ECUDA = -5,     /* a CUDA call or kernel launch failed                  */
    GBH_ETIMEOUT = -6,  /* a bounded device-side wait expired (batched plans)   */
    GBH_ENOMEM = -7,    /* host or device allocation failed (plans only)        */
    GBH_EUNSUPPORTED = -8 /* option not available for this shape or dtype       */
} gbh_status;

/* Transform selector. */
typedef enum {
    GBH_HIERARCHIZE = 0,    /* nodal -> hierarchical (Alg. 1)                    */
    GBH_DEHIERARCHIZE = 1,  /* hierarchical -> nodal (inverse of Alg. 1)         */
    GBH_ADJOINT = 2,        /* transpose of Alg. 1                               */
    GBH_DEHIERARCHIZE_ADJOINT = 3  /* transpose of the inverse (per-dimension path,
                                      native arithmetic whatever `arith` says)  */
} gbh_op;

/* ------------------------------------------------------------------------ */
/* Single grid (the paper's problem statement: "a d dimensional combination  */
/* grid of level vector (l_1, ..., l_d)", Sec. 3, Flop Count)                */
/* ------------------------------------------------------------------------ */

/*
 * Hierarchize in place: Alg. 1 (Sec. 3) in its boundary form.  For every
 * dimension and every 1-D pole along it, every interior point i of level j
 * becomes u[i] - 0.5 * (u[i - s] + u[i + s]), s = 2^{l_k - j}, computed from
 * the nodal values; boundary points are unchanged.
 *   data   : device pointer to N = prod_k (2^{l_k}+1) elements of `dtype`
 *   d      : number of dimensions, 1..16
 *   levels : host array of d levels, each 0..30 (level 0 = two points)
 *   dtype  : GBH_F32 or GBH_F64
 *   stream : cudaStream_t as void*
 */
int gbh_hierarchize(void *data, int d, const int32_t *levels, int dtype, void *stream);

/*
 * Dehierarchize in place: the exact inverse of gbh_hierarchize (the
 * hierarchical-to-nodal step of the iterated combination technique, Sec. 2).
 * Per pole, coarse to fine: u[i] = alpha[i] + 0.5 * (u[i - s] + u[i + s]).
 * Arguments as for gbh_hierarchize.
 */
int gbh_dehierarchize(void *data, int d, const int32_t *levels, int dtype, void *stream);

/*
 * Adjoint in place: the exact transpose of gbh_hierarchize.  Per pole, every
 * point p collects y[p] = x[p] - 0.5 * (sum of x over the points whose
 * hierarchical predecessor p is).  Arguments as for gbh_hierarchize.
 */
int gbh_hierarchize_adjoint(void *data, int d, const int32_t *levels, int dtype, void *stream);

/*
 * Transpose of gbh_dehierarchize, in place: per pole, fine to coarse, every
 * interior point adds half of its accumulated value to both hierarchical
 * predecessors (boundary points change too).  It is the inverse of
 * gbh_hierarchize_adjoint, and the backward step through the
 * dehierarchization that follows the scatter of the iterated combination
 * technique (Sec. 2).  Computed on the per-dimension path in native
 * arithmetic, in the serial operation order (fp64 bit-identical to a serial
 * run).  Arguments as for gbh_hierarchize.
 */
int gbh_dehierarchize_adjoint(void *data, int d, const int32_t *levels, int dtype, void *stream);

/* Execution path of gbh_transform. */
typedef enum {
    GBH_PATH_AUTO = 0,   /* planner's choice (fused when available)             */
    GBH_PATH_PLAIN = 1,  /* one sweep kernel per dimension (native arithmetic
                            unless arith = 2)                                   */
    GBH_PATH_FUSED = 2,  /* dyadic-tile kernels, all dimensions per tile
                            (hierarchize and dehierarchize, d in [2, 6];
                            GBH_EUNSUPPORTED otherwise)                         */
    GBH_PATH_GROUPED = 3 /* one pass per group of consecutive dimensions whose
                            pole sets fit in a shared-memory tile (hierarchize
                            and dehierarchize; GBH_EUNSUPPORTED for a level of
                            13 or more, d > 8 or the transpose)                 */
} gbh_path;

/* Options of gbh_transform.  Zero-initialise, then set what is wanted. */
typedef struct {
    int32_t path;          /* gbh_path                                          */
    int32_t tile_exp[16];  /* fused path: tile exponent m_k per dimension
                              (tile edge 2^{m_k}+1, 0 <= m_k <= l_k); all 0 =
                              the planner chooses                               */
    int32_t arith;         /* GBH_F64 only: 0 = the path's default (native fp64
                              on GBH_PATH_PLAIN, int64 block fixed point on the
                              others), 1 = native fp64, 2 = int64 block fixed
                              point (one binary scale per tile or pole group)    */
    int32_t variant;       /* kernel choice within a path, same results
                              within the stated tolerance.  Fused path, 3-D
                              fp64 fixed point with tile exponents (5,4,4):
                              0 = the interior class on its own kernel
                              (default), 1 = the generic tile kernel for every
                              class.  Plain path with native arithmetic:
                              0 = two consecutive dimensions per pass where
                              their poles fit a pair tile (default; results
                              bit-identical to 1), 1 = one pass per dimension */
    int32_t reserved[5];
} gbh_options;

/*
 * General form of the four single-grid calls with an explicit op and
 * execution options (NULL = defaults).  Used by tests and the tuner to pin a
 * path; the results of every path agree with the oracle within the stated
 * tolerance.
 */
int gbh_transform(void *data, int d, const int32_t *levels, int dtype, int op,
                  const gbh_options *opt, void *stream);

/*
 * Same-shape batch: `batch` grids of one level vector stored back to back
 * (grid b starts at element b * N), each transformed as by gbh_transform.
 * batch >= 1; the other arguments as for gbh_transform.  Used for the
 * differentiation workload (a batch of equal grids).
 */
int gbh_transform_batched(void *data, int64_t batch, int d, const int32_t *levels, int dtype,
                          int op, const gbh_options *opt, void *stream);

/*
 * Number of grid points prod_k (2^{l_k}+1) into *out.  Host only.
 */
int gbh_num_points(int d, const int32_t *levels, int64_t *out);

/*
 * Tile exponents the fused path would use for (d, levels, dtype, op): the
 * planner's choice, written to m_out[0..d-1].  Host only (no device work).
 * GBH_EUNSUPPORTED if the fused path does not take this shape.
 */
int gbh_tile_plan(int d, const int32_t *levels, int dtype, int op, int32_t *m_out);

/* ------------------------------------------------------------------------ */
/* Autotuner                                                                  */
/* ------------------------------------------------------------------------ */

/*
 * The tile shapes gbh_autotune times on the fused path for (d, levels, dtype,
 * op), best estimate first: up to max_count vectors of d tile exponents into
 * m_out (host array [max_count][d]), their number into *count.  Host only.
 * GBH_EUNSUPPORTED if the fused path does not take the shape.
 */
int gbh_tile_candidates(int d, const int32_t *levels, int dtype, int op, int max_count, int32_t *m_out, int *count);

/* Outcome of gbh_autotune. */
typedef struct {
    int32_t path;              /* chosen gbh_path: GBH_PATH_PLAIN, _FUSED or _GROUPED */
    int32_t tile_exp[16];      /* GBH_PATH_FUSED: chosen tile exponents m_k          */
    int32_t candidates;        /* configurations timed                               */
    double ms_tuned;           /* median time of the chosen configuration            */
    double ms_model;           /* median time of the cost model's configuration      */
    int32_t model_path;        /* the cost model's configuration                     */
    int32_t model_tile_exp[16];
    int32_t reserved[4];
} gbh_tune_result;

/*
 * Measured choice of the execution path and of the dyadic tile shape for one
 * level vector (the dimension fusion and tile shape per level vector; the
 * cost model alone ranks tiles by estimated DRAM bytes).  Times, on a scratch
 * grid of that shape allocated for the call (values in [-1, 1)), the
 * per-dimension sweeps, the six best-estimated tile shapes of the dyadic path
 * and the dimension-group path (each the median of three runs), and records
 * the fastest: later gbh_transform calls with the default path
 * (GBH_PATH_AUTO, all tile_exp 0) and the four single-grid calls use it for
 * this (d, levels, dtype, op).  The record lives in the process and is
 * shared by all threads.  Synchronous; allocates and frees the scratch grid
 * (twice the grid's bytes) on the current device.  GBH_ENOMEM if that fails.
 */
int gbh_autotune(int d, const int32_t *levels, int dtype, int op, gbh_tune_result *out);

/* Drops every recorded choice: the cost model decides again. */
int gbh_autotune_reset(void);

/* ------------------------------------------------------------------------ */
/* Combination scheme (Sec. 2): batched transform and sparse-grid gather     */
/* ------------------------------------------------------------------------ */

typedef struct gbh_plan gbh_plan;

/*
 * Plan for the regular combination scheme of dimension d and level n: every
 * level vector with l_k >= 1 and |l|_1 = n + d - 1 - q, q = 0..d-1, with
 * coefficient (-1)^q C(d-1, q) (Sec. 2, "The Combination Technique").  Grids
 * are enumerated q ascending, then lexicographically (l_0 most significant).
 * The plan owns its device work tables (allocated here; freed by
 * gbh_plan_destroy) but not the grids.
 *   d in [1, 8], n >= 1, dtype GBH_F32 or GBH_F64.  *out receives the plan.
 */
int gbh_plan_create_scheme(int d, int n, int dtype, gbh_plan **out);

/*
 * Scheme plan over a subset of the scheme's grids, for one rank of a job that
 * splits the grids over ranks (the coarse parallelism of the combination
 * technique, Sec. 2).  owned: host array of n_owned >= 1 strictly increasing
 * indexes into the enumeration of gbh_plan_create_scheme; the plan holds
 * those grids (in that order) with their coefficients and the whole sparse
 * grid.  Its gather sums only these grids (a partial sparse vector that a sum
 * over ranks completes, equal to a full plan's gather with the other
 * coefficients set to 0); its scatter and execute touch only these grids.
 * GBH_EINVAL for an empty, unordered or out-of-range list.
 */
int gbh_plan_create_scheme_subset(int d, int n, int dtype, int n_owned, const int32_t *owned, gbh_plan **out);

/*
 * Plan for an arbitrary list of grids: levels is a host array [n_grids][d],
 * d in [1, 8], every level in [0, 17] (GBH_ERANGE otherwise).  Coefficients
 * are 1; gbh_plan_gather needs a plan made by gbh_plan_create_scheme.
 */
int gbh_plan_create(int n_grids, int d, const int32_t *levels, int dtype, gbh_plan **out);

int gbh_plan_destroy(gbh_plan *plan);

/* Number of grids; level vector of grid g (d values) into levels_out. */
int gbh_plan_num_grids(const gbh_plan *plan, int *out);
int gbh_plan_grid_levels(const gbh_plan *plan, int g, int32_t *levels_out);
/* Combination coefficients of all grids (n_grids doubles) into coeffs_out. */
int gbh_plan_coeffs(const gbh_plan *plan, double *coeffs_out);
/* Replace the combination coefficients (host array of n_grids doubles; copied
 * synchronously).  A coefficient of 0 leaves that grid out of the gather, which
 * is how a rank gathers only the grids it owns. */
int gbh_plan_set_coeffs(gbh_plan *plan, const double *coeffs);
/* Points of the sparse grid (scheme plans), total grid points (all plans). */
int gbh_plan_sparse_points(const gbh_plan *plan, int64_t *out);
int gbh_plan_total_points(const gbh_plan *plan, int64_t *out);

/*
 * Bind the device pointers of the grids: host array of n_grids device
 * pointers, grid g holding gbh_num_points(levels of g) elements.  The table is
 * copied to the device on `stream`; later executions use it until the next
 * bind.  Must be called before gbh_plan_execute.
 */
int gbh_plan_bind(gbh_plan *plan, void *const *grid_ptrs, void *stream);

/*
 * Transform every bound grid in place (op = GBH_HIERARCHIZE or
 * GBH_DEHIERARCHIZE; GBH_EUNSUPPORTED for the transposes) with one persistent
 * kernel launch driven by a device work queue.  Each grid is transformed group
 * of dimensions by group of dimensions (consecutive dimensions whose pole sets
 * fit a shared-memory tile), fp64 in int64 fixed point per tile; results agree
 * with the single-grid calls within the fp64 / fp32 tolerance.  Stream-ordered;
 * device-side wait timeouts are reported by gbh_plan_status.
 */
int gbh_plan_execute(gbh_plan *plan, int op, void *stream);

/*
 * Gather (Sec. 2, "Hierarchization as preprocessing"): sparse[p] = sum over
 * the grids containing p of c_g * alpha_g(p), added in grid enumeration order
 * in fp64, starting from 0, one fused multiply-add per term.  The grids must
 * hold surpluses (hierarchized).
 * sparse: device array of gbh_plan_sparse_points doubles, subspace-major
 * layout (blocks of hierarchical subspaces j, lexicographic, j_0 most
 * significant; inside a block dimension 0 fastest; level 0 = the two
 * boundary points).  Works for GBH_F32 grids too (read and promoted).
 */
int gbh_plan_gather(gbh_plan *plan, double *sparse, void *stream);

/*
 * Scatter, the step back of the iterated combination technique (Sec. 2,
 * "Hierarchization as preprocessing"): every bound grid receives the
 * sparse-grid surpluses of its own points, alpha_g(x) = sparse[p(x)], or
 * c_g * sparse[p(x)] (one fp64 product) when scaled != 0, which makes the map
 * the transpose of gbh_plan_gather.  Every subspace of a grid of the scheme is
 * a subspace of the sparse grid, so every point of every grid is written; a
 * following gbh_plan_execute(GBH_DEHIERARCHIZE) leaves on each grid the
 * combined sparse-grid function at that grid's points (hats of finer
 * subspaces vanish there).
 *   sparse : device array of gbh_plan_sparse_points doubles in the layout of
 *            gbh_plan_gather; only read
 *   scaled : 0 = plain restriction, nonzero = times the grid's coefficient
 * Scheme plans only (GBH_EUNSUPPORTED otherwise); the grids must be bound
 * (GBH_EINVAL otherwise).  GBH_F32 grids receive the value rounded to float.
 * Stream-ordered.
 */
int gbh_plan_scatter(gbh_plan *plan, const double *sparse, int scaled, void *stream);

/*
 * Host only, no GPU: out[f] = position in the sparse grid of the scheme
 * (d, n) (the layout of gbh_plan_gather) of point f of the grid of level
 * vector `levels`, for every f < gbh_num_points(d, levels).  The grid must lie
 * in the sparse grid: 0 <= l_k <= n and sum_k max(l_k, 1) <= n + d - 1
 * (GBH_ERANGE otherwise).  d in [1, 8], n in [1, 30] (GBH_EINVAL otherwise).
 * out: host array owned by the caller.
 */
int gbh_sparse_index_of_grid(int d, int n, const int32_t *levels, int64_t *out);

/*
 * Batched transform that allocates nothing, for callers that may not call
 * cudaMalloc (a framework's caching allocator owns the device, a strict memory
 * budget, or a context where allocation is not allowed).  The paper has no
 * counterpart: a persistent batched kernel like gbh_plan_execute's (one phase
 * per dimension, int64 fixed point per grid) whose work queue, counters and
 * per-grid tables live in one fixed device array of 4 MiB inside the library
 * (held by every GPU that loads the library until exit) instead of in a
 * plan.
 *   n_grids   : 1..2048 grids; levels: host array [n_grids][d], d in [1, 8]
 *   grid_ptrs : HOST array of n_grids DEVICE pointers (grid g holds
 *               prod_k (2^{l_k}+1) elements of dtype), transformed in place
 *   op        : GBH_HIERARCHIZE or GBH_DEHIERARCHIZE
 * Results agree with those of a plan for the same grids within the fp64 /
 * fp32 tolerance.  Returns
 * GBH_ERANGE when the grids need more work items than the array holds
 * (roughly 80,000 items of 65,536 points).  The first call on a device looks
 * up the array's device address.  Every call rewrites the shared array and clears its counters: calls whose
 * kernels overlap on the GPU (other streams, other threads) race, so order
 * them on one stream.  Not thread-safe on the host.  The return code covers
 * argument and launch errors only; a bounded device-side wait that gives up
 * (the grids' contents are then unspecified) is reported by
 * gbh_batched_transform_noalloc_status.
 */
int gbh_batched_transform_noalloc(int n_grids, int d, const int32_t *levels, void *const *grid_ptrs,
                                  int dtype, int op, void *stream);

/*
 * Device-side status of the allocation-free transform on the current device:
 * GBH_ETIMEOUT if a bounded wait of any call since the last read gave up,
 * else GBH_OK (GBH_ECUDA if the status could not be read).  The word lives in
 * the same fixed array, outside the part that every call clears, so it stays
 * set across later calls until this function reads it; reading it clears it.
 * Synchronises `stream` (cudaStream_t as void*).  Allocates nothing.
 */
int gbh_batched_transform_noalloc_status(void *stream);

/*
 * Failure injection for tests of the allocation-free transform: with
 * grid >= 0, the following calls make every work item of grid `grid` wait for
 * a dependency that is never released; the waits give up after `spin_limit`
 * polls and set the status word.  grid = -1 restores normal operation.  Host
 * state only; no GPU fault, trap or hang is involved.
 */
int gbh_batched_transform_noalloc_test_stall(int grid, long long spin_limit);

/*
 * Execution parameters of gbh_plan_execute for op (GBH_HIERARCHIZE or
 * GBH_DEHIERARCHIZE): resident CTAs per SM of the persistent kernel
 * (0..32; 0 = as many as fit, more than fit = as many as fit) and the size in
 * MiB of the L2 waves the work queue is ordered in (1..4096; grids are cut
 * into waves of about that many bytes, items run along (wave, phase)
 * diagonals).  Results do not depend on them.  Host call; when the wave
 * changes it waits for the device to be idle, then rewrites the plan's work
 * list.
 */
int gbh_plan_set_params(gbh_plan *plan, int op, int ctas_per_sm, int wave_mb);
int gbh_plan_get_params(const gbh_plan *plan, int op, int *ctas_per_sm, int *wave_mb);

/* Outcome of gbh_plan_autotune. */
typedef struct {
    int32_t ctas_per_sm;       /* chosen resident CTAs per SM                         */
    int32_t wave_mb;           /* chosen L2 wave (MiB)                                */
    int32_t candidates;        /* configurations timed                                */
    int32_t max_ctas_per_sm;   /* the most that fit (the untuned setting)             */
    double ms_tuned;           /* median time of the chosen configuration             */
    double ms_model;           /* median time of the untuned configuration            */
    int32_t reserved[4];
} gbh_plan_tune_result;

/*
 * Measured choice of the execution parameters of op for this plan: times every
 * CTAs-per-SM count that fits and L2 waves of 8, 16, 32 and 64 MiB (median of
 * three executions each) on scratch grids of the plan's shapes (allocated for
 * the call: the plan's total points of dtype; values in [-1, 1)), keeps the
 * fastest in the plan and, for plans made by gbh_plan_create_scheme, for
 * every later plan of the same (d, n, dtype) in this process.  The caller's
 * bound grids are untouched and bound again afterwards.  Synchronises
 * `stream`; GBH_ENOMEM if the scratch grids cannot be allocated.
 */
int gbh_plan_autotune(gbh_plan *plan, int op, void *stream, gbh_plan_tune_result *out);

/*
 * Failure injection for tests.  With grid >= 0, the next executions of the plan
 * make every work item of that grid wait for a dependency that is never
 * released; the bounded waits give up after `spin_limit` polls, record
 * GBH_ETIMEOUT in the plan's status word and the kernel returns (the grids'
 * contents are then unspecified).  grid = -1 restores normal operation.  No
 * GPU fault, trap or hang is involved.
 */
int gbh_plan_test_stall(gbh_plan *plan, int grid, long long spin_limit);

/* Sticky device-side status of a plan: GBH_ETIMEOUT if a bounded wait of any
 * execution since the last read gave up, else GBH_OK.  Later executions do
 * not clear it; reading it does.  Synchronises the stream given. */
int gbh_plan_status(gbh_plan *plan, void *stream);

/* ------------------------------------------------------------------------ */
/* Diagnostics                                                                */
/* ------------------------------------------------------------------------ */

/* Human-readable name of a status code (static string). */
const char *gbh_status_string(int status);

/* Count of kernels this library has launched in this process. */
int gbh_launch_count(uint64_t *out);

/*
 * Kernel timing.  While enabled, the library brackets each of its kernel
 * launches with a pair of CUDA events recorded on the launch stream and
 * accumulates the durations per kernel name.  gbh_profile_read synchronises
 * on the recorded events, then reports entry `idx` (0-based; GBH_ERANGE past
 * the last): its name (copied into name_buf, NUL-terminated, truncated to
 * buf_len), its launch count and its summed duration in milliseconds.
 * gbh_profile_reset drops every entry and pending event.
 */
int gbh_profile_enable(int on);
int gbh_profile_read(int idx, char *name_buf, int buf_len, uint64_t *launches, double *total_ms,
                     double *total_bytes);
int gbh_profile_reset(void);

/* Library version as major*10000 + minor*100 + patch. */
int gbh_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GBH_H */
