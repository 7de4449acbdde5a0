/*
 * gbh_oracle.c -- plain, serial, fp64 CPU oracle for hierarchization of
 * sparse-grid combination grids (P. Hupp, "Hierarchization for the Sparse Grid
 * Combination Technique", arXiv 1309.0392).
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. The GPU library never
 * links, includes or calls it, and it shares no code with the GPU library.
 *
 * Conventions (the paper numbers dimensions 1..d with x_1 fastest; here they
 * are 0..d-1 with dimension 0 contiguous):
 *   - a combination grid of level vector l has n_k = 2^{l_k} + 1 points in
 *     dimension k (boundary included), index i_k in [0, 2^{l_k}], coordinate
 *     x = i_k 2^{-l_k};
 *   - flat offset = i_0 + n_0 (i_1 + n_1 (i_2 + ...)), "standard row major
 *     order" of Sec. 3 (Func / Ind paragraphs);
 *   - an interior index i has hierarchical level j = l - ctz(i); its two
 *     hierarchical predecessors (Sec. 3, definition under Alg. 1) are i - s
 *     and i + s with s = 2^{l-j} = lowbit(i).  The boundary points i = 0 and
 *     i = 2^l have level 0 and no predecessors.
 *
 * Readings of the paper taken here:
 *   - Boundary grids: the paper's grids have no boundary (level 1 is one point,
 *     the outermost points of a level have one predecessor).  With boundary
 *     points the missing predecessors are the boundary points, so the level
 *     loop of Alg. 1 runs l..1 instead of l..2.  orc_hierarchize_nobnd() keeps
 *     the paper's own boundary-free form for comparison.
 *   - The update is written in the reduced-op form of Sec. 3 ("Flop Count"):
 *     x[i] = x[i] - 0.5 * (left + right).
 *   - Dehierarchization is named (Sec. 2, iterated combination technique) but
 *     not given; it is the exact inverse: coarse to fine,
 *     u[i] = a[i] + 0.5 * (u[left] + u[right]).
 *   - The adjoint is the exact transpose: coarse to fine, each point scatters
 *     -0.5 times its own (still original) value into both predecessors.
 *   - The transpose of the dehierarchization runs fine to coarse: each point
 *     adds 0.5 times its accumulated value to both predecessors.
 *   - Combination scheme (Sec. 2, "The Combination Technique"): level vectors
 *     with l_k >= 1 and |l|_1 = n + d - 1 - q, q = 0..d-1, coefficient
 *     (-1)^q C(d-1, q); enumerated by q ascending, then lexicographically
 *     with l_0 most significant.
 *   - Sparse grid storage for the gather (unspecified in the paper):
 *     subspace-major.  Subspace j in N_0^d (j_k = 0 is the pair of boundary
 *     points) exists iff sum_k max(j_k,1) <= n + d - 1; blocks are in
 *     lexicographic order of j (j_0 most significant); inside a block the
 *     position p_k runs dimension 0 fastest, p_k in [0, 2) for j_k = 0
 *     (x = 0, x = 1) and p_k in [0, 2^{j_k-1}) for j_k >= 1 (x = (2p+1)2^{-j}).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no FMA contraction,
 * so every operation rounds exactly as written).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_MAXD 16

/* ------------------------------------------------------------------------ */
/* grid geometry                                                              */
/* ------------------------------------------------------------------------ */

/* Number of points of the boundary grid of level vector levels[0..d-1]. */
int64_t orc_num_points(int d, const int *levels)
{
    int64_t n = 1;
    for (int k = 0; k < d; ++k) n *= ((int64_t)1 << levels[k]) + 1;
    return n;
}

/* Element stride of dimension k (product of the lower extents). */
static int64_t stride_of(int d, const int *levels, int k)
{
    int64_t s = 1;
    for (int m = 0; m < k && m < d; ++m) s *= ((int64_t)1 << levels[m]) + 1;
    return s;
}

/* Hierarchical level of 1-D index i in a boundary pole of level l. */
static int level_of(int64_t i, int l)
{
    if (i == 0 || i == ((int64_t)1 << l)) return 0;
    int tz = 0;
    while (((i >> tz) & 1) == 0) ++tz;
    return l - tz;
}

/* ------------------------------------------------------------------------ */
/* 1-D pole transforms (the two inner loops of Alg. 1)                        */
/* ------------------------------------------------------------------------ */

/* Alg. 1 inner loops, boundary form: levels l down to 1; every point of a level
 * reads its two predecessors, which lie on coarser levels and so still hold
 * nodal values. */
static void pole_hierarchize(double *u, int64_t S, int l)
{
    const int64_t last = (int64_t)1 << l;
    for (int lev = l; lev >= 1; --lev) {
        const int64_t s = (int64_t)1 << (l - lev);
        for (int64_t i = s; i < last; i += 2 * s)
            u[i * S] = u[i * S] - 0.5 * (u[(i - s) * S] + u[(i + s) * S]);
    }
}

/* Inverse: levels 1 up to l; the predecessors already hold nodal values. */
static void pole_dehierarchize(double *u, int64_t S, int l)
{
    const int64_t last = (int64_t)1 << l;
    for (int lev = 1; lev <= l; ++lev) {
        const int64_t s = (int64_t)1 << (l - lev);
        for (int64_t i = s; i < last; i += 2 * s)
            u[i * S] = u[i * S] + 0.5 * (u[(i - s) * S] + u[(i + s) * S]);
    }
}

/* Transpose of pole_hierarchize: levels 1 up to l; a point's own value is
 * changed only by finer points, so it is still original when it scatters. */
static void pole_adjoint(double *y, int64_t S, int l)
{
    const int64_t last = (int64_t)1 << l;
    for (int lev = 1; lev <= l; ++lev) {
        const int64_t s = (int64_t)1 << (l - lev);
        for (int64_t i = s; i < last; i += 2 * s) {
            y[(i - s) * S] = y[(i - s) * S] - 0.5 * y[i * S];
            y[(i + s) * S] = y[(i + s) * S] - 0.5 * y[i * S];
        }
    }
}

/* Transpose of pole_dehierarchize (the inverse read backwards): levels l down
 * to 1; every point of a level adds half of its value, which already holds
 * the contributions of all finer points, to both predecessors. */
static void pole_dehierarchize_adjoint(double *y, int64_t S, int l)
{
    const int64_t last = (int64_t)1 << l;
    for (int lev = l; lev >= 1; --lev) {
        const int64_t s = (int64_t)1 << (l - lev);
        for (int64_t i = s; i < last; i += 2 * s) {
            y[(i - s) * S] = y[(i - s) * S] + 0.5 * y[i * S];
            y[(i + s) * S] = y[(i + s) * S] + 0.5 * y[i * S];
        }
    }
}

typedef void (*pole_fn)(double *, int64_t, int);

/* Outer two loops of Alg. 1: for each dimension, for every 1-D pole in it. */
static void sweep_all_dims(double *u, int d, const int *levels, pole_fn fn)
{
    const int64_t N = orc_num_points(d, levels);
    for (int k = 0; k < d; ++k) {
        const int64_t S = stride_of(d, levels, k);
        const int64_t n = ((int64_t)1 << levels[k]) + 1;
        const int64_t outer = N / (S * n);
        for (int64_t o = 0; o < outer; ++o)
            for (int64_t j = 0; j < S; ++j)
                fn(u + o * S * n + j, S, levels[k]);
    }
}

/* Alg. 1 (Sec. 3), boundary form, in place. */
void orc_hierarchize(double *u, int d, const int *levels)
{
    sweep_all_dims(u, d, levels, pole_hierarchize);
}

/* Exact inverse of orc_hierarchize, in place. */
void orc_dehierarchize(double *u, int d, const int *levels)
{
    sweep_all_dims(u, d, levels, pole_dehierarchize);
}

/* Exact transpose of orc_hierarchize, in place. */
void orc_hierarchize_adjoint(double *u, int d, const int *levels)
{
    sweep_all_dims(u, d, levels, pole_adjoint);
}

/* Exact transpose of orc_dehierarchize (the inverse of the transpose of
 * orc_hierarchize), in place: differentiates through the dehierarchization
 * that follows the scatter of the iterated combination technique (Sec. 2). */
void orc_dehierarchize_adjoint(double *u, int d, const int *levels)
{
    sweep_all_dims(u, d, levels, pole_dehierarchize_adjoint);
}

/* ------------------------------------------------------------------------ */
/* One-point forms: the tensor-product definitions, evaluated at one point   */
/* ------------------------------------------------------------------------ */

/* Per-dimension row of a 1-D operator: list of (index, weight). */
typedef struct { int cnt; int64_t idx[2 * 32 + 2]; double w[2 * 32 + 2]; } row1d;

/* Row i of H_k: e_i - 1/2 e_{i-s} - 1/2 e_{i+s} (identity on the boundary). */
static void row_hier(row1d *r, int64_t i, int l)
{
    r->cnt = 0;
    r->idx[r->cnt] = i; r->w[r->cnt++] = 1.0;
    if (level_of(i, l) > 0) {
        int64_t s = i & (-i);
        r->idx[r->cnt] = i - s; r->w[r->cnt++] = -0.5;
        r->idx[r->cnt] = i + s; r->w[r->cnt++] = -0.5;
    }
}

/* Row i of the nodal evaluation (inverse): u(x_i) = sum_a alpha_a phi_a(x_i).
 * phi_0 = 1 - x, phi_{2^l} = x, interior hats phi_a(x) = max(0, 1-|x-x_a|/h_a)
 * with h_a = 2^{-level(a)}. */
static void row_dehier(row1d *r, int64_t i, int l)
{
    const int64_t last = (int64_t)1 << l;
    const double x = (double)i / (double)last;
    r->cnt = 0;
    r->idx[r->cnt] = 0;    r->w[r->cnt++] = 1.0 - x;
    r->idx[r->cnt] = last; r->w[r->cnt++] = x;
    for (int lev = 1; lev <= l; ++lev) {
        const int64_t s = (int64_t)1 << (l - lev);
        /* the level-lev hat whose support contains x_i (at most one) */
        int64_t a = (i / (2 * s)) * (2 * s) + s;
        if (a >= last) continue;
        double dist = fabs((double)(i - a)) / (double)s;
        double w = 1.0 - dist;
        if (w > 0.0) { r->idx[r->cnt] = a; r->w[r->cnt++] = w; }
    }
}

/* Row p of H_k^T: column p of H_k.  Point p collects -1/2 from each point
 * whose predecessor it is. */
static void row_adjoint(row1d *r, int64_t p, int l)
{
    const int64_t last = (int64_t)1 << l;
    r->cnt = 0;
    r->idx[r->cnt] = p; r->w[r->cnt++] = 1.0;
    for (int64_t i = 1; i < last; ++i) {
        int64_t s = i & (-i);
        if (i - s == p || i + s == p) { r->idx[r->cnt] = i; r->w[r->cnt++] = -0.5; }
    }
}

typedef void (*row_fn)(row1d *, int64_t, int);

static double apply_tensor_row(const double *u, int d, const int *levels,
                               int64_t flat, row_fn fn)
{
    row1d rows[ORC_MAXD];
    int64_t strides[ORC_MAXD];
    int64_t rem = flat;
    for (int k = 0; k < d; ++k) {
        const int64_t n = ((int64_t)1 << levels[k]) + 1;
        strides[k] = stride_of(d, levels, k);
        fn(&rows[k], rem % n, levels[k]);
        rem /= n;
    }
    /* sum over the tensor product of the d rows */
    int c[ORC_MAXD];
    for (int k = 0; k < d; ++k) c[k] = 0;
    double acc = 0.0;
    for (;;) {
        double w = 1.0;
        int64_t off = 0;
        for (int k = 0; k < d; ++k) {
            w *= rows[k].w[c[k]];
            off += rows[k].idx[c[k]] * strides[k];
        }
        acc += w * u[off];
        int k = 0;
        while (k < d && ++c[k] == rows[k].cnt) { c[k] = 0; ++k; }
        if (k == d) break;
    }
    return acc;
}

/* Surplus at one point: ((H_{d-1} x ... x H_0) u)[flat]. */
double orc_hierarchize_at(const double *u, int d, const int *levels, int64_t flat)
{
    return apply_tensor_row(u, d, levels, flat, row_hier);
}

/* Nodal value at one point from surpluses: sum of tensor hats at x_flat. */
double orc_dehierarchize_at(const double *a, int d, const int *levels, int64_t flat)
{
    return apply_tensor_row(a, d, levels, flat, row_dehier);
}

/* Adjoint at one point: ((H_{d-1} x ... x H_0)^T y)[flat]. */
double orc_adjoint_at(const double *y, int d, const int *levels, int64_t flat)
{
    return apply_tensor_row(y, d, levels, flat, row_adjoint);
}

/* ------------------------------------------------------------------------ */
/* The paper's own boundary-free Alg. 1, instrumented (Sec. 3, Flop Count)    */
/* ------------------------------------------------------------------------ */

/* Grid of level vector l without boundary: 2^{l_k} - 1 points per dimension,
 * array index i-1 for i in [1, 2^l - 1]; level 1 is the single root point.
 * Level loop l..2; the outermost points of a level have one predecessor.
 * reduced_op = 0: two subtractions (as printed in Alg. 1);
 * reduced_op = 1: add both predecessors first, one multiply (Sec. 3).
 * Counts floating-point additions and multiplications into n_add / n_mul. */
void orc_hierarchize_nobnd(double *u, int d, const int *levels, int reduced_op,
                           int64_t *n_add, int64_t *n_mul)
{
    int64_t ext[ORC_MAXD], str[ORC_MAXD], N = 1;
    for (int k = 0; k < d; ++k) { ext[k] = ((int64_t)1 << levels[k]) - 1; str[k] = N; N *= ext[k]; }
    int64_t adds = 0, muls = 0;
    for (int k = 0; k < d; ++k) {
        const int l = levels[k];
        const int64_t S = str[k], n = ext[k], outer = N / (S * n);
        for (int64_t o = 0; o < outer; ++o)
            for (int64_t j = 0; j < S; ++j) {
                double *p = u + o * S * n + j;            /* p[(i-1)*S] is point i */
                for (int lev = l; lev >= 2; --lev) {
                    const int64_t s = (int64_t)1 << (l - lev);
                    for (int64_t i = s; i <= n; i += 2 * s) {
                        const int hasL = (i - s) >= 1, hasR = (i + s) <= n;
                        double *x = &p[(i - 1) * S];
                        if (reduced_op && hasL && hasR) {
                            *x = *x - 0.5 * (p[(i - s - 1) * S] + p[(i + s - 1) * S]);
                            adds += 2; muls += 1;
                        } else {
                            if (hasL) { *x = *x - 0.5 * p[(i - s - 1) * S]; adds++; muls++; }
                            if (hasR) { *x = *x - 0.5 * p[(i + s - 1) * S]; adds++; muls++; }
                        }
                    }
                }
            }
    }
    if (n_add) *n_add = adds;
    if (n_mul) *n_mul = muls;
}

/* ------------------------------------------------------------------------ */
/* Combination scheme and sparse-grid gather (Sec. 2)                         */
/* ------------------------------------------------------------------------ */

static double binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

/* Next composition of `sum` into d parts >= 1 in lexicographic order
 * (l[0] most significant).  Returns 0 when exhausted. */
static int next_composition(int *l, int d)
{
    /* find the rightmost position k < d-1 that can be increased: the suffix
     * after it must keep at least one per part */
    for (int k = d - 2; k >= 0; --k) {
        int tail = 0;
        for (int m = k + 1; m < d; ++m) tail += l[m];
        if (tail - (d - 1 - k) >= 1) {           /* suffix can give one away */
            l[k] += 1;
            tail -= 1;
            for (int m = k + 1; m < d - 1; ++m) { l[m] = 1; tail -= 1; }
            l[d - 1] = tail;
            return 1;
        }
    }
    return 0;
}

/* Number of grids of the scheme (d, n). */
int orc_scheme_count(int d, int n)
{
    int cnt = 0;
    for (int q = 0; q < d; ++q) {
        int s = n + d - 1 - q;
        if (s < d) continue;
        cnt += (int)binom(s - 1, d - 1);
    }
    return cnt;
}

/* Fills levels_out[g*d + k] and coeffs_out[g]; returns the grid count. */
int orc_scheme_levels(int d, int n, int *levels_out, double *coeffs_out)
{
    int g = 0;
    for (int q = 0; q < d; ++q) {
        int s = n + d - 1 - q;
        if (s < d) continue;
        double c = ((q & 1) ? -1.0 : 1.0) * binom(d - 1, q);
        int l[ORC_MAXD];
        for (int k = 0; k < d - 1; ++k) l[k] = 1;
        l[d - 1] = s - (d - 1);
        do {
            for (int k = 0; k < d; ++k) levels_out[g * d + k] = l[k];
            coeffs_out[g] = c;
            ++g;
        } while (next_composition(l, d));
    }
    return g;
}

static int64_t subspace_size(int d, const int *j)
{
    int64_t s = 1;
    for (int k = 0; k < d; ++k) s *= (j[k] == 0) ? 2 : ((int64_t)1 << (j[k] - 1));
    return s;
}

static int subspace_exists(int d, int n, const int *j)
{
    int t = 0;
    for (int k = 0; k < d; ++k) t += j[k] > 1 ? j[k] : 1;
    return t <= n + d - 1;
}

/* Offsets of every subspace block in a dense table indexed by
 * j_0 (n+1)^{d-1} + ... + j_{d-1} (lexicographic, j_0 most significant);
 * -1 for subspaces not in the sparse grid.  Returns the total point count. */
static int64_t build_offsets(int d, int n, int64_t *table)
{
    int j[ORC_MAXD];
    for (int k = 0; k < d; ++k) j[k] = 0;
    int64_t off = 0, t = 0;
    for (;;) {
        if (subspace_exists(d, n, j)) { table[t] = off; off += subspace_size(d, j); }
        else table[t] = -1;
        ++t;
        int k = d - 1;                      /* j_{d-1} runs fastest */
        while (k >= 0 && ++j[k] > n) { j[k] = 0; --k; }
        if (k < 0) break;
    }
    return off;
}

static int64_t table_len(int d, int n)
{
    int64_t len = 1;
    for (int k = 0; k < d; ++k) len *= (n + 1);
    return len;
}

/* Number of points of the boundary sparse grid of the scheme (d, n). */
int64_t orc_sparse_num_points(int d, int n)
{
    int64_t *tab = (int64_t *)malloc(sizeof(int64_t) * table_len(d, n));
    int64_t tot = build_offsets(d, n, tab);
    free(tab);
    return tot;
}

/* Sparse-grid index of 1-D grid index i of a pole of level l: returns the
 * subspace level j and the position p within it. */
static void hier_pos(int64_t i, int l, int *j, int64_t *p)
{
    if (i == 0) { *j = 0; *p = 0; return; }
    if (i == ((int64_t)1 << l)) { *j = 0; *p = 1; return; }
    int lev = level_of(i, l);
    *j = lev;
    *p = i >> (l - lev + 1);            /* i = (2p+1) 2^{l-lev} */
}

/* Sparse index of every point of grid `levels` (out[flat] = sparse index). */
void orc_sparse_index_of_grid(int d, int n, const int *levels, int64_t *out)
{
    int64_t *tab = (int64_t *)malloc(sizeof(int64_t) * table_len(d, n));
    build_offsets(d, n, tab);
    const int64_t N = orc_num_points(d, levels);
    for (int64_t f = 0; f < N; ++f) {
        int64_t rem = f, pos = 0, mul = 1, t = 0;
        int j[ORC_MAXD];
        int64_t p[ORC_MAXD];
        for (int k = 0; k < d; ++k) {
            const int64_t nk = ((int64_t)1 << levels[k]) + 1;
            hier_pos(rem % nk, levels[k], &j[k], &p[k]);
            rem /= nk;
        }
        for (int k = 0; k < d; ++k) t = t * (n + 1) + j[k];
        for (int k = 0; k < d; ++k) {
            pos += p[k] * mul;
            mul *= (j[k] == 0) ? 2 : ((int64_t)1 << (j[k] - 1));
        }
        out[f] = tab[t] + pos;
    }
    free(tab);
}

/* Gather (Sec. 2, "Hierarchization as preprocessing"): sparse = sum over the
 * grids of coeff_g * alpha_g, where a point absent from a grid contributes 0.
 * Grids are added in the order given (scheme enumeration order), starting
 * from 0, each term as one fused multiply-add, sparse[p] = fma(c, alpha,
 * sparse[p]) (one rounding per term; the paper fixes no rounding order). */
void orc_gather(int d, int n, int ngrids, const int *levels, const double *coeffs,
                const double *const *grids, double *sparse)
{
    const int64_t M = orc_sparse_num_points(d, n);
    for (int64_t p = 0; p < M; ++p) sparse[p] = 0.0;
    for (int g = 0; g < ngrids; ++g) {
        const int *l = levels + (int64_t)g * d;
        const int64_t N = orc_num_points(d, l);
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * N);
        orc_sparse_index_of_grid(d, n, l, idx);
        for (int64_t f = 0; f < N; ++f) sparse[idx[f]] = fma(coeffs[g], grids[g][f], sparse[idx[f]]);
        free(idx);
    }
}

/* Scatter, the step back of the iterated combination technique (Sec. 2,
 * "Hierarchization as preprocessing"): every component grid receives the
 * combined sparse-grid surpluses of its own points.  Each subspace of grid g
 * is a subspace of the sparse grid, so point f of grid g takes
 * sparse[index of f]; dehierarchizing the result gives the combined
 * sparse-grid function at the points of grid g (hats of finer subspaces vanish
 * there).  With scaled != 0 the value is multiplied by coeffs[g], one fp64
 * product, which makes this map the transpose of orc_gather. */
void orc_scatter(int d, int n, int ngrids, const int *levels, const double *coeffs, int scaled,
                 const double *sparse, double *const *grids)
{
    for (int g = 0; g < ngrids; ++g) {
        const int *l = levels + (int64_t)g * d;
        const int64_t N = orc_num_points(d, l);
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * N);
        orc_sparse_index_of_grid(d, n, l, idx);
        for (int64_t f = 0; f < N; ++f) grids[g][f] = scaled ? coeffs[g] * sparse[idx[f]] : sparse[idx[f]];
        free(idx);
    }
}

/* ------------------------------------------------------------------------ */
/* Loss weights of the differentiation workload                               */
/* ------------------------------------------------------------------------ */

/* w[flat] = 2^{-sum_k level(i_k)}, boundary level 0. */
void orc_level_weights(int d, const int *levels, double *w)
{
    const int64_t N = orc_num_points(d, levels);
    for (int64_t f = 0; f < N; ++f) {
        int64_t rem = f;
        int s = 0;
        for (int k = 0; k < d; ++k) {
            const int64_t nk = ((int64_t)1 << levels[k]) + 1;
            s += level_of(rem % nk, levels[k]);
            rem /= nk;
        }
        w[f] = ldexp(1.0, -s);
    }
}
