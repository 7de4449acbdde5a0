// Combination-scheme plans (Sec. 2): every grid of a scheme transformed by one
// persistent kernel driven by a device work queue, and the fp64 gather of the
// hierarchical surpluses into the sparse grid.
//
// Work items.  Each grid runs through phases; items are (grid, phase, tile)
// and are handed out by an atomic ticket in a fixed order: grids are grouped
// into waves that fit in L2 together, and within a wave the items run
// phase-major, so phase p+1 of a grid mostly reads phase p's output from L2.
// An item of phase p waits (bounded spin) until every item of the previous
// phase of its grid has finished; tickets are taken in order by resident
// CTAs, so every dependency is already owned by a running CTA.
//
// Two kernels share this queue.  k_fused (plans): a phase is a group of
// consecutive dimensions whose pole sets fit in one shared-memory tile, so a
// grid crosses memory once per group; fp64 tiles compute in exact int64 fixed
// point with their own binary scale.  k_batched (the allocation-free entry
// point): one phase per dimension, with a per-grid exponent scan and int64
// fixed point held in place between phases (the same 8 bytes per point); the
// first sweep converts, the last converts back.  Either way hierarchization
// uses the doubling form 2u - L - R, so it rounds once per stored value.
#include <algorithm>
#include <map>
#include <mutex>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "gbh_internal.h"

namespace gbh {
namespace {

constexpr int kPlanMaxD = 8;
constexpr int kBThreads = 256;
constexpr int64_t kItemPoints = 32768;        // target points per item
constexpr double kWaveBytes = 16.0 * 1024 * 1024;
constexpr long long kSpinLimit = 1ll << 24;   // bounded waits (~ seconds)

enum { OP_H = GBH_HIERARCHIZE, OP_D = GBH_DEHIERARCHIZE };
enum ItemKind {
    K_SCAN = 0, K_CONV_IN = 1, K_CONV_OUT = 2, K_ROWS = 3, K_POLES = 4, K_GROUP = 5, K_LATT = 6,
    K_FUSED = 7,         // tile of pole sets of a dimension group (fused kernel)
    K_LATT_NAT = 8       // coarse lattice of a split dimension, native arithmetic (fused kernel)
};

// t / S as __umul64hi(t, ceil(2^64 / S)), exact for t < 2^64 / S; S = 1 is
// marked by m = 0.
struct FastDiv {
    unsigned long long m;
};
__host__ inline FastDiv make_fastdiv(int64_t S)
{
    FastDiv f;
    f.m = S == 1 ? 0ull : (~0ull / (unsigned long long)S) + 1ull;
    return f;
}
__device__ __forceinline__ int64_t fdiv(int64_t t, FastDiv f)
{
    return f.m ? (int64_t)__umul64hi((unsigned long long)t, f.m) : t;
}

struct GridInfo {
    int l[kPlanMaxD];
    int64_t S[kPlanMaxD];
    FastDiv divS[kPlanMaxD];
    int64_t N;
    int first_dim;       // first and last dimension with a sweep (-1: none)
    int last_dim;
    int g0;              // fixed point: input scale bits (per op)
    int g0_d;
    int passes;          // dimensions with a sweep
    int ngroups;         // dimension groups of the fused kernel
    signed char grp_lo[kPlanMaxD];     // group q covers dimensions grp_lo..grp_hi
    signed char grp_hi[kPlanMaxD];
    signed char grp_m[kPlanMaxD];      // block level of a split dimension (-1: whole poles)
    signed char grp_g0[2][kPlanMaxD];  // fixed-point input scale bits (hierarchize, inverse)
};

struct Item {
    int grid;
    int phase;           // 0 = scan (fp64), 1 + k = sweep of dimension k
    int kind;
    int dim;
    int64_t start;       // first row / pole / element
    int64_t count;
    int wait;            // phase that must be complete first (-1: none)
    int blk;             // block index (K_GROUP)
};

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// fp64 <-> fixed point (see fused.cu for the derivation): the grid's largest
// magnitude sits just below 2^{g0}.
__device__ __noinline__ long long b_to_fixed_slow(double x, int emax, int c);
__device__ __noinline__ double b_from_fixed_slow(long long v, int X);

// Fast forms for grids whose largest exponent lies in [64, 1900]: zeros and
// subnormals fall out of the shift, every nonzero result is a normal number.
__device__ __forceinline__ long long b_to_fixed_fast(double x, int emax, int c)
{
    const long long bits = __double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7FF);
    const unsigned long long M = ((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int P = c > 0 ? c : 0;
    int rs = emax - e + P - c;
    rs = rs > 63 ? 63 : rs;
    const long long v = (long long)((M << P) >> rs);
    return bits < 0 ? -v : v;
}
__device__ __forceinline__ double b_from_fixed_fast(long long v, int X)
{
    const long long b = __double_as_longlong(__ll2double_rn(v));
    return __longlong_as_double(v == 0 ? 0ll : b + ((long long)X << 52));
}

__device__ __noinline__ long long b_to_fixed_slow(double x, int emax, int c)
{
    const long long bits = __double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7FF);
    if (e == 0) return 0;
    const unsigned long long M = ((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = c - (emax - e);
    long long v;
    if (sh >= 0) v = (long long)(M << sh);
    else v = (-sh >= 63) ? 0 : (long long)(M >> (-sh));
    return bits < 0 ? -v : v;
}

__device__ __noinline__ double b_from_fixed_slow(long long v, int X)
{
    if (v == 0) return 0.0;
    const double r = __ll2double_rn(v);
    const long long b = __double_as_longlong(r);
    const int ne = (int)((b >> 52) & 0x7FF) + X;
    if (ne > 0 && ne < 2047) return __longlong_as_double(b + ((long long)X << 52));
    return ldexp(r, X);
}

struct BatchParams {
    const Item *items;
    int nitems;
    const GridInfo *grids;
    void *const *ptrs;
    int *done;           // [ngrids * kPhases]
    const int *need;     // items per (grid, phase)
    int *emax;           // per grid
    unsigned *ticket;
    int *status;         // this launch: nonzero stops every CTA
    int *sticky;         // kept across launches until read by a status call
    int op;
    long long spin_limit;   // bounded waits: polls before giving up
    int stall_grid;         // test hook: every item of this grid waits on a
                            // dependency that nothing releases (-1: none)
};

// Phases of a grid: 0 exponent scan and 1 conversion to fixed point (fp64
// only), then two sub-phases per dimension (a long dimension splits into a
// block part and a coarse-lattice part), then the conversion back.
constexpr int kPhases = 3 + 2 * kPlanMaxD;
constexpr int kPhaseOut = kPhases - 1;
constexpr int kGroupLevel = 12;                  // block level of long dimensions
constexpr int kGroupElems = 8208;               // shared-memory elements per item
// fused kernel: tile size (elements), CTAs per SM, and the block level of
// dimensions longer than a tile
constexpr int kFusedElems = 8192;
constexpr int kFusedCtas64 = 3;                  // resident CTAs per SM, fp64 / fp32 plans
constexpr int kFusedCtas32 = 5;
constexpr int kGroupedCtas = 3;                  // single-grid grouped launches
constexpr int kSplitLevel = 12;

template <int OP>
__device__ __forceinline__ long long fx_op(long long v, long long L, long long R)
{
    if (OP == OP_H) return (v + v) - L - R;
    return v + ((L + R) >> 1);
}
template <int OP, typename F>
__device__ __forceinline__ F fl_op(F v, F L, F R)
{
    if (OP == OP_H) return v - F(0.5) * (L + R);
    return v + F(0.5) * (L + R);
}
template <int OP, typename V>
__device__ __forceinline__ V any_op(V v, V L, V R)
{
    if constexpr (std::is_same<V, long long>::value) return fx_op<OP>(v, L, R);
    else return fl_op<OP, V>(v, L, R);
}

// A pole of level L held in registers: hierarchize (fine to coarse) or
// dehierarchize (coarse to fine).  Fixed point doubles the two ends too, so
// one sweep scales every point by 2.
template <typename V, int L, int OP>
__device__ __forceinline__ void b_pole_regs(V *v)
{
    constexpr int last = 1 << L;
    if constexpr (OP == OP_H) {
#pragma unroll
        for (int lev = L; lev >= 1; --lev) {
            const int s = 1 << (L - lev);
#pragma unroll
            for (int i = s; i < last; i += 2 * s) v[i] = any_op<OP>(v[i], v[i - s], v[i + s]);
        }
        if constexpr (std::is_same<V, long long>::value) {
            v[0] = v[0] + v[0];
            v[last] = v[last] + v[last];
        }
    } else {
#pragma unroll
        for (int lev = 1; lev <= L; ++lev) {
            const int s = 1 << (L - lev);
#pragma unroll
            for (int i = s; i < last; i += 2 * s) v[i] = any_op<OP>(v[i], v[i - s], v[i + s]);
        }
    }
}

template <typename V, int L, int OP>
__device__ __forceinline__ void b_rows_regs(V *sv, int rows)
{
    constexpr int n = (1 << L) + 1;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        V v[n];
#pragma unroll
        for (int i = 0; i < n; ++i) v[i] = sv[r * n + i];
        b_pole_regs<V, L, OP>(v);
#pragma unroll
        for (int i = 0; i < n; ++i) sv[r * n + i] = v[i];
    }
}

// `count` poles starting at pole `start`: pole t of a dimension with stride S
// and extent n starts at (t / S) S n + t % S; the pole's points sit at stride
// `st` from there (a coarse lattice uses st = 2^m S).  One thread per pole,
// loads and stores all independent.
template <typename V, int L, int OP>
__device__ __forceinline__ void b_poles_regs(V *base, int64_t S, FastDiv dS, int64_t n, int64_t st, int64_t start,
                                             int64_t count)
{
    constexpr int np = (1 << L) + 1;
    for (int64_t t = start + threadIdx.x; t < start + count; t += blockDim.x) {
        const int64_t o = fdiv(t, dS), j = t - o * S;
        V *pp = base + o * S * n + j;
        V v[np];
#pragma unroll
        for (int i = 0; i < np; ++i) v[i] = __ldcg(pp + i * st);
        b_pole_regs<V, L, OP>(v);
#pragma unroll
        for (int i = 0; i < np; ++i) __stcg(pp + i * st, v[i]);
    }
}

template <typename V, int OP>
__device__ __forceinline__ void b_poles_dispatch(int L, V *base, int64_t S, FastDiv dS, int64_t n, int64_t st,
                                                 int64_t start, int64_t count)
{
    switch (L) {
        case 1: b_poles_regs<V, 1, OP>(base, S, dS, n, st, start, count); break;
        case 2: b_poles_regs<V, 2, OP>(base, S, dS, n, st, start, count); break;
        case 3: b_poles_regs<V, 3, OP>(base, S, dS, n, st, start, count); break;
        case 4: b_poles_regs<V, 4, OP>(base, S, dS, n, st, start, count); break;
        case 5: b_poles_regs<V, 5, OP>(base, S, dS, n, st, start, count); break;
        default: break;
    }
}

// Level-ordered sweep of `rows` poles of level L staged in shared memory
// (pole r at sv + r * pitch); with `ends` the two ends are doubled (fixed
// point) at the end.
template <typename V, int OP>
__device__ __forceinline__ void b_smem_sweep(V *sv, int rows, int pitch, int L, bool ends)
{
    const int last = 1 << L;
    if (OP == OP_H) {
        for (int lev = L; lev >= 1; --lev) {
            const int s = 1 << (L - lev), per = 1 << (lev - 1);
            for (int q = threadIdx.x; q < rows * per; q += blockDim.x) {
                const int r = q >> (lev - 1), i = (2 * (q & (per - 1)) + 1) * s;
                V *row = sv + r * pitch;
                row[i] = any_op<OP>(row[i], row[i - s], row[i + s]);
            }
            __syncthreads();
        }
        if constexpr (std::is_same<V, long long>::value) {
            if (ends) {
                for (int r = threadIdx.x; r < rows; r += blockDim.x) {
                    sv[r * pitch] += sv[r * pitch];
                    sv[r * pitch + last] += sv[r * pitch + last];
                }
                __syncthreads();
            }
        }
    } else {
        for (int lev = 1; lev <= L; ++lev) {
            const int s = 1 << (L - lev), per = 1 << (lev - 1);
            for (int q = threadIdx.x; q < rows * per; q += blockDim.x) {
                const int r = q >> (lev - 1), i = (2 * (q & (per - 1)) + 1) * s;
                V *row = sv + r * pitch;
                row[i] = any_op<OP>(row[i], row[i - s], row[i + s]);
            }
            __syncthreads();
        }
    }
}

// Streams `count` elements: src(e) -> dst(e, value), with up to kU loads in
// flight per thread (all loads of a group issue before its stores).
constexpr int kU = 8;
template <typename T, typename Src, typename Dst>
__device__ __forceinline__ void stream_elems(int64_t count, Src src, Dst dst)
{
    for (int64_t e0 = threadIdx.x; e0 < count; e0 += (int64_t)blockDim.x * kU) {
        T tmp[kU];
#pragma unroll
        for (int q = 0; q < kU; ++q) {
            const int64_t e = e0 + (int64_t)q * blockDim.x;
            if (e < count) tmp[q] = src(e);
        }
#pragma unroll
        for (int q = 0; q < kU; ++q) {
            const int64_t e = e0 + (int64_t)q * blockDim.x;
            if (e < count) dst(e, tmp[q]);
        }
    }
}

// Thread 0 takes the next ticket (or the one prefetched in `pref`) and waits
// (bounded) until the item's dependency -- every item of the previous phase
// of its grid -- has finished.
// Returns the item index, or -1 when the queue is empty, the wait gave up
// (status GBH_ETIMEOUT) or another CTA reported an error.  Every thread of
// the CTA calls it.
__device__ __forceinline__ int next_item(const BatchParams &P, int *s_item, int *s_abort, int *pref = nullptr)
{
    if (threadIdx.x == 0) {
        *s_item = (pref && *pref >= 0) ? *pref : (int)atomicAdd(P.ticket, 1u);
        *s_abort = 0;
        if (*s_item < P.nitems) {
            const Item it = P.items[*s_item];
            int wait = it.wait, want = 0;
            if (it.grid == P.stall_grid) {
                wait = kPhaseOut;
                want = 0x7FFFFFFF;
            } else if (wait >= 0) {
                want = P.need[it.grid * kPhases + wait];
            }
            if (wait >= 0) {
                const int *cnt = P.done + it.grid * kPhases + wait;
                long long spins = 0;
                while (ld_acquire(cnt) < want) {
                    if (++spins > P.spin_limit) {
                        atomicExch(P.status, GBH_ETIMEOUT);
                        atomicExch(P.sticky, GBH_ETIMEOUT);
                        *s_abort = 1;
                        break;
                    }
                    __nanosleep(64);
                }
            }
        }
        // the following ticket, taken now so that its latency hides behind
        // this item (tickets stay in order: a CTA holds at most one ticket
        // beyond the one it works on, and dependencies point to smaller ones)
        if (pref) *pref = (*s_item < P.nitems && !*s_abort) ? (int)atomicAdd(P.ticket, 1u) : -1;
    }
    __syncthreads();
    const int idx = *s_item;
    if (idx >= P.nitems || *s_abort || ld_acquire(P.status) != 0) return -1;
    return idx;
}

template <typename ST, int OP>
__global__ void __launch_bounds__(kBThreads, 2) k_batched(const BatchParams P)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_item;
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    using V = typename std::conditional<sizeof(ST) == 8, long long, ST>::type;
    V *sv = reinterpret_cast<V *>(sm);

    for (;;) {
        const int idx = next_item(P, &s_item, &s_abort);
        if (idx < 0) return;
        const Item it = P.items[idx];
        const GridInfo &gi = P.grids[it.grid];
        ST *sbase = reinterpret_cast<ST *>(P.ptrs[it.grid]);
        V *base = reinterpret_cast<V *>(P.ptrs[it.grid]);

        if (it.kind == K_SCAN) {
            int em = 0;
            const long long *b = reinterpret_cast<const long long *>(sbase) + it.start;
            stream_elems<long long>(it.count, [&](int64_t e) { return __ldcg(b + e); },
                                    [&](int64_t, long long v) {
                                        const int ex = (int)((v >> 52) & 0x7FF);
                                        em = ex > em ? ex : em;
                                    });
            em = __reduce_max_sync(0xFFFFFFFFu, (unsigned)em);
            if ((tid & 31) == 0 && em > 0) atomicMax(P.emax + it.grid, em);
        } else if (it.kind == K_CONV_IN || it.kind == K_CONV_OUT) {
            if constexpr (sizeof(ST) == 8) {
                const int emax = ld_acquire(P.emax + it.grid);
                const int c = (OP == OP_H ? gi.g0 : gi.g0_d) - 53;
                const int X = emax - 1075 - c - (OP == OP_H ? gi.passes : 0);
                long long *b = reinterpret_cast<long long *>(sbase);
                const bool fast = emax >= 64 && emax <= 1900;
                long long *bb = b + it.start;
                if (fast && it.kind == K_CONV_IN) {
                    stream_elems<long long>(it.count, [&](int64_t e) { return __ldcg(bb + e); },
                                            [&](int64_t e, long long v) {
                                                __stcg(bb + e, b_to_fixed_fast(__longlong_as_double(v), emax, c));
                                            });
                } else if (fast) {
                    stream_elems<long long>(it.count, [&](int64_t e) { return __ldcg(bb + e); },
                                            [&](int64_t e, long long v) {
                                                __stcg(bb + e, __double_as_longlong(b_from_fixed_fast(v, X)));
                                            });
                } else {
                    for (int64_t i = it.start + tid; i < it.start + it.count; i += blockDim.x) {
                        const long long v = __ldcg(b + i);
                        __stcg(b + i, it.kind == K_CONV_IN ? b_to_fixed_slow(__longlong_as_double(v), emax, c)
                                                           : __double_as_longlong(b_from_fixed_slow(v, X)));
                    }
                }
            }
        } else {
            const int k = it.dim, l = gi.l[k];
            const int64_t n = ((int64_t)1 << l) + 1, S = gi.S[k];
            if (it.kind == K_ROWS) {
                // dimension 0: `count` whole rows staged in shared memory
                const int64_t e0 = it.start * n;
                const int cnt = (int)(it.count * n);
                V *src = base + e0;
                stream_elems<V>(cnt, [&](int64_t e) { return __ldcg(src + e); }, [&](int64_t e, V v) { sv[e] = v; });
                __syncthreads();
                const int rows = (int)it.count;
                switch (l) {
                    case 1: b_rows_regs<V, 1, OP>(sv, rows); __syncthreads(); break;
                    case 2: b_rows_regs<V, 2, OP>(sv, rows); __syncthreads(); break;
                    case 3: b_rows_regs<V, 3, OP>(sv, rows); __syncthreads(); break;
                    case 4: b_rows_regs<V, 4, OP>(sv, rows); __syncthreads(); break;
                    case 5: b_rows_regs<V, 5, OP>(sv, rows); __syncthreads(); break;
                    default: b_smem_sweep<V, OP>(sv, rows, (int)n, l, true); break;
                }
                stream_elems<V>(cnt, [&](int64_t e) { return sv[e]; }, [&](int64_t e, V v) { __stcg(src + e, v); });
            } else if (it.kind == K_POLES) {
                b_poles_dispatch<V, OP>(l, base, S, gi.divS[k], n, S, it.start, it.count);
            } else if (it.kind == K_LATT) {
                // coarse lattice of a long dimension: points a 2^m, stride 2^m S
                const int m = l < kGroupLevel ? l : kGroupLevel;
                b_poles_dispatch<V, OP>(l - m, base, S, gi.divS[k], n, S << m, it.start, it.count);
            } else {
                // K_GROUP: block `blk` (2^m + 1 points) of `count` poles in
                // shared memory; a block covering the whole pole writes it
                // all, otherwise only the block interior
                const int m = l < kGroupLevel ? l : kGroupLevel;
                const int nb = (1 << m) + 1;
                const int G = (int)it.count;
                const unsigned magG = G == 1 ? 0u : (0xFFFFFFFFu / (unsigned)G) + 1u;
                const int64_t off0 = (int64_t)it.blk << m;
                int64_t *pb = reinterpret_cast<int64_t *>(sm + (size_t)kGroupElems * sizeof(V));
                for (int g = tid; g < G; g += blockDim.x) {
                    const int64_t t = it.start + g, o = fdiv(t, gi.divS[k]);
                    pb[g] = o * S * n + (t - o * S) + off0 * S;
                }
                __syncthreads();
                stream_elems<V>(
                    (int64_t)G * nb,
                    [&](int64_t w) {
                        const int i = magG ? (int)__umulhi((unsigned)w, magG) : (int)w, g = (int)w - i * G;
                        return __ldcg(base + pb[g] + (int64_t)i * S);
                    },
                    [&](int64_t w, V v) {
                        const int i = magG ? (int)__umulhi((unsigned)w, magG) : (int)w, g = (int)w - i * G;
                        sv[g * nb + i] = v;
                    });
                __syncthreads();
                b_smem_sweep<V, OP>(sv, G, nb, m, m == l);
                const int lo = m == l ? 0 : 1, hi = m == l ? nb : nb - 1;
                for (int w = tid; w < G * (hi - lo); w += blockDim.x) {
                    const int q = magG ? (int)__umulhi((unsigned)w, magG) : w, g = w - q * G, i = lo + q;
                    __stcg(base + pb[g] + (int64_t)i * S, sv[g * nb + i]);
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(P.done + it.grid * kPhases + it.phase, 1);
        }
    }
}

// ---------------------------------------------------------------------------
// fused kernel: dimension groups staged in shared memory
// ---------------------------------------------------------------------------
//
// The plan's kernel.  A grid's dimensions are cut into groups of consecutive
// dimensions whose pole sets (every point of the group's dimensions, the
// other coordinates fixed) fit in one tile; a dimension longer than a tile is
// a group of its own, split into blocks of 2^13 + 1 points and the coarse
// lattice of the block ends (hierarchize: blocks, then lattice; the inverse:
// lattice first).  An item is a tile of pole sets: loaded, transformed along
// every dimension of its group in shared memory, stored, so a grid crosses
// memory once per group instead of once per dimension plus conversions.
// fp64 computes in int64 fixed point with the tile's own binary scale (exact
// for the hierarchization, one rounding per point at the store); lattice
// items, a few points per pole, compute natively.

// Poles of one dimension of a tile.  Element i of pole set g sits at
// sv[g sG + i sI]: pole sets one after another (sG = M, sI = 1) when their
// points are contiguous in memory, side by side (sG = 1, sI = Gc) when pole
// sets are strided -- either way shared memory follows the order of the
// global accesses.  The dimension has local stride sk (product of the extents
// of the group's lower dimensions) and extent nk, so pole (g, a, b) holds the
// points i = a + sk (j + nk b), j = 0..nk-1.  Poles are numbered so that
// neighbouring threads touch neighbouring words.
struct TilePoles {
    int Gc, pps, sk, nk, sG, sI;
    bool gfast;
    unsigned magA, magK;

    __device__ __forceinline__ int base(int p) const
    {
        int g, r;
        if (gfast) {
            r = magA ? (int)__umulhi((unsigned)p, magA) : p;
            g = p - r * Gc;
        } else {
            g = magA ? (int)__umulhi((unsigned)p, magA) : p;
            r = p - g * pps;
        }
        const int b = magK ? (int)__umulhi((unsigned)r, magK) : r;
        const int a = r - b * sk;
        return g * sG + (a + b * sk * nk) * sI;
    }
};

// x / dv as __umulhi(x, magic), exact for x * dv < 2^32; dv = 1 gives 0
__host__ __device__ __forceinline__ unsigned magic_u32(int dv)
{
    return dv == 1 ? 0u : (0xFFFFFFFFu / (unsigned)dv) + 1u;
}

// Short poles (level L <= 5): one thread per pole, held in registers.  CONV
// converts the staged fp64 bits to fixed point on the way in.
template <typename V, int L, int OP, bool CONV>
__device__ __forceinline__ void tile_regs(V *sv, const TilePoles &tp, int poles, int emax, int c)
{
    constexpr int n = (1 << L) + 1;
    const int st = tp.sk * tp.sI;
    for (int p = threadIdx.x; p < poles; p += blockDim.x) {
        V *q = sv + tp.base(p);
        V v[n];
#pragma unroll
        for (int i = 0; i < n; ++i) {
            V x = q[i * st];
            if constexpr (CONV) x = (V)b_to_fixed_fast(__longlong_as_double((long long)x), emax, c);
            v[i] = x;
        }
        b_pole_regs<V, L, OP>(v);
#pragma unroll
        for (int i = 0; i < n; ++i) q[i * st] = v[i];
    }
}

template <typename V, int OP, bool CONV>
__device__ __forceinline__ void tile_regs_dispatch(int L, V *sv, const TilePoles &tp, int poles, int emax, int c)
{
    switch (L) {
        case 1: tile_regs<V, 1, OP, CONV>(sv, tp, poles, emax, c); break;
        case 2: tile_regs<V, 2, OP, CONV>(sv, tp, poles, emax, c); break;
        case 3: tile_regs<V, 3, OP, CONV>(sv, tp, poles, emax, c); break;
        case 4: tile_regs<V, 4, OP, CONV>(sv, tp, poles, emax, c); break;
        default: tile_regs<V, 5, OP, CONV>(sv, tp, poles, emax, c); break;
    }
}

// Long poles: level by level in shared memory (hierarchize fine to coarse: a
// point's two parents are coarser, hence still nodal; the inverse coarse to
// fine: a point's parents are final before it is computed); fixed point
// doubles the two ends of every pole too.  At least 4 poles: a group of
// lanes of one warp per pole (one lane when there are many poles, the whole
// warp when there are few; warp-level barriers only); fewer: the whole CTA
// sweeps every pole level by level.
template <typename V, int OP>
__device__ __forceinline__ void tile_long(V *sv, const TilePoles &tp, int poles, int lk)
{
    const int st = tp.sk * tp.sI, last = 1 << lk;
    constexpr bool kEnds = OP == OP_H && std::is_same<V, long long>::value;
    const int nw = blockDim.x >> 5;
    if (poles >= 4) {
        // lpp lanes of one warp per pole (a power of two, as many as the
        // poles leave room for): the lanes split each level, warp barriers
        // between levels; every lane of a warp runs every level
        int lpp = 1;
        while (lpp < 32 && 2 * lpp * poles <= (int)blockDim.x) lpp *= 2;
        const int lane = threadIdx.x & 31, sub = lane & (lpp - 1);
        const int per_warp = 32 / lpp;
        for (int p0 = (threadIdx.x >> 5) * per_warp; p0 < poles; p0 += nw * per_warp) {
            const int p = p0 + lane / lpp;
            const bool on = p < poles;
            V *q = sv + (on ? tp.base(p) : 0);
            for (int step = 1; step <= lk; ++step) {
                const int lev = OP == OP_H ? lk + 1 - step : step;
                const int s = 1 << (lk - lev), per = 1 << (lev - 1);
                if (on) {
                    for (int j = sub; j < per; j += lpp) {
                        const int i = (2 * j + 1) * s;
                        q[i * st] = any_op<OP>(q[i * st], q[(i - s) * st], q[(i + s) * st]);
                    }
                }
                __syncwarp();
            }
            if constexpr (kEnds) {
                if (on)
                    for (int e = sub; e < 2; e += lpp) q[e * last * st] += q[e * last * st];
                __syncwarp();
            }
        }
        return;
    }
    const unsigned magP = magic_u32(poles);
    for (int step = 1; step <= lk; ++step) {
        const int lev = OP == OP_H ? lk + 1 - step : step;
        const int s = 1 << (lk - lev), per = 1 << (lev - 1);
        const int tot = poles * per;
        for (int w = threadIdx.x; w < tot; w += blockDim.x) {
            const int pi = magP ? (int)__umulhi((unsigned)w, magP) : w;
            V *q = sv + tp.base(w - pi * poles);
            const int i = (2 * pi + 1) * s;
            q[i * st] = any_op<OP>(q[i * st], q[(i - s) * st], q[(i + s) * st]);
        }
        __syncthreads();
    }
    if constexpr (kEnds) {
        for (int w = threadIdx.x; w < 2 * poles; w += blockDim.x) {
            V *q = sv + tp.base(w >> 1) + (w & 1) * last * st;
            q[0] += q[0];
        }
    }
}

// Coarse-lattice poles of a split dimension (at most 2^5 + 1 points, a small
// fraction of the grid): level by level through global memory, one thread
// per pole, neighbouring threads on neighbouring poles.
template <typename V, int OP>
__device__ __forceinline__ void b_poles_loop(int L, V *base, int64_t S, FastDiv dS, int64_t n, int64_t st,
                                             int64_t start, int64_t count)
{
    const int last = 1 << L;
    for (int64_t t = start + threadIdx.x; t < start + count; t += blockDim.x) {
        const int64_t o = fdiv(t, dS), j = t - o * S;
        V *pp = base + o * S * n + j;
        for (int step = 1; step <= L; ++step) {
            const int lev = OP == OP_H ? L + 1 - step : step;
            const int s = 1 << (L - lev);
            for (int i = s; i < last; i += 2 * s)
                __stcg(pp + i * st, any_op<OP>(__ldcg(pp + i * st), __ldcg(pp + (i - s) * st), __ldcg(pp + (i + s) * st)));
        }
    }
}

// One K_FUSED item: `count` pole sets of group q starting at pole set
// `start` (block `blk` of a split dimension).
template <typename ST, int OP>
__device__ __forceinline__ void fused_item(const Item &it, const GridInfo &gi, ST *sbase, unsigned char *sm,
                                           int *s_em)
{
    using V = typename std::conditional<sizeof(ST) == 8, long long, ST>::type;
    // poles up to level kRegLevel are held in registers (one thread per pole)
    constexpr int kRegLevel = sizeof(V) == 8 ? 4 : 5;
    V *sv = reinterpret_cast<V *>(sm);
    V *base = reinterpret_cast<V *>(sbase);
    const int tid = threadIdx.x;
    const int q = it.dim, lo = gi.grp_lo[q], hi = gi.grp_hi[q], m = gi.grp_m[q];
    const bool split = m >= 0;
    int M = 1, pdims = 0;
    for (int k = lo; k <= hi; ++k) {
        M *= (1 << gi.l[k]) + 1;
        pdims += gi.l[k] > 0;
    }
    const int64_t Sa = gi.S[lo], Sout = Sa * M;    // Sout: stride of dimension hi + 1
    if (split) M = (1 << m) + 1;
    const int Gc = (int)it.count;
    const int cnt = Gc * M;
    const bool contig = Sa == 1 && !split;
    const unsigned magG = magic_u32(Gc), magM = magic_u32(M);
    // pole set t starts at (t / Sa) Sout + t % Sa (+ the block offset of a
    // split dimension); a tile never crosses a multiple of Sa, so its pole
    // sets are consecutive in memory (Sa > 1) or Sout apart (Sa = 1)
    int64_t base0;
    {
        const int64_t o = fdiv(it.start, gi.divS[lo]);
        base0 = o * Sout + (it.start - o * Sa) + (split ? ((int64_t)it.blk << m) * Sa : 0);
    }
    // offset of element w of the tile from its first point (its shared-memory
    // slot is w) and its index i within the pole set; 32-bit when the tile's
    // span allows (every plan grid below 2^31 points)
    const bool narrow = gi.N < ((int64_t)1 << 31);
    const int Sout32 = (int)Sout, Sa32 = (int)Sa;
    auto gaddr = [&](int w, int &i) -> int64_t {
        if (contig) {
            i = 0;
            return base0 + w;
        }
        if (Sa == 1) {
            const int g = magM ? (int)__umulhi((unsigned)w, magM) : w;
            i = w - g * M;
            return narrow ? base0 + (g * Sout32 + i) : base0 + (int64_t)g * Sout + i;
        }
        i = magG ? (int)__umulhi((unsigned)w, magG) : w;
        return narrow ? base0 + ((w - i * Gc) + i * Sa32) : base0 + (w - i * Gc) + (int64_t)i * Sa;
    };
    // every load of the tile in flight at once.  Other CTAs wrote this grid's
    // previous phase; the dependency wait (an acquire at gpu scope, then the
    // CTA barrier) orders their released stores before these loads.
    for (int w = tid; w < cnt; w += blockDim.x) {
        int i;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(sv + w);
        const V *src = base + gaddr(w, i);
        if constexpr (sizeof(V) == 8)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
        else
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    int X = 0, emax = 0, c = 0;
    bool fast = true, conv = false;
    int first = lo;
    while (gi.l[first] == 0) ++first;
    const int lfirst = split ? m : gi.l[first];
    if constexpr (sizeof(ST) == 8) {
        for (int e = tid; e < cnt; e += blockDim.x) {
            const int ex = (int)((sv[e] >> 52) & 0x7FF);
            emax = ex > emax ? ex : emax;
        }
        emax = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)emax);
        if ((tid & 31) == 0) atomicMax(s_em, emax);
        __syncthreads();
        emax = *s_em;
        c = gi.grp_g0[OP == OP_H ? 0 : 1][q] - 53;
        X = emax - 1075 - c - (OP == OP_H ? pdims : 0);
        fast = emax >= 64 && emax <= 1900;
        conv = true;
        // the conversion rides on the first sweep when that one keeps its
        // poles in registers
        if (!fast || lfirst > kRegLevel) {
            for (int e = tid; e < cnt; e += blockDim.x) {
                const double x = __longlong_as_double((long long)sv[e]);
                sv[e] = (V)(fast ? b_to_fixed_fast(x, emax, c) : b_to_fixed_slow(x, emax, c));
            }
            conv = false;
            __syncthreads();
        }
    }
    TilePoles tp;
    tp.Gc = Gc;
    tp.gfast = Sa > 1;
    tp.sG = tp.gfast ? 1 : M;
    tp.sI = tp.gfast ? Gc : 1;
    tp.sk = 1;
    for (int k = lo; k <= hi; ++k) {
        const int lk = split ? m : gi.l[k];
        tp.nk = (1 << lk) + 1;
        if (lk > 0) {
            tp.pps = M / tp.nk;
            tp.magA = magic_u32(tp.gfast ? Gc : tp.pps);
            tp.magK = magic_u32(tp.sk);
            const int poles = Gc * tp.pps;
            if (lk <= kRegLevel) {
                if (conv) tile_regs_dispatch<V, OP, sizeof(ST) == 8>(lk, sv, tp, poles, emax, c);
                else tile_regs_dispatch<V, OP, false>(lk, sv, tp, poles, emax, c);
            } else {
                tile_long<V, OP>(sv, tp, poles, lk);
            }
            conv = false;
            __syncthreads();
        }
        tp.sk *= tp.nk;
    }
    // a split dimension's block ends belong to the lattice: not stored
    for (int w = tid; w < cnt; w += blockDim.x) {
        int i;
        const int64_t a = gaddr(w, i);
        if (split && (i == 0 || i == M - 1)) continue;
        if constexpr (sizeof(ST) == 8) {
            const long long v = (long long)sv[w];
            const double r = fast ? b_from_fixed_fast(v, X) : b_from_fixed_slow(v, X);
            __stcg(base + a, (V)__double_as_longlong(r));
        } else {
            __stcg(base + a, sv[w]);
        }
    }
}

template <typename ST, int OP>
__global__ void __launch_bounds__(kBThreads, sizeof(ST) == 8 ? kFusedCtas64 : kFusedCtas32) k_fused(const BatchParams P)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_item;
    __shared__ int s_abort;
    __shared__ int s_em;
    int pref = -1;     // thread 0: prefetched ticket
    for (;;) {
        if (threadIdx.x == 0) s_em = 0;
        const int idx = next_item(P, &s_item, &s_abort, &pref);
        if (idx < 0) return;
        const Item it = P.items[idx];
        const GridInfo &gi = P.grids[it.grid];
        ST *sbase = reinterpret_cast<ST *>(P.ptrs[it.grid]);
        if (it.kind == K_FUSED) {
            fused_item<ST, OP>(it, gi, sbase, sm, &s_em);
        } else {
            // coarse lattice of a split dimension: points a 2^m, stride 2^m S
            const int k = gi.grp_lo[it.dim], l = gi.l[k], m = gi.grp_m[it.dim];
            const int64_t n = ((int64_t)1 << l) + 1, S = gi.S[k];
            const int L = l - m;    // at most 17 - kSplitLevel = 5
            const int64_t st = S << m;
            b_poles_loop<ST, OP>(L, sbase, S, gi.divS[k], n, st, it.start, it.count);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(P.done + it.grid * kPhases + it.phase, 1);
        }
    }
}


// ---------------------------------------------------------------------------
// single grids by dimension groups (non-persistent)
// ---------------------------------------------------------------------------
//
// A single grid (or a same-shape batch) transformed group by group: one
// launch per group of dimensions, one CTA per tile, the batched kernel's
// item body.  The default path takes it when grouping crosses memory fewer
// times than one sweep per dimension (e.g. (6,6,5,5,5): dimensions {0,1},
// {2,3}, {4}).  Tiles never cross a multiple of Sa (the stride of the group's
// first dimension).
struct GroupLaunch {
    GridInfo gi;
    int q;
    int64_t Sa, G, tiles_per_o, sets;
};

template <typename ST, int OP>
__global__ void __launch_bounds__(kBThreads, kGroupedCtas) k_grouped(const __grid_constant__ GroupLaunch L, ST *u)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int s_em;
    if (threadIdx.x == 0) s_em = 0;
    __syncthreads();
    Item it{};
    const int64_t b = blockIdx.x;
    if (L.Sa == 1) {
        it.start = b * L.G;
        it.count = L.sets - it.start < L.G ? L.sets - it.start : L.G;
    } else {
        const int64_t o = b / L.tiles_per_o;
        it.start = o * L.Sa + (b - o * L.tiles_per_o) * L.G;
        const int64_t end = (o + 1) * L.Sa;
        it.count = end - it.start < L.G ? end - it.start : L.G;
    }
    it.dim = L.q;
    it.kind = K_FUSED;
    fused_item<ST, OP>(it, L.gi, u + (int64_t)blockIdx.y * L.gi.N, sm, &s_em);
}

// Items of the fused kernel for one grid and phase: group q runs in phases
// 2 + 2q (+1 for the second part of a split dimension).
template <typename Push>
bool emit_fused_items(const GridInfo &gi, int op, int phase, int64_t chunk, Push push)
{
    if (phase < 2 || phase == kPhaseOut) return true;
    const int q = (phase - 2) / 2, sub = (phase - 2) % 2;
    if (q >= gi.ngroups) return true;
    const int lo = gi.grp_lo[q], hi = gi.grp_hi[q], m = gi.grp_m[q];
    int64_t M = 1;
    int pdims = 0;
    for (int k = lo; k <= hi; ++k) {
        M *= ((int64_t)1 << gi.l[k]) + 1;
        pdims += gi.l[k] > 0;
    }
    if (pdims == 0) return true;
    const int64_t sets = gi.N / M;
    // tiles of G pole sets that never cross a multiple of Sa (the stride of
    // dimension lo), so that a tile's pole sets are evenly spaced in memory
    const int64_t Sa = gi.S[lo];
    auto tiles = [&](int64_t G, int blk) {
        for (int64_t o = 0; o < sets; o += Sa)
            for (int64_t t = o; t < o + Sa; t += G)
                if (!push(K_FUSED, q, t, std::min(G, o + Sa - t), blk)) return false;
        return true;
    };
    if (Sa == 1) {
        // pole sets evenly spaced whatever the tile: no cut needed
        auto rows = [&](int64_t G, int blk) {
            for (int64_t t = 0; t < sets; t += G)
                if (!push(K_FUSED, q, t, std::min(G, sets - t), blk)) return false;
            return true;
        };
        if (m < 0) return sub ? true : rows(std::max<int64_t>(1, kFusedElems / M), 0);
        const int l = gi.l[lo];
        const bool blocks_now = (op == GBH_HIERARCHIZE) == (sub == 0);
        if (!blocks_now) {
            const int64_t ppi = std::max<int64_t>(kBThreads, chunk >> (l - m));
            for (int64_t t = 0; t < sets; t += ppi)
                if (!push(K_LATT_NAT, q, t, std::min(ppi, sets - t), 0)) return false;
            return true;
        }
        const int64_t G = std::max<int64_t>(1, kFusedElems / (((int64_t)1 << m) + 1));
        for (int64_t a = 0; a < ((int64_t)1 << (l - m)); ++a)
            if (!rows(G, (int)a)) return false;
        return true;
    }
    if (m < 0) {
        if (sub) return true;
        return tiles(std::max<int64_t>(1, kFusedElems / M), 0);
    }
    // split dimension: hierarchize blocks then lattice, the inverse the reverse
    const int l = gi.l[lo];
    const bool blocks_now = (op == GBH_HIERARCHIZE) == (sub == 0);
    if (!blocks_now) {
        const int64_t ppi = std::max<int64_t>(kBThreads, chunk >> (l - m));
        for (int64_t t = 0; t < sets; t += ppi)
            if (!push(K_LATT_NAT, q, t, std::min(ppi, sets - t), 0)) return false;
        return true;
    }
    const int64_t G = std::max<int64_t>(1, kFusedElems / (((int64_t)1 << m) + 1));
    for (int64_t a = 0; a < ((int64_t)1 << (l - m)); ++a)
        if (!tiles(G, (int)a)) return false;
    return true;
}

// Work items of one grid and phase, in the order they are handed out.  `push`
// takes (kind, dim, start, count, blk) and returns false when full.
template <typename Push>
bool emit_items(const GridInfo &gi, int d, int dtype, int op, int phase, int64_t chunk, Push push)
{
    if (phase == 0 || phase == 1 || phase == kPhaseOut) {
        if (dtype != GBH_F64) return true;
        const int kind = phase == 0 ? K_SCAN : phase == 1 ? K_CONV_IN : K_CONV_OUT;
        for (int64_t s = 0; s < gi.N; s += chunk * 2)
            if (!push(kind, 0, s, std::min<int64_t>(chunk * 2, gi.N - s), 0)) return false;
        return true;
    }
    const int k = (phase - 2) / 2, sub = (phase - 2) % 2;
    if (k >= d || gi.l[k] == 0) return true;
    const int l = gi.l[k];
    const int64_t n = ((int64_t)1 << l) + 1, poles = gi.N / n;
    if (k == 0 && n <= kGroupElems) {
        if (sub) return true;
        const int64_t rpi = std::max<int64_t>(1, std::min<int64_t>(kGroupElems / n, std::max<int64_t>(1, chunk / n)));
        for (int64_t s = 0; s < poles; s += rpi)
            if (!push(K_ROWS, 0, s, std::min(rpi, poles - s), 0)) return false;
        return true;
    }
    if (l <= 5) {
        if (sub) return true;
        const int64_t ppi = std::max<int64_t>(kBThreads, chunk / n);
        for (int64_t s = 0; s < poles; s += ppi)
            if (!push(K_POLES, k, s, std::min(ppi, poles - s), 0)) return false;
        return true;
    }
    const int m = std::min(l, kGroupLevel);
    const bool split = m < l;
    // hierarchize: blocks, then the lattice; the inverse: lattice first
    const bool blocks_now = !split ? (sub == 0) : ((op == GBH_HIERARCHIZE) == (sub == 0));
    if (!blocks_now) {
        if (!split) return true;
        const int64_t ppi = std::max<int64_t>(kBThreads, chunk >> (l - m));
        for (int64_t s = 0; s < poles; s += ppi)
            if (!push(K_LATT, k, s, std::min(ppi, poles - s), 0)) return false;
        return true;
    }
    const int64_t nb = ((int64_t)1 << m) + 1;
    const int64_t G = std::max<int64_t>(1, kGroupElems / nb);
    for (int64_t a = 0; a < ((int64_t)1 << (l - m)); ++a)
        for (int64_t s = 0; s < poles; s += G)
            if (!push(K_GROUP, k, s, std::min(G, poles - s), (int)a)) return false;
    return true;
}

// ---------------------------------------------------------------------------
// gather into the sparse grid
// ---------------------------------------------------------------------------

struct GatherParams {
    int d;
    const int64_t *sub_off;     // [nsub + 1] first sparse point of every subspace
    const int *sub_j;           // [nsub * d] subspace levels
    const int *list_off;        // [nsub + 1]
    const int *list;            // grids containing each subspace, enumeration order
    const int2 *chunks;         // (subspace, first point in it) of every CTA's chunk
    int nchunks;
    const GridInfo *grids;
    void *const *ptrs;
    const double *coeffs;
    double *sparse;
    int fp64;
};

// read-only loads of isolated elements, L2 fill limited to 64 bytes
__device__ __forceinline__ double g_ld64(const double *p)
{
    double v;
    asm("ld.global.nc.L2::64B.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float g_ld32(const float *p)
{
    float v;
    asm("ld.global.nc.L2::64B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

constexpr int kGatherPer = 2;                      // points per thread
constexpr int kGatherChunk = kGatherPer * 256;     // points per CTA chunk
constexpr int kGatherAhead = 4;                    // grids whose loads are in flight together
// staged path per element type (measured): fp64 grids stage chunks of up to
// 256 points, 8192 values per sub-batch (64 KB), three CTAs per SM; fp32
// grids chunks of up to 128 points, 4096 values (32 KB), four CTAs per SM
template <bool F64> struct GatherCfg {
    static constexpr int small = F64 ? 256 : 128, stage = F64 ? 8192 : 4096, ctas = F64 ? 3 : 4;
};

// A CTA takes a chunk of one subspace block (positions p, dimension 0
// fastest) and runs through the grids containing the subspace in enumeration
// order, 256 at a time: for grid g its point of position (p_k) sits at
// B_g + sum_k p_k T_gk, with B_g = sum_{j_k >= 1} S_k 2^{l_k - j_k} and
// T_gk = S_k 2^{l_k - j_k + 1} (j_k >= 1) or S_k 2^{l_k} (j_k = 0, the two
// boundary points).  Every term is one fused multiply-add, in grid order;
// the loads of the next kGatherAhead grids are in flight while the current
// ones are summed.  A chunk of at most GatherCfg::small points (the coarse
// subspaces, whose grid lists are the longest) would leave most threads idle
// and each point's thread with a long chain of dependent loads; there all
// threads load the terms of up to GatherCfg::stage / points grids at once into
// shared memory, and each point's thread then runs its fused multiply-adds
// over them in the same grid order.
template <bool F64>
__global__ void __launch_bounds__(256, GatherCfg<F64>::ctas) k_gather(const GatherParams P)
{
    extern __shared__ double sV[];   // GatherCfg::stage staged values (small chunks)
    __shared__ int64_t sB[256];
    __shared__ int64_t sT[256][kPlanMaxD];
    __shared__ double sC[256];
    __shared__ const void *sP[256];
    __shared__ int sj[kPlanMaxD], sbits[kPlanMaxD];
    const int d = P.d, tid = threadIdx.x;
    for (int c = blockIdx.x; c < P.nchunks; c += gridDim.x) {
        const int2 ch = P.chunks[c];
        const int sb = ch.x;
        const int64_t size = P.sub_off[sb + 1] - P.sub_off[sb];
        if (tid < d) {
            const int j = P.sub_j[sb * d + tid];
            sj[tid] = j;
            sbits[tid] = j == 0 ? 1 : j - 1;   // bits of the position along dimension tid
        }
        __syncthreads();
        int npts = 0;
#pragma unroll
        for (int r = 0; r < kGatherPer; ++r)
            if ((int64_t)ch.y + tid + r * 256 < size) npts = r + 1;
        double acc[kGatherPer];
#pragma unroll
        for (int r = 0; r < kGatherPer; ++r) acc[r] = 0.0;
        // value of this thread's point r in batch grid b (0 if absent)
        auto fetch = [&](int b, int r) -> double {
            int64_t f = sB[b], rest = (int64_t)ch.y + tid + r * 256;
#pragma unroll
            for (int k = 0; k < kPlanMaxD; ++k)
                if (k < d) {
                    f += (rest & ((1ll << sbits[k]) - 1)) * sT[b][k];
                    rest >>= sbits[k];
                }
            return P.fp64 ? g_ld64(reinterpret_cast<const double *>(sP[b]) + f)
                          : (double)g_ld32(reinterpret_cast<const float *>(sP[b]) + f);
        };
        const int q0 = P.list_off[sb], q1 = P.list_off[sb + 1];
        const int64_t left = size - ch.y;
        const int ppts = left < kGatherChunk ? (int)left : kGatherChunk;   // points of the chunk
        const bool small = ppts <= GatherCfg<F64>::small;
        // value of the chunk's point pt in batch grid b
        auto fetch_pt = [&](int b, int pt) -> double {
            int64_t f = sB[b], rest = (int64_t)ch.y + pt;
#pragma unroll
            for (int k = 0; k < kPlanMaxD; ++k)
                if (k < d) {
                    f += (rest & ((1ll << sbits[k]) - 1)) * sT[b][k];
                    rest >>= sbits[k];
                }
            return P.fp64 ? g_ld64(reinterpret_cast<const double *>(sP[b]) + f)
                          : (double)g_ld32(reinterpret_cast<const float *>(sP[b]) + f);
        };
        for (int qb = q0; qb < q1; qb += 256) {
            const int nb = q1 - qb < 256 ? q1 - qb : 256;
            if (tid < nb) {
                const int g = P.list[qb + tid];
                const GridInfo &gi = P.grids[g];
                int64_t B = 0;
                for (int k = 0; k < kPlanMaxD; ++k) {
                    int64_t T = 0;
                    if (k < d) {
                        const int l = gi.l[k], j = sj[k];
                        T = j == 0 ? gi.S[k] << l : gi.S[k] << (l - j + 1);
                        if (j > 0) B += gi.S[k] << (l - j);
                    }
                    sT[tid][k] = T;
                }
                sB[tid] = B;
                sC[tid] = P.coeffs[g];
                sP[tid] = P.ptrs[g];
            }
            __syncthreads();
            if (small) {
                const int GB = GatherCfg<F64>::stage / ppts;    // grids per sub-batch (>= 16)
                for (int b0 = 0; b0 < nb; b0 += GB) {
                    const int cnt = (nb - b0 < GB ? nb - b0 : GB) * ppts;
                    for (int w = tid; w < cnt; w += 256) {
                        const int b = w / ppts;
                        sV[w] = fetch_pt(b0 + b, w - b * ppts);
                    }
                    __syncthreads();
                    if (tid < ppts)
                        for (int w = tid, b = b0; w < cnt; w += ppts, ++b) acc[0] = __fma_rn(sC[b], sV[w], acc[0]);
                    __syncthreads();
                }
            } else if (npts > 0) {
                double cur[kGatherAhead][kGatherPer];
#pragma unroll
                for (int a = 0; a < kGatherAhead; ++a)
#pragma unroll
                    for (int r = 0; r < kGatherPer; ++r) cur[a][r] = (a < nb && r < npts) ? fetch(a, r) : 0.0;
                for (int b0 = 0; b0 < nb; b0 += kGatherAhead) {
                    double nxt[kGatherAhead][kGatherPer];
#pragma unroll
                    for (int a = 0; a < kGatherAhead; ++a) {
                        const int b = b0 + kGatherAhead + a;
#pragma unroll
                        for (int r = 0; r < kGatherPer; ++r) nxt[a][r] = (b < nb && r < npts) ? fetch(b, r) : 0.0;
                    }
#pragma unroll
                    for (int a = 0; a < kGatherAhead; ++a) {
                        if (b0 + a < nb) {
                            const double cg = sC[b0 + a];
#pragma unroll
                            for (int r = 0; r < kGatherPer; ++r)
                                if (r < npts) acc[r] = __fma_rn(cg, cur[a][r], acc[r]);
                        }
                    }
#pragma unroll
                    for (int a = 0; a < kGatherAhead; ++a)
#pragma unroll
                        for (int r = 0; r < kGatherPer; ++r) cur[a][r] = nxt[a][r];
                }
            }
            __syncthreads();
        }
        double *out = P.sparse + P.sub_off[sb] + ch.y;
#pragma unroll
        for (int r = 0; r < kGatherPer; ++r)
            if (r < npts) out[tid + r * 256] = acc[r];
    }
}

// ---------------------------------------------------------------------------
// scatter from the sparse grid back onto the grids
// ---------------------------------------------------------------------------

// Position of a subspace block in the sparse grid without a table over all
// subspaces.  With T = n + d - 1 and omega(0) = 2, omega(j) = 2^{j-1} points
// per dimension, let C_k(b) be the number of points of all suffixes
// (j_k, ..., j_{d-1}) with sum_{m>=k} max(j_m, 1) <= b.  Blocks before j in
// lexicographic order (j_0 most significant) agree with j on j_0..j_{k-1} and
// have a smaller j_k for exactly one k, so
//   offset(j) = sum_k W_k R_k(j_k, b_k),  W_k = prod_{m<k} omega(j_m),
//   R_k(jj, b) = sum_{j' < jj} omega(j') C_{k+1}(b - max(j', 1)),
// with b_0 = T and b_{k+1} = b_k - max(j_k, 1).  rank[(k (n+1) + jj) (T+1) + b]
// holds R_k(jj, b).
std::vector<int64_t> build_rank(int d, int n)
{
    const int T = n + d - 1, nj = n + 1, nb = T + 1;
    auto omega = [](int j) -> int64_t { return j == 0 ? 2 : (int64_t)1 << (j - 1); };
    std::vector<int64_t> C((size_t)(d + 1) * nb, 0), R((size_t)d * nj * nb, 0);
    for (int b = 0; b < nb; ++b) C[(size_t)d * nb + b] = 1;
    for (int k = d - 1; k >= 0; --k)
        for (int b = 0; b < nb; ++b) {
            int64_t acc = 0;
            for (int jj = 0; jj < nj; ++jj) {
                R[((size_t)k * nj + jj) * nb + b] = acc;
                const int r = b - std::max(jj, 1);
                if (r >= 0) acc += omega(jj) * C[(size_t)(k + 1) * nb + r];
            }
            C[(size_t)k * nb + b] = acc;
        }
    return R;
}

// Sparse-grid position contributed by dimension k of a point with index i on
// level l: subspace j_k = l - ctz(i) (0 at the two boundary points) and
// position p_k with i = (2 p_k + 1) 2^{l - j_k} (p_k = 0, 1 at the boundary),
// dimension 0 fastest inside a block.  Updates the budget b and the block
// weight W for the next dimension.
__host__ __device__ __forceinline__ void level_pos(int l, int i, int &j, int &p)
{
    if (i == 0 || i == (1 << l)) {
        j = 0;
        p = i != 0;
    } else {
#ifdef __CUDA_ARCH__
        const int tz = __ffs(i) - 1;
#else
        const int tz = __builtin_ctz((unsigned)i);
#endif
        j = l - tz;
        p = i >> (tz + 1);
    }
}

template <typename IDX>
__host__ __device__ __forceinline__ IDX sparse_pos(int k, int l, int i, int nj, int nb, const IDX *rank, int &b,
                                                   IDX &W)
{
    int j, p;
    level_pos(l, i, j, p);
    const IDX add = W * (rank[(k * nj + j) * nb + b] + p);
    W <<= j == 0 ? 1 : j - 1;
    b -= j > 1 ? j : 1;
    return add;
}

// Position of a point from its dimension-0 part and the part of the other
// dimensions: with m = max(j_0, 1), out_m = sum_{k>=1} W'_k (R_k(j_k, b_k) + p_k)
// taken with b_1 = T - m and W'_1 = 1, the position is
// R_0(j_0, T) + p_0 + omega(j_0) out_m.
template <typename IDX>
__host__ __device__ __forceinline__ IDX point_pos(const IDX *rank, int nb, int T, int j0, int p0, IDX out_m)
{
    return rank[j0 * nb + T] + p0 + (out_m << (j0 == 0 ? 1 : j0 - 1));
}

// A chunk of consecutive points of one grid, with the sizes of its tables
// and the 32-bit reciprocals its threads divide by (computed on the host).
struct ScatterChunk {
    int grid;
    int t0;          // first point's index along dimension 0
    int npts;        // points (<= kScatterChunk)
    int nent;        // parts of dimensions >= 1: rows x values of max(j_0, 1)
    int nent2;       // parts of dimensions >= 2: planes x values of max(j_0, 1) + max(j_1, 1)
    int nbud, nb2;   // values of max(j_0, 1); of max(j_0, 1) + max(j_1, 1)
    int n0;
    unsigned mag0, magb, magb2, pad;
    int64_t row;     // first point's row (pole along dimension 0)
    int64_t plane;   // first row's plane (dimensions 0 and 1)
};

struct ScatterParams {
    int d, nj, nb, T;
    const int64_t *rank;          // [d][n+1][T+1]
    int rank_len, max_ent;        // shared-memory layout: rank, parts >= 1, parts >= 2
    const ScatterChunk *chunks;
    int64_t nchunks;
    const GridInfo *grids;
    void *const *ptrs;
    const double *coeffs;
    const double *sparse;
    int scaled, fp64;
};

constexpr int kScatterPer = 8;                       // points per thread
constexpr int kScatterChunk = kScatterPer * 256;     // points per CTA chunk

// t / n0 for t < n0 + kScatterChunk: exact by the 32-bit reciprocal when
// n0 <= kScatterChunk (t n0 < 2^32), and in {0, 1} for longer rows.
__host__ __device__ __forceinline__ int div_row(int t, int n0, unsigned mag)
{
#ifdef __CUDA_ARCH__
    return n0 > kScatterChunk ? (t >= n0) : (int)__umulhi((unsigned)t, mag);
#else
    return n0 > kScatterChunk ? (t >= n0) : (int)(((uint64_t)(unsigned)t * mag) >> 32);
#endif
}

// Tables of one chunk.  With l0' = max(l_0, 1) and l1' = max(l_1, 1): the
// rows it touches times l0' values of max(j_0, 1), and the planes those rows
// touch times l0' + l1' - 1 values of max(j_0, 1) + max(j_1, 1).
ScatterChunk make_chunk(int g, const int *l, int d, int64_t N, int64_t f0)
{
    ScatterChunk c{};
    const int64_t n0 = ((int64_t)1 << l[0]) + 1;
    const int64_t n1 = d > 1 ? ((int64_t)1 << l[1]) + 1 : 1;
    c.grid = g;
    c.n0 = (int)n0;
    c.t0 = (int)(f0 % n0);
    c.row = f0 / n0;
    c.npts = (int)std::min<int64_t>(kScatterChunk, N - f0);
    const int64_t rows = (f0 + c.npts - 1) / n0 - c.row + 1;
    c.plane = c.row / n1;
    const int64_t planes = (c.row + rows - 1) / n1 - c.plane + 1;
    c.nbud = std::max(l[0], 1);
    c.nb2 = d > 2 ? c.nbud + std::max(l[1], 1) - 1 : 0;
    c.nent = (int)rows * c.nbud;
    c.nent2 = d > 2 ? (int)planes * c.nb2 : 0;
    c.mag0 = magic_u32((int)std::min<int64_t>(n0, 1 << 30));
    c.magb = magic_u32(c.nbud);
    c.magb2 = c.nb2 > 0 ? magic_u32(c.nb2) : 0;
    return c;
}

// A CTA takes a chunk of consecutive points of one grid.  Its threads first
// compute the part of the position due to dimensions >= 2 for every plane
// the chunk touches and every budget those dimensions can have, then from it
// the part due to dimensions >= 1 for every row and value of max(j_0, 1);
// then thread t writes points t, t + 256, ... (coalesced), each resolving
// only its dimension-0 level, with all eight loads issued before the stores.
// Consecutive points of one level along dimension 0 read consecutive
// positions.  IDX = int when every position fits in 31 bits.
template <typename IDX>
__global__ void __launch_bounds__(256) k_scatter(const ScatterParams P)
{
    extern __shared__ int64_t s_mem[];
    IDX *s_rank = reinterpret_cast<IDX *>(s_mem);
    IDX *s_out = s_rank + P.rank_len;
    IDX *s_out2 = s_out + P.max_ent;
    for (int e = threadIdx.x; e < P.rank_len; e += blockDim.x) s_rank[e] = (IDX)P.rank[e];
    __syncthreads();
    const int d = P.d;
    for (int64_t c = blockIdx.x; c < P.nchunks; c += gridDim.x) {
        const ScatterChunk ch = P.chunks[c];
        const GridInfo &gi = P.grids[ch.grid];
        const int l0 = gi.l[0], n0 = ch.n0, nbud = ch.nbud;
        // parts of dimensions >= 2, per plane and value s = max(j_0,1) + max(j_1,1)
        for (int e = threadIdx.x; e < ch.nent2; e += blockDim.x) {
            const int pp = ch.magb2 ? (int)__umulhi((unsigned)e, ch.magb2) : e, s = e - pp * ch.nb2 + 2;
            const int64_t plane = ch.plane + pp, fp = plane * gi.S[2];   // first point of the plane
            IDX out = 0, W = 1;
            int b = P.T - s;
            int64_t q = plane;                     // fp / S_2
            for (int k = 2; k < d; ++k) {
                const int64_t q1 = k + 1 < d ? fdiv(fp, gi.divS[k + 1]) : 0;
                out += sparse_pos<IDX>(k, gi.l[k], (int)(q - q1 * (((int64_t)1 << gi.l[k]) + 1)), P.nj, P.nb,
                                       s_rank, b, W);
                q = q1;
            }
            s_out2[e] = out;
        }
        if (d > 2) __syncthreads();
        // parts of dimensions >= 1, per row and value m = max(j_0, 1)
        for (int e = threadIdx.x; e < ch.nent; e += blockDim.x) {
            const int rr = ch.magb ? (int)__umulhi((unsigned)e, ch.magb) : e, m = e - rr * nbud + 1;
            IDX out = 0;
            if (d > 1) {
                const int64_t row = ch.row + rr;
                const int64_t plane = d > 2 ? fdiv(row * n0, gi.divS[2]) : 0;
                const int l1 = gi.l[1];
                int j1, p1;
                level_pos(l1, (int)(row - plane * (((int64_t)1 << l1) + 1)), j1, p1);
                out = s_rank[(P.nj + j1) * P.nb + P.T - m] + p1;
                if (d > 2) {
                    const int s = m + (j1 > 1 ? j1 : 1);
                    out += s_out2[(int)(plane - ch.plane) * ch.nb2 + s - 2] << (j1 == 0 ? 1 : j1 - 1);
                }
            }
            s_out[e] = out;
        }
        __syncthreads();
        IDX idx[kScatterPer];
#pragma unroll
        for (int r = 0; r < kScatterPer; ++r) {
            const int o = r * 256 + threadIdx.x;
            idx[r] = -1;
            if (o < ch.npts) {
                const int t = ch.t0 + o, rr = div_row(t, n0, ch.mag0);
                int j0, p0;
                level_pos(l0, t - rr * n0, j0, p0);
                const int m = j0 > 1 ? j0 : 1;
                idx[r] = point_pos<IDX>(s_rank, P.nb, P.T, j0, p0, s_out[rr * nbud + m - 1]);
            }
        }
        double v[kScatterPer];
#pragma unroll
        for (int r = 0; r < kScatterPer; ++r) v[r] = idx[r] >= 0 ? __ldg(P.sparse + idx[r]) : 0.0;
        const double cg = P.scaled ? P.coeffs[ch.grid] : 1.0;
        const int64_t f0 = ch.row * n0 + ch.t0;
        if (P.fp64) {
            double *dst = reinterpret_cast<double *>(P.ptrs[ch.grid]) + f0;
#pragma unroll
            for (int r = 0; r < kScatterPer; ++r)
                if (idx[r] >= 0) dst[r * 256 + threadIdx.x] = P.scaled ? cg * v[r] : v[r];
        } else {
            float *dst = reinterpret_cast<float *>(P.ptrs[ch.grid]) + f0;
#pragma unroll
            for (int r = 0; r < kScatterPer; ++r)
                if (idx[r] >= 0) dst[r * 256 + threadIdx.x] = (float)(P.scaled ? cg * v[r] : v[r]);
        }
        __syncthreads();
    }
}

double dgrowth(int lev)
{
    const int n = (1 << lev) + 1;
    double best = 0.0;
    for (int i = 0; i < n; ++i) {
        double s = 1.0;
        for (int j = 1; j <= lev; ++j) {
            const int st = 1 << (lev - j);
            const int a = (i / (2 * st)) * (2 * st) + st;
            if (a >= n - 1) continue;
            const double w = 1.0 - std::fabs((double)(i - a)) / (double)st;
            if (w > 0) s += w;
        }
        best = std::max(best, s);
    }
    return best;
}

// Dimension groups of the fused kernel: consecutive dimensions whose pole
// sets (product of their extents) fit in one tile, greedily from dimension 0;
// a dimension longer than a tile is a group of its own, split at block level
// kSplitLevel.  Fixed-point scales: hierarchization grows by at most 4 per
// swept dimension (doubling form), the inverse by the largest sum of hat
// weights along a pole per swept dimension.
static_assert(((1 << kSplitLevel) + 1) <= kFusedElems, "a block must fit in a tile");
static_assert(kGroupLevel + 5 - kSplitLevel <= 5, "the fused kernel's lattice poles have at most 5 levels");

void make_groups(GridInfo &gi, int d)
{
    int q = 0;
    auto ext = [&](int k) { return ((int64_t)1 << gi.l[k]) + 1; };
    for (int k = 0; k < d;) {
        int hi = k, m = -1;
        int64_t M = ext(k);
        if (M > kFusedElems) {
            m = kSplitLevel;
        } else {
            while (hi + 1 < d && M * ext(hi + 1) <= kFusedElems) {
                ++hi;
                M *= ext(hi);
            }
        }
        int pdims = 0;
        double growth = 1.0;
        for (int j = k; j <= hi; ++j)
            if (gi.l[j] > 0) {
                ++pdims;
                growth *= dgrowth(m >= 0 ? m : gi.l[j]);
            }
        gi.grp_lo[q] = (signed char)k;
        gi.grp_hi[q] = (signed char)hi;
        gi.grp_m[q] = (signed char)m;
        gi.grp_g0[0][q] = (signed char)(62 - 2 * pdims);
        gi.grp_g0[1][q] = (signed char)(61 - (int)std::ceil(std::log2(growth) + 1e-9));
        ++q;
        k = hi + 1;
    }
    gi.ngroups = q;
}

template <typename ST, int OP>
int run_grouped(const GridInfo &gi, int64_t batch, ST *u, cudaStream_t st)
{
    const size_t smem = kFusedElems * sizeof(ST);
    cudaFuncSetAttribute(k_grouped<ST, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int q = 0; q < gi.ngroups; ++q) {
        GroupLaunch L{};
        L.gi = gi;
        L.q = q;
        int64_t M = 1;
        int pdims = 0;
        for (int k = gi.grp_lo[q]; k <= gi.grp_hi[q]; ++k) {
            M *= ((int64_t)1 << gi.l[k]) + 1;
            pdims += gi.l[k] > 0;
        }
        if (pdims == 0) continue;
        L.Sa = gi.S[gi.grp_lo[q]];
        L.sets = gi.N / M;
        L.G = std::max<int64_t>(1, kFusedElems / M);
        int64_t tiles;
        if (L.Sa == 1) {
            tiles = (L.sets + L.G - 1) / L.G;
        } else {
            L.tiles_per_o = (L.Sa + L.G - 1) / L.G;
            tiles = (L.sets / L.Sa) * L.tiles_per_o;
        }
        if (tiles > INT32_MAX || batch > 65535) return GBH_ERANGE;
        ProfScope ps("grouped", st, 2.0 * sizeof(ST) * (double)gi.N * batch);
        k_grouped<ST, OP><<<dim3((unsigned)tiles, (unsigned)batch), kBThreads, smem, st>>>(L, u);
        ps.done();
        count_launches(1);
        if (int e = check_launch()) return e;
    }
    return GBH_OK;
}

bool make_grid_info(const Geom &g, GridInfo *gi)
{
    if (g.d > kPlanMaxD) return false;
    std::memset(gi, 0, sizeof(*gi));
    for (int k = 0; k < g.d; ++k) {
        gi->l[k] = g.l[k];
        gi->S[k] = g.S[k];
        gi->divS[k] = make_fastdiv(g.S[k]);
    }
    gi->N = g.N;
    make_groups(*gi, g.d);
    for (int q = 0; q < gi->ngroups; ++q)
        if (gi->grp_m[q] >= 0) return false;          // a dimension longer than a tile
    return true;
}

}  // namespace

int grouped_transform(void *data, const Geom &g, int dtype, int op, cudaStream_t s)
{
    if (op != GBH_HIERARCHIZE && op != GBH_DEHIERARCHIZE) return GBH_EUNSUPPORTED;
    GridInfo gi;
    if (!make_grid_info(g, &gi)) return GBH_EUNSUPPORTED;
    if (dtype == GBH_F64) {
        double *u = static_cast<double *>(data);
        return op == GBH_HIERARCHIZE ? run_grouped<double, OP_H>(gi, g.batch, u, s) : run_grouped<double, OP_D>(gi, g.batch, u, s);
    }
    float *u = static_cast<float *>(data);
    return op == GBH_HIERARCHIZE ? run_grouped<float, OP_H>(gi, g.batch, u, s) : run_grouped<float, OP_D>(gi, g.batch, u, s);
}

}  // namespace gbh

using namespace gbh;

struct gbh_plan {
    int d = 0, dtype = 0, n = -1, ngrids = 0;
    std::vector<int32_t> levels;       // [G][d]
    std::vector<double> coeffs;
    std::vector<GridInfo> info;
    std::vector<Item> items[2];        // per op (hierarchize, dehierarchize)
    std::vector<int> need[2];          // [G][kPhases]
    int64_t total_points = 0, sparse_points = 0;
    // device
    GridInfo *d_info = nullptr;
    Item *d_items[2] = {nullptr, nullptr};
    int *d_need[2] = {nullptr, nullptr};
    void **d_ptrs = nullptr;
    double *d_coeffs = nullptr;
    unsigned char *d_scratch = nullptr;   // ticket | status | emax[G] | done[G][kPhases] | sticky status
    size_t scratch_bytes = 0;
    int64_t *d_sub_off = nullptr;
    int *d_sub_j = nullptr, *d_list_off = nullptr, *d_list = nullptr;
    int2 *d_chunks = nullptr;
    int nsub = 0, nchunks = 0;
    int64_t *d_rank = nullptr;        // scatter: subspace ranking table [d][n+1][n+d]
    ScatterChunk *d_scat = nullptr;   // scatter: chunk list
    int64_t nscat = 0;
    int rank_len = 0;
    int scat_ent = 0, scat_ent2 = 0;  // scatter: largest part tables of a chunk
    bool scat_idx32 = false;          // scatter: sparse positions fit in 31 bits
    void **h_ptrs = nullptr;          // pinned staging for bind
    bool bound = false;
    int dev = 0;
    int stall_grid = -1;              // test hook: a dependency nothing releases
    long long spin_limit = kSpinLimit;
    // execution parameters per op (autotuned or set): resident CTAs per SM
    // (0 = as many as fit) and the L2 wave of the ticket order
    int ctas_per_sm[2] = {0, 0};
    double wave_bytes[2] = {kWaveBytes, kWaveBytes};
    bool full_scheme = false;         // gbh_plan_create_scheme: the tuned-scheme cache applies
};

namespace {

void free_plan(gbh_plan *p)
{
    if (!p) return;
    cudaFree(p->d_info);
    for (int o = 0; o < 2; ++o) {
        cudaFree(p->d_items[o]);
        cudaFree(p->d_need[o]);
    }
    cudaFree(p->d_ptrs);
    cudaFree(p->d_coeffs);
    cudaFree(p->d_scratch);
    cudaFree(p->d_sub_off);
    cudaFree(p->d_sub_j);
    cudaFree(p->d_list_off);
    cudaFree(p->d_list);
    cudaFree(p->d_chunks);
    cudaFree(p->d_rank);
    cudaFree(p->d_scat);
    if (p->h_ptrs) cudaFreeHost(p->h_ptrs);
    delete p;
}

template <typename T>
int upload(T **dst, const std::vector<T> &src)
{
    const size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
    if (cudaMalloc(reinterpret_cast<void **>(dst), bytes) != cudaSuccess) return GBH_ENOMEM;
    if (!src.empty() && cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return GBH_ECUDA;
    return GBH_OK;
}

// Ticket order: grids (largest first) are cut into waves of about kWaveBytes;
// items are issued along diagonals of (wave, phase): all items with
// wave + phase = t, then t + 1, ...  An item's dependency (the previous phase of
// its grid) lies on an earlier diagonal, so consecutive tickets are
// independent while a few waves stay resident in L2.
template <typename Push>
bool order_items(const GridInfo *info, int ngrids, int d, int dtype, int op, int64_t chunk, double wave_bytes,
                 bool fused, int *order, int *wave_of, int *prev, int *need, Push push)
{
    const int es = dtype == GBH_F64 ? 8 : 4;
    for (int g = 0; g < ngrids; ++g) order[g] = g;
    std::sort(order, order + ngrids, [&](int a, int b) { return info[a].N > info[b].N || (info[a].N == info[b].N && a < b); });
    int nwaves = 0;
    {
        int w0 = 0;
        while (w0 < ngrids) {
            int w1 = w0;
            double bytes = 0.0;
            while (w1 < ngrids && (w1 == w0 || bytes + (double)info[order[w1]].N * es <= wave_bytes)) {
                bytes += (double)info[order[w1]].N * es;
                wave_of[w1] = nwaves;
                ++w1;
            }
            ++nwaves;
            w0 = w1;
        }
    }
    for (int i = 0; i < ngrids; ++i) prev[i] = -1;
    for (int i = 0; i < ngrids * kPhases; ++i) need[i] = 0;
    for (int t = 0; t < nwaves + kPhases - 1; ++t) {
        int gi0 = 0;
        for (int w = 0; w < nwaves; ++w) {
            while (gi0 < ngrids && wave_of[gi0] < w) ++gi0;
            const int ph = t - w;
            if (ph < 0 || ph >= kPhases) continue;
            for (int i = gi0; i < ngrids && wave_of[i] == w; ++i) {
                const int g = order[i];
                if (info[g].first_dim < 0) continue;
                int cnt = 0;
                const int wait = prev[i];
                auto put = [&](int kind, int dim, int64_t st, int64_t c, int blk) {
                    if (!push(Item{g, ph, kind, dim, st, c, wait, blk})) return false;
                    ++cnt;
                    return true;
                };
                const bool ok = fused ? emit_fused_items(info[g], op, ph, chunk, put)
                                      : emit_items(info[g], d, dtype, op, ph, chunk, put);
                if (!ok) return false;
                need[(size_t)g * kPhases + ph] = cnt;
                if (cnt > 0) prev[i] = ph;
            }
        }
    }
    return true;
}

int build_items(gbh_plan *p, int op, std::vector<Item> &items, std::vector<int> &need)
{
    need.assign((size_t)p->ngrids * kPhases, 0);
    items.clear();
    std::vector<int> order(p->ngrids), wave(p->ngrids), prev(p->ngrids);
    order_items(p->info.data(), p->ngrids, p->d, p->dtype, op, kItemPoints, p->wave_bytes[op], true, order.data(), wave.data(),
                prev.data(), need.data(), [&](const Item &it) {
                    items.push_back(it);
                    return true;
                });
    return GBH_OK;
}

// Execution parameters of op (0 CTAs = as many as fit); a new wave reorders
// the items (the same items, so the device arrays keep their size).
int set_params(gbh_plan *p, int op, int ctas, double wave)
{
    p->ctas_per_sm[op] = ctas;
    if (wave == p->wave_bytes[op]) return GBH_OK;
    // the work list is rewritten: no execution of the plan may still read it
    if (cudaDeviceSynchronize() != cudaSuccess) return GBH_ECUDA;
    p->wave_bytes[op] = wave;
    std::vector<Item> items;
    std::vector<int> need;
    if (int e = build_items(p, op, items, need)) return e;
    if (items.size() != p->items[op].size()) return GBH_ECUDA;
    p->items[op].swap(items);
    p->need[op].swap(need);
    if (!p->items[op].empty() &&
        cudaMemcpy(p->d_items[op], p->items[op].data(), sizeof(Item) * p->items[op].size(), cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return GBH_ECUDA;
    if (cudaMemcpy(p->d_need[op], p->need[op].data(), sizeof(int) * p->need[op].size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return GBH_ECUDA;
    return GBH_OK;
}

// Parameters the autotuner measured for full scheme plans: (d, n, dtype, op)
// -> (CTAs per SM, wave bytes); new plans of the same scheme start with them.
std::mutex g_scheme_tune_mu;
std::map<std::vector<int>, std::pair<int, double>> g_scheme_tuned;

int finish_plan(gbh_plan *p)
{
    const int d = p->d;
    p->info.resize(p->ngrids);
    p->total_points = 0;
    for (int g = 0; g < p->ngrids; ++g) {
        GridInfo &gi = p->info[g];
        std::memset(&gi, 0, sizeof(gi));
        int64_t N = 1;
        gi.first_dim = gi.last_dim = -1;
        int passes = 0;
        double growth = 1.0;
        for (int k = 0; k < d; ++k) {
            const int l = p->levels[(size_t)g * d + k];
            if (l < 0 || l > kGroupLevel + 5) return GBH_ERANGE;
            gi.l[k] = l;
            gi.S[k] = N;
            gi.divS[k] = make_fastdiv(N);
            const int64_t nk = ((int64_t)1 << l) + 1;
            if (N > INT64_MAX / 8 / nk) return GBH_ERANGE;
            N *= nk;
            if (l > 0) {
                if (gi.first_dim < 0) gi.first_dim = k;
                gi.last_dim = k;
                ++passes;
                growth *= dgrowth(std::min(l, 16));
            }
        }
        gi.N = N;
        gi.passes = passes;
        gi.g0 = 61 - 2 * passes;
        gi.g0_d = 61 - (int)std::ceil(std::log2(growth) + 1e-9);
        make_groups(gi, d);
        p->total_points += N;
    }
    for (int o = 0; o < 2; ++o) {
        if (int e = build_items(p, o, p->items[o], p->need[o])) return e;
        if (int e = upload(&p->d_items[o], p->items[o])) return e;
        if (int e = upload(&p->d_need[o], p->need[o])) return e;
    }
    if (int e = upload(&p->d_info, p->info)) return e;
    if (int e = upload(&p->d_coeffs, p->coeffs)) return e;
    if (cudaMalloc(reinterpret_cast<void **>(&p->d_ptrs), sizeof(void *) * p->ngrids) != cudaSuccess) return GBH_ENOMEM;
    // the per-execution part (cleared by every execution), then the sticky
    // status word behind it
    p->scratch_bytes = (64 + sizeof(int) * (size_t)p->ngrids * (1 + kPhases) + 15) / 16 * 16;
    if (cudaMalloc(reinterpret_cast<void **>(&p->d_scratch), p->scratch_bytes + 16) != cudaSuccess) return GBH_ENOMEM;
    if (cudaMemset(p->d_scratch, 0, p->scratch_bytes + 16) != cudaSuccess) return GBH_ECUDA;
    if (cudaMallocHost(reinterpret_cast<void **>(&p->h_ptrs), sizeof(void *) * p->ngrids) != cudaSuccess) return GBH_ENOMEM;
    cudaGetDevice(&p->dev);
    return GBH_OK;
}

// sparse-grid subspaces of the scheme (d, n): lexicographic j, j_0 most significant
int build_sparse(gbh_plan *p)
{
    const int d = p->d, n = p->n;
    std::vector<int64_t> off;
    std::vector<int> js, loff, list;
    std::vector<int> j(d, 0);
    int64_t acc = 0;
    for (;;) {
        int t = 0;
        for (int k = 0; k < d; ++k) t += std::max(j[k], 1);
        if (t <= n + d - 1) {
            off.push_back(acc);
            int64_t sz = 1;
            for (int k = 0; k < d; ++k) sz *= (j[k] == 0) ? 2 : ((int64_t)1 << (j[k] - 1));
            acc += sz;
            for (int k = 0; k < d; ++k) js.push_back(j[k]);
            loff.push_back((int)list.size());
            for (int g = 0; g < p->ngrids; ++g) {
                bool in = true;
                for (int k = 0; k < d; ++k) in &= j[k] <= p->levels[(size_t)g * d + k];
                if (in) list.push_back(g);
            }
        }
        int k = d - 1;                             // j_{d-1} fastest
        while (k >= 0 && ++j[k] > n) { j[k] = 0; --k; }
        if (k < 0) break;
    }
    off.push_back(acc);
    loff.push_back((int)list.size());
    p->nsub = (int)js.size() / d;
    p->sparse_points = acc;
    std::vector<int2> chunks;
    for (int sb = 0; sb < p->nsub; ++sb)
        for (int64_t q = 0; q < off[sb + 1] - off[sb]; q += kGatherChunk) {
            if (q > INT32_MAX) return GBH_ERANGE;
            chunks.push_back(make_int2(sb, (int)q));
        }
    // costliest chunks first (points x grids containing the subspace), so
    // that the long grid lists of the coarse subspaces do not finish last;
    // each sparse point is still summed by one thread in grid order
    {
        auto cost = [&](const int2 &c) {
            const int64_t pts = std::min<int64_t>(kGatherChunk, off[c.x + 1] - off[c.x] - c.y);
            return pts * (int64_t)(loff[c.x + 1] - loff[c.x]);
        };
        std::stable_sort(chunks.begin(), chunks.end(), [&](const int2 &a, const int2 &b) { return cost(a) > cost(b); });
    }
    p->nchunks = (int)chunks.size();
    if (int e = upload(&p->d_chunks, chunks)) return e;
    if (int e = upload(&p->d_sub_off, off)) return e;
    if (int e = upload(&p->d_sub_j, js)) return e;
    if (int e = upload(&p->d_list_off, loff)) return e;
    if (int e = upload(&p->d_list, list)) return e;
    const std::vector<int64_t> rank = build_rank(d, n);
    p->rank_len = (int)rank.size();
    std::vector<ScatterChunk> sch;
    for (int g = 0; g < p->ngrids; ++g)
        for (int64_t f0 = 0; f0 < p->info[g].N; f0 += kScatterChunk) {
            sch.push_back(make_chunk(g, p->info[g].l, d, p->info[g].N, f0));
            p->scat_ent = std::max(p->scat_ent, sch.back().nent);
            p->scat_ent2 = std::max(p->scat_ent2, sch.back().nent2);
        }
    p->nscat = (int64_t)sch.size();
    p->scat_idx32 = p->sparse_points < ((int64_t)1 << 31) &&
                    *std::max_element(rank.begin(), rank.end()) < ((int64_t)1 << 31);
    if (int e = upload(&p->d_rank, rank)) return e;
    if (int e = upload(&p->d_scat, sch)) return e;
    return GBH_OK;
}

// Appends every l in N_{>=1}^d with |l|_1 = s in lexicographic order (l_0
// most significant): an odometer over l_0..l_{d-2}, l_{d-1} takes the rest.
void add_compositions(gbh_plan *p, int s, double c)
{
    const int d = p->d;
    std::vector<int> l(d, 1);
    for (;;) {
        int head = 0;
        for (int k = 0; k < d - 1; ++k) head += l[k];
        if (s - head >= 1) {
            for (int k = 0; k < d - 1; ++k) p->levels.push_back(l[k]);
            p->levels.push_back(s - head);
            p->coeffs.push_back(c);
        }
        if (d == 1) break;
        int k = d - 2;
        while (k >= 0) {
            ++l[k];
            int h = 0;
            for (int m = 0; m <= k; ++m) h += l[m];
            if (h + (d - 1 - k) <= s) break;        // the tail still gets >= 1 each
            l[k] = 1;
            --k;
        }
        if (k < 0) break;
    }
}

double binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

}  // namespace

extern "C" {

int gbh_plan_create_scheme(int d, int n, int dtype, gbh_plan **out)
{
    return gbh_plan_create_scheme_subset(d, n, dtype, -1, nullptr, out);
}

int gbh_plan_create_scheme_subset(int d, int n, int dtype, int n_owned, const int32_t *owned, gbh_plan **out)
{
    if (!out) return GBH_EINVAL;
    *out = nullptr;
    if (d < 1 || d > kPlanMaxD || n < 1) return GBH_EINVAL;
    if (dtype != GBH_F32 && dtype != GBH_F64) return GBH_EDTYPE;
    if (n + d - 1 > 30 + d - 1) return GBH_ERANGE;
    if (n_owned >= 0 && (n_owned < 1 || !owned)) return GBH_EINVAL;
    gbh_plan *p = new (std::nothrow) gbh_plan();
    if (!p) return GBH_ENOMEM;
    p->d = d;
    p->dtype = dtype;
    p->n = n;
    // every l with l_k >= 1 and |l|_1 = n + d - 1 - q; q ascending, then
    // lexicographic order with l_0 most significant
    for (int q = 0; q < d; ++q) {
        const int s = n + d - 1 - q;
        if (s < d) continue;
        const double c = ((q & 1) ? -1.0 : 1.0) * binom(d - 1, q);
        add_compositions(p, s, c);
    }
    if (n_owned >= 0) {
        // keep the listed grids (strictly increasing scheme indexes)
        const int all = (int)p->coeffs.size();
        std::vector<int32_t> lv;
        std::vector<double> cf;
        for (int i = 0; i < n_owned; ++i) {
            const int g = owned[i];
            if (g < 0 || g >= all || (i > 0 && g <= owned[i - 1])) { delete p; return GBH_EINVAL; }
            lv.insert(lv.end(), p->levels.begin() + (size_t)g * d, p->levels.begin() + (size_t)(g + 1) * d);
            cf.push_back(p->coeffs[g]);
        }
        p->levels.swap(lv);
        p->coeffs.swap(cf);
    }
    p->ngrids = (int)p->coeffs.size();
    int e = finish_plan(p);
    if (!e) e = build_sparse(p);
    p->full_scheme = n_owned < 0;
    if (!e && p->full_scheme) {
        for (int op = 0; op < 2 && !e; ++op) {
            std::pair<int, double> t{0, 0.0};
            bool have = false;
            {
                std::lock_guard<std::mutex> lk(g_scheme_tune_mu);
                auto it = g_scheme_tuned.find(std::vector<int>{d, n, dtype, op});
                if (it != g_scheme_tuned.end()) { t = it->second; have = true; }
            }
            if (have) e = set_params(p, op, t.first, t.second);
        }
    }
    if (e) { free_plan(p); return e; }
    *out = p;
    return GBH_OK;
}

int gbh_plan_create(int n_grids, int d, const int32_t *levels, int dtype, gbh_plan **out)
{
    if (!out) return GBH_EINVAL;
    *out = nullptr;
    if (n_grids < 1 || d < 1 || d > kPlanMaxD || !levels) return GBH_EINVAL;
    if (dtype != GBH_F32 && dtype != GBH_F64) return GBH_EDTYPE;
    gbh_plan *p = new (std::nothrow) gbh_plan();
    if (!p) return GBH_ENOMEM;
    p->d = d;
    p->dtype = dtype;
    p->ngrids = n_grids;
    p->levels.assign(levels, levels + (size_t)n_grids * d);
    p->coeffs.assign(n_grids, 1.0);
    if (int e = finish_plan(p)) { free_plan(p); return e; }
    *out = p;
    return GBH_OK;
}

int gbh_plan_destroy(gbh_plan *plan)
{
    if (!plan) return GBH_EINVAL;
    free_plan(plan);
    return GBH_OK;
}

int gbh_plan_num_grids(const gbh_plan *plan, int *out)
{
    if (!plan || !out) return GBH_EINVAL;
    *out = plan->ngrids;
    return GBH_OK;
}

int gbh_plan_grid_levels(const gbh_plan *plan, int g, int32_t *levels_out)
{
    if (!plan || !levels_out || g < 0 || g >= plan->ngrids) return GBH_EINVAL;
    for (int k = 0; k < plan->d; ++k) levels_out[k] = plan->levels[(size_t)g * plan->d + k];
    return GBH_OK;
}

int gbh_plan_coeffs(const gbh_plan *plan, double *coeffs_out)
{
    if (!plan || !coeffs_out) return GBH_EINVAL;
    std::memcpy(coeffs_out, plan->coeffs.data(), sizeof(double) * plan->ngrids);
    return GBH_OK;
}

int gbh_plan_set_coeffs(gbh_plan *plan, const double *coeffs)
{
    if (!plan || !coeffs) return GBH_EINVAL;
    std::memcpy(plan->coeffs.data(), coeffs, sizeof(double) * plan->ngrids);
    if (cudaMemcpy(plan->d_coeffs, coeffs, sizeof(double) * plan->ngrids, cudaMemcpyHostToDevice) != cudaSuccess)
        return GBH_ECUDA;
    return GBH_OK;
}

int gbh_plan_sparse_points(const gbh_plan *plan, int64_t *out)
{
    if (!plan || !out) return GBH_EINVAL;
    if (plan->n < 0) return GBH_EUNSUPPORTED;
    *out = plan->sparse_points;
    return GBH_OK;
}

int gbh_plan_total_points(const gbh_plan *plan, int64_t *out)
{
    if (!plan || !out) return GBH_EINVAL;
    *out = plan->total_points;
    return GBH_OK;
}

int gbh_plan_bind(gbh_plan *plan, void *const *grid_ptrs, void *stream)
{
    if (!plan || !grid_ptrs) return GBH_EINVAL;
    const size_t es = plan->dtype == GBH_F64 ? 8 : 4;
    for (int g = 0; g < plan->ngrids; ++g) {
        if (!grid_ptrs[g]) return GBH_EINVAL;
        if (reinterpret_cast<uintptr_t>(grid_ptrs[g]) % es) return GBH_EALIGN;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the staging buffer may still feed an earlier copy
    if (cudaStreamSynchronize(s) != cudaSuccess) return GBH_ECUDA;
    std::memcpy(plan->h_ptrs, grid_ptrs, sizeof(void *) * plan->ngrids);
    if (cudaMemcpyAsync(plan->d_ptrs, plan->h_ptrs, sizeof(void *) * plan->ngrids, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return GBH_ECUDA;
    plan->bound = true;
    return GBH_OK;
}

int gbh_plan_execute(gbh_plan *plan, int op, void *stream)
{
    if (!plan) return GBH_EINVAL;
    if (op != GBH_HIERARCHIZE && op != GBH_DEHIERARCHIZE) return (op == GBH_ADJOINT || op == GBH_DEHIERARCHIZE_ADJOINT) ? GBH_EUNSUPPORTED : GBH_EINVAL;
    if (!plan->bound) return GBH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // queue, status and counters restart with every execution
    if (cudaMemsetAsync(plan->d_scratch, 0, plan->scratch_bytes, s) != cudaSuccess) return GBH_ECUDA;
    BatchParams P{};
    P.items = plan->d_items[op];
    P.nitems = (int)plan->items[op].size();
    P.grids = plan->d_info;
    P.ptrs = plan->d_ptrs;
    P.ticket = reinterpret_cast<unsigned *>(plan->d_scratch);
    P.status = reinterpret_cast<int *>(plan->d_scratch + 32);
    P.sticky = reinterpret_cast<int *>(plan->d_scratch + plan->scratch_bytes);
    P.emax = reinterpret_cast<int *>(plan->d_scratch + 64);
    P.done = P.emax + plan->ngrids;
    P.need = plan->d_need[op];
    P.op = op;
    P.spin_limit = plan->spin_limit;
    P.stall_grid = plan->stall_grid;
    const size_t es = plan->dtype == GBH_F64 ? 8 : 4;
    const size_t smem = kFusedElems * es;
    auto launch = [&](auto kern) -> int {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBThreads, smem);
        if (per_sm < 1) return GBH_EUNSUPPORTED;
        if (plan->ctas_per_sm[op] > 0) per_sm = std::min(per_sm, plan->ctas_per_sm[op]);
        const int grid = std::max(1, std::min(num_sms() * per_sm, P.nitems));
        ProfScope ps("batched", s, 2.0 * es * (double)plan->total_points);
        kern<<<grid, kBThreads, smem, s>>>(P);
        ps.done();
        count_launches(1);
        return check_launch();
    };
    if (plan->dtype == GBH_F64)
        return op == GBH_HIERARCHIZE ? launch(k_fused<double, OP_H>) : launch(k_fused<double, OP_D>);
    return op == GBH_HIERARCHIZE ? launch(k_fused<float, OP_H>) : launch(k_fused<float, OP_D>);
}

int gbh_plan_gather(gbh_plan *plan, double *sparse, void *stream)
{
    if (!plan || !sparse) return GBH_EINVAL;
    if (plan->n < 0) return GBH_EUNSUPPORTED;
    if (!plan->bound) return GBH_EINVAL;
    if (reinterpret_cast<uintptr_t>(sparse) % 8) return GBH_EALIGN;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GatherParams G{};
    G.d = plan->d;
    G.sub_off = plan->d_sub_off;
    G.sub_j = plan->d_sub_j;
    G.list_off = plan->d_list_off;
    G.list = plan->d_list;
    G.chunks = plan->d_chunks;
    G.nchunks = plan->nchunks;
    G.grids = plan->d_info;
    G.ptrs = plan->d_ptrs;
    G.coeffs = plan->d_coeffs;
    G.sparse = sparse;
    G.fp64 = plan->dtype == GBH_F64;
    const int grid = std::max(1, std::min(G.nchunks, num_sms() * 4));
    ProfScope ps("gather", s, (double)plan->total_points * (plan->dtype == GBH_F64 ? 8 : 4) + 8.0 * plan->sparse_points);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_gather<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(GatherCfg<true>::stage * sizeof(double)));
        cudaFuncSetAttribute(k_gather<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(GatherCfg<false>::stage * sizeof(double)));
        attr = true;
    }
    if (G.fp64) k_gather<true><<<grid, 256, GatherCfg<true>::stage * sizeof(double), s>>>(G);
    else k_gather<false><<<grid, 256, GatherCfg<false>::stage * sizeof(double), s>>>(G);
    ps.done();
    count_launches(1);
    return check_launch();
}

int gbh_plan_scatter(gbh_plan *plan, const double *sparse, int scaled, void *stream)
{
    if (!plan || !sparse) return GBH_EINVAL;
    if (plan->n < 0) return GBH_EUNSUPPORTED;
    if (!plan->bound) return GBH_EINVAL;
    if (reinterpret_cast<uintptr_t>(sparse) % 8) return GBH_EALIGN;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ScatterParams P{};
    P.d = plan->d;
    P.T = plan->n + plan->d - 1;
    P.nj = plan->n + 1;
    P.nb = P.T + 1;
    P.rank = plan->d_rank;
    P.rank_len = plan->rank_len;
    P.max_ent = plan->scat_ent;
    P.chunks = plan->d_scat;
    P.nchunks = plan->nscat;
    P.grids = plan->d_info;
    P.ptrs = plan->d_ptrs;
    P.coeffs = plan->d_coeffs;
    P.sparse = sparse;
    P.scaled = scaled != 0;
    P.fp64 = plan->dtype == GBH_F64;
    auto kern = plan->scat_idx32 ? k_scatter<int> : k_scatter<int64_t>;
    const size_t smem = (plan->scat_idx32 ? sizeof(int) : sizeof(int64_t)) *
                        ((size_t)plan->rank_len + plan->scat_ent + plan->scat_ent2);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GBH_ECUDA;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(P.nchunks, (int64_t)num_sms() * 8));
    ProfScope ps("scatter", s, (double)plan->total_points * (plan->dtype == GBH_F64 ? 8 : 4) + 8.0 * plan->sparse_points);
    kern<<<(int)grid, 256, smem, s>>>(P);
    ps.done();
    count_launches(1);
    return check_launch();
}

int gbh_sparse_index_of_grid(int d, int n, const int32_t *levels, int64_t *out)
{
    if (!levels || !out) return GBH_EINVAL;
    if (d < 1 || d > kPlanMaxD || n < 1 || n > 30) return GBH_EINVAL;
    int t = 0;
    int64_t N = 1, S[kPlanMaxD];
    for (int k = 0; k < d; ++k) {
        if (levels[k] < 0 || levels[k] > n) return GBH_ERANGE;
        t += std::max(levels[k], 1);
        S[k] = N;
        const int64_t nk = ((int64_t)1 << levels[k]) + 1;
        if (N > INT64_MAX / 8 / nk) return GBH_ERANGE;
        N *= nk;
    }
    if (t > n + d - 1) return GBH_ERANGE;
    const std::vector<int64_t> rank = build_rank(d, n);
    const int nj = n + 1, nb = n + d, T = n + d - 1;
    const int64_t n0 = ((int64_t)1 << levels[0]) + 1;
    for (int64_t f = 0; f < N; ++f) {
        int j0, p0;
        level_pos(levels[0], (int)(f % n0), j0, p0);
        int64_t out_m = 0, W = 1;
        int b = T - std::max(j0, 1);
        for (int k = 1; k < d; ++k) {
            const int i = (int)((f / S[k]) % (((int64_t)1 << levels[k]) + 1));
            out_m += sparse_pos<int64_t>(k, levels[k], i, nj, nb, rank.data(), b, W);
        }
        out[f] = point_pos<int64_t>(rank.data(), nb, T, j0, p0, out_m);
    }
    return GBH_OK;
}

int gbh_plan_test_stall(gbh_plan *plan, int grid, long long spin_limit)
{
    if (!plan || grid < -1 || grid >= plan->ngrids || spin_limit < 1) return GBH_EINVAL;
    plan->stall_grid = grid;
    plan->spin_limit = grid < 0 ? kSpinLimit : spin_limit;
    return GBH_OK;
}

int gbh_plan_set_params(gbh_plan *plan, int op, int ctas_per_sm, int wave_mb)
{
    if (!plan) return GBH_EINVAL;
    if (op != GBH_HIERARCHIZE && op != GBH_DEHIERARCHIZE) return GBH_EINVAL;
    if (ctas_per_sm < 0 || ctas_per_sm > 32 || wave_mb < 1 || wave_mb > 4096) return GBH_EINVAL;
    return set_params(plan, op, ctas_per_sm, (double)wave_mb * 1024.0 * 1024.0);
}

int gbh_plan_get_params(const gbh_plan *plan, int op, int *ctas_per_sm, int *wave_mb)
{
    if (!plan || !ctas_per_sm || !wave_mb) return GBH_EINVAL;
    if (op != GBH_HIERARCHIZE && op != GBH_DEHIERARCHIZE) return GBH_EINVAL;
    *ctas_per_sm = plan->ctas_per_sm[op];
    *wave_mb = (int)(plan->wave_bytes[op] / (1024.0 * 1024.0) + 0.5);
    return GBH_OK;
}

int gbh_plan_autotune(gbh_plan *plan, int op, void *stream, gbh_plan_tune_result *out)
{
    if (!plan || !out) return GBH_EINVAL;
    if (op != GBH_HIERARCHIZE && op != GBH_DEHIERARCHIZE) return GBH_EINVAL;
    std::memset(out, 0, sizeof(*out));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t es = plan->dtype == GBH_F64 ? 8 : 4;
    // resident CTAs the kernel allows
    int maxc = 0;
    {
        const size_t smem = kFusedElems * es;
        auto query = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxc, kern, kBThreads, smem);
        };
        if (plan->dtype == GBH_F64) {
            if (op == OP_H) query(k_fused<double, OP_H>);
            else query(k_fused<double, OP_D>);
        } else {
            if (op == OP_H) query(k_fused<float, OP_H>);
            else query(k_fused<float, OP_D>);
        }
        if (maxc < 1) return GBH_EUNSUPPORTED;
    }
    // scratch grids of the plan's shapes, bound in place of the caller's
    unsigned char *scratch = nullptr;
    if (cudaMalloc(reinterpret_cast<void **>(&scratch), (size_t)plan->total_points * es) != cudaSuccess)
        return GBH_ENOMEM;
    std::vector<void *> saved(plan->h_ptrs, plan->h_ptrs + plan->ngrids);
    const bool was_bound = plan->bound;
    std::vector<void *> sp(plan->ngrids);
    {
        size_t off = 0;
        for (int g = 0; g < plan->ngrids; ++g) {
            sp[g] = scratch + off * es;
            off += (size_t)plan->info[g].N;
        }
    }
    const int c0 = plan->ctas_per_sm[op];
    const double w0 = plan->wave_bytes[op];
    int status = gbh_plan_bind(plan, sp.data(), stream);
    if (!status) status = launch_fill(scratch, plan->total_points, plan->dtype, 777u, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int other = op == GBH_HIERARCHIZE ? GBH_DEHIERARCHIZE : GBH_HIERARCHIZE;
    // median of three timed executions of op; the inverse runs between them
    // (untimed) so that the values keep their magnitude
    auto time_of = [&](int ctas, double wave, double *ms) -> int {
        if (int e = set_params(plan, op, ctas, wave)) return e;
        if (int e = gbh_plan_execute(plan, op, stream)) return e;
        if (int e = gbh_plan_execute(plan, other, stream)) return e;
        double t[3];
        for (int r = 0; r < 3; ++r) {
            cudaEventRecord(e0, s);
            if (int e = gbh_plan_execute(plan, op, stream)) return e;
            cudaEventRecord(e1, s);
            if (int e = gbh_plan_execute(plan, other, stream)) return e;
            if (cudaEventSynchronize(e1) != cudaSuccess) return GBH_ECUDA;
            float f = 0.f;
            cudaEventElapsedTime(&f, e0, e1);
            t[r] = f;
        }
        std::sort(t, t + 3);
        *ms = t[1];
        return GBH_OK;
    };
    double best = 1e300;
    int bc = 0;
    double bw = kWaveBytes;
    const double waves[4] = {8.0, 16.0, 32.0, 64.0};
    for (int ci = 1; ci <= maxc && !status; ++ci) {
        for (int wi = 0; wi < 4 && !status; ++wi) {
            double ms = 0.0;
            status = time_of(ci, waves[wi] * 1024.0 * 1024.0, &ms);
            if (status) break;
            ++out->candidates;
            if (ms < best) { best = ms; bc = ci; bw = waves[wi] * 1024.0 * 1024.0; }
            if (ci == maxc && waves[wi] * 1024.0 * 1024.0 == kWaveBytes) out->ms_model = ms;
        }
    }
    if (!status) status = gbh_plan_status(plan, stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the caller's grids again
    if (was_bound) {
        const int e = gbh_plan_bind(plan, saved.data(), stream);
        if (!status) status = e;
    } else {
        plan->bound = false;
    }
    cudaStreamSynchronize(s);
    cudaFree(scratch);
    if (status) {
        set_params(plan, op, c0, w0);
        return status;
    }
    out->ctas_per_sm = bc;
    out->wave_mb = (int)(bw / (1024.0 * 1024.0) + 0.5);
    out->ms_tuned = best;
    out->max_ctas_per_sm = maxc;
    if (int e = set_params(plan, op, bc, bw)) return e;
    if (plan->full_scheme) {
        std::lock_guard<std::mutex> lk(g_scheme_tune_mu);
        g_scheme_tuned[std::vector<int>{plan->d, plan->n, plan->dtype, op}] = std::make_pair(bc, bw);
    }
    return GBH_OK;
}

int gbh_plan_status(gbh_plan *plan, void *stream)
{
    if (!plan) return GBH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int st = 0;
    unsigned char *word = plan->d_scratch + plan->scratch_bytes;
    if (cudaMemcpyAsync(&st, word, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return GBH_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GBH_ECUDA;
    if (st != 0) {
        if (cudaMemsetAsync(word, 0, sizeof(int), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
            return GBH_ECUDA;
    }
    return st;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched transform without any allocation
// ---------------------------------------------------------------------------
//
// For callers that must not allocate device memory: code that runs while a
// framework's caching allocator owns the whole device, code inside a memory
// budget that forbids hidden allocations, or code that may not call
// cudaMalloc at all at that point.  The work queue, its counters and the
// per-grid tables live in one file-scope device array of fixed size instead of
// in a plan; the kernel is the plan's k_batched.  The array's device address
// is looked up once per device (by the first call on that device).  Every
// call shares the array
// and rewrites it: calls that overlap on the GPU race; the counters are
// cleared by every call.  The first 256 bytes hold a status word that no call
// clears: a bounded wait that gives up sets it to GBH_ETIMEOUT, and
// gbh_batched_transform_noalloc_status reads and clears it.

namespace {

constexpr size_t kNoAllocBytes = 4u << 20;        // device work tables, per device
constexpr int kNoAllocMaxGrids = 2048;
constexpr int64_t kNoAllocItemPoints = 65536;      // points per work item

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocHost {
    GridInfo info[kNoAllocMaxGrids];
    int need[kNoAllocMaxGrids * kPhases];
    void *ptrs[kNoAllocMaxGrids];
    int order[kNoAllocMaxGrids];
    Item items[kNoAllocBytes / sizeof(Item)];
};
static NoAllocHost g_na_host;                      // host staging, no heap
static unsigned char *g_na_dev[64];                // symbol address per device
static int g_na_stall_grid = -1;                   // failure injection (tests)
static long long g_na_spin_limit = kSpinLimit;

size_t na_align(size_t x) { return (x + 255) / 256 * 256; }

// The array's device address on the current device (looked up once).
unsigned char *na_base()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!g_na_dev[dev]) {
        unsigned char *ptr = nullptr;
        if (cudaGetSymbolAddress(reinterpret_cast<void **>(&ptr), g_noalloc_scratch) != cudaSuccess || !ptr)
            return nullptr;
        g_na_dev[dev] = ptr;
    }
    return g_na_dev[dev];
}

}  // namespace

extern "C" int gbh_batched_transform_noalloc(int n_grids, int d, const int32_t *levels, void *const *grid_ptrs,
                                             int dtype, int op, void *stream)
{
    if (!levels || !grid_ptrs || n_grids < 1 || d < 1 || d > kPlanMaxD) return GBH_EINVAL;
    if (dtype != GBH_F32 && dtype != GBH_F64) return GBH_EDTYPE;
    if (op != GBH_HIERARCHIZE && op != GBH_DEHIERARCHIZE) return (op == GBH_ADJOINT || op == GBH_DEHIERARCHIZE_ADJOINT) ? GBH_EUNSUPPORTED : GBH_EINVAL;
    if (n_grids > kNoAllocMaxGrids) return GBH_ERANGE;
    const size_t es = dtype == GBH_F64 ? 8 : 4;
    // per-grid geometry
    for (int g = 0; g < n_grids; ++g) {
        if (!grid_ptrs[g]) return GBH_EINVAL;
        if (reinterpret_cast<uintptr_t>(grid_ptrs[g]) % es) return GBH_EALIGN;
        GridInfo &gi = g_na_host.info[g];
        std::memset(&gi, 0, sizeof(gi));
        gi.first_dim = gi.last_dim = -1;
        int64_t N = 1;
        double growth = 1.0;
        for (int k = 0; k < d; ++k) {
            const int l = levels[(size_t)g * d + k];
            if (l < 0 || l > kGroupLevel + 5) return GBH_ERANGE;
            const int64_t nk = ((int64_t)1 << l) + 1;
            if (N > INT64_MAX / 8 / nk) return GBH_ERANGE;
            gi.l[k] = l;
            gi.S[k] = N;
            gi.divS[k] = make_fastdiv(N);
            N *= nk;
            if (l > 0) {
                if (gi.first_dim < 0) gi.first_dim = k;
                gi.last_dim = k;
                ++gi.passes;
                growth *= dgrowth(std::min(l, 16));
            }
        }
        gi.N = N;
        gi.g0 = 61 - 2 * gi.passes;
        gi.g0_d = 61 - (int)std::ceil(std::log2(growth) + 1e-9);
        g_na_host.ptrs[g] = grid_ptrs[g];
        g_na_host.order[g] = g;
    }
    // device layout: sticky status | counters | need | ptrs | info | items
    const size_t o_sticky = 0, o_ticket = 256, o_status = 288, o_emax = 320;
    const size_t o_done = na_align(o_emax + sizeof(int) * (size_t)n_grids);
    const size_t o_need = na_align(o_done + sizeof(int) * (size_t)n_grids * kPhases);
    const size_t o_ptrs = na_align(o_need + sizeof(int) * (size_t)n_grids * kPhases);
    const size_t o_info = na_align(o_ptrs + sizeof(void *) * (size_t)n_grids);
    const size_t o_items = na_align(o_info + sizeof(GridInfo) * (size_t)n_grids);
    if (o_items >= kNoAllocBytes) return GBH_ERANGE;
    const int cap = (int)std::min<size_t>((kNoAllocBytes - o_items) / sizeof(Item),
                                          sizeof(g_na_host.items) / sizeof(Item));
    // items in the plan's ticket order
    int nitems = 0;
    static int na_wave[kNoAllocMaxGrids], na_prev[kNoAllocMaxGrids];
    const bool ok = order_items(g_na_host.info, n_grids, d, dtype, op, kNoAllocItemPoints, kWaveBytes, false,
                                g_na_host.order, na_wave, na_prev, g_na_host.need, [&](const Item &it) {
                                    if (nitems >= cap) return false;
                                    g_na_host.items[nitems++] = it;
                                    return true;
                                });
    if (!ok) return GBH_ERANGE;
    // set-up: the array's device address, once per device
    unsigned char *base = na_base();
    if (!base) return GBH_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // counters start at zero; the tables are rewritten by every call; the
    // sticky status word is left alone
    if (cudaMemsetAsync(base + o_ticket, 0, o_need - o_ticket, s) != cudaSuccess) return GBH_ECUDA;
    if (cudaMemcpyAsync(base + o_need, g_na_host.need, sizeof(int) * (size_t)n_grids * kPhases, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(base + o_ptrs, g_na_host.ptrs, sizeof(void *) * (size_t)n_grids, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(base + o_info, g_na_host.info, sizeof(GridInfo) * (size_t)n_grids, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(base + o_items, g_na_host.items, sizeof(Item) * (size_t)nitems, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return GBH_ECUDA;
    BatchParams P{};
    P.spin_limit = g_na_spin_limit;
    P.stall_grid = g_na_stall_grid < n_grids ? g_na_stall_grid : -1;
    P.items = reinterpret_cast<const Item *>(base + o_items);
    P.nitems = nitems;
    P.grids = reinterpret_cast<const GridInfo *>(base + o_info);
    P.ptrs = reinterpret_cast<void *const *>(base + o_ptrs);
    P.ticket = reinterpret_cast<unsigned *>(base + o_ticket);
    P.status = reinterpret_cast<int *>(base + o_status);
    P.sticky = reinterpret_cast<int *>(base + o_sticky);
    P.emax = reinterpret_cast<int *>(base + o_emax);
    P.done = reinterpret_cast<int *>(base + o_done);
    P.need = reinterpret_cast<const int *>(base + o_need);
    P.op = op;
    if (nitems == 0) return GBH_OK;
    const size_t smem = kGroupElems * es + kGroupElems * sizeof(int64_t) / 2;
    auto launch = [&](auto kern) -> int {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBThreads, smem);
        if (per_sm < 1) return GBH_EUNSUPPORTED;
        const int grid = std::max(1, std::min(num_sms() * per_sm, nitems));
        kern<<<grid, kBThreads, smem, s>>>(P);
        count_launches(1);
        return check_launch();
    };
    if (dtype == GBH_F64)
        return op == GBH_HIERARCHIZE ? launch(k_batched<double, OP_H>) : launch(k_batched<double, OP_D>);
    return op == GBH_HIERARCHIZE ? launch(k_batched<float, OP_H>) : launch(k_batched<float, OP_D>);
}

extern "C" int gbh_batched_transform_noalloc_status(void *stream)
{
    unsigned char *base = na_base();
    if (!base) return GBH_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int st = 0;    // pageable host memory: the copy has completed when the call returns
    if (cudaMemcpyAsync(&st, base, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GBH_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GBH_ECUDA;
    const int out = st;
    if (out != 0) {
        if (cudaMemsetAsync(base, 0, sizeof(int), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
            return GBH_ECUDA;
    }
    return out;
}

extern "C" int gbh_batched_transform_noalloc_test_stall(int grid, long long spin_limit)
{
    if (grid < -1 || grid >= kNoAllocMaxGrids || spin_limit < 1) return GBH_EINVAL;
    g_na_stall_grid = grid;
    g_na_spin_limit = grid < 0 ? kSpinLimit : spin_limit;
    return GBH_OK;
}
