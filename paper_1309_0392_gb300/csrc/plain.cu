// Plain path: one in-place sweep kernel per dimension.  With native fp32/fp64
// arithmetic every point is computed in the operation order of the serial
// algorithm (so fp64 results are bit-identical to a serial run of Alg. 1 in
// dimension order 0..d-1); fp64 may instead compute in int64 fixed point.
//
//   pole-group kernel  any dimension whose poles fit in shared memory: a CTA
//                      stages a group of poles (rows of dimension 0, or
//                      neighbouring poles of an outer dimension side by side),
//                      so that every global access is coalesced whichever way
//                      the poles run through memory (Sec. 3 discusses the
//                      cost of working along versus across the data layout).
//   pole kernel        short poles of dimensions k >= 1 (up to 33 points):
//                      one thread per pole, held in registers; neighbouring
//                      threads own neighbouring poles (Sec. 3, Fig. 3 right).
//   level kernel       any dimension with few, long poles: one launch per level,
//                      threads over (pole, point of that level).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "gbh_internal.h"

namespace gbh {
namespace {

enum { OP_H = GBH_HIERARCHIZE, OP_D = GBH_DEHIERARCHIZE, OP_A = GBH_ADJOINT, OP_DT = GBH_DEHIERARCHIZE_ADJOINT };

constexpr int kRegPoleMaxLevel = 5;      // poles up to 33 points kept in registers (65 for fp32)
constexpr int64_t kMinPolesForThreadPerPole = 152 * 64;

// ---------------------------------------------------------------------------
// 1-D pole transforms; the loop order is that of Alg. 1 (fine to coarse) for
// hierarchization, coarse to fine for the inverse and the transpose, fine to
// coarse for the transpose of the inverse.
// ---------------------------------------------------------------------------

template <typename T, int OP, int L>
__device__ __forceinline__ void transform_regs(T *v)
{
    constexpr int last = 1 << L;
    if (OP == OP_H) {
#pragma unroll
        for (int lev = L; lev >= 1; --lev) {
            const int s = 1 << (L - lev);
#pragma unroll
            for (int i = s; i < last; i += 2 * s) v[i] = v[i] - T(0.5) * (v[i - s] + v[i + s]);
        }
    } else if (OP == OP_D) {
#pragma unroll
        for (int lev = 1; lev <= L; ++lev) {
            const int s = 1 << (L - lev);
#pragma unroll
            for (int i = s; i < last; i += 2 * s) v[i] = v[i] + T(0.5) * (v[i - s] + v[i + s]);
        }
    } else if (OP == OP_A) {
#pragma unroll
        for (int lev = 1; lev <= L; ++lev) {
            const int s = 1 << (L - lev);
#pragma unroll
            for (int i = s; i < last; i += 2 * s) {
                v[i - s] = v[i - s] - T(0.5) * v[i];
                v[i + s] = v[i + s] - T(0.5) * v[i];
            }
        }
    } else {
#pragma unroll
        for (int lev = L; lev >= 1; --lev) {
            const int s = 1 << (L - lev);
#pragma unroll
            for (int i = s; i < last; i += 2 * s) {
                v[i - s] = v[i - s] + T(0.5) * v[i];
                v[i + s] = v[i + s] + T(0.5) * v[i];
            }
        }
    }
}

template <typename T, int OP>
__device__ __forceinline__ void transform_global(T *__restrict__ p, int64_t S, int l)
{
    const int64_t last = (int64_t)1 << l;
    if (OP == OP_H) {
        for (int lev = l; lev >= 1; --lev) {
            const int64_t s = (int64_t)1 << (l - lev);
            for (int64_t i = s; i < last; i += 2 * s)
                p[i * S] = p[i * S] - T(0.5) * (p[(i - s) * S] + p[(i + s) * S]);
        }
    } else if (OP == OP_D) {
        for (int lev = 1; lev <= l; ++lev) {
            const int64_t s = (int64_t)1 << (l - lev);
            for (int64_t i = s; i < last; i += 2 * s)
                p[i * S] = p[i * S] + T(0.5) * (p[(i - s) * S] + p[(i + s) * S]);
        }
    } else if (OP == OP_A) {
        for (int lev = 1; lev <= l; ++lev) {
            const int64_t s = (int64_t)1 << (l - lev);
            for (int64_t i = s; i < last; i += 2 * s) {
                const T v = p[i * S];
                p[(i - s) * S] = p[(i - s) * S] - T(0.5) * v;
                p[(i + s) * S] = p[(i + s) * S] - T(0.5) * v;
            }
        }
    } else {
        for (int lev = l; lev >= 1; --lev) {
            const int64_t s = (int64_t)1 << (l - lev);
            for (int64_t i = s; i < last; i += 2 * s) {
                const T v = p[i * S];
                p[(i - s) * S] = p[(i - s) * S] + T(0.5) * v;
                p[(i + s) * S] = p[(i + s) * S] + T(0.5) * v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// pole kernel: one thread per pole of dimension k >= 1
// ---------------------------------------------------------------------------

template <typename T, int OP, int L>
__global__ void __launch_bounds__(256) k_pole_regs(T *__restrict__ u, int64_t S, int64_t poles)
{
    constexpr int n = (1 << L) + 1;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < poles;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = t / S, j = t - o * S;
        T *p = u + o * S * n + j;
        T v[n];
#pragma unroll
        for (int i = 0; i < n; ++i) v[i] = p[i * S];
        transform_regs<T, OP, L>(v);
#pragma unroll
        for (int i = 0; i < n; ++i)
            if (OP == OP_A || OP == OP_DT || (i > 0 && i < n - 1)) p[i * S] = v[i];
    }
}

template <typename T, int OP>
__global__ void __launch_bounds__(256) k_pole_global(T *__restrict__ u, int64_t S, int64_t poles, int l)
{
    const int64_t n = ((int64_t)1 << l) + 1;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < poles;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = t / S, j = t - o * S;
        transform_global<T, OP>(u + o * S * n + j, S, l);
    }
}

// ---------------------------------------------------------------------------
// level kernel: one launch per level, threads over (pole, point of the level)
// ---------------------------------------------------------------------------

// H / D: the level-lev points i = (2q+1) s of every pole.
// Transposes: the points p = 2 s q that receive from level-lev children
// p -/+ s (left, then right: the order of the serial scatter).
template <typename T, int OP>
__global__ void __launch_bounds__(256) k_level(T *__restrict__ u, int64_t S, int64_t n, int64_t outer,
                                               int l, int lev)
{
    const int64_t s = (int64_t)1 << (l - lev);
    const int64_t per = (OP == OP_A || OP == OP_DT) ? (((int64_t)1 << (lev - 1)) + 1) : ((int64_t)1 << (lev - 1));
    const int64_t items = outer * S * per;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < items;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = w % S;
        const int64_t rest = w / S;
        const int64_t q = rest % per, o = rest / per;
        T *p = u + o * S * n + j;
        if (OP == OP_A || OP == OP_DT) {
            const int64_t i = 2 * s * q;
            T y = p[i * S];
            if (OP == OP_A) {
                if (q > 0) y = y - T(0.5) * p[(i - s) * S];
                if (q < per - 1) y = y - T(0.5) * p[(i + s) * S];
            } else {
                if (q > 0) y = y + T(0.5) * p[(i - s) * S];
                if (q < per - 1) y = y + T(0.5) * p[(i + s) * S];
            }
            p[i * S] = y;
        } else {
            const int64_t i = (2 * q + 1) * s;
            const T sum = p[(i - s) * S] + p[(i + s) * S];
            p[i * S] = (OP == OP_H) ? p[i * S] - T(0.5) * sum : p[i * S] + T(0.5) * sum;
        }
    }
}

// ---------------------------------------------------------------------------
// pole-group kernel: a group of poles staged in shared memory
// ---------------------------------------------------------------------------
//
// G poles of one dimension (length n = 2^l + 1, stride S) per CTA.  Poles of
// dimension k >= 1 are loaded side by side (neighbouring poles are contiguous,
// Sec. 3, Fig. 3 right: work orthogonal to the poles), rows of dimension 0
// row after row; either way every global access is coalesced, and all loads
// of the group are in flight at once (cp.async).  Then:
//   H  every surplus from the staged nodal values in one step (the two
//      neighbours of a point are always coarser, hence still nodal);
//   D  level by level, coarse to fine, in shared memory;
//   A  y[p] = x[p] - 1/2 sum over the children of p: in fixed point every
//      point at once from the staged values; natively level by level, coarse
//      to fine, each parent gathering from its two children of that level
//      (left, then right: the order of the serial scatter).
// Boundary points are not stored back by H and D (they do not change).
// FIX (fp64 only): the group is scaled by its largest binary exponent and
// computed in int64 fixed point: H and A exactly (doubling forms 2u - L - R
// and 2x - sum of children), D with halved sums; one int64 -> fp64 conversion
// per stored point replaces the fp64 arithmetic.
constexpr int kGroupElems = 8192;        // elements staged per CTA (target)
constexpr int kGroupMaxElems = 16385;    // longest pole staged whole

__device__ __forceinline__ void pg_cp8(void *smem_dst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void pg_cp4(void *smem_dst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void pg_commit_wait()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ long long g_to_fixed(long long bits, int emax, int c)
{
    const int e = (int)((unsigned long long)bits >> 52) & 0x7FF;
    if (e == 0) return 0;
    const unsigned long long M = ((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = c - (emax - e);
    long long v;
    if (sh >= 0) v = (long long)(M << sh);
    else v = (-sh >= 63) ? 0 : (long long)(M >> (-sh));
    return bits < 0 ? -v : v;
}

// v * 2^X for any X (slow path: exponents near the ends of the range)
__device__ __noinline__ double g_from_fixed_slow(long long v, int X)
{
    if (v == 0) return 0.0;
    return ldexp(__ll2double_rn(v), X);
}

// v * 2^X by adding X to the exponent field; valid while the result stays
// normal, which the caller guarantees (group exponent in [64, 1900])
__device__ __forceinline__ double g_from_fixed_fast(long long v, long long Xhi)
{
    const long long b = __double_as_longlong(__ll2double_rn(v));
    return __longlong_as_double(v == 0 ? 0ll : b + Xhi);
}

// ROWS: poles are rows of n contiguous elements, row r starting at r * rs
// (rs = n for the rows of dimension 0; rs = n - 1 for the dyadic blocks of a
// long pole, which share their end points).  Otherwise pole t is the pole
// (t / S, t % S) of a dimension with stride S.
template <typename T, int OP, bool FIX, bool ROWS>
__global__ void __launch_bounds__(256) k_pole_group(T *__restrict__ u, int64_t S, int64_t poles, int l, int G,
                                                    int g0, int64_t rs)
{
    using V = typename std::conditional<FIX, long long, T>::type;
    extern __shared__ __align__(16) unsigned char smr[];
    V *sv = reinterpret_cast<V *>(smr);
    __shared__ int s_emax;
    const int n = (1 << l) + 1, last = 1 << l;
    const int64_t t0 = (int64_t)blockIdx.x * G;
    const int Gc = (poles - t0) < (int64_t)G ? (int)(poles - t0) : G;
    const int cnt = Gc * n;
    int64_t *pb = reinterpret_cast<int64_t *>(smr + (((size_t)G * n * sizeof(V) + 15) & ~(size_t)15));
    const unsigned magG = Gc == 1 ? 0u : (0xFFFFFFFFu / (unsigned)Gc) + 1u;
    const unsigned magN = (0xFFFFFFFFu / (unsigned)n) + 1u;
    if (!ROWS) {
        for (int g = threadIdx.x; g < Gc; g += blockDim.x) {
            const int64_t t = t0 + g, o = t / S;
            pb[g] = o * S * n + (t - o * S);
        }
    }
    if (threadIdx.x == 0) s_emax = 0;
    __syncthreads();
    // element w of the group (the order of the global accesses): its global
    // address, its shared-memory slot and its index i along the pole
    auto locate = [&](int w, int &sidx, int &i) -> int64_t {
        if (ROWS) {
            sidx = w;
            const int r = (int)__umulhi((unsigned)w, magN);
            i = w - r * n;
            return (t0 + r) * rs + i;
        }
        i = magG ? (int)__umulhi((unsigned)w, magG) : w;
        const int g = w - i * Gc;
        sidx = g * n + i;
        return pb[g] + (int64_t)i * S;
    };
    for (int w = threadIdx.x; w < cnt; w += blockDim.x) {
        int sidx, i;
        const int64_t a = locate(w, sidx, i);
        if constexpr (sizeof(T) == 8) pg_cp8(sv + sidx, u + a);
        else pg_cp4(sv + sidx, u + a);
    }
    pg_commit_wait();
    __syncthreads();

    int X = 0;
    long long Xhi = 0;
    bool fast = true;
    if constexpr (FIX) {
        int emax = 0;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x)
            emax = max(emax, (int)((unsigned long long)sv[e] >> 52) & 0x7FF);
        emax = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)emax);
        if ((threadIdx.x & 31) == 0) atomicMax(&s_emax, emax);
        __syncthreads();
        emax = s_emax;
        const int c = g0 - 53;
        X = emax - 1075 - c - (OP == OP_D ? 0 : 1);    // H and A: doubled results
        Xhi = (long long)X << 52;
        fast = emax >= 64 && emax <= 1900;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) sv[e] = g_to_fixed((long long)sv[e], emax, c);
        __syncthreads();
    }
    auto put = [&](int64_t a, V y) {
        if constexpr (FIX) u[a] = fast ? g_from_fixed_fast(y, Xhi) : g_from_fixed_slow(y, X);
        else u[a] = y;
    };
    if (OP == OP_H) {
        for (int w = threadIdx.x; w < cnt; w += blockDim.x) {
            int sidx, i;
            const int64_t a = locate(w, sidx, i);
            if (i == 0 || i == last) continue;
            const int s = i & (-i);
            const V *p = sv + sidx;
            if constexpr (FIX) put(a, (p[0] + p[0]) - p[-s] - p[s]);
            else put(a, p[0] - V(0.5) * (p[-s] + p[s]));
        }
    } else if (OP == OP_D) {
        for (int lev = 1; lev <= l; ++lev) {
            const int s = 1 << (l - lev), per = 1 << (lev - 1);
            for (int q = threadIdx.x; q < Gc * per; q += blockDim.x) {
                const int r = q >> (lev - 1), i = (2 * (q & (per - 1)) + 1) * s;
                V *row = sv + r * n;
                if constexpr (FIX) row[i] = row[i] + ((row[i - s] + row[i + s]) >> 1);
                else row[i] = row[i] + V(0.5) * (row[i - s] + row[i + s]);
            }
            __syncthreads();
        }
        for (int w = threadIdx.x; w < cnt; w += blockDim.x) {
            int sidx, i;
            const int64_t a = locate(w, sidx, i);
            if (i == 0 || i == last) continue;
            put(a, sv[sidx]);
        }
    } else if (OP == OP_DT) {
        // level by level, fine to coarse: the parents p = 2 s q of level-lev
        // children take half of each child's value (left, then right); a
        // child's value is final once every finer level has been gathered
        for (int lev = l; lev >= 1; --lev) {
            const int s = 1 << (l - lev), per = (1 << (lev - 1)) + 1;
            for (int w = threadIdx.x; w < Gc * per; w += blockDim.x) {
                const int r = w / per, q = w - r * per, p = 2 * s * q;
                V *row = sv + r * n;
                V y = row[p];
                if (q > 0) y = y + V(0.5) * row[p - s];
                if (q < per - 1) y = y + V(0.5) * row[p + s];
                row[p] = y;
            }
            __syncthreads();
        }
        for (int w = threadIdx.x; w < cnt; w += blockDim.x) {
            int sidx, i;
            const int64_t a = locate(w, sidx, i);
            put(a, sv[sidx]);
        }
    } else if constexpr (FIX) {
        // every point at once from the staged values (exact):
        // 2 y[p] = 2 x[p] - sum_{t < lowbit(p)} (x[p - t] + x[p + t])
        for (int w = threadIdx.x; w < cnt; w += blockDim.x) {
            int sidx, i;
            const int64_t a = locate(w, sidx, i);
            const V *p = sv + sidx;
            const int top = (i == 0 || i == last) ? (last >> 1) : ((i & (-i)) >> 1);
            V y = p[0] + p[0];
            for (int t = top; t >= 1; t >>= 1) {
                if (i != 0) y -= p[-t];
                if (i != last) y -= p[t];
            }
            put(a, y);
        }
    } else {
        // level by level, coarse to fine: the parents p = 2 s q of level-lev
        // children take their contributions (left, then right); a child's own
        // value changes only at finer levels, so it is still x when read
        for (int lev = 1; lev <= l; ++lev) {
            const int s = 1 << (l - lev), per = (1 << (lev - 1)) + 1;
            for (int w = threadIdx.x; w < Gc * per; w += blockDim.x) {
                const int r = w / per, q = w - r * per, p = 2 * s * q;
                V *row = sv + r * n;
                V y = row[p];
                if (q > 0) y = y - V(0.5) * row[p - s];
                if (q < per - 1) y = y - V(0.5) * row[p + s];
                row[p] = y;
            }
            __syncthreads();
        }
        for (int w = threadIdx.x; w < cnt; w += blockDim.x) {
            int sidx, i;
            const int64_t a = locate(w, sidx, i);
            put(a, sv[sidx]);
        }
    }
}

// ---------------------------------------------------------------------------
// host dispatch
// ---------------------------------------------------------------------------

int grid_for(int64_t items, int threads)
{
    const int64_t want = (items + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * 32;
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

template <typename T, int OP, int L>
int launch_pole_regs(T *u, int64_t S, int64_t poles, cudaStream_t st)
{
    ProfScope ps("plain_pole_regs", st, 2.0 * sizeof(T) * (double)poles * ((1 << L) + 1));
    k_pole_regs<T, OP, L><<<grid_for(poles, 256), 256, 0, st>>>(u, S, poles);
    ps.done();
    count_launches(1);
    return check_launch();
}

template <typename T, int OP>
int sweep_level(T *u, const Geom &g, int k, cudaStream_t st)
{
    const int l = g.l[k];
    const int64_t outer = g.total / (g.S[k] * g.n[k]);
    if (OP == OP_H) {
        for (int lev = l; lev >= 1; --lev) {
            const int64_t items = outer * g.S[k] * ((int64_t)1 << (lev - 1));
            ProfScope ps("plain_level", st, 2.0 * sizeof(T) * (double)items);
            k_level<T, OP><<<grid_for(items, 256), 256, 0, st>>>(u, g.S[k], g.n[k], outer, l, lev);
            ps.done();
            count_launches(1);
            if (int e = check_launch()) return e;
        }
    } else if (OP == OP_DT) {
        for (int lev = l; lev >= 1; --lev) {
            const int64_t items = outer * g.S[k] * (((int64_t)1 << (lev - 1)) + 1);
            ProfScope ps("plain_level", st, 2.0 * sizeof(T) * (double)items);
            k_level<T, OP><<<grid_for(items, 256), 256, 0, st>>>(u, g.S[k], g.n[k], outer, l, lev);
            ps.done();
            count_launches(1);
            if (int e = check_launch()) return e;
        }
    } else {
        for (int lev = 1; lev <= l; ++lev) {
            const int64_t per = (OP == OP_A) ? (((int64_t)1 << (lev - 1)) + 1) : ((int64_t)1 << (lev - 1));
            const int64_t items = outer * g.S[k] * per;
            ProfScope ps("plain_level", st, 2.0 * sizeof(T) * (double)items);
            k_level<T, OP><<<grid_for(items, 256), 256, 0, st>>>(u, g.S[k], g.n[k], outer, l, lev);
            ps.done();
            count_launches(1);
            if (int e = check_launch()) return e;
        }
    }
    return GBH_OK;
}

// poles of level l: rows at stride rs (ROWS), else the poles of a dimension
// of stride S; `bytes` is the launch's algorithmic traffic
template <typename T, int OP, bool FIX, bool ROWS>
int launch_group_raw(T *u, int64_t S, int64_t rs, int64_t poles, int l, double bytes, cudaStream_t st)
{
    const int n = (1 << l) + 1;
    const int G = std::max(1, kGroupElems / n);
    const int64_t blocks = (poles + G - 1) / G;
    if (blocks > INT32_MAX) return GBH_ERANGE;
    using V = typename std::conditional<FIX, long long, T>::type;
    const size_t smem = (((size_t)G * n * sizeof(V) + 15) & ~(size_t)15) + (ROWS ? 0 : (size_t)G * sizeof(int64_t));
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_pole_group<T, OP, FIX, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((kGroupMaxElems + kGroupElems / 3 + 4) * sizeof(long long)));
        attr = true;
    }
    // fixed-point headroom below 2^63: H doubles once (|2u - L - R| <= 4 max);
    // D grows by at most l + 1 (hat weights along a pole sum to at most l + 1);
    // A sums at most 2 l children besides the doubled point
    const int g0 = OP == OP_H ? 59 : 59 - (int)std::ceil(std::log2((double)l + 1.0));
    ProfScope ps(ROWS ? "plain_rows_group" : "plain_pole_group", st, bytes);
    k_pole_group<T, OP, FIX, ROWS><<<(unsigned)blocks, 256, smem, st>>>(u, S, poles, l, G, g0, rs);
    ps.done();
    count_launches(1);
    return check_launch();
}

template <typename T, int OP, bool FIX, bool ROWS>
int launch_group(T *u, const Geom &g, int k, cudaStream_t st)
{
    return launch_group_raw<T, OP, FIX, ROWS>(u, g.S[k], g.n[k], g.total / g.n[k], g.l[k],
                                              2.0 * sizeof(T) * (double)g.total, st);
}

// One long pole (a single grid of one dimension, level 14 < L <= 28) by the
// dyadic split of its index set: with blocks of level m, the points that are
// not multiples of 2^m have both predecessors inside their block
// [a 2^m, (a+1) 2^m], so hierarchization is a level-m transform of every
// block (end points read, never written) followed by a level L-m transform
// of the coarse pole of the multiples of 2^m, which reads only those.  The
// inverse runs the two parts in the opposite order.  Each transform keeps
// the per-point operation of Alg. 1, so results equal the per-level sweep.
template <typename T, int OP, bool FIX>
int long_pole_split(T *u, int L, cudaStream_t st)
{
    const int m = std::max(13, L - 14);
    const int64_t bm = (int64_t)1 << m, blocks = (int64_t)1 << (L - m);
    const double bytes = 2.0 * sizeof(T) * (double)(((int64_t)1 << L) + 1);
    auto fine = [&] { return launch_group_raw<T, OP, FIX, true>(u, 1, bm, blocks, m, bytes, st); };
    auto coarse = [&] {
        return launch_group_raw<T, OP, FIX, false>(u, bm, 0, 1, L - m, 2.0 * sizeof(T) * (double)(blocks + 1), st);
    };
    if (OP == OP_H) {
        if (int e = fine()) return e;
        return coarse();
    }
    if (int e = coarse()) return e;
    return fine();
}

template <typename T, int OP>
int sweep_dim(T *u, const Geom &g, int k, cudaStream_t st, bool fixed)
{
    const int l = g.l[k];
    const int64_t poles = g.total / g.n[k];
    // fp64 may compute in fixed point; the transpose of D runs natively
    constexpr bool kFixable = sizeof(T) == 8 && OP != OP_DT;
    const bool fix = kFixable && fixed;
    if (k == 0) {
        if (g.n[0] > kGroupMaxElems) {
            if ((OP == OP_H || OP == OP_D) && g.d == 1 && g.batch == 1 && l <= 28)
                return fix ? long_pole_split<T, OP, kFixable>(u, l, st) : long_pole_split<T, OP, false>(u, l, st);
            return sweep_level<T, OP>(u, g, 0, st);
        }
        return fix ? launch_group<T, OP, kFixable, true>(u, g, 0, st) : launch_group<T, OP, false, true>(u, g, 0, st);
    }
    if (fix && g.n[k] <= kGroupElems) return launch_group<T, OP, kFixable, false>(u, g, k, st);
    // fp32 poles of 65 points still fit in registers
    if constexpr (sizeof(T) == 4)
        if (l == kRegPoleMaxLevel + 1) return launch_pole_regs<T, OP, kRegPoleMaxLevel + 1>(u, g.S[k], poles, st);
    if (l <= kRegPoleMaxLevel) {
        switch (l) {
            case 1: return launch_pole_regs<T, OP, 1>(u, g.S[k], poles, st);
            case 2: return launch_pole_regs<T, OP, 2>(u, g.S[k], poles, st);
            case 3: return launch_pole_regs<T, OP, 3>(u, g.S[k], poles, st);
            case 4: return launch_pole_regs<T, OP, 4>(u, g.S[k], poles, st);
            default: return launch_pole_regs<T, OP, 5>(u, g.S[k], poles, st);
        }
    }
    if (g.n[k] <= kGroupElems) return launch_group<T, OP, false, false>(u, g, k, st);
    if (poles < kMinPolesForThreadPerPole) return sweep_level<T, OP>(u, g, k, st);
    ProfScope ps("plain_pole_global", st, 2.0 * sizeof(T) * (double)g.total);
    k_pole_global<T, OP><<<grid_for(poles, 256), 256, 0, st>>>(u, g.S[k], poles, l);
    ps.done();
    count_launches(1);
    return check_launch();
}

template <typename T, int OP>
int plain_all(T *u, const Geom &g, cudaStream_t st, bool fixed)
{
    for (int k = 0; k < g.d; ++k) {
        if (g.l[k] == 0) continue;
        if (int e = sweep_dim<T, OP>(u, g, k, st, fixed)) return e;
    }
    return GBH_OK;
}

template <typename T>
int plain_dispatch(T *u, const Geom &g, int op, cudaStream_t st, bool fixed)
{
    switch (op) {
        case OP_H: return plain_all<T, OP_H>(u, g, st, fixed);
        case OP_D: return plain_all<T, OP_D>(u, g, st, fixed);
        case OP_A: return plain_all<T, OP_A>(u, g, st, fixed);
        case OP_DT: return plain_all<T, OP_DT>(u, g, st, false);
        default: return GBH_EINVAL;
    }
}

}  // namespace

int plain_transform(void *data, const Geom &g, int dtype, int op, cudaStream_t s, bool fixed64)
{
    if (dtype == GBH_F64) return plain_dispatch<double>(static_cast<double *>(data), g, op, s, fixed64);
    if (dtype == GBH_F32) return plain_dispatch<float>(static_cast<float *>(data), g, op, s, false);
    return GBH_EDTYPE;
}

}  // namespace gbh
