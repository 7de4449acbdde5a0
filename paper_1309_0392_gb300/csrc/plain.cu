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
// pair kernel: dimensions a and a+1 in one pass (native arithmetic)
// ---------------------------------------------------------------------------
//
// A CTA stages a tile that holds whole poles of both dimensions, sweeps
// dimension a and then dimension a+1 in shared memory (one thread per pole,
// the pole held in registers as in the pole kernel) and stores the tile back:
// one crossing of memory for two dimensions.  Every point receives the same
// operations in the same order as from two single-dimension sweeps, so the
// results are bit-identical to them.
//   a = 0   (ROWS) Q consecutive planes of n0 x n1 points: one contiguous
//           range, copied in 16-byte pieces (the range's first element sits
//           at the shared-memory offset that makes both sides aligned).
//   a >= 1  B consecutive positions j of the dimensions below a (a run of B
//           elements at every (i_a, i_{a+1})), B a power of two, for one
//           index o of the dimensions above a+1; shared index jj + B r with
//           r = i_a + n_a i_{a+1}.  Neighbouring threads own neighbouring
//           poles, so the strided pole reads are free of bank conflicts.
constexpr int kPairThreads = 256;
constexpr int kPairBytes = 104 * 1024;   // two CTAs per SM

template <typename T>
__host__ __device__ constexpr int pair_max_level()
{
    return sizeof(T) == 4 ? 6 : 5;       // pole of 65 (fp32) or 33 (fp64) in registers
}

__device__ __forceinline__ void lds_val(float &v, unsigned a)
{
    asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(a));
}
__device__ __forceinline__ void lds_val(double &v, unsigned a)
{
    asm volatile("ld.shared.f64 %0, [%1];\n" : "=d"(v) : "r"(a));
}
__device__ __forceinline__ void sts_val(unsigned a, float v)
{
    asm volatile("st.shared.f32 [%0], %1;\n" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void sts_val(unsigned a, double v)
{
    asm volatile("st.shared.f64 [%0], %1;\n" ::"r"(a), "d"(v) : "memory");
}

// One pole of 2^L + 1 points at shared address a, stride st bytes: loaded
// into registers, transformed, stored.  The store addresses start from an
// opaque copy of a, so that they are recomputed rather than kept live from
// the loads (which would hold one register per point).
template <typename T, int OP, int L>
__device__ __forceinline__ void pole_via_regs(unsigned a, unsigned st)
{
    constexpr int n = (1 << L) + 1;
    T v[n];
#pragma unroll
    for (int i = 0; i < n; ++i) lds_val(v[i], a + i * st);
    transform_regs<T, OP, L>(v);
    unsigned b;
    asm volatile("mov.b32 %0, %1;\n" : "=r"(b) : "r"(a));
#pragma unroll
    for (int i = 0; i < n; ++i)
        if (OP == OP_A || OP == OP_DT || (i > 0 && i < n - 1)) sts_val(b + i * st, v[i]);
}

// pole at p (shared memory), stride st elements, level l
template <typename T, int OP>
__device__ __forceinline__ void pole_shared(T *p, int st, int l)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p), sb = (unsigned)(st * (int)sizeof(T));
    switch (l) {
        case 1: pole_via_regs<T, OP, 1>(a, sb); break;
        case 2: pole_via_regs<T, OP, 2>(a, sb); break;
        case 3: pole_via_regs<T, OP, 3>(a, sb); break;
        case 4: pole_via_regs<T, OP, 4>(a, sb); break;
        case 5: pole_via_regs<T, OP, 5>(a, sb); break;
        default:
            if constexpr (pair_max_level<T>() >= 6) pole_via_regs<T, OP, 6>(a, sb);
            break;
    }
}

__device__ __forceinline__ void pg_cp16(void *smem_dst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}

template <typename T>
__device__ __forceinline__ void pg_cp(T *smem_dst, const T *gsrc)
{
    if constexpr (sizeof(T) == 8) pg_cp8(smem_dst, gsrc);
    else pg_cp4(smem_dst, gsrc);
}

// ROWS: units = planes, Q planes per CTA.  Otherwise units = bundles of Q
// positions (bpo per index o), Sa = stride of dimension a.
template <typename T, int OP, bool ROWS>
__global__ void __launch_bounds__(kPairThreads, 2)
k_pair(T *__restrict__ u, int64_t units, int64_t Sa, int64_t bpo, int la, int lb, int Q)
{
    extern __shared__ __align__(16) unsigned char smr[];
    T *sv = reinterpret_cast<T *>(smr);
    const int na = (1 << la) + 1, nb = (1 << lb) + 1, M = na * nb;
    const int tid = threadIdx.x;
    if constexpr (ROWS) {
        constexpr int VEC = 16 / sizeof(T);
        const int64_t p0 = (int64_t)blockIdx.x * Q;
        const int Qc = (int)((units - p0) < (int64_t)Q ? (units - p0) : (int64_t)Q);
        const int cnt = Qc * M;
        T *g = u + p0 * M;
        const int mis = (int)((reinterpret_cast<uintptr_t>(g) / sizeof(T)) & (VEC - 1));
        const int head = min(cnt, (VEC - mis) & (VEC - 1));
        const int body = (cnt - head) / VEC;
        const int tail = head + body * VEC;
        T *s = sv + mis;    // element e of the range at s[e]; s + head is 16-byte aligned
        for (int e = tid; e < head; e += kPairThreads) pg_cp(s + e, g + e);
        for (int c = tid; c < body; c += kPairThreads) pg_cp16(s + head + c * VEC, g + head + c * VEC);
        for (int e = tail + tid; e < cnt; e += kPairThreads) pg_cp(s + e, g + e);
        pg_commit_wait();
        __syncthreads();
        for (int q = tid; q < Qc * nb; q += kPairThreads) pole_shared<T, OP>(s + q * na, 1, la);
        __syncthreads();
        for (int q = tid; q < Qc * na; q += kPairThreads) {
            const int p = q / na, ia = q - p * na;
            pole_shared<T, OP>(s + p * M + ia, na, lb);
        }
        __syncthreads();
        for (int e = tid; e < head; e += kPairThreads) g[e] = s[e];
        for (int c = tid; c < body; c += kPairThreads)
            *reinterpret_cast<uint4 *>(g + head + c * VEC) = *reinterpret_cast<const uint4 *>(s + head + c * VEC);
        for (int e = tail + tid; e < cnt; e += kPairThreads) g[e] = s[e];
    } else {
        const int64_t o = (int64_t)blockIdx.x / bpo;
        const int64_t j0 = ((int64_t)blockIdx.x - o * bpo) * Q;
        const int Bc = (int)((Sa - j0) < (int64_t)Q ? (Sa - j0) : (int64_t)Q);
        T *g = u + o * Sa * M + j0;
        const int lgB = __ffs(Q) - 1;
        const int cnt = Q * M;
        // Q divides the block size: a thread keeps its jj, r steps by kPairThreads / Q
        const int jj = tid & (Q - 1);
        const int rstep = kPairThreads >> lgB;
        if (jj < Bc)
            for (int w = tid, r = tid >> lgB; w < cnt; w += kPairThreads, r += rstep)
                pg_cp(sv + w, g + jj + Sa * r);
        pg_commit_wait();
        __syncthreads();
        for (int q = tid; q < Q * nb; q += kPairThreads) {
            const int ib = q >> lgB;
            if (jj < Bc) pole_shared<T, OP>(sv + ib * na * Q + jj, Q, la);
        }
        __syncthreads();
        for (int q = tid; q < Q * na; q += kPairThreads) {
            const int ia = q >> lgB;
            if (jj < Bc) pole_shared<T, OP>(sv + ia * Q + jj, na * Q, lb);
        }
        __syncthreads();
        if (jj < Bc)
            for (int w = tid, r = tid >> lgB; w < cnt; w += kPairThreads, r += rstep)
                g[jj + Sa * r] = sv[w];
    }
}

// Square pairs of outer dimensions (a >= 1, l_a = l_b = L <= 5): no staging
// copy.  A CTA owns B consecutive positions j (square_run: runs of at least
// 64 bytes, more positions for short poles) and n = 2^L + 1 threads per
// position.  Thread (jj, q) loads the pole
// of dimension a at i_{a+1} = q straight from global memory into registers
// (a warp reads whole runs: coalesced), transforms it and parks it in shared
// memory; after one barrier it takes the pole of dimension a+1 at i_a = q
// from shared memory, transforms it and stores it to global memory.  Shared
// memory serves only the exchange between the two dimensions (one store and
// one load per point), and every thread keeps a whole pole of loads in
// flight.  Shared index (i_{a+1} n + i_a) B + jj: the two positions of q in
// a warp fall on opposite bank halves in both phases.
// positions per CTA: runs of at least 64 bytes, and for short poles as many
// positions as keep the CTA near 256 threads (a power of two)
template <typename T, int L>
__host__ __device__ constexpr int square_run()
{
    constexpr int n = (1 << L) + 1, by_bytes = 64 / (int)sizeof(T);
    constexpr int by_threads = 256 / n >= 64 ? 64 : 256 / n >= 32 ? 32 : 256 / n >= 16 ? 16 : 256 / n >= 8 ? 8 : 4;
    return by_bytes > by_threads ? by_bytes : by_threads;
}

template <typename T, int OP, int L>
__global__ void __launch_bounds__(square_run<T, L>() * ((1 << L) + 1), 2)
k_pair_square(T *__restrict__ u, int64_t Sa, int64_t bpo)
{
    constexpr int n = (1 << L) + 1, B = square_run<T, L>();
    extern __shared__ __align__(16) unsigned char smr[];
    T *sv = reinterpret_cast<T *>(smr);
    const int tid = threadIdx.x;
    const int jj = tid & (B - 1), q = tid / B;
    const int64_t o = (int64_t)blockIdx.x / bpo;
    const int64_t j0 = ((int64_t)blockIdx.x - o * bpo) * B;
    const bool act = j0 + jj < Sa;
    T *g = u + o * Sa * n * n + j0 + jj;
    T v[n];
    if (act) {
        const T *p = g + Sa * n * q;            // pole of dimension a at i_{a+1} = q
#pragma unroll
        for (int i = 0; i < n; ++i) v[i] = p[Sa * i];
        transform_regs<T, OP, L>(v);
#pragma unroll
        for (int i = 0; i < n; ++i) sv[(q * n + i) * B + jj] = v[i];
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int i = 0; i < n; ++i) v[i] = sv[(i * n + q) * B + jj];
        transform_regs<T, OP, L>(v);
        T *p = g + Sa * q;                      // pole of dimension a+1 at i_a = q
#pragma unroll
        for (int i = 0; i < n; ++i) p[Sa * n * i] = v[i];
    }
}

template <typename T, int OP, int L>
int launch_pair_square(T *u, const Geom &g, int k, cudaStream_t st)
{
    constexpr int n = (1 << L) + 1, B = square_run<T, L>();
    const int64_t Sa = g.S[k];
    const int64_t bpo = (Sa + B - 1) / B;
    const int64_t blocks = g.total / (Sa * n * n) * bpo;
    if (blocks > INT32_MAX) return GBH_ERANGE;
    const size_t smem = (size_t)B * n * n * sizeof(T);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_pair_square<T, OP, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    ProfScope ps("plain_pair_square", st, 2.0 * sizeof(T) * (double)g.total);
    k_pair_square<T, OP, L><<<(unsigned)blocks, B * n, smem, st>>>(u, Sa, bpo);
    ps.done();
    count_launches(1);
    return check_launch();
}

// the square kernel takes the pair (k, k+1) when k >= 1, l_k = l_{k+1} in
// [1, 5] and at least one run of positions lies below k
template <typename T>
bool pair_square_fits(const Geom &g, int k)
{
    if (!(k >= 1 && k + 1 < g.d && g.l[k] == g.l[k + 1] && g.l[k] >= 1 && g.l[k] <= 5)) return false;
    int B = 0;
    switch (g.l[k]) {
        case 1: B = square_run<T, 1>(); break;
        case 2: B = square_run<T, 2>(); break;
        case 3: B = square_run<T, 3>(); break;
        case 4: B = square_run<T, 4>(); break;
        default: B = square_run<T, 5>(); break;
    }
    return g.S[k] >= B;
}

template <typename T, int OP>
int launch_pair_square_any(T *u, const Geom &g, int k, cudaStream_t st)
{
    switch (g.l[k]) {
        case 1: return launch_pair_square<T, OP, 1>(u, g, k, st);
        case 2: return launch_pair_square<T, OP, 2>(u, g, k, st);
        case 3: return launch_pair_square<T, OP, 3>(u, g, k, st);
        case 4: return launch_pair_square<T, OP, 4>(u, g, k, st);
        default: return launch_pair_square<T, OP, 5>(u, g, k, st);
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

// Tile of the pair pass over dimensions (k, k+1): planes per CTA (k = 0) or
// bundle width B (k >= 1); 0 when the pair does not fit (a pole longer than
// the register pole, a tile over the shared-memory budget, or fewer than 8
// positions below k, which would leave the runs of a bundle uncoalesced).
template <typename T>
int pair_tile(const Geom &g, int k)
{
    if (k + 1 >= g.d) return 0;
    const int la = g.l[k], lb = g.l[k + 1];
    if (la < 1 || lb < 1 || la > pair_max_level<T>() || lb > pair_max_level<T>()) return 0;
    const int64_t M = g.n[k] * g.n[k + 1];
    const int64_t cap = kPairBytes / (int64_t)sizeof(T);
    if (k == 0) {
        const int64_t Q = (cap - 16 / (int64_t)sizeof(T)) / M;
        return Q >= 1 ? (int)std::min<int64_t>(Q, 256) : 0;
    }
    int64_t B = 128;
    while (B > 8 && (B * M > cap || B > g.S[k])) B >>= 1;
    return (B * M <= cap && B <= g.S[k]) ? (int)B : 0;
}

template <typename T, int OP>
int launch_pair(T *u, const Geom &g, int k, int Q, cudaStream_t st)
{
    const int la = g.l[k], lb = g.l[k + 1];
    const int64_t M = g.n[k] * g.n[k + 1];
    static bool attr[2] = {false, false};
    const bool rows = k == 0;
    if (!attr[rows]) {
        if (rows) cudaFuncSetAttribute(k_pair<T, OP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairBytes + 16);
        else cudaFuncSetAttribute(k_pair<T, OP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairBytes + 16);
        attr[rows] = true;
    }
    ProfScope ps(rows ? "plain_pair_planes" : "plain_pair_bundles", st, 2.0 * sizeof(T) * (double)g.total);
    if (rows) {
        const int64_t planes = g.total / M;
        const int64_t blocks = (planes + Q - 1) / Q;
        if (blocks > INT32_MAX) return GBH_ERANGE;
        const size_t smem = ((size_t)Q * M + 16 / sizeof(T)) * sizeof(T);
        k_pair<T, OP, true><<<(unsigned)blocks, kPairThreads, smem, st>>>(u, planes, 1, 1, la, lb, Q);
    } else {
        const int64_t Sa = g.S[k];
        const int64_t outer = g.total / (Sa * M);
        const int64_t bpo = (Sa + Q - 1) / Q;
        if (outer * bpo > INT32_MAX) return GBH_ERANGE;
        const size_t smem = (size_t)Q * M * sizeof(T);
        k_pair<T, OP, false><<<(unsigned)(outer * bpo), kPairThreads, smem, st>>>(u, outer * bpo, Sa, bpo, la, lb, Q);
    }
    ps.done();
    count_launches(1);
    return check_launch();
}

// pairs: two consecutive dimensions per pass where they fit a pair tile
// (native arithmetic only).  short_native: with fixed point, dimensions of
// level 1 still compute natively -- a 3-point pole costs two fp64 operations,
// less than its fixed-point scale pass and conversions -- and so can pair.
constexpr int kShortNativeLevel = 1;

template <typename T, int OP>
int plain_all(T *u, const Geom &g, cudaStream_t st, bool fixed, bool pairs, bool short_native)
{
    constexpr bool kFixable = sizeof(T) == 8 && OP != OP_DT;
    auto native = [&](int k) {
        return !(kFixable && fixed) || (short_native && g.l[k] <= kShortNativeLevel);
    };
    for (int k = 0; k < g.d; ++k) {
        if (g.l[k] == 0) continue;
        const bool nat = native(k), nat2 = nat && k + 1 < g.d && native(k + 1);
        if (pairs && nat2 && pair_square_fits<T>(g, k)) {
            if (int e = launch_pair_square_any<T, OP>(u, g, k, st)) return e;
            ++k;
            continue;
        }
        if (pairs && nat2) {
            if (const int Q = pair_tile<T>(g, k)) {
                if (int e = launch_pair<T, OP>(u, g, k, Q, st)) return e;
                ++k;
                continue;
            }
        }
        if (int e = sweep_dim<T, OP>(u, g, k, st, fixed && !nat)) return e;
    }
    return GBH_OK;
}

template <typename T>
int plain_dispatch(T *u, const Geom &g, int op, cudaStream_t st, bool fixed, bool pairs, bool short_native)
{
    switch (op) {
        case OP_H: return plain_all<T, OP_H>(u, g, st, fixed, pairs, short_native);
        case OP_D: return plain_all<T, OP_D>(u, g, st, fixed, pairs, short_native);
        case OP_A: return plain_all<T, OP_A>(u, g, st, fixed, pairs, short_native);
        case OP_DT: return plain_all<T, OP_DT>(u, g, st, false, pairs, short_native);
        default: return GBH_EINVAL;
    }
}

}  // namespace

int plain_transform(void *data, const Geom &g, int dtype, int op, cudaStream_t s, bool fixed64, bool pairs,
                    bool short_native)
{
    if (dtype == GBH_F64)
        return plain_dispatch<double>(static_cast<double *>(data), g, op, s, fixed64, pairs, short_native);
    if (dtype == GBH_F32) return plain_dispatch<float>(static_cast<float *>(data), g, op, s, false, pairs, false);
    return GBH_EDTYPE;
}

}  // namespace gbh
