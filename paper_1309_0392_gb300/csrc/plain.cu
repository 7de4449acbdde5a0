// Plain path: one in-place sweep kernel per dimension, native fp32/fp64
// arithmetic, in the operation order of the serial algorithm (so fp64 results
// are bit-identical to a serial run of Alg. 1 in dimension order 0..d-1).
//
//   rows kernel       dimension 0: a CTA stages whole contiguous rows in shared
//                     memory (coalesced), then every point is computed from
//                     the staged copy (Sec. 3: "working in direction of the
//                     data layout vectorization is difficult" -- here the
//                     staging makes it a plain coalesced stream).
//   pole kernel       dimensions k >= 1: one thread per pole; neighbouring
//                     threads own neighbouring poles, which are contiguous in
//                     memory (Sec. 3, Fig. 3 right: work orthogonal to the
//                     poles), so every load and store is coalesced.
//   level kernel      any dimension with few, long poles: one launch per level,
//                     threads over (pole, point of that level).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "gbh_internal.h"

namespace gbh {
namespace {

enum { OP_H = GBH_HIERARCHIZE, OP_D = GBH_DEHIERARCHIZE, OP_A = GBH_ADJOINT };

constexpr int kRowCapElems = 16385;      // longest row staged in shared memory
constexpr int kRowChunk = 4096;          // elements staged per CTA for short rows
constexpr int kRegPoleMaxLevel = 5;      // poles up to 33 points kept in registers
constexpr int64_t kMinPolesForThreadPerPole = 152 * 64;

// ---------------------------------------------------------------------------
// 1-D pole transforms; the loop order is that of Alg. 1 (fine to coarse) for
// hierarchization, coarse to fine for the inverse and the transpose.
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
    } else {
#pragma unroll
        for (int lev = 1; lev <= L; ++lev) {
            const int s = 1 << (L - lev);
#pragma unroll
            for (int i = s; i < last; i += 2 * s) {
                v[i - s] = v[i - s] - T(0.5) * v[i];
                v[i + s] = v[i + s] - T(0.5) * v[i];
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
    } else {
        for (int lev = 1; lev <= l; ++lev) {
            const int64_t s = (int64_t)1 << (l - lev);
            for (int64_t i = s; i < last; i += 2 * s) {
                const T v = p[i * S];
                p[(i - s) * S] = p[(i - s) * S] - T(0.5) * v;
                p[(i + s) * S] = p[(i + s) * S] - T(0.5) * v;
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
            if (OP == OP_A || (i > 0 && i < n - 1)) p[i * S] = v[i];
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
// rows kernel: dimension 0, rows staged in shared memory
// ---------------------------------------------------------------------------

template <typename T, int OP>
__global__ void __launch_bounds__(256) k_rows(T *__restrict__ u, int64_t rows, int l, int rows_per_cta)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);
    const int n = (1 << l) + 1;
    const int64_t row0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t left = rows - row0;
    const int R = left < rows_per_cta ? (int)left : rows_per_cta;
    const int64_t base = row0 * n;
    const int cnt = R * n;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) s[e] = u[base + e];
    __syncthreads();
    if (OP == OP_H) {
        // every surplus from the staged nodal values: one step per point
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            const int i = e % n;
            if (i > 0 && i < n - 1) {
                const int lb = i & (-i);
                u[base + e] = s[e] - T(0.5) * (s[e - lb] + s[e + lb]);
            }
        }
    } else if (OP == OP_D) {
        for (int lev = 1; lev <= l; ++lev) {
            const int st = 1 << (l - lev);
            const int per_row = 1 << (lev - 1);
            const int tot = R * per_row;
            for (int q = threadIdx.x; q < tot; q += blockDim.x) {
                const int r = q >> (lev - 1), k = q & (per_row - 1);
                const int e = r * n + (2 * k + 1) * st;
                s[e] = s[e] + T(0.5) * (s[e - st] + s[e + st]);
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            const int i = e % n;
            if (i > 0 && i < n - 1) u[base + e] = s[e];
        }
    } else {
        // gather form of the transpose; contributions are taken coarse to fine,
        // left before right, as the serial scatter applies them
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            const int i = e % n;
            T y = s[e];
            if (i == 0) {
                for (int t = 1 << (l - 1); t >= 1; t >>= 1) y = y - T(0.5) * s[e + t];
            } else if (i == n - 1) {
                for (int t = 1 << (l - 1); t >= 1; t >>= 1) y = y - T(0.5) * s[e - t];
            } else {
                for (int t = (i & (-i)) >> 1; t >= 1; t >>= 1) {
                    y = y - T(0.5) * s[e - t];
                    y = y - T(0.5) * s[e + t];
                }
            }
            u[base + e] = y;
        }
    }
}

// ---------------------------------------------------------------------------
// level kernel: one launch per level, threads over (pole, point of the level)
// ---------------------------------------------------------------------------

// H / D: the level-lev points i = (2q+1) s of every pole.
// Adjoint: the points p = 2 s q that receive from level-lev children p -/+ s.
template <typename T, int OP>
__global__ void __launch_bounds__(256) k_level(T *__restrict__ u, int64_t S, int64_t n, int64_t outer,
                                               int l, int lev)
{
    const int64_t s = (int64_t)1 << (l - lev);
    const int64_t per = (OP == OP_A) ? (((int64_t)1 << (lev - 1)) + 1) : ((int64_t)1 << (lev - 1));
    const int64_t items = outer * S * per;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < items;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = w % S;
        const int64_t rest = w / S;
        const int64_t q = rest % per, o = rest / per;
        T *p = u + o * S * n + j;
        if (OP == OP_A) {
            const int64_t i = 2 * s * q;
            T y = p[i * S];
            if (q > 0) y = y - T(0.5) * p[(i - s) * S];
            if (q < per - 1) y = y - T(0.5) * p[(i + s) * S];
            p[i * S] = y;
        } else {
            const int64_t i = (2 * q + 1) * s;
            const T sum = p[(i - s) * S] + p[(i + s) * S];
            p[i * S] = (OP == OP_H) ? p[i * S] - T(0.5) * sum : p[i * S] + T(0.5) * sum;
        }
    }
}

// ---------------------------------------------------------------------------
// pole-group kernel: a group of neighbouring poles staged in shared memory
// ---------------------------------------------------------------------------
//
// G poles of one dimension (length n = 2^l + 1, stride S) per CTA, loaded with
// neighbouring poles side by side (coalesced), swept level by level in shared
// memory, written back.  Rows of dimension 0 (S = 1) load row after row.
// FIX (fp64 only): the group is scaled by its largest binary exponent and
// swept in int64 fixed point (hierarchize exact in the doubling form; the
// inverse and the transpose add halved sums); one int64 -> fp64 conversion per
// point instead of two fp64 operations per point.
constexpr int kGroupElems = 8192;

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

__device__ __forceinline__ double g_from_fixed(long long v, int X)
{
    if (v == 0) return 0.0;
    return ldexp(__ll2double_rn(v), X);
}

__device__ __forceinline__ double g_from_fixed_fast(long long v, long long Xhi)
{
    const long long b = __double_as_longlong(__ll2double_rn(v));
    return __longlong_as_double(v == 0 ? 0ll : b + Xhi);
}

template <typename T, int OP, bool FIX, bool ROWS>
__global__ void __launch_bounds__(256) k_pole_group(T *__restrict__ u, int64_t S, int64_t poles, int l, int G,
                                                    int g0)
{
    using V = typename std::conditional<FIX, long long, T>::type;
    extern __shared__ __align__(16) unsigned char smr[];
    V *sv = reinterpret_cast<V *>(smr);
    int64_t *pb = reinterpret_cast<int64_t *>(smr + (size_t)kGroupElems * sizeof(V));
    __shared__ int s_emax;
    const int n = (1 << l) + 1, last = 1 << l;
    const int64_t t0 = (int64_t)blockIdx.x * G;
    const int Gc = (poles - t0) < (int64_t)G ? (int)(poles - t0) : G;
    const int cnt = Gc * n;
    const unsigned magG = Gc == 1 ? 0u : (0xFFFFFFFFu / (unsigned)Gc) + 1u;
    if (!ROWS)
        for (int g = threadIdx.x; g < Gc; g += blockDim.x) {
            const int64_t t = t0 + g, o = t / S;
            pb[g] = o * S * n + (t - o * S);
        }
    if (threadIdx.x == 0) s_emax = 0;
    __syncthreads();
    // element w of the group: rows go row after row, poles side by side
    auto gaddr = [&](int w, int &sidx) -> int64_t {
        if (ROWS) {
            sidx = w;
            return t0 * n + w;
        }
        const int i = magG ? (int)__umulhi((unsigned)w, magG) : w, g = w - i * Gc;
        sidx = g * n + i;
        return pb[g] + (int64_t)i * S;
    };
    int emax = 0;
    for (int w0 = threadIdx.x; w0 < cnt; w0 += blockDim.x * 4) {
        T tmp[4];
        int sid[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int w = w0 + q * blockDim.x;
            if (w < cnt) tmp[q] = u[gaddr(w, sid[q])];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int w = w0 + q * blockDim.x;
            if (w < cnt) {
                if constexpr (FIX) {
                    const long long bits = __double_as_longlong((double)tmp[q]);
                    emax = max(emax, (int)((unsigned long long)bits >> 52) & 0x7FF);
                    sv[sid[q]] = (V)bits;
                } else {
                    sv[sid[q]] = (V)tmp[q];
                }
            }
        }
    }
    int X = 0;
    long long Xhi = 0;
    bool fast = true;
    if constexpr (FIX) {
        emax = __reduce_max_sync(0xFFFFFFFFu, (unsigned)emax);
        if ((threadIdx.x & 31) == 0) atomicMax(&s_emax, emax);
        __syncthreads();
        emax = s_emax;
        const int c = g0 - 53;
        X = emax - 1075 - c - (OP == OP_H ? 1 : 0);
        Xhi = (long long)X << 52;
        fast = emax >= 64 && emax <= 1900;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) sv[e] = g_to_fixed((long long)sv[e], emax, c);
    }
    __syncthreads();
    // level-ordered sweeps, all poles of the group at once
    if (OP == OP_H) {
        for (int lev = l; lev >= 1; --lev) {
            const int s = 1 << (l - lev), per = 1 << (lev - 1);
            for (int q = threadIdx.x; q < Gc * per; q += blockDim.x) {
                const int r = q >> (lev - 1), i = (2 * (q & (per - 1)) + 1) * s;
                V *row = sv + r * n;
                if constexpr (FIX) row[i] = (row[i] + row[i]) - row[i - s] - row[i + s];
                else row[i] = row[i] - V(0.5) * (row[i - s] + row[i + s]);
            }
            __syncthreads();
        }
        if constexpr (FIX) {
            for (int r = threadIdx.x; r < Gc; r += blockDim.x) {
                sv[r * n] += sv[r * n];
                sv[r * n + last] += sv[r * n + last];
            }
            __syncthreads();
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
    } else {
        // transpose: level by level coarse to fine, every parent p = 2 s q
        // collects its two children of this level (left, then right)
        for (int lev = 1; lev <= l; ++lev) {
            const int s = 1 << (l - lev), per = (1 << (lev - 1)) + 1;
            for (int w = threadIdx.x; w < Gc * per; w += blockDim.x) {
                const int r = w / per, q = w - r * per, p = 2 * s * q;
                V *row = sv + r * n;
                if constexpr (FIX) {
                    const V lc = q > 0 ? row[p - s] : V(0), rc = q < per - 1 ? row[p + s] : V(0);
                    row[p] = row[p] - ((lc + rc) >> 1);
                } else {
                    V y = row[p];
                    if (q > 0) y = y - V(0.5) * row[p - s];
                    if (q < per - 1) y = y - V(0.5) * row[p + s];
                    row[p] = y;
                }
            }
            __syncthreads();
        }
    }
    for (int w = threadIdx.x; w < cnt; w += blockDim.x) {
        int sidx;
        const int64_t a = gaddr(w, sidx);
        if constexpr (FIX) u[a] = fast ? (T)g_from_fixed_fast((long long)sv[sidx], Xhi) : (T)g_from_fixed((long long)sv[sidx], X);
        else u[a] = (T)sv[sidx];
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

template <typename T, int OP, bool FIX, bool ROWS>
int launch_group(T *u, const Geom &g, int k, cudaStream_t st)
{
    const int l = g.l[k];
    const int n = (int)g.n[k];
    const int64_t poles = g.total / g.n[k];
    const int G = std::max(1, kGroupElems / n);
    const int64_t blocks = (poles + G - 1) / G;
    if (blocks > INT32_MAX) return GBH_ERANGE;
    using V = typename std::conditional<FIX, long long, T>::type;
    const size_t smem = (size_t)kGroupElems * sizeof(V) + (size_t)G * sizeof(int64_t) + 16;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_pole_group<T, OP, FIX, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kGroupElems * sizeof(long long) + kGroupElems * sizeof(int64_t) + 16));
        attr = true;
    }
    // fixed point headroom: hierarchize doubles once; the inverse grows by at
    // most l + 1 (sum of hat weights); the transpose by at most l + 1
    const int g0 = OP == OP_H ? 59 : 59 - (int)std::ceil(std::log2((double)l + 1.0));
    ProfScope ps(ROWS ? "plain_rows_group" : "plain_pole_group", st, 2.0 * sizeof(T) * (double)g.total);
    k_pole_group<T, OP, FIX, ROWS><<<(unsigned)blocks, 256, smem, st>>>(u, g.S[k], poles, l, G, g0);
    ps.done();
    count_launches(1);
    return check_launch();
}

template <typename T, int OP>
int sweep_dim(T *u, const Geom &g, int k, cudaStream_t st, bool fixed)
{
    const int l = g.l[k];
    const int64_t poles = g.total / g.n[k];
    if constexpr (sizeof(T) == 8) {
        if (fixed && g.n[k] <= kGroupElems) {
            if (k == 0) return launch_group<T, OP, true, true>(u, g, k, st);
            return launch_group<T, OP, true, false>(u, g, k, st);
        }
    }
    if (k == 0) {
        if (g.n[0] > kRowCapElems) return sweep_level<T, OP>(u, g, 0, st);
        const int n = (int)g.n[0];
        const int rpc = std::max(1, kRowChunk / n);
        const int64_t blocks = (poles + rpc - 1) / rpc;
        const size_t smem = (size_t)rpc * n * sizeof(T);
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_rows<T, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kRowCapElems * (int)sizeof(double));
            attr_set = true;
        }
        if (blocks > INT32_MAX) return GBH_ERANGE;
        ProfScope ps("plain_rows", st, 2.0 * sizeof(T) * (double)g.total);
        k_rows<T, OP><<<(unsigned)blocks, 256, smem, st>>>(u, poles, l, rpc);
        ps.done();
        count_launches(1);
        return check_launch();
    }
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
