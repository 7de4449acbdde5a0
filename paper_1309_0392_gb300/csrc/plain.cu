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

template <typename T, int OP>
int sweep_dim(T *u, const Geom &g, int k, cudaStream_t st)
{
    const int l = g.l[k];
    const int64_t poles = g.total / g.n[k];
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
    if (poles < kMinPolesForThreadPerPole) return sweep_level<T, OP>(u, g, k, st);
    ProfScope ps("plain_pole_global", st, 2.0 * sizeof(T) * (double)g.total);
    k_pole_global<T, OP><<<grid_for(poles, 256), 256, 0, st>>>(u, g.S[k], poles, l);
    ps.done();
    count_launches(1);
    return check_launch();
}

template <typename T, int OP>
int plain_all(T *u, const Geom &g, cudaStream_t st)
{
    for (int k = 0; k < g.d; ++k) {
        if (g.l[k] == 0) continue;
        if (int e = sweep_dim<T, OP>(u, g, k, st)) return e;
    }
    return GBH_OK;
}

template <typename T>
int plain_dispatch(T *u, const Geom &g, int op, cudaStream_t st)
{
    switch (op) {
        case OP_H: return plain_all<T, OP_H>(u, g, st);
        case OP_D: return plain_all<T, OP_D>(u, g, st);
        case OP_A: return plain_all<T, OP_A>(u, g, st);
        default: return GBH_EINVAL;
    }
}

}  // namespace

int plain_transform(void *data, const Geom &g, int dtype, int op, cudaStream_t s)
{
    if (dtype == GBH_F64) return plain_dispatch<double>(static_cast<double *>(data), g, op, s);
    if (dtype == GBH_F32) return plain_dispatch<float>(static_cast<float *>(data), g, op, s);
    return GBH_EDTYPE;
}

}  // namespace gbh
