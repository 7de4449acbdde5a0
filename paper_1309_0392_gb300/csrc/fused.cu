// Fused path: every dimension of a grid in one shared-memory round trip per
// tile, in place, without scratch memory.
//
// Dyadic split (derived from the predecessor structure of Alg. 1, Sec. 3).
// Pick a tile exponent m_k per dimension and write i_k = a 2^{m_k} + r_k.  A
// point with r_k != 0 has both predecessors inside its dyadic block
// [a 2^{m_k}, (a+1) 2^{m_k}]; a point with r_k = 0 (a "lattice" point) has
// lattice predecessors only.  Give every point the class C = {k : r_k = 0}.
// The surplus of a class-C point depends only on the values of points of
// classes containing C inside its "closure": the block closure in the
// dimensions outside C times the lattice in the dimensions of C.  On that
// closure it is the ordinary hierarchization of a small dense grid (levels
// m_k outside C, l_k - m_k inside C).
//
// In-place schedule.  Hierarchization reads only classes containing C, so the
// classes are processed by increasing |C| (one launch per |C|): when class C
// is written, every reader of its nodal values has finished.  The inverse goes
// the other way (|C| decreasing): class C reads final nodal values on the
// closure faces and surpluses inside.  A lattice dimension whose closure would
// not fit in shared memory becomes a "point" dimension: the closure is taken
// at one lattice position and the lattice transform along that dimension is
// applied by a separate strided pass over the class's points.
//
// Arithmetic.  fp32 grids compute in fp32.  fp64 grids compute in exact int64
// block fixed point by default: GB300 issues fp64 instructions at about 1/64
// of the fp32 rate, so fp64 arithmetic, not HBM, would bound the sweep.  Each
// closure is scaled by its largest binary exponent; hierarchization uses the
// doubling form 2u - L - R (exact, no rounding at all), dehierarchization adds
// halved predecessor sums; the result is rounded to fp64 once.  Inputs are
// truncated to 2^{-(g0-1)} of the closure's largest magnitude, far below the
// fp64 rounding of the serial algorithm.  Inputs must be finite; subnormal
// inputs count as zero.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "gbh_internal.h"

namespace gbh {
namespace {

constexpr int kFD = 6;            // dimensions handled by the fused path
// largest closure extent (poles are held in registers): 65 for 4-byte
// values, 33 for 8-byte values
__host__ __device__ constexpr int max_extent(int value_bytes) { return value_bytes == 8 ? 33 : 65; }
constexpr int kMaxCls = 20;       // classes of one |C| (C(6,3))
constexpr int kThreads = 256;
constexpr int64_t kMinClosures = 256;   // closures of an all-lattice class (see make_class)

enum { OP_H = GBH_HIERARCHIZE, OP_D = GBH_DEHIERARCHIZE };
enum Mode { BLOCK = 0, LATTICE = 1, POINT = 2 };

// One class of one grid shape.
struct ClassDesc {
    int e[kFD];          // closure extent per dimension
    unsigned mag[kFD];   // __umulhi magic of e[k]
    int ss[kFD];         // shared-memory stride
    int mode[kFD];
    int lev[kFD];        // local transform level (0 = no pass)
    int we[kFD];         // write-box extent
    int wlo[kFD];        // write-box start
    unsigned wmag[kFD];  // __umulhi magic of we[k]
    int64_t gstride[kFD];  // global element stride of one closure step
    int64_t gstep[kFD];    // global element offset of one group step
    int64_t ngrp[kFD];     // groups along each dimension
    int64_t groups;
    int64_t grp_base;    // first group of this class within the launch
    int V;               // closure points
    int rows;            // V / e[0]
    int W;               // write-box points
    int wrows;           // W / we[0]
    int g0;              // fixed point: bits of the input scale
    int doublings;       // fixed point: doubling passes (hierarchization)
    int growth_bits;     // fixed point, inverse: bits the block stage may add
};

struct LaunchParams {
    int d;
    int ncls;
    int64_t per_grid;    // groups of one grid (sum over classes)
    int64_t total;       // per_grid * batch
    int64_t N;           // points per grid (batch stride)
    int off_wg;          // byte offsets in dynamic shared memory: write-row
    int off_ws;          //   global bases, write-row shared bases, values
    int off_vals;
    ClassDesc cls[kMaxCls];
};

// n / e for 0 <= n < 2^32 / e as __umulhi(n, ceil(2^32 / e)); e = 1 has no
// 32-bit magic and is marked by 0.
__host__ __device__ inline unsigned magic_of(int e) { return e == 1 ? 0u : (unsigned)(0xFFFFFFFFu / (unsigned)e) + 1u; }
__device__ __forceinline__ int udiv(int n, unsigned mag) { return mag ? (int)__umulhi((unsigned)n, mag) : n; }

// plain loads with the L2 fill limited to 64 bytes (isolated elements)
__device__ __forceinline__ double ld_l2_64(const double *p)
{
    double v;
    asm volatile("ld.global.L2::64B.f64 %0, [%1];\n" : "=d"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ float ld_l2_64(const float *p)
{
    float v;
    asm volatile("ld.global.L2::64B.f32 %0, [%1];\n" : "=f"(v) : "l"(p) : "memory");
    return v;
}

// ---------------------------------------------------------------------------
// fixed point <-> fp64
// ---------------------------------------------------------------------------

// v = sign * M * 2^{c - (emax - e)}, M the 53-bit significand: the input scaled
// so that the largest magnitude of the closure sits just below 2^{g0}
// (c = g0 - 53).  Computed as (M << P) >> rs with P = max(c, 0) and
// rs = emax - e + P - c >= 0; shifts past the significand give 0, so zeros and
// subnormals (e = 0) become 0 whenever emax >= 64 (checked per closure).
__device__ __forceinline__ long long to_fixed(long long bits, int emax, int P, int rbias)
{
    const int e = (int)((unsigned long long)bits >> 52) & 0x7FF;
    const unsigned long long M = (((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << P;
    int rs = emax - e + rbias;
    rs = rs > 63 ? 63 : rs;
    const long long v = (long long)(M >> rs);
    return bits < 0 ? -v : v;
}

// v * 2^X rounded to fp64 once: the integer-to-fp64 conversion rounds, the
// power of two is an exponent-field add.  Valid for every nonzero v when the
// closure's exponent range is moderate (checked per closure).
__device__ __forceinline__ double from_fixed(long long v, long long Xhi)
{
    const long long b = __double_as_longlong(__ll2double_rn(v));
    return __longlong_as_double(v == 0 ? 0ll : b + Xhi);
}

// to_fixed with the pre-shift PC = max(c, 0) known at compile time and
// emaxp = emax + PC - c: no branches, the 64-bit right shift clamps at 63.
template <int PC>
__device__ __forceinline__ long long to_fixed_pc(long long bits, int emaxp)
{
    const int e = (int)((unsigned long long)bits >> 52) & 0x7FF;
    const unsigned long long M = ((((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52))) << PC;
    const int rs = min(emaxp - e, 63);
    const long long v = (long long)(M >> rs);
    return bits < 0 ? -v : v;
}

// Out-of-range closures (all values below 2^-960 or near the fp64 maximum):
// exact but slow conversions.
__device__ __noinline__ long long to_fixed_slow(long long bits, int emax, int c)
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

__device__ __noinline__ double from_fixed_slow(long long v, int X)
{
    if (v == 0) return 0.0;
    return ldexp(__ll2double_rn(v), X);
}

// ---------------------------------------------------------------------------
// 1-D pole operations on a register copy of a shared-memory pole
// ---------------------------------------------------------------------------

enum PoleOp { P_H_DBL, P_H_HALF, P_D_FIX, P_H_NAT, P_D_NAT };

template <int E>
struct LevelOf { static constexpr int v = (E <= 2) ? 0 : 1 + LevelOf<(E + 1) / 2>::v; };
template <>
struct LevelOf<1> { static constexpr int v = 0; };

template <typename V, int E, int PO>
__device__ __forceinline__ void pole_regs(V *v)
{
    constexpr int L = LevelOf<E>::v;
    constexpr int last = 1 << L;
    if constexpr (PO == P_H_DBL || PO == P_H_HALF || PO == P_H_NAT) {
#pragma unroll
        for (int lev = L; lev >= 1; --lev) {
            const int s = 1 << (L - lev);
#pragma unroll
            for (int i = s; i < last; i += 2 * s) {
                if constexpr (PO == P_H_DBL) v[i] = (v[i] + v[i]) - v[i - s] - v[i + s];
                else if constexpr (PO == P_H_HALF) v[i] = v[i] - ((v[i - s] + v[i + s]) >> 1);
                else v[i] = v[i] - V(0.5) * (v[i - s] + v[i + s]);
            }
        }
        if constexpr (PO == P_H_DBL) {
            v[0] = v[0] + v[0];
            v[last] = v[last] + v[last];
        }
    } else {
#pragma unroll
        for (int lev = 1; lev <= L; ++lev) {
            const int s = 1 << (L - lev);
#pragma unroll
            for (int i = s; i < last; i += 2 * s) {
                if constexpr (PO == P_D_FIX) v[i] = v[i] + ((v[i - s] + v[i + s]) >> 1);
                else v[i] = v[i] + V(0.5) * (v[i - s] + v[i + s]);
            }
        }
    }
}

template <typename V, int E, int PO>
__device__ __forceinline__ void pole_smem(V *s, int st)
{
    V v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = s[i * st];
    pole_regs<V, E, PO>(v);
#pragma unroll
    for (int i = 0; i < E; ++i) s[i * st] = v[i];
}

// two poles of the same shape at once (independent loads in flight together)
template <typename V, int E, int PO>
__device__ __forceinline__ void pole_smem2(V *a, V *b, int st)
{
    V va[E], vb[E];
#pragma unroll
    for (int i = 0; i < E; ++i) { va[i] = a[i * st]; vb[i] = b[i * st]; }
    pole_regs<V, E, PO>(va);
    pole_regs<V, E, PO>(vb);
#pragma unroll
    for (int i = 0; i < E; ++i) { a[i * st] = va[i]; b[i * st] = vb[i]; }
}

template <typename V, int PO>
__device__ __forceinline__ void pole_dispatch(V *s, int st, int e)
{
    switch (e) {
        case 3: pole_smem<V, 3, PO>(s, st); break;
        case 5: pole_smem<V, 5, PO>(s, st); break;
        case 9: pole_smem<V, 9, PO>(s, st); break;
        case 17: pole_smem<V, 17, PO>(s, st); break;
        case 33: pole_smem<V, 33, PO>(s, st); break;
        case 65:
            if constexpr (max_extent(sizeof(V)) >= 65) pole_smem<V, 65, PO>(s, st);
            break;
        default: break;
    }
}

// Which poles of a pass: all, those whose other block coordinates are all
// interior, or those with some other block coordinate on the block boundary.
enum PoleSet { ALL = 0, INTERIOR = 1, FACE = 2 };

template <typename V, int E, int PO>
__device__ __forceinline__ unsigned long long pole_smem_or(V *s, int st)
{
    V v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = s[i * st];
    pole_regs<V, E, PO>(v);
    unsigned long long o = 0ull;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        s[i * st] = v[i];
        if constexpr (std::is_same<V, long long>::value) o |= (unsigned long long)(v[i] ^ (v[i] >> 63));
    }
    return o;
}

template <typename V, int PO>
__device__ __forceinline__ unsigned long long pole_dispatch_or(V *s, int st, int e)
{
    switch (e) {
        case 3: return pole_smem_or<V, 3, PO>(s, st);
        case 5: return pole_smem_or<V, 5, PO>(s, st);
        case 9: return pole_smem_or<V, 9, PO>(s, st);
        case 17: return pole_smem_or<V, 17, PO>(s, st);
        case 33: return pole_smem_or<V, 33, PO>(s, st);
        case 65:
            if constexpr (max_extent(sizeof(V)) >= 65) return pole_smem_or<V, 65, PO>(s, st);
            return 0ull;
        default: return 0ull;
    }
}

// Applies pole operation PO along closure dimension k to the poles of `set`;
// returns the OR of the magnitudes written (fixed point; 0 otherwise).
template <typename V, int PO>
__device__ unsigned long long pass_dim(V *vals, const ClassDesc &C, int d, int k, int set)
{
    const int ek = C.e[k];
    const int npoles = C.V / ek;
    unsigned long long orv = 0ull;
    for (int p = threadIdx.x; p < npoles; p += blockDim.x) {
        int rem = p, off = 0;
        bool interior = true;
#pragma unroll
        for (int j = 0; j < kFD; ++j) {
            if (j >= d || j == k) continue;
            const int q = udiv(rem, C.mag[j]);
            const int c = rem - q * C.e[j];
            rem = q;
            off += c * C.ss[j];
            if (C.mode[j] == BLOCK && (c == 0 || c == C.e[j] - 1)) interior = false;
        }
        if (set == INTERIOR && !interior) continue;
        if (set == FACE && interior) continue;
        if (set == ALL) pole_dispatch<V, PO>(vals + off, C.ss[k], ek);
        else orv |= pole_dispatch_or<V, PO>(vals + off, C.ss[k], ek);
    }
    return orv;
}

// ---------------------------------------------------------------------------
// closure kernel
// ---------------------------------------------------------------------------

// ST: storage type; FIX: int64 fixed-point arithmetic (fp64 storage only).
template <typename ST, bool FIX, int OP>
__global__ void __launch_bounds__(kThreads, 2) k_closure(const __grid_constant__ LaunchParams P,
                                                      ST *__restrict__ u)
{
    using V = typename std::conditional<FIX, long long, ST>::type;
    extern __shared__ __align__(16) unsigned char sm[];
    int64_t *rowg = reinterpret_cast<int64_t *>(sm);           // global base of every closure row
    int64_t *s_wg = reinterpret_cast<int64_t *>(sm + P.off_wg); // global base of every write row
    int *s_ws = reinterpret_cast<int *>(sm + P.off_ws);         // shared base of every write row
    V *vals = reinterpret_cast<V *>(sm + P.off_vals);
    __shared__ int s_emax;
    __shared__ unsigned long long s_or;
    const int tid = threadIdx.x, T = blockDim.x;
    const int d = P.d;

    for (int64_t G = blockIdx.x; G < P.total; G += gridDim.x) {
        const int64_t b = G / P.per_grid;
        const int64_t gl = G - b * P.per_grid;
        int c = 0;
        while (c + 1 < P.ncls && gl >= P.cls[c + 1].grp_base) ++c;
        const ClassDesc &C = P.cls[c];
        // group coordinates -> global base of the closure
        int64_t g = gl - C.grp_base;
        int64_t base = b * P.N;
#pragma unroll
        for (int k = 0; k < kFD; ++k) {
            if (k >= d) break;
            const int64_t q = g / C.ngrp[k];
            base += (g - q * C.ngrp[k]) * C.gstep[k];
            g = q;
        }
        // row tables: closure rows (global base) and write rows
        for (int r = tid; r < C.rows; r += T) {
            int rem = r;
            int64_t off = base;
#pragma unroll
            for (int k = 1; k < kFD; ++k) {
                if (k >= d) break;
                const int q = udiv(rem, C.mag[k]);
                off += (int64_t)(rem - q * C.e[k]) * C.gstride[k];
                rem = q;
            }
            rowg[r] = off;
        }
        for (int r = tid; r < C.wrows; r += T) {
            int rem = r, crow = 0, rstride = 1;
#pragma unroll
            for (int k = 1; k < kFD; ++k) {
                if (k >= d) break;
                const int q = udiv(rem, C.wmag[k]);
                crow += (rem - q * C.we[k] + C.wlo[k]) * rstride;
                rstride *= C.e[k];
                rem = q;
            }
            s_ws[r] = crow * C.e[0] + C.wlo[0];
            s_wg[r] = crow;       // closure row; global base filled below
        }
        if (tid == 0) { s_emax = 0; s_or = 0ull; }
        __syncthreads();
        for (int r = tid; r < C.wrows; r += T) s_wg[r] = rowg[s_wg[r]] + (int64_t)C.wlo[0] * C.gstride[0];

        // load the closure
        int emax = 0;
        {
            const int e0 = C.e[0];
            const int64_t gs0 = C.gstride[0];
            constexpr int U = 8;
            for (int e = tid; e < C.V; e += T * U) {
                ST tmp[U];
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const int ee = e + q * T;
                    if (ee < C.V) {
                        const int r = udiv(ee, C.mag[0]);
                        const ST *src = u + rowg[r] + (int64_t)(ee - r * e0) * gs0;
                        tmp[q] = gs0 == 1 ? *src : ld_l2_64(src);
                    }
                }
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const int ee = e + q * T;
                    if (ee < C.V) {
                        if constexpr (FIX) {
                            const long long bits = __double_as_longlong((double)tmp[q]);
                            const int ex = (int)((bits >> 52) & 0x7FF);
                            emax = ex > emax ? ex : emax;
                            vals[ee] = (V)bits;
                        } else {
                            vals[ee] = (V)tmp[q];
                        }
                    }
                }
            }
        }
        int X = 0;
        bool fast = true;
        if constexpr (FIX) {
            emax = __reduce_max_sync(0xFFFFFFFFu, (unsigned)emax);
            if ((tid & 31) == 0) atomicMax(&s_emax, emax);
            __syncthreads();
            emax = s_emax;
            const int cshift = C.g0 - 53;
            X = emax - 1075 - cshift - (OP == OP_H ? C.doublings : 0);
            fast = emax >= 64 && emax <= 1900;
            if (fast) {
                const int P = cshift > 0 ? cshift : 0;
                const int rbias = P - cshift;
                for (int e = tid; e < C.V; e += T) vals[e] = (V)to_fixed((long long)vals[e], emax, P, rbias);
            } else {
                for (int e = tid; e < C.V; e += T) vals[e] = (V)to_fixed_slow((long long)vals[e], emax, cshift);
            }
        }
        __syncthreads();

        // transform
        if constexpr (OP == OP_H) {
            for (int k = 0; k < d; ++k) {
                if (C.lev[k] == 0) continue;
                pass_dim<V, FIX ? P_H_DBL : P_H_NAT>(vals, C, d, k, ALL);
                __syncthreads();
            }
        } else {
            // stage A.  Lattice dimensions: surpluses -> partial nodal values,
            // interior poles only
            unsigned long long orv = 0ull;
            for (int k = 0; k < d; ++k) {
                if (C.lev[k] == 0 || C.mode[k] != LATTICE) continue;
                orv |= pass_dim<V, FIX ? P_D_FIX : P_D_NAT>(vals, C, d, k, INTERIOR);
                __syncthreads();
            }
            // block faces hold final nodal values: hierarchize them in the
            // block dimensions, so the closure holds one consistent vector
            for (int k = 0; k < d; ++k) {
                if (C.lev[k] == 0 || C.mode[k] != BLOCK) continue;
                orv |= pass_dim<V, FIX ? P_H_HALF : P_H_NAT>(vals, C, d, k, FACE);
                __syncthreads();
            }
            if constexpr (FIX) {
                // renormalise to the magnitude stage A reached, leaving room
                // for the growth of the block stage
                orv |= (1ull << C.g0) - 1ull;
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) orv |= __shfl_xor_sync(0xFFFFFFFFu, orv, o);
                if ((tid & 31) == 0) atomicOr(&s_or, orv);
                __syncthreads();
                int shift = (64 - __clzll((long long)s_or)) + C.growth_bits - 62;
                if (shift > 0) {
                    for (int e = tid; e < C.V; e += T) vals[e] = vals[e] >> shift;
                    X += shift;
                    __syncthreads();
                }
            }
            // stage B: the block dehierarchization on the whole closure
            for (int k = 0; k < d; ++k) {
                if (C.lev[k] == 0 || C.mode[k] != BLOCK) continue;
                pass_dim<V, FIX ? P_D_FIX : P_D_NAT>(vals, C, d, k, ALL);
                __syncthreads();
            }
        }

        // write the class's points
        {
            const int we0 = C.we[0];
            const int64_t gs0 = C.gstride[0];
            const long long Xhi = (long long)X << 52;
            for (int e = tid; e < C.W; e += T) {
                const int r = udiv(e, C.wmag[0]);
                const int x = e - r * we0;
                const V v = vals[s_ws[r] + x];
                ST out;
                if constexpr (FIX) out = fast ? (ST)from_fixed((long long)v, Xhi) : (ST)from_fixed_slow((long long)v, X);
                else out = (ST)v;
                u[s_wg[r] + (int64_t)x * gs0] = out;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// interior class of a 3-D grid with a compile-time tile E0 x E1 x E2
// ---------------------------------------------------------------------------
//
// The same computation as k_closure for the class of points interior to their
// tile in every dimension, with the index arithmetic resolved at compile time:
// the first pass converts rows to fixed point while it transforms them, the
// last pass writes the tile's interior straight from registers.  Dehierarchize
// runs in two fixed-point stages: the tile faces (final nodal values) are
// hierarchized, the values are renormalised to the magnitude they actually
// reached, then the block dehierarchization runs on the whole tile.

struct Tile3Params {
    int64_t S1, S2;          // grid strides of dimensions 1 and 2
    int64_t gs0, gs1, gs2;   // global element stride of one closure step
    int64_t step0, step1, step2;  // global offset of one group step
    int64_t nb0, nb1;        // groups along dimensions 0 and 1
    int64_t tiles;           // tiles per grid
    int64_t total;           // tiles * batch
    int64_t N;               // points per grid
    int g0;                  // fixed point: input scale bits
    int growth_bits;         // dehierarchize: bits the block stage may add
    int pairs;               // 16-byte staging: rows contiguous, strides 1 and 2 odd
};

template <typename V>
__device__ __forceinline__ unsigned long long mag_bits_or(V v)
{
    if constexpr (std::is_same<V, long long>::value) return (unsigned long long)(v ^ (v >> 63));
    else return 0ull;
}

__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
// the same with the L2 fill limited to 64 bytes around the element (isolated
// elements of a lattice along dimension 0)
__device__ __forceinline__ void cp_async8_l2_64(void *smem_dst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global.L2::64B [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4_l2_64(void *smem_dst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global.L2::64B [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// compile-time pre-shift of the fast conversion: c = g0 - 53 of the
// interior kernel (hierarchize g0 = 55, dehierarchize g0 = 58)
template <int OP>
struct kT3Pre { static constexpr int v = OP == GBH_HIERARCHIZE ? 2 : 5; };

constexpr int kTile3Threads = 320;

// One CTA per closure (the block scheduler overlaps the loads of new closures
// with the arithmetic of resident ones): the closure streams in with
// cp.async, then three register-pole passes.  fp64 closures whose rows are
// contiguous and whose row strides along dimensions 1 and 2 are odd (every
// grid with 2^l + 1 points per dimension, outside the lattice classes) stage
// in 16-byte copies: consecutive closure rows alternate in the parity of
// their global element offset exactly as they do in a dense shared-memory
// layout of odd pitch E0, so shifting the layout by the parity of the first
// row aligns every row's 16-byte pairs in both memories; each row is one
// 8-byte copy and (E0 - 1) / 2 16-byte copies.  LM marks the lattice dimensions
// of the class (bit k: dimension k is on the block lattice; 0 is the interior
// class): a lattice dimension takes global strides 2^{m_k} S_k, has no group
// index, and its whole extent is written.
template <typename ST, bool FIX, int OP, int E0, int E1, int E2, int LM>
__global__ void __launch_bounds__(kTile3Threads, 2) k_tile3(const __grid_constant__ Tile3Params P, ST *__restrict__ u)
{
    using V = typename std::conditional<FIX, long long, ST>::type;
    static_assert(sizeof(V) == sizeof(ST), "in-place conversion needs equal sizes");
    constexpr bool L0 = LM & 1, L1 = LM & 2, L2 = LM & 4;
    constexpr int T = kTile3Threads;
    constexpr int NV = E0 * E1 * E2, R = E1 * E2, P1 = E0 * E2, P2 = E0 * E1;
    constexpr int B0 = E0 - 1, B1 = E1 - 1, B2 = E2 - 1;
    constexpr int NBLOCK = (L0 ? 0 : 1) + (L1 ? 0 : 1) + (L2 ? 0 : 1);
    extern __shared__ __align__(16) unsigned char sm[];
    V *vals = reinterpret_cast<V *>(sm);     // shifted by one value below (16-byte staging)
    __shared__ int s_emax;
    __shared__ unsigned long long s_or;
    const int tid = threadIdx.x;

    // block coordinate c of extent E is interior (or the dimension is a lattice)
    auto inner0 = [](int c) { return L0 || (c > 0 && c < B0); };
    auto inner1 = [](int c) { return L1 || (c > 0 && c < B1); };
    auto inner2 = [](int c) { return L2 || (c > 0 && c < B2); };

    const int64_t G = blockIdx.x;
    const int64_t b = G / P.tiles;
    int64_t t = G - b * P.tiles;
    const int64_t bx = t % P.nb0;
    t /= P.nb0;
    const int64_t by = t % P.nb1, bz = t / P.nb1;
    ST *__restrict__ ub = u + b * P.N + bx * P.step0 + by * P.step1 + bz * P.step2;
    if (tid == 0) { s_emax = 0; s_or = 0ull; }
    // tile-relative offsets in 32 bits (the host checks that the closure's
    // span fits)
    const int g0s = (int)P.gs0, g1s = (int)P.gs1, g2s = (int)P.gs2;
    constexpr bool V16 = sizeof(ST) == 8 && !L0 && (E0 & 1);
    if (V16 && P.pairs) {
        // row r = y + E1 z starts at global parity o = o00 ^ (r & 1) and at
        // shared parity (E0 r + o00) & 1, the same; copy c of row r is
        // element 0 alone (o = 1) or element E0 - 1 alone (o = 0) for c = 0,
        // else the pair starting at element 2c - 1 (o = 1) or 2c - 2 (o = 0)
        const int o00 = (int)(((unsigned long long)(uintptr_t)ub >> 3) & 1ull);
        vals += o00;
        constexpr int CH = (E0 + 1) / 2, RW = T / CH;
        if (tid < CH * RW) {
            const int c = tid % CH;
            for (int r = tid / CH; r < R; r += RW) {
                const int y = r % E1, z = r / E1;
                const int o = o00 ^ (r & 1);
                const ST *src = ub + (y * g1s + z * g2s);
                V *dst = vals + r * E0;
                if (c == 0) {
                    const int x = o ? 0 : E0 - 1;
                    cp_async8(dst + x, src + x);
                } else {
                    const int x = 2 * c - 2 + o;
                    cp_async16(dst + x, src + x);
                }
            }
        }
    } else {
    for (int e = tid; e < NV; e += T) {
        const int x = e % E0, r = e / E0;
        const ST *src = ub + (x * g0s + (r % E1) * g1s + (r / E1) * g2s);
        if constexpr (L0) {
            if constexpr (sizeof(ST) == 8) cp_async8_l2_64(vals + e, src);
            else cp_async4_l2_64(vals + e, src);
        } else {
            if constexpr (sizeof(ST) == 8) cp_async8(vals + e, src);
            else cp_async4(vals + e, src);
        }
    }
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();

    int X = 0, emax = 0, P_ = 0, rbias = 0, cshift = 0;
    bool fast = true;
    if constexpr (FIX) {
        // largest binary exponent of the closure (high words only)
        const unsigned *hw = reinterpret_cast<const unsigned *>(vals);
        for (int e = tid; e < NV; e += T) {
            const int ex = (int)(hw[2 * e + 1] >> 20) & 0x7FF;
            emax = ex > emax ? ex : emax;
        }
        emax = __reduce_max_sync(0xFFFFFFFFu, (unsigned)emax);
        if ((tid & 31) == 0) atomicMax(&s_emax, emax);
        __syncthreads();
        emax = s_emax;
        cshift = P.g0 - 53;
        P_ = cshift > 0 ? cshift : 0;
        rbias = P_ - cshift;
        X = emax - 1075 - cshift - (OP == OP_H ? 3 : 0);
        fast = emax >= 64 && emax <= 1900;
    }

    if constexpr (OP == OP_D && LM == 0 && FIX) {
        // Interior class, inverse.  The faces of the closure hold nodal
        // values, its interior surpluses.  Dimension 0 swept over the
        // interior rows needs the rows' ends (the x faces) hierarchical in
        // dimensions 1 and 2; dimension 1 over poles with x, z interior needs
        // their ends (the y faces) hierarchical in dimension 2; dimension 2
        // needs its ends (the z faces) nodal, as they are.  Stage A brings the
        // x and y faces there (scale c); stage B converts the interior at the
        // renormalised scale c - shift as it loads it and sweeps dimensions
        // 0, 1, 2 over interior poles only.
        auto cvt = [&](long long bits, int cs, int Pp, int rb) -> long long {
            return fast ? to_fixed(bits, emax, Pp, rb) : to_fixed_slow(bits, emax, cs);
        };
        constexpr int NXF = 2 * E1 * E2, NYF = 2 * (E0 - 2) * E2;
        for (int w = tid; w < NXF + NYF; w += T) {
            int e;
            if (w < NXF) {
                const int f = w / (E1 * E2), r = w - f * (E1 * E2);
                e = f * B0 + r * E0;
            } else {
                const int w2 = w - NXF, t = w2 / (E0 - 2), x = 1 + w2 - t * (E0 - 2);
                const int z = t >> 1, f = t & 1;
                e = x + E0 * (f * B1 + E1 * z);
            }
            vals[e] = (V)cvt((long long)vals[e], cshift, P_, rbias);
        }
        __syncthreads();
        unsigned long long ora = (1ull << P.g0) - 1ull;
        // x faces along y (every z); y faces along z (x interior)
        for (int p = tid; p < 2 * E2 + 2 * (E0 - 2); p += T) {
            if (p < 2 * E2) {
                const int f = p / E2, z = p - f * E2;
                ora |= pole_smem_or<V, E1, P_H_HALF>(vals + f * B0 + E0 * E1 * z, E0);
            } else {
                const int q = p - 2 * E2, f = q & 1, x = 1 + (q >> 1);
                ora |= pole_smem_or<V, E2, P_H_HALF>(vals + x + E0 * f * B1, E0 * E1);
            }
        }
        __syncthreads();
        // x faces along z (y interior)
        for (int p = tid; p < 2 * (E1 - 2); p += T) {
            const int f = p & 1, y = 1 + (p >> 1);
            ora |= pole_smem_or<V, E2, P_H_HALF>(vals + f * B0 + E0 * y, E0 * E1);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) ora |= __shfl_xor_sync(0xFFFFFFFFu, ora, o);
        if ((tid & 31) == 0) atomicOr(&s_or, ora);
        __syncthreads();
        int shift = (64 - __clzll((long long)s_or)) + P.growth_bits - 62;
        shift = shift > 0 ? shift : 0;
        const int cs2 = cshift - shift, P2s = cs2 > 0 ? cs2 : 0, rb2 = P2s - cs2;
        X += shift;
        // stage B, dimension 0: rows with y, z interior
        for (int r = tid; r < (E1 - 2) * (E2 - 2); r += T) {
            const int zz = r / (E1 - 2), y = 1 + r - zz * (E1 - 2), z = 1 + zz;
            V *row = vals + E0 * (y + E1 * z);
            V v[E0];
            v[0] = row[0] >> shift;
            v[B0] = row[B0] >> shift;
#pragma unroll
            for (int i = 1; i < B0; ++i) v[i] = (V)cvt((long long)row[i], cs2, P2s, rb2);
            pole_regs<V, E0, P_D_FIX>(v);
#pragma unroll
            for (int i = 1; i < B0; ++i) row[i] = v[i];
        }
        __syncthreads();
        // dimension 1: poles with x, z interior
        for (int p = tid; p < (E0 - 2) * (E2 - 2); p += T) {
            const int zz = p / (E0 - 2), x = 1 + p - zz * (E0 - 2), z = 1 + zz;
            V *sp = vals + x + E0 * E1 * z;
            V v[E1];
            v[0] = sp[0] >> shift;
            v[B1] = sp[B1 * E0] >> shift;
#pragma unroll
            for (int i = 1; i < B1; ++i) v[i] = sp[i * E0];
            pole_regs<V, E1, P_D_FIX>(v);
#pragma unroll
            for (int i = 1; i < B1; ++i) sp[i * E0] = v[i];
        }
        __syncthreads();
        // dimension 2: poles with x, y interior; the z faces converted here;
        // the interior points go to global memory
        const long long Xhi = (long long)X << 52;
        for (int p = tid; p < (E0 - 2) * (E1 - 2); p += T) {
            const int yy = p / (E0 - 2), x = 1 + p - yy * (E0 - 2), y = 1 + yy;
            V *sp = vals + x + E0 * y;
            V v[E2];
            v[0] = (V)cvt((long long)sp[0], cs2, P2s, rb2);
            v[B2] = (V)cvt((long long)sp[B2 * E0 * E1], cs2, P2s, rb2);
#pragma unroll
            for (int i = 1; i < B2; ++i) v[i] = sp[i * E0 * E1];
            pole_regs<V, E2, P_D_FIX>(v);
            ST *o = ub + x * P.gs0 + y * P.gs1;
#pragma unroll
            for (int i = 1; i < B2; ++i)
                o[i * P.gs2] = fast ? (ST)from_fixed((long long)v[i], Xhi) : (ST)from_fixed_slow((long long)v[i], X);
        }
        return;
    }

    unsigned long long orv = 0ull;
    // stage A of the inverse along one dimension: a lattice dimension
    // dehierarchizes the poles through class points (block coordinates
    // interior), a block dimension hierarchizes the face poles
    // dimension 0: convert every row, then transform
    for (int r = tid; r < R; r += T) {
        const int y = r % E1, z = r / E1;
        V v[E0];
#pragma unroll
        for (int i = 0; i < E0; ++i) {
            V w = vals[r * E0 + i];
            if constexpr (FIX) w = fast ? to_fixed((long long)w, emax, P_, rbias) : to_fixed_slow((long long)w, emax, cshift);
            v[i] = w;
        }
        bool changed = OP == OP_H;
        if constexpr (OP == OP_H) {
            pole_regs<V, E0, FIX ? P_H_DBL : P_H_NAT>(v);
        } else if constexpr (L0) {
            if (inner1(y) && inner2(z)) {
                pole_regs<V, E0, FIX ? P_D_FIX : P_D_NAT>(v);
                changed = true;
            }
        } else if (!(inner1(y) && inner2(z))) {
            pole_regs<V, E0, FIX ? P_H_HALF : P_H_NAT>(v);
            changed = true;
        }
        // magnitudes for the renormalisation: rows left as converted stay
        // below 2^g0, which the OR covers anyway
        if constexpr (OP == OP_D) {
            if (changed) {
#pragma unroll
                for (int i = 0; i < E0; ++i) orv |= mag_bits_or(v[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < E0; ++i) vals[r * E0 + i] = v[i];
    }
    __syncthreads();
    // dimension 1 (hierarchize, interior class: the x faces are not needed
    // any more, so only poles with x interior, numbered compactly)
    constexpr int XS = (OP == OP_H && LM == 0) ? 1 : 0, XE = E0 - 2 * XS;
    for (int p = tid; p < XE * E2; p += T) {
        const int x = XS + p % XE, z = p / XE;
        V *sp = vals + x + z * E0 * E1;
        if constexpr (OP == OP_H) {
            pole_smem<V, E1, FIX ? P_H_DBL : P_H_NAT>(sp, E0);
        } else if constexpr (L1) {
            if (inner0(x) && inner2(z)) orv |= pole_smem_or<V, E1, FIX ? P_D_FIX : P_D_NAT>(sp, E0);
        } else if (!(inner0(x) && inner2(z))) {
            orv |= pole_smem_or<V, E1, FIX ? P_H_HALF : P_H_NAT>(sp, E0);
        }
    }
    __syncthreads();
    if constexpr (OP == OP_D) {
        // dimension 2, stage A; renormalise; stage B on the block dimensions
        for (int p = tid; p < P2; p += T) {
            const int x = p % E0, y = p / E0;
            V *sp = vals + x + y * E0;
            if constexpr (L2) {
                if (inner0(x) && inner1(y)) orv |= pole_smem_or<V, E2, FIX ? P_D_FIX : P_D_NAT>(sp, E0 * E1);
            } else if (!(inner0(x) && inner1(y))) {
                orv |= pole_smem_or<V, E2, FIX ? P_H_HALF : P_H_NAT>(sp, E0 * E1);
            }
        }
        int shift = 0;
        if constexpr (FIX) {
            orv |= (1ull << P.g0) - 1ull;
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) orv |= __shfl_xor_sync(0xFFFFFFFFu, orv, o);
            if ((tid & 31) == 0) atomicOr(&s_or, orv);
            __syncthreads();
            shift = (64 - __clzll((long long)s_or)) + P.growth_bits - 62;
            shift = shift > 0 ? shift : 0;
            X += shift;
        } else {
            __syncthreads();
        }
        if constexpr (!L0) {
            for (int r = tid; r < R; r += T) {
                V v[E0];
#pragma unroll
                for (int i = 0; i < E0; ++i) {
                    V w = vals[r * E0 + i];
                    if constexpr (FIX) w = w >> shift;
                    v[i] = w;
                }
                pole_regs<V, E0, FIX ? P_D_FIX : P_D_NAT>(v);
#pragma unroll
                for (int i = 0; i < E0; ++i) vals[r * E0 + i] = v[i];
            }
        } else if constexpr (FIX) {
            for (int e = tid; e < NV; e += T) vals[e] = vals[e] >> shift;
        }
        __syncthreads();
        if constexpr (!L1) {
            for (int p = tid; p < P1; p += T) {
                const int x = p % E0, z = p / E0;
                pole_smem<V, E1, FIX ? P_D_FIX : P_D_NAT>(vals + x + z * E0 * E1, E0);
            }
            __syncthreads();
        }
    }
    // dimension 2 (hierarchize; block stage of the inverse), then the class
    // points go to global memory
    const long long Xhi = (long long)X << 52;
    // only poles whose points are stored, numbered compactly
    constexpr int X0 = L0 ? 0 : 1, NX = L0 ? E0 : E0 - 2, Y0 = L1 ? 0 : 1, NY = L1 ? E1 : E1 - 2;
    for (int p = tid; p < NX * NY; p += T) {
        const int x = X0 + p % NX, y = Y0 + p / NX;
        V *sp = vals + x + y * E0;
        V v[E2];
#pragma unroll
        for (int i = 0; i < E2; ++i) v[i] = sp[i * E0 * E1];
        if constexpr (OP == OP_H) pole_regs<V, E2, FIX ? P_H_DBL : P_H_NAT>(v);
        else if constexpr (!L2) pole_regs<V, E2, FIX ? P_D_FIX : P_D_NAT>(v);
        if (inner0(x) && inner1(y)) {
            ST *o = ub + x * P.gs0 + y * P.gs1;
#pragma unroll
            for (int i = L2 ? 0 : 1; i < (L2 ? E2 : E2 - 1); ++i) {
                ST out;
                if constexpr (FIX) out = fast ? (ST)from_fixed((long long)v[i], Xhi) : (ST)from_fixed_slow((long long)v[i], X);
                else out = (ST)v[i];
                o[i * P.gs2] = out;
            }
        }
    }
    (void)NBLOCK;
}

// ---------------------------------------------------------------------------
// lattice pass: transform along one point dimension of a class, native
// arithmetic, one thread per lattice pole (all other coordinates fixed)
// ---------------------------------------------------------------------------

struct LatticeParams {
    int d;
    int k;                 // pole dimension
    int lev;               // pole level (l_k - m_k)
    int64_t pstride;       // 2^{m_k} S_k
    int kind[kFD];         // 0: block-interior positions, 1: lattice positions
    int64_t cnt[kFD];      // positions per dimension (1 for k)
    int64_t m_pow[kFD];    // 2^{m_j}
    int64_t S[kFD];
    int64_t poles;         // per grid
    int64_t total;         // poles * batch
    int64_t N;
};

template <typename ST, int OP, int LEV>
__device__ __forceinline__ void lattice_pole(ST *pp, int64_t S)
{
    // the pole's 2^LEV + 1 points in registers: every load in flight at once
    constexpr int n = (1 << LEV) + 1, last = 1 << LEV;
    ST v[n];
#pragma unroll
    for (int i = 0; i < n; ++i) v[i] = ld_l2_64(pp + i * S);
    if constexpr (OP == OP_H) {
#pragma unroll
        for (int lev = LEV; lev >= 1; --lev) {
            const int s = 1 << (LEV - lev);
#pragma unroll
            for (int i = s; i < last; i += 2 * s) v[i] = v[i] - ST(0.5) * (v[i - s] + v[i + s]);
        }
    } else {
#pragma unroll
        for (int lev = 1; lev <= LEV; ++lev) {
            const int s = 1 << (LEV - lev);
#pragma unroll
            for (int i = s; i < last; i += 2 * s) v[i] = v[i] + ST(0.5) * (v[i - s] + v[i + s]);
        }
    }
#pragma unroll
    for (int i = 1; i < last; ++i) pp[i * S] = v[i];
}

template <typename ST, int OP>
__global__ void __launch_bounds__(kThreads) k_lattice(const __grid_constant__ LatticeParams L, ST *__restrict__ u)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < L.total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / L.poles;
        int64_t p = t - b * L.poles;
        int64_t off = b * L.N;
        for (int j = 0; j < L.d; ++j) {
            if (j == L.k) continue;
            const int64_t q = p / L.cnt[j];
            const int64_t pos = p - q * L.cnt[j];
            p = q;
            int64_t coord;
            if (L.kind[j] == 0) {
                const int64_t w = L.m_pow[j] - 1;
                const int64_t blk = pos / w;
                coord = blk * L.m_pow[j] + (pos - blk * w) + 1;
            } else {
                coord = pos * L.m_pow[j];
            }
            off += coord * L.S[j];
        }
        ST *pp = u + off;
        const int64_t S = L.pstride;
        switch (L.lev) {
            case 1: lattice_pole<ST, OP, 1>(pp, S); break;
            case 2: lattice_pole<ST, OP, 2>(pp, S); break;
            case 3: lattice_pole<ST, OP, 3>(pp, S); break;
            case 4: lattice_pole<ST, OP, 4>(pp, S); break;
            case 5: lattice_pole<ST, OP, 5>(pp, S); break;
            default: {
                const int64_t last = (int64_t)1 << L.lev;
                if (OP == OP_H) {
                    for (int lev = L.lev; lev >= 1; --lev) {
                        const int64_t s = (int64_t)1 << (L.lev - lev);
                        for (int64_t i = s; i < last; i += 2 * s)
                            pp[i * S] = pp[i * S] - ST(0.5) * (pp[(i - s) * S] + pp[(i + s) * S]);
                    }
                } else {
                    for (int lev = 1; lev <= L.lev; ++lev) {
                        const int64_t s = (int64_t)1 << (L.lev - lev);
                        for (int64_t i = s; i < last; i += 2 * s)
                            pp[i * S] = pp[i * S] + ST(0.5) * (pp[(i - s) * S] + pp[(i + s) * S]);
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host planner
// ---------------------------------------------------------------------------

// Largest row sum of |weights| of the 1-D nodal evaluation of a level-lev pole
// (how much dehierarchization can grow a vector in the max norm).
double dehier_growth(int lev)
{
    const int n = (1 << lev) + 1;
    double best = 0.0;
    for (int i = 0; i < n; ++i) {
        // nodal value at i of unit surpluses of absolute weight: sum of hats
        const double x = (double)i / (double)(n - 1);
        double s = 1.0;   // the two boundary hats sum to one
        for (int j = 1; j <= lev; ++j) {
            const int st = 1 << (lev - j);
            const int a = (i / (2 * st)) * (2 * st) + st;
            if (a >= n - 1) continue;
            const double w = 1.0 - std::fabs((double)(i - a)) / (double)st;
            if (w > 0) s += w;
        }
        (void)x;
        best = std::max(best, s);
    }
    return best;
}

struct ClassPlan {
    unsigned mask;
    ClassDesc desc;
    int point_dims[kFD];
    int npoint;
    size_t smem;
};

struct Plan {
    int d;
    int m[kFD];
    std::vector<std::vector<ClassPlan>> by_size;   // index |C|
};

int popc(unsigned x) { return __builtin_popcount(x); }

size_t al16(size_t x) { return (x + 15) / 16 * 16; }

size_t closure_smem(const ClassDesc &c, int es)
{
    return al16((size_t)c.rows * 8) + al16((size_t)c.wrows * 8) + al16((size_t)c.wrows * 4) + (size_t)c.V * es;
}

// Builds the closure descriptor of class `mask`; returns false if the class
// has no points.  Lattice dimensions are turned into point dimensions (the
// largest first) until the closure fits `cap` bytes and every extent <= 65.
bool make_class(const Geom &g, const int *m, unsigned mask, int es, size_t cap, int op, ClassPlan *out)
{
    const int d = g.d;
    ClassPlan cp{};
    cp.mask = mask;
    ClassDesc &c = cp.desc;
    for (int k = 0; k < d; ++k) {
        const bool inC = (mask >> k) & 1u;
        if (!inC && m[k] == 0) return false;          // no block interior: empty class
        if (inC) {
            c.mode[k] = LATTICE;
            c.e[k] = (1 << (g.l[k] - m[k])) + 1;
            c.lev[k] = g.l[k] - m[k];
            c.gstride[k] = ((int64_t)1 << m[k]) * g.S[k];
            c.gstep[k] = 0;
            c.ngrp[k] = 1;
            c.we[k] = c.e[k];
            c.wlo[k] = 0;
        } else {
            c.mode[k] = BLOCK;
            c.e[k] = (1 << m[k]) + 1;
            c.lev[k] = m[k];
            c.gstride[k] = g.S[k];
            c.gstep[k] = ((int64_t)1 << m[k]) * g.S[k];
            c.ngrp[k] = (int64_t)1 << (g.l[k] - m[k]);
            c.we[k] = c.e[k] - 2;
            c.wlo[k] = 1;
        }
    }
    auto to_point = [&](int k) {
        c.mode[k] = POINT;
        const int ext = (1 << (g.l[k] - m[k])) + 1;
        c.e[k] = 1;
        c.lev[k] = 0;
        c.ngrp[k] = ext;
        c.gstep[k] = ((int64_t)1 << m[k]) * g.S[k];
        c.we[k] = 1;
        c.wlo[k] = 0;
    };
    for (int k = 0; k < d; ++k)
        if (c.mode[k] == LATTICE && c.e[k] > max_extent(es)) to_point(k);
    auto volume = [&]() {
        int64_t v = 1;
        for (int k = 0; k < d; ++k) v *= c.e[k];
        return v;
    };
    auto wvolume = [&]() {
        int64_t v = 1;
        for (int k = 1; k < d; ++k) v *= (c.mode[k] == BLOCK ? c.e[k] - 2 : c.e[k]);
        return v;
    };
    auto closures = [&]() {
        int64_t v = 1;
        for (int k = 0; k < d; ++k) v *= c.ngrp[k];
        return v;
    };
    // a class with every dimension on the lattice has one closure, which would
    // leave all SMs but one idle: its lattice dimensions become point
    // dimensions until it has kMinClosures closures
    bool all_lattice = true;
    for (int k = 0; k < d; ++k) all_lattice &= c.mode[k] != BLOCK;
    for (;;) {
        c.V = (int)std::min<int64_t>(volume(), INT32_MAX);
        c.rows = c.V / c.e[0];
        c.wrows = (int)std::min<int64_t>(wvolume(), INT32_MAX);
        const bool fits = closure_smem(c, es) <= cap;
        if (fits && (!all_lattice || closures() >= kMinClosures)) break;
        int best = -1;
        for (int k = 0; k < d; ++k)
            if (c.mode[k] == LATTICE && (fits ? c.e[k] > 2 : true) && (best < 0 || c.e[k] > c.e[best])) best = k;
        if (best < 0) {
            if (fits) break;
            return false;                               // block closure alone too big
        }
        to_point(best);
    }
    int ss = 1;
    c.W = 1;
    for (int k = 0; k < d; ++k) {
        c.ss[k] = ss;
        ss *= c.e[k];
        c.mag[k] = magic_of(c.e[k]);
        c.wmag[k] = magic_of(c.we[k]);
        c.W *= c.we[k];
    }
    c.wrows = c.W / c.we[0];
    c.groups = 1;
    for (int k = 0; k < d; ++k) c.groups *= c.ngrp[k];
    // fixed-point headroom.  Hierarchization: each pass at most quadruples
    // 2u - L - R.  Inverse, stage A: lattice dehierarchization of the
    // interior (growth prod gD) and face hierarchization (2 per block
    // dimension) touch disjoint points; stage B: block dehierarchization.
    int passes = 0;
    double gA_lat = 1.0, gA_face = 1.0, gB = 1.0;
    for (int k = 0; k < d; ++k) {
        if (c.lev[k] == 0) continue;
        ++passes;
        if (c.mode[k] == BLOCK) { gA_face *= 2.0; gB *= dehier_growth(c.lev[k]); }
        else gA_lat *= dehier_growth(c.lev[k]);
    }
    c.doublings = passes;
    if (op == OP_H) {
        c.g0 = 61 - 2 * passes;
        c.growth_bits = 0;
    } else {
        c.g0 = 61 - (int)std::ceil(std::log2(std::max(gA_lat, gA_face)) + 1e-9);
        c.growth_bits = (int)std::ceil(std::log2(gB) + 1e-9);
    }
    cp.npoint = 0;
    for (int k = 0; k < d; ++k)
        if (c.mode[k] == POINT) cp.point_dims[cp.npoint++] = k;
    cp.smem = closure_smem(c, es);
    *out = cp;
    return true;
}

// Estimated DRAM bytes of one transform with tile exponents m.
double estimate_bytes(const Geom &g, const int *m, int es, int op, size_t cap, bool *ok)
{
    const int d = g.d;
    double bytes = 0.0;
    *ok = true;
    for (unsigned mask = 0; mask < (1u << d); ++mask) {
        ClassPlan cp;
        if (!make_class(g, m, mask, es, mask == 0 ? cap / 2 : cap, op, &cp)) {
            bool empty = false;
            for (int k = 0; k < d; ++k)
                if (!((mask >> k) & 1u) && m[k] == 0) empty = true;
            if (!empty) { *ok = false; return 1e300; }
            continue;
        }
        const ClassDesc &c = cp.desc;
        // dimension 0 strided (lattice or point): one 32-byte sector per element
        const bool strided0 = c.mode[0] != BLOCK && m[0] > 0;
        const double waste0 = strided0 ? std::max(1.0, 32.0 / es) : (c.mode[0] == BLOCK ? (c.e[0] * es + 24.0) / (c.e[0] * es) : 1.0);
        double points = (double)c.groups * c.W;
        bytes += (double)c.groups * c.V * es * waste0 + points * es * waste0;
        for (int i = 0; i < cp.npoint; ++i) {
            const int k = cp.point_dims[i];
            const double w = (k == 0 || strided0) ? std::max(1.0, 32.0 / es) : 1.0;
            bytes += 2.0 * points * es * w;
        }
    }
    return bytes;
}

// Plan cache: one class plan per (d, element size, op, levels), the cost
// model's choice unless the autotuner pinned another one.
std::mutex g_plan_mu;
std::map<std::vector<int>, Plan> g_plans;

std::vector<int> plan_key(const Geom &g, int es, int op)
{
    std::vector<int> key;
    key.push_back(g.d);
    key.push_back(es);
    key.push_back(op);
    for (int k = 0; k < g.d; ++k) key.push_back(g.l[k]);
    return key;
}

bool tile3_shape_ok(int es, int E0, int E1, int E2);

// Tile exponents minimising the estimated DRAM bytes, subject to: every
// dimension of level >= 1 has a block interior (m_k >= 1); every lattice
// extent 2^{l_k - m_k} + 1 and block extent 2^{m_k} + 1 fits a register pole;
// the interior-class closure fits half the shared-memory budget (two CTAs
// per SM).  Returns false when no such m exists (e.g. one very long
// dimension): the plain path then takes the grid.
// Feasible tile exponents ranked by estimated DRAM bytes (at most K):
// every dimension of level >= 1 has a block interior (m_k >= 1); every
// lattice extent 2^{l_k - m_k} + 1 and block extent 2^{m_k} + 1 fits a
// register pole; the interior-class closure fits half the shared-memory
// budget (two CTAs per SM).  For 3-D grids the tiles that have a
// compile-time interior kernel come first.  Empty when no such m exists
// (e.g. one very long dimension): the plain path then takes the grid.
std::vector<std::vector<int>> rank_m(const Geom &g, int es, int op, int K)
{
    const int d = g.d;
    const size_t cap = 200 * 1024;
    const int emax_lev = max_extent(es) == 65 ? 6 : 5;
    int lo[kFD], hi[kFD], m[kFD];
    for (int k = 0; k < d; ++k) {
        if (g.l[k] == 0) { lo[k] = hi[k] = 0; continue; }
        lo[k] = std::max(1, g.l[k] - emax_lev);
        hi[k] = std::min(g.l[k], emax_lev);
        if (lo[k] > hi[k]) return {};
    }
    struct Cand { bool t3; double bytes; std::vector<int> m; };
    std::vector<Cand> cands;
    for (int k = 0; k < d; ++k) m[k] = lo[k];
    for (;;) {
        int64_t vol = 1;
        for (int k = 0; k < d; ++k) vol *= (int64_t)(1 << m[k]) + 1;
        if ((size_t)vol * es <= cap / 2) {
            bool ok;
            const double b = estimate_bytes(g, m, es, op, cap, &ok);
            if (ok) {
                const bool t3 = d == 3 && tile3_shape_ok(es, (1 << m[0]) + 1, (1 << m[1]) + 1, (1 << m[2]) + 1);
                cands.push_back(Cand{t3, b, std::vector<int>(m, m + d)});
            }
        }
        int k = 0;
        while (k < d && ++m[k] > hi[k]) { m[k] = lo[k]; ++k; }
        if (k == d) break;
    }
    std::stable_sort(cands.begin(), cands.end(), [](const Cand &a, const Cand &b) {
        return a.t3 != b.t3 ? a.t3 : a.bytes < b.bytes;
    });
    std::vector<std::vector<int>> out;
    for (const Cand &c : cands) {
        if ((int)out.size() >= K) break;
        out.push_back(c.m);
    }
    return out;
}

// The cost model's choice: the first ranked tile.
bool choose_m(const Geom &g, int es, int op, int *m_out)
{
    const auto r = rank_m(g, es, op, 1);
    if (r.empty()) return false;
    for (int k = 0; k < g.d; ++k) m_out[k] = r[0][k];
    return true;
}

// Class plans for explicit tile exponents m.
bool build_plan_m(const Geom &g, int es, int op, const int *m, Plan *plan)
{
    const int d = g.d;
    const size_t cap = 200 * 1024;
    plan->d = d;
    for (int k = 0; k < d; ++k) plan->m[k] = m[k];
    plan->by_size.assign(d + 1, {});
    for (unsigned mask = 0; mask < (1u << d); ++mask) {
        ClassPlan cp;
        if (!make_class(g, m, mask, es, mask == 0 ? cap / 2 : cap, op, &cp)) {
            bool empty = false;
            for (int k = 0; k < d; ++k)
                if (!((mask >> k) & 1u) && m[k] == 0) empty = true;
            if (!empty) return false;
            continue;
        }
        plan->by_size[popc(mask)].push_back(cp);
    }
    return true;
}

// Plan for requested tile exponents (any nonzero entry), else the cached
// planner choice for this shape.
bool build_plan(const Geom &g, int es, int op, const int *m_req, Plan *plan)
{
    const int d = g.d;
    bool explicit_m = false;
    if (m_req)
        for (int k = 0; k < d; ++k) explicit_m |= m_req[k] != 0;
    if (explicit_m) {
        for (int k = 0; k < d; ++k)
            if (m_req[k] < 0 || m_req[k] > g.l[k] || (1 << m_req[k]) + 1 > max_extent(es)) return false;
        return build_plan_m(g, es, op, m_req, plan);
    }
    const std::vector<int> key = plan_key(g, es, op);
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        auto it = g_plans.find(key);
        if (it != g_plans.end()) { *plan = it->second; return true; }
    }
    int m[kFD];
    if (!choose_m(g, es, op, m)) return false;
    Plan p;
    if (!build_plan_m(g, es, op, m, &p)) return false;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans[key] = p;
    *plan = p;
    return true;
}

template <typename ST, bool FIX, int OP>
int launch_closure(const Plan &pl, const std::vector<ClassPlan> &cls, const Geom &g, ST *u, cudaStream_t st)
{
    if (cls.empty()) return GBH_OK;
    LaunchParams P{};
    P.d = pl.d;
    P.ncls = (int)cls.size();
    P.N = g.N;
    size_t smem_rows = 0, smem_wrows = 0, smem_vals = 0;
    int64_t acc = 0;
    double pts = 0.0;
    for (int i = 0; i < P.ncls; ++i) {
        P.cls[i] = cls[i].desc;
        P.cls[i].grp_base = acc;
        acc += cls[i].desc.groups;
        smem_rows = std::max(smem_rows, (size_t)cls[i].desc.rows);
        smem_wrows = std::max(smem_wrows, (size_t)cls[i].desc.wrows);
        smem_vals = std::max(smem_vals, (size_t)cls[i].desc.V * sizeof(typename std::conditional<FIX, long long, ST>::type));
        pts += (double)cls[i].desc.groups * cls[i].desc.W;
    }
    P.per_grid = acc;
    P.total = acc * g.batch;
    P.off_wg = (int)al16(smem_rows * 8);
    P.off_ws = P.off_wg + (int)al16(smem_wrows * 8);
    P.off_vals = P.off_ws + (int)al16(smem_wrows * 4);
    const size_t smem = P.off_vals + smem_vals;
    static int attr_done[2][2][2] = {};
    int &flag = attr_done[sizeof(ST) == 8][FIX][OP == OP_D];
    if (!flag) {
        cudaFuncSetAttribute(k_closure<ST, FIX, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        flag = 1;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_closure<ST, FIX, OP>, kThreads, smem);
    if (per_sm < 1) return GBH_EUNSUPPORTED;
    const int64_t grid = std::min<int64_t>(P.total, (int64_t)num_sms() * per_sm);
    static const char *names[4] = {"fused_class0", "fused_class1", "fused_class2", "fused_class3+"};
    const int csz = popc(cls[0].mask);
    ProfScope ps(names[std::min(csz, 3)], st, 2.0 * sizeof(ST) * pts * g.batch);
    k_closure<ST, FIX, OP><<<(unsigned)grid, kThreads, smem, st>>>(P, u);
    ps.done();
    count_launches(1);
    return check_launch();
}

// Compile-time closures of the 3-D kernel: (storage, E0, E1, E2, lattice mask).
// The interior class (mask 0) and the three one-dimensional lattice classes of
// the planner's usual 3-D tiles.
#define GBH_T3_F64(X) X(33, 17, 17, 0) X(17, 17, 17, 0) X(33, 17, 9, 0) \
    X(17, 17, 17, 1) X(9, 17, 17, 1) X(33, 33, 17, 2) X(33, 17, 17, 2) X(33, 17, 33, 4) X(33, 17, 17, 4)
#define GBH_T3_F32(X) X(65, 17, 17, 0) X(65, 17, 9, 0) X(33, 17, 17, 0) X(17, 17, 17, 0) X(33, 17, 9, 0) \
    X(9, 17, 17, 1) X(5, 17, 17, 1) X(65, 33, 17, 2) X(65, 17, 17, 2) X(65, 17, 33, 4) X(65, 17, 17, 4)

bool tile3_shape_ok(int es, int E0, int E1, int E2)
{
#define GBH_T3_CMP(a, b, c, m) if (m == 0 && E0 == a && E1 == b && E2 == c) return true;
    if (es == 8) { GBH_T3_F64(GBH_T3_CMP) }
    else { GBH_T3_F32(GBH_T3_CMP) }
#undef GBH_T3_CMP
    return false;
}

template <typename ST, bool FIX, int OP, int E0, int E1, int E2, int LM>
int launch_tile3_shape(const Tile3Params &P, ST *u, cudaStream_t st, double alg_bytes, const char *name)
{
    // one spare value: the 16-byte staging shifts the closure by one value
    constexpr size_t smem = ((size_t)E0 * E1 * E2 + 1) * sizeof(ST);
    auto kern = k_tile3<ST, FIX, OP, E0, E1, E2, LM>;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTile3Threads, smem);
    if (per_sm < 1) return GBH_EUNSUPPORTED;
    if (P.total > INT32_MAX) return 1;
    ProfScope ps(name, st, alg_bytes);
    kern<<<(unsigned)P.total, kTile3Threads, smem, st>>>(P, u);
    ps.done();
    count_launches(1);
    return check_launch();
}

// Launches the compile-time kernel for a 3-D class whose lattice dimensions
// are all held in the closure (no point dimensions); returns 1 if no
// compile-time closure matches (the generic kernel then runs).
template <typename ST, bool FIX, int OP>
int launch_tile3(const Plan &pl, const ClassPlan &cp, const Geom &g, ST *u, cudaStream_t st)
{
    const ClassDesc &c = cp.desc;
    if (pl.d != 3 || cp.npoint != 0) return 1;
    if (cp.mask != 0 && cp.mask != 1 && cp.mask != 2 && cp.mask != 4) return 1;
    for (int k = 0; k < 3; ++k)
        if (c.lev[k] < 1) return 1;
    const int E0 = c.e[0], E1 = c.e[1], E2 = c.e[2], LM = (int)cp.mask;
    if ((size_t)E0 * E1 * E2 * sizeof(ST) > 200 * 1024) return 1;
    // closure-relative offsets are 32-bit in the kernel
    if ((double)(E0 - 1) * c.gstride[0] + (double)(E1 - 1) * c.gstride[1] + (double)(E2 - 1) * c.gstride[2] >= 2147483647.0)
        return 1;
    Tile3Params P{};
    P.S1 = g.S[1];
    P.S2 = g.S[2];
    P.gs0 = c.gstride[0];
    P.gs1 = c.gstride[1];
    P.gs2 = c.gstride[2];
    P.step0 = c.gstep[0];
    P.step1 = c.gstep[1];
    P.step2 = c.gstep[2];
    P.nb0 = c.ngrp[0];
    P.nb1 = c.ngrp[1];
    P.tiles = c.ngrp[0] * c.ngrp[1] * c.ngrp[2];
    P.total = P.tiles * g.batch;
    P.N = g.N;
    P.g0 = c.g0;
    P.growth_bits = c.growth_bits;
    P.pairs = c.gstride[0] == 1 && (c.gstride[1] & 1) && (c.gstride[2] & 1) && (c.e[0] & 1);
    const double bytes = 2.0 * sizeof(ST) * (double)P.total * c.W;
    const char *name = cp.mask == 0 ? "fused_class0" : cp.mask == 1 ? "fused_class1_d0" : cp.mask == 2 ? "fused_class1_d1" : "fused_class1_d2";
#define GBH_T3_CALL(a, b, cc, m) \
    if (LM == m && E0 == a && E1 == b && E2 == cc) return launch_tile3_shape<ST, FIX, OP, a, b, cc, m>(P, u, st, bytes, name);
    if constexpr (sizeof(ST) == 8) {
        GBH_T3_F64(GBH_T3_CALL)
    } else {
        GBH_T3_F32(GBH_T3_CALL)
    }
#undef GBH_T3_CALL
    return 1;
}

template <typename ST, int OP>
int launch_lattice(const Plan &pl, const ClassPlan &cp, int k, const Geom &g, ST *u, cudaStream_t st)
{
    LatticeParams L{};
    L.d = pl.d;
    L.k = k;
    L.lev = g.l[k] - pl.m[k];
    L.pstride = ((int64_t)1 << pl.m[k]) * g.S[k];
    int64_t poles = 1;
    for (int j = 0; j < pl.d; ++j) {
        L.S[j] = g.S[j];
        L.m_pow[j] = (int64_t)1 << pl.m[j];
        if (j == k) { L.cnt[j] = 1; L.kind[j] = 1; continue; }
        if ((cp.mask >> j) & 1u) {
            L.kind[j] = 1;
            L.cnt[j] = ((int64_t)1 << (g.l[j] - pl.m[j])) + 1;
        } else {
            L.kind[j] = 0;
            L.cnt[j] = ((int64_t)1 << (g.l[j] - pl.m[j])) * (L.m_pow[j] - 1);
        }
        poles *= L.cnt[j];
    }
    L.poles = poles;
    L.total = poles * g.batch;
    L.N = g.N;
    const int64_t want = (L.total + kThreads - 1) / kThreads;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * 16));
    ProfScope ps("fused_lattice", st, 2.0 * sizeof(ST) * (double)L.total * ((1 << L.lev) + 1));
    k_lattice<ST, OP><<<(unsigned)grid, kThreads, 0, st>>>(L, u);
    ps.done();
    count_launches(1);
    return check_launch();
}

// Kernel variants of a plan (gbh_options.variant): 0 the interior-class
// kernel of interior3.cu where it takes the tile, 1 the generic tile kernels
// only.
// Side streams of the one-lattice-dimension classes.  Classes of equal size
// are independent: a class-C surplus reads only points of classes that
// contain C (all of them larger, or C itself) and writes only class-C
// points.  The classes of size 1 of a 3-D tile therefore run concurrently:
// the first on the caller's stream, the others on two side streams that
// fork from it and join it again by events (the dimension-0 lattice class,
// latency bound on isolated 8-byte values, then overlaps the other two).
// Created on the first fused call on a device; the enqueue sequence holds a
// mutex so that concurrent host threads cannot interleave their event
// records.
struct SideStreams {
    cudaStream_t s[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
    bool ok = false;
};
std::mutex g_side_mu;
SideStreams g_side[64];

// with g_side_mu held
SideStreams *side_streams()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    SideStreams &ss = g_side[dev];
    if (!ss.ok) {
        bool good = cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; i < 2 && good; ++i)
            good = cudaStreamCreateWithFlags(&ss.s[i], cudaStreamNonBlocking) == cudaSuccess &&
                   cudaEventCreateWithFlags(&ss.join[i], cudaEventDisableTiming) == cudaSuccess;
        if (!good) {
            cudaGetLastError();
            return nullptr;
        }
        ss.ok = true;
    }
    return &ss;
}

template <typename ST, bool FIX, int OP>
int run_plan(const Plan &pl, const Geom &g, ST *u, cudaStream_t st, bool int3)
{
    const int d = pl.d;
    auto closure = [&](int c) -> int {
        if (c > 1) return launch_closure<ST, FIX, OP>(pl, pl.by_size[c], g, u, st);
        // classes with a compile-time kernel go one by one, the rest together
        std::vector<ClassPlan> rest;
        // size-1 classes with compile-time kernels: the second and third on
        // the side streams
        std::unique_lock<std::mutex> lk(g_side_mu, std::defer_lock);
        SideStreams *ss = nullptr;
        int nside = 0;
        if (c == 1 && d == 3 && pl.by_size[1].size() > 1) {
            lk.lock();
            ss = side_streams();
            if (ss && cudaEventRecord(ss->fork, st) != cudaSuccess) return check_launch();
        }
        // with side streams the classes are enqueued last to first: the later
        // classes (one-lattice classes of dimensions 1 and 2, large closures)
        // then take their SM slots first and the dimension-0 lattice class
        // (small closures) fills the room beside them
        const int ncls = (int)pl.by_size[c].size();
        for (int idx = 0; idx < ncls; ++idx) {
            const int pos = ss ? ncls - 1 - idx : idx;
            const ClassPlan &cp = pl.by_size[c][pos];
            if (int3 && cp.mask == 0u) {
                const int r = interior3_transform(reinterpret_cast<double *>(u), g, pl.m, OP, st);
                if (r != 1) {
                    if (r != GBH_OK) return r;
                    continue;
                }
            }
            cudaStream_t cs = st;
            if (ss && pos > 0 && nside < 2) {
                cs = ss->s[nside];
                if (cudaStreamWaitEvent(cs, ss->fork, 0) != cudaSuccess) return check_launch();
            }
            const int r = launch_tile3<ST, FIX, OP>(pl, cp, g, u, cs);
            if (r == 1) rest.push_back(cp);
            else if (r != GBH_OK) return r;
            if (cs != st) {
                if (cudaEventRecord(ss->join[nside], cs) != cudaSuccess ||
                    cudaStreamWaitEvent(st, ss->join[nside], 0) != cudaSuccess)
                    return check_launch();
                ++nside;
            }
        }
        if (lk.owns_lock()) lk.unlock();
        return launch_closure<ST, FIX, OP>(pl, rest, g, u, st);
    };
    if (OP == OP_H) {
        for (int c = 0; c <= d; ++c) {
            if (int e = closure(c)) return e;
            for (const ClassPlan &cp : pl.by_size[c])
                for (int i = 0; i < cp.npoint; ++i)
                    if (int e = launch_lattice<ST, OP>(pl, cp, cp.point_dims[i], g, u, st)) return e;
        }
    } else {
        for (int c = d; c >= 0; --c) {
            for (const ClassPlan &cp : pl.by_size[c])
                for (int i = 0; i < cp.npoint; ++i)
                    if (int e = launch_lattice<ST, OP>(pl, cp, cp.point_dims[i], g, u, st)) return e;
            if (int e = closure(c)) return e;
        }
    }
    return GBH_OK;
}

}  // namespace

bool fused_supported(const Geom &g, int dtype, int op)
{
    if (op != GBH_HIERARCHIZE && op != GBH_DEHIERARCHIZE) return false;
    (void)dtype;
    return g.d >= 2 && g.d <= kFD;       // one dimension is one pass already
}

bool fused_preferred(const Geom &g, int dtype, int op)
{
    if (!fused_supported(g, dtype, op)) return false;
    const int es = dtype == GBH_F64 ? 8 : 4;
    Plan pl;
    if (!build_plan(g, es, op, nullptr, &pl)) return false;
    bool ok = false;
    const double fused = estimate_bytes(g, pl.m, es, op, 200 * 1024, &ok);
    int passes = 0;
    for (int k = 0; k < g.d; ++k) passes += g.l[k] > 0;
    const double plain = 2.0 * es * (double)g.N * passes;
    return ok && fused < 0.7 * plain;
}

bool fused_candidates(const Geom &g, int dtype, int op, int K, std::vector<std::vector<int>> *out)
{
    if (!fused_supported(g, dtype, op)) return false;
    *out = rank_m(g, dtype == GBH_F64 ? 8 : 4, op, K);
    return !out->empty();
}

bool fused_pin_tiles(const Geom &g, int dtype, int op, const int *m)
{
    const int es = dtype == GBH_F64 ? 8 : 4;
    Plan p;
    if (!build_plan_m(g, es, op, m, &p)) return false;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans[plan_key(g, es, op)] = p;
    return true;
}

void fused_forget_pins()
{
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans.clear();
}

bool fused_tiles(const Geom &g, int dtype, int op, int *m_out)
{
    if (!fused_supported(g, dtype, op)) return false;
    Plan pl;
    if (!build_plan(g, dtype == GBH_F64 ? 8 : 4, op, nullptr, &pl)) return false;
    for (int k = 0; k < g.d; ++k) m_out[k] = pl.m[k];
    return true;
}

int fused_transform(void *data, const Geom &g, int dtype, int op, const gbh_options *opt, cudaStream_t s)
{
    const int es = dtype == GBH_F64 ? 8 : 4;
    Plan pl;
    const int *m_req = opt ? opt->tile_exp : nullptr;
    if (!build_plan(g, es, op, m_req, &pl)) return GBH_EUNSUPPORTED;
    const int arith = opt ? opt->arith : 0;
    if (dtype == GBH_F64) {
        double *u = static_cast<double *>(data);
        const bool fix = arith != 1;
        const bool int3 = fix && !(opt && opt->variant == 1);
        if (op == OP_H) return fix ? run_plan<double, true, OP_H>(pl, g, u, s, int3) : run_plan<double, false, OP_H>(pl, g, u, s, false);
        return fix ? run_plan<double, true, OP_D>(pl, g, u, s, int3) : run_plan<double, false, OP_D>(pl, g, u, s, false);
    }
    float *u = static_cast<float *>(data);
    if (op == OP_H) return run_plan<float, false, OP_H>(pl, g, u, s, false);
    return run_plan<float, false, OP_D>(pl, g, u, s, false);
}

}  // namespace gbh
