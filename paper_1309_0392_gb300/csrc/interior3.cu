// Interior class of the fused path for 3-D fp64 grids with tile exponents
// (5, 4, 4), in int64 block fixed point: one CTA per closure of 33 x 17 x 17
// points, two CTAs per SM.
//
// Dyadic split (derived from the predecessor structure of Alg. 1, Sec. 3):
// with tile exponents m = (m0, m1, m2), a point whose coordinate i_k is not a
// multiple of 2^{m_k} has both predecessors along k inside its dyadic block
// [a 2^{m_k}, (a+1) 2^{m_k}].  A point interior to its tile in every
// dimension therefore has its surplus determined by the tile's closure, on
// which it is the ordinary hierarchization of a small dense grid; nothing
// else reads it, so it is written in place as soon as it is known (the
// classes on the block lattices run after this launch for the
// hierarchization, before it for the inverse: fused.cu).
//
// Hierarchization: rows along dimension 0 (every row), then dimension-1
// poles with x interior, then dimension-2 poles with x and y interior,
// written to global memory from registers.  Inverse: the closure's faces hold
// final nodal values of the lattice classes; the x faces are hierarchized
// along dimensions 1 and 2 and the y faces along dimension 2 (what the block
// inverse needs at its pole ends), then the block inverse runs over the rows,
// dimension-1 and dimension-2 poles of the interior.
//
// Loads: every closure row (33 values, odd length and odd strides) as 16
// 16-byte cp.async copies and one 8-byte copy; the shared-memory layout is
// shifted by the parity of the closure's first element, which aligns the
// 16-byte pairs of every row in both memories.
//
// Arithmetic: exact int64 block fixed point per closure (GB300 issues fp64
// instructions at about 1/64 of the fp32 rate).  A closure is scaled by its
// largest binary exponent so that its largest magnitude keeps all 53 bits.
// Hierarchization uses the doubling form 2u - L - R (no rounding at all); the
// inverse adds rounded halves of predecessor sums; every result is rounded to
// fp64 once (half of them converted with integer instructions, half on the
// fp64 pipe, so that neither unit alone holds up the last pass).  Inputs must
// be finite; subnormal inputs count as zero.
#include <cmath>

#include "gbh_internal.h"

namespace gbh {
namespace {

constexpr int kIT = 320;                   // threads of a CTA
constexpr int kE0 = 33, kE1 = 17, kE2 = 17;
constexpr int kXC = kE0 - 1;               // x step of one tile
constexpr int kLX = 5;                     // kXC = 2^kLX
constexpr int kNV = kE0 * kE1 * kE2;       // closure points
constexpr int kNVP = kNV + 1;              // one spare value: parity shift of the layout
constexpr int kRows = kE1 * kE2;           // closure rows along dimension 0
constexpr int kPlane = kE0 * kE1;          // shared-memory stride along dimension 2
constexpr int kPairs = kXC / 2;            // 16-byte copies of a row
static_assert(kXC == (1 << kLX), "tile step");
static_assert(kRows <= kIT && (kPairs + 1) * kE1 <= kIT, "rows and copies fit a CTA");

struct Int3Params {
    int64_t S1, S2;          // grid strides of dimensions 1 and 2
    int64_t N;               // points per grid
    int nb0, nb1;            // tiles along dimensions 0 and 1
    int64_t tiles;           // tiles per grid
};

template <int E>
struct Lev { static constexpr int v = (E <= 2) ? 0 : 1 + Lev<(E + 1) / 2>::v; };
template <>
struct Lev<1> { static constexpr int v = 0; };

__device__ __forceinline__ unsigned long long shr_u64(unsigned long long v, unsigned s)
{
    unsigned long long r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"(s));   // shifts >= 64 give 0
    return r;
}

// fp64 bits -> fixed point v = x * 2^{1075 + C - emax} (truncated toward 0),
// emax the largest biased exponent of the closure (64 <= emax <= 1900): the
// 53-bit significand shifted right by emax - e; zeros and subnormals (e = 0)
// shift out completely.
template <int C>
__device__ __forceinline__ long long fx_in(long long bits, int emax)
{
    const unsigned hi = (unsigned)((unsigned long long)bits >> 32);
    const unsigned rs = (unsigned)(emax - (int)((hi >> 20) & 0x7FFu));
    unsigned long long M = ((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    if (C) M <<= C;
    const long long v = (long long)shr_u64(M, rs);
    const long long s = bits >> 63;
    return (v ^ s) - s;
}

// Exact conversion for closures outside that exponent range (all values below
// 2^-959 or near the fp64 maximum).
__device__ __forceinline__ long long fx_in_slow(long long bits, int emax, int C)
{
    const int e = (int)((unsigned long long)bits >> 52) & 0x7FF;
    if (e == 0) return 0;
    const unsigned long long M = ((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = C - (emax - e);
    long long v;
    if (sh >= 0) v = (long long)(M << sh);
    else v = (-sh >= 63) ? 0 : (long long)(M >> (-sh));
    return bits < 0 ? -v : v;
}

// v * 2^X rounded to fp64 once: the conversion rounds, the power of two is an
// add to the exponent field (valid while the result is a normal number, which
// the exponent range of fast closures guarantees).
__device__ __forceinline__ double fx_out(long long v, int X)
{
    const long long b = __double_as_longlong(__ll2double_rn(v));
    return __longlong_as_double(v == 0 ? 0ll : b + ((long long)X << 52));
}

// The same for any X: results beyond the normal range round once more (to
// a subnormal, zero or infinity).
__device__ __forceinline__ double fx_out_slow(long long v, int X)
{
    if (v == 0) return 0.0;
    const double dv = __ll2double_rn(v);
    const long long b = __double_as_longlong(dv);
    const int t = (int)((b >> 52) & 0x7FF) + X;   // biased exponent of the result
    if (t >= 1 && t <= 2046) return __longlong_as_double(b + ((long long)X << 52));
    if (t > 2046) return dv > 0.0 ? __longlong_as_double(0x7FF0000000000000ll) : __longlong_as_double((long long)0xFFF0000000000000ull);
    if (t < -60) return dv > 0.0 ? 0.0 : -0.0;
    // exact scaling into the normal range, then one rounding multiply
    const double r = __longlong_as_double(b + ((long long)(X + 600) << 52));
    return r * 0x1p-600;
}

// Converts n values of a register array; `fast` is uniform over the CTA.
template <int C, int n>
__device__ __forceinline__ void cvt_in_all(long long *v, int emax, bool fast)
{
    if (fast) {
#pragma unroll
        for (int i = 0; i < n; ++i) v[i] = fx_in<C>(v[i], emax);
    } else {
#pragma unroll
        for (int i = 0; i < n; ++i) v[i] = fx_in_slow(v[i], emax, C);
    }
}

// 1-D pole transforms on a register copy of a pole of E = 2^L + 1 points.
// Hierarchization, doubling form (exact): interior i -> 2 v_i - v_{i-s} - v_{i+s};
// ENDS: the two end points are doubled too (one scale for the whole pole).
template <int E, bool ENDS>
__device__ __forceinline__ void h_dbl(long long *v)
{
    constexpr int L = Lev<E>::v, last = 1 << L;
#pragma unroll
    for (int lev = L; lev >= 1; --lev) {
        const int s = 1 << (L - lev);
#pragma unroll
        for (int i = s; i < last; i += 2 * s) v[i] = (v[i] + v[i]) - v[i - s] - v[i + s];
    }
    if (ENDS) {
        v[0] += v[0];
        v[last] += v[last];
    }
}

// Hierarchization without doubling: v_i - round((v_{i-s} + v_{i+s}) / 2).
template <int E>
__device__ __forceinline__ void h_half(long long *v)
{
    constexpr int L = Lev<E>::v, last = 1 << L;
#pragma unroll
    for (int lev = L; lev >= 1; --lev) {
        const int s = 1 << (L - lev);
#pragma unroll
        for (int i = s; i < last; i += 2 * s) v[i] = v[i] - ((v[i - s] + v[i + s] + 1) >> 1);
    }
}

// Dehierarchization, coarse to fine: v_i + round((v_{i-s} + v_{i+s}) / 2).
template <int E>
__device__ __forceinline__ void d_fix(long long *v)
{
    constexpr int L = Lev<E>::v, last = 1 << L;
#pragma unroll
    for (int lev = 1; lev <= L; ++lev) {
        const int s = 1 << (L - lev);
#pragma unroll
        for (int i = s; i < last; i += 2 * s) v[i] = v[i] + ((v[i - s] + v[i + s] + 1) >> 1);
    }
}

__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Parity (in 8-byte units) of a closure's first element; the shared-memory
// layout of the closure is shifted by it, which aligns every row's 16-byte
// pairs in both memories (rows have odd length, odd strides).
__device__ __forceinline__ int parity_of(const double *p) { return (int)(((uintptr_t)p >> 3) & 1u); }

// The copies of one closure at src0 into vb0 (16-byte aligned, kNVP values):
// row r = y + E1 z has global and shared parity (o00 + r) & 1.  Thread gt
// takes one y and every z (row steps of E1, plane steps of S2): one 16-byte
// pair per row (threads below kPairs E1), or the row's single 8-byte element
// (the next E1 threads); the pair's offset alternates with the parity.
__device__ __forceinline__ void issue_closure(const double *src0, long long *vb0, int S1, int S2, int gt)
{
    const int o00 = parity_of(src0);
    int y0, c;
    bool single;
    if (gt < kPairs * kE1) { y0 = gt / kPairs; c = gt % kPairs; single = false; }
    else if (gt < (kPairs + 1) * kE1) { y0 = gt - kPairs * kE1; c = 0; single = true; }
    else return;
    // element of the row for even and odd row parity
    const int xe = single ? kE0 - 1 : 2 * c, xo = single ? 0 : 2 * c + 1;
    const int p0 = (o00 + y0) & 1;   // parity of row (y0, z = 0)
    long long *dst = vb0 + o00 + y0 * kE0;
    const double *src = src0 + y0 * S1;
#pragma unroll
    for (int z = 0; z < kE2; ++z) {
        const int x = ((p0 + z) & 1) ? xo : xe;
        if (single) cp_async8(dst + z * kPlane + x, src + (int64_t)z * S2 + x);
        else cp_async16(dst + z * kPlane + x, src + (int64_t)z * S2 + x);
    }
}

__device__ __forceinline__ unsigned hi_mag(long long b) { return (unsigned)((unsigned long long)b >> 32) & 0x7FFFFFFFu; }

// int64 -> fp64 with integer instructions (round to nearest even, from the
// IEEE-754 binary64 layout), times 2^X: the same result as fx_out for
// |v| < 2^62 and a normal result, without the fp64 pipe.
__device__ __forceinline__ double fx_out_int(long long v, int X)
{
    const unsigned long long sg = (unsigned long long)(v >> 63);
    unsigned long long a = ((unsigned long long)v ^ sg) - sg;
    const int n = __clzll((long long)a);            // >= 2; 64 for v = 0
    a <<= (unsigned)(n - 1) & 63u;                  // leading one at bit 62
    a += 0x1FFull + ((a >> 10) & 1ull);             // ties to even at bit 10
    const unsigned long long m = a >> 10;           // in [2^52, 2^53]
    const unsigned long long b = ((unsigned long long)(long long)(1085 - n + X) << 52) + m;
    return __longlong_as_double(v == 0 ? 0ll : (long long)(b | (sg & 0x8000000000000000ull)));
}

// Writes the 15 interior values w[1..15] of a dimension-2 pole to o (stride
// S2): every second value converted with integer instructions, the others on
// the fp64 pipe.
__device__ __forceinline__ void out_pole(const long long *w, int X, bool fast, double *o, int S2)
{
    if (fast) {
#pragma unroll
        for (int z = 1; z < kE2 - 1; ++z) o[(int64_t)z * S2] = (z & 1) ? fx_out(w[z], X) : fx_out_int(w[z], X);
    } else {
#pragma unroll
        for (int z = 1; z < kE2 - 1; ++z) o[(int64_t)z * S2] = fx_out_slow(w[z], X);
    }
}

// Largest magnitude over the CTA into *slot (reset beforehand).
__device__ __forceinline__ void block_max(unsigned m, unsigned *slot)
{
    m = __reduce_max_sync(0xFFFFFFFFu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(slot, m);
}

// Row r of a closure into registers and back: rows of one parity use 16-byte
// accesses (par: parity of the row's first element).
__device__ __forceinline__ void load_row(const long long *row, int par, long long *v)
{
    if (par == 0) {
#pragma unroll
        for (int i = 0; i < kPairs; ++i) {
            const longlong2 t = reinterpret_cast<const longlong2 *>(row)[i];
            v[2 * i] = t.x;
            v[2 * i + 1] = t.y;
        }
        v[kXC] = row[kXC];
    } else {
        v[0] = row[0];
#pragma unroll
        for (int i = 0; i < kPairs; ++i) {
            const longlong2 t = reinterpret_cast<const longlong2 *>(row + 1)[i];
            v[2 * i + 1] = t.x;
            v[2 * i + 2] = t.y;
        }
    }
}

__device__ __forceinline__ void store_row(long long *row, int par, const long long *v)
{
    if (par == 0) {
#pragma unroll
        for (int i = 0; i < kPairs; ++i) reinterpret_cast<longlong2 *>(row)[i] = make_longlong2(v[2 * i], v[2 * i + 1]);
        row[kXC] = v[kXC];
    } else {
        row[0] = v[0];
#pragma unroll
        for (int i = 0; i < kPairs; ++i)
            reinterpret_cast<longlong2 *>(row + 1)[i] = make_longlong2(v[2 * i + 1], v[2 * i + 2]);
    }
}

// j-th row with y, z in [1, E - 2] and y + z of parity q: per pair of planes
// (z odd, z even) 15 rows, 8 then 7 (q = 0) or 7 then 8 (q = 1).
__device__ __forceinline__ void inner2_row(int q, int j, int &y, int &z)
{
    const int codd = q ? 7 : 8;   // rows in the odd plane of a pair
    const int P = j / 15, rem = j - 15 * P;
    z = 2 * P + 1 + (rem >= codd);
    const int k = rem >= codd ? rem - codd : rem;
    y = (((q - z) & 1) ? 1 : 2) + 2 * k;
}

template <int OP>
__global__ void __launch_bounds__(kIT, 2) k_int3(const __grid_constant__ Int3Params P, double *__restrict__ u)
{
    constexpr int C = 0;
    extern __shared__ __align__(16) unsigned char sm[];
    long long *buf = reinterpret_cast<long long *>(sm);
    __shared__ unsigned s_hmax;
    const int tid = threadIdx.x;
    const int S1 = (int)P.S1, S2 = (int)P.S2;

    // closure origin
    const unsigned G = blockIdx.x, tl = (unsigned)P.tiles;
    const unsigned b = G / tl, t = G - b * tl;
    const unsigned bx = t % (unsigned)P.nb0, t2 = t / (unsigned)P.nb0;
    const unsigned by = t2 % (unsigned)P.nb1, bz = t2 / (unsigned)P.nb1;
    double *ub = u + (int64_t)b * P.N + (int64_t)bx * kXC + (int64_t)by * (kE1 - 1) * P.S1 + (int64_t)bz * (kE2 - 1) * P.S2;
    const int o00 = parity_of(ub);
    long long *vb = buf + o00;
    if (tid == 0) s_hmax = 0u;
    issue_closure(ub, buf, S1, S2, tid);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();

    // largest exponent: rows, even ones on threads 0..159, odd on 160..319
    const int xr = tid < kIT / 2 ? 2 * tid : 2 * (tid - kIT / 2) + 1;
    const int par = (o00 + xr) & 1;
    {
        unsigned hm = 0u;
        if (xr < kRows) {
            long long v[kE0];
            load_row(vb + xr * kE0, par, v);
#pragma unroll
            for (int i = 0; i < kE0; ++i) hm = max(hm, hi_mag(v[i]));
        }
        block_max(hm, &s_hmax);
    }
    __syncthreads();
    const int emax = (int)(s_hmax >> 20);
    const bool fast = emax >= 64 && emax <= 1900;

    if constexpr (OP == GBH_HIERARCHIZE) {
        // dimension 0: every row
        if (xr < kRows) {
            long long v[kE0];
            load_row(vb + xr * kE0, par, v);
            cvt_in_all<C, kE0>(v, emax, fast);
            h_dbl<kE0, true>(v);
            store_row(vb + xr * kE0, par, v);
        }
        __syncthreads();
        // dimension 1: poles (x interior, every z), two per thread
        {
            constexpr int NP = (kE0 - 2) * kE2, H = (NP + 1) / 2;   // 527, 264
            if (tid < H) {
                const int p1 = tid, p2 = tid + H;
                long long *q1 = vb + 1 + p1 % (kE0 - 2) + kPlane * (p1 / (kE0 - 2));
                long long *q2 = vb + 1 + p2 % (kE0 - 2) + kPlane * (p2 / (kE0 - 2));
                const bool two = p2 < NP;
                long long w[kE1], w2[kE1];
#pragma unroll
                for (int y = 0; y < kE1; ++y) {
                    w[y] = q1[kE0 * y];
                    if (two) w2[y] = q2[kE0 * y];
                }
                h_dbl<kE1, false>(w);
#pragma unroll
                for (int y = 1; y < kE1 - 1; ++y) q1[kE0 * y] = w[y];
                if (two) {
                    h_dbl<kE1, false>(w2);
#pragma unroll
                    for (int y = 1; y < kE1 - 1; ++y) q2[kE0 * y] = w2[y];
                }
            }
        }
        __syncthreads();
        // dimension 2: poles (x, y interior), two per thread; the interior
        // points to global memory
        {
            constexpr int NP = (kE0 - 2) * (kE1 - 2), H = (NP + 1) / 2;   // 465, 233
            const int X = emax - 1075 - C - 3;
            if (tid < H) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int pi = tid + h * H;
                    if (pi < NP) {
                        const int x = 1 + pi % (kE0 - 2), y = 1 + pi / (kE0 - 2);
                        const long long *q = vb + x + kE0 * y;
                        long long w[kE2];
#pragma unroll
                        for (int z = 0; z < kE2; ++z) w[z] = q[kPlane * z];
                        h_dbl<kE2, false>(w);
                        out_pole(w, X, fast, ub + x + (int64_t)y * S1, S2);
                    }
                }
            }
        }
    } else {
        // stage A1: x faces along y (every z), y faces along z (x interior)
        if (tid < 2 * kE2) {
            const int f = tid / kE2, z = tid - f * kE2;
            long long *q = vb + f * kXC + kPlane * z;
            long long w[kE1];
#pragma unroll
            for (int y = 0; y < kE1; ++y) w[y] = q[kE0 * y];
            cvt_in_all<C, kE1>(w, emax, fast);
            h_half<kE1>(w);
#pragma unroll
            for (int y = 1; y < kE1 - 1; ++y) q[kE0 * y] = w[y];
        } else if (tid < 2 * kE2 + 2 * (kE0 - 2)) {
            const int k = tid - 2 * kE2, f = k / (kE0 - 2), x = 1 + k - f * (kE0 - 2);
            long long *q = vb + x + kE0 * f * (kE1 - 1);
            long long w[kE2];
#pragma unroll
            for (int z = 0; z < kE2; ++z) w[z] = q[kPlane * z];
            cvt_in_all<C, kE2>(w, emax, fast);
            h_half<kE2>(w);
#pragma unroll
            for (int z = 1; z < kE2 - 1; ++z) q[kPlane * z] = w[z];
        }
        __syncthreads();
        // stage A2: x faces along z (y interior)
        if (tid < 2 * (kE1 - 2)) {
            const int f = tid / (kE1 - 2), y = 1 + tid - f * (kE1 - 2);
            long long *q = vb + f * kXC + kE0 * y;
            long long w[kE2];
#pragma unroll
            for (int z = 0; z < kE2; ++z) w[z] = q[kPlane * z];
            h_half<kE2>(w);
#pragma unroll
            for (int z = 1; z < kE2 - 1; ++z) q[kPlane * z] = w[z];
        }
        __syncthreads();
        // stage B, dimension 0: rows with y, z interior (ends from stage A,
        // the interior converted here); even y + z on threads 0..112, odd
        // on 160..271
        {
            const int q = tid >= kIT / 2, j = q ? tid - kIT / 2 : tid;
            if (j < (q ? 112 : 113)) {
                int y, z;
                inner2_row(q, j, y, z);
                const int r = y + kE1 * z, rp = (o00 + r) & 1;
                long long v[kE0];
                load_row(vb + r * kE0, rp, v);
                const long long e0 = v[0], e1 = v[kXC];
                cvt_in_all<C, kE0>(v, emax, fast);
                v[0] = e0;
                v[kXC] = e1;
                d_fix<kE0>(v);
                store_row(vb + r * kE0, rp, v);
            }
        }
        __syncthreads();
        // dimension 1: poles (x, z interior), two per thread
        {
            constexpr int NP = (kE0 - 2) * (kE2 - 2), H = (NP + 1) / 2;   // 465, 233
            if (tid < H) {
                const int p1 = tid, p2 = tid + H;
                long long *q1 = vb + 1 + p1 % (kE0 - 2) + kPlane * (1 + p1 / (kE0 - 2));
                long long *q2 = vb + 1 + p2 % (kE0 - 2) + kPlane * (1 + p2 / (kE0 - 2));
                const bool two = p2 < NP;
                long long w[kE1], w2[kE1];
#pragma unroll
                for (int y = 0; y < kE1; ++y) {
                    w[y] = q1[kE0 * y];
                    if (two) w2[y] = q2[kE0 * y];
                }
                d_fix<kE1>(w);
#pragma unroll
                for (int y = 1; y < kE1 - 1; ++y) q1[kE0 * y] = w[y];
                if (two) {
                    d_fix<kE1>(w2);
#pragma unroll
                    for (int y = 1; y < kE1 - 1; ++y) q2[kE0 * y] = w2[y];
                }
            }
        }
        __syncthreads();
        // dimension 2: poles (x, y interior), two per thread; the ends (z
        // faces, final nodal values) converted here; the interior points to
        // global memory
        {
            constexpr int NP = (kE0 - 2) * (kE1 - 2), H = (NP + 1) / 2;
            const int X = emax - 1075 - C;
            if (tid < H) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int pi = tid + h * H;
                    if (pi < NP) {
                        const int x = 1 + pi % (kE0 - 2), y = 1 + pi / (kE0 - 2);
                        const long long *q = vb + x + kE0 * y;
                        long long w[kE2];
#pragma unroll
                        for (int z = 0; z < kE2; ++z) w[z] = q[kPlane * z];
                        cvt_in_all<C, 1>(&w[0], emax, fast);
                        cvt_in_all<C, 1>(&w[kE2 - 1], emax, fast);
                        d_fix<kE2>(w);
                        out_pole(w, X, fast, ub + x + (int64_t)y * S1, S2);
                    }
                }
            }
        }
    }
}

template <int OP>
int launch_int3(const Geom &g, double *u, cudaStream_t st)
{
    constexpr size_t smem = (size_t)kNVP * 8;
    Int3Params P{};
    P.S1 = g.S[1];
    P.S2 = g.S[2];
    P.N = g.N;
    P.nb0 = 1 << (g.l[0] - kLX);
    P.nb1 = 1 << (g.l[1] - 4);
    P.tiles = (int64_t)P.nb0 * P.nb1 << (g.l[2] - 4);
    const int64_t total = P.tiles * g.batch;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_int3<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const double pts = (double)total * (kE0 - 2) * (kE1 - 2) * (kE2 - 2);
    ProfScope ps("fused_class0", st, 16.0 * pts);
    k_int3<OP><<<(unsigned)total, kIT, smem, st>>>(P, u);
    ps.done();
    count_launches(1);
    return check_launch();
}

}  // namespace

bool interior3_applicable(const Geom &g, const int *m)
{
    if (g.d != 3) return false;
    if (m[0] != kLX || m[1] != 4 || m[2] != 4) return false;
    if (g.l[0] < kLX || g.l[1] < 4 || g.l[2] < 4) return false;
    const int64_t total = ((int64_t)1 << (g.l[0] - kLX + g.l[1] - 4 + g.l[2] - 4)) * g.batch;
    if (total >= ((int64_t)1 << 31)) return false;
    if ((double)(kE1 - 1) * g.S[1] + (double)(kE2 - 1) * g.S[2] + kE0 >= 2147483647.0) return false;
    return true;
}

int interior3_transform(double *u, const Geom &g, const int *m, int op, cudaStream_t st)
{
    if (!interior3_applicable(g, m)) return 1;
    if (op == GBH_HIERARCHIZE) return launch_int3<GBH_HIERARCHIZE>(g, u, st);
    if (op == GBH_DEHIERARCHIZE) return launch_int3<GBH_DEHIERARCHIZE>(g, u, st);
    return 1;
}

}  // namespace gbh
