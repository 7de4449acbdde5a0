// Interior class of a 3-D fp64 grid on the fused path: every point whose three
// coordinates are all off the block lattice of its dyadic tile (the class
// C = {} of the dyadic split described in fused.cu; derived from the
// predecessor structure of Alg. 1, Sec. 3).  Such a point's surplus is the
// hierarchization of its tile closure E0 x E1 x E2 (E_k = 2^{m_k} + 1) with
// the closure faces as block ends, so one closure load, three pole passes and
// one store of the interior finalise it.
//
// Execution.  A persistent kernel: one CTA per SM walks the tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  Closures stream into two shared-
// memory buffers with one bulk asynchronous copy per closure row
// (cp.async.bulk, completion on an mbarrier), so the rows of tile k+1 are in
// flight while tile k is computed.  A bulk copy needs 16-byte aligned
// addresses: row starts alternate between 8 and 0 modulo 16 (rows are
// 2^{l_0}+1 doubles long), so every row copy starts at the even element at or
// below the closure row and takes E0+1 doubles; the row's data sits at offset
// 0 or 1 of its shared-memory slot.  Rows of the two offsets are kept in
// separate halves of the buffer (slot = r/2, or r/2 + half for odd r), so a
// warp's rows share one offset and the row pass reads them with conflict-free
// 16-byte shared loads and a compile-time register layout.
//
// Arithmetic (GB300 issues fp64 at a small fraction of its integer rate).
// Each closure is converted once to int64 block fixed point at the scale of
// its largest binary exponent, chosen so that no later step can overflow:
// hierarchization (doubling form 2u - L - R, exact) gains at most 2 bits per
// pass, 6 in all; the inverse gains at most 2 bits hierarchizing the faces
// (halving form) and at most log2 of the product of the largest hat-basis row
// sums (4.5625 * 3.875 * 3.875 for blocks of levels 5, 4, 4) dehierarchizing
// the closure.  The interior is rounded back to fp64 once.  Inputs are
// truncated at 2^-(g0-1) of the closure's largest magnitude; the inverse
// rounds each halving to nearest.  Closures whose largest exponent lies
// outside [64, 1900] (all values tiny, or near the fp64 limit) take exact but
// slow conversions.  Inputs must be finite.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "gbh_internal.h"

namespace gbh {

// Device status of the single-grid kernels (bounded waits); read and cleared by
// gbh_device_status.
__device__ int g_single_status = 0;

namespace {

constexpr int kI3Threads = 544;                 // 17 warps
constexpr long long kI3SpinLimit = 1ll << 22;   // mbarrier polls before giving up

enum { OP_H = GBH_HIERARCHIZE, OP_D = GBH_DEHIERARCHIZE };

struct Int3Params {
    int64_t S1, S2;            // grid strides of dimensions 1 and 2 (elements)
    int64_t step0, step1, step2;   // offset of one tile step per dimension
    int64_t nb0, nb1;          // tiles along dimensions 0 and 1
    int64_t tiles;             // tiles per grid
    int64_t total;             // tiles * batch
    int64_t N;                 // points per grid
    const double *lo, *hi;     // first element and one past the last of all grids
    int S1i, S2i;              // the strides as 32-bit values (closure spans fit)
};

// ---------------------------------------------------------------------------
// PTX helpers: mbarrier and bulk copies
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase of the given parity; false if it gave up
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity)
{
    for (long long i = 0; i < kI3SpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy ones (a bulk copy into a buffer the CTA has written)
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// fp64 <-> int64 block fixed point
// ---------------------------------------------------------------------------

// v = trunc(x * 2^{c - (emax - 1075)}) for x = (hi:lo) with |x| < 2^{emax-1022}:
// the significand M (53 bits, implicit bit set) placed at bits 62..10, shifted
// right by K - e (K = emax - c + 10, clamped at 63: far smaller values give
// 0; zero has e = 0 and gives 0), then the sign applied.
__device__ __forceinline__ long long fix_fast(unsigned lo, unsigned hi, int K)
{
    const unsigned e = (hi >> 20) & 0x7FFu;
    const int t = min(K - (int)e, 63);
    const unsigned mh = (__funnelshift_l(lo, hi, 10) & 0x3FFFFFFFu) | 0x40000000u;
    const unsigned long long m = ((unsigned long long)mh << 32) | (unsigned long long)(lo << 10);
    const long long r = (long long)(m >> t);
    const long long s = (long long)((int)hi >> 31);
    return (r ^ s) - s;
}

// exact conversion for closures outside the fast exponent range
__device__ __noinline__ long long fix_slow(long long bits, int emax, int c)
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

// v * 2^X rounded once: the int64 -> fp64 conversion rounds to nearest, the
// power of two is an add to the exponent field (Xs = X << 20 on the high
// word); a nonzero v converts to a high word >= 0x3FF00000, zero to 0.
__device__ __forceinline__ double unfix_fast(long long v, int Xs)
{
    const double d = __ll2double_rn(v);
    const int h = __double2hiint(d);
    return __hiloint2double(h == 0 ? 0 : h + Xs, __double2loint(d));
}

__device__ __noinline__ double unfix_slow(long long v, int X)
{
    if (v == 0) return 0.0;
    return ldexp(__ll2double_rn(v), X);
}

// ---------------------------------------------------------------------------
// register poles
// ---------------------------------------------------------------------------

template <int E>
struct Lev { static constexpr int v = (E <= 2) ? 0 : 1 + Lev<(E + 1) / 2>::v; };
template <>
struct Lev<1> { static constexpr int v = 0; };

// hierarchization, doubling form: every interior point becomes 2u - L - R
// (twice its surplus, exact); the ends keep their value
template <int E>
__device__ __forceinline__ void pole_h2(long long *v)
{
    constexpr int L = Lev<E>::v, last = 1 << L;
#pragma unroll
    for (int lev = L; lev >= 1; --lev) {
        const int s = 1 << (L - lev);
#pragma unroll
        for (int i = s; i < last; i += 2 * s) v[i] = (v[i] + v[i]) - v[i - s] - v[i + s];
    }
}

// hierarchization, halving form (scale kept): u - round((L + R) / 2)
template <int E>
__device__ __forceinline__ void pole_h1(long long *v)
{
    constexpr int L = Lev<E>::v, last = 1 << L;
#pragma unroll
    for (int lev = L; lev >= 1; --lev) {
        const int s = 1 << (L - lev);
#pragma unroll
        for (int i = s; i < last; i += 2 * s) v[i] = v[i] - ((v[i - s] + v[i + s] + 1) >> 1);
    }
}

// dehierarchization, coarse to fine: u = alpha + round((L + R) / 2)
template <int E>
__device__ __forceinline__ void pole_d(long long *v)
{
    constexpr int L = Lev<E>::v, last = 1 << L;
#pragma unroll
    for (int lev = 1; lev <= L; ++lev) {
        const int s = 1 << (L - lev);
#pragma unroll
        for (int i = s; i < last; i += 2 * s) v[i] = v[i] + ((v[i - s] + v[i + s] + 1) >> 1);
    }
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------

// shared-memory geometry of one closure buffer
template <int E0, int E1, int E2>
struct I3Geom {
    static constexpr int R = E1 * E2;                 // closure rows
    static constexpr int NEVEN = (R + 1) / 2;         // rows of even index (slots 0..NEVEN-1)
    static constexpr int ROWP = E0 + 1;               // doubles per slot (even: 16-byte rows)
    static constexpr int ELEMS = R * ROWP;
    static constexpr int PAIRS = ELEMS / 2;
    static constexpr int ODD_T0 = (NEVEN + 31) / 32 * 32;   // first thread of the odd rows
    static_assert(E0 % 2 == 1 && E1 % 2 == 1 && E2 % 2 == 1, "closure extents are 2^m + 1");
    static_assert(ODD_T0 + (R - NEVEN) <= kI3Threads, "one thread per row");
    static_assert((E0 - 2) * E2 <= kI3Threads && (E0 - 2) * (E1 - 2) <= kI3Threads, "one thread per pole");
};

// slot of closure row r (r = y + E1 z)
template <int NEVEN>
__device__ __forceinline__ int slot_of(int r) { return (r >> 1) + (r & 1) * NEVEN; }

// Row pass for a row whose data starts at element OFF of its slot: 16-byte
// loads into registers, the conversion (CONV) and the dimension-0 pole
// operation, 16-byte stores back.
template <int E0, int OFF, int MODE>
__device__ __forceinline__ void row_pass(long long *row)
{
    constexpr int NP = (E0 + 1) / 2;
    long long w[2 * NP];
    const longlong2 *p = reinterpret_cast<const longlong2 *>(row);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const longlong2 q = p[k];
        w[2 * k] = q.x;
        w[2 * k + 1] = q.y;
    }
    long long *v = w + OFF;
    if constexpr (MODE == 0) pole_h2<E0>(v);
    else pole_d<E0>(v);
    longlong2 *o = reinterpret_cast<longlong2 *>(row);
#pragma unroll
    for (int k = 0; k < NP; ++k) o[k] = make_longlong2(w[2 * k], w[2 * k + 1]);
}

template <int OP, int E0, int E1, int E2>
__global__ void __launch_bounds__(kI3Threads, 1) k_int3(const __grid_constant__ Int3Params P, double *__restrict__ u)
{
    using G = I3Geom<E0, E1, E2>;
    constexpr int R = G::R, NEVEN = G::NEVEN, ROWP = G::ROWP, ELEMS = G::ELEMS, PAIRS = G::PAIRS;
    constexpr int T = kI3Threads;
    constexpr int B0 = E0 - 1, B1 = E1 - 1, B2 = E2 - 1;
    // fixed-point scale: bits of the largest converted magnitude
    constexpr int g0 = OP == OP_H ? 55 : 54;
    constexpr int c = g0 - 53;

    extern __shared__ __align__(128) unsigned char sm[];
    long long *bufs = reinterpret_cast<long long *>(sm);
    __shared__ __align__(8) unsigned long long full[2];
    __shared__ unsigned s_red[2];
    __shared__ double *s_base[2];     // tile base of each buffer (set by the producer)
    const int tid = threadIdx.x;

    auto tile_base = [&](int64_t t) -> double * {
        const int64_t b = t / P.tiles;
        int64_t r = t - b * P.tiles;
        const int64_t bx = r % P.nb0;
        r /= P.nb0;
        const int64_t by = r % P.nb1, bz = r / P.nb1;
        return u + b * P.N + bx * P.step0 + by * P.step1 + bz * P.step2;
    };
    // producer: thread 0 issues the closure rows of tile t into buffer j
    auto issue = [&](int64_t t, int j) {
        double *base = tile_base(t);
        s_base[j] = base;
        const int par0 = (int)((reinterpret_cast<uintptr_t>(base) >> 3) & 1u);
        long long *buf = bufs + (size_t)j * ELEMS;
        const double *first = base - par0;
        const double *last = base + (int64_t)B1 * P.S1 + (int64_t)B2 * P.S2 - (par0 ^ ((B1 + B2) & 1)) + ROWP;
        if (first >= P.lo && last <= P.hi) {
            mbar_arrive_expect_tx(&full[j], (unsigned)(R * ROWP * 8));
            for (int r = 0; r < R; ++r) {
                const int y = r % E1, z = r / E1;
                const int off = par0 ^ (r & 1);
                const double *src = base + (int64_t)y * P.S1 + (int64_t)z * P.S2 - off;
                bulk_g2s(buf + (size_t)slot_of<NEVEN>(r) * ROWP, src, ROWP * 8, &full[j]);
            }
        } else {
            // a closure at the very start or end of the grids: rows whose
            // 16-byte span leaves the grids are copied element by element
            unsigned bytes = 0;
            for (int r = 0; r < R; ++r) {
                const int y = r % E1, z = r / E1;
                const int off = par0 ^ (r & 1);
                const double *src = base + (int64_t)y * P.S1 + (int64_t)z * P.S2 - off;
                if (src >= P.lo && src + ROWP <= P.hi) bytes += ROWP * 8;
            }
            for (int r = 0; r < R; ++r) {
                const int y = r % E1, z = r / E1;
                const int off = par0 ^ (r & 1);
                const double *row = base + (int64_t)y * P.S1 + (int64_t)z * P.S2;
                long long *dst = buf + (size_t)slot_of<NEVEN>(r) * ROWP;
                if (row - off >= P.lo && row - off + ROWP <= P.hi) continue;
                for (int x = 0; x < E0; ++x) dst[off + x] = __double_as_longlong(row[x]);
            }
            mbar_arrive_expect_tx(&full[j], bytes);
            for (int r = 0; r < R; ++r) {
                const int y = r % E1, z = r / E1;
                const int off = par0 ^ (r & 1);
                const double *src = base + (int64_t)y * P.S1 + (int64_t)z * P.S2 - off;
                if (src >= P.lo && src + ROWP <= P.hi)
                    bulk_g2s(buf + (size_t)slot_of<NEVEN>(r) * ROWP, src, ROWP * 8, &full[j]);
            }
        }
    };

    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        s_red[0] = s_red[1] = 0;
        s_base[0] = s_base[1] = u;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const int64_t t0 = blockIdx.x;
    if (tid == 0) {
        if (t0 < P.total) issue(t0, 0);
        if (t0 + gridDim.x < P.total) issue(t0 + gridDim.x, 1);
    }

    int k = 0;
    for (int64_t t = t0; t < P.total; t += gridDim.x, ++k) {
        const int j = k & 1;
        long long *buf = bufs + (size_t)j * ELEMS;
        if (tid == 0) s_red[j ^ 1] = 0;
        const bool ok = mbar_wait(&full[j], (unsigned)((k >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(&g_single_status, GBH_ETIMEOUT);
            // give the copies in flight one more bounded wait, then leave
            if (!ok) mbar_wait(&full[j], (unsigned)((k >> 1) & 1));
            return;
        }
        double *base = s_base[j];
        const int par0 = (int)((reinterpret_cast<uintptr_t>(base) >> 3) & 1u);
        // the pad element of every slot (the neighbour the 16-byte row copy
        // brought along) takes no part in the scale
        if (tid < R) {
            const int r = tid < NEVEN ? 2 * tid : 2 * (tid - NEVEN) + 1;
            const int off = par0 ^ (r & 1);
            buf[(size_t)tid * ROWP + (off ? 0 : E0)] = 0;
        }
        __syncthreads();
        // largest binary exponent of the closure (high words)
        {
            unsigned m = 0;
            const uint4 *q = reinterpret_cast<const uint4 *>(buf);
            for (int p = tid; p < PAIRS; p += T) {
                const uint4 w = q[p];
                m = max(m, max(w.y & 0x7FFFFFFFu, w.w & 0x7FFFFFFFu));
            }
            m = __reduce_max_sync(0xFFFFFFFFu, m);
            if ((tid & 31) == 0) atomicMax(&s_red[j], m);
        }
        __syncthreads();
        const int emax = (int)(s_red[j] >> 20);
        const bool fast = emax >= 64 && emax <= 1900;
        const int X = emax - 1075 - c - (OP == OP_H ? 3 : 0);
        // conversion to fixed point, in place
        if (fast) {
            const int K = emax - c + 10;
            longlong2 *q = reinterpret_cast<longlong2 *>(buf);
            for (int p = tid; p < PAIRS; p += T) {
                const uint4 w = reinterpret_cast<const uint4 *>(q)[p];
                q[p] = make_longlong2(fix_fast(w.x, w.y, K), fix_fast(w.z, w.w, K));
            }
        } else {
            for (int e = tid; e < ELEMS; e += T) buf[e] = fix_slow(buf[e], emax, c);
        }
        __syncthreads();

        // thread -> row of the row passes: even rows first, odd rows from a
        // warp boundary on (a warp's rows share their offset)
        int rslot = -1, roff = 0;
        if (tid < NEVEN) { rslot = tid; roff = par0; }
        else if (tid >= G::ODD_T0 && tid < G::ODD_T0 + (R - NEVEN)) { rslot = NEVEN + tid - G::ODD_T0; roff = par0 ^ 1; }

        if constexpr (OP == OP_H) {
            // dimension 0 on every row
            if (rslot >= 0) {
                long long *row = buf + (size_t)rslot * ROWP;
                if (roff) row_pass<E0, 1, 0>(row);
                else row_pass<E0, 0, 0>(row);
            }
            __syncthreads();
            // dimension 1 on the poles with x interior (every z)
            if (tid < (E0 - 2) * E2) {
                const int x = 1 + tid % (E0 - 2), z = tid / (E0 - 2);
                const int r0 = E1 * z;
                const int eo = r0 & 1;   // parity of the row of y = 0
                // y even: rows of parity eo; y odd: the other parity
                const int se = (r0 >> 1) + eo * NEVEN, so = ((r0 + 1) >> 1) + (eo ^ 1) * NEVEN;
                long long *pe = buf + (size_t)se * ROWP + (par0 ^ eo) + x;
                long long *po = buf + (size_t)so * ROWP + (par0 ^ eo ^ 1) + x;
                long long v[E1];
#pragma unroll
                for (int y = 0; y < E1; ++y) v[y] = (y & 1) ? po[(y >> 1) * ROWP] : pe[(y >> 1) * ROWP];
                pole_h2<E1>(v);
#pragma unroll
                for (int y = 1; y < B1; ++y) {
                    if (y & 1) po[(y >> 1) * ROWP] = v[y];
                    else pe[(y >> 1) * ROWP] = v[y];
                }
            }
            __syncthreads();
            // dimension 2 on the poles with x, y interior; the interior goes
            // to global memory
            if (tid < (E0 - 2) * (E1 - 2)) {
                const int x = 1 + tid % (E0 - 2), y = 1 + tid / (E0 - 2);
                const int ey = y & 1;    // parity of the row of z = 0
                const int se = (y >> 1) + ey * NEVEN, so = ((y + E1) >> 1) + (ey ^ 1) * NEVEN;
                const long long *pe = buf + (size_t)se * ROWP + (par0 ^ ey) + x;
                const long long *po = buf + (size_t)so * ROWP + (par0 ^ ey ^ 1) + x;
                long long v[E2];
#pragma unroll
                for (int z = 0; z < E2; ++z) v[z] = (z & 1) ? po[(z >> 1) * E1 * ROWP] : pe[(z >> 1) * E1 * ROWP];
                pole_h2<E2>(v);
                double *o = base + x + (int64_t)y * P.S1;
                const int Xs = X << 20;
#pragma unroll
                for (int z = 1; z < B2; ++z)
                    o[(int64_t)z * P.S2i] = fast ? unfix_fast(v[z], Xs) : unfix_slow(v[z], X);
            }
        } else {
            // Inverse.  The closure faces hold final nodal values, its
            // interior surpluses.  Stage A: the x faces are hierarchized along
            // y (every z) and then along z (y interior), the y faces along z
            // (x interior): the ends of every interior pole of the
            // dehierarchization then hold what that dimension expects.
            // Stage B: dimensions 0, 1, 2 dehierarchized over interior poles.
            if (tid < 2 * E2) {
                const int f = tid & 1, z = tid >> 1, x = f * B0;
                const int r0 = E1 * z, eo = r0 & 1;
                const int se = (r0 >> 1) + eo * NEVEN, so = ((r0 + 1) >> 1) + (eo ^ 1) * NEVEN;
                long long *pe = buf + (size_t)se * ROWP + (par0 ^ eo) + x;
                long long *po = buf + (size_t)so * ROWP + (par0 ^ eo ^ 1) + x;
                long long v[E1];
#pragma unroll
                for (int y = 0; y < E1; ++y) v[y] = (y & 1) ? po[(y >> 1) * ROWP] : pe[(y >> 1) * ROWP];
                pole_h1<E1>(v);
#pragma unroll
                for (int y = 1; y < B1; ++y) {
                    if (y & 1) po[(y >> 1) * ROWP] = v[y];
                    else pe[(y >> 1) * ROWP] = v[y];
                }
            }
            __syncthreads();
            if (tid < 2 * (E1 - 2) + 2 * (E0 - 2)) {
                int x, y;
                if (tid < 2 * (E1 - 2)) { x = (tid & 1) * B0; y = 1 + (tid >> 1); }
                else { const int q = tid - 2 * (E1 - 2); x = 1 + (q >> 1); y = (q & 1) * B1; }
                const int ey = y & 1;
                const int se = (y >> 1) + ey * NEVEN, so = ((y + E1) >> 1) + (ey ^ 1) * NEVEN;
                long long *pe = buf + (size_t)se * ROWP + (par0 ^ ey) + x;
                long long *po = buf + (size_t)so * ROWP + (par0 ^ ey ^ 1) + x;
                long long v[E2];
#pragma unroll
                for (int z = 0; z < E2; ++z) v[z] = (z & 1) ? po[(z >> 1) * E1 * ROWP] : pe[(z >> 1) * E1 * ROWP];
                pole_h1<E2>(v);
#pragma unroll
                for (int z = 1; z < B2; ++z) {
                    if (z & 1) po[(z >> 1) * E1 * ROWP] = v[z];
                    else pe[(z >> 1) * E1 * ROWP] = v[z];
                }
            }
            __syncthreads();
            // dimension 0 on the rows with y, z interior
            if (rslot >= 0) {
                const int r = rslot < NEVEN ? 2 * rslot : 2 * (rslot - NEVEN) + 1;
                const int y = r % E1, z = r / E1;
                if (y > 0 && y < B1 && z > 0 && z < B2) {
                    long long *row = buf + (size_t)rslot * ROWP;
                    if (roff) row_pass<E0, 1, 1>(row);
                    else row_pass<E0, 0, 1>(row);
                }
            }
            __syncthreads();
            // dimension 1 on the poles with x, z interior
            if (tid < (E0 - 2) * (E2 - 2)) {
                const int x = 1 + tid % (E0 - 2), z = 1 + tid / (E0 - 2);
                const int r0 = E1 * z, eo = r0 & 1;
                const int se = (r0 >> 1) + eo * NEVEN, so = ((r0 + 1) >> 1) + (eo ^ 1) * NEVEN;
                long long *pe = buf + (size_t)se * ROWP + (par0 ^ eo) + x;
                long long *po = buf + (size_t)so * ROWP + (par0 ^ eo ^ 1) + x;
                long long v[E1];
#pragma unroll
                for (int y = 0; y < E1; ++y) v[y] = (y & 1) ? po[(y >> 1) * ROWP] : pe[(y >> 1) * ROWP];
                pole_d<E1>(v);
#pragma unroll
                for (int y = 1; y < B1; ++y) {
                    if (y & 1) po[(y >> 1) * ROWP] = v[y];
                    else pe[(y >> 1) * ROWP] = v[y];
                }
            }
            __syncthreads();
            // dimension 2 on the poles with x, y interior; the interior goes
            // to global memory
            if (tid < (E0 - 2) * (E1 - 2)) {
                const int x = 1 + tid % (E0 - 2), y = 1 + tid / (E0 - 2);
                const int ey = y & 1;
                const int se = (y >> 1) + ey * NEVEN, so = ((y + E1) >> 1) + (ey ^ 1) * NEVEN;
                const long long *pe = buf + (size_t)se * ROWP + (par0 ^ ey) + x;
                const long long *po = buf + (size_t)so * ROWP + (par0 ^ ey ^ 1) + x;
                long long v[E2];
#pragma unroll
                for (int z = 0; z < E2; ++z) v[z] = (z & 1) ? po[(z >> 1) * E1 * ROWP] : pe[(z >> 1) * E1 * ROWP];
                pole_d<E2>(v);
                double *o = base + x + (int64_t)y * P.S1;
                const int Xs = X << 20;
#pragma unroll
                for (int z = 1; z < B2; ++z)
                    o[(int64_t)z * P.S2i] = fast ? unfix_fast(v[z], Xs) : unfix_slow(v[z], X);
            }
        }
        // every thread's shared-memory writes to this buffer come before the
        // bulk copies that will overwrite it
        fence_proxy_async_smem();
        __syncthreads();
        // the buffer is free: the rows of the tile after next go into it
        if (tid == 0) {
            const int64_t tn = t + 2 * (int64_t)gridDim.x;
            if (tn < P.total) issue(tn, j);
        }
    }
}

// Compile-time closures (E0, E1, E2) of the interior kernel.
#define GBH_I3_SHAPES(X) X(33, 17, 17) X(17, 17, 17)

template <int OP, int E0, int E1, int E2>
int launch_shape(const Int3Params &P, double *u, cudaStream_t st, double alg_bytes)
{
    using G = I3Geom<E0, E1, E2>;
    constexpr size_t smem = 2 * (size_t)G::ELEMS * 8;
    auto kern = k_int3<OP, E0, E1, E2>;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return GBH_ECUDA;
        attr = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kI3Threads, smem);
    if (per_sm < 1) return GBH_EUNSUPPORTED;
    const int64_t grid = std::min<int64_t>(P.total, (int64_t)num_sms() * per_sm);
    ProfScope ps("fused_class0", st, alg_bytes);
    kern<<<(unsigned)grid, kI3Threads, smem, st>>>(P, u);
    ps.done();
    count_launches(1);
    return check_launch();
}

}  // namespace

bool interior3_supported(const Geom &g, const int *m)
{
    if (g.d != 3) return false;
    for (int k = 0; k < 3; ++k)
        if (m[k] < 1 || m[k] > g.l[k]) return false;
    const int E0 = (1 << m[0]) + 1, E1 = (1 << m[1]) + 1, E2 = (1 << m[2]) + 1;
    bool shape = false;
#define GBH_I3_CMP(a, b, cc) shape |= (E0 == a && E1 == b && E2 == cc);
    GBH_I3_SHAPES(GBH_I3_CMP)
#undef GBH_I3_CMP
    if (!shape) return false;
    // closure spans in 32-bit element offsets
    return (double)(E2 - 1) * (double)g.S[2] + (double)(E1 - 1) * (double)g.S[1] + E0 < 2147483647.0;
}

int interior3_transform(double *u, const Geom &g, const int *m, int op, cudaStream_t s)
{
    if (!interior3_supported(g, m)) return 1;
    Int3Params P{};
    P.S1 = g.S[1];
    P.S2 = g.S[2];
    P.S1i = (int)g.S[1];
    P.S2i = (int)g.S[2];
    P.step0 = (int64_t)1 << m[0];
    P.step1 = ((int64_t)1 << m[1]) * g.S[1];
    P.step2 = ((int64_t)1 << m[2]) * g.S[2];
    P.nb0 = (int64_t)1 << (g.l[0] - m[0]);
    P.nb1 = (int64_t)1 << (g.l[1] - m[1]);
    P.tiles = P.nb0 * P.nb1 * ((int64_t)1 << (g.l[2] - m[2]));
    P.total = P.tiles * g.batch;
    P.N = g.N;
    P.lo = u;
    P.hi = u + g.N * g.batch;
    const int E0 = (1 << m[0]) + 1, E1 = (1 << m[1]) + 1, E2 = (1 << m[2]) + 1;
    const double bytes = 16.0 * (double)P.total * (E0 - 2) * (E1 - 2) * (E2 - 2);
#define GBH_I3_CALL(a, b, cc)                                                                      \
    if (E0 == a && E1 == b && E2 == cc)                                                            \
        return op == OP_H ? launch_shape<OP_H, a, b, cc>(P, u, s, bytes) : launch_shape<OP_D, a, b, cc>(P, u, s, bytes);
    GBH_I3_SHAPES(GBH_I3_CALL)
#undef GBH_I3_CALL
    return 1;
}

}  // namespace gbh

extern "C" int gbh_device_status(void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return GBH_ECUDA;
    int st = 0;
    if (cudaMemcpyFromSymbol(&st, gbh::g_single_status, sizeof(int)) != cudaSuccess) return GBH_ECUDA;
    if (st != 0) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(gbh::g_single_status, &zero, sizeof(int)) != cudaSuccess) return GBH_ECUDA;
    }
    return st;
}
