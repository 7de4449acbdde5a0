"""CPU model of the interior-class kernel of 3-D fp64 grids (csrc/interior3.cu):
its row copies, shared-memory slots, pole addressing, fixed-point conversion
and stores, emulated with Python integers and checked before any GPU run:

- every bulk row copy starts 16-byte aligned, stays inside the grids and
  lands 16-byte aligned inside its buffer; rows at the ends of the grids are
  copied element by element;
- the slot and offset arithmetic of the three pole passes addresses the same
  closure element as the producer wrote, inside the buffer;
- the stores cover exactly the interior-class points, once each;
- the fixed-point steps never exceed int64, and the result matches the
  oracle's hierarchization and dehierarchization of those points within the
  fp64 tolerance.

The dyadic split behind the kernel: a point off the block lattice in every
dimension has its surplus determined by its tile closure (Alg. 1, Sec. 3,
predecessors of a point lie inside its dyadic block)."""
import numpy as np
import pytest

import oracle
from paper_1309_0392_gb300 import inputs

INT64_MAX = 2 ** 63 - 1


def lev_of(E):
    return (E - 1).bit_length() - 1


def pole_h2(v):
    L = lev_of(len(v))
    last = 1 << L
    for lev in range(L, 0, -1):
        s = 1 << (L - lev)
        for i in range(s, last, 2 * s):
            v[i] = 2 * v[i] - v[i - s] - v[i + s]


def pole_h1(v):
    L = lev_of(len(v))
    last = 1 << L
    for lev in range(L, 0, -1):
        s = 1 << (L - lev)
        for i in range(s, last, 2 * s):
            v[i] = v[i] - ((v[i - s] + v[i + s] + 1) >> 1)


def pole_d(v):
    L = lev_of(len(v))
    last = 1 << L
    for lev in range(1, L + 1):
        s = 1 << (L - lev)
        for i in range(s, last, 2 * s):
            v[i] = v[i] + ((v[i - s] + v[i + s] + 1) >> 1)


def bits_of(x):
    return int(np.array([x], dtype=np.float64).view(np.uint64)[0])


def fix_fast(x, K):
    b = bits_of(x)
    hi, lo = b >> 32, b & 0xFFFFFFFF
    e = (hi >> 20) & 0x7FF
    t = min(K - e, 63)
    mh = ((((hi << 10) | (lo >> 22)) & 0xFFFFFFFF) & 0x3FFFFFFF) | 0x40000000
    m = (mh << 32) | ((lo << 10) & 0xFFFFFFFF)
    r = m >> t
    return -r if hi >> 31 else r


def unfix(v, X):
    return float(np.ldexp(np.float64(v), X)) if v else 0.0


class Buffer:
    """One closure buffer: slots of ROWP doubles, every access bounds-checked."""

    def __init__(self, E0, E1, E2):
        self.E0, self.E1, self.E2 = E0, E1, E2
        self.R = E1 * E2
        self.NEVEN = (self.R + 1) // 2
        self.ROWP = E0 + 1
        self.data = [None] * (self.R * self.ROWP)

    def slot(self, r):
        return (r >> 1) + (r & 1) * self.NEVEN

    def __getitem__(self, i):
        assert 0 <= i < len(self.data), i
        assert self.data[i] is not None, i
        return self.data[i]

    def __setitem__(self, i, v):
        assert 0 <= i < len(self.data), i
        self.data[i] = v


def run_model(u, levels, m, op, p8, batch=1):
    """Emulates the kernel on `batch` grids stored back to back whose first
    element sits at an address of parity p8 (in 8-byte units)."""
    n = [(1 << l) + 1 for l in levels]
    S1, S2 = n[0], n[0] * n[1]
    N = n[0] * n[1] * n[2]
    E0, E1, E2 = [(1 << mk) + 1 for mk in m]
    B0, B1, B2 = E0 - 1, E1 - 1, E2 - 1
    nb = [1 << (l - mk) for l, mk in zip(levels, m)]
    tiles = nb[0] * nb[1] * nb[2]
    total = tiles * batch
    g0 = 55 if op == "h" else 54
    c = g0 - 53
    out = u.copy()
    written = np.zeros(u.size, dtype=np.int64)
    lo_i, hi_i = 0, N * batch
    for t in range(total):
        b, r_ = divmod(t, tiles)
        bx = r_ % nb[0]
        r_ //= nb[0]
        by, bz = r_ % nb[1], r_ // nb[1]
        base = b * N + bx * B0 + by * B1 * S1 + bz * B2 * S2
        par0 = (p8 + base) & 1
        buf = Buffer(E0, E1, E2)
        # producer
        for r in range(buf.R):
            y, z = r % E1, r // E1
            off = par0 ^ (r & 1)
            row = base + y * S1 + z * S2
            # the row's own parity is the one the kernel derives
            assert (p8 + row) & 1 == off
            dst = buf.slot(r) * buf.ROWP
            assert (dst * 8) % 16 == 0
            src = row - off
            if lo_i <= src and src + buf.ROWP <= hi_i:
                assert ((p8 + src) * 8) % 16 == 0
                for q in range(buf.ROWP):
                    buf[dst + q] = float(u[src + q])
            else:
                for x in range(E0):
                    buf[dst + off + x] = float(u[row + x])
                buf[dst + (0 if off else E0)] = 0.0
        # pads zeroed
        for sl in range(buf.R):
            r = 2 * sl if sl < buf.NEVEN else 2 * (sl - buf.NEVEN) + 1
            off = par0 ^ (r & 1)
            buf[sl * buf.ROWP + (0 if off else E0)] = 0.0
        emax = max(((bits_of(v) >> 52) & 0x7FF) for v in buf.data)
        assert 64 <= emax <= 1900
        K = emax - c + 10
        for i in range(len(buf.data)):
            buf[i] = fix_fast(buf[i], K)
        X = emax - 1075 - c - (3 if op == "h" else 0)

        def pole_addrs_y(x, z):
            r0 = E1 * z
            eo = r0 & 1
            se = (r0 >> 1) + eo * buf.NEVEN
            so = ((r0 + 1) >> 1) + (eo ^ 1) * buf.NEVEN
            pe = se * buf.ROWP + (par0 ^ eo) + x
            po = so * buf.ROWP + (par0 ^ eo ^ 1) + x
            addrs = [(po if y & 1 else pe) + (y >> 1) * buf.ROWP for y in range(E1)]
            # the same element the producer wrote for (x, y, z)
            for y in range(E1):
                r = y + E1 * z
                assert addrs[y] == buf.slot(r) * buf.ROWP + (par0 ^ (r & 1)) + x
            return addrs

        def pole_addrs_z(x, y):
            ey = y & 1
            se = (y >> 1) + ey * buf.NEVEN
            so = ((y + E1) >> 1) + (ey ^ 1) * buf.NEVEN
            pe = se * buf.ROWP + (par0 ^ ey) + x
            po = so * buf.ROWP + (par0 ^ ey ^ 1) + x
            addrs = [(po if z & 1 else pe) + (z >> 1) * E1 * buf.ROWP for z in range(E2)]
            for z in range(E2):
                r = y + E1 * z
                assert addrs[z] == buf.slot(r) * buf.ROWP + (par0 ^ (r & 1)) + x
            return addrs

        def run_pole(addrs, fn, write_range):
            v = [buf[a] for a in addrs]
            fn(v)
            assert all(abs(q) <= INT64_MAX for q in v)
            for i in write_range:
                buf[addrs[i]] = v[i]
            return v

        def row_addrs(sl):
            r = 2 * sl if sl < buf.NEVEN else 2 * (sl - buf.NEVEN) + 1
            off = par0 ^ (r & 1)
            return r, [sl * buf.ROWP + off + x for x in range(E0)]

        def store(x, y, v):
            for z in range(1, B2):
                gi = base + x + y * S1 + z * S2
                assert lo_i <= gi < hi_i
                out[gi] = unfix(v[z], X)
                written[gi] += 1

        if op == "h":
            for sl in range(buf.R):
                _, a = row_addrs(sl)
                run_pole(a, pole_h2, range(E0))
            for z in range(E2):
                for x in range(1, B0):
                    run_pole(pole_addrs_y(x, z), pole_h2, range(1, B1))
            for y in range(1, B1):
                for x in range(1, B0):
                    v = run_pole(pole_addrs_z(x, y), pole_h2, [])
                    store(x, y, v)
        else:
            for z in range(E2):
                for x in (0, B0):
                    run_pole(pole_addrs_y(x, z), pole_h1, range(1, B1))
            for y in range(1, B1):
                for x in (0, B0):
                    run_pole(pole_addrs_z(x, y), pole_h1, range(1, B2))
            for x in range(1, B0):
                for y in (0, B1):
                    run_pole(pole_addrs_z(x, y), pole_h1, range(1, B2))
            for sl in range(buf.R):
                r, a = row_addrs(sl)
                y, z = r % E1, r // E1
                if 0 < y < B1 and 0 < z < B2:
                    run_pole(a, pole_d, range(E0))
            for z in range(1, B2):
                for x in range(1, B0):
                    run_pole(pole_addrs_y(x, z), pole_d, range(1, B1))
            for y in range(1, B1):
                for x in range(1, B0):
                    v = run_pole(pole_addrs_z(x, y), pole_d, [])
                    store(x, y, v)
    return out, written


def interior_mask(levels, m, batch=1):
    masks = []
    for l, mk in zip(levels, m):
        i = np.arange((1 << l) + 1)
        masks.append((i % (1 << mk)) != 0)
    full = np.ones(1, dtype=bool)
    for mk in reversed(masks):
        full = np.kron(full, mk).astype(bool)
    return np.tile(full, batch)


@pytest.mark.parametrize("levels,m", [((5, 5, 5), (4, 4, 4)), ((6, 5, 4), (5, 4, 4)), ((5, 4, 5), (4, 4, 4))])
@pytest.mark.parametrize("op", ["h", "d"])
@pytest.mark.parametrize("p8", [0, 1])
def test_interior3_model(levels, m, op, p8):
    """Hierarchization: the interior class runs first, on nodal values.  The
    inverse: it runs last, when every other class holds its final nodal
    values and the interior still holds surpluses."""
    u = inputs.uniform(levels, 31 + p8)
    mask = interior_mask(levels, m)
    ref = oracle.hierarchize(u, levels) if op == "h" else oracle.dehierarchize(u, levels)
    u_in = u.copy()
    if op == "d":
        u_in[~mask] = ref[~mask]
    out, written = run_model(u_in, levels, m, op, p8)
    assert np.array_equal(written, mask.astype(np.int64))
    scale = np.abs(u).max() if op == "h" else np.abs(ref).max()
    assert np.abs(out[mask] - ref[mask]).max() <= 1e-13 * scale
    assert np.array_equal(out[~mask], u_in[~mask])


def test_interior3_model_batch_of_two():
    levels, m = (5, 4, 4), (4, 4, 4)
    N = inputs.num_points(levels)
    u = np.concatenate([inputs.uniform(levels, 41), inputs.uniform(levels, 42)])
    out, written = run_model(u, levels, m, "h", 1, batch=2)
    mask = interior_mask(levels, m, batch=2)
    assert np.array_equal(written, mask.astype(np.int64))
    for b in range(2):
        ref = oracle.hierarchize(u[b * N:(b + 1) * N], levels)
        mb = mask[b * N:(b + 1) * N]
        assert np.abs(out[b * N:(b + 1) * N][mb] - ref[mb]).max() <= 1e-13 * np.abs(u).max()
