"""A CPU model of the interior-class kernel (``csrc/interior3.cu``), checked
before and beside its GPU runs.  CPU only.

- index arithmetic: every copy the loader issues (16-byte pairs and single
  8-byte elements, one y and every z per thread, the parity-shifted shared
  layout of a 33 x 17 x 17 closure), the row and pole assignments of the
  passes, and the interior points the kernel writes;
- arithmetic: the kernel's steps restated in numpy (int64 fixed point per
  closure with truncation, doubling-form hierarchization, rounded-half
  inverse with its face stage) on small grids, compared with the oracle at
  the points the kernel finalises (interior to their tile in every
  dimension).

The GPU tests check the kernel itself against the oracle."""
import numpy as np
import pytest

E0, E1, E2 = 33, 17, 17
XC = E0 - 1
NV, NVP = E0 * E1 * E2, E0 * E1 * E2 + 1
ROWS, PLANE = E1 * E2, E0 * E1
T = 320
NPR = XC // 2


def geom(levels):
    n = [(1 << l) + 1 for l in levels]
    return n, n[0], n[0] * n[1]


# ---------------------------------------------------------------------------
# index arithmetic
# ---------------------------------------------------------------------------

def loader_copies(o00, S1, S2):
    """(shared index, global offset from the closure origin, size, row, x) of
    every copy: a thread takes one y and every z."""
    out = []
    for gt in range(T):
        if gt < NPR * E1:
            y0, c, single = gt // NPR, gt % NPR, False
        elif gt < (NPR + 1) * E1:
            y0, c, single = gt - NPR * E1, 0, True
        else:
            continue
        xe, xo = (E0 - 1, 0) if single else (2 * c, 2 * c + 1)
        p0 = (o00 + y0) & 1
        for z in range(E2):
            x = xo if (p0 + z) & 1 else xe
            r = y0 + E1 * z
            out.append((o00 + y0 * E0 + z * PLANE + x, y0 * S1 + z * S2 + x, 8 if single else 16, r, x))
    return out


@pytest.mark.parametrize("levels", [(9, 9, 9), (6, 5, 5), (5, 4, 4), (9, 10, 4)])
@pytest.mark.parametrize("ualign", [0, 1])
def test_loader_copies_cover_the_closure_once_aligned(levels, ualign):
    _, S1, S2 = geom(levels)
    for origin in (0, 32, 16 * S1, 16 * S2 + 32, 16 * S1 + 16 * S2 + 64):
        o00 = (ualign + origin) & 1
        seen = np.zeros(NVP, dtype=np.int64)
        for s, g, size, r, x in loader_copies(o00, S1, S2):
            y, z = r % E1, r // E1
            assert g == x + y * S1 + z * S2
            n = size // 8
            assert 0 <= s and s + n <= NVP
            if size == 16:
                assert s % 2 == 0, "shared destination not 16-byte aligned"
                assert (ualign + origin + g) % 2 == 0, "global source not 16-byte aligned"
            assert s - o00 == r * E0 + x
            seen[s:s + n] += 1
        assert seen[o00:o00 + NV].min() == 1 and seen.max() == 1


def inner2_row(q, j):
    """j-th row with y, z in [1, 15] and y + z of parity q."""
    codd = 7 if q else 8
    P, rem = divmod(j, 15)
    z = 2 * P + 1 + (rem >= codd)
    k = rem - codd if rem >= codd else rem
    y = (1 if (q - z) & 1 else 2) + 2 * k
    return y, z


def test_pass_mappings():
    _, S1, S2 = geom((9, 9, 9))
    for _, g, _, _, _ in loader_copies(0, S1, S2):
        assert 0 <= g < 2 ** 31
    assert (NPR + 1) * E1 <= T
    # rows: even rows on threads 0..159, odd rows on 160..319 (one parity and
    # one 16-byte access pattern per warp)
    xr = [2 * t if t < T // 2 else 2 * (t - T // 2) + 1 for t in range(T)]
    assert sorted(r for r in xr if r < ROWS) == list(range(ROWS))
    for w in range(T // 32):
        assert len({xr[t] & 1 for t in range(32 * w, 32 * w + 32)}) == 1
    # inverse stage B rows: y, z interior by parity of y + z
    rows = []
    for tid in range(T):
        q = int(tid >= T // 2)
        j = tid - q * T // 2
        if j < (112 if q else 113):
            y, z = inner2_row(q, j)
            assert 1 <= y <= 15 and 1 <= z <= 15 and (y + z) % 2 == q
            rows.append((y, z))
    assert sorted(rows) == sorted((y, z) for y in range(1, 16) for z in range(1, 16))
    # dimension-1 poles (x interior, every z: hierarchization; x, z interior:
    # inverse), two per thread
    for nz, z0 in ((E2, 0), (E2 - 2, 1)):
        NP = (E0 - 2) * nz
        H = (NP + 1) // 2
        got = [(1 + p % (E0 - 2), z0 + p // (E0 - 2)) for tid in range(H) for p in (tid, tid + H) if p < NP]
        assert sorted(got) == sorted((x, z) for x in range(1, E0 - 1) for z in range(z0, z0 + nz)) and H <= T
    # dimension-2 poles (x, y interior): the interior points, each once
    NP = (E0 - 2) * (E1 - 2)
    H = (NP + 1) // 2
    got = [(1 + p % (E0 - 2), 1 + p // (E0 - 2)) for tid in range(H) for p in (tid, tid + H) if p < NP]
    assert sorted(got) == sorted((x, y) for x in range(1, E0 - 1) for y in range(1, E1 - 1))
    # inverse stage A1: x faces along y (every z), y faces along z (x interior)
    a1 = [divmod(tid, E2) for tid in range(2 * E2)]
    assert sorted((f * XC, z) for f, z in a1) == sorted((x, z) for x in (0, XC) for z in range(E2))
    a1y = []
    for tid in range(2 * E2, 2 * E2 + 2 * (E0 - 2)):
        f, x = divmod(tid - 2 * E2, E0 - 2)
        a1y.append((1 + x, f * (E1 - 1)))
    assert sorted(a1y) == sorted((x, y) for x in range(1, E0 - 1) for y in (0, E1 - 1))
    assert 2 * E2 + 2 * (E0 - 2) <= T
    # stage A2: x faces along z (y interior)
    a2 = [divmod(tid, E1 - 2) for tid in range(2 * (E1 - 2))]
    assert sorted((f * XC, 1 + y) for f, y in a2) == sorted((x, y) for x in (0, XC) for y in range(1, E1 - 1))


# ---------------------------------------------------------------------------
# arithmetic
# ---------------------------------------------------------------------------

def lev_of(e):
    return (e - 1).bit_length() - 1 if e > 2 else 0


def bits_of(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def emax_of(a):
    return int(((bits_of(a) >> np.uint64(52)) & np.uint64(0x7FF)).max())


def fx_in(a, emax):
    """Truncating int64 fixed point with the closure's largest exponent."""
    b = bits_of(a)
    e = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    M = (b & np.uint64((1 << 52) - 1)) | np.uint64(1 << 52)
    rs = emax - e
    assert (rs >= 0).all()
    v = np.where(rs >= 64, np.uint64(0), M >> np.minimum(rs, 63).astype(np.uint64)).astype(np.int64)
    return np.where(a < 0, -v, v).reshape(np.shape(a))


def fx_out(v, X):
    return np.ldexp(v.astype(np.float64), X)


def along(a, axis):
    return np.moveaxis(a, axis, -1)


def h_dbl(a, axis, ends):
    w = along(a, axis)
    L = lev_of(w.shape[-1])
    last = 1 << L
    for lev in range(L, 0, -1):
        s = 1 << (L - lev)
        i = np.arange(s, last, 2 * s)
        w[..., i] = (w[..., i] + w[..., i]) - w[..., i - s] - w[..., i + s]
    if ends:
        w[..., 0] += w[..., 0]
        w[..., last] += w[..., last]


def h_half(a, axis):
    w = along(a, axis)
    L = lev_of(w.shape[-1])
    last = 1 << L
    for lev in range(L, 0, -1):
        s = 1 << (L - lev)
        i = np.arange(s, last, 2 * s)
        w[..., i] = w[..., i] - ((w[..., i - s] + w[..., i + s] + 1) >> 1)


def d_fix(a, axis):
    w = along(a, axis)
    L = lev_of(w.shape[-1])
    last = 1 << L
    for lev in range(1, L + 1):
        s = 1 << (L - lev)
        i = np.arange(s, last, 2 * s)
        w[..., i] = w[..., i] + ((w[..., i - s] + w[..., i + s] + 1) >> 1)


def tiles(levels):
    for bz in range(1 << (levels[2] - 4)):
        for by in range(1 << (levels[1] - 4)):
            for bx in range(1 << (levels[0] - 5)):
                yield (slice(16 * bz, 16 * bz + 17), slice(16 * by, 16 * by + 17), slice(32 * bx, 32 * bx + 33))


def model_forward(u3, levels):
    out = u3.copy()
    for zs, ys, xs in tiles(levels):
        c = u3[zs, ys, xs]
        emax = emax_of(c)
        v = fx_in(c, emax)
        h_dbl(v, 2, True)
        h_dbl(v, 1, False)
        h_dbl(v, 0, False)
        assert np.abs(v).max() < 2 ** 62
        out[zs, ys, xs][1:16, 1:16, 1:32] = fx_out(v[1:16, 1:16, 1:32], emax - 1075 - 3)
    return out


def model_inverse(u3, levels):
    """u3 holds final nodal values outside the interior class, surpluses on it."""
    out = u3.copy()
    for zs, ys, xs in tiles(levels):
        c = u3[zs, ys, xs]
        emax = emax_of(c)
        v = fx_in(c, emax)                       # [z][y][x]
        for f in (0, XC):                        # A1: x faces along y, every z
            face = v[:, :, f]
            h_half(face, 1)
        for f in (0, E1 - 1):                    # A1: y faces along z, x interior
            face = v[:, f, 1:XC]
            h_half(face, 0)
        for f in (0, XC):                        # A2: x faces along z, y interior
            face = v[:, 1:E1 - 1, f]
            h_half(face, 0)
        rows = v[1:E2 - 1, 1:E1 - 1, :]          # B: rows y, z interior
        d_fix(rows, 2)
        poles = v[1:E2 - 1, :, 1:XC]             # dimension 1: x, z interior
        d_fix(poles, 1)
        poles = v[:, 1:E1 - 1, 1:XC]             # dimension 2: x, y interior
        d_fix(poles, 0)
        assert np.abs(v).max() < 2 ** 62
        out[zs, ys, xs][1:16, 1:16, 1:32] = fx_out(v[1:16, 1:16, 1:32], emax - 1075)
    return out


def interior_mask(levels):
    n = [(1 << l) + 1 for l in levels]
    i0 = np.arange(n[0]) % 32 != 0
    i1 = np.arange(n[1]) % 16 != 0
    i2 = np.arange(n[2]) % 16 != 0
    return i2[:, None, None] & i1[None, :, None] & i0[None, None, :]


@pytest.mark.parametrize("levels", [(6, 5, 5), (5, 4, 4), (7, 4, 5)])
def test_model_forward_matches_oracle_on_interior_points(orc, levels):
    from paper_1309_0392_gb300 import inputs
    u = inputs.uniform(levels, 31)
    n = [(1 << l) + 1 for l in levels]
    ref = orc.hierarchize(u, levels).reshape(n[2], n[1], n[0])
    got = model_forward(u.reshape(n[2], n[1], n[0]), levels)
    m = interior_mask(levels)
    assert np.abs(got - ref)[m].max() / np.abs(u).max() <= 1e-14


@pytest.mark.parametrize("levels", [(6, 5, 5), (5, 4, 4), (7, 4, 5)])
def test_model_inverse_matches_oracle_on_interior_points(orc, levels):
    from paper_1309_0392_gb300 import inputs
    a = inputs.uniform(levels, 32)
    n = [(1 << l) + 1 for l in levels]
    ref = orc.dehierarchize(a, levels).reshape(n[2], n[1], n[0])
    m = interior_mask(levels)
    state = np.where(m, a.reshape(n[2], n[1], n[0]), ref)
    got = model_inverse(state, levels)
    assert np.abs(got - ref)[m].max() / np.abs(ref).max() <= 1e-14


def test_model_inverse_headroom_on_growth_extremes(orc):
    """Surpluses of one sign everywhere (the largest nodal growth): no int64
    overflow (asserted inside the model), result within tolerance."""
    levels = (6, 5, 5)
    n = [(1 << l) + 1 for l in levels]
    a = np.ones(n[0] * n[1] * n[2])
    ref = orc.dehierarchize(a, levels).reshape(n[2], n[1], n[0])
    m = interior_mask(levels)
    state = np.where(m, a.reshape(n[2], n[1], n[0]), ref)
    got = model_inverse(state, levels)
    assert np.abs(got - ref)[m].max() / np.abs(ref).max() <= 1e-14
