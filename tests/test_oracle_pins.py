"""Pins of the CPU oracle against facts that do not come from the oracle:
brute-force solves in the hat basis, closed forms, invariants, the paper's
boundary-free Alg. 1 and its operation counts (Sec. 3, Eq. 1), and the
partition of unity of the combination technique (Sec. 2).

CPU only (no GPU marker)."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1309_0392_gb300 import inputs

LEVELS_SMALL = [(0,), (1,), (3,), (2, 1), (1, 3), (3, 2), (0, 2), (2, 0, 1), (1, 2, 2), (3, 1, 1),
                (2, 2, 2)]


# ---------------------------------------------------------------------------
# brute force: the hierarchical hat basis written out from its definition
# ---------------------------------------------------------------------------

def hat_matrix_1d(l):
    """Phi[i, a] = phi_a(x_i) for the boundary hierarchical basis of level l:
    phi_0 = 1 - x, phi_{2^l} = x, interior phi_a a hat of half-width 2^{-level(a)}."""
    n = 2 ** l + 1
    x = np.arange(n) / 2 ** l
    phi = np.zeros((n, n))
    phi[:, 0] = 1 - x
    phi[:, n - 1] = x
    for a in range(1, n - 1):
        tz = (a & -a).bit_length() - 1
        h = 2.0 ** -(l - tz)
        phi[:, a] = np.maximum(0.0, 1 - np.abs(x - x[a]) / h)
    return phi


def hat_matrix(levels):
    """Full tensor matrix in flat order (dimension 0 fastest)."""
    m = np.ones((1, 1))
    for l in reversed(levels):          # np.kron(A, B): B's index runs fastest
        m = np.kron(m, hat_matrix_1d(l))
    return m


@pytest.mark.parametrize("levels", LEVELS_SMALL)
def test_brute_force_hat_basis(orc, levels):
    rng = np.random.default_rng(11)
    phi = hat_matrix(list(levels))
    u = rng.uniform(-1, 1, phi.shape[0])
    alpha = np.linalg.solve(phi, u)
    scale = np.abs(u).max()
    assert np.abs(orc.hierarchize(u, levels) - alpha).max() <= 1e-12 * scale
    assert np.abs(orc.dehierarchize(alpha, levels) - phi @ alpha).max() <= 1e-12 * scale
    # the transpose of Phi^{-1}
    y = rng.uniform(-1, 1, phi.shape[0])
    assert np.abs(orc.hierarchize_adjoint(y, levels) - np.linalg.solve(phi.T, y)).max() <= 1e-12
    # the transpose of Phi
    assert np.abs(orc.dehierarchize_adjoint(y, levels) - phi.T @ y).max() <= 1e-12 * np.abs(phi.T @ y).max()


@pytest.mark.parametrize("levels", LEVELS_SMALL)
def test_point_forms_match_sweeps(orc, levels):
    rng = np.random.default_rng(3)
    n = orc.num_points(levels)
    u = rng.uniform(-1, 1, n)
    idx = np.arange(n)
    assert np.abs(orc.hierarchize_at(u, levels, idx) - orc.hierarchize(u, levels)).max() <= 1e-14
    assert np.abs(orc.dehierarchize_at(u, levels, idx) - orc.dehierarchize(u, levels)).max() <= 1e-13
    assert np.abs(orc.adjoint_at(u, levels, idx) - orc.hierarchize_adjoint(u, levels)).max() <= 1e-14


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

def point_levels(levels):
    """Per-point array of per-dimension hierarchical levels, shape [N, d]."""
    per_dim = []
    for l in levels:
        i = np.arange(2 ** l + 1)
        lev = np.zeros_like(i)
        inner = (i > 0) & (i < 2 ** l)
        tz = np.array([(int(v) & -int(v)).bit_length() - 1 if v else 0 for v in i])
        lev[inner] = l - tz[inner]
        per_dim.append(lev)
    grids = np.meshgrid(*per_dim[::-1], indexing="ij")
    return np.stack([g.reshape(-1) for g in grids[::-1]], axis=1)


@pytest.mark.parametrize("levels", [(3,), (2, 3), (3, 1, 2), (1, 1, 1, 2)])
def test_multilinear_has_zero_surplus(orc, levels):
    rng = np.random.default_rng(7)
    a, b = rng.uniform(-2, 2, len(levels)), rng.uniform(-2, 2, len(levels))
    u = inputs.sample(levels, lambda *xs: math.prod([a[k] + b[k] * x for k, x in enumerate(xs)]))
    al = orc.hierarchize(u, levels)
    lev = point_levels(levels)
    interior = (lev > 0).any(axis=1)
    assert np.abs(al[interior]).max() <= 1e-14
    assert np.array_equal(al[~interior], u[~interior])


@pytest.mark.parametrize("levels,k", [((5,), 0), ((3, 4), 0), ((3, 4), 1), ((2, 3, 2), 2)])
def test_square_closed_form(orc, levels, k):
    """f = x_k^2: surplus -h_j^2 = -4^{-j} at points interior in dimension k and
    on the boundary in every other dimension; 0 at points interior in another
    dimension; nodal values at the corners.  Dyadic throughout: bit-exact."""
    u = inputs.sample(levels, lambda *xs: xs[k] ** 2)
    al = orc.hierarchize(u, levels)
    lev = point_levels(levels)
    others = np.delete(lev, k, axis=1)
    expect = np.zeros_like(u)
    edge = (lev[:, k] > 0) & (others == 0).all(axis=1)
    expect[edge] = -(4.0 ** -lev[edge, k])
    corner = (lev == 0).all(axis=1)
    expect[corner] = u[corner]
    assert np.array_equal(al, expect)


def test_cfg1b_closed_form(orc):
    """x^2 + 3xy on level (5,5): -4^{-j_x} at (x interior, y boundary), 0 at
    every point interior in y, corners 0, 1, 0, 4.  Bit-exact."""
    levels, u = inputs.cfg1b()
    al = orc.hierarchize(u, levels).reshape(33, 33)     # [y, x]
    lev = point_levels(levels).reshape(33, 33, 2)
    expect = np.zeros((33, 33))
    for iy in (0, 32):
        for ix in range(1, 32):
            expect[iy, ix] = -(4.0 ** -lev[iy, ix, 0])
    expect[0, 0], expect[0, 32], expect[32, 0], expect[32, 32] = 0.0, 1.0, 0.0, 4.0
    assert np.array_equal(al, expect)


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("levels", [(7,), (4, 5), (3, 4, 2), (2, 1, 3, 2), (0, 3, 1)])
def test_round_trip(orc, levels):
    rng = np.random.default_rng(5)
    u = rng.uniform(-1, 1, orc.num_points(levels))
    assert np.abs(orc.dehierarchize(orc.hierarchize(u, levels), levels) - u).max() <= 1e-14
    assert np.abs(orc.hierarchize(orc.dehierarchize(u, levels), levels) - u).max() <= 1e-13


@pytest.mark.parametrize("levels", [(6,), (4, 3), (3, 3, 3), (2, 2, 1, 2)])
def test_adjoint_dot_product(orc, levels):
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, orc.num_points(levels))
    y = rng.uniform(-1, 1, orc.num_points(levels))
    hx = orc.hierarchize(x, levels)
    lhs, rhs = hx @ y, x @ orc.hierarchize_adjoint(y, levels)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(hx) * np.linalg.norm(y)


@pytest.mark.parametrize("levels", [(6,), (4, 3), (3, 3, 3), (2, 2, 1, 2)])
def test_dehierarchize_adjoint_dot_product_and_inverse(orc, levels):
    """<D x, y> = <x, D^T y>, and D^T inverts the transpose of hierarchization
    (D^T H^T = (H D)^T = I)."""
    rng = np.random.default_rng(10)
    x = rng.uniform(-1, 1, orc.num_points(levels))
    y = rng.uniform(-1, 1, orc.num_points(levels))
    dx = orc.dehierarchize(x, levels)
    dty = orc.dehierarchize_adjoint(y, levels)
    assert abs(dx @ y - x @ dty) <= 1e-12 * np.linalg.norm(dx) * np.linalg.norm(y)
    assert np.abs(orc.dehierarchize_adjoint(orc.hierarchize_adjoint(y, levels), levels) - y).max() <= 1e-13
    assert np.abs(orc.hierarchize_adjoint(dty, levels) - y).max() <= 1e-13 * np.abs(dty).max()


def test_dehierarchize_adjoint_1d_closed_form(orc):
    """One pole: (D^T y)[p] = sum_i phi_p(x_i) y_i, so with y = 1 the value at
    p is the sum of its hat over the nodes: 2^l / 2^{level(p)} for an interior
    p, (2^l + 1) / 2 at either boundary point (exact, dyadic)."""
    l = 6
    n = 2 ** l + 1
    got = orc.dehierarchize_adjoint(np.ones(n), (l,))
    want = np.empty(n)
    for p in range(n):
        if p in (0, n - 1):
            want[p] = (2 ** l + 1) / 2
        else:
            tz = (p & -p).bit_length() - 1
            want[p] = 2.0 ** tz          # hat of half-width 2^tz nodes sums to 2^tz
    assert np.array_equal(got, want)


@pytest.mark.parametrize("levels", [(3, 4), (2, 3, 2)])
def test_dimension_order_independence(orc, levels):
    """The per-dimension operators commute; on dyadic data of few bits every
    order rounds nothing, so permuted sweeps agree bit for bit."""
    rng = np.random.default_rng(1)
    n = orc.num_points(levels)
    u = rng.integers(-64, 64, n).astype(np.float64) / 64.0
    ref = orc.hierarchize(u, levels)
    d = len(levels)
    shp = inputs.shape_of(levels)
    for perm in itertools.permutations(range(d)):
        # new dimension m is old dimension perm[m]
        new_levels = [levels[p] for p in perm]
        arr = u.reshape(shp)                           # axes: old dims reversed
        axes = [d - 1 - perm[m] for m in reversed(range(d))]
        moved = np.ascontiguousarray(np.transpose(arr, axes)).reshape(-1)
        out = orc.hierarchize(moved, new_levels).reshape(inputs.shape_of(new_levels))
        back = np.transpose(out, np.argsort(axes)).reshape(-1)
        assert np.array_equal(back, ref), perm


# ---------------------------------------------------------------------------
# the paper's boundary-free Alg. 1 and its operation counts (Sec. 3, Eq. 1)
# ---------------------------------------------------------------------------

def eq1_corrected(levels):
    """Eq. 1 with the inner term 2^{l_i+1} - 2 l_i - 2 (adds; flops = 2 x adds)."""
    d = len(levels)
    tot = 0
    for i in range(d):
        p = 1
        for j in range(d):
            if j != i:
                p *= 2 ** levels[j] - 1
        tot += (2 ** (levels[i] + 1) - 2 * levels[i] - 2) * p
    return 2 * tot


def eq1_printed(levels):
    d = len(levels)
    tot = 0
    for i in range(d):
        p = 1
        for j in range(d):
            if j != i:
                p *= 2 ** levels[j] - 1
        tot += (2 ** levels[i] - 2 * levels[i] - 2) * p
    return 2 * tot


def mults_reduced(levels):
    """M(d, l) of Sec. 3 (reduced-op multiplications)."""
    d = len(levels)
    tot = 0
    for i in range(d):
        p = 1
        for j in range(d):
            if j != i:
                p *= 2 ** levels[j] - 1
        tot += (2 ** levels[i] - 2) * p
    return tot


@pytest.mark.parametrize("levels", [(2,), (3,), (5,), (2, 3), (4, 2), (3, 3, 2), (1, 4), (2, 2, 2, 2)])
def test_flop_counts(orc, levels):
    n = int(np.prod([2 ** l - 1 for l in levels]))
    u = np.ones(n)
    _, adds, muls = orc.hierarchize_nobnd(u, levels, reduced_op=False)
    assert adds == muls and adds + muls == eq1_corrected(levels)
    _, adds_r, muls_r = orc.hierarchize_nobnd(u, levels, reduced_op=True)
    assert muls_r == mults_reduced(levels)
    assert adds_r == eq1_corrected(levels) // 2          # A = F / 2


def test_eq1_as_printed_is_off():
    # the printed inner term gives a negative count for l = 2; counting gives 2 adds
    assert eq1_printed([2]) == -4 and eq1_corrected([2]) == 4
    assert eq1_corrected([3]) == 16


@pytest.mark.parametrize("levels", [(4,), (3, 2), (2, 3, 2)])
def test_boundary_zero_reduces_to_paper_alg1(orc, levels):
    """With zero boundary values the boundary grid's interior is the paper's
    boundary-free grid of the same level, and the results agree."""
    rng = np.random.default_rng(2)
    inner_shape = tuple(2 ** l - 1 for l in reversed(levels))
    v = rng.uniform(-1, 1, inner_shape)
    full = np.zeros(inputs.shape_of(levels))
    full[tuple(slice(1, -1) for _ in levels)] = v
    ours = orc.hierarchize(full.reshape(-1), levels).reshape(full.shape)
    ours_inner = ours[tuple(slice(1, -1) for _ in levels)].reshape(-1)
    red, _, _ = orc.hierarchize_nobnd(v.reshape(-1), levels, reduced_op=True)
    two, _, _ = orc.hierarchize_nobnd(v.reshape(-1), levels, reduced_op=False)
    assert np.array_equal(ours_inner, red)
    assert np.abs(ours_inner - two).max() <= 1e-15


# ---------------------------------------------------------------------------
# combination scheme and gather (Sec. 2)
# ---------------------------------------------------------------------------

def test_scheme_enumeration(orc):
    lv, c = orc.scheme(4, 14)
    assert lv.shape == (1665, 4)
    sums = lv.sum(axis=1)
    counts = [int((sums == 17 - q).sum()) for q in range(4)]
    assert counts == [560, 455, 364, 286]
    assert (lv >= 1).all()
    for q, coef in enumerate([1, -3, 3, -1]):
        assert (c[sums == 17 - q] == coef).all()
    # q ascending, then lexicographic (l_0 most significant)
    keys = [(-int(s),) + tuple(int(v) for v in row) for s, row in zip(sums, lv)]
    assert keys == sorted(keys)
    assert len({tuple(r) for r in lv.tolist()}) == 1665


def subspaces(d, n):
    return [j for j in itertools.product(range(n + 1), repeat=d)
            if sum(max(v, 1) for v in j) <= n + d - 1]


def test_sparse_size(orc):
    for d, n in [(2, 3), (3, 4), (4, 14)]:
        tot = sum(int(np.prod([2 if v == 0 else 2 ** (v - 1) for v in j])) for j in subspaces(d, n))
        assert orc.sparse_num_points(d, n) == tot
    assert orc.sparse_num_points(4, 14) == 25_362_433


def _coord_key(levels, flat):
    rem, key = int(flat), []
    for l in levels:
        l = int(l)
        n = 2 ** l + 1
        key.append(Fraction(rem % n, 2 ** l))
        rem //= n
    return tuple(key)


@pytest.mark.parametrize("d,n", [(2, 3), (3, 3), (2, 5)])
def test_gather_matches_coordinate_dictionary(orc, d, n):
    """Brute force: sum c_g alpha_g keyed by exact point coordinates."""
    lv, c = orc.scheme(d, n)
    rng = np.random.default_rng(4)
    grids = [rng.uniform(-1, 1, orc.num_points(l)) for l in lv]
    sparse = orc.gather(d, n, lv, c, grids)
    acc = {}
    for l, cg, g in zip(lv, c, grids):
        for f in range(g.size):
            key = _coord_key(l, f)
            acc[key] = acc.get(key, 0.0) + cg * g[f]
    assert len(acc) == sparse.size
    # map coordinates to the subspace-major layout
    for l, g in zip(lv, grids):
        idx = orc.sparse_index_of_grid(d, n, l)
        for f in range(g.size):
            assert sparse[idx[f]] == pytest.approx(acc[_coord_key(l, f)], abs=1e-14)
    # the layout: subspace-major, lexicographic j (j_0 most significant), dim 0 fastest
    off = 0
    for j in subspaces(d, n):
        size = int(np.prod([2 if v == 0 else 2 ** (v - 1) for v in j]))
        for pos in range(size):
            rem, x = pos, []
            for v in j:
                w = 2 if v == 0 else 2 ** (v - 1)
                p = rem % w
                rem //= w
                x.append(Fraction(p, 1) if v == 0 else Fraction(2 * p + 1, 2 ** v))
            assert sparse[off + pos] == pytest.approx(acc[tuple(x)], abs=1e-14)
        off += size


@pytest.mark.parametrize("d,n", [(2, 4), (3, 4), (4, 3)])
def test_partition_of_unity(orc, d, n):
    lv, c = orc.scheme(d, n)
    grids = [np.ones(orc.num_points(l)) for l in lv]
    assert np.array_equal(orc.gather(d, n, lv, c, grids), np.ones(orc.sparse_num_points(d, n)))


@pytest.mark.parametrize("d,n", [(2, 4), (3, 3)])
def test_gather_of_one_function_is_its_sparse_surplus(orc, d, n):
    """Every grid samples the same f.  The surplus of a point depends only on f
    at the point and at its predecessors at its own spacing 2^{-j_k}, so the
    combination returns that 3^d-stencil value (computed here from f)."""
    def f(*xs):
        return math.prod(math.sin(1.0 + (k + 1) * x) for k, x in enumerate(xs))

    fv = lambda *xs: math.prod([np.sin(1.0 + (k + 1) * x) for k, x in enumerate(xs)])
    lv, c = orc.scheme(d, n)
    grids = [orc.hierarchize(inputs.sample(l, fv), l) for l in lv]
    sparse = orc.gather(d, n, lv, c, grids)
    off = 0
    for j in subspaces(d, n):
        size = int(np.prod([2 if v == 0 else 2 ** (v - 1) for v in j]))
        for pos in range(size):
            rem, x, h = pos, [], []
            for v in j:
                w = 2 if v == 0 else 2 ** (v - 1)
                p = rem % w
                rem //= w
                x.append(float(p) if v == 0 else (2 * p + 1) / 2 ** v)
                h.append(0.0 if v == 0 else 2.0 ** -v)
            val = 0.0
            for delta in itertools.product((-1, 0, 1), repeat=d):
                wt = 1.0
                for k in range(d):
                    if delta[k] != 0:
                        wt *= 0.0 if h[k] == 0.0 else -0.5
                if wt != 0.0:
                    val += wt * f(*[x[k] + delta[k] * h[k] for k in range(d)])
            assert sparse[off + pos] == pytest.approx(val, abs=1e-13)
        off += size


def _sparse_layout(d, n):
    """Sparse-grid points in subspace-major order, written out from the layout
    definition: (subspace j, position p, coordinates as Fractions)."""
    out = []
    for j in subspaces(d, n):
        size = int(np.prod([2 if v == 0 else 2 ** (v - 1) for v in j]))
        for pos in range(size):
            rem, x, p = pos, [], []
            for v in j:
                w = 2 if v == 0 else 2 ** (v - 1)
                pk = rem % w
                rem //= w
                p.append(pk)
                x.append(Fraction(pk, 1) if v == 0 else Fraction(2 * pk + 1, 2 ** v))
            out.append((j, tuple(p), tuple(x)))
    return out


@pytest.mark.parametrize("d,n", [(2, 3), (3, 3), (2, 5), (4, 2)])
@pytest.mark.parametrize("scaled", [False, True])
def test_scatter_matches_coordinate_dictionary(orc, d, n, scaled):
    """Every grid point takes the sparse value at its own coordinates."""
    lv, c = orc.scheme(d, n)
    layout = _sparse_layout(d, n)
    where = {x: q for q, (_, _, x) in enumerate(layout)}
    sparse = np.random.default_rng(11).uniform(-1, 1, len(layout))
    grids = orc.scatter(d, n, lv, c, sparse, scaled=scaled)
    for l, cg, g in zip(lv, c, grids):
        assert g.size == orc.num_points(l)
        for f in range(g.size):
            v = sparse[where[_coord_key(l, f)]]
            assert g[f] == (cg * v if scaled else v)


@pytest.mark.parametrize("d,n", [(2, 4), (3, 3), (4, 3)])
def test_scaled_scatter_is_transpose_of_gather(orc, d, n):
    """<gather(alpha), s> = sum_g <alpha_g, scatter_scaled(s)_g>, exact on
    small integers."""
    lv, c = orc.scheme(d, n)
    rng = np.random.default_rng(12)
    alphas = [rng.integers(-8, 9, orc.num_points(l)).astype(np.float64) for l in lv]
    s = rng.integers(-8, 9, orc.sparse_num_points(d, n)).astype(np.float64)
    lhs = int(np.dot(orc.gather(d, n, lv, c, alphas).astype(np.int64), s.astype(np.int64)))
    back = orc.scatter(d, n, lv, c, s, scaled=True)
    rhs = sum(int(np.dot(a.astype(np.int64), b.astype(np.int64))) for a, b in zip(alphas, back))
    assert lhs == rhs


@pytest.mark.parametrize("d,n", [(2, 4), (3, 4), (4, 3)])
def test_gather_after_scatter_is_identity(orc, d, n):
    """Partition of unity: the coefficients of the grids holding a point sum
    to 1, so gathering the scattered sparse grid returns it (exact on
    values with few mantissa bits)."""
    lv, c = orc.scheme(d, n)
    s = np.random.default_rng(13).integers(-1000, 1001, orc.sparse_num_points(d, n)) / 1024.0
    assert np.array_equal(orc.gather(d, n, lv, c, orc.scatter(d, n, lv, c, s)), s)


@pytest.mark.parametrize("d,n", [(2, 3), (2, 4), (3, 3)])
def test_iterated_round_gives_sparse_interpolant(orc, d, n):
    """One round of the iterated combination technique (hierarchize, gather,
    scatter, dehierarchize) leaves on every grid the combined sparse-grid
    function at that grid's points, evaluated here as a sum over the sparse
    hat basis."""
    fv = lambda *xs: math.prod([np.cos(0.5 + (k + 2) * x) for k, x in enumerate(xs)])
    lv, c = orc.scheme(d, n)
    grids = [orc.hierarchize(inputs.sample(l, fv), l) for l in lv]
    sparse = orc.gather(d, n, lv, c, grids)
    back = [orc.dehierarchize(g, l) for g, l in zip(orc.scatter(d, n, lv, c, sparse), lv)]
    layout = _sparse_layout(d, n)

    def hat(j, p, x):
        if j == 0:
            return 1.0 - x if p == 0 else x
        return max(0.0, 1.0 - abs(x - (2 * p + 1) * 2.0 ** -j) * 2.0 ** j)

    for l, g in zip(lv, back):
        for f in range(g.size):
            x = [float(v) for v in _coord_key(l, f)]
            want = sum(sparse[q] * math.prod(hat(j[k], p[k], x[k]) for k in range(d))
                       for q, (j, p, _) in enumerate(layout))
            assert g[f] == pytest.approx(want, abs=1e-13)


@pytest.mark.parametrize("d,n", [(2, 3), (3, 3)])
def test_exact_gather_is_order_free_and_close_to_the_ordered_one(orc, d, n):
    """The exactly rounded gather: equal to the ordered fma gather when every
    partial sum is exact (few mantissa bits), independent of the grid order,
    and within a few units of the last place of the ordered gather on
    general data."""
    lv, c = orc.scheme(d, n)
    rng = np.random.default_rng(23)
    dyadic = [rng.integers(-64, 65, orc.num_points(l)) / 64.0 for l in lv]
    assert np.array_equal(orc.gather_exact(d, n, lv, c, dyadic), orc.gather(d, n, lv, c, dyadic))
    grids = [rng.uniform(-1, 1, orc.num_points(l)) for l in lv]
    exact = orc.gather_exact(d, n, lv, c, grids)
    perm = rng.permutation(len(lv))
    assert np.array_equal(orc.gather_exact(d, n, lv[perm], c[perm], [grids[i] for i in perm]), exact)
    ordered = orc.gather(d, n, lv, c, grids)
    bound = len(lv) * np.finfo(float).eps * sum(abs(cg) * np.abs(g).max() for cg, g in zip(c, grids))
    assert np.abs(ordered - exact).max() <= bound


def test_level_weights(orc):
    levels = (2, 1)
    w = orc.level_weights(levels).reshape(3, 5)
    lev_x = np.array([0, 2, 1, 2, 0])
    lev_y = np.array([0, 1, 0])
    assert np.array_equal(w, 2.0 ** -(lev_y[:, None] + lev_x[None, :]))
