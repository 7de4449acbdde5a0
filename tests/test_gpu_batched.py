"""GPU parity of combination-scheme plans: the batched persistent transform of
every grid of a scheme, the fp64 gather into the sparse grid and the scatter
back onto the grids (Sec. 2), against the CPU oracle."""
import numpy as np
import pytest

import oracle
from parity import TOL32, TOL64, gather_bound, rel_err
from paper_1309_0392_gb300 import inputs

torch = pytest.importorskip("torch")
gbh = pytest.importorskip("paper_1309_0392_gb300")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,n", [(1, 5), (2, 5), (3, 4), (4, 4), (4, 14), (5, 3)])
def test_scheme_matches_oracle(d, n):
    plan = gbh.Plan.scheme(d, n)
    lv, c = oracle.scheme(d, n)
    assert plan.num_grids == len(lv)
    assert np.array_equal(plan.levels(), lv)
    assert np.array_equal(plan.coeffs(), c)
    assert plan.sparse_points == oracle.sparse_num_points(d, n)
    assert plan.total_points == sum(oracle.num_points(l) for l in lv)


def _grids(lv, dtype, seed0=1000):
    return [torch.tensor(inputs.scheme_grid(l, seed0 + g), dtype=dtype, device="cuda") for g, l in enumerate(lv)]


@pytest.mark.parametrize("d,n", [(2, 6), (3, 5), (4, 5), (2, 12), (5, 3)])
@pytest.mark.parametrize("op", [gbh.GBH_HIERARCHIZE, gbh.GBH_DEHIERARCHIZE])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_transform(d, n, op, dtype):
    plan = gbh.Plan.scheme(d, n, dtype=str(dtype))
    lv = plan.levels()
    grids = _grids(lv, dtype)
    host = [g.cpu().double().numpy() for g in grids]
    plan.bind(grids)
    plan.execute(op)
    assert plan.status() == 0
    fn = oracle.hierarchize if op == gbh.GBH_HIERARCHIZE else oracle.dehierarchize
    o = "h" if op == gbh.GBH_HIERARCHIZE else "d"
    tol = TOL64 if dtype == torch.float64 else TOL32
    for l, g, u in zip(lv, grids, host):
        assert rel_err(g.cpu().double().numpy(), fn(u, l), u, o) <= tol, tuple(l)


@pytest.mark.parametrize("op", [gbh.GBH_HIERARCHIZE, gbh.GBH_DEHIERARCHIZE])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_long_dimensions(op, dtype):
    """Levels 6..17: shared-memory pole groups, and above 12 the block /
    coarse-lattice split."""
    levels = np.array([[14, 1], [1, 14], [13, 2, 1], [1, 2, 16], [17, 1], [6, 7], [8, 1, 9],
                       [12, 1], [1, 12], [3, 13]], dtype=object)
    levels = [np.array(l, dtype=np.int32) for l in levels]
    for lv_group in ([l for l in levels if len(l) == 2], [l for l in levels if len(l) == 3]):
        lv = np.stack(lv_group)
        plan = gbh.Plan.from_levels(lv, dtype=str(dtype))
        grids = _grids(lv, dtype)
        host = [g.cpu().double().numpy() for g in grids]
        plan.bind(grids)
        plan.execute(op)
        assert plan.status() == 0
        fn = oracle.hierarchize if op == gbh.GBH_HIERARCHIZE else oracle.dehierarchize
        o = "h" if op == gbh.GBH_HIERARCHIZE else "d"
        tol = TOL64 if dtype == torch.float64 else TOL32
        for l, g, u in zip(lv, grids, host):
            assert rel_err(g.cpu().double().numpy(), fn(u, l), u, o) <= tol, tuple(l)


def test_batched_round_trip_twice():
    plan = gbh.Plan.scheme(3, 6)
    grids = _grids(plan.levels(), torch.float64)
    ref = [g.clone() for g in grids]
    plan.bind(grids)
    for _ in range(2):
        plan.execute(gbh.GBH_HIERARCHIZE)
        plan.execute(gbh.GBH_DEHIERARCHIZE)
    assert plan.status() == 0
    for g, r in zip(grids, ref):
        assert (g - r).abs().max().item() <= 1e-13


def test_batched_arbitrary_levels_with_zero_levels():
    levels = np.array([[3, 0, 2], [0, 0, 0], [5, 1, 0], [2, 2, 2], [0, 4, 1]], dtype=np.int32)
    plan = gbh.Plan.from_levels(levels)
    grids = _grids(levels, torch.float64)
    host = [g.cpu().numpy() for g in grids]
    plan.bind(grids)
    plan.execute(gbh.GBH_HIERARCHIZE)
    assert plan.status() == 0
    for l, g, u in zip(levels, grids, host):
        assert rel_err(g.cpu().numpy(), oracle.hierarchize(u, l), u, "h") <= TOL64


@pytest.mark.parametrize("d,n", [(2, 5), (3, 4), (4, 4), (2, 9), (4, 10)])
def test_gather_bit_exact_on_oracle_surpluses(d, n):
    """Same surpluses in, same summation order: the fp64 gather is bit-exact.
    (4, 10): 589 grids, so the coarse subspaces' grid lists run over several
    batches of 256 grids and several staged sub-batches of their small
    chunks."""
    plan = gbh.Plan.scheme(d, n)
    lv, c = oracle.scheme(d, n)
    alphas = [oracle.hierarchize(inputs.scheme_grid(l, 1000 + g), l) for g, l in enumerate(lv)]
    grids = [torch.tensor(a, device="cuda") for a in alphas]
    plan.bind(grids)
    sparse = torch.empty(plan.sparse_points, dtype=torch.float64, device="cuda")
    plan.gather(sparse)
    ref = oracle.gather(d, n, lv, c, alphas)
    assert np.array_equal(sparse.cpu().numpy(), ref)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_hierarchize_then_gather(dtype):
    """Batched hierarchization, then the gather.  The gather of the GPU's own
    surpluses is bit-exact against the oracle's gather of those surpluses
    (same inputs, same order); against the oracle's whole chain, every sparse
    point stays within the error the coefficients carry over from the
    per-grid tolerance, sum_g |c_g| tol max|u_g|, plus the rounding of the
    two summation chains (tests/parity.py, gather_bound)."""
    d, n = 3, 5
    plan = gbh.Plan.scheme(d, n, dtype=str(dtype))
    lv, c = oracle.scheme(d, n)
    grids = _grids(lv, dtype)
    host = [g.cpu().double().numpy() for g in grids]
    plan.bind(grids)
    plan.execute(gbh.GBH_HIERARCHIZE)
    sparse = torch.empty(plan.sparse_points, dtype=torch.float64, device="cuda")
    plan.gather(sparse)
    got = sparse.cpu().numpy()
    gpu_alphas = [g.cpu().double().numpy() for g in grids]
    assert np.array_equal(got, oracle.gather(d, n, lv, c, gpu_alphas))
    alphas = [oracle.hierarchize(u, l) for u, l in zip(host, lv)]
    ref = oracle.gather(d, n, lv, c, alphas)
    tol = TOL64 if dtype == torch.float64 else TOL32
    bound = gather_bound(d, n, lv, c, alphas, [tol * np.abs(u).max() for u in host])
    assert np.all(np.abs(got - ref) <= bound)


def test_gather_partition_of_unity():
    d, n = 4, 6
    plan = gbh.Plan.scheme(d, n)
    grids = [torch.ones(oracle.num_points(l), dtype=torch.float64, device="cuda") for l in plan.levels()]
    plan.bind(grids)
    sparse = torch.empty(plan.sparse_points, dtype=torch.float64, device="cuda")
    plan.gather(sparse)
    assert torch.equal(sparse, torch.ones_like(sparse))


def test_full_scheme_d4_n14_sampled():
    """The full batched workload (1665 grids, 218.8 M points): sampled grids
    against the oracle."""
    plan = gbh.Plan.scheme(4, 14)
    lv = plan.levels()
    rng = np.random.default_rng(0)
    picks = set(int(v) for v in rng.choice(len(lv), 12, replace=False)) | {0, len(lv) - 1}
    grids = []
    for g, l in enumerate(lv):
        t = torch.empty(oracle.num_points(l), dtype=torch.float64, device="cuda")
        if g in picks:
            t.copy_(torch.from_numpy(inputs.scheme_grid(l, 1000 + g)))
        else:
            t.uniform_(-1, 1)
        grids.append(t)
    host = {g: grids[g].cpu().numpy() for g in picks}
    plan.bind(grids)
    plan.execute(gbh.GBH_HIERARCHIZE)
    assert plan.status() == 0
    for g in picks:
        assert rel_err(grids[g].cpu().numpy(), oracle.hierarchize(host[g], lv[g]), host[g], "h") <= TOL64


@pytest.mark.parametrize("d,n", [(1, 6), (2, 5), (3, 4), (4, 4), (2, 9), (5, 3)])
@pytest.mark.parametrize("scaled", [False, True])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_scatter_bit_exact(d, n, scaled, dtype):
    """Every point of every grid receives its sparse-grid value (times c_g when
    scaled), bit for bit; fp32 grids the same value rounded to float."""
    plan = gbh.Plan.scheme(d, n, dtype=str(dtype))
    lv, c = oracle.scheme(d, n)
    s = np.random.default_rng(31).uniform(-1, 1, oracle.sparse_num_points(d, n))
    grids = [torch.full((oracle.num_points(l),), float("nan"), dtype=dtype, device="cuda") for l in lv]
    plan.bind(grids)
    plan.scatter(torch.tensor(s, device="cuda"), scaled=scaled)
    ref = oracle.scatter(d, n, lv, c, s, scaled=scaled)
    for g, r in zip(grids, ref):
        want = r if dtype == torch.float64 else r.astype(np.float32)
        assert np.array_equal(g.cpu().numpy(), want)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_iterated_round(dtype):
    """Hierarchize, gather, scatter, dehierarchize on the GPU against the same
    chain in the oracle."""
    d, n = 3, 6
    plan = gbh.Plan.scheme(d, n, dtype=str(dtype))
    lv, c = oracle.scheme(d, n)
    grids = _grids(lv, dtype)
    host = [g.cpu().double().numpy() for g in grids]
    plan.bind(grids)
    sparse = torch.empty(plan.sparse_points, dtype=torch.float64, device="cuda")
    tol = TOL64 if dtype == torch.float64 else TOL32
    np_dt = np.float64 if dtype == torch.float64 else np.float32
    # every step against the oracle on that step's own input, at its own
    # tolerance: hierarchize, gather (bit-exact), scatter (bit-exact),
    # dehierarchize
    plan.execute(gbh.GBH_HIERARCHIZE)
    alphas = [g.cpu().double().numpy() for g in grids]
    for l, a, u in zip(lv, alphas, host):
        assert rel_err(a, oracle.hierarchize(u, l), u, "h") <= tol
    plan.gather(sparse)
    s = sparse.cpu().numpy()
    assert np.array_equal(s, oracle.gather(d, n, lv, c, alphas))
    plan.scatter(sparse)
    scat = oracle.scatter(d, n, lv, c, s)
    for g, r in zip(grids, scat):
        assert np.array_equal(g.cpu().numpy(), r.astype(np_dt))
    scat = [g.cpu().double().numpy() for g in grids]
    plan.execute(gbh.GBH_DEHIERARCHIZE)
    for l, g, a in zip(lv, grids, scat):
        assert rel_err(g.cpu().double().numpy(), oracle.dehierarchize(a, l), a, "d") <= tol


def test_scatter_full_scheme_d4_n14():
    """The full 4-d level-14 scheme (1665 grids, 218.8 M points, sparse grid
    25.4 M points): sampled grids bit-exact against the oracle's index, and
    gather after scatter returns the sparse grid exactly (the coefficients of
    the grids holding a point sum to 1; values with few mantissa bits)."""
    d, n = 4, 14
    plan = gbh.Plan.scheme(d, n)
    lv = plan.levels()
    s = np.random.default_rng(32).integers(-1000, 1001, plan.sparse_points) / 1024.0
    sparse = torch.tensor(s, device="cuda")
    grids = [torch.full((oracle.num_points(l),), float("nan"), dtype=torch.float64, device="cuda") for l in lv]
    plan.bind(grids)
    plan.scatter(sparse)
    rng = np.random.default_rng(0)
    for g in sorted(set(int(v) for v in rng.choice(len(lv), 10, replace=False)) | {0, len(lv) - 1}):
        assert np.array_equal(grids[g].cpu().numpy(), s[oracle.sparse_index_of_grid(d, n, lv[g])])
    back = torch.empty_like(sparse)
    plan.gather(back)
    assert torch.equal(back, sparse)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_subset_plans_of_two_ranks(dtype):
    """Plans over each rank's share of the grids: partial gathers are bit-exact
    against the oracle with the other coefficients 0 and sum to the full
    gather; scatter and execute touch only the rank's grids."""
    from paper_1309_0392_gb300 import shard
    d, n = 3, 5
    lv, c = oracle.scheme(d, n)
    parts = shard.partition_grids([oracle.num_points(l) for l in lv], 2)
    host = [inputs.scheme_grid(l, 1000 + g) for g, l in enumerate(lv)]
    if dtype == torch.float32:
        host = [h.astype(np.float32).astype(np.float64) for h in host]
    alphas = [oracle.hierarchize(h, l) for h, l in zip(host, lv)]
    total = np.zeros(oracle.sparse_num_points(d, n))
    for own in parts:
        plan = gbh.Plan.scheme(d, n, dtype=str(dtype), owned=own)
        assert np.array_equal(plan.levels(), lv[own]) and np.array_equal(plan.coeffs(), c[own])
        grids = [torch.tensor(host[g], dtype=dtype, device="cuda") for g in own]
        plan.bind(grids)
        plan.execute(gbh.GBH_HIERARCHIZE)
        tol = TOL64 if dtype == torch.float64 else TOL32
        for t, g in zip(grids, own):
            assert rel_err(t.cpu().double().numpy(), alphas[g], host[g], "h") <= tol
        if dtype == torch.float64:
            exact = [torch.tensor(alphas[g], device="cuda") for g in own]
            plan.bind(exact)
        sparse = torch.empty(plan.sparse_points, dtype=torch.float64, device="cuda")
        plan.gather(sparse)
        if dtype == torch.float64:
            assert np.array_equal(sparse.cpu().numpy(), oracle.gather(d, n, lv, shard.owned_coeffs(c, own), alphas))
        total += sparse.cpu().numpy()
        s = np.random.default_rng(33).uniform(-1, 1, plan.sparse_points)
        plan.scatter(torch.tensor(s, device="cuda"))
        back = oracle.scatter(d, n, lv[own], c[own], s)
        for t, r in zip(plan._bound, back):
            want = r if dtype == torch.float64 else r.astype(np.float32)
            assert np.array_equal(t.cpu().numpy(), want)
    full = oracle.gather(d, n, lv, c, alphas)
    # fp64: each partial is bit-exact, so the two sums differ only by the
    # rounding of the partial chains and of their sum: one unit in the last
    # place per term and one for the final addition (gather_bound with no
    # carried error).  fp32: the gathered grids hold the GPU's fp32
    # surpluses, each within tol max|u_g| of the oracle's.
    err = [0.0 if dtype == torch.float64 else TOL32 * np.abs(h).max() for h in host]
    bound = gather_bound(d, n, lv, c, alphas, err) + 2.0 ** -52 * np.abs(full)
    assert np.all(np.abs(total - full) <= bound)


def test_subset_plan_rejects_bad_lists():
    for owned in ([], [3, 1], [0, 0], [-1], [10 ** 6]):
        with pytest.raises(gbh.GbhError):
            gbh.Plan.scheme(3, 4, owned=owned)


def test_scatter_argument_errors():
    plan = gbh.Plan.scheme(2, 4)
    sparse = torch.zeros(plan.sparse_points, dtype=torch.float64, device="cuda")
    with pytest.raises(gbh.GbhError):
        plan.scatter(sparse)                        # grids not bound
    with pytest.raises(ValueError):
        plan.scatter(sparse[:-1])                   # wrong size
    with pytest.raises(ValueError):
        plan.scatter(sparse.float())                # wrong dtype
    other = gbh.Plan.from_levels([[2, 2], [3, 1]])
    other.bind([torch.zeros(oracle.num_points(l), dtype=torch.float64, device="cuda") for l in [(2, 2), (3, 1)]])
    with pytest.raises(gbh.GbhError):
        other.scatter(sparse)                       # a plan without a sparse grid
    with pytest.raises(gbh.GbhError):
        other.gather(sparse)


def test_bounded_wait_reports_timeout():
    """A dependency that nothing releases: the waits give up, the plan reports
    GBH_ETIMEOUT, the context stays usable, and normal operation resumes."""
    plan = gbh.Plan.scheme(3, 5)
    lv = plan.levels()
    grids = _grids(lv, torch.float64)
    plan.bind(grids)
    plan.test_stall(3, spin_limit=1 << 12)
    plan.execute(gbh.GBH_HIERARCHIZE)
    assert plan.status() == -6
    assert plan.status() == 0                       # reading clears it
    plan.test_stall(-1)
    fresh = _grids(lv, torch.float64)
    host = [g.cpu().numpy() for g in fresh]
    plan.bind(fresh)
    plan.execute(gbh.GBH_HIERARCHIZE)
    assert plan.status() == 0
    for l, g, u in zip(lv, fresh, host):
        assert rel_err(g.cpu().numpy(), oracle.hierarchize(u, l), u, "h") <= TOL64
