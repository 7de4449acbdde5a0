"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

fp64 plain path: the kernels apply the serial operation order, so results are
bit-identical to the oracle.  Every other fp64 path: within 1e-13 relative to
max|u|.  fp32: within 1e-5 relative to max|u| against the oracle run on the
same fp32 input promoted to fp64.  u is the nodal vector: the input of a
hierarchization or of a transpose, the output of a dehierarchization.
"""
import numpy as np
import pytest

import oracle
from golden_io import load
from parity import TOL32, TOL64, rel_err
from paper_1309_0392_gb300 import inputs

torch = pytest.importorskip("torch")
gbh = pytest.importorskip("paper_1309_0392_gb300")

pytestmark = pytest.mark.gpu

OPS = {"h": gbh.GBH_HIERARCHIZE, "d": gbh.GBH_DEHIERARCHIZE, "a": gbh.GBH_ADJOINT,
       "t": gbh.GBH_DEHIERARCHIZE_ADJOINT}
ORACLE = {"h": oracle.hierarchize, "d": oracle.dehierarchize, "a": oracle.hierarchize_adjoint,
          "t": oracle.dehierarchize_adjoint}


def run(u, levels, op, dtype=torch.float64, **kw):
    t = torch.tensor(u, dtype=dtype, device="cuda")
    gbh.transform(t, levels, OPS[op], **kw)
    torch.cuda.synchronize()
    return t.cpu().double().numpy()


@pytest.mark.parametrize("op,name", [("h", "cfg1a_hierarchize.txt"), ("d", "cfg1a_dehierarchize.txt"),
                                     ("a", "cfg1a_adjoint.txt"), ("t", "cfg1a_dehier_adjoint.txt")])
@pytest.mark.parametrize("path", [gbh.GBH_PATH_PLAIN, gbh.GBH_PATH_AUTO])
def test_cfg1a_golden(op, name, path):
    levels, u = inputs.cfg1a()
    got = run(u, levels, op, path=path)
    ref = load(name)
    if path == gbh.GBH_PATH_PLAIN:
        assert np.array_equal(got, ref)
    else:
        assert rel_err(got, ref, u, op) <= TOL64


@pytest.mark.parametrize("path", [gbh.GBH_PATH_PLAIN, gbh.GBH_PATH_AUTO])
def test_cfg1b_closed_form_bit_exact(path):
    levels, u = inputs.cfg1b()
    assert np.array_equal(run(u, levels, "h", path=path), load("cfg1b_hierarchize.txt"))


def random_levels(rng, count):
    out = []
    for _ in range(count):
        d = int(rng.integers(1, 7))
        budget = 16 if d <= 3 else 14
        lv = []
        for _ in range(d):
            lv.append(int(rng.integers(0, 9)))
        while sum(lv) > budget:
            k = int(np.argmax(lv))
            lv[k] -= 1
        out.append(tuple(lv))
    return out


LEVELS = [(1,), (5,), (12,), (3, 4), (9, 0), (0, 9), (1, 1, 1), (5, 4, 4), (4, 6, 3), (2, 3, 1, 4),
          (3, 3, 2, 2, 2), (1, 2, 1, 2, 1, 2)] + random_levels(np.random.default_rng(2024), 12)


@pytest.mark.parametrize("levels", LEVELS)
@pytest.mark.parametrize("op", ["h", "d", "a"])
def test_plain_fp64_bit_exact(levels, op):
    u = inputs.uniform(levels, 100 + len(levels))
    assert np.array_equal(run(u, levels, op, path=gbh.GBH_PATH_PLAIN), ORACLE[op](u, levels))


@pytest.mark.parametrize("levels", LEVELS)
@pytest.mark.parametrize("op", ["h", "d", "a"])
def test_auto_fp64(levels, op):
    u = inputs.uniform(levels, 200 + len(levels))
    assert rel_err(run(u, levels, op), ORACLE[op](u, levels), u, op) <= TOL64


@pytest.mark.parametrize("levels", LEVELS)
@pytest.mark.parametrize("op", ["h", "d", "a"])
def test_plain_fixed_point_fp64(levels, op):
    """Sweeps in int64 fixed point, one binary scale per pole group."""
    u = inputs.uniform(levels, 250 + len(levels))
    assert rel_err(run(u, levels, op, path=gbh.GBH_PATH_PLAIN, arith=2), ORACLE[op](u, levels), u, op) <= TOL64


@pytest.mark.parametrize("levels", [l for l in LEVELS if len(l) >= 2 and max(l) <= 12]
                         + [(6, 6, 5, 5, 5), (3, 3, 3, 3, 3, 3, 2, 2), (12, 3), (2, 2, 11)])
@pytest.mark.parametrize("op", ["h", "d"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_grouped_path(levels, op, dtype):
    """One pass per group of consecutive dimensions (shared-memory tiles of
    pole sets, per-tile fixed point in fp64)."""
    tol = TOL64 if dtype == torch.float64 else TOL32
    u = inputs.uniform(levels, 400 + len(levels), dtype=np.float64 if dtype == torch.float64 else np.float32)
    got = run(u, levels, op, dtype=dtype, path=gbh.GBH_PATH_GROUPED)
    ud = u.astype(np.float64)
    assert rel_err(got, ORACLE[op](ud, levels), ud, op) <= tol


def test_grouped_path_declines():
    for levels, op in [((13, 2), gbh.GBH_HIERARCHIZE), ((4, 4), gbh.GBH_ADJOINT), ((1,) * 9, gbh.GBH_HIERARCHIZE)]:
        t = torch.zeros(inputs.num_points(levels), dtype=torch.float64, device="cuda")
        with pytest.raises(gbh.GbhError):
            gbh.transform(t, levels, op, path=gbh.GBH_PATH_GROUPED)


@pytest.mark.parametrize("op", ["h", "d", "a"])
def test_plain_fixed_point_wide_range(op):
    """Pole groups whose values span many binades, and groups of zeros next to
    groups of tiny values: every group takes its own scale."""
    levels = (6, 7, 3)
    rng = np.random.default_rng(9)
    u = rng.uniform(-1, 1, inputs.num_points(levels)) * 2.0 ** rng.integers(-40, 40, inputs.num_points(levels))
    u.reshape(9, 129, 65)[:2] *= 1e-300
    u.reshape(9, 129, 65)[2] = 0.0
    ref = ORACLE[op](u, levels)
    got = run(u, levels, op, path=gbh.GBH_PATH_PLAIN, arith=2)
    assert rel_err(got, ref, u, op) <= TOL64


@pytest.mark.parametrize("levels", LEVELS)
@pytest.mark.parametrize("op", ["h", "d", "a"])
@pytest.mark.parametrize("path", [gbh.GBH_PATH_PLAIN, gbh.GBH_PATH_AUTO])
def test_fp32(levels, op, path):
    u32 = inputs.uniform(levels, 300 + len(levels), dtype=np.float32)
    u = u32.astype(np.float64)
    assert rel_err(run(u32, levels, op, dtype=torch.float32, path=path), ORACLE[op](u, levels), u, op) <= TOL32


@pytest.mark.parametrize("levels", [(16,), (15,), (2, 13), (1, 1, 14), (14, 1, 1, 1)])
@pytest.mark.parametrize("op", ["h", "d", "a"])
def test_long_poles(levels, op):
    """Rows longer than the staged-row limit and dimensions with few long
    poles take the per-level kernels."""
    u = inputs.uniform(levels, 7)
    assert np.array_equal(run(u, levels, op, path=gbh.GBH_PATH_PLAIN), ORACLE[op](u, levels))
    assert rel_err(run(u, levels, op), ORACLE[op](u, levels), u, op) <= TOL64


@pytest.mark.parametrize("levels", [(27,), (12,) + (1,) * 9, (1,) * 9 + (12,)])
@pytest.mark.parametrize("op", ["h", "d", "a"])
def test_dim0_heavy_shapes(levels, op):
    """The paper's extreme shapes (Sec. 4): one pole of level 27 (134 M points),
    and ten dimensions with one long dimension and 3 points in every other;
    bit-exact on the plain path, within the tolerance on the default path."""
    u = inputs.uniform(levels, 9)
    ref = ORACLE[op](u, levels)
    assert np.array_equal(run(u, levels, op, path=gbh.GBH_PATH_PLAIN), ref)
    assert rel_err(run(u, levels, op), ref, u, op) <= TOL64


@pytest.mark.parametrize("levels", [(28,), (20,)])
@pytest.mark.parametrize("op", ["h", "d"])
def test_long_pole_split(levels, op):
    """A single long pole splits into dyadic blocks of level max(13, L - 14)
    and their coarse pole (the largest blocks at level 28); the split keeps
    the serial operation order, so the plain path stays bit-exact."""
    u = inputs.uniform(levels, 11)
    ref = ORACLE[op](u, levels)
    assert np.array_equal(run(u, levels, op, path=gbh.GBH_PATH_PLAIN), ref)
    assert rel_err(run(u, levels, op), ref, u, op) <= TOL64


@pytest.mark.parametrize("levels", LEVELS + [(16,), (2, 13), (14, 1, 1, 1), (1, 1, 14), (6,) * 3])
def test_dehierarchize_adjoint(levels):
    """Transpose of the dehierarchization: native on every path, in the serial
    operation order, so fp64 is bit-exact; fp32 within the tolerance."""
    u = inputs.uniform(levels, 13)
    ref = ORACLE["t"](u, levels)
    assert np.array_equal(run(u, levels, "t", path=gbh.GBH_PATH_PLAIN), ref)
    assert np.array_equal(run(u, levels, "t"), ref)
    u32 = u.astype(np.float32).astype(np.float64)
    assert rel_err(run(u32, levels, "t", dtype=torch.float32), ORACLE["t"](u32, levels), u32, "t") <= TOL32


def test_dehierarchize_adjoint_unsupported_paths():
    t = torch.zeros(inputs.num_points((4, 4)), dtype=torch.float64, device="cuda")
    for path in (gbh.GBH_PATH_FUSED, gbh.GBH_PATH_GROUPED):
        with pytest.raises(gbh.GbhError):
            gbh.transform(t, (4, 4), gbh.GBH_DEHIERARCHIZE_ADJOINT, path=path)


def test_headline_workload_full_size():
    """The headline workload at full size in the bench's launch configuration:
    level (9,9,9) (135 M points, fp64), the bench's input recipe, the default
    path.  Hierarchization against the oracle at every point, then the
    dehierarchization of that result against the oracle's, and the round trip."""
    levels, u = inputs.cfg2()
    t = torch.tensor(u, device="cuda")
    gbh.hierarchize(t, levels)
    torch.cuda.synchronize()
    alpha = t.cpu().numpy()
    assert rel_err(alpha, oracle.hierarchize(u, levels), u, "h") <= TOL64
    gbh.dehierarchize(t, levels)
    torch.cuda.synchronize()
    back = t.cpu().numpy()
    assert rel_err(back, oracle.dehierarchize(alpha, levels), alpha, "d") <= TOL64
    assert rel_err(back, u, alpha, "d") <= TOL64


def test_fp32_form_full_size():
    """The fp32 workload at full size: level (6,6,5,5,5), 152 M points, the
    bench's input recipe, default path, against the oracle on the fp32 input."""
    levels, u = inputs.cfg3()
    u32 = u.astype(np.float32)
    ref_in = u32.astype(np.float64)
    t = torch.tensor(u32, device="cuda")
    gbh.hierarchize(t, levels)
    torch.cuda.synchronize()
    assert rel_err(t.cpu().double().numpy(), oracle.hierarchize(ref_in, levels), ref_in, "h") <= TOL32


@pytest.mark.parametrize("op", ["h", "d", "a", "t"])
def test_same_shape_batch(op):
    levels, B = (4, 3, 5), 5
    n = inputs.num_points(levels)
    u = np.random.default_rng(3).uniform(-1, 1, (B, n))
    got = run(u.reshape(-1), levels, op, batch=B).reshape(B, n)
    for b in range(B):
        assert rel_err(got[b], ORACLE[op](u[b], levels), u[b], op) <= TOL64


def test_degenerate_level_zero():
    """All-boundary grids (every level 0) are unchanged by every op."""
    levels = (0, 0, 0)
    u = inputs.uniform(levels, 1)
    for op in "hda":
        assert np.array_equal(run(u, levels, op), u)
