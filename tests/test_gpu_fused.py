"""GPU parity of the fused dyadic-tile path (all dimensions per tile, in place)
against the CPU oracle: every class schedule the planner can build -- block,
lattice and point dimensions -- for hierarchization and its inverse, in fp64
(int64 fixed point and native) and fp32."""
import numpy as np
import pytest

import oracle
from golden_io import load
from parity import TOL32, TOL64, rel_err
from paper_1309_0392_gb300 import inputs

torch = pytest.importorskip("torch")
gbh = pytest.importorskip("paper_1309_0392_gb300")

pytestmark = pytest.mark.gpu

OPS = {"h": gbh.GBH_HIERARCHIZE, "d": gbh.GBH_DEHIERARCHIZE}
ORACLE = {"h": oracle.hierarchize, "d": oracle.dehierarchize}
FIX, NAT = gbh.GBH_ARITH_FIXED, gbh.GBH_ARITH_NATIVE


def run(u, levels, op, dtype=torch.float64, **kw):
    t = torch.tensor(u, dtype=dtype, device="cuda")
    gbh.transform(t, levels, OPS[op], path=gbh.GBH_PATH_FUSED, **kw)
    torch.cuda.synchronize()
    return t.cpu().double().numpy()


# (levels, tile exponents); None = the planner's choice
CASES = [
    ((5, 5), (2, 3)), ((5, 5), (5, 5)), ((5, 5), (1, 1)), ((6, 4), (3, 2)), ((3, 7), (3, 2)),
    ((9, 9), (2, 2)),                      # long lattices: point dimensions
    ((4, 4, 4), (2, 2, 2)), ((5, 4, 3), (3, 1, 2)), ((6, 5, 4), None), ((7, 6, 5), (5, 4, 3)),
    ((2, 0, 3), (1, 0, 2)), ((0, 4, 4), (0, 2, 2)), ((1, 1, 1), (1, 1, 1)),
    ((3, 3, 2, 2), (2, 2, 1, 1)), ((4, 3, 3, 2), None), ((5, 4, 4, 4), None),
    ((2, 2, 2, 2, 2), (1, 1, 1, 1, 1)), ((3, 3, 2, 2, 2), None), ((2, 2, 2, 2, 2, 2), None),
    ((8, 8, 8), None), ((9, 5, 5), None),
]


@pytest.mark.parametrize("levels,tile", CASES)
@pytest.mark.parametrize("op", ["h", "d"])
def test_fused_fp64_fixed(levels, tile, op):
    u = inputs.uniform(levels, 11 + sum(levels))
    got = run(u, levels, op, tile=tile, arith=FIX)
    assert rel_err(got, ORACLE[op](u, levels), u, op) <= TOL64


@pytest.mark.parametrize("levels,tile", CASES)
@pytest.mark.parametrize("op", ["h", "d"])
def test_fused_fp64_native(levels, tile, op):
    u = inputs.uniform(levels, 13 + sum(levels))
    got = run(u, levels, op, tile=tile, arith=NAT)
    assert rel_err(got, ORACLE[op](u, levels), u, op) <= TOL64


@pytest.mark.parametrize("levels,tile", CASES)
@pytest.mark.parametrize("op", ["h", "d"])
def test_fused_fp32(levels, tile, op):
    if tile is not None and max(tile) > 6:
        pytest.skip("fp32 tiles go to 2^6+1")
    u32 = inputs.uniform(levels, 17 + sum(levels), dtype=np.float32)
    u = u32.astype(np.float64)
    got = run(u32, levels, op, dtype=torch.float32, tile=tile)
    assert rel_err(got, ORACLE[op](u, levels), u, op) <= TOL32


@pytest.mark.parametrize("levels,tile", [((5, 5), (2, 3)), ((4, 4, 4), (2, 2, 2)), ((6, 5, 4), None)])
def test_fused_round_trip(levels, tile):
    u = inputs.uniform(levels, 5)
    t = torch.tensor(u, device="cuda")
    for _ in range(3):
        gbh.transform(t, levels, gbh.GBH_HIERARCHIZE, path=gbh.GBH_PATH_FUSED, tile=tile)
        gbh.transform(t, levels, gbh.GBH_DEHIERARCHIZE, path=gbh.GBH_PATH_FUSED, tile=tile)
    torch.cuda.synchronize()
    assert np.abs(t.cpu().numpy() - u).max() <= 1e-13


def test_fused_closed_form_bit_exact():
    """x^2 + 3xy: dyadic inputs, the fixed-point path is exact."""
    levels, u = inputs.cfg1b()
    for tile in [(2, 3), (5, 5), (3, 1), (1, 1)]:
        assert np.array_equal(run(u, levels, "h", tile=tile, arith=FIX), load("cfg1b_hierarchize.txt"))


def test_fused_wide_dynamic_range():
    """Values spanning many binades inside one tile: the fixed-point error
    stays within the tolerance relative to max|u|."""
    levels = (6, 5, 4)
    rng = np.random.default_rng(8)
    u = rng.uniform(-1, 1, inputs.num_points(levels)) * 10.0 ** rng.integers(-12, 3, inputs.num_points(levels))
    for op in "hd":
        got = run(u, levels, op)
        assert rel_err(got, ORACLE[op](u, levels), u, op) <= TOL64


def test_fused_zero_and_tiny_tiles():
    """Tiles of zeros next to tiles whose values are all near 1e-300 (normal
    numbers far below the fast conversion's range): the tiny tiles keep the
    full relative accuracy, measured against the tiny values themselves."""
    levels = (5, 4, 4)
    rng = np.random.default_rng(21)
    u = np.zeros(inputs.num_points(levels))
    u[:100] = 1e-300
    u[200:300] = rng.uniform(-1, 1, 100) * 1e-300
    for op in "hd":
        ref = ORACLE[op](u, levels)
        got = run(u, levels, op)
        assert np.abs(ref).max() > 0.0
        assert rel_err(got, ref, u, op) <= TOL64


@pytest.mark.parametrize("op", ["h", "d"])
def test_fused_same_shape_batch(op):
    levels, B = (5, 4, 4), 3
    n = inputs.num_points(levels)
    u = np.random.default_rng(4).uniform(-1, 1, (B, n))
    t = torch.tensor(u.reshape(-1), device="cuda")
    gbh.transform(t, levels, OPS[op], path=gbh.GBH_PATH_FUSED, batch=B)
    got = t.cpu().numpy().reshape(B, n)
    for b in range(B):
        assert rel_err(got[b], ORACLE[op](u[b], levels), u[b], op) <= TOL64


def test_planner_choice_is_used_by_default():
    from paper_1309_0392_gb300 import _lib
    assert _lib.tile_plan((9, 9, 9), 1, 0) == (5, 4, 4)
