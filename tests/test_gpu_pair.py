"""GPU parity of the plain path's pair kernel (two consecutive dimensions per
pass, native arithmetic) against the CPU oracle and against one pass per
dimension (variant 1), which it must match bit for bit: both apply the same
operations to every point in the same order.  Shapes cover planes of
dimensions (0, 1) with a ragged last CTA, bundles of positions below an
outer pair with a ragged last bundle (down to one position), pairs next to
dimensions that do not pair (a level above the register pole, a level 0),
batches, and grid pointers off a 16-byte boundary (the plane copies switch
between single elements and 16-byte pieces)."""
import numpy as np
import pytest

import oracle
from parity import TOL32, rel_err
from paper_1309_0392_gb300 import inputs

torch = pytest.importorskip("torch")
gbh = pytest.importorskip("paper_1309_0392_gb300")

pytestmark = pytest.mark.gpu

OPS = {"h": gbh.GBH_HIERARCHIZE, "d": gbh.GBH_DEHIERARCHIZE, "a": gbh.GBH_ADJOINT,
       "t": gbh.GBH_DEHIERARCHIZE_ADJOINT}
ORACLE = {"h": oracle.hierarchize, "d": oracle.dehierarchize, "a": oracle.hierarchize_adjoint,
          "t": oracle.dehierarchize_adjoint}
DT = {"f32": (np.float32, torch.float32), "f64": (np.float64, torch.float64)}

# (levels, pairs taken in fp32, pairs taken in fp64)
SHAPES = [
    ((6, 6), 1, 0),             # fp32: planes of 65 x 65; fp64: level 6 is above its register pole
    ((3, 4), 1, 1),             # many small planes per CTA
    ((5, 5, 5, 5), 2, 2),       # planes, then bundles over 1089 positions (ragged last bundle)
    ((1, 1, 1, 1, 1, 1), 3, 3), # bundles over 9 positions: the second holds one
    ((2, 6, 6), 1, 0),
    ((4, 2, 6, 5, 1), 2, 2),    # (0,1); dimension 2 alone (its pair tile is too large); (3,4)
    ((7, 3, 3), 1, 1),          # level 7 alone, pair (1,2) over 129 positions
    ((0, 5, 5), 0, 0),          # a dimension of one point: nothing below the pair to bundle
    ((5, 0, 5), 0, 0),
    ((2, 3, 2, 3, 2, 3), 3, 3),
    ((1, 1, 4, 4, 4, 4), 3, 3),   # more tiles than resident CTAs: CTAs take two or more in turn
]


def run(u, levels, op, dt, variant=0, offset=0, batch=None):
    npt, tt = DT[dt]
    buf = torch.zeros(u.size + offset, dtype=tt, device="cuda")
    t = buf[offset:]
    t.copy_(torch.from_numpy(np.ascontiguousarray(u, dtype=npt).reshape(-1)))
    gbh.transform(t, levels, OPS[op], path=gbh.GBH_PATH_PLAIN, variant=variant, batch=batch)
    torch.cuda.synchronize()
    return t.cpu().numpy()


def check_oracle(got, u, levels, op, dt):
    ref = ORACLE[op](u.astype(np.float64), levels)
    if dt == "f64" and op != "t":
        # native fp64 in the serial operation order: bit-identical
        assert np.array_equal(got, ref)
    elif dt == "f64":
        assert rel_err(got, ref, u, op) <= 1e-13
    else:
        assert rel_err(got.astype(np.float64), ref, u.astype(np.float64), op) <= TOL32


@pytest.mark.parametrize("levels,p32,p64", SHAPES)
@pytest.mark.parametrize("op", ["h", "d", "a", "t"])
@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_pair_against_oracle_and_single_passes(levels, p32, p64, op, dt):
    u = inputs.uniform(levels, 500 + sum(levels), dtype=DT[dt][0])
    got = run(u, levels, op, dt)
    check_oracle(got, u, levels, op, dt)
    assert np.array_equal(got, run(u, levels, op, dt, variant=1))


@pytest.mark.parametrize("offset", [1, 2, 3])
@pytest.mark.parametrize("op", ["h", "d"])
def test_pair_unaligned_fp32(offset, op):
    levels = (5, 4, 3)
    u = inputs.uniform(levels, 510 + offset, dtype=np.float32)
    got = run(u, levels, op, "f32", offset=offset)
    check_oracle(got, u, levels, op, "f32")
    assert np.array_equal(got, run(u, levels, op, "f32", variant=1, offset=offset))


@pytest.mark.parametrize("op", ["h", "d", "a"])
def test_pair_unaligned_fp64(op):
    levels = (4, 5, 2, 2)
    u = inputs.uniform(levels, 520, dtype=np.float64)
    check_oracle(run(u, levels, op, "f64", offset=1), u, levels, op, "f64")


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("op", ["h", "d"])
def test_pair_batch(dt, op):
    """Three grids of an odd point count back to back: planes and bundles
    run across the grid boundaries."""
    levels, B = (3, 2, 4, 3), 3
    n = inputs.num_points(levels)
    u = np.random.default_rng(530).uniform(-1, 1, (B, n)).astype(DT[dt][0])
    got = run(u, levels, op, dt, batch=B).reshape(B, n)
    for b in range(B):
        check_oracle(got[b], u[b], levels, op, dt)
    assert np.array_equal(got.reshape(-1), run(u, levels, op, dt, variant=1, batch=B))


@pytest.mark.parametrize("levels,p32,p64", SHAPES)
@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_pair_launches(levels, p32, p64, dt):
    """One pair launch per pair the host logic takes; variant 1 takes none."""
    from paper_1309_0392_gb300 import _lib
    u = inputs.uniform(levels, 540, dtype=DT[dt][0])
    for variant, want in ((0, p32 if dt == "f32" else p64), (1, 0)):
        _lib.profile_enable(True)
        _lib.profile_reset()
        run(u, levels, "h", dt, variant=variant)
        names = _lib.profile_read()
        _lib.profile_enable(False)
        got = sum(names.get(k, (0,))[0] for k in ("plain_pair_planes", "plain_pair_bundles", "plain_pair_square"))
        assert got == want
