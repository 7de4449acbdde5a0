"""GPU parity of the 3-D fp64 fixed-point kernels of the fused path with tile
exponents (5,4,4) against the CPU oracle: the interior class on its own
kernel (interior3.cu, the default) and the generic tile kernel for every
class, over shapes with one to 512 tiles per plane, batches, a grid pointer
that is not 16-byte aligned, and closures outside the fast exponent range."""
import numpy as np
import pytest

import oracle
from parity import TOL64, rel_err
from paper_1309_0392_gb300 import inputs

torch = pytest.importorskip("torch")
gbh = pytest.importorskip("paper_1309_0392_gb300")

pytestmark = pytest.mark.gpu

OPS = {"h": gbh.GBH_HIERARCHIZE, "d": gbh.GBH_DEHIERARCHIZE}
ORACLE = {"h": oracle.hierarchize, "d": oracle.dehierarchize}
TILE = (5, 4, 4)
SHAPES = [(5, 4, 4), (6, 4, 4), (6, 5, 4), (7, 4, 5), (8, 5, 5), (9, 4, 4), (9, 5, 6), (6, 6, 6), (7, 8, 8), (6, 8, 9)]


def run(u, levels, op, variant=0, batch=None, offset=0):
    buf = torch.zeros(u.size + offset, dtype=torch.float64, device="cuda")
    t = buf[offset:]
    t.copy_(torch.from_numpy(np.ascontiguousarray(u).reshape(-1)))
    gbh.transform(t, levels, OPS[op], path=gbh.GBH_PATH_FUSED, tile=TILE, variant=variant, batch=batch)
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("levels", SHAPES)
@pytest.mark.parametrize("op", ["h", "d"])
@pytest.mark.parametrize("variant", [0, 1])
def test_interior_against_oracle(levels, op, variant):
    u = inputs.uniform(levels, 41 + sum(levels))
    assert rel_err(run(u, levels, op, variant), ORACLE[op](u, levels), u, op) <= TOL64


@pytest.mark.parametrize("op", ["h", "d"])
@pytest.mark.parametrize("variant", [0, 1])
def test_interior_unaligned_grid_pointer(op, variant):
    """The grid starts 8 bytes past a 16-byte boundary: every row's copies
    swap between the single element and the pairs."""
    levels = (7, 5, 4)
    u = inputs.uniform(levels, 43)
    assert rel_err(run(u, levels, op, variant=variant, offset=1), ORACLE[op](u, levels), u, op) <= TOL64


@pytest.mark.parametrize("op", ["h", "d"])
@pytest.mark.parametrize("variant", [0, 1])
def test_interior_batch(op, variant):
    """Three grids back to back (odd grid size: the second grid starts at the
    other parity)."""
    levels, B = (6, 5, 5), 3
    n = inputs.num_points(levels)
    u = np.random.default_rng(44).uniform(-1, 1, (B, n))
    got = run(u, levels, op, variant=variant, batch=B).reshape(B, n)
    for b in range(B):
        assert rel_err(got[b], ORACLE[op](u[b], levels), u[b], op) <= TOL64


@pytest.mark.parametrize("op", ["h", "d"])
@pytest.mark.parametrize("variant", [0, 1])
def test_interior_exponent_extremes(op, variant):
    """Tiles of zeros, of values near 1e-300 and near 1e300 next to ordinary
    ones: the slow conversions keep the accuracy relative to each closure's
    own magnitude."""
    levels = (6, 5, 5)
    n = [(1 << l) + 1 for l in levels]
    rng = np.random.default_rng(45)
    u = rng.uniform(-1, 1, (n[2], n[1], n[0]))
    u[:17, :17, :] = 0.0                                    # tiles (*, 0, 0) and their faces
    u[16:, :17, :] *= 1e-300                                # tiles (*, 0, 1)
    u[:17, 16:, :] *= 1e300                                 # tiles (*, 1, 0)
    u = u.reshape(-1)
    got = run(u, levels, op, variant=variant).reshape(n[2], n[1], n[0])
    ref = ORACLE[op](u, levels).reshape(n[2], n[1], n[0])
    u3 = u.reshape(n[2], n[1], n[0])
    for b2 in range(2):
        for b1 in range(2):
            # the tiles' interior points along dimensions 1 and 2, and their
            # closures (faces shared with the neighbouring tiles), whose
            # largest magnitude sets the scale
            pts = np.s_[16 * b2 + 1:16 * b2 + 16, 16 * b1 + 1:16 * b1 + 16, :]
            clo = np.s_[16 * b2:16 * b2 + 17, 16 * b1:16 * b1 + 17, :]
            scale = max(np.abs(u3[clo]).max(), np.abs(ref[clo]).max())
            if scale == 0.0:
                assert np.abs(got[pts]).max() == 0.0
            else:
                assert np.abs(got[pts] - ref[pts]).max() / scale <= TOL64


@pytest.mark.parametrize("variant", [0, 1])
def test_interior_round_trip(variant):
    levels = (9, 5, 5)
    u = inputs.uniform(levels, 46)
    t = torch.tensor(u, device="cuda")
    for _ in range(3):
        gbh.transform(t, levels, gbh.GBH_HIERARCHIZE, path=gbh.GBH_PATH_FUSED, tile=TILE, variant=variant)
        gbh.transform(t, levels, gbh.GBH_DEHIERARCHIZE, path=gbh.GBH_PATH_FUSED, tile=TILE, variant=variant)
    torch.cuda.synchronize()
    assert np.abs(t.cpu().numpy() - u).max() / np.abs(u).max() <= 1e-13


@pytest.mark.parametrize("variant,name", [(0, "fused_class0"), (1, "fused_class0")])
def test_variant_launches(variant, name):
    """Both variants report the interior class as one launch; the default
    runs the interior3 kernel (fewer instructions per point), variant 1 the
    generic tile kernel."""
    from paper_1309_0392_gb300 import _lib
    levels = (8, 6, 6)
    t = torch.tensor(inputs.uniform(levels, 47), device="cuda")
    _lib.profile_enable(True)
    _lib.profile_reset()
    n0 = _lib.launch_count()
    gbh.transform(t, levels, gbh.GBH_HIERARCHIZE, path=gbh.GBH_PATH_FUSED, tile=TILE, variant=variant)
    torch.cuda.synchronize()
    names = _lib.profile_read()
    _lib.profile_enable(False)
    assert names[name][0] == 1
    assert _lib.launch_count() > n0
