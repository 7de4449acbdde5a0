"""Guard words around device buffers: every path and operation writes only
inside its grid (and a plan only inside its grids and its sparse vector).
The grid is a view into a larger buffer whose first and last GUARD elements
hold a sentinel; after the call they must be unchanged.

Kept in a file that pytest collects last, after the parity tests."""
import numpy as np
import pytest

import oracle
from paper_1309_0392_gb300 import inputs

torch = pytest.importorskip("torch")
gbh = pytest.importorskip("paper_1309_0392_gb300")

pytestmark = pytest.mark.gpu

GUARD = 128                 # elements on each side (keeps 16-byte alignment)
SENTINEL = -7.25            # exact in fp32 and fp64

OPS = {"h": gbh.GBH_HIERARCHIZE, "d": gbh.GBH_DEHIERARCHIZE, "a": gbh.GBH_ADJOINT,
       "t": gbh.GBH_DEHIERARCHIZE_ADJOINT}


def guarded(values, dtype):
    """(buffer, view): the view holds `values`, the guards the sentinel."""
    n = values.size
    buf = torch.full((n + 2 * GUARD,), SENTINEL, dtype=dtype, device="cuda")
    view = buf[GUARD:GUARD + n]
    view.copy_(torch.as_tensor(values, dtype=dtype))
    return buf, view


def guards_intact(buf):
    torch.cuda.synchronize()
    ref = torch.full((GUARD,), SENTINEL, dtype=buf.dtype, device="cuda")
    return torch.equal(buf[:GUARD], ref) and torch.equal(buf[-GUARD:], ref)


SHAPES = [(1,), (7,), (16,), (20,), (2, 13), (5, 4, 4), (6, 5, 4), (9, 9, 8), (3, 3, 2, 2, 2),
          (14, 1, 1, 1), (1, 1, 14), (0, 3, 1)]


@pytest.mark.parametrize("levels", SHAPES)
@pytest.mark.parametrize("op", ["h", "d", "a", "t"])
@pytest.mark.parametrize("path", [gbh.GBH_PATH_AUTO, gbh.GBH_PATH_PLAIN])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_single_grid_writes_stay_inside(levels, op, path, dtype):
    u = inputs.uniform(levels, 21)
    buf, view = guarded(u, dtype)
    gbh.transform(view, levels, OPS[op], path=path)
    assert guards_intact(buf)


@pytest.mark.parametrize("levels", [(5, 4, 4), (9, 9, 8)])
def test_batched_single_shape_writes_stay_inside(levels):
    B = 3
    u = np.random.default_rng(22).uniform(-1, 1, B * inputs.num_points(levels))
    buf, view = guarded(u, torch.float64)
    gbh.transform(view, levels, gbh.GBH_HIERARCHIZE, batch=B)
    gbh.transform(view, levels, gbh.GBH_DEHIERARCHIZE, batch=B)
    assert guards_intact(buf)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_plan_writes_stay_inside(dtype):
    d, n = 3, 6
    plan = gbh.Plan.scheme(d, n, dtype=str(dtype))
    lv = plan.levels()
    pairs = [guarded(inputs.scheme_grid(l, 1000 + g), dtype) for g, l in enumerate(lv)]
    plan.bind([v for _, v in pairs])
    sbuf, sparse = guarded(np.zeros(plan.sparse_points), torch.float64)
    plan.execute(gbh.GBH_HIERARCHIZE)
    plan.gather(sparse)
    plan.scatter(sparse)
    plan.scatter(sparse, scaled=True)
    plan.execute(gbh.GBH_DEHIERARCHIZE)
    assert plan.status() == 0
    assert all(guards_intact(b) for b, _ in pairs)
    assert guards_intact(sbuf)
