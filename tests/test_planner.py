"""Host-side tile planner (no GPU): the fused path's tile choices respect the
register-pole and shared-memory limits, and decline shapes it cannot tile."""
import pytest

from paper_1309_0392_gb300 import _lib, build


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


@pytest.mark.parametrize("levels", [(9, 9, 9), (8, 8, 8), (6, 6, 5, 5, 5), (5, 4, 4, 4), (7, 7),
                                    (4, 4, 4, 5), (2, 2, 2, 2, 2, 2), (9, 5, 5)])
@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("op", [0, 1])
def test_tiles_respect_limits(levels, dtype, op):
    m = _lib.tile_plan(levels, dtype, op)
    assert m is not None
    maxlev = 5 if dtype == 1 else 6
    es = 8 if dtype == 1 else 4
    vol = 1
    for l, mk in zip(levels, m):
        assert 0 <= mk <= l and mk <= maxlev
        if l >= 1:
            assert mk >= 1 and l - mk <= maxlev
        vol *= 2 ** mk + 1
    assert vol * es <= 100 * 1024


@pytest.mark.parametrize("levels", [(16,), (12,), (14, 1, 1, 1), (1, 1, 1, 14), (1,) * 7])
def test_planner_declines(levels):
    assert _lib.tile_plan(levels, 1, 0) is None


def test_headline_tiles():
    assert _lib.tile_plan((9, 9, 9), 1, 0) == (5, 4, 4)
