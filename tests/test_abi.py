"""C ABI: the library builds, loads and exports every symbol include/gbh.h
declares; host-only entry points and argument validation (no kernel is
launched here, so these run without a GPU)."""
import ctypes

import pytest

import paper_1309_0392_gb300 as gbh
from paper_1309_0392_gb300 import _lib, build


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.lib()


def test_exports_every_declared_symbol(L):
    syms = _lib.header_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(L, s), s
    # and every declared symbol has a ctypes signature in the binding
    assert set(syms) == set(_lib._SIGS)


def test_version_and_status_strings(L):
    assert L.gbh_version() >= 100
    assert L.gbh_status_string(0) == b"ok"
    for code in range(-8, 0):
        assert L.gbh_status_string(code) != b"unknown status"


def test_num_points(L):
    assert gbh.num_points((9, 9, 9)) == 513 ** 3
    assert gbh.num_points((0,)) == 2
    assert gbh.num_points((6, 6, 5, 5, 5)) == 65 * 65 * 33 ** 3
    out = ctypes.c_int64(0)
    assert L.gbh_num_points(0, _lib.levels_arg([1]), ctypes.byref(out)) == -1       # d < 1
    assert L.gbh_num_points(17, _lib.levels_arg([1] * 17), ctypes.byref(out)) == -1  # d > 16
    assert L.gbh_num_points(1, _lib.levels_arg([31]), ctypes.byref(out)) == -4      # level > 30
    assert L.gbh_num_points(1, _lib.levels_arg([-1]), ctypes.byref(out)) == -4
    # 16 dims of level 30: the point count overflows int64
    assert L.gbh_num_points(16, _lib.levels_arg([30] * 16), ctypes.byref(out)) == -4


def test_argument_errors_launch_nothing(L):
    lv = _lib.levels_arg([2, 2])
    before = _lib.launch_count()
    fake = ctypes.c_void_p(0x1000)                 # never dereferenced: calls fail validation
    assert L.gbh_hierarchize(None, 2, lv, 1, None) == -1                       # null data
    assert L.gbh_hierarchize(fake, 2, lv, 7, None) == -2                       # dtype
    assert L.gbh_hierarchize(ctypes.c_void_p(0x1004), 2, lv, 1, None) == -3    # fp64 alignment
    assert L.gbh_hierarchize(fake, 0, lv, 1, None) == -1                       # d
    assert L.gbh_hierarchize(fake, 1, _lib.levels_arg([40]), 1, None) == -4    # level
    assert L.gbh_transform(fake, 2, lv, 1, 9, None, None) == -1                # op
    opt = _lib.Options()
    opt.path = 7
    assert L.gbh_transform(fake, 2, lv, 1, 0, ctypes.byref(opt), None) == -1   # path
    assert L.gbh_transform_batched(fake, 0, 2, lv, 1, 0, None, None) == -1     # batch
    # the transpose of the dehierarchization runs on the per-dimension path only
    for path in (2, 3):                                                        # fused, grouped
        opt.path = path
        assert L.gbh_transform(fake, 2, lv, 1, 3, ctypes.byref(opt), None) == -8
    # scheme plans: invalid arguments and owned-grid lists fail before any
    # device allocation
    h = ctypes.c_void_p()
    assert L.gbh_plan_create_scheme(0, 4, 1, ctypes.byref(h)) == -1
    assert L.gbh_plan_create_scheme(3, 4, 7, ctypes.byref(h)) == -2
    for owned in ([], [3, 1], [0, 0], [-1], [10 ** 6]):
        arr = _lib.levels_arg(owned) if owned else None
        assert L.gbh_plan_create_scheme_subset(3, 4, 1, len(owned), arr, ctypes.byref(h)) == -1
    assert not h.value
    assert L.gbh_plan_scatter(None, fake, 0, None) == -1
    assert L.gbh_plan_gather(None, fake, None) == -1
    assert _lib.launch_count() == before


def test_python_layer_rejects_host_tensors():
    torch = pytest.importorskip("torch")
    t = torch.zeros(25, dtype=torch.float64)
    with pytest.raises(ValueError):
        gbh.hierarchize(t, (2, 2))


@pytest.mark.parametrize("d,n", [(1, 6), (2, 5), (3, 4), (4, 4), (5, 3), (8, 2)])
def test_sparse_index_of_grid_matches_oracle(L, d, n):
    """The library's subspace ranking (the index the scatter kernel uses) gives
    the oracle's sparse-grid position for every point of every grid."""
    import numpy as np
    import oracle
    lv, _ = oracle.scheme(d, n)
    seen = np.zeros(oracle.sparse_num_points(d, n), dtype=bool)
    for l in lv:
        got = gbh.sparse_index_of_grid(d, n, l)
        assert np.array_equal(got, oracle.sparse_index_of_grid(d, n, l))
        seen[got] = True
    assert seen.all()          # the scheme covers the sparse grid
    # a grid inside the sparse grid that is not in the scheme
    small = [1] * d
    assert np.array_equal(gbh.sparse_index_of_grid(d, n, small), oracle.sparse_index_of_grid(d, n, small))


def test_sparse_index_of_grid_full_scheme_sampled(L):
    """The 4-d level-14 scheme (1665 grids): sampled grids, bit-exact."""
    import numpy as np
    import oracle
    lv, _ = oracle.scheme(4, 14)
    rng = np.random.default_rng(3)
    for g in sorted(set(int(v) for v in rng.choice(len(lv), 6, replace=False)) | {0, len(lv) - 1}):
        assert np.array_equal(gbh.sparse_index_of_grid(4, 14, lv[g]), oracle.sparse_index_of_grid(4, 14, lv[g]))


def test_sparse_index_of_grid_rejects_grids_outside(L):
    out = (ctypes.c_int64 * 64)()
    assert L.gbh_sparse_index_of_grid(2, 3, _lib.levels_arg([4, 1]), out) == -4   # level above n
    assert L.gbh_sparse_index_of_grid(2, 3, _lib.levels_arg([3, 2]), out) == -4   # |l| too large
    assert L.gbh_sparse_index_of_grid(0, 3, _lib.levels_arg([1]), out) == -1
    assert L.gbh_sparse_index_of_grid(9, 3, _lib.levels_arg([1] * 9), out) == -1
    assert L.gbh_sparse_index_of_grid(2, 0, _lib.levels_arg([0, 0]), out) == -1
