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
    assert _lib.launch_count() == before


def test_python_layer_rejects_host_tensors():
    torch = pytest.importorskip("torch")
    t = torch.zeros(25, dtype=torch.float64)
    with pytest.raises(ValueError):
        gbh.hierarchize(t, (2, 2))
