"""ctypes declarations of the C ABI in include/gbh.h (libgbh.so).

Argument marshalling only: every transform runs in the library's CUDA kernels.
The library is built in-tree (``paper_1309_0392_gb300/libgbh.so``); loading
fails loudly when it is missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libgbh.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "gbh.h")

GBH_F32, GBH_F64 = 0, 1
GBH_HIERARCHIZE, GBH_DEHIERARCHIZE, GBH_ADJOINT, GBH_DEHIERARCHIZE_ADJOINT = 0, 1, 2, 3
GBH_PATH_AUTO, GBH_PATH_PLAIN, GBH_PATH_FUSED, GBH_PATH_GROUPED = 0, 1, 2, 3
GBH_ARITH_AUTO, GBH_ARITH_NATIVE, GBH_ARITH_FIXED = 0, 1, 2

STATUS = {0: "GBH_OK", -1: "GBH_EINVAL", -2: "GBH_EDTYPE", -3: "GBH_EALIGN", -4: "GBH_ERANGE",
          -5: "GBH_ECUDA", -6: "GBH_ETIMEOUT", -7: "GBH_ENOMEM", -8: "GBH_EUNSUPPORTED"}


class GbhError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)} ({status})")


class TuneResult(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("tile_exp", ctypes.c_int32 * 16), ("candidates", ctypes.c_int32),
                ("ms_tuned", ctypes.c_double), ("ms_model", ctypes.c_double), ("model_path", ctypes.c_int32),
                ("model_tile_exp", ctypes.c_int32 * 16), ("reserved", ctypes.c_int32 * 4)]


class PlanTuneResult(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("wave_mb", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("max_ctas_per_sm", ctypes.c_int32), ("ms_tuned", ctypes.c_double), ("ms_model", ctypes.c_double),
                ("reserved", ctypes.c_int32 * 4)]


class Options(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("tile_exp", ctypes.c_int32 * 16),
                ("arith", ctypes.c_int32), ("variant", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


_I32P = ctypes.POINTER(ctypes.c_int32)
_VP = ctypes.c_void_p

_SIGS = {
    "gbh_hierarchize": (ctypes.c_int, [_VP, ctypes.c_int, _I32P, ctypes.c_int, _VP]),
    "gbh_dehierarchize": (ctypes.c_int, [_VP, ctypes.c_int, _I32P, ctypes.c_int, _VP]),
    "gbh_hierarchize_adjoint": (ctypes.c_int, [_VP, ctypes.c_int, _I32P, ctypes.c_int, _VP]),
    "gbh_dehierarchize_adjoint": (ctypes.c_int, [_VP, ctypes.c_int, _I32P, ctypes.c_int, _VP]),
    "gbh_transform": (ctypes.c_int, [_VP, ctypes.c_int, _I32P, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(Options), _VP]),
    "gbh_transform_batched": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int, _I32P, ctypes.c_int,
                                             ctypes.c_int, ctypes.POINTER(Options), _VP]),
    "gbh_num_points": (ctypes.c_int, [ctypes.c_int, _I32P, ctypes.POINTER(ctypes.c_int64)]),
    "gbh_tile_plan": (ctypes.c_int, [ctypes.c_int, _I32P, ctypes.c_int, ctypes.c_int, _I32P]),
    "gbh_plan_create_scheme": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(_VP)]),
    "gbh_plan_create_scheme_subset": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                     _I32P, ctypes.POINTER(_VP)]),
    "gbh_plan_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _I32P, ctypes.c_int,
                                       ctypes.POINTER(_VP)]),
    "gbh_plan_destroy": (ctypes.c_int, [_VP]),
    "gbh_plan_num_grids": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "gbh_plan_grid_levels": (ctypes.c_int, [_VP, ctypes.c_int, _I32P]),
    "gbh_plan_coeffs": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "gbh_plan_set_coeffs": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "gbh_plan_sparse_points": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    "gbh_plan_total_points": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    "gbh_plan_bind": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), _VP]),
    "gbh_plan_execute": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "gbh_plan_gather": (ctypes.c_int, [_VP, _VP, _VP]),
    "gbh_plan_scatter": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP]),
    "gbh_sparse_index_of_grid": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _I32P,
                                                ctypes.POINTER(ctypes.c_int64)]),
    "gbh_plan_status": (ctypes.c_int, [_VP, _VP]),
    "gbh_plan_set_params": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "gbh_plan_get_params": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]),
    "gbh_plan_autotune": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.POINTER(PlanTuneResult)]),
    "gbh_autotune": (ctypes.c_int, [ctypes.c_int, _I32P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(TuneResult)]),
    "gbh_autotune_reset": (ctypes.c_int, []),
    "gbh_tile_candidates": (ctypes.c_int, [ctypes.c_int, _I32P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _I32P,
                                           ctypes.POINTER(ctypes.c_int)]),
    "gbh_plan_test_stall": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_longlong]),
    "gbh_batched_transform_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _I32P, ctypes.POINTER(_VP),
                                                     ctypes.c_int, ctypes.c_int, _VP]),
    "gbh_batched_transform_noalloc_status": (ctypes.c_int, [_VP]),
    "gbh_batched_transform_noalloc_test_stall": (ctypes.c_int, [ctypes.c_int, ctypes.c_longlong]),
    "gbh_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gbh_launch_count": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64)]),
    "gbh_version": (ctypes.c_int, []),
    "gbh_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "gbh_profile_read": (ctypes.c_int, [ctypes.c_int, ctypes.c_char_p, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]),
    "gbh_profile_reset": (ctypes.c_int, []),
}

_lock = threading.Lock()
_lib = None


def header_symbols():
    """Function names declared in include/gbh.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gbh_[a-z0-9_]+)\s*\(", text)))


def lib():
    """The loaded library (raises if libgbh.so was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with "
                                  "`python -m paper_1309_0392_gb300.build` (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(status: int, what: str):
    if status != 0:
        raise GbhError(status, what)


def levels_arg(levels):
    arr = (ctypes.c_int32 * len(levels))(*[int(v) for v in levels])
    return arr


def launch_count() -> int:
    v = ctypes.c_uint64(0)
    check(lib().gbh_launch_count(ctypes.byref(v)), "gbh_launch_count")
    return int(v.value)


def profile_enable(on: bool = True):
    check(lib().gbh_profile_enable(1 if on else 0), "gbh_profile_enable")


def profile_reset():
    check(lib().gbh_profile_reset(), "gbh_profile_reset")


def profile_read():
    """{kernel name: (launches, total_ms, total_algorithmic_bytes)} of the
    library's timed launches."""
    out = {}
    i = 0
    buf = ctypes.create_string_buffer(128)
    while True:
        n, ms, by = ctypes.c_uint64(0), ctypes.c_double(0.0), ctypes.c_double(0.0)
        st = lib().gbh_profile_read(i, buf, 128, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by))
        if st != 0:
            break
        out[buf.value.decode()] = (int(n.value), float(ms.value), float(by.value))
        i += 1
    return out


def sparse_index_of_grid(d: int, n: int, levels):
    """Sparse-grid position of every point of grid `levels` in the scheme
    (d, n) (int64 numpy array, flat grid order).  Host only."""
    import numpy as np
    lv = [int(v) for v in levels]
    if len(lv) != d:
        raise ValueError("one level per dimension")
    N = 1
    for v in lv:
        N *= (1 << v) + 1
    out = np.empty(N, dtype=np.int64)
    check(lib().gbh_sparse_index_of_grid(d, n, levels_arg(lv),
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
          "gbh_sparse_index_of_grid")
    return out


def tile_plan(levels, dtype_code=GBH_F64, op=GBH_HIERARCHIZE):
    """Tile exponents the fused path chooses for this shape (None if it does
    not take the shape).  Host only."""
    out = (ctypes.c_int32 * len(levels))()
    st = lib().gbh_tile_plan(len(levels), levels_arg(levels), dtype_code, op, out)
    if st == -8:
        return None
    check(st, "gbh_tile_plan")
    return tuple(int(v) for v in out)


def tile_candidates(levels, dtype_code=GBH_F64, op=GBH_HIERARCHIZE, max_count=6):
    """Tile shapes the autotuner times on the fused path, best estimate first
    ([] if the fused path does not take the shape).  Host only."""
    d = len(levels)
    out = (ctypes.c_int32 * (max_count * d))()
    cnt = ctypes.c_int(0)
    st = lib().gbh_tile_candidates(d, levels_arg(levels), dtype_code, op, max_count, out, ctypes.byref(cnt))
    if st == -8:
        return []
    check(st, "gbh_tile_candidates")
    return [tuple(int(out[i * d + k]) for k in range(d)) for i in range(cnt.value)]
