"""ctypes wrapper of the serial fp64 CPU oracle (``gbh_oracle.c``).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The GPU library never
imports it and shares no code with it.

Every array argument is a C-contiguous float64 numpy array in the grid layout
of Sec. 3 (row-major, dimension 0 contiguous):
``u.reshape(n_{d-1}, ..., n_0)`` in numpy terms, ``n_k = 2**levels[k] + 1``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gbh_oracle.c")
_LIB = os.path.join(_HERE, "libgbh_oracle.so")
_lock = threading.Lock()
_lib = None

_I64 = ctypes.c_int64
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
_I64P = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) and return the .so path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC",
                               "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_num_points.restype = _I64
            lib.orc_num_points.argtypes = [ctypes.c_int, _IP]
            for name in ("orc_hierarchize", "orc_dehierarchize", "orc_hierarchize_adjoint",
                         "orc_dehierarchize_adjoint"):
                f = getattr(lib, name)
                f.restype = None
                f.argtypes = [_DP, ctypes.c_int, _IP]
            for name in ("orc_hierarchize_at", "orc_dehierarchize_at", "orc_adjoint_at"):
                f = getattr(lib, name)
                f.restype = ctypes.c_double
                f.argtypes = [_DP, ctypes.c_int, _IP, _I64]
            lib.orc_hierarchize_nobnd.restype = None
            lib.orc_hierarchize_nobnd.argtypes = [_DP, ctypes.c_int, _IP, ctypes.c_int, _I64P, _I64P]
            lib.orc_scheme_count.restype = ctypes.c_int
            lib.orc_scheme_count.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.orc_scheme_levels.restype = ctypes.c_int
            lib.orc_scheme_levels.argtypes = [ctypes.c_int, ctypes.c_int, _IP, _DP]
            lib.orc_sparse_num_points.restype = _I64
            lib.orc_sparse_num_points.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.orc_sparse_index_of_grid.restype = None
            lib.orc_sparse_index_of_grid.argtypes = [ctypes.c_int, ctypes.c_int, _IP, _I64P]
            lib.orc_gather.restype = None
            lib.orc_gather.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _IP, _DP,
                                       ctypes.POINTER(_DP), _DP]
            lib.orc_scatter.restype = None
            lib.orc_scatter.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _IP, _DP, ctypes.c_int,
                                        _DP, ctypes.POINTER(_DP)]
            lib.orc_level_weights.restype = None
            lib.orc_level_weights.argtypes = [ctypes.c_int, _IP, _DP]
            _lib = lib
    return _lib


def _levels(levels):
    lv = np.ascontiguousarray(np.asarray(levels, dtype=np.int32).reshape(-1))
    return lv, lv.ctypes.data_as(_IP)


def _f64(u):
    u = np.asarray(u)
    if u.dtype != np.float64 or not u.flags.c_contiguous:
        raise TypeError("oracle arrays must be C-contiguous float64")
    return u.ctypes.data_as(_DP)


def num_points(levels) -> int:
    lv, p = _levels(levels)
    return int(_load().orc_num_points(len(lv), p))


def shape_of(levels):
    """numpy shape (n_{d-1}, ..., n_0) of a grid; dimension 0 is the last axis."""
    return tuple(2 ** int(l) + 1 for l in reversed(list(levels)))


def _transform(name, u, levels):
    lv, p = _levels(levels)
    out = np.array(u, dtype=np.float64, order="C", copy=True)
    if out.size != num_points(lv):
        raise ValueError("array size does not match the level vector")
    getattr(_load(), name)(_f64(out), len(lv), p)
    return out


def hierarchize(u, levels):
    """Alg. 1 (boundary form) on a copy of ``u``."""
    return _transform("orc_hierarchize", u, levels)


def dehierarchize(a, levels):
    """Exact inverse of :func:`hierarchize` on a copy of ``a``."""
    return _transform("orc_dehierarchize", a, levels)


def hierarchize_adjoint(y, levels):
    """Exact transpose of :func:`hierarchize` on a copy of ``y``."""
    return _transform("orc_hierarchize_adjoint", y, levels)


def dehierarchize_adjoint(y, levels):
    """Exact transpose of :func:`dehierarchize` on a copy of ``y``."""
    return _transform("orc_dehierarchize_adjoint", y, levels)


def _at(name, u, levels, flat_indices):
    lv, p = _levels(levels)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    f = getattr(_load(), name)
    up = _f64(u)
    return np.array([f(up, len(lv), p, int(i)) for i in np.asarray(flat_indices).reshape(-1)])


def hierarchize_at(u, levels, flat_indices):
    """Surpluses at the given flat indices, from the tensor-product rows of H."""
    return _at("orc_hierarchize_at", u, levels, flat_indices)


def dehierarchize_at(a, levels, flat_indices):
    """Nodal values at the given flat indices: sum of tensor hats."""
    return _at("orc_dehierarchize_at", a, levels, flat_indices)


def adjoint_at(y, levels, flat_indices):
    """Adjoint values at the given flat indices: columns of H."""
    return _at("orc_adjoint_at", y, levels, flat_indices)


def hierarchize_nobnd(u, levels, reduced_op=False):
    """The paper's boundary-free Alg. 1 (2^l - 1 points per dimension),
    instrumented.  Returns (result, n_add, n_mul)."""
    lv, p = _levels(levels)
    out = np.array(u, dtype=np.float64, order="C", copy=True)
    na, nm = ctypes.c_int64(0), ctypes.c_int64(0)
    _load().orc_hierarchize_nobnd(_f64(out), len(lv), p, int(bool(reduced_op)),
                                  ctypes.byref(na), ctypes.byref(nm))
    return out, na.value, nm.value


def scheme(d: int, n: int):
    """Combination scheme: (levels[G, d] int32, coeffs[G] float64)."""
    lib = _load()
    g = lib.orc_scheme_count(d, n)
    lv = np.zeros((g, d), dtype=np.int32)
    c = np.zeros(g, dtype=np.float64)
    got = lib.orc_scheme_levels(d, n, lv.ctypes.data_as(_IP), c.ctypes.data_as(_DP))
    assert got == g
    return lv, c


def sparse_num_points(d: int, n: int) -> int:
    return int(_load().orc_sparse_num_points(d, n))


def sparse_index_of_grid(d: int, n: int, levels):
    lv, p = _levels(levels)
    out = np.zeros(num_points(lv), dtype=np.int64)
    _load().orc_sparse_index_of_grid(d, n, p, out.ctypes.data_as(_I64P))
    return out


def gather(d: int, n: int, levels, coeffs, grids):
    """sparse = sum_g coeffs[g] * alpha_g, in the order given."""
    lv = np.ascontiguousarray(np.asarray(levels, dtype=np.int32).reshape(-1, d))
    cf = np.ascontiguousarray(coeffs, dtype=np.float64)
    gs = [np.ascontiguousarray(g, dtype=np.float64).reshape(-1) for g in grids]
    ptrs = (_DP * len(gs))(*[_f64(g) for g in gs])
    out = np.zeros(sparse_num_points(d, n), dtype=np.float64)
    _load().orc_gather(d, n, len(gs), lv.ctypes.data_as(_IP), _f64(cf), ptrs, _f64(out))
    return out


def gather_exact(d: int, n: int, levels, coeffs, grids):
    """sparse = sum_g coeffs[g] * alpha_g summed exactly (rational arithmetic)
    and rounded once to the nearest double: the reading of the gather (Sec. 2)
    that does not depend on the order of the grids.  Pure Python, small
    schemes only."""
    from fractions import Fraction
    lv = np.ascontiguousarray(np.asarray(levels, dtype=np.int32).reshape(-1, d))
    acc = [Fraction(0)] * sparse_num_points(d, n)
    for l, c, g in zip(lv, np.asarray(coeffs, dtype=np.float64), grids):
        idx = sparse_index_of_grid(d, n, l)
        cf = Fraction(float(c))
        for f, v in enumerate(np.asarray(g, dtype=np.float64).reshape(-1)):
            acc[idx[f]] += cf * Fraction(float(v))
    return np.array([float(a) for a in acc], dtype=np.float64)


def scatter(d: int, n: int, levels, coeffs, sparse, scaled: bool = False):
    """alpha_g = sparse restricted to the points of grid g (times coeffs[g]
    when scaled: the transpose of gather); one array per grid."""
    lv = np.ascontiguousarray(np.asarray(levels, dtype=np.int32).reshape(-1, d))
    cf = np.ascontiguousarray(coeffs, dtype=np.float64)
    sp = np.ascontiguousarray(sparse, dtype=np.float64)
    outs = [np.zeros(num_points(l), dtype=np.float64) for l in lv]
    ptrs = (_DP * len(outs))(*[_f64(o) for o in outs])
    _load().orc_scatter(d, n, len(outs), lv.ctypes.data_as(_IP), _f64(cf), 1 if scaled else 0, _f64(sp), ptrs)
    return outs


def level_weights(levels):
    """w = 2^{-sum_k level(i_k)} per point."""
    lv, p = _levels(levels)
    out = np.zeros(num_points(lv), dtype=np.float64)
    _load().orc_level_weights(len(lv), p, _f64(out))
    return out
