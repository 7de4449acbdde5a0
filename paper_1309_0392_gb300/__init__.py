"""GB300-native hierarchization of sparse-grid combination grids.

Thin Python layer over the C ABI of ``libgbh.so`` (include/gbh.h).  PyTorch
provides device memory and streams only; every transform runs in the
library's CUDA kernels (sm_103a).  A grid of level vector ``levels`` is a
contiguous CUDA tensor of ``prod(2**l + 1)`` elements (float32 or float64),
dimension 0 contiguous (P. Hupp, arXiv 1309.0392, Sec. 3).
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import (GBH_ADJOINT, GBH_DEHIERARCHIZE, GBH_DEHIERARCHIZE_ADJOINT, GBH_HIERARCHIZE,  # noqa: F401
                   GBH_PATH_AUTO, GBH_PATH_FUSED, GBH_PATH_GROUPED, GBH_PATH_PLAIN, GBH_ARITH_AUTO,
                   GBH_ARITH_NATIVE, GBH_ARITH_FIXED, GbhError, sparse_index_of_grid)

__all__ = ["hierarchize", "dehierarchize", "hierarchize_adjoint", "dehierarchize_adjoint", "transform", "num_points",
           "autotune", "autotune_reset", "Plan", "HierarchizeFn", "DehierarchizeFn", "GbhError", "sparse_index_of_grid"]


def num_points(levels) -> int:
    out = ctypes.c_int64(0)
    _lib.check(_lib.lib().gbh_num_points(len(levels), _lib.levels_arg(levels), ctypes.byref(out)),
               "gbh_num_points")
    return int(out.value)


def _dtype_code(t):
    import torch
    if t.dtype == torch.float64:
        return _lib.GBH_F64
    if t.dtype == torch.float32:
        return _lib.GBH_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _stream_ptr(t, stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream(t.device)
    return ctypes.c_void_p(s.cuda_stream)


def transform(t, levels, op=GBH_HIERARCHIZE, *, path=GBH_PATH_AUTO, tile=None, arith=0,
              variant=0, stream=None, batch=None):
    """In-place transform of grid tensor ``t`` (op: GBH_HIERARCHIZE,
    GBH_DEHIERARCHIZE, GBH_ADJOINT or GBH_DEHIERARCHIZE_ADJOINT).  With
    ``batch=B`` the tensor holds B grids of the level vector back to back.
    ``variant`` picks kernels within a path (same results within the
    stated tolerance): fused path, 3-D fp64 tiles (5,4,4): 0 the interior
    class on its own kernel, 1 the generic tile kernels; plain path with
    native arithmetic: 0 two consecutive dimensions per pass where they fit
    a pair tile, 1 one pass per dimension (bit-identical results).
    Returns ``t``."""
    B = 1 if batch is None else int(batch)
    if B < 1:
        raise ValueError("batch must be >= 1")
    if not t.is_cuda:
        raise ValueError("grid tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("grid tensor must be contiguous")
    if t.numel() != B * num_points(levels):
        raise ValueError(f"tensor has {t.numel()} elements, {B} grid(s) of level vector "
                         f"{tuple(levels)} need {B * num_points(levels)}")
    opt = _lib.Options()
    opt.path = int(path)
    opt.arith = int(arith)
    opt.variant = int(variant)
    if tile is not None:
        for k, m in enumerate(tile):
            opt.tile_exp[k] = int(m)
    with _device(t):
        st = _lib.lib().gbh_transform_batched(ctypes.c_void_p(t.data_ptr()), B, len(levels),
                                              _lib.levels_arg(levels), _dtype_code(t), int(op),
                                              ctypes.byref(opt), _stream_ptr(t, stream))
    _lib.check(st, "gbh_transform_batched")
    return t


class _device:
    def __init__(self, t):
        self.dev = t.device

    def __enter__(self):
        import torch
        self.ctx = torch.cuda.device(self.dev)
        self.ctx.__enter__()

    def __exit__(self, *a):
        self.ctx.__exit__(*a)


def hierarchize(t, levels, **kw):
    """Alg. 1 (boundary form) in place: nodal values -> hierarchical surpluses."""
    return transform(t, levels, GBH_HIERARCHIZE, **kw)


def dehierarchize(t, levels, **kw):
    """Inverse of :func:`hierarchize` in place: surpluses -> nodal values."""
    return transform(t, levels, GBH_DEHIERARCHIZE, **kw)


def hierarchize_adjoint(t, levels, **kw):
    """Transpose of :func:`hierarchize` in place."""
    return transform(t, levels, GBH_ADJOINT, **kw)


def dehierarchize_adjoint(t, levels, **kw):
    """Transpose of :func:`dehierarchize` in place."""
    return transform(t, levels, GBH_DEHIERARCHIZE_ADJOINT, **kw)


def autotune(levels, dtype="float64", op=GBH_HIERARCHIZE):
    """Times the execution paths and tile shapes of the single-grid transform
    for this level vector on a scratch grid and records the fastest for the
    default path (gbh_autotune).  Returns the choice and the times."""
    code = _lib.GBH_F64 if str(dtype).endswith("float64") else _lib.GBH_F32
    r = _lib.TuneResult()
    _lib.check(_lib.lib().gbh_autotune(len(levels), _lib.levels_arg(levels), code, int(op), ctypes.byref(r)),
               "gbh_autotune")
    d = len(levels)
    return {"path": int(r.path), "tile_exp": tuple(int(v) for v in r.tile_exp[:d]), "candidates": int(r.candidates),
            "ms_tuned": float(r.ms_tuned), "ms_model": float(r.ms_model), "model_path": int(r.model_path),
            "model_tile_exp": tuple(int(v) for v in r.model_tile_exp[:d])}


def autotune_reset():
    """Drops every recorded autotuner choice (gbh_autotune_reset)."""
    _lib.check(_lib.lib().gbh_autotune_reset(), "gbh_autotune_reset")


from .plan import Plan  # noqa: E402
from .autograd import DehierarchizeFn, HierarchizeFn  # noqa: E402
