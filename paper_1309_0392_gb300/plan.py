"""Combination-scheme plans: batched transform of many grids in one persistent
launch, the fp64 gather into the sparse grid and the scatter back onto the
grids (Sec. 2)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib


class Plan:
    """Owns a gbh_plan (device work tables); the grids stay the caller's."""

    def __init__(self, handle, d, dtype_code):
        self._h = handle
        self.d = d
        self.dtype_code = dtype_code
        self._bound = None

    @classmethod
    def scheme(cls, d: int, n: int, dtype="float64", owned=None):
        """Plan of the combination scheme (d, n); with `owned` (increasing
        indexes into the scheme's enumeration) only those grids, for one rank
        of a sharded job."""
        code = _lib.GBH_F64 if str(dtype).endswith("float64") else _lib.GBH_F32
        h = ctypes.c_void_p()
        if owned is None:
            _lib.check(_lib.lib().gbh_plan_create_scheme(d, n, code, ctypes.byref(h)), "gbh_plan_create_scheme")
        else:
            own = [int(g) for g in owned]
            _lib.check(_lib.lib().gbh_plan_create_scheme_subset(d, n, code, len(own), _lib.levels_arg(own),
                                                                ctypes.byref(h)), "gbh_plan_create_scheme_subset")
        return cls(h, d, code)

    @classmethod
    def from_levels(cls, levels, dtype="float64"):
        lv = np.ascontiguousarray(np.asarray(levels, dtype=np.int32))
        g, d = lv.shape
        code = _lib.GBH_F64 if str(dtype).endswith("float64") else _lib.GBH_F32
        h = ctypes.c_void_p()
        _lib.check(_lib.lib().gbh_plan_create(g, d, lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                              code, ctypes.byref(h)), "gbh_plan_create")
        return cls(h, d, code)

    def close(self):
        if self._h is not None and self._h.value:
            _lib.lib().gbh_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_grids(self) -> int:
        v = ctypes.c_int(0)
        _lib.check(_lib.lib().gbh_plan_num_grids(self._h, ctypes.byref(v)), "gbh_plan_num_grids")
        return int(v.value)

    def levels(self):
        out = np.zeros((self.num_grids, self.d), dtype=np.int32)
        for g in range(out.shape[0]):
            _lib.check(_lib.lib().gbh_plan_grid_levels(
                self._h, g, out[g].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "gbh_plan_grid_levels")
        return out

    def coeffs(self):
        out = np.zeros(self.num_grids, dtype=np.float64)
        _lib.check(_lib.lib().gbh_plan_coeffs(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                   "gbh_plan_coeffs")
        return out

    def set_coeffs(self, coeffs):
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
        if c.shape != (self.num_grids,):
            raise ValueError("one coefficient per grid")
        _lib.check(_lib.lib().gbh_plan_set_coeffs(self._h, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                   "gbh_plan_set_coeffs")

    @property
    def sparse_points(self) -> int:
        v = ctypes.c_int64(0)
        _lib.check(_lib.lib().gbh_plan_sparse_points(self._h, ctypes.byref(v)), "gbh_plan_sparse_points")
        return int(v.value)

    @property
    def total_points(self) -> int:
        v = ctypes.c_int64(0)
        _lib.check(_lib.lib().gbh_plan_total_points(self._h, ctypes.byref(v)), "gbh_plan_total_points")
        return int(v.value)

    def bind(self, grids, stream=None):
        """Bind device tensors (one per grid, in plan order)."""
        import torch
        ptrs = (ctypes.c_void_p * len(grids))(*[ctypes.c_void_p(t.data_ptr()) for t in grids])
        s = stream if stream is not None else torch.cuda.current_stream()
        _lib.check(_lib.lib().gbh_plan_bind(self._h, ptrs, ctypes.c_void_p(s.cuda_stream)), "gbh_plan_bind")
        self._bound = list(grids)

    def execute(self, op=_lib.GBH_HIERARCHIZE, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        _lib.check(_lib.lib().gbh_plan_execute(self._h, int(op), ctypes.c_void_p(s.cuda_stream)),
                   "gbh_plan_execute")

    def _check_sparse(self, sparse):
        import torch
        if not (isinstance(sparse, torch.Tensor) and sparse.is_cuda and sparse.dtype == torch.float64
                and sparse.is_contiguous() and sparse.numel() == self.sparse_points):
            raise ValueError(f"sparse must be a contiguous float64 CUDA tensor of {self.sparse_points} points")

    def gather(self, sparse, stream=None):
        import torch
        self._check_sparse(sparse)
        s = stream if stream is not None else torch.cuda.current_stream()
        _lib.check(_lib.lib().gbh_plan_gather(self._h, ctypes.c_void_p(sparse.data_ptr()),
                                              ctypes.c_void_p(s.cuda_stream)), "gbh_plan_gather")
        return sparse

    def scatter(self, sparse, scaled: bool = False, stream=None):
        """Every bound grid receives the sparse-grid surpluses of its points
        (times its coefficient when scaled: the transpose of gather)."""
        import torch
        self._check_sparse(sparse)
        s = stream if stream is not None else torch.cuda.current_stream()
        _lib.check(_lib.lib().gbh_plan_scatter(self._h, ctypes.c_void_p(sparse.data_ptr()), 1 if scaled else 0,
                                               ctypes.c_void_p(s.cuda_stream)), "gbh_plan_scatter")

    def set_params(self, op, ctas_per_sm: int, wave_mb: int):
        """Execution parameters of op: resident CTAs per SM (0 = as many as
        fit) and the L2 wave of the work queue in MiB."""
        _lib.check(_lib.lib().gbh_plan_set_params(self._h, int(op), int(ctas_per_sm), int(wave_mb)),
                   "gbh_plan_set_params")

    def get_params(self, op):
        c, w = ctypes.c_int(0), ctypes.c_int(0)
        _lib.check(_lib.lib().gbh_plan_get_params(self._h, int(op), ctypes.byref(c), ctypes.byref(w)),
                   "gbh_plan_get_params")
        return int(c.value), int(w.value)

    def autotune(self, op=_lib.GBH_HIERARCHIZE, stream=None):
        """Times the execution parameters of op on scratch grids and keeps the
        fastest (gbh_plan_autotune); the bound grids are untouched."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        r = _lib.PlanTuneResult()
        _lib.check(_lib.lib().gbh_plan_autotune(self._h, int(op), ctypes.c_void_p(s.cuda_stream), ctypes.byref(r)),
                   "gbh_plan_autotune")
        return {"ctas_per_sm": int(r.ctas_per_sm), "wave_mb": int(r.wave_mb), "candidates": int(r.candidates),
                "max_ctas_per_sm": int(r.max_ctas_per_sm), "ms_tuned": float(r.ms_tuned),
                "ms_model": float(r.ms_model)}

    def test_stall(self, grid: int, spin_limit: int = 1 << 14):
        """Failure injection: the grid's work items wait on a dependency that
        is never released (grid=-1 restores normal operation)."""
        _lib.check(_lib.lib().gbh_plan_test_stall(self._h, int(grid), int(spin_limit)), "gbh_plan_test_stall")

    def status(self, stream=None) -> int:
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return int(_lib.lib().gbh_plan_status(self._h, ctypes.c_void_p(s.cuda_stream)))
