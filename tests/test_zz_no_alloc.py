"""The batched transform that allocates nothing (gbh_batched_transform_noalloc),
for callers that may not call cudaMalloc: its work tables live in a fixed
device array inside the library.  Checked through the C ABI against the plan
entry point (gbh_plan_execute) on the same grids, two calls in a row.

Kept in a file of its own that pytest collects last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
gbh = pytest.importorskip("paper_1309_0392_gb300")
from paper_1309_0392_gb300 import _lib  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-13, torch.float32: 1e-5}


def noalloc(grids, levels, op, dtype_code):
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    ptrs = (ctypes.c_void_p * len(grids))(*[ctypes.c_void_p(g.data_ptr()) for g in grids])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return _lib.lib().gbh_batched_transform_noalloc(len(grids), lv.shape[1],
                                                     lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                     ptrs, dtype_code, op, stream)


def max_rel(a_list, b_list):
    err, scale = 0.0, 0.0
    for a, b in zip(a_list, b_list):
        err = max(err, (a.double() - b.double()).abs().max().item())
        scale = max(scale, b.double().abs().max().item())
    return err / max(scale, 1e-300)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_matches_plan_two_calls(dtype):
    code = _lib.GBH_F64 if dtype == torch.float64 else _lib.GBH_F32
    levels = gbh.Plan.scheme(4, 6).levels()
    gen = torch.Generator(device="cuda").manual_seed(7)
    ours = [torch.rand(gbh.num_points(l), dtype=dtype, device="cuda", generator=gen) * 2 - 1 for l in levels]
    ref = [t.clone() for t in ours]
    plan = gbh.Plan.from_levels(levels, dtype=str(dtype))
    plan.bind(ref)
    for op in (gbh.GBH_HIERARCHIZE, gbh.GBH_DEHIERARCHIZE):
        assert noalloc(ours, levels, op, code) == 0
        plan.execute(op)
        torch.cuda.synchronize()
        assert plan.status() == 0
        assert max_rel(ours, ref) <= TOL[dtype]


def test_noalloc_scheme_d3_uneven_grids_twice():
    levels = np.array([[3, 0, 2], [0, 0, 0], [9, 1, 1], [2, 2, 2], [0, 4, 1], [1, 1, 12]], dtype=np.int32)
    ours = [torch.rand(gbh.num_points(l), dtype=torch.float64, device="cuda") for l in levels]
    ref = [t.clone() for t in ours]
    plan = gbh.Plan.from_levels(levels)
    plan.bind(ref)
    for _ in range(2):
        assert noalloc(ours, levels, gbh.GBH_HIERARCHIZE, _lib.GBH_F64) == 0
        plan.execute(gbh.GBH_HIERARCHIZE)
        torch.cuda.synchronize()
        assert max_rel(ours, ref) <= 1e-13


def test_noalloc_rejects_too_many_grids():
    levels = np.ones((2049, 2), dtype=np.int32)
    fake = [torch.empty(0, device="cuda")] * 1
    lv = np.ascontiguousarray(levels)
    ptrs = (ctypes.c_void_p * 2049)(*([ctypes.c_void_p(fake[0].data_ptr() or 256)] * 2049))
    st = _lib.lib().gbh_batched_transform_noalloc(2049, 2, lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                   ptrs, _lib.GBH_F64, gbh.GBH_HIERARCHIZE, None)
    assert st == -4        # GBH_ERANGE, nothing launched
