"""The batched transform that allocates nothing (gbh_batched_transform_noalloc),
for callers that may not call cudaMalloc: its work tables live in a fixed
device array inside the library.  Checked through the C ABI, two calls in a
row, against the plan entry point (gbh_plan_execute) on the same grids and
against the CPU oracle; its status word reports a bounded wait that gave up.

Kept in a file of its own that pytest collects last."""
import ctypes

import numpy as np
import pytest

import oracle
from parity import TOL32, TOL64, rel_err

torch = pytest.importorskip("torch")
gbh = pytest.importorskip("paper_1309_0392_gb300")
from paper_1309_0392_gb300 import _lib  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {torch.float64: TOL64, torch.float32: TOL32}
ORACLE = {gbh.GBH_HIERARCHIZE: (oracle.hierarchize, "h"), gbh.GBH_DEHIERARCHIZE: (oracle.dehierarchize, "d")}


def noalloc(grids, levels, op, dtype_code):
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    ptrs = (ctypes.c_void_p * len(grids))(*[ctypes.c_void_p(g.data_ptr()) for g in grids])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return _lib.lib().gbh_batched_transform_noalloc(len(grids), lv.shape[1],
                                                     lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                     ptrs, dtype_code, op, stream)


def noalloc_status():
    return _lib.lib().gbh_batched_transform_noalloc_status(
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def max_rel(a_list, b_list):
    err, scale = 0.0, 0.0
    for a, b in zip(a_list, b_list):
        err = max(err, (a.double() - b.double()).abs().max().item())
        scale = max(scale, b.double().abs().max().item())
    return err / max(scale, 1e-300)


def check_against_oracle(grids, levels, before, op, dtype):
    fn, o = ORACLE[op]
    for l, g, u in zip(levels, grids, before):
        assert rel_err(g.cpu().double().numpy(), fn(u, tuple(l)), u, o) <= TOL[dtype], tuple(l)


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
        before = [t.cpu().double().numpy() for t in ours]
        assert noalloc(ours, levels, op, code) == 0
        plan.execute(op)
        torch.cuda.synchronize()
        assert plan.status() == 0
        assert noalloc_status() == 0
        assert max_rel(ours, ref) <= TOL[dtype]
        check_against_oracle(ours, levels, before, op, dtype)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_scheme_d3_uneven_grids_twice(dtype):
    """Uneven grids, level-0 dimensions and a level-12 dimension (the block /
    coarse-lattice split), two hierarchizations in a row."""
    code = _lib.GBH_F64 if dtype == torch.float64 else _lib.GBH_F32
    levels = np.array([[3, 0, 2], [0, 0, 0], [9, 1, 1], [2, 2, 2], [0, 4, 1], [1, 1, 12]], dtype=np.int32)
    gen = torch.Generator(device="cuda").manual_seed(8)
    ours = [torch.rand(gbh.num_points(l), dtype=dtype, device="cuda", generator=gen) for l in levels]
    ref = [t.clone() for t in ours]
    plan = gbh.Plan.from_levels(levels, dtype=str(dtype))
    plan.bind(ref)
    for _ in range(2):
        before = [t.cpu().double().numpy() for t in ours]
        assert noalloc(ours, levels, gbh.GBH_HIERARCHIZE, code) == 0
        plan.execute(gbh.GBH_HIERARCHIZE)
        torch.cuda.synchronize()
        assert noalloc_status() == 0
        assert max_rel(ours, ref) <= TOL[dtype]
        check_against_oracle(ours, levels, before, gbh.GBH_HIERARCHIZE, dtype)


def test_noalloc_reports_a_wait_that_gave_up():
    """A dependency that nothing releases (injected from the host): the bounded
    waits give up, the status word says GBH_ETIMEOUT and stays set across a
    later call until it is read; reading clears it, and normal calls work
    again afterwards."""
    levels = gbh.Plan.scheme(3, 5).levels()
    grids = [torch.rand(gbh.num_points(l), dtype=torch.float64, device="cuda") for l in levels]
    assert noalloc_status() == 0
    lib = _lib.lib()
    assert lib.gbh_batched_transform_noalloc_test_stall(3, 1 << 12) == 0
    try:
        assert noalloc(grids, levels, gbh.GBH_HIERARCHIZE, _lib.GBH_F64) == 0
    finally:
        assert lib.gbh_batched_transform_noalloc_test_stall(-1, 1) == 0
    torch.cuda.synchronize()
    # a normal call in between does not clear the word
    other = [torch.rand(gbh.num_points(l), dtype=torch.float64, device="cuda") for l in levels]
    assert noalloc(other, levels, gbh.GBH_HIERARCHIZE, _lib.GBH_F64) == 0
    assert noalloc_status() == -6
    assert noalloc_status() == 0
    fresh = [torch.rand(gbh.num_points(l), dtype=torch.float64, device="cuda") for l in levels]
    before = [t.cpu().numpy() for t in fresh]
    assert noalloc(fresh, levels, gbh.GBH_HIERARCHIZE, _lib.GBH_F64) == 0
    torch.cuda.synchronize()
    assert noalloc_status() == 0
    check_against_oracle(fresh, levels, before, gbh.GBH_HIERARCHIZE, torch.float64)


def _fake_call(levels, op=gbh.GBH_HIERARCHIZE, dtype_code=_lib.GBH_F64):
    """Calls the entry point with a placeholder device pointer for every grid:
    only for requests that are rejected before anything is launched."""
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    g = lv.shape[0]
    ptrs = (ctypes.c_void_p * g)(*([ctypes.c_void_p(256)] * g))
    return _lib.lib().gbh_batched_transform_noalloc(g, lv.shape[1], lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                     ptrs, dtype_code, op, None)


def test_noalloc_rejects_too_many_grids():
    assert _fake_call(np.ones((2049, 2), dtype=np.int32)) == -4        # GBH_ERANGE, nothing launched


def test_noalloc_rejects_too_many_work_items():
    """2000 grids of level (12, 12): far more work items than the fixed array
    holds."""
    assert _fake_call(np.full((2000, 2), 12, dtype=np.int32)) == -4    # GBH_ERANGE, nothing launched


def test_noalloc_rejects_the_transposes():
    for op in (gbh.GBH_ADJOINT, gbh.GBH_DEHIERARCHIZE_ADJOINT):
        assert _fake_call(np.ones((3, 2), dtype=np.int32), op=op) == -8   # GBH_EUNSUPPORTED
