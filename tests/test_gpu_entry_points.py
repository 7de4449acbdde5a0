"""The four single-grid entry points of the C ABI (gbh_hierarchize,
gbh_dehierarchize, gbh_hierarchize_adjoint, gbh_dehierarchize_adjoint; the
paper's problem statement, Sec. 3) called directly through ctypes with valid
device data, a CUDA graph that captures a plan's batched transform and its
gather, replayed and compared with the oracle (Sec. 2), and a graph that
captures a single-grid fused hierarchization with its forked streams."""
import ctypes

import numpy as np
import pytest

import oracle
from parity import TOL32, TOL64, rel_err
from paper_1309_0392_gb300 import _lib, inputs

torch = pytest.importorskip("torch")
gbh = pytest.importorskip("paper_1309_0392_gb300")

pytestmark = pytest.mark.gpu

ENTRY = {"h": "gbh_hierarchize", "d": "gbh_dehierarchize", "a": "gbh_hierarchize_adjoint",
         "t": "gbh_dehierarchize_adjoint"}
ORACLE = {"h": oracle.hierarchize, "d": oracle.dehierarchize, "a": oracle.hierarchize_adjoint,
          "t": oracle.dehierarchize_adjoint}


def call_entry(op, t, levels, stream=None):
    code = _lib.GBH_F64 if t.dtype == torch.float64 else _lib.GBH_F32
    s = stream if stream is not None else torch.cuda.current_stream()
    fn = getattr(_lib.lib(), ENTRY[op])
    return fn(ctypes.c_void_p(t.data_ptr()), len(levels), _lib.levels_arg(levels), code,
              ctypes.c_void_p(s.cuda_stream))


SHAPES = [(5, 5), (9, 9, 9), (6, 5, 4), (3, 3, 2, 2, 2), (14,), (2, 3, 1, 4), (0, 7), (12,) + (1,) * 9]


@pytest.mark.parametrize("levels", SHAPES)
@pytest.mark.parametrize("op", ["h", "d", "a", "t"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_single_grid_entry_points(levels, op, dtype):
    if levels == (9, 9, 9) and (dtype == torch.float32 or op in "at"):
        pytest.skip("full-size headline grid: fp64 hierarchize / dehierarchize only")
    np_dt = np.float64 if dtype == torch.float64 else np.float32
    u = inputs.uniform(levels, 500 + sum(levels), dtype=np_dt)
    t = torch.tensor(u, device="cuda")
    assert call_entry(op, t, levels) == 0
    torch.cuda.synchronize()
    ud = u.astype(np.float64)
    ref = ORACLE[op](ud, levels)
    tol = TOL64 if dtype == torch.float64 else TOL32
    assert rel_err(t.cpu().double().numpy(), ref, ud, op) <= tol


def test_entry_point_argument_errors_touch_nothing():
    t = torch.ones(inputs.num_points((3, 3)), dtype=torch.float64, device="cuda")
    before = t.clone()
    lib = _lib.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    bad_levels = _lib.levels_arg((3, 31))
    assert lib.gbh_hierarchize(ctypes.c_void_p(t.data_ptr()), 2, bad_levels, _lib.GBH_F64, stream) == -4
    assert lib.gbh_dehierarchize(ctypes.c_void_p(t.data_ptr()), 0, _lib.levels_arg((3, 3)), _lib.GBH_F64,
                                 stream) == -1
    assert lib.gbh_hierarchize_adjoint(ctypes.c_void_p(t.data_ptr() + 4), 2, _lib.levels_arg((3, 3)),
                                       _lib.GBH_F64, stream) == -3
    assert lib.gbh_dehierarchize_adjoint(ctypes.c_void_p(t.data_ptr()), 2, _lib.levels_arg((3, 3)), 7,
                                         stream) == -2
    torch.cuda.synchronize()
    assert torch.equal(t, before)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_graph_replay_of_batched_transform_and_gather(dtype):
    """A CUDA graph captures the plan's batched hierarchization and the gather
    into the sparse grid; it is replayed twice, the second time after binding
    fresh grids (the graph reads the bound grid table from device memory, so
    a re-bind between replays redirects it).  Every grid and the sparse vector
    are compared with the oracle after each replay."""
    d, n = 3, 6
    plan = gbh.Plan.scheme(d, n, dtype=str(dtype))
    lv, c = oracle.scheme(d, n)
    np_dt = np.float64 if dtype == torch.float64 else np.float32
    tol = TOL64 if dtype == torch.float64 else TOL32

    def fresh(seed0):
        host = [inputs.scheme_grid(l, seed0 + g).astype(np_dt) for g, l in enumerate(lv)]
        return host, [torch.tensor(h, device="cuda") for h in host]

    host, grids = fresh(1000)
    plan.bind(grids)
    sparse = torch.zeros(plan.sparse_points, dtype=torch.float64, device="cuda")
    # warm up on a side stream (the plan's first execution sets kernel
    # attributes), then put the grids back
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.execute(gbh.GBH_HIERARCHIZE, stream=side)
        plan.gather(sparse, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    for g, h in zip(grids, host):
        g.copy_(torch.from_numpy(h))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.execute(gbh.GBH_HIERARCHIZE)
        plan.gather(sparse)
    torch.cuda.synchronize()

    for replay, seed0 in enumerate((1000, 3000)):
        if replay == 1:
            host, grids = fresh(seed0)
            plan.bind(grids)
        graph.replay()
        torch.cuda.synchronize()
        assert plan.status() == 0
        alphas = []
        for l, g, h in zip(lv, grids, host):
            a = g.cpu().double().numpy()
            assert rel_err(a, oracle.hierarchize(h.astype(np.float64), l), h, "h") <= tol, (replay, tuple(l))
            alphas.append(a)
        # the gather of the replay's own surpluses, bit for bit
        assert np.array_equal(sparse.cpu().numpy(), oracle.gather(d, n, lv, c, alphas)), replay


def test_graph_replay_of_fused_single_grid_hierarchization():
    """A 3-D fp64 grid on the fused path (tiles (5,4,4)) forks its
    one-lattice-dimension classes onto side streams and joins them back by
    events.  Captured in a CUDA graph, the fork and join become graph edges;
    two replays on fresh data match the oracle."""
    levels = (9, 8, 8)
    st = torch.cuda.Stream()
    t = torch.empty(inputs.num_points(levels), dtype=torch.float64, device="cuda")
    # warm-up outside the capture (first calls create the side streams and
    # set kernel attributes)
    with torch.cuda.stream(st):
        t.copy_(torch.from_numpy(inputs.uniform(levels, 61)))
        gbh.hierarchize(t, levels)
        gbh.dehierarchize(t, levels)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        gbh.hierarchize(t, levels)
    for seed in (62, 63):
        u = inputs.uniform(levels, seed)
        t.copy_(torch.from_numpy(u))
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        assert rel_err(t.cpu().numpy(), oracle.hierarchize(u, levels), u, "h") <= TOL64
