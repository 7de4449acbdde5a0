"""The autotuner (tile shape and dimension fusion chosen per level vector by
measurement) and the plan tuner (resident CTAs per SM and L2 waves of the work
queue): every configuration either can choose is run against the CPU oracle,
and the choices they record are used by the default path and by new plans."""
import numpy as np
import pytest

import oracle
from parity import TOL32, TOL64, rel_err
from paper_1309_0392_gb300 import _lib, inputs

torch = pytest.importorskip("torch")
gbh = pytest.importorskip("paper_1309_0392_gb300")

pytestmark = pytest.mark.gpu

OPS = {"h": gbh.GBH_HIERARCHIZE, "d": gbh.GBH_DEHIERARCHIZE}
ORACLE = {"h": oracle.hierarchize, "d": oracle.dehierarchize}
SHAPES = [(6, 5, 4), (9, 5, 5), (5, 4, 4, 4), (3, 3, 2, 2, 2), (12, 2)]


def run(u, levels, op, dtype, **kw):
    t = torch.tensor(u, dtype=dtype, device="cuda")
    gbh.transform(t, levels, OPS[op], **kw)
    torch.cuda.synchronize()
    return t.cpu().double().numpy()


@pytest.mark.parametrize("levels", SHAPES)
@pytest.mark.parametrize("op", ["h", "d"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_every_tuner_candidate_matches_oracle(levels, op, dtype):
    """The per-dimension sweeps, every tile shape the tuner times and the
    dimension groups, each against the oracle."""
    code = _lib.GBH_F64 if dtype == torch.float64 else _lib.GBH_F32
    np_dt = np.float64 if dtype == torch.float64 else np.float32
    tol = TOL64 if dtype == torch.float64 else TOL32
    u = inputs.uniform(levels, 600 + sum(levels), dtype=np_dt)
    ud = u.astype(np.float64)
    ref = ORACLE[op](ud, levels)
    configs = [dict(path=gbh.GBH_PATH_PLAIN, arith=2 if dtype == torch.float64 else 0)]
    configs += [dict(path=gbh.GBH_PATH_FUSED, tile=m) for m in _lib.tile_candidates(levels, code, OPS[op])]
    configs += [dict(path=gbh.GBH_PATH_GROUPED)]
    for kw in configs:
        assert rel_err(run(u, levels, op, dtype, **kw), ref, ud, op) <= tol, kw


@pytest.mark.parametrize("levels", [(6, 5, 4), (5, 4, 4, 4), (12, 2)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_autotune_records_choice_for_default_path(levels, dtype):
    gbh.autotune_reset()
    try:
        for op in ("h", "d"):
            r = gbh.autotune(levels, dtype=str(dtype), op=OPS[op])
            assert r["candidates"] >= 2
            assert r["ms_tuned"] > 0 and r["ms_model"] > 0
            assert r["ms_tuned"] <= r["ms_model"] * 1.0000001
            assert r["path"] in (gbh.GBH_PATH_PLAIN, gbh.GBH_PATH_FUSED, gbh.GBH_PATH_GROUPED)
            if r["path"] == gbh.GBH_PATH_FUSED:
                code = _lib.GBH_F64 if dtype == torch.float64 else _lib.GBH_F32
                assert r["tile_exp"] in _lib.tile_candidates(levels, code, OPS[op])
                assert _lib.tile_plan(levels, code, OPS[op]) == r["tile_exp"]
            # the default path now runs the recorded choice; results stay
            # within the tolerance
            np_dt = np.float64 if dtype == torch.float64 else np.float32
            u = inputs.uniform(levels, 700, dtype=np_dt)
            ud = u.astype(np.float64)
            tol = TOL64 if dtype == torch.float64 else TOL32
            assert rel_err(run(u, levels, op, dtype), ORACLE[op](ud, levels), ud, op) <= tol
    finally:
        gbh.autotune_reset()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_every_plan_configuration_matches_oracle(dtype):
    d, n = 3, 6
    plan = gbh.Plan.scheme(d, n, dtype=str(dtype))
    lv = plan.levels()
    np_dt = np.float64 if dtype == torch.float64 else np.float32
    tol = TOL64 if dtype == torch.float64 else TOL32
    host = [inputs.scheme_grid(l, 900 + g).astype(np_dt) for g, l in enumerate(lv)]
    refs = {o: [ORACLE[o](h.astype(np.float64), l) for h, l in zip(host, lv)] for o in ("h", "d")}
    for ctas in (1, 2, 0):
        for wave in (1, 8, 64):
            for o in ("h", "d"):
                plan.set_params(OPS[o], ctas, wave)
                assert plan.get_params(OPS[o]) == (ctas, wave)
                grids = [torch.tensor(h, device="cuda") for h in host]
                plan.bind(grids)
                plan.execute(OPS[o])
                assert plan.status() == 0
                for g, r, h in zip(grids, refs[o], host):
                    assert rel_err(g.cpu().double().numpy(), r, h.astype(np.float64), o) <= tol, (ctas, wave, o)


def test_plan_autotune_keeps_bound_grids_and_is_reused():
    d, n = 3, 7
    plan = gbh.Plan.scheme(d, n)
    lv = plan.levels()
    host = [inputs.scheme_grid(l, 950 + g) for g, l in enumerate(lv)]
    grids = [torch.tensor(h, device="cuda") for h in host]
    plan.bind(grids)
    res = {}
    for o in ("h", "d"):
        r = plan.autotune(OPS[o])
        assert r["candidates"] == 4 * r["max_ctas_per_sm"]
        assert 1 <= r["ctas_per_sm"] <= r["max_ctas_per_sm"] and r["wave_mb"] in (8, 16, 32, 64)
        assert r["ms_tuned"] <= r["ms_model"] * 1.0000001
        assert plan.get_params(OPS[o]) == (r["ctas_per_sm"], r["wave_mb"])
        res[o] = r
    torch.cuda.synchronize()
    for g, h in zip(grids, host):
        assert np.array_equal(g.cpu().numpy(), h)        # the caller's grids were not touched
    plan.execute(gbh.GBH_HIERARCHIZE)
    assert plan.status() == 0
    for g, h, l in zip(grids, host, lv):
        assert rel_err(g.cpu().numpy(), oracle.hierarchize(h, l), h, "h") <= TOL64
    # a new plan of the same scheme starts with the tuned parameters
    again = gbh.Plan.scheme(d, n)
    for o in ("h", "d"):
        assert again.get_params(OPS[o]) == (res[o]["ctas_per_sm"], res[o]["wave_mb"])


def test_tuner_arguments():
    with pytest.raises(gbh.GbhError):
        gbh.autotune((3, 31))
    plan = gbh.Plan.scheme(2, 4)
    for bad in ((gbh.GBH_ADJOINT, 1, 8), (gbh.GBH_HIERARCHIZE, -1, 8), (gbh.GBH_HIERARCHIZE, 1, 0)):
        with pytest.raises(gbh.GbhError):
            plan.set_params(*bad)


def test_plan_autotune_first_in_process():
    """The plan tuner in a fresh process, before any plan has executed (its
    kernel attributes are set by the tuner itself)."""
    import subprocess
    import sys
    code = ("import torch, paper_1309_0392_gb300 as gbh;"
            "p = gbh.Plan.scheme(3, 5);"
            "r = p.autotune(gbh.GBH_HIERARCHIZE);"
            "assert r['candidates'] > 0, r")
    root = __import__("os").path.dirname(__import__("os").path.dirname(__import__("os").path.abspath(__file__)))
    subprocess.run([sys.executable, "-c", code], check=True, cwd=root, timeout=600)
