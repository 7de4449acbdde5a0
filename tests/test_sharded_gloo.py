"""The multi-rank path on CPU (gloo, world size 2): grids of a combination
scheme are split over ranks, every rank gathers its own grids with the other
ranks' coefficients set to 0, and one sum all-reduce of the sparse vector
gives the single-rank gather; every rank then scatters the sparse vector onto
its own grids with no further exchange.  The per-rank gather here is the CPU oracle
(the GPU gather computes the same sum)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1309_0392_gb300 import inputs, shard  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, d, n, out):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lv, c = oracle.scheme(d, n)
    owned = shard.partition_grids([oracle.num_points(l) for l in lv], world)[rank]
    alphas = [oracle.hierarchize(inputs.scheme_grid(l, 1000 + g), l) for g, l in enumerate(lv)]
    part = torch.from_numpy(oracle.gather(d, n, lv, shard.owned_coeffs(c, owned), alphas))
    shard.allreduce_sparse(part)
    if rank == 0:
        full = oracle.gather(d, n, lv, c, alphas)
        out.put(float(np.abs(part.numpy() - full).max() / max(np.abs(full).max(), 1e-300)))
    dist.barrier()
    dist.destroy_process_group()


def _round_worker(rank, world, port, d, n, out):
    """One iterated round on two ranks: hierarchize own grids, partial gather,
    all-reduce, scatter onto own grids, dehierarchize them."""
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lv, c = oracle.scheme(d, n)
    owned = shard.partition_grids([oracle.num_points(l) for l in lv], world)[rank]
    alphas = [oracle.hierarchize(inputs.scheme_grid(l, 1000 + g), l) for g, l in enumerate(lv)]
    part = torch.from_numpy(oracle.gather(d, n, lv, shard.owned_coeffs(c, owned), alphas))
    shard.allreduce_sparse(part)
    mine = oracle.scatter(d, n, lv[owned], c[owned], part.numpy())
    mine = [oracle.dehierarchize(a, lv[g]) for a, g in zip(mine, owned)]
    full_sparse = oracle.gather(d, n, lv, c, alphas)
    full = oracle.scatter(d, n, lv, c, full_sparse)
    err = max(float(np.abs(a - oracle.dehierarchize(full[g], lv[g])).max()) for a, g in zip(mine, owned))
    out.put((rank, len(owned), err))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_is_disjoint_complete_and_balanced():
    pts = [2 ** (i % 7) * 100 + i for i in range(97)]
    parts = shard.partition_grids(pts, 4)
    flat = sorted(g for p in parts for g in p)
    assert flat == list(range(97))
    loads = [sum(pts[g] for g in p) for p in parts]
    assert max(loads) - min(loads) <= max(pts)


def test_owned_coeffs_sum_to_full():
    c = np.array([1.0, -3.0, 3.0, -1.0, 2.0])
    parts = shard.partition_grids([5, 4, 3, 2, 1], 2)
    assert np.array_equal(sum(shard.owned_coeffs(c, p) for p in parts), c)


@pytest.mark.parametrize("d,n", [(2, 5), (3, 4)])
def test_two_rank_gather_matches_single_rank(d, n):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, d, n, out)) for r in range(2)]
    for p in procs:
        p.start()
    err = out.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert err <= 1e-14


@pytest.mark.parametrize("d,n", [(2, 5), (3, 4)])
def test_two_rank_iterated_round_matches_single_rank(d, n):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_round_worker, args=(r, 2, port, d, n, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = [out.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    assert sum(k for _, k, _ in got) == len(oracle.scheme(d, n)[0])
    assert max(e for _, _, e in got) <= 1e-14
