"""Two and three ranks on CPU (gloo) draw disjoint sample-id ranges of one
seed with the oracle; the exact integer all-reduce of
paper_2409_08975_gb300.dist gives the single-run sums, and the library's
tc_estimate_from_sums (host arithmetic, no GPU needed) the estimate."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from _graphs import small_random_graph

C4 = [(0, 1), (1, 2), (2, 3), (3, 0)]
K_TOTAL = 20_001
SEED = 31


def _graph():
    src, dst, t = small_random_graph(77, 6, 60, 60, dup_frac=0.3)
    g = oracle.build_csr(6, src, dst, t)
    plan = oracle.compile_motif(C4)
    pre = oracle.prefix_sum(oracle.path_weights(g, plan, 20)["w"])
    return g, plan, pre


def _worker(rank, world, port, queue):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2409_08975_gb300 import dist as tcdist
    g, plan, pre = _graph()
    off, cnt = tcdist.rank_range(K_TOTAL, rank, world)
    sums, _ = oracle.sample_run(g, plan, 20, pre, cnt, SEED, off)
    merged = tcdist.merge_runs(sums, int(pre[-1]))
    # values above 2^64 survive the limb split
    big = tcdist.allreduce_exact([(1 << 100) + rank])
    if rank == 0:
        queue.put((merged, big))
    dist.barrier()
    dist.destroy_process_group()


def _batch_worker(rank, world, port, queue):
    # every rank answers the same two queries over its own id range
    # [rank * k, (rank + 1) * k), as the batched benchmark does
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2409_08975_gb300 import dist as tcdist
    g, plan, pre = _graph()
    plan2 = oracle.compile_motif([(0, 1), (0, 2), (1, 2)])
    pre2 = oracle.prefix_sum(oracle.path_weights(g, plan2, 10)["w"])
    local = []
    for pl, delta, pr, k in ((plan, 20, pre, 3000), (plan2, 10, pre2, 1700)):
        sums, _ = oracle.sample_run(g, pl, delta, pr, k, SEED, rank * k)
        local.append(dict(sums, W=int(pr[-1])))
    merged = tcdist.merge_batch(local)
    if rank == 0:
        queue.put(merged)
    dist.barrier()
    dist.destroy_process_group()


def _built():
    from paper_2409_08975_gb300 import _build
    _build.build()  # once, before the ranks load the library


@pytest.mark.parametrize("world", [2, 3])
def test_batch_runs_merge_per_query(world):
    _built()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    g, plan, pre = _graph()
    plan2 = oracle.compile_motif([(0, 1), (0, 2), (1, 2)])
    pre2 = oracle.prefix_sum(oracle.path_weights(g, plan2, 10)["w"])
    for m, (pl, delta, pr, k) in zip(merged, ((plan, 20, pre, 3000), (plan2, 10, pre2, 1700))):
        single, _ = oracle.sample_run(g, pl, delta, pr, world * k, SEED, 0)
        for key in ("sum_x", "sum_x2", "hits", "k"):
            assert m[key] == single[key], key
        est, _ = oracle.estimate(single["sum_x"], single["sum_x2"], world * k, int(pr[-1]))
        assert m["estimate"] == pytest.approx(est, rel=1e-12)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_disjoint_ranges_merge_to_single_run(world):
    _built()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    merged, big = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    g, plan, pre = _graph()
    single, _ = oracle.sample_run(g, plan, 20, pre, K_TOTAL, SEED, 0)
    for key in ("sum_x", "sum_x2", "hits", "k"):
        assert merged[key] == single[key]
    est, se = oracle.estimate(single["sum_x"], single["sum_x2"], K_TOTAL, int(pre[-1]))
    assert merged["estimate"] == pytest.approx(est, rel=1e-12)
    assert big == [world * (1 << 100) + sum(range(world))]


def test_rank_ranges_partition():
    from paper_2409_08975_gb300 import dist as tcdist
    for k, world in ((10, 3), (7, 7), (5, 8), (10 ** 9 + 7, 6)):
        ranges = [tcdist.rank_range(k, r, world) for r in range(world)]
        assert ranges[0][0] == 0
        for (o1, c1), (o2, c2) in zip(ranges, ranges[1:]):
            assert o1 + c1 == o2
        assert sum(c for _, c in ranges) == k
