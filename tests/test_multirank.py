"""The multi-rank path of the benchmark on CPU (gloo, world size 2): each
rank steps its own boxes with no data-path collective; the whole-job figures
sum the pair-interactions over the ranks and take the slowest rank's times,
and the seeded generators give each rank its own realisation."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    import bench
    pairs = 1000.0 * (rank + 1)
    ms, gf = 10.0 + rank, 4.0 + 2.0 * rank
    tot, ms_max, gf_max = bench.aggregate(world, pairs, ms, gf, "cpu")
    w, name = bench.make_workload("lognormal", 4096, seed=rank)
    out.put((rank, tot, ms_max, gf_max, float(w["x"].sum()), name))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_aggregate_and_own_boxes():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=180) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, tot, ms_max, gf_max, _, name in res:
        assert tot == 3000.0 and ms_max == 11.0 and gf_max == 6.0, (rank, tot, ms_max, gf_max)
        assert name == "lognormal3d_4096_mfv_exact"
    assert res[0][4] != res[1][4]          # different realisations per rank


def _stepping_worker(rank, world, port, out):
    import time
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    import bench
    import oracle
    # each rank steps its own realisation (the oracle stands in for the GPU
    # step here: the same pairs, counted the same way)
    w, _ = bench.make_workload("lognormal", 4096, seed=rank)
    cfg = oracle.config(gamma=w["gamma"])
    t0 = time.perf_counter()
    _, _, info = oracle.step(cfg, w, -1.0)
    ms = 1000.0 * (time.perf_counter() - t0)
    pairs = info["grad_pairs"] + info["flux"]["pairs"]
    tot, ms_max, _ = bench.aggregate(world, pairs, ms, ms, "cpu")
    out.put((rank, pairs, ms, tot, ms_max, info["status"]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_step_their_own_boxes():
    """Both ranks step a box of their own; the whole-job pair count is the sum
    of the two steps' counts and the time the slower rank's."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_stepping_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, p0, ms0, tot0, max0, st0), (_, p1, ms1, tot1, max1, st1) = res
    assert st0 in (0, -5) and st1 in (0, -5)
    assert p0 > 0 and p1 > 0 and p0 != p1          # two realisations, two pair counts
    assert tot0 == tot1 == p0 + p1
    assert max0 == max1 == max(ms0, ms1)


def test_single_rank_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(1, 5.0, 2.0, 1.0, "cpu") == (5.0, 2.0, 1.0)
