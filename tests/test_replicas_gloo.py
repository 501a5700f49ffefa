"""The multi-GPU path of the benchmark runs independent replicas (one
lattice per rank, no data-path collective): ranks meet at barriers around
the timed region and the reported rate uses the slowest rank's time.  This
exercises that logic with two gloo ranks on the CPU."""
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
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port,
                            rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    assert (r, w) == (rank, world)
    bench.barrier(world)
    ms = 10.0 + 5.0 * rank            # rank 1 is the slow replica
    worst = bench.max_over_ranks(ms, world)
    bench.barrier(world)
    dist.destroy_process_group()
    out.put((rank, worst, bench.whole_job_mlups(1000, 20, world, worst)))


def test_two_gloo_replicas_report_the_slowest_rank():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q))
             for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slow rank's 15 ms; 2 x 1000 nodes x 20 steps in
    # 15 ms = 2.667 MLUPS
    assert [w for _, w, _ in res] == [15.0, 15.0]
    assert all(abs(v - 2 * 1000 * 20 / 15e3) < 1e-12 for _, _, v in res)
