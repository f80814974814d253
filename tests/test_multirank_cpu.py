"""The N > 1 host path of bench.py as world-size-2 gloo process groups on the
CPU: ranks shard windows with no exchange, the job's time is the slowest
rank's (MAX all-reduce), the whole-job rate counts every rank's windows, and
under torchrun only rank 0 runs the CPU reference arm."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_env()
    t = bench.reduce_max(10.0 + 5.0 * rank, dist, torch.device("cpu"))  # rank 1 is the slowest
    rate = bench.whole_job_rate(w, 256, 4, t)
    q.put((r, w, bench.first_window(r, 256), t, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, f0, t0, v0), (r1, w1, f1, t1, v1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert (f0, f1) == (0, 256)        # disjoint window ranges, no exchange
    assert t0 == t1 == 15.0            # both ranks see the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 256 * 4 / 0.015)


def test_reference_arm_runs_on_rank_0_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 1, 2

    bench.run_reference(A(), bench.workload("bf16_b256_3x256x128"), rank=1)
    assert capsys.readouterr().out == ""
