"""Host logic of the multi-GPU bench (replicas: every rank transports its own
packets, no data-path collective), run as two gloo ranks on the CPU: the job's
time is the largest rank time, its events the sum over ranks; rank seeds
differ; the reference arm runs on rank 0 alone."""
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


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]
    ev = [1.0e6, 3.0e6][rank]
    q.put((rank, bench.reduce_over_ranks(ms, ev, dist, device="cpu"), bench.replica_seed(7, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_max_time_summed_events():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got.sort()
    assert [g[1] for g in got] == [(20.0, 4.0e6), (20.0, 4.0e6)]
    assert got[0][2] != got[1][2]


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        workload, packets, steps, warmup = "sphere", 1000, 1, 0
    bench.run_reference(Args(), rank=1, world=2)
    assert capsys.readouterr().out == ""
