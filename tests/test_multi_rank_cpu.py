"""The N-replica path of bench.py on CPU: two gloo ranks (127.0.0.1).

Checks the max-over-ranks job time, the whole-job throughput (every replica
solves its own RHS block), distinct per-replica sources, and that only rank 0
runs and prints the reference arm.  No GPU and no compute call.
"""
import multiprocessing as mp
import os
import socket

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = [1.5, 2.5][rank]
        t_job = bench.max_over_ranks(t_local, world, "cpu")
        value = bench.job_throughput(48, 5, world, t_job)
        seed = bench.replica_source_seed(dict(bench.WORKLOAD), rank)
        dist.barrier()
        q.put((rank, t_job, value, seed))
    finally:
        dist.destroy_process_group()


def test_two_replicas_time_is_the_slowest_rank_and_value_counts_both():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    (r0, t0, v0, s0), (r1, t1, v1, s1) = got
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 2.5                       # the slowest rank sets the job time
    assert v0 == v1 == 48 * 5 * 2 / 2.5          # both replicas' RHS counted
    assert s0 != s1                              # each replica solves its own sources


def test_single_rank_helpers():
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.job_throughput(48, 5, 1, 2.0) == 120.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class A:
        steps, warmup = 1, 0
    bench.run_reference(A(), rank=1, world=2)    # returns before any work
    assert capsys.readouterr().out == ""
