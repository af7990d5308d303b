"""The N > 1 path of bench.py on CPU: two gloo ranks.

The method shards by independent replicas (no exchange step), so the only
multi-rank logic is the replica seeding, the max-over-ranks time, the
whole-job throughput and the oracle arm run by rank 0 alone; these run here
with world_size 2 over gloo."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    t = bench.max_over_ranks(10.0 + 5.0 * rank)      # the slower rank defines the job time
    seed = bench.replica_seed(12345, r)
    value = bench.job_throughput(8000 * 256, 4, ws, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ws, r, t, seed, value))


def test_two_gloo_ranks_max_time_and_replica_seeds():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ws0, _, t0, s0, v0), (r1, ws1, _, t1, s1, v1) = out
    assert ws0 == ws1 == 2
    assert t0 == t1 == pytest.approx(15.0)           # max over ranks
    assert s0 != s1                                    # independent replicas
    assert v0 == v1 == pytest.approx(2 * 8000 * 256 * 4 / 0.015)


def _ref_worker(rank, world, port, q):
    import contextlib
    import io
    import types
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    buf = io.StringIO()
    args = types.SimpleNamespace(workload="mgo8000", ncell=10, steps=1, warmup=0)
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, buf.getvalue()))


def test_reference_arm_prints_on_rank_zero_only():
    # under torchrun the oracle arm runs on rank 0 alone; the other ranks exit without work
    import json
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_ref_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[1] == ""
    line = json.loads(out[0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["cores"] >= 1
