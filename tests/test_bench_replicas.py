"""The N > 1 path of bench.py (independent replicas, one per rank) on CPU
with the gloo backend, world size 2: the barrier, the max over ranks of the
timed region, the whole-job rate, and the reference arm printing on rank 0
only.  The GPU work of each replica is that of N = 1."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    # per-rank summed step times: rank 1 is the slow one
    per_step = [10.0 + rank * 5.0, 12.0, 11.0]
    bench.barrier(ws)
    total = bench.reduce_max(sum(per_step), ws, "cpu")
    rate = bench.whole_job_rate(ws, len(per_step), total)
    out.put((r, ws, local, total, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_max_over_ranks_and_aggregate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slow = 10.0 + 5.0 + 12.0 + 11.0
    for r, (rank, ws, local, total, rate) in enumerate(res):
        assert (rank, ws, local) == (r, 2, r)
        assert total == slow                       # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 3 / (slow / 1000.0))


def test_reference_arm_prints_only_on_rank_zero(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = bench.argparse.Namespace(warmup=3, steps=1, ref_cycles=1)
    bench.run_reference(args)                      # rank 1: no work, no output
    assert capsys.readouterr().out == ""


def test_whole_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(1, 20, 400.0) == pytest.approx(50.0)
    assert bench.reduce_max(3.5, 1) == 3.5        # identity without a process group
