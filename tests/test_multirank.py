"""The N > 1 path of bench.py as world-size-2 gloo process groups on the CPU: the job's
step time is the maximum over ranks, the value counts every rank's replica apply, each
rank works on its own right-hand side, and under torchrun the reference arm runs on rank
0 only (the other ranks exit without work)."""
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [12.5, 40.0][rank]
    t = bench.reduce_step_time(local_ms, world, dist, device="cpu")
    q.put((rank, t, bench.whole_job_value(2.0e12, world, t), bench.rank_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_and_count_both_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [40.0, 40.0]          # max over ranks, seen by both
    assert out[0][2] == out[1][2] == 2.0e12 * 2 / 0.040  # both replicas' interactions
    assert out[0][3] != out[1][3]                       # independent right-hand sides


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_step_time(7.0, 1, None) == 7.0
    assert bench.whole_job_value(1.0e12, 1, 500.0) == 2.0e12


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"workload": "ball12_k2", "steps": 1, "warmup": 0, "gpus": 2})()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""
