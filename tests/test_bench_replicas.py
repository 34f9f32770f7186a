"""The N > 1 path of bench.py on CPU: two gloo ranks (world_size 2) run as
replicas; the job time is the slowest rank's, the rate counts every rank's
units, and the reference arm runs on rank 0 only."""
import io
import os
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank                              # rank 1 is the slower replica
        t = bench.max_over_ranks(ms, world, "cpu")
        rate = bench.whole_job_rate(world, 4, 1000, t)
        dist.barrier()
        out.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == 150.0
        assert rate == pytest.approx(2 * 4 * 1000 / 0.150)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_rate(1, 5, 200, 1000.0) == pytest.approx(1000.0)


def test_reference_arm_rank_nonzero_does_no_work():
    sys.path.insert(0, ROOT)
    import bench
    class A:
        workload = "3p3n_nmax2"; warmup = 3; steps = 2; cpu_rows = 40; gpus = 2
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A, rank=1)
    assert buf.getvalue() == ""


def test_reference_arm_rank_zero_prints_one_line():
    sys.path.insert(0, ROOT)
    import json
    import bench

    class A:
        workload = "3p3n_nmax2"; warmup = 3; steps = 2; cpu_rows = 400; gpus = 1
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A, rank=0)
    lines = buf.getvalue().strip().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "nnz/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_oracle_one_thread_child_process():
    """The single-thread oracle timing runs in a child with OMP_NUM_THREADS=1
    and reports the same kind of sample as the all-core run."""
    sys.path.insert(0, ROOT)
    import bench
    r, n, dt, th = bench.oracle_rate_one_thread("3p3n_nmax2", 200)
    assert th == 1 and n > 0 and dt > 0 and r == pytest.approx(n / dt)
