"""bench.py's multi-replica host logic on CPU (gloo, world size 2): every
rank sees the slowest rank's time, the job's throughput counts every
replica's units over that time, and the reference arm runs on rank 0 only.
Also the clock sampler's timed-region window."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank            # rank 1 is the slow one
    got = bench.max_over_ranks(ms, dist, "cpu")
    q.put((rank, got, bench.job_rate(20, world, got)))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in out:
        assert ms == 15.0                       # the slowest rank's time on every rank
        assert abs(rate - 2 * 20 / 0.015) < 1e-9


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert abs(bench.job_rate(10, 1, 100.0) - 100.0) < 1e-12


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun the other ranks exit without work or output."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(None)
    assert buf.getvalue() == ""


def test_clock_samples_inside_the_timed_region():
    """Only samples read inside [mark, stop] count; throttle reasons are
    reported by name; with none inside, the first one after the mark is
    kept.  (Samples are planted by hand: no nvidia-smi process runs.)"""
    sys.path.insert(0, ROOT)
    import time
    import bench
    c = bench.Clocks()
    c.mark()
    t = c.t0
    row = lambda sm, thermal: [str(sm), "2032", "900.0", "Not Active",
                               "Active" if thermal else "Not Active", "Not Active", "Active"]
    c.samples = [(t - 1.0, row(1000, True)),      # before the region: ignored
                 (t + 0.001, row(2032, False)),
                 (t + 0.002, row(2010, False))]
    out = c.stop()
    assert out["samples"] == 2 and out["sm_max_mhz"] == 2032.0
    assert out["sm_mhz"] in (2010.0, 2032.0)
    assert out["reasons"] == ["sw_power_cap"]
    c2 = bench.Clocks()
    c2.mark()
    c2.samples = [(c2.t0 + 10.0, row(1500, True))]   # read after the region ended
    out2 = c2.stop()
    assert out2["samples"] == 1 and out2["sm_mhz"] == 1500.0
    assert out2["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert time.perf_counter() > c2.t0
