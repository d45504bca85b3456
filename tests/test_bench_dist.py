"""Host-side checks of the benchmark's multi-rank path on CPU: two ranks on
the gloo backend (127.0.0.1) run the rank setup, the max-over-ranks timing
reduction and the whole-job throughput that the N-GPU run uses (replicas:
every rank processes its own cube, no data exchange), and the reference arm
does its work on rank 0 only."""

import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist, w, r, local = bench._dist_setup(world, backend="gloo")
    # rank-dependent timings: the job's time is the slowest rank's
    mine = [10.0 + 4.0 * rank, 3.0 - rank]
    got = bench._max_over_ranks(dist, mine, "cpu")
    rate = bench._job_rate(w, 1.0e6, 5, got[0])
    out.put((r, w, local, got, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reduce_timings_and_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for pr in procs:
        pr.start()
    results = sorted(out.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert [res[0] for res in results] == [0, 1]
    for r, w, local, got, rate in results:
        assert w == 2 and local == r
        assert got == [14.0, 3.0]
        # 2 ranks x 1e6 units x 5 steps in 14 ms
        assert rate == pytest.approx(2 * 1.0e6 * 5 / 0.014 / 1e6)


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    dist, w, r, local = bench._dist_setup(1)
    assert dist is None and (w, r) == (1, 0)
    assert bench._max_over_ranks(None, [2.5, 7], "cpu") == [2.5, 7.0]
    assert bench._job_rate(1, 95737680, 10, 11.53) == pytest.approx(
        95737680 * 10 / 0.01153 / 1e6)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    """Under torchrun with N > 1 only rank 0 times the oracle and prints."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = SimpleNamespace(steps=1, warmup=0, cpu_cols=8, gpus=2)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""


@pytest.mark.slow
def test_reference_arm_rank0_line(monkeypatch):
    """Rank 0 of a two-rank reference run prints one JSON line for the job."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "0")
    args = SimpleNamespace(steps=1, warmup=0, cpu_cols=32, gpus=2)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["unit"] == "Mvoxel/s" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
