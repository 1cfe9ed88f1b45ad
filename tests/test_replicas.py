"""The N > 1 path of bench.py runs independent replicas, one per rank, and
aggregates on the host: the time is the maximum over ranks and the work the
sum over ranks.  Checked here with world-size-2 gloo ranks on the CPU (no GPU
involved); the reference arm runs on rank 0 only."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, _ = bench.dist_env()
        t_max = bench.max_over_ranks(1.5 + rank, ws)       # per-rank step times
        work = bench.sum_over_ranks(100.0 * (rank + 1), ws)   # per-rank shift-iterations
        bench.barrier(ws)
        q.put((rank, got_ws, got_rank, t_max, work))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_summed_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, got_rank, t_max, work in out:
        assert ws == 2 and got_rank == rank
        assert t_max == 2.5            # the slowest rank sets the time
        assert work == 300.0           # every rank's work counts
    # value = total work / max time, as bench.py reports it
    assert out[0][4] / out[0][3] == 120.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})(), None) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_line(monkeypatch, capsys):
    """The reference arm on one process: the oracle timed on a bounded sample
    (here the 6^3 x 4 workload, 30 seed iterations) and one JSON line with the
    keys the benchmark contract asks for, its e2e and cpu_baseline equal to
    its own value."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    from paper_0802_0748_gb300 import inputs
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    wl = inputs.workload("anderson", "small")
    real = bench.oracle_sample
    monkeypatch.setattr(bench, "oracle_sample", lambda w, n_shift=16, n_iter=800: real(w, n_shift, 30))
    bench.run_reference(type("A", (), {"steps": 2, "warmup": 1, "gpus": 1})(), wl)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling", "dtype",
                "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["value"] == line["value"] == line["e2e"]["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
