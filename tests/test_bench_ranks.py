"""bench.py's multi-rank host logic on CPU, with world-size-2 gloo ranks.

Under torchrun each rank runs one replica of the workload (the path has no
data-path collective); the job's time is the slowest rank's, its value counts
every rank's atom-steps, and the reference arm runs on rank 0 alone.
"""
import json
import os
import socket
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, str(ROOT))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(times[rank], world, "cpu")
    v = bench.whole_job_value(1000, 10, world, t)
    dist.destroy_process_group()
    Path(out_dir, f"rank{rank}.json").write_text(json.dumps({"t": t, "v": v}))


def test_slowest_rank_sets_the_job_time_gloo(tmp_path):
    import torch.multiprocessing as mp
    world, times = 2, [2.0, 5.0]
    mp.start_processes(_rank, args=(world, _free_port(), times, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        got = json.loads((tmp_path / f"rank{r}.json").read_text())
        assert got["t"] == 5.0
        assert got["v"] == pytest.approx(1000 * 10 * world / 5e-3)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_value(1_000_000, 1000, 1, 2800.0) == pytest.approx(1e6 * 1000 / 2.8)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, str(ROOT))
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(bench.args_parse()) is None
    assert capsys.readouterr().out == ""
