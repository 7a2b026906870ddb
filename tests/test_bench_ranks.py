"""The replica path of bench.py on CPU: two gloo ranks combine their timed
milliseconds (the slowest rank) and their rows (the sum), as the benchmark does
over NCCL with one rank per GPU; the reference arm prints only on rank 0."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
rank, world, local = bench.dist_env()
dist.init_process_group("gloo")
t_max, rows = bench.combine_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), world, "cpu")
with open(os.path.join({out!r}, f"rank{{rank}}.json"), "w") as f:  # one file per rank: no interleaved lines
    json.dump({{"rank": rank, "t_max": t_max, "rows": rows}}, f)
dist.destroy_process_group()
"""


def test_two_gloo_ranks_combine_max_time_and_summed_rows(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT, out=str(tmp_path)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=29561", str(script)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=240, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    import json
    lines = [json.loads((tmp_path / f"rank{i}.json").read_text()) for i in range(2)]
    assert sorted(x["rank"] for x in lines) == [0, 1]
    for x in lines:
        assert x["t_max"] == 15.0 and x["rows"] == 3000.0


def test_single_rank_passes_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(12.5, 7, 1, "cpu") == (12.5, 7)


def test_reference_arm_prints_only_on_rank_zero(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload = "pairwise_uniform"
        size = "full"
        steps = 1
        warmup = 1
        gpus = 2

    bench.run_reference(Args)
    assert capsys.readouterr().out == ""
