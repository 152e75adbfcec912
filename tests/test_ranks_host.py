"""Multi-rank logic of bench.py on the CPU (gloo, world size 2): the path runs replicas, one
per GPU, so the only cross-rank steps are the barrier around the timed region, the maximum
of the per-rank times, and the whole-job rate (all ranks' units / the slowest rank's time);
single-GPU arms (reference, serving, refinement) run on rank 0 and return on the others."""
import json
import os
import socket
import subprocess
import sys
import textwrap
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_job_rate_and_single_rank_max():
    assert bench._max_over_ranks(3.5, 1) == 3.5
    assert bench._job_rate(200, 4, 500.0) == pytest.approx(1600.0)  # 4 x 200 units in 0.5 s


def test_max_over_two_gloo_ranks_under_torchrun(tmp_path):
    """Each rank times a different region; both learn the slowest, and the job rate counts
    every rank's units over that time."""
    script = tmp_path / "ranks.py"
    script.write_text(textwrap.dedent(f"""
        import json, os, sys
        sys.path.insert(0, {ROOT!r})
        import torch.distributed as dist
        import bench
        world, rank, local = bench._dist()
        dist.init_process_group("gloo")
        ms = 100.0 * (rank + 1)              # rank 1 is the slow one
        dist.barrier()
        mx = bench._max_over_ranks(ms, world, device="cpu")
        rate = bench._job_rate(50, world, mx)
        with open(os.path.join({str(tmp_path)!r}, f"rank{{rank}}.json"), "w") as f:  # one file per rank
            json.dump({{"rank": rank, "world": world, "local": local, "max": mx, "rate": rate}}, f)
        dist.destroy_process_group()
    """))
    env = dict(os.environ, PYTHONUNBUFFERED="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), str(script)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=240, env=env, cwd=str(tmp_path))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads((tmp_path / f"rank{q}.json").read_text()) for q in range(2)]
    assert sorted(d["rank"] for d in lines) == [0, 1]
    for d in lines:
        assert d["world"] == 2 and d["local"] == d["rank"]
        assert d["max"] == 200.0
        assert d["rate"] == pytest.approx(2 * 50 / 0.2)


@pytest.mark.parametrize("arm", ["run_reference", "run_serving", "run_refine"])
def test_single_gpu_arms_return_on_other_ranks(arm, monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = SimpleNamespace(workload="sphere_655360", steps=2, warmup=1, serve=4, serve_nmax=20000, serve_kmax=2.0,
                           serve_slots=1, serve_group=1, refine_pmin=12, restart=0)
    assert getattr(bench, arm)(args) is None
    assert capsys.readouterr().out == ""
