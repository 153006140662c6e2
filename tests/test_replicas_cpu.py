"""Replicas-only multi-GPU path, host logic on CPU: two gloo ranks under
torch.distributed.run agree on the slowest rank's time and on the whole-job rate, and the
reference arm does no work on ranks other than 0."""
import json
import os
import socket
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_max_time_and_rate():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", os.path.join(ROOT, "tests", "replica_worker.py")]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout  # rank 0 alone prints
    res = json.loads(lines[0])
    assert res["world"] == 2 and res["seconds"] == 3.0
    assert abs(res["rate"] - 2 * 100.0 * 4 / 3.0) < 1e-9


def test_single_rank_helpers():
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.whole_job_rate(10.0, 3, 2.0, 1) == 15.0


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, eps = 1, 0, 1e-9
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
