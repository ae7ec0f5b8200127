"""The multi-rank path of bench.py on the CPU: world_size 2 over gloo (no GPU).

Every rank runs its own replica of the workload (weak scaling, no data-path
collective); the ranks meet only in barriers and in the max-over-ranks timing, and the
reported value is the whole job's seconds per solve."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


_WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import bench
dist = bench.dist_init("gloo")
ws, rank, _ = bench.dist_env()
assert dist is not None and ws == 2
# each rank times its own replica; the slower one decides
ms = bench.dist_max(dist, 100.0 + 50.0 * rank, "cpu")
assert ms == 150.0, ms
value = bench.whole_job_seconds_per_solve(ms, steps=3, solves_per_step=4, world_size=ws)
assert abs(value - 0.150 / 24) < 1e-15, value
dist.barrier()
dist.destroy_process_group()
print("rank", rank, "ok", flush=True)
"""


def test_two_gloo_ranks_take_the_max_and_report_the_whole_job():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", _WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    outs = []
    for p in procs:
        try:
            out, _ = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            p.kill()
            out, _ = p.communicate()
        outs.append((p.returncode, out))
    for rank, (rc, out) in enumerate(outs):
        assert rc == 0, out
        assert f"rank {rank} ok" in out


def test_single_rank_needs_no_process_group():
    assert bench.dist_init("gloo") is None or int(os.environ.get("WORLD_SIZE", "1")) > 1
    assert bench.dist_max(None, 12.5, "cpu") == 12.5
    assert bench.whole_job_seconds_per_solve(400.0, 2, 4, 1) == pytest.approx(0.05)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.run_reference(bench.parse()) == 0


def test_reference_arm_prints_the_contract_line():
    """Rank 0 of the reference arm times the oracle and prints one JSON line with the
    keys the benchmark contract names (a small grid keeps it to a second or two)."""
    import json
    env = dict(os.environ, WORLD_SIZE="1", RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--m1", "15", "--nt", "16"], capture_output=True, text=True,
                         timeout=300, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is False
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["m1"] == 15 and d["config"]["n"] == 16
