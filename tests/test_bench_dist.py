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


@pytest.mark.parametrize("ws", [1, 2, 3, 4])
def test_batched_problems_are_split_without_overlap_and_balanced(ws):
    costs = [(i * 37) % 11 + 1.0 for i in range(64)]  # uneven sizes
    shards = [bench.shard_by_work(costs, r, ws) for r in range(ws)]
    flat = sorted(i for sh in shards for i in sh)
    assert flat == list(range(64))  # every problem exactly once
    loads = [sum(costs[i] for i in sh) for sh in shards]
    assert max(loads) - min(loads) <= max(costs)  # greedy largest-first balance
    assert bench.shard_by_work(costs, 0, 1) == list(range(64))  # one rank keeps the order


_SHARD_WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import torch.distributed as td
import bench
dist = bench.dist_init("gloo")
ws, rank, _ = bench.dist_env()
costs = [float((7 * i) % 13 + 1) for i in range(64)]
mine = bench.shard_by_work(costs, rank, ws)
got = [None] * ws
td.all_gather_object(got, mine)
flat = sorted(i for sh in got for i in sh)
assert flat == list(range(64)), flat
assert bench.dist_sum(dist, float(len(mine)), "cpu") == 64.0
dist.barrier()
dist.destroy_process_group()
print("rank", rank, "ok", flush=True)
"""


def test_two_gloo_ranks_take_complementary_shares():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", _SHARD_WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    for rank, p in enumerate(procs):
        out, _ = p.communicate(timeout=120)
        assert p.returncode == 0, out
        assert f"rank {rank} ok" in out


def test_batched_extra_logic_with_fake_solvers(monkeypatch):
    """The batched section of the benchmark on the host: fake solvers and events stand in
    for the GPU, so the wave split, the per-rank share and the reported fields are
    checked without a device (one rank)."""
    import time
    import types

    import torch

    import paper_2410_22686_gb300 as pkg
    import synthetic

    class FakeSolver:
        def __init__(self, dim, m1, n, *a, **k):
            self.len = 2 * n * m1 ** dim

        def build_rhs(self, f, g, y0):
            return torch.ones(self.len, dtype=torch.float64)

        def solve(self, b, rtol=1e-8, raise_on_nonconv=True):
            return b, 7, 1e-9

        def close(self):
            pass

    class FakeBatch:
        def __init__(self, sols, bs, rtol=1e-8, maxit=None):
            self.k = len(sols)

        def solve(self, raise_on_nonconv=True):
            return [7] * self.k, [1e-9] * self.k

        def close(self):
            pass

    class FakeEvent:
        def __init__(self, enable_timing=True):
            self.t = 0.0

        def record(self):
            self.t = time.perf_counter()

        def elapsed_time(self, other):
            return 1000.0 * (other.t - self.t)

    monkeypatch.setattr(pkg, "Solver", FakeSolver)
    monkeypatch.setattr(pkg, "Batch", FakeBatch)
    # Krylov storage of 1000 bytes per problem in a pool of 10 KB: several memory waves
    monkeypatch.setattr(pkg, "krylov_bytes", lambda *a, **k: 1000)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a, **k: (400e9, 400e9))
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    args = types.SimpleNamespace(skip_3d=True, skip_fst=True, skip_fe_var=True, skip_grad=True, skip_batched=False, skip_ideal=True,
                                 batch_gb=1e-5)
    out = bench._extra_workloads(args, torch, "cpu")["batched_64"]
    assert out["problems"] == 64 and out["ranks"] == 1 and out["converged"] == 64 and out["max_iters"] == 7
    assert out["graph_launches"] == 1 and out["batch_seconds"] >= 0.0
    # 64 storages of 1024 bytes (256-byte aligned) in a 10000-byte pool: 9 per wave
    assert out["memory_waves"] == 8 and out["krylov_pool_gb"] == 1e-5
    assert out["total_unknowns"] == sum(q.unknowns for q in synthetic.batched_problems(64))


def test_gpus_flag_starts_the_ranks_itself():
    """`bench.py --gpus 2` without a torchrun environment starts two ranks of one job;
    each runs its replica, rank 0 alone prints the line, n_gpus is 2 and the value is
    the whole job's seconds per solve (slowest rank's time over both ranks' solves)."""
    import json
    env_keep = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        argv = ["--gpus", "2", "--steps", "2", "--warmup", "3", "--m1", "7", "--nt", "4", "--skip-fp64",
                "--skip-e2e", "--skip-bf16", "--skip-3d", "--skip-grad", "--skip-batched", "--skip-fst", "--skip-fe-var",
                "--skip-graph", "--skip-sweep", "--skip-ideal", "--no-cpu-baseline"]
        rc, outs = bench.launch_local_ranks(2, argv, script=os.path.join(ROOT, "tests", "bench_fake_rank.py"),
                                            capture=True, timeout=240)
    finally:
        os.environ.update(env_keep)
    assert rc == 0, outs
    assert "fake rank 0 of 2" in outs[0] and "fake rank 1 of 2" in outs[1]
    lines = [ln for out in outs for ln in out.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1 and lines[0] in outs[0]
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["scaling"] == "weak" and d["steps"] == 2
    # rank 1 sleeps 20 ms per solve: 2 steps x 4 solves = 160 ms at least, over 16 solves
    assert d["value"] >= 0.160 / 16 * 0.99
    assert abs(d["value"] - d["ms_per_step"] * 2 / 1000.0 / 16) <= 1e-12
    assert d["gpu_launches"] == 2 * (2 * 4 * 10)  # both ranks


def test_gpus_flag_under_torchrun_environment_does_not_relaunch(monkeypatch):
    called = []
    monkeypatch.setattr(bench, "launch_local_ranks", lambda *a, **k: called.append(a) or 0)
    monkeypatch.setattr(bench, "run_reference", lambda args: 0)
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--gpus", "2", "--impl", "reference"])
    assert bench.main() == 0 and not called
    monkeypatch.delenv("WORLD_SIZE")
    assert bench.main() == 0 and called and called[0][0] == 2
