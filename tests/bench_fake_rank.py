"""One rank of bench.py's own arm on the CPU, for tests/test_bench_dist.py.

The GPU pieces are replaced by host fakes before the benchmark's main() runs:
the process group is gloo, the rank's device is the CPU, CUDA events are
host clocks, and Solver returns fixed iteration counts.  Everything else --
argument parsing, the rank launcher's environment, barriers, the max over
ranks and the whole-job value -- is the benchmark's own code.  Each rank
prints a marker line with its rank and world size."""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

import bench  # noqa: E402
import paper_2410_22686_gb300 as pkg  # noqa: E402
from paper_2410_22686_gb300 import build as pbuild  # noqa: E402

SOLVE_S = 0.01 * (1 + int(os.environ.get("RANK", "0")))  # rank 1 is the slower one


class FakeEvent:
    def __init__(self, enable_timing=True):
        self.t = 0.0

    def record(self, *a):
        self.t = time.perf_counter()

    def elapsed_time(self, other):
        return 1000.0 * (other.t - self.t)


class FakeSolver:
    def __init__(self, dim, m1, n, *a, **k):
        self.len = 2 * n * m1 ** dim
        self.launches = 0

    def build_rhs(self, f, g, y0):
        return torch.ones(self.len, dtype=torch.float64)

    def solve(self, b, rtol=1e-8, raise_on_nonconv=True, **k):
        time.sleep(SOLVE_S)
        self.launches += 10
        return b, 7, 1e-9

    def stats_reset(self):
        self.launches = 0

    def profile(self, on=True, classes=None):
        pass

    def launch_count(self):
        return self.launches

    def stats(self):
        return {"arnoldi_dot": {"launches": 7, "ms": 1.0, "bytes": 8.0e9, "flops": 1.0e9},
                "arnoldi_update_norm": {"launches": 7, "ms": 0.5, "bytes": 8.0e9, "flops": 1.0e9}}

    def residual_history(self):
        return [1.0, 1e-9]

    def apply_precond(self, v, out=None):
        return out

    def close(self):
        pass


bench.BACKEND = "gloo"
bench.rank_device = lambda local: torch.device("cpu")
pkg.Solver = FakeSolver
pkg.measure_peaks = lambda: (1.0, 60.0)
pbuild.build = lambda *a, **k: None
torch.cuda.Event = FakeEvent
torch.cuda.synchronize = lambda *a, **k: None
torch.cuda.empty_cache = lambda *a, **k: None

ws, rank, _ = bench.dist_env()
print(f"fake rank {rank} of {ws}", file=sys.stderr, flush=True)
sys.argv = ["bench.py", *sys.argv[1:]]
sys.exit(bench.main())
