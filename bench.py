"""Benchmark: preconditioned GMRES solve time on the 2D variable-coefficient
workload (255 x 255 interior grid, n = 256 time blocks, T = 1,
a = 1 + 0.5 sin(2 pi x1) cos(2 pi x2), eps = sqrt(tau), 16-mode target, f = 0,
y0 = 0), gamma in {1e-2, 1e-4, 1e-6, 1e-8}: FP32 preconditioner inside flexible
GMRES (FP64 Arnoldi, Givens, matvec and true residual) against the plain FP64
solve, to a relative residual of 1e-8.

One step = the four gamma solves of the mixed-precision path, right-hand
sides resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the CPU oracle (plain numpy FP64) on the machine's host
cores on a bounded sample of the same workload.

Beyond the contract keys (metric, value, unit, n_gpus, steps, warmup, ms_per_step,
higher_is_better, scaling, vs_baseline, dtype, data, config, roofline, cpu_baseline,
clocks, e2e, gpu_launches) the line carries: fp64_solve_s, mixed_graph_solve_s (the
same solves as one CUDA-graph launch each), bf16_storage_solve_s, iteration counts and
final residuals, residual_history_mixed, unknowns_iters_per_s, precond_apply (GB/s of
the preconditioner alone), kernel_breakdown (CUDA-event time per kernel class in the
timed region) and other_workloads (3D random field with its kernel breakdown,
constant-coefficient sine-transform solves with finite differences and elements, one
gradient, the 64-problem batch).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# the oracle runs single-threaded (numpy FFT and elementwise code are; pin BLAS too)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

METRIC = "GMRES solve time to 1e-8 rel. residual, mixed vs FP64; precond-apply HBM GB/s"
GAMMAS = (1e-2, 1e-4, 1e-6, 1e-8)
M1, NT = 255, 256
RTOL = 1e-8
# Iterations reported by the paper for its variable-coefficient example at the same
# number of unknowns (h = tau = 2^-8, gamma = 1e-4; Table 6): used only to scale the
# oracle's per-iteration time to a solve in the reference arm.
PAPER_ITERS_H8 = 15


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cap", type=int, default=60, help="Krylov basis capacity")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # smaller cases for profiling runs (the default is the benchmark workload)
    ap.add_argument("--m1", type=int, default=255)
    ap.add_argument("--nt", type=int, default=256)
    ap.add_argument("--gammas", default=",".join(str(g) for g in GAMMAS))
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-bf16", action="store_true")
    ap.add_argument("--skip-3d", action="store_true")
    ap.add_argument("--skip-grad", action="store_true")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-fst", action="store_true")
    ap.add_argument("--skip-graph", action="store_true")
    ap.add_argument("--batch-gb", type=float, default=110.0, help="device memory per batched wave (GB)")
    a = ap.parse_args()
    a.gammas = tuple(float(x) for x in a.gammas.split(","))
    return a


def workload_config(m1=M1, nt=NT, gammas=GAMMAS):
    vec_mb = 2 * m1 * m1 * nt * 8 / 1e6
    return {"workload": f"2D variable-a parabolic control, {m1}x{m1} grid, n={nt} time blocks, "
                        f"gamma in {{{','.join(f'{g:g}' for g in gammas)}}}, eps=sqrt(tau), rtol 1e-8",
            "m1": m1, "n": nt, "dim": 2, "unknowns_per_solve": 2 * m1 * m1 * nt,
            "gammas": list(gammas), "rtol": RTOL,
            "l2": f"inputs larger than L2 (each all-at-once vector is {vec_mb:.0f} MB)" if vec_mb > 129
                  else f"vectors of {vec_mb:.0f} MB: not larger than L2"}


# ----------------------------------------------------------------------------- distributed helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(backend):
    import torch.distributed as dist
    ws, rank, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=ws)
    return dist if ws > 1 else None


def whole_job_seconds_per_solve(max_ms, steps, solves_per_step, world_size):
    """Seconds per solve over the whole job: every rank ran steps x solves_per_step
    independent solves (its own replica of the workload) within the slowest rank's time."""
    return max_ms / 1000.0 / (steps * solves_per_step * world_size)


def dist_max(dist, value, device):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_sum(dist, value, device):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard_by_work(costs, rank, world_size):
    """Indices of the independent problems rank `rank` solves: largest cost first, each
    to the least-loaded rank (ties to the lower rank).  Every rank computes the same
    assignment, so no collective is needed."""
    load = [0.0] * world_size
    owner = [0] * len(costs)
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world_size), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += costs[i]
    return [i for i in range(len(costs)) if owner[i] == rank]


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for ln in fh:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names[1:], parts[5:9]):
                    if v.lower() in ("active", "0x1") or v == "1":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle timing
def oracle_iteration_seconds(gamma=1e-4, m1=M1, nt=NT):
    """Time one right-preconditioned (flexible) GMRES iteration of the CPU oracle on
    the full workload: P_eps^{-1} v (FFT, one V-cycle per shifted system, inverse
    FFT), A z, and the Gram-Schmidt step against the first basis vector."""
    import synthetic as S
    from oracle import precond as opc, system as osy
    prob = S.variable_2d_problem(gamma=gamma, m1=m1, n=nt)
    tau, alpha = prob.tau, osy.alpha_weight(prob.T, prob.n, gamma)
    b = osy.build_rhs(prob.f, prob.g, prob.y0, tau, gamma)
    mg = opc.MGSpatialSolver(prob.a_nodes, tau)
    t0 = time.perf_counter()
    v = b / np.linalg.norm(b)
    z = opc.apply_Peps_inv(v, prob.n, alpha, prob.eps, mg)
    w = osy.apply_A(z, prob.a_nodes, tau, alpha)
    h = float(np.vdot(w.ravel(), v.ravel()))
    w = w - h * v
    _ = np.linalg.norm(w)
    return time.perf_counter() - t0


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_iteration_seconds(m1=args.m1, nt=args.nt)
    times = [oracle_iteration_seconds(m1=args.m1, nt=args.nt) for _ in range(args.steps)]
    per_iter = statistics.median(times)
    value = per_iter * PAPER_ITERS_H8
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s/solve",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * statistics.mean(times), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.m1, args.nt, args.gammas),
        "cpu_baseline": {"value": value, "unit": "s/solve", "cores": 1, "kind": "oracle",
                         "sample": f"one oracle GMRES iteration (preconditioner apply, matvec, one Gram-Schmidt "
                                   f"step) on the full workload at gamma=1e-4 per step, median of {args.steps}, "
                                   f"times {PAPER_ITERS_H8} iterations (the paper's count at this size)"},
        "e2e": {"value": value, "unit": "s/solve", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def _e2e(args, sols, rhs, gammas, torch):
    """Same metric through the public host-buffer call (copies inside the timed region)."""
    hb = [torch.empty(b.shape, dtype=torch.float64, pin_memory=True) for b in rhs]
    for h_, b in zip(hb, rhs):
        h_.copy_(b)
    hx = [torch.empty(b.shape, dtype=torch.float64, pin_memory=True) for b in rhs]
    from paper_2410_22686_gb300 import solve_host_pipelined
    jobs = list(zip(sols, hb, hx))
    solve_host_pipelined(jobs, rtol=RTOL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solve_host_pipelined(jobs, rtol=RTOL)
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / (args.steps * len(gammas))


def _extra_workloads(args, torch, dev, dist=None, ws=1, rank=0):
    """Timed extras on the other workloads of the path (not part of `value`).  With
    several ranks the batched workload's problems are split between them (they are
    independent); the other extras run as one replica per rank."""
    import synthetic as S
    from paper_2410_22686_gb300 import Batch, Solver
    from paper_2410_22686_gb300 import autograd as pag
    out = {}

    def sync_time(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = None
        for _ in range(reps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0 / reps, r

    if not args.skip_3d:
        p = S.gaussian_field_3d_problem()
        res = {}
        for prec in ("fp32", "bf16s", "fp64"):
            sol = Solver(3, p.m1, p.n, p.T, p.gamma, p.eps, p.a_nodes, spatial="mg", precision=prec, max_iter=60)
            b = sol.build_rhs(torch.from_numpy(p.f).to(dev), torch.from_numpy(p.g).to(dev),
                              torch.from_numpy(p.y0).to(dev))
            t, r = sync_time(lambda: sol.solve(b, rtol=RTOL, raise_on_nonconv=False), 2)
            res[prec] = {"solve_s": t, "iters": r[1], "relres": r[2]}
            if prec == "fp32":  # per-kernel CUDA-event breakdown of one more solve
                sol.stats_reset()
                sol.profile(True)
                sol.solve(b, rtol=RTOL, raise_on_nonconv=False)
                torch.cuda.synchronize()
                sol.profile(False)
                st = sol.stats()
                tot = sum(v["ms"] for v in st.values()) or 1.0
                res[prec]["kernel_breakdown"] = {
                    k: {"share": v["ms"] / tot, "avg_us": 1000 * v["ms"] / v["launches"],
                        "gbs": v["bytes"] / (v["ms"] * 1e-3) / 1e9 if v["ms"] else None}
                    for k, v in sorted(st.items(), key=lambda kv: -kv[1]["ms"])[:8] if v["launches"]}
            sol.close()
            del b
            torch.cuda.empty_cache()
        out["grf_3d_63cubed_n128"] = {"unknowns": p.unknowns, "gamma": p.gamma, **res}

    if not args.skip_fst:
        # constant a: sine-transform solves, finite differences and bilinear finite elements
        p = S.example1_problem(M1, NT, 1e-4)
        eps = math.sqrt(p.tau)
        res = {}
        for space in ("fd", "fe"):
            for prec in ("fp32", "fp64"):
                sol = Solver(2, p.m1, p.n, p.T, p.gamma, eps, None, spatial="fst", precision=prec, max_iter=60,
                             space=space)
                b = sol.build_rhs(torch.from_numpy(p.f).to(dev), torch.from_numpy(p.g).to(dev),
                                  torch.from_numpy(p.y0).to(dev))
                t, r = sync_time(lambda: sol.solve(b, rtol=RTOL, raise_on_nonconv=False), 2)
                res[f"{space}_{prec}"] = {"solve_s": t, "iters": r[1], "relres": r[2]}
                sol.close()
                del b
                torch.cuda.empty_cache()
        out["const_a_fst_255sq_n256"] = {"data": "Example 1 fields, a = 1, gamma 1e-4, eps = sqrt(tau)",
                                         "fd": "finite differences (M = I)",
                                         "fe": "bilinear finite elements (mass matrix M)", **res}

    if not args.skip_grad:
        p = S.gradient_problem()
        sol = Solver(2, p.m1, p.n, p.T, p.gamma, p.eps, p.a_nodes, spatial="mg", precision="fp64", max_iter=80)
        g = torch.from_numpy(p.g).to(dev)
        la0 = torch.from_numpy(np.log(p.a_nodes[1:-1, 1:-1]).copy()).to(dev)

        def grad_once():
            la = la0.clone().requires_grad_(True)
            gg = g.clone().requires_grad_(True)
            x = pag.solve(sol, la, gg, rtol=1e-10)
            J = pag.objective(x, gg, sol)
            J.backward()
            return J.item()

        t, _ = sync_time(grad_once, 2)
        out["gradient_127sq_n128"] = {"seconds_per_gradient": t, "params": p.m1 * p.m1 + p.g.size,
                                      "includes": "set_log_coefficient, forward solve (1e-10), objective, "
                                                  "objective gradient, coefficient reset, adjoint solve, "
                                                  "stencil derivative, target gradient"}
        sol.close()
        torch.cuda.empty_cache()

    if not args.skip_batched:
        all_probs = S.batched_problems(64)
        probs = [all_probs[i] for i in shard_by_work([q.unknowns for q in all_probs], rank, ws)]
        cap = 48
        waves, cur, cur_b = [], [], 0.0
        for q in probs:
            need = q.unknowns * (12.0 * cap + 60.0) / 1e9
            if cur and cur_b + need > args.batch_gb:
                waves.append(cur)
                cur, cur_b = [], 0.0
            cur.append(q)
            cur_b += need
        if cur:
            waves.append(cur)
        t_batch, t_seq, iters, rels, unk_it = 0.0, 0.0, [], [], 0.0
        for wave in waves:
            sols, bs = [], []
            for q in wave:
                so = Solver(2, q.m1, q.n, q.T, q.gamma, q.eps, q.a_nodes, spatial="mg", precision="fp32",
                            max_iter=cap)
                bs.append(so.build_rhs(torch.from_numpy(q.f).to(dev), torch.from_numpy(q.g).to(dev),
                                       torch.from_numpy(q.y0).to(dev)))
                sols.append(so)
            bt = Batch(sols, bs, rtol=RTOL, maxit=cap)
            tb, r = sync_time(lambda: bt.solve(raise_on_nonconv=False), 2)
            t_batch += tb
            iters += r[0]
            rels += r[1]
            unk_it += sum(q.unknowns * it for q, it in zip(wave, r[0]))

            def seq():
                for so, bb in zip(sols, bs):
                    so.solve(bb, rtol=RTOL, raise_on_nonconv=False)

            ts, _ = sync_time(seq, 1)
            t_seq += ts
            bt.close()
            for so in sols:
                so.close()
            del bs, sols
            torch.cuda.empty_cache()
        # the job ends when the slowest rank's share is done
        t_batch = dist_max(dist, t_batch, dev)
        t_seq = dist_max(dist, t_seq, dev)
        unk_it = dist_sum(dist, unk_it, dev)
        conv = int(dist_sum(dist, float(sum(1 for r in rels if r <= RTOL)), dev))
        max_it = int(dist_max(dist, float(max(iters) if iters else 0), dev))
        out["batched_64"] = {"problems": len(all_probs), "ranks": ws, "waves": len(waves), "batch_seconds": t_batch,
                             "sequential_seconds": t_seq, "speedup": t_seq / t_batch if t_batch else None,
                             "unknowns_iters_per_s": unk_it / t_batch if t_batch else None,
                             "total_unknowns": sum(q.unknowns for q in all_probs), "max_iters": max_it,
                             "converged": conv,
                             "how": "each wave is one graph launch (pc_batch_solve), FP32 preconditioner; "
                                    "sequential = the same problems one host-driven solve after another; "
                                    "with several ranks each takes a share balanced by size, times are the "
                                    "slowest rank's"}
    return out


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init("nccl")
    import synthetic as S
    from paper_2410_22686_gb300 import Solver
    from paper_2410_22686_gb300 import build as pbuild
    pbuild.build()

    GAM = args.gammas
    probs = [S.variable_2d_problem(gamma=g, m1=args.m1, n=args.nt) for g in GAM]
    U = probs[0].unknowns
    f = torch.from_numpy(probs[0].f).to(dev)
    y0 = torch.from_numpy(probs[0].y0).to(dev)

    def make(precision):
        sols, rhs = [], []
        for p in probs:
            s = Solver(2, args.m1, args.nt, p.T, p.gamma, p.eps, p.a_nodes, spatial="mg", precision=precision,
                       max_iter=args.cap)
            rhs.append(s.build_rhs(f, torch.from_numpy(p.g).to(dev), y0))
            sols.append(s)
        torch.cuda.synchronize()
        return sols, rhs

    def step(sols, rhs, record):
        for s, b in zip(sols, rhs):
            x, it, rr = s.solve(b, rtol=RTOL, raise_on_nonconv=False)
            record.append((it, rr))

    def timed(sols, rhs, steps, warmup, profile=False):
        for _ in range(warmup):
            step(sols, rhs, [])
        for s in sols:
            s.stats_reset()
            s.profile(profile)
        rec = []
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step(sols, rhs, rec)
        e1.record()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clocks = clk.stop()
        ms = dist_max(dist, e0.elapsed_time(e1), dev)
        for s in sols:
            s.profile(False)
        return ms, rec, clocks

    # ---------------- mixed precision (the timed headline)
    sols, rhs = make("fp32")
    ms_mixed, rec_mixed, clocks = timed(sols, rhs, args.steps, args.warmup, profile=True)
    launches = sum(s.launch_count() for s in sols)
    stats = {}
    for s in sols:
        for k, v in s.stats().items():
            a = stats.setdefault(k, {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0})
            for q in a:
                a[q] += v[q]
    iters_mixed = [it for it, _ in rec_mixed[: len(GAM)]]
    relres_mixed = [rr for _, rr in rec_mixed[: len(GAM)]]
    # whole job: every rank runs its own replica of the four solves (weak scaling)
    value = whole_job_seconds_per_solve(ms_mixed, args.steps, len(GAM), ws)

    # the Givens residual estimates of the last timed solve at the second gamma
    s0 = sols[min(1, len(sols) - 1)]
    history = [float(f"{r:.3e}") for r in s0.residual_history()]

    # precond-apply GB/s (mixed): the apply alone, on the same handle and launch configuration
    v = torch.randn(U, dtype=torch.float64, device=dev)
    w = torch.empty_like(v)
    for _ in range(3):
        s0.apply_precond(v, out=w)
    s0.stats_reset()
    reps = 10
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ea.record()
    for _ in range(reps):
        s0.apply_precond(v, out=w)
    eb.record()
    torch.cuda.synchronize()
    pstats = s0.stats()
    p_bytes = sum(x["bytes"] for x in pstats.values()) / reps
    p_ms = ea.elapsed_time(eb) / reps
    precond_gbs = p_bytes / (p_ms * 1e-3) / 1e9

    # ---------------- the same four solves, each one CUDA-graph launch (device-side stop)
    graph_s = None
    if not args.skip_graph:
        xg = [torch.empty_like(b) for b in rhs]
        for s, b, x in zip(sols, rhs, xg):  # capture and one replay each
            s.solve_graph(b, x, rtol=RTOL, raise_on_nonconv=False)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ga.record()
        for s, b, x in zip(sols, rhs, xg):
            s.solve_graph(b, x, rtol=RTOL, raise_on_nonconv=False)
        gb.record()
        torch.cuda.synchronize()
        graph_s = whole_job_seconds_per_solve(dist_max(dist, ga.elapsed_time(gb), dev), 1, len(GAM), ws)
        del xg

    # ---------------- end to end through host buffers (same metric)
    e2e_s = None
    if not args.skip_e2e:
        e2e_rank = _e2e(args, sols, rhs, GAM, torch)  # seconds per solve on this rank
        if dist is not None:
            dist.barrier()
        e2e_s = dist_max(dist, e2e_rank, dev) / ws
    for s in sols:
        s.close()
    del sols
    torch.cuda.empty_cache()

    # ---------------- plain FP64 solve (comparison)
    fp64_s, iters64 = None, None
    if not args.skip_fp64:
        sols64, rhs64 = make("fp64")
        ms64, rec64, _ = timed(sols64, rhs64, args.steps, 1)
        iters64 = [it for it, _ in rec64[: len(GAM)]]
        fp64_s = whole_job_seconds_per_solve(ms64, args.steps, len(GAM), ws)
        for s in sols64:
            s.close()
        del sols64

    # ---------------- BF16-storage smoother variant (FP32 arithmetic)
    bf16_s, iters_bf16 = None, None
    if not args.skip_bf16:
        solsb, rhsb = make("bf16s")
        msb, recb, _ = timed(solsb, rhsb, args.steps, 1)
        iters_bf16 = [it for it, _ in recb[: len(GAM)]]
        bf16_s = whole_job_seconds_per_solve(msb, args.steps, len(GAM), ws)
        for s in solsb:
            s.close()
        del solsb
        torch.cuda.empty_cache()

    # ---------------- the other workloads of the path
    extras = _extra_workloads(args, torch, dev, dist, ws, rank)

    # ---------------- roofline of the dominant kernel class
    # DRAM bytes (read + write) over algorithmic bytes of one launch, from the ncu
    # capture summarised in profiles/kernels_gmres_mixed_255x255_n128.md (255^2 x 128,
    # four basis vectors); a full-size launch moves the same bytes per unknown, so the
    # traffic of the average timed launch is this ratio times its algorithmic bytes
    ncu_traffic_ratio = {"arnoldi_dot": (665.9 + 4.0) / 665.8, "arnoldi_update_norm": (665.9 + 176.8) / 865.6}
    tot_ms = sum(v["ms"] for v in stats.values())
    dom_name, dom = max(stats.items(), key=lambda kv: kv[1]["ms"])
    peaks, peak_src = {}, "fallback 6.8 TB/s (of fallback)"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
        peak_src = "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    fp64_peak_tflops = 152 * 2 * 2 * 2.07e9 / 1e12     # 2 FP64 FMA/clk/SM at 2070 MHz
    dom_avg_ms = dom["ms"] / max(dom["launches"], 1)
    dom_bytes = dom["bytes"] / max(dom["launches"], 1)
    dom_flops = dom["flops"] / max(dom["launches"], 1)
    gbs = dom_bytes / (dom_avg_ms * 1e-3) / 1e9
    tfl = dom_flops / (dom_avg_ms * 1e-3) / 1e12
    if dom_name in ("arnoldi_dot", "arnoldi_update_norm", "matvec", "x_update") and tfl / fp64_peak_tflops > gbs / hbm_peak:
        roof = {"bound": "alu", "achieved": tfl, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                "frac": tfl / fp64_peak_tflops, "traffic": None, "kernel": dom_name,
                "peak_source": "FP64: 152 SMs x 2 FMA/clk x 2 flop x 2070 MHz (derived)",
                "hbm_achieved_gbs": gbs, "hbm_frac": gbs / hbm_peak}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "traffic": None, "kernel": dom_name, "peak_source": peak_src}
    if dom_name in ncu_traffic_ratio:
        roof["traffic"] = ncu_traffic_ratio[dom_name] * dom_bytes
        roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the same kernel at "
                                  "255^2 x 128 (profiles/kernels_gmres_mixed_255x255_n128.md), scaled to "
                                  "this launch by its algorithmic bytes")
    roof["share_of_kernel_time"] = dom["ms"] / tot_ms if tot_ms else None
    breakdown = {k: {"share": v["ms"] / tot_ms if tot_ms else None, "launches": v["launches"],
                     "avg_us": 1000 * v["ms"] / v["launches"] if v["launches"] else None,
                     "gbs": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] else None}
                 for k, v in sorted(stats.items(), key=lambda kv: -kv[1]["ms"]) if v["launches"]}

    line = {
        "metric": METRIC, "value": value, "unit": "s/solve", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": workload_config(args.m1, args.nt, GAM),
        "fp64_solve_s": fp64_s, "mixed_solve_s": value, "mixed_graph_solve_s": graph_s,
        "mixed_speedup_vs_fp64": (fp64_s / value) if fp64_s else None,
        "bf16_storage_solve_s": bf16_s, "iters_bf16_storage": iters_bf16,
        "iters_mixed": iters_mixed, "iters_fp64": iters64, "relres_mixed": relres_mixed,
        "residual_history_mixed": {"gamma": GAM[min(1, len(GAM) - 1)], "estimates": history},
        "unknowns_iters_per_s": ws * sum(U * it for it in iters_mixed) / (ms_mixed / 1000.0 / args.steps),
        "precond_apply": {"gbs": precond_gbs, "ms": p_ms, "frac_of_hbm": precond_gbs / hbm_peak,
                          "bytes": p_bytes, "precision": "fp32"},
        "roofline": roof, "kernel_breakdown": breakdown, "other_workloads": extras,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": {"value": e2e_s, "unit": "s/solve", "h2d_bytes_per_step": 8 * U * len(GAM) * ws,
                "d2h_bytes_per_step": 8 * U * len(GAM) * ws,
                "how": "solve_host_pipelined: pinned host b -> device, GMRES, device x -> pinned host for each "
                       "of the step's solves, the copies of the next b and the previous x on a second stream "
                       "during the current solve"},
    }
    if rank == 0 and not args.no_cpu_baseline:
        t_iter = oracle_iteration_seconds(m1=args.m1, nt=args.nt)
        mean_it = sum(iters_mixed) / len(iters_mixed)
        line["cpu_baseline"] = {"value": t_iter * mean_it, "unit": "s/solve", "cores": 1, "kind": "oracle",
                                "sample": "one oracle GMRES iteration (preconditioner apply, matvec, one "
                                          "Gram-Schmidt step) on the full workload at gamma=1e-4, times the "
                                          f"mean GPU iteration count {mean_it:.1f}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
