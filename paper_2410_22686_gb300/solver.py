"""Python front end over the C ABI: one ``Solver`` per problem.

Tensors are torch float64 CUDA tensors; all-at-once vectors have shape
``(2, n) + (m1,)*dim`` (or any shape with ``2*n*m1**dim`` elements) laid out as
[half][time block][space] with x1 fastest (include/pcopt.h).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import capi, tuning

_SPATIAL = {"auto": capi.PC_SPATIAL_AUTO, "fst": capi.PC_SPATIAL_FST, "mg": capi.PC_SPATIAL_MG}
_PREC = {"fp64": capi.PC_PREC_FP64, "fp32": capi.PC_PREC_MIXED_FP32, "mixed": capi.PC_PREC_MIXED_FP32,
         "bf16s": capi.PC_PREC_MIXED_BF16S, "auto": capi.PC_PREC_AUTO}
_PREC_NAME = {capi.PC_PREC_FP64: "fp64", capi.PC_PREC_MIXED_FP32: "fp32", capi.PC_PREC_MIXED_BF16S: "bf16s"}
_MODE = {"right": capi.PC_GMRES_RIGHT, "left": capi.PC_GMRES_LEFT}
_SPACE = {"fd": capi.PC_SPACE_FD, "fe": capi.PC_SPACE_FE}
_SMOOTHER = {"red-black": capi.PC_SMOOTHER_RED_BLACK, "lexicographic": capi.PC_SMOOTHER_LEXICOGRAPHIC}
_PRECOND = {"eps-circulant": capi.PC_PRECOND_EPS_CIRCULANT, "ideal": capi.PC_PRECOND_IDEAL_RBD}
_ARNOLDI = {"auto": capi.PC_ARNOLDI_AUTO, "fp64": capi.PC_ARNOLDI_FP64, "fp64-strict": capi.PC_ARNOLDI_FP64_STRICT,
            "double-float": capi.PC_ARNOLDI_DOUBLE_FLOAT}


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Solver:
    """Handle for one discrete optimal-control problem (pc_setup ... pc_destroy)."""

    def __init__(self, dim: int, m1: int, n: int, T: float, gamma: float, eps: float,
                 a_nodes: np.ndarray | None = None, spatial: str = "auto", precision: str = "fp64",
                 max_iter: int = 60, tiles: str | dict | None = "table", space: str = "fd",
                 smoother: str = "red-black", krylov: torch.Tensor | None = None):
        """space: "fd" finite differences (M = I) or "fe" bilinear / trilinear finite
        elements (mass matrix M; constant a, sine-transform solves).
        smoother: Gauss-Seidel ordering of the multigrid pre-smoother, "red-black"
        (parallel) or "lexicographic" (the natural order: the paper's Table 7 counts).
        tiles: "table" applies the stored autotune table's entry for this shape
        (if any), "auto" runs the autotuner now, a dict sets the shapes, None keeps
        the built-in defaults.
        krylov: a CUDA uint8 tensor (view) holding the Krylov storage instead of the
        handle's own (pc_setup_shared; at least krylov_bytes(...) bytes, 256-byte
        aligned).  Handles whose storage overlaps must not solve at the same time; a
        Batch orders them."""
        for name, val, table in (("spatial", spatial, _SPATIAL), ("precision", precision, _PREC),
                                 ("space", space, _SPACE), ("smoother", smoother, _SMOOTHER)):
            if val not in table:
                raise ValueError(f"{name} must be one of {sorted(table)}, got {val!r}")
        if not (tiles in ("table", "auto", None) or isinstance(tiles, dict)):
            raise ValueError("tiles must be 'table', 'auto', a dict or None")
        self.lib = capi.load()
        if not torch.cuda.is_available():
            raise RuntimeError("pcopt needs a CUDA device")
        self.dim, self.m1, self.n = dim, m1, n
        self.T, self.gamma, self.eps = T, gamma, eps
        self.max_iter = max_iter
        prm = capi.pc_params(dim, m1, n, T, gamma, eps, _SPATIAL[spatial], _PREC[precision], max_iter,
                             _SPACE[space], _SMOOTHER[smoother])
        a_ptr = None
        if a_nodes is not None:
            self._a = np.ascontiguousarray(a_nodes, dtype=np.float64)
            if self._a.size != (m1 + 2) ** dim:
                raise ValueError("a_nodes must have (m1+2)^dim entries")
            a_ptr = self._a.ctypes.data_as(ctypes.c_void_p)
        h = ctypes.c_void_p()
        if krylov is None:
            capi.check(self.lib.pc_setup(ctypes.byref(prm), a_ptr, _stream(), ctypes.byref(h)))
        else:
            if not (krylov.is_cuda and krylov.dtype == torch.uint8 and krylov.dim() == 1 and krylov.is_contiguous()):
                raise ValueError("krylov must be a contiguous 1-D uint8 CUDA tensor")
            self._krylov = krylov  # the handle borrows it
            capi.check(self.lib.pc_setup_shared(ctypes.byref(prm), a_ptr, ctypes.c_void_p(krylov.data_ptr()),
                                                krylov.numel(), _stream(), ctypes.byref(h)))
        self.h = h
        self.ms = m1 ** dim
        self.vec_len = 2 * n * self.ms
        self.tau = T / (n + 1)
        resolved = ctypes.c_int(0)
        capi.check(self.lib.pc_precision_of(self.h, ctypes.byref(resolved)))
        self.precision = _PREC_NAME[resolved.value]  # "auto" resolved by eps (pc_precision)
        self.spatial = spatial
        self.space = space
        if tiles == "table":
            entry = tuning.lookup(dim, m1, n, self.precision, spatial) if space == "fd" else None
            if entry:
                self.set_tiles(**entry)
        elif tiles == "auto":
            self.autotune()
        elif isinstance(tiles, dict):
            self.set_tiles(**tiles)
        elif tiles is not None:
            raise ValueError("tiles must be 'table', 'auto', a dict or None")

    # ---------------------------------------------------------------- lifetime
    def close(self):
        if getattr(self, "h", None):
            self.lib.pc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_coefficient(self, a_nodes: np.ndarray | None):
        """Replace a(x) (host array of (m1+2)^dim nodal values) without reallocating."""
        ptr = None
        if a_nodes is not None:
            self._a = np.ascontiguousarray(a_nodes, dtype=np.float64)
            if self._a.size != (self.m1 + 2) ** self.dim:
                raise ValueError("a_nodes must have (m1+2)^dim entries")
            ptr = self._a.ctypes.data_as(ctypes.c_void_p)
        capi.check(self.lib.pc_set_coefficient(self.h, ptr, _stream()))

    def set_log_coefficient(self, log_a: torch.Tensor):
        """a = exp(log_a) at the interior nodes, on the device (pc_set_log_coefficient);
        log_a: float64 CUDA tensor of m1^dim values.  The boundary keeps its values."""
        if log_a.numel() != self.ms:
            raise ValueError(f"log_a must hold {self.ms} values")
        capi.check(self.lib.pc_set_log_coefficient(self.h, _ptr(log_a), _stream()))

    def set_arnoldi(self, mode: str):
        """Arnoldi precision of later solves: "auto" (FP64 handles FP64, mixed handles
        a double-float basis), "fp64", "fp64-strict" (FP64 products everywhere) or
        "double-float" (pc_set_arnoldi)."""
        if mode not in _ARNOLDI:
            raise ValueError(f"mode must be one of {sorted(_ARNOLDI)}, got {mode!r}")
        capi.check(self.lib.pc_set_arnoldi(self.h, _ARNOLDI[mode]))
        self.arnoldi = mode

    def set_preconditioner(self, kind: str):
        """"eps-circulant" (P_eps, the default) or "ideal" (P of Eq. matrix_P by block
        substitution in time: the paper's comparison preconditioner)."""
        if kind not in _PRECOND:
            raise ValueError(f"kind must be one of {sorted(_PRECOND)}, got {kind!r}")
        capi.check(self.lib.pc_set_preconditioner(self.h, _PRECOND[kind]))
        self.precond_kind = kind

    # ---------------------------------------------------------------- helpers
    def empty_vector(self):
        return torch.empty((2, self.n) + (self.m1,) * self.dim, dtype=torch.float64, device="cuda")

    def _vec(self, t):
        if t.numel() != self.vec_len:
            raise ValueError(f"expected {self.vec_len} entries, got {t.numel()}")
        return t

    # ---------------------------------------------------------------- operators
    def matvec(self, x, out=None, transpose=False):
        self._vec(x)
        y = torch.empty_like(x) if out is None else out
        fn = self.lib.pc_matvec_transpose if transpose else self.lib.pc_matvec
        capi.check(fn(self.h, _ptr(x), _ptr(y), _stream()))
        return y

    def matvec_f32(self, x32, out=None):
        """y = A x for an FP32 tensor x (double-float arithmetic, FP64 result)."""
        if not x32.is_cuda or x32.dtype != torch.float32 or not x32.is_contiguous():
            raise ValueError("expected a contiguous float32 CUDA tensor")
        y = torch.empty(x32.shape, dtype=torch.float64, device="cuda") if out is None else out
        capi.check(self.lib.pc_matvec_f32(self.h, ctypes.c_void_p(x32.data_ptr()), _ptr(y), _stream()))
        return y

    def apply_precond(self, v, out=None):
        self._vec(v)
        w = torch.empty_like(v) if out is None else out
        capi.check(self.lib.pc_apply_precond(self.h, _ptr(v), _ptr(w), _stream()))
        return w

    def build_rhs(self, f, g, y0=None, out=None):
        b = self.empty_vector() if out is None else out
        capi.check(self.lib.pc_build_rhs(self.h, _ptr(f), _ptr(g), _ptr(y0), _ptr(b), _stream()))
        return b

    def solve(self, b, x0=None, rtol=1e-8, maxit=None, mode="right", raise_on_nonconv=True, out=None):
        """GMRES on A x = b; returns (x, iterations, relative residual).  out: a device
        vector to solve into (zeroed first unless x0 is given; no allocation then)."""
        self._vec(b)
        if out is not None:
            self._vec(out)
            x = out
            if x0 is None:
                x.zero_()
            elif x0.data_ptr() != x.data_ptr():
                x.copy_(x0)
        else:
            x = torch.zeros_like(b) if x0 is None else x0.clone()
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = self.lib.pc_gmres_solve(self.h, _ptr(b), _ptr(x), rtol, maxit or self.max_iter, _MODE[mode],
                                     ctypes.byref(it), ctypes.byref(rr), _stream())
        if st != capi.PC_ERR_NOT_CONVERGED or raise_on_nonconv:
            capi.check(st)
        return x, it.value, rr.value

    def solve_graph(self, b, x=None, rtol=1e-8, maxit=None, raise_on_nonconv=True):
        """The same FGMRES solve (zero initial guess) as one CUDA-graph launch with
        device-side convergence control; returns (x, iterations, relative residual)."""
        self._vec(b)
        x = torch.empty_like(b) if x is None else x
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = self.lib.pc_gmres_solve_graph(self.h, _ptr(b), _ptr(x), rtol, maxit or self.max_iter,
                                           ctypes.byref(it), ctypes.byref(rr), _stream())
        if st != capi.PC_ERR_NOT_CONVERGED or raise_on_nonconv:
            capi.check(st)
        return x, it.value, rr.value

    def residual_history(self, cap: int | None = None) -> list:
        """Relative residual estimates of the last solve on this handle: entry 0 the
        initial one, entry i the GMRES estimate after iteration i (non-increasing)."""
        cap = (self.max_iter + 1) if cap is None else cap
        out = (ctypes.c_double * max(cap, 1))()
        cnt = ctypes.c_int(0)
        capi.check(self.lib.pc_residual_history(self.h, out, cap, ctypes.byref(cnt), _stream()))
        return [out[i] for i in range(cnt.value)]

    def solve_host(self, b_host, x_host=None, rtol=1e-8, maxit=None, mode="right", raise_on_nonconv=True):
        """Solve from a HOST right-hand side: copy b to the device, run GMRES,
        copy x back into ``x_host`` (pinned CPU tensors give asynchronous copies).
        Returns (x_host, iterations, relative residual)."""
        if b_host.is_cuda or b_host.dtype != torch.float64:
            raise ValueError("b_host must be a float64 CPU tensor")
        b = torch.empty(b_host.shape, dtype=torch.float64, device="cuda")
        b.copy_(b_host, non_blocking=True)
        x, it, rr = self.solve(b, rtol=rtol, maxit=maxit, mode=mode, raise_on_nonconv=raise_on_nonconv)
        if x_host is None:
            x_host = torch.empty(b_host.shape, dtype=torch.float64, pin_memory=True)
        x_host.copy_(x, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return x_host, it, rr

    def adjoint_solve(self, c, lam0=None, rtol=1e-8, maxit=None, mode="right"):
        """GMRES on A^T lam = c; returns (lam, iterations, relative residual)."""
        self._vec(c)
        lam = torch.zeros_like(c) if lam0 is None else lam0.clone()
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        capi.check(self.lib.pc_adjoint_solve(self.h, _ptr(c), _ptr(lam), rtol, maxit or self.max_iter,
                                             _MODE[mode], ctypes.byref(it), ctypes.byref(rr), _stream()))
        return lam, it.value, rr.value

    def grad_log_a(self, x, lam, out=None):
        g = torch.empty((self.m1,) * self.dim, dtype=torch.float64, device="cuda") if out is None else out
        capi.check(self.lib.pc_grad_log_a(self.h, _ptr(x), _ptr(lam), _ptr(g), _stream()))
        return g

    def grad_g(self, lam, out=None):
        """tau * lam1: the gradient with respect to the target g (pc_grad_g)."""
        self._vec(lam)
        gg = torch.empty((self.n,) + (self.m1,) * self.dim, dtype=torch.float64, device="cuda") if out is None else out
        if gg.numel() != self.n * self.ms:
            raise ValueError("out must hold n * m1^dim values")
        capi.check(self.lib.pc_grad_g(self.h, _ptr(lam), _ptr(gg), _stream()))
        return gg

    def objective(self, x, g, out=None):
        """J_h(x; g) as a 0-d device tensor (pc_objective)."""
        self._vec(x)
        if g.numel() != self.n * self.ms:
            raise ValueError("g must hold n * m1^dim values")
        J = torch.empty((), dtype=torch.float64, device="cuda") if out is None else out
        capi.check(self.lib.pc_objective(self.h, _ptr(x), _ptr(g), _ptr(J), _stream()))
        return J

    def objective_grad(self, x, g, gJ=None, gx=None, gg=None):
        """(dJ/dx, explicit dJ/dg) times the device scalar gJ (pc_objective_grad)."""
        self._vec(x)
        if g.numel() != self.n * self.ms:
            raise ValueError("g must hold n * m1^dim values")
        gx = torch.empty_like(x) if gx is None else gx
        gg = torch.empty_like(g) if gg is None else gg
        capi.check(self.lib.pc_objective_grad(self.h, _ptr(x), _ptr(g), _ptr(gJ), _ptr(gx), _ptr(gg), _stream()))
        return gx, gg

    def end_point_solves(self, x, f_T=None, g_0=None, y0=None, p_N=None, rtol=1e-12, maxit=500):
        """y^(N) and p^(0) of the time discretisation from a solution x (pc_end_point_solves)."""
        self._vec(x)
        for v in (f_T, g_0, y0, p_N):
            if v is not None and v.numel() != self.ms:
                raise ValueError("f_T, g_0, y0 and p_N hold m1^dim values")
        yN = torch.empty((self.m1,) * self.dim, dtype=torch.float64, device="cuda")
        p0 = torch.empty_like(yN)
        it = ctypes.c_int(0)
        capi.check(self.lib.pc_end_point_solves(self.h, _ptr(x), _ptr(f_T), _ptr(g_0), _ptr(y0), _ptr(p_N),
                                                _ptr(yN), _ptr(p0), rtol, maxit, ctypes.byref(it), _stream()))
        return yN, p0, it.value

    # ---------------------------------------------------------------- tile shapes
    def get_tiles(self) -> dict:
        t = capi.pc_tiles()
        capi.check(self.lib.pc_get_tiles(self.h, ctypes.byref(t)))
        return {f: getattr(t, f) for f, _ in capi.pc_tiles._fields_}

    def set_tiles(self, **shape):
        cur = self.get_tiles()
        unknown = set(shape) - set(cur)
        if unknown:
            raise ValueError(f"unknown tile fields {sorted(unknown)}")
        cur.update(shape)
        t = capi.pc_tiles(**cur)
        capi.check(self.lib.pc_set_tiles(self.h, ctypes.byref(t)))

    def autotune(self, reps: int = 3) -> dict:
        """Time candidate tile shapes on this handle and keep the fastest (pc_autotune)."""
        t = capi.pc_tiles()
        capi.check(self.lib.pc_autotune(self.h, reps, ctypes.byref(t), _stream()))
        return {f: getattr(t, f) for f, _ in capi.pc_tiles._fields_}

    # ---------------------------------------------------------------- instrumentation
    def profile(self, on=True, classes=None):
        """Time kernels with CUDA events (pc_profile); classes: names of the kernel classes
        to time (pc_profile_classes), None for all."""
        capi.check(self.lib.pc_profile_classes(self.h, ",".join(classes).encode() if classes else None))
        capi.check(self.lib.pc_profile(self.h, 1 if on else 0))

    def stats(self):
        arr = (capi.pc_kernel_stat * 64)()
        cnt = ctypes.c_int(0)
        capi.check(self.lib.pc_stats(self.h, arr, 64, ctypes.byref(cnt)))
        out = {}
        for i in range(cnt.value):
            s = arr[i]
            out[s.name.decode()] = {"launches": s.launches, "ms": s.total_ms, "bytes": s.bytes, "flops": s.flops}
        return out

    def stats_reset(self):
        capi.check(self.lib.pc_stats_reset(self.h))

    def launch_count(self):
        return int(self.lib.pc_launch_count(self.h))


def krylov_bytes(dim: int, m1: int, n: int, eps: float, precision: str = "fp64", max_iter: int = 60) -> int:
    """Bytes of the Krylov storage of a handle with these parameters (pc_krylov_bytes)."""
    if precision not in _PREC:
        raise ValueError(f"precision must be one of {sorted(_PREC)}, got {precision!r}")
    lib = capi.load()
    prm = capi.pc_params(dim, m1, n, 1.0, 1.0, eps, capi.PC_SPATIAL_AUTO, _PREC[precision], max_iter,
                         capi.PC_SPACE_FD, capi.PC_SMOOTHER_RED_BLACK)
    out = ctypes.c_size_t(0)
    capi.check(lib.pc_krylov_bytes(ctypes.byref(prm), ctypes.byref(out)))
    return int(out.value)


def pack_krylov(sizes, pool_bytes: int, align: int = 256):
    """Offsets of Krylov storages of the given sizes in one pool: in order, side by
    side until the pool is full, then again from the start (the next memory wave).
    Storages of one wave never overlap; a storage of a later wave overlaps those of
    earlier waves that share its bytes, and a Batch runs it after them."""
    offsets, cur = [], 0
    for b in sizes:
        need = (int(b) + align - 1) // align * align
        if need > pool_bytes:
            raise ValueError(f"a Krylov storage of {b} bytes does not fit a pool of {pool_bytes}")
        if cur + need > pool_bytes:
            cur = 0
        offsets.append(cur)
        cur += need
    return offsets


def measure_peaks():
    """Measured FP64 and FP32 FMA rates of the current GPU in TFLOP/s (pc_measure_peaks)."""
    lib = capi.load()
    f64, f32 = ctypes.c_double(0.0), ctypes.c_double(0.0)
    capi.check(lib.pc_measure_peaks(ctypes.byref(f64), ctypes.byref(f32), _stream()))
    return f64.value, f32.value


def solve_host_pipelined(jobs, rtol=1e-8, maxit=None, mode="right", raise_on_nonconv=True):
    """Solve several problems from pinned HOST buffers with the host<->device copies
    overlapped with the solves.

    jobs: sequence of (solver, b_host, x_host), pinned float64 CPU tensors of each
    solver's vector length.  While problem i is solved on the current stream, the
    right-hand side of problem i+1 is copied in and the solution of problem i-1 copied
    out on a second stream (events order each copy after what it depends on).  Every
    byte still crosses between host and device inside the call; returns
    [(iterations, relative residual), ...] once all solutions are in their x_host."""
    jobs = list(jobs)
    for s, bh, xh in jobs:
        if bh.is_cuda or xh.is_cuda or bh.dtype != torch.float64 or xh.dtype != torch.float64:
            raise ValueError("b_host and x_host must be float64 CPU tensors")
        if bh.numel() != s.vec_len or xh.numel() != s.vec_len:
            raise ValueError("host buffers must hold the solver's vector length")
    cur = torch.cuda.current_stream()
    cp = torch.cuda.Stream()
    # device buffers live on the solvers and are reused by later calls: allocating
    # inside the loop could make the caching allocator wait for the copy stream
    dev_b, dev_x, seen = [], [], set()
    for s, bh, _ in jobs:
        bufs = getattr(s, "_pipe_bufs", None)
        if id(s) in seen:  # a solver listed twice needs a second pair for this call
            bufs = None
        elif bufs is None or bufs[0].shape != bh.shape:
            bufs = None
        if bufs is None:
            bufs = (torch.empty(bh.shape, dtype=torch.float64, device="cuda"),
                    torch.empty(bh.shape, dtype=torch.float64, device="cuda"))
            if id(s) not in seen:
                s._pipe_bufs = bufs
        seen.add(id(s))
        dev_b.append(bufs[0])
        dev_x.append(bufs[1])
    cp.wait_stream(cur)  # the buffers are free before the copy stream writes them

    def copy_in(i):
        with torch.cuda.stream(cp):
            dev_b[i].copy_(jobs[i][1], non_blocking=True)
            return cp.record_event()

    out = []
    ev_in = copy_in(0) if jobs else None
    for i, (s, _, xh) in enumerate(jobs):
        ev_next = copy_in(i + 1) if i + 1 < len(jobs) else None
        cur.wait_event(ev_in)
        x, it, rr = s.solve(dev_b[i], rtol=rtol, maxit=maxit, mode=mode, raise_on_nonconv=raise_on_nonconv,
                            out=dev_x[i])
        ev_done = cur.record_event()
        with torch.cuda.stream(cp):
            cp.wait_event(ev_done)
            xh.copy_(x, non_blocking=True)
        out.append((it, rr))
        ev_in = ev_next
    cp.synchronize()
    return out


class Batch:
    """Independent problems solved by one graph launch (pc_batch_*).  ``solvers``
    are distinct Solver objects; ``bs`` their right-hand sides; ``xs`` receive the
    solutions (allocated if None).  Keep the solvers and tensors alive while the
    batch exists."""

    def __init__(self, solvers, bs, xs=None, rtol=1e-8, maxit=None):
        self.lib = capi.load()
        self.solvers = list(solvers)
        self.bs = list(bs)
        self.xs = [torch.empty_like(b) for b in self.bs] if xs is None else list(xs)
        n = len(self.solvers)
        hs = (ctypes.c_void_p * n)(*[s.h for s in self.solvers])
        bp = (ctypes.c_void_p * n)(*[_ptr(b) for b in self.bs])
        xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in self.xs])
        maxit = maxit or min(s.max_iter for s in self.solvers)
        bt = ctypes.c_void_p()
        capi.check(self.lib.pc_batch_create(hs, n, bp, xp, rtol, maxit, ctypes.byref(bt)))
        self.bt = bt

    def solve(self, raise_on_nonconv=True):
        n = len(self.solvers)
        it = (ctypes.c_int * n)()
        rr = (ctypes.c_double * n)()
        st = self.lib.pc_batch_solve(self.bt, it, rr, _stream())
        if st != capi.PC_ERR_NOT_CONVERGED or raise_on_nonconv:
            capi.check(st)
        return list(it), list(rr)

    def close(self):
        if getattr(self, "bt", None):
            self.lib.pc_batch_destroy(self.bt)
            self.bt = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
