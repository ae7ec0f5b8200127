"""The checked build (libpcopt_debug.so, -DPCOPT_DEBUG) on the GPU: the operators and
solves of the odd and tiny shapes and of the double-float Krylov path run with every
index check passing (pc_debug_status code 0) and give the release build's results."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu

_WORKER = r"""
import ctypes, sys
sys.path.insert(0, {root!r})
import numpy as np, torch
import synthetic as S
from paper_2410_22686_gb300 import Solver, capi
lib = capi.load()
assert lib._name.endswith("libpcopt_debug.so"), lib._name
code = ctypes.c_int(-1)
assert lib.pc_debug_status(1, ctypes.byref(code)) == capi.PC_OK
out = []
for d, m1, n, prec, sp in [(2, 1, 1, "fp64", "mg"), (2, 3, 2, "fp32", "mg"), (2, 7, 5, "fp32", "mg"),
                           (3, 7, 4, "fp32", "mg"), (2, 31, 32, "fp32", "mg"), (2, 20, 3, "fp64", "fst"),
                           (2, 63, 64, "bf16s", "mg")]:
    a = None if sp == "fst" else np.exp(0.3 * S.random_vector((m1 + 2,) * d, m1 + n))
    s = Solver(d, m1, n, 1.0, 1e-3, 0.3, a, spatial=sp, precision=prec, max_iter=60)
    v = torch.from_numpy(S.random_vector((2, n) + (m1,) * d, 5)).cuda()
    y = s.matvec(v)
    w = s.apply_precond(v)
    x, it, rr = s.solve(v, rtol=1e-8, raise_on_nonconv=False)
    torch.cuda.synchronize()
    out.append((float(y.norm()), float(w.norm()), it, float(x.norm())))
    s.close()
assert lib.pc_debug_status(0, ctypes.byref(code)) == capi.PC_OK
print("CODE", code.value)
print("OUT", out)
"""


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", _WORKER.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    return r


def test_debug_build_checks_pass_and_match_the_release_build():
    from paper_2410_22686_gb300 import build
    build.build()
    build.build(debug=True)
    r = _run({"PCOPT_LIBRARY": "debug"})
    assert r.returncode == 0, r.stdout + r.stderr
    code = int([ln for ln in r.stdout.splitlines() if ln.startswith("CODE")][0].split()[1])
    assert code == 0, code
    out_dbg = [ln for ln in r.stdout.splitlines() if ln.startswith("OUT")][0]
    # the release build, same worker without the checks (its status call answers UNSUPPORTED)
    worker_rel = _WORKER.replace('assert lib._name.endswith("libpcopt_debug.so"), lib._name', "pass").replace(
        "== capi.PC_OK", "in (capi.PC_OK, capi.PC_ERR_UNSUPPORTED)")
    rr = subprocess.run([sys.executable, "-c", worker_rel.format(root=ROOT)], capture_output=True, text=True,
                        timeout=900, cwd=ROOT, env={k: v for k, v in os.environ.items() if k != "PCOPT_LIBRARY"})
    assert rr.returncode == 0, rr.stdout + rr.stderr
    out_rel = [ln for ln in rr.stdout.splitlines() if ln.startswith("OUT")][0]
    import ast
    for a, b in zip(ast.literal_eval(out_dbg[4:]), ast.literal_eval(out_rel[4:])):
        assert a[2] == b[2], (a, b)  # iteration counts
        for p, q in ((a[0], b[0]), (a[1], b[1]), (a[3], b[3])):
            assert abs(p - q) <= 1e-9 * abs(q), (a, b)
