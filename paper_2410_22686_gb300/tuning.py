"""Stored tile shapes per problem shape, written by the autotuner.

``pc_autotune`` times candidate tile shapes of the tunable kernels on one handle
(fused multigrid down leg: tile width and CTAs per SM; prolongation planes per
CTA; shared-memory or register-marching down leg; streaming or one-CTA-per-tile
time FFTs; matvec time blocks per thread) and keeps the fastest.  This module keeps
the chosen shapes in a JSON table next to the package, keyed by
(dim, m1, n, precision, spatial solver), so that ``Solver(..., tiles="table")`` (the default)
starts with the tuned shapes without re-timing.  Shapes missing from the table
run with the built-in defaults.

Regenerate the table on the target GPU with

    python -m paper_2410_22686_gb300.tuning --write [--reps 5] [--out PATH]

which autotunes every workload shape listed in ``WORKLOADS``.
"""
from __future__ import annotations

import argparse
import json
import os

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiles_gb300.json")
FIELDS = ("mg_cx", "mg_ctas", "mv_tj", "pro_pch", "fft_stream", "mg_march", "mg_seg", "fst_stream")

# (dim, m1, n, precision, spatial solver): the bench and test workloads, each shape once
WORKLOADS = tuple(dict.fromkeys(
    [(2, 255, 256, p, "mg") for p in ("mixed", "bf16s", "fp64")]
    + [(2, 255, 128, "mixed", "mg")]  # the small case the kernel profiles are captured on
    + [(3, 63, 128, p, "mg") for p in ("mixed", "bf16s", "fp64")]
    + [(2, 127, 128, p, "mg") for p in ("fp64", "mixed")]
    + [(2, 31, 32, "fp64", "fst")]
    + [(2, 255, 256, p, "fst") for p in ("mixed", "fp64")]
    + [(2, m, n, "mixed", "mg") for m in (31, 63, 127, 255) for n in (16, 64, 256, 512)]
))

_cache: dict | None = None


_PREC_ALIAS = {"fp32": "mixed"}


def key(dim: int, m1: int, n: int, precision: str, spatial: str = "mg") -> str:
    k = f"{dim}d_m{m1}_n{n}_{_PREC_ALIAS.get(precision, precision)}"
    return k + "_fst" if spatial == "fst" else k


def load(path: str = TABLE) -> dict:
    """The table as {key: {field: value}} (empty when there is no file)."""
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        data = json.load(fh)
    return data.get("entries", {})


def lookup(dim: int, m1: int, n: int, precision: str, spatial: str | None = None) -> dict | None:
    """Tile shapes stored for this problem shape, or None."""
    global _cache
    if _cache is None:
        _cache = load()
    e = _cache.get(key(dim, m1, n, precision, spatial or "mg"))
    if not e:
        return None
    return {f: int(e[f]) for f in FIELDS if f in e}


def _tune_one(dim, m1, n, precision, spatial, reps):
    import numpy as np
    import torch

    from .solver import Solver

    tau = 1.0 / (n + 1)
    M = m1 + 2
    x = np.linspace(0.0, 1.0, M)
    if dim == 2:
        X1, X2 = np.meshgrid(x, x, indexing="xy")
        a = 1.0 + 0.5 * np.sin(2 * np.pi * X1) * np.cos(2 * np.pi * X2)
    else:
        X1, X2, X3 = np.meshgrid(x, x, x, indexing="ij")
        a = np.exp(0.25 * np.sin(2 * np.pi * X1) * np.cos(2 * np.pi * X2) * np.sin(np.pi * X3))
    s = Solver(dim, m1, n, 1.0, 1e-4, float(np.sqrt(tau)), a_nodes=None if spatial == "fst" else a,
               spatial=spatial, precision=precision, max_iter=2, tiles=None)
    try:
        t = s.autotune(reps)
        torch.cuda.synchronize()
        return t
    finally:
        s.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--write", action="store_true", help="autotune every workload shape and write the table")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--missing", action="store_true",
                    help="with --write: tune only the shapes the table lacks and keep the rest")
    args = ap.parse_args(argv)
    if not args.write:
        print(json.dumps(load(args.out), indent=1, sort_keys=True))
        return 0
    import torch

    entries = load(args.out) if args.missing else {}
    for (dim, m1, n, prec, spatial) in WORKLOADS:
        k = key(dim, m1, n, prec, spatial)
        if k in entries:
            continue
        t = _tune_one(dim, m1, n, prec, spatial, args.reps)
        entries[k] = t
        print(k, t, flush=True)
    doc = {"device": torch.cuda.get_device_name(0), "reps": args.reps,
           "fields": {"mg_cx": "fused 2D down-leg tile (coarse points per axis)",
                      "mg_ctas": "fused down-leg CTAs per SM",
                      "mv_tj": "matvec time blocks per thread",
                      "pro_pch": "prolongation / 3D per-level planes per CTA",
                      "fft_stream": "time FFTs: 0 one CTA per tile, 1 persistent streaming CTAs",
                      "mg_march": "fused down leg: 0 shared-memory tiles, 1 register-marching warps",
                      "mg_seg": "register-marching down leg: coarse rows per warp",
                      "fst_stream": "sine transforms with persistent streaming CTAs: bit 0 axis passes, "
                                    "bit 1 the fused last-axis pass"},
           "entries": entries}
    with open(args.out, "w") as fh:
        json.dump(doc, fh, indent=1, sort_keys=True)
        fh.write("\n")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
