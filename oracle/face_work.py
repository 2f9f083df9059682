"""Algorithmic work of one face, counted by the oracle (TEST AND MEASUREMENT
INFRASTRUCTURE ONLY).

For each benchmark workload this runs the oracle's stages (density, E and B,
limited gradients) on a small sample of the same generator and counts the
operations of its per-face routine with the counting build
(flopcount.cpp).  Two runs at the Riemann tolerances 1e-12 and 2e-6 (the
mixed path's) change only the number of Newton iterations, which separates
the work per face from the work per iteration:

    ops(tol) = faces * base + iterations(tol) * per_iter

Reported per workload (each add, sub, mul, div, sqrt and pow one flop; the
special-function operations a GPU issues for them: one per division and
square root, two per power):

    flop_base, flop_per_iter, mufu_base, mufu_per_iter

    python -m oracle.face_work      # prints the table the benchmark holds
"""
from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# samples of the benchmark's generators (small enough for a few seconds)
SAMPLES = {
    "sod": ("sod", 16, "exact"),
    "sedov": ("sedov", 24, "exact"),
    "lognormal": ("lognormal", 1 << 14, "exact"),
    "wave": ("wave", 16, "hllc"),
}


def _workload(kind, n):
    from paper_2211_12243_gb300 import workloads as W
    if kind == "sod":
        return W.sod(n)
    if kind == "sedov":
        return W.sedov(n)
    if kind == "lognormal":
        return W.lognormal(n, seed=1, grid=16)
    return W.lattice_wave(n)


def _flops(c):
    return c["add"] + c["mul"] + c["div"] + c["sqrt"] + c["pow"]


def _mufu(c):
    return c["div"] + c["sqrt"] + 2 * c["pow"]


def face_op_counts(kind):
    import oracle
    wk, n, riemann = SAMPLES[kind]
    w = _workload(wk, n)
    runs = []
    for tol in (1e-12, 2e-6):
        cfg = oracle.config(gamma=w["gamma"], riemann=riemann, p_tol=tol)
        x, y, z, L = w["x"], w["y"], w["z"], w["L"]
        h, om, _, _ = oracle.density(cfg, x, y, z, L, w["h"])
        prims = oracle.primitives(cfg, w["m"], w["px"], w["py"], w["pz"], w["E"], w["U"], om)
        B6, _, nc = oracle.matrices(cfg, x, y, z, L, h, om)
        grad, alpha, _ = oracle.gradients(cfg, x, y, z, L, h, om, prims, B6, nc)
        pairs = oracle.flux_pairs(x, y, z, L, h)
        runs.append(oracle.count_face_ops(cfg, x, y, z, L, h, om, B6, prims, grad, alpha, 1e-4,
                                          pairs))
    a, b = runs
    faces = a["faces"]
    di = a["newton_iters"] - b["newton_iters"]
    out = {"faces": faces, "iters_per_face": b["newton_iters"] / faces}
    for key, f in (("flop", _flops), ("mufu", _mufu)):
        per_iter = (f(a) - f(b)) / di if di > 0 else 0.0
        out[f"{key}_per_iter"] = per_iter
        out[f"{key}_base"] = (f(b) - b["newton_iters"] * per_iter) / faces
    return out


def table():
    return {kind: face_op_counts(kind) for kind in SAMPLES}


if __name__ == "__main__":
    t = table()
    for kind, v in t.items():
        print(f"{kind:10s} " + "  ".join(f"{k}={v[k]:.3f}" for k in (
            "flop_base", "flop_per_iter", "mufu_base", "mufu_per_iter", "iters_per_face")))
    print(json.dumps({k: {q: round(v[q], 3) for q in ("flop_base", "flop_per_iter", "mufu_base",
                                                        "mufu_per_iter")} for k, v in t.items()}))
