#!/usr/bin/env python
"""Benchmark of the MFV/MFM hydro step on GB300.

Metric: hydro pair-interactions per second -- directed gradient pairs
(j != i, r_ij < h_i) plus unordered flux pairs (r_ij < max(h_i, h_j)) --
divided by the device time of the gradient and flux stages (CUDA events
recorded by the library around each stage, summed over the timed steps).
The throughput over the whole step (neighbour search, density, gradients,
fluxes, update) is reported beside it as `step_rate`.

Default workload: one clustered log-normal box of 2^27 particles (density
contrast 1e4 on a 256^3 Gaussian field, P ~ rho^gamma, Gaussian velocities
of 0.1 c_s, gamma = 5/3, Wendland C2, N_NGB = 32, exact Riemann solver,
MFV), mixed precision with the adaptive learned starting pressure.  Every
step starts from the initial state with its converged smoothing lengths.
Before the timed region (untimed) the network is trained on the GPU by the
library's kernels on hard faces recorded from steps of the workload itself,
a small log-normal field and a Sedov blast.  After it, on the same initial
state: the mixed step with the plain guess, and the plain FP64 step, which
also gives the mixed step's error at full size; the oracle times a sample of
the same generator on the host cores and checks the GPU on that sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload lognormal|sod|sedov|batch|wave] [--n N]

One JSON line on stdout (rank 0).  Under torchrun each rank steps its own
independent box (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "hydro pair-interactions/s (grad+flux), mixed+learned vs plain FP64, 1 GB300"
UNIT = "pair-interactions/s"
# default sizes: Sod resolution n (78: 1,067,742 particles), Sedov lattice
# side, log-normal particles, number of boxes, wave lattice side
DEFAULT_N = {"sod": 78, "sedov": 128, "lognormal": 1 << 27, "batch": 512, "wave": 32}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lognormal",
                    choices=["sod", "sedov", "lognormal", "batch", "wave"],
                    help="lognormal: clustered log-normal box of n particles (default); sod: 3D "
                         "Sod tube; sedov: Sedov-Taylor blast on an n^3 lattice; batch: n "
                         "independent periodic boxes of 4k-64k particles in one launch; wave: "
                         "n^3 jittered lattice with a density wave (HLLC)")
    ap.add_argument("--n", type=int, default=None,
                    help="size: log-normal particle count (2^27), Sod resolution (78: "
                         "1,067,742), Sedov lattice side (128), number of boxes (512), wave "
                         "lattice side (32)")
    ap.add_argument("--riemann", default=None, choices=["exact", "hllc"],
                    help="Riemann solver (default: exact; hllc for the wave)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch parameters (no hydro_autotune)")
    ap.add_argument("--no-graph", action="store_true", help="host-driven steps (no CUDA graph)")
    ap.add_argument("--scheme", default="mfv")
    ap.add_argument("--precision", default="mixed")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-learned", action="store_true", help="headline without the learned guess")
    ap.add_argument("--train-steps", type=int, default=20000)
    ap.add_argument("--riemann-polish", action="store_true",
                    help="mixed path: one FP64 Newton step after the float iteration "
                         "(hydro_config.riemann_polish)")
    ap.add_argument("--restart", action="store_true",
                    help="start every step (warm-up and timed) from the initial state "
                         "(default for the log-normal box, whose state develops negative "
                         "internal energies after a few steps)")
    ap.add_argument("--cpu-n", type=int, default=None,
                    help="size of the CPU sample (Sod 40, Sedov 32, log-normal 2^15)")
    ap.add_argument("--cpu-reps", type=int, default=6)
    ap.add_argument("--gravity", action="store_true",
                    help="step with a seeded external acceleration field (hydro_set_gravity)")
    ap.add_argument("--entropy", action="store_true",
                    help="step with the entropy switch on (hydro_set_entropy)")
    ap.add_argument("--rungs", type=float, default=None, metavar="K",
                    help="time base steps of individual timesteps (hydro_step_rungs) with "
                         "dt0 = K times the CFL dt of the initial state; value = pairs over "
                         "the whole base step")
    ap.add_argument("--caller-order", action="store_true",
                    help="keep the particles in the generator's order (sorted_output = 0): every "
                         "step gathers them from and scatters them back to that order")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the short runs of the Sod tube, the Sedov blast and the batch of "
                         "boxes that the default workload's line carries under other_workloads")
    return ap.parse_args()


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# --------------------------------------------------------------------------
# CPU oracle baseline (test infrastructure, timed as it stands)
# --------------------------------------------------------------------------
def workload_name(kind, n):
    n = n or DEFAULT_N[kind]
    if kind == "sedov":
        return f"sedov3d_{n}cubed_mfv_exact"
    if kind == "lognormal":
        return f"lognormal3d_{n}_mfv_exact"
    if kind == "batch":
        return f"batch_{n}_boxes_4k_64k_mfv_exact"
    if kind == "wave":
        return f"wave3d_{n}cubed_mfv_hllc"
    return "sod3d_1067742_mfv_exact" if n == 78 else f"sod3d_n{n}"


def make_workload(kind, n, seed=0):
    """The workload of one rank: the seeded generators (log-normal, batch)
    draw a different realisation per seed, the lattice problems are the same
    on every rank."""
    from paper_2211_12243_gb300 import workloads as W
    name = workload_name(kind, n)
    n = n or DEFAULT_N[kind]
    if kind == "sedov":
        return W.sedov(n), name
    if kind == "lognormal":
        return W.lognormal(n, seed=seed), name
    if kind == "batch":
        return W.batch(n, seed=seed), name
    if kind == "wave":
        return W.lattice_wave(n), name
    return W.sod(n), name


def oracle_sample_rate(kind, n, reps, threads=None):
    """The oracle's gradient + flux stages on a small case of the same
    generator (density solved first, untimed); pairs counted like the GPU
    metric.  threads: OpenMP threads of the timed passes (default: all)."""
    import oracle
    if n is None:
        n = {"sod": 40, "sedov": 32, "lognormal": 1 << 15, "batch": 6, "wave": 32}[kind]
    w, _ = make_workload(kind, n)
    if kind == "batch":   # the oracle takes one periodic box at a time
        off, bl = w["box_off"], w["box_len"].reshape(-1, 3)
        boxes = [({k: w[k][off[b]:off[b + 1]] for k in ("x", "y", "z", "m", "px", "py", "pz",
                                                          "E", "U", "h")}, bl[b])
                 for b in range(len(off) - 1)]
    else:
        boxes = [(w, w["L"])]
    cfg = oracle.config(gamma=w["gamma"])
    prep = []
    gpairs = 0
    for wb, L in boxes:
        x, y, z = wb["x"], wb["y"], wb["z"]
        h, om, _, _ = oracle.density(cfg, x, y, z, L, wb["h"])
        prims = oracle.primitives(cfg, wb["m"], wb["px"], wb["py"], wb["pz"], wb["E"], wb["U"], om)
        off_l, idx = oracle.neighbours(x, y, z, L, h)
        gpairs += int(idx.size - x.size)
        prep.append((x, y, z, L, h, om, prims))
    t = 0.0
    fpairs = 0
    all_threads = oracle.num_threads()
    if threads:
        oracle.set_num_threads(threads)
    for _ in range(reps):
        fpairs = 0
        for x, y, z, L, h, om, prims in prep:
            t0 = time.perf_counter()
            B6, _, nc = oracle.matrices(cfg, x, y, z, L, h, om)
            grad, alpha, _ = oracle.gradients(cfg, x, y, z, L, h, om, prims, B6, nc)
            pairs = oracle.flux_pairs(x, y, z, L, h)
            oracle.fluxes(cfg, x, y, z, L, h, om, B6, prims, grad, alpha, 1e-4, pairs=pairs)
            t += time.perf_counter() - t0
            fpairs += len(pairs)
    total = reps * (gpairs + fpairs)
    npart = sum(len(p[0]) for p in prep)
    cores = oracle.num_threads()
    oracle.set_num_threads(all_threads)
    return dict(value=total / t, unit=UNIT, cores=cores, kind="oracle",
                sample=f"{kind} generator at n={n} ({npart} particles), oracle gradient+flux stages "
                       f"(E/B/N_cond, gradients+limiter, pair enumeration, fluxes), {reps} passes, "
                       f"{total} pair-interactions in {t:.2f} s"), t


def aggregate(world, pairs, ms, gf_ms, device):
    """Whole-job figures of a multi-rank run (one process per GPU, each on
    its own boxes, no data-path collective): pair-interactions summed over
    the ranks, step and stage times the maximum over the ranks."""
    if world <= 1:
        return float(pairs), float(ms), float(gf_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms, gf_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(p[0].item()), float(t[0].item()), float(t[1].item())


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    rate = None
    times = []
    for k in range(args.warmup + args.steps):
        r, t = oracle_sample_rate(args.workload, args.cpu_n, 1)
        if k >= args.warmup:
            times.append(t)
            rate = r
    import oracle
    ms = 1000.0 * sum(times) / len(times)
    pairs_per_step = rate["value"] * (sum(times) / len(times))
    value = pairs_per_step / (sum(times) / len(times))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.workload, args.n), "sample": rate["sample"],
                   "l2": "CPU run (no device caches)"},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": rate["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def boxes_of(hydro, w):
    """(box_off, box_len) of a workload: its own for a batch, else one box."""
    if w.get("box_off") is not None:
        return w["box_off"], w["box_len"]
    return hydro.single_box(w)


def train_network(hydro, workloads, w, kind, steps):
    """Record the hard faces of a few mixed steps of the workload itself (a
    2^21-particle sample of its generator when it is larger than 2^22), a
    log-normal field, a Sod tube and a Sedov blast, and train the
    starting-pressure network on them with the library's kernels
    (untimed)."""
    import numpy as np
    import torch
    t0 = time.time()
    big = kind == "lognormal" and w["x"].size > (1 << 22)
    own = make_workload(kind, 1 << 21, seed=9)[0] if big else w
    sets = [(own, 2, 1.0), (workloads.lognormal(1 << 16, seed=5, grid=32), 2, 0.5),
            (workloads.sod(24), 4, 1.0), (workloads.sedov(48), 8, 1.0)]
    bufs = []
    for wk, nstep, keep in sets:
        Hr = hydro.Hydro(hydro.default_config(gamma=wk["gamma"], precision="mixed",
                                              search_margin=2.0))
        Hr.set_boxes(*boxes_of(hydro, wk))
        s = hydro.to_device(wk)
        cap = 1 << 21
        buf = torch.zeros((7, cap), dtype=torch.float32, device="cuda")
        Hr.record_faces(buf, keep=keep, hard_only=True)
        for _ in range(nstep):
            Hr.step(s, check=False)
        bufs.append(buf[:, :min(Hr.recorded_faces(), cap)])
        Hr.close()
    faces = torch.cat(bufs, 1).contiguous()
    Ht = hydro.Hydro(hydro.default_config(gamma=w["gamma"], precision="mixed"))
    loss = Ht.mlp_train(faces, steps=steps, batch=2048, lr=2e-3, seed=11)
    torch.cuda.synchronize()
    theta = Ht.mlp_get()
    l = loss.cpu().numpy()
    Ht.close()
    return {"theta": theta, "faces": int(faces.shape[1]), "steps": steps, "batch": 2048,
            "loss_first": float(np.mean(l[:50])), "loss_last": float(np.mean(l[-200:])),
            "seconds": time.time() - t0}


KEYS = ("x", "y", "z", "m", "px", "py", "pz", "E", "U", "h")


def timed_steps(hydro, Hc, state, k, warm, restart, ok_status, flush, stream, dt=-1.0):
    """k timed steps (CUDA events on the stream, L2 flushed before each)
    after `warm` untimed ones; with restart every step starts from the state
    given.  Returns the summed stage times and counters."""
    import torch
    saved = {kk: v.clone() for kk, v in state.items()} if restart else None
    for _ in range(warm):
        if restart:
            for kk, v in saved.items():
                state[kk].copy_(v)
        s = Hc.step(state, dt, check=False)
        assert s["status"] in ok_status, s
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    acc = dict(pairs=0, flux_ms=0.0, grad_ms=0.0, kern_ms=0.0, hard_ms=0.0, flux_pairs=0,
               iters=0, hard=0, learned=0, fallbacks=0, active=0, graph_steps=0)
    launches0 = hydro.kernel_launches()
    stats = None
    for i in range(k):
        if restart:
            for kk, v in saved.items():
                state[kk].copy_(v)
        flush.zero_()
        ev0[i].record(stream)
        stats = Hc.step(state, dt, check=False)
        ev1[i].record(stream)
        assert stats["status"] in ok_status, stats
        acc["pairs"] += stats["grad_pairs"] + stats["flux_pairs"]
        acc["flux_ms"] += stats["ms_fluxes"]
        acc["grad_ms"] += stats["ms_gradients"]
        acc["kern_ms"] += stats["ms_flux_kernel"]
        acc["hard_ms"] += stats["ms_hard_faces"]
        acc["flux_pairs"] += stats["flux_pairs"]
        acc["iters"] += stats["newton_iters"]
        acc["hard"] += stats["hard_faces"]
        acc["learned"] += stats["learned_faces"]
        acc["fallbacks"] += stats["guess_fallbacks"]
        acc["active"] += stats["learned_active"]
        acc["graph_steps"] += stats["graph"] == 1
    torch.cuda.synchronize()
    acc["launches"] = hydro.kernel_launches() - launches0
    acc["each_ms"] = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    acc["ms"] = sum(acc["each_ms"])
    acc["gf_ms"] = acc["grad_ms"] + acc["flux_ms"]
    acc["last"] = stats
    del saved
    return acc


def one_step_host(Hc, hydro, w, dt):
    """One step of the workload's initial state with a fixed dt; the state
    after it on the host (float64 numpy) and the step's statistics."""
    import torch
    st = hydro.to_device(w)
    stats = Hc.step(st, dt, check=False)
    torch.cuda.synchronize()
    out = {k: st[k].cpu().numpy() for k in KEYS + ("omega",)}
    del st
    return out, stats


def error_vs_fp64(w, mixed, fp64):
    """The mixed step's error at full size against the plain FP64 step from
    the same state with the same dt (the FP64 path itself matches the FP64
    oracle to 1e-12 in the tests): per conserved component, the largest
    difference of the step's change over the largest change; h relative."""
    import numpy as np
    out = {}
    for k in ("m", "px", "py", "pz", "E"):
        d_m = mixed[k] - w[k]
        d_f = fp64[k] - w[k]
        scale = float(np.abs(d_f).max()) + 1e-300
        err = np.abs(d_m - d_f) / scale
        out[k] = {"max": float(err.max()), "p999": float(np.quantile(err, 0.999))}
    dh = np.abs(mixed["h"] - fp64["h"]) / np.abs(fp64["h"])
    out["h_max_rel"] = float(dh.max())
    # particles whose h differs beyond the double-class refinement: N_cond
    # guard decisions (a threshold on a float-accumulated E) that came out
    # the other way, which move h by (1.2)^(1/3) per growth round
    out["h_differs_1e-9"] = int(np.sum(dh > 1e-9))
    errs = np.stack([np.abs((mixed[k] - w[k]) - (fp64[k] - w[k])) /
                     (np.abs(fp64[k] - w[k]).max() + 1e-300) for k in ("m", "px", "py", "pz", "E")], 1)
    out["particles_above_1e-5"] = int(np.sum(errs.max(1) > 1e-5))
    out["note"] = ("|dQ_mixed - dQ_fp64| / max|dQ_fp64| per component over all particles, one "
                   "step from the initial state with the same dt")
    return out


def conservation_of(stats, w):
    """Relative drift of the step's totals (compensated sums before and after
    the update, from hydro_stats): mass and energy over sum |X|, momentum per
    axis over sum m (|v| + c_s)."""
    import numpy as np
    m = w["m"]
    v = np.stack([w["px"], w["py"], w["pz"]], 1) / m[:, None]
    cs = np.sqrt(np.maximum(w["gamma"] * (w["gamma"] - 1) * w["U"] / m, 0))
    ps = math.fsum(m * (np.linalg.norm(v, axis=1) + cs))
    out = {"M": abs(stats["mass"][1] - stats["mass"][0]) / math.fsum(np.abs(m)),
           "E": abs(stats["energy"][1] - stats["energy"][0]) / math.fsum(np.abs(w["E"]))}
    for a, k in enumerate(("px", "py", "pz")):
        out[k] = abs(stats["mom"][1][a] - stats["mom"][0][a]) / ps
    return out


def oracle_sample_parity(kind, hydro, n=None):
    """The GPU's mixed step against the FP64 oracle's step on a sample of the
    same generator: the per-particle flux error of each conserved component,
    normalised by the particle's sum over its faces of |c| (the net can
    cancel; a component that vanishes on every face takes the momentum
    flux's scale through c_s), and the conservation drift of both."""
    import numpy as np
    import oracle
    n = n or {"sod": 16, "sedov": 24, "lognormal": 1 << 14, "batch": 1 << 14, "wave": 16}[kind]
    w, _ = make_workload("lognormal" if kind == "batch" else kind, n)
    riemann = "hllc" if kind == "wave" else "exact"
    cfg = oracle.config(gamma=w["gamma"], riemann=riemann)
    so, out_o, info = oracle.step(cfg, w, -1.0)
    Hs = hydro.Hydro(hydro.default_config(gamma=w["gamma"], precision="mixed", riemann=riemann))
    Hs.set_boxes(*boxes_of(hydro, w))
    sg, stats = one_step_host(Hs, hydro, w, info["dt"])
    Hs.close()
    prims = oracle.primitives(cfg, w["m"], w["px"], w["py"], w["pz"], w["E"], w["U"], so["omega"])
    _, _, _, dQabs = oracle.fluxes(cfg, w["x"], w["y"], w["z"], w["L"], so["h"], so["omega"],
                                   out_o["B6"], prims, out_o["grad"], out_o["alpha"], info["dt"],
                                   want_abs=True)
    rho, _, _, _, p = prims
    cs = np.sqrt(w["gamma"] * p / rho)
    pm = dQabs[:, 1] + dQabs[:, 2] + dQabs[:, 3]
    sc = np.stack([np.maximum(dQabs[:, 0], pm / cs), pm, pm, pm,
                   np.maximum(dQabs[:, 4], pm * cs)], 1) + 1e-300
    keys = ("m", "px", "py", "pz", "E")
    d = np.stack([(sg[k] - w[k]) - (so[k] - w[k]) for k in keys], 1)
    err = np.abs(d) / sc
    return {"particles": int(w["x"].size), "status_gpu": stats["status"],
            "status_oracle": info["status"],
            "flux_err_max": float(err.max()), "flux_err_p999": float(np.quantile(err, 0.999)),
            "above_1e-5": int(np.sum(err.max(1) > 1e-5)),
            "conservation_gpu": conservation_of(stats, w),
            "note": "per-particle |dQ_gpu - dQ_oracle| / sum over faces |c|, one step, same dt"}


def other_workloads(hydro, flush, stream, steps=10, warm=3):
    """Short runs of the other configurations at their full sizes -- the
    1,067,742-particle Sod tube, the 128^3 Sedov blast and the 512 boxes of
    4k-64k particles in one context -- each with its mixed step (plain guess,
    autotuned, graph steps, L2 flushed before every step) against one plain
    FP64 step of the same state: the metric, the whole-step rate and the
    times of both; the state kept in the library's order (sorted_output)."""
    import numpy as np
    import torch
    out = {}
    for kind in ("sod", "sedov", "batch"):
        w, name = make_workload(kind, DEFAULT_N[kind])
        n = w["x"].size
        restart = kind == "batch"
        ok = (0, -5) if kind == "batch" else (0,)
        common = dict(gamma=w["gamma"], riemann="exact", search_margin=1.15, graph=1,
                      sorted_output=1)
        H = hydro.Hydro(hydro.default_config(precision="mixed", **common))
        H.set_boxes(*boxes_of(hydro, w))
        H.reserve(n, 96)
        st = hydro.to_device(w)
        # one step on a copy: the library's order for the state (and, for the
        # restarted batch, the converged h of the initial state)
        tmp = {k: v.clone() for k, v in st.items()}
        s0 = H.step(tmp, -1.0, check=False)
        assert s0["status"] in ok, s0
        perm = H.get_order().cpu().numpy()
        for k in KEYS:
            w[k] = tmp[k].cpu().numpy() if (restart and k == "h") else np.ascontiguousarray(w[k][perm])
        del tmp
        st = hydro.to_device(w)
        tuning = H.autotune(st)
        r = timed_steps(hydro, H, st, steps, warm, restart, ok, flush, stream)
        H.close()
        del st
        torch.cuda.empty_cache()
        H64 = hydro.Hydro(hydro.default_config(precision="fp64", **common))
        H64.set_boxes(*boxes_of(hydro, w))
        H64.set_tuning(dict(tuning, grad_min_ctas=1, flux_min_ctas=4))
        st = hydro.to_device(w)
        r64 = timed_steps(hydro, H64, st, 1, 1, restart, ok, flush, stream)
        H64.close()
        del st
        torch.cuda.empty_cache()
        out[name] = {
            "particles": n, "value": r["pairs"] / (r["gf_ms"] / 1000.0),
            "step_rate": r["pairs"] / (r["ms"] / 1000.0), "ms_per_step": r["ms"] / steps,
            "grad_flux_ms_per_step": r["gf_ms"] / steps, "steps": steps,
            "timed_steps": "each from the initial state" if restart else "consecutive",
            "plain_fp64": {"value": r64["pairs"] / (r64["gf_ms"] / 1000.0),
                           "ms_per_step": r64["ms"], "steps": 1},
            "vs_plain_fp64": (r["pairs"] / r["gf_ms"]) / (r64["pairs"] / r64["gf_ms"]),
            "note": "mixed step with the plain starting guess (no network trained for it)"}
    return out


def measured_peaks():
    """This GPU's arithmetic throughput by the library's probes."""
    from paper_2211_12243_gb300 import hydro
    return {u: hydro.probe_peak(u) for u in ("fp32", "mufu", "fp64")}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.rungs is not None:
        return bench_rungs(args)
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2211_12243_gb300 import build, hydro, workloads
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    t_setup = time.time()
    w, wname = make_workload(args.workload, args.n, seed=rank)
    n = w["x"].size
    big = n > (1 << 25)
    learned = args.precision == "mixed" and not args.no_learned
    riemann = args.riemann or ("hllc" if args.workload == "wave" else "exact")
    learned = learned and riemann == "exact"
    training = train_network(hydro, workloads, w, args.workload, args.train_steps) if learned else None
    margin = 1.15
    graph = 0 if args.no_graph else 1
    common = dict(gamma=w["gamma"], scheme=args.scheme, riemann=riemann, search_margin=margin,
                  graph=graph)
    sorted_out = not args.caller_order
    common["sorted_output"] = int(sorted_out)
    cfg = hydro.default_config(precision=args.precision, learned_guess=int(learned),
                               riemann_polish=int(args.riemann_polish), **common)
    H = hydro.Hydro(cfg)
    if learned:
        H.mlp_load(training["theta"])
    H.set_boxes(*boxes_of(hydro, w))
    H.reserve(n, 96)
    st = hydro.to_device(w)
    if args.gravity:
        # a seeded acceleration field of order the sound speed squared over the box
        g = np.random.default_rng(20221122 + 7).normal(0.0, 0.1, (n, 3))
        acc = torch.as_tensor(g, device="cuda").contiguous()
        H.set_gravity(acc)
    if args.entropy:
        H.set_config(entropy_switch=1)
        st["A"] = torch.zeros(n, dtype=torch.float64, device="cuda")   # unset: set by the first step
        H.set_entropy(st["A"])
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    stream = torch.cuda.current_stream()

    # the log-normal box has isolated particles whose E stays ill-conditioned
    # after the N_NGB growths; the step completes and reports them (ENCOND)
    ok_status = (0, -5) if args.workload in ("lognormal", "batch") else (0,)

    restart = args.restart or args.workload in ("lognormal", "batch")
    # the initial state's CFL dt (and, for restarted workloads, its
    # converged smoothing lengths, which a running simulation carries: the
    # generator's h are rough guesses from a coarse density grid)
    tmp = {kk: v.clone() for kk, v in st.items()}
    s0 = H.step(tmp, -1.0, check=False)
    assert s0["status"] in ok_status, s0
    dt_cmp = s0["dt"]
    if restart:
        w["h"] = tmp["h"].cpu().numpy()
    if sorted_out:
        # the state kept in the library's own (Morton) order, as a simulation
        # that keeps sorted_output on carries it from step to step (tmp, the
        # step's output, is already in that order)
        perm = H.get_order().cpu().numpy()
        for kk in KEYS:
            if not (restart and kk == "h"):
                w[kk] = np.ascontiguousarray(w[kk][perm])
        st = hydro.to_device(w)
        if args.gravity:
            acc = acc[torch.as_tensor(perm, device="cuda").long()].contiguous()
            H.set_gravity(acc)
        if args.entropy:
            st["A"] = torch.zeros(n, dtype=torch.float64, device="cuda")
            H.set_entropy(st["A"])
    elif restart:
        st["h"].copy_(tmp["h"])
    del tmp

    tuning = None if args.no_autotune else H.autotune(st)
    setup_s = time.time() - t_setup

    # ---- timed region: the mixed step
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    r = timed_steps(hydro, H, st, args.steps, args.warmup, restart, ok_status, flush, stream)
    clocks = clk.stop()
    pairs_all, ms_max, gf_max = aggregate(world, r["pairs"], r["ms"], r["gf_ms"], "cuda")
    ms_per_step = ms_max / args.steps
    # the metric: pairs over the gradient + flux stage time; whole-step rate beside it
    value = pairs_all / (gf_max / 1000.0)
    step_rate = pairs_all / (ms_max / 1000.0)
    last = r["last"]
    conservation = conservation_of(last, w) if restart else None

    # ---- end to end through the public API with host buffers: every step
    # copies its inputs in (pinned host -> device), steps, and reads its state
    # back (device -> pinned host), sequentially and then pipelined (below).
    # One sequential step first (untimed) gives the three phases on their
    # own.  Every step, copy and event runs on streams of its own: work on the
    # legacy default stream would wait on the copy streams.
    es = torch.cuda.Stream()
    with torch.cuda.stream(es):
        host = {k: torch.as_tensor(w[k]).pin_memory() for k in KEYS}
        host_out = {k: torch.empty(n, dtype=torch.float64).pin_memory() for k in KEYS + ("omega",)}
        e2e_steps = args.steps
        st2 = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k in KEYS + ("omega",)}
        stage = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k in KEYS + ("omega",)}
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        flush.zero_()
        ev[0].record(es)
        for kk in KEYS:
            st2[kk].copy_(host[kk], non_blocking=True)
        ev[1].record(es)
        s2 = H.step(st2, -1.0, check=False, stream=es)
        assert s2["status"] in ok_status, s2
        ev[2].record(es)
        for kk in KEYS + ("omega",):
            host_out[kk].copy_(st2[kk], non_blocking=True)
        ev[3].record(es)
        torch.cuda.synchronize()
        phases = {"h2d": ev[0].elapsed_time(ev[1]), "step": ev[1].elapsed_time(ev[2]),
                  "d2h": ev[2].elapsed_time(ev[3])}
        # sequential: each step's read-back before the next step's copy-in
        e_seq0 = torch.cuda.Event(enable_timing=True)
        e_seq1 = torch.cuda.Event(enable_timing=True)
        seq_pairs = 0
        e_seq0.record(es)
        for k in range(e2e_steps):
            flush.zero_()
            for kk in KEYS:
                st2[kk].copy_(host[kk], non_blocking=True)
            s2 = H.step(st2, -1.0, check=False, stream=es)
            assert s2["status"] in ok_status, s2
            seq_pairs += s2["grad_pairs"] + s2["flux_pairs"]
            for kk in KEYS + ("omega",):
                host_out[kk].copy_(st2[kk], non_blocking=True)
        e_seq1.record(es)
        torch.cuda.synchronize()
        seq_ms = e_seq0.elapsed_time(e_seq1)
        # overlapped: each step's inputs arrive in a device staging copy on a
        # copy stream while the previous step runs, and its state leaves from a
        # staging copy on another while the next step runs (device-to-device
        # copies into and out of the step's own arrays); the first H2D and the
        # last D2H are inside the timed region
        in_stage = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k in KEYS}
        cs_in = torch.cuda.Stream()
        cs = torch.cuda.Stream()
        e_start = torch.cuda.Event(enable_timing=True)
        e_end = torch.cuda.Event(enable_timing=True)
        d2h_done = None
        e2e_pairs = 0
        e_start.record(es)
        cs_in.wait_stream(es)
        with torch.cuda.stream(cs_in):
            for kk in KEYS:
                in_stage[kk].copy_(host[kk], non_blocking=True)
        in_ready = torch.cuda.Event()
        in_ready.record(cs_in)
        for k in range(e2e_steps):
            flush.zero_()
            es.wait_event(in_ready)
            for kk in KEYS:
                st2[kk].copy_(in_stage[kk], non_blocking=True)
            if k + 1 < e2e_steps:
                # the next step's inputs, once the staging copy is free again
                in_free = torch.cuda.Event()
                in_free.record(es)
                cs_in.wait_event(in_free)
                with torch.cuda.stream(cs_in):
                    for kk in KEYS:
                        in_stage[kk].copy_(host[kk], non_blocking=True)
                in_ready = torch.cuda.Event()
                in_ready.record(cs_in)
            s2 = H.step(st2, -1.0, check=False, stream=es)
            assert s2["status"] in ok_status, s2
            e2e_pairs += s2["grad_pairs"] + s2["flux_pairs"]
            if d2h_done is not None:
                es.wait_event(d2h_done)   # (the staging buffers are free again)
            for kk in KEYS + ("omega",):
                stage[kk].copy_(st2[kk], non_blocking=True)
            staged = torch.cuda.Event()
            staged.record(es)
            cs.wait_event(staged)
            with torch.cuda.stream(cs):
                for kk in KEYS + ("omega",):
                    host_out[kk].copy_(stage[kk], non_blocking=True)
            d2h_done = torch.cuda.Event()
            d2h_done.record(cs)
        es.wait_event(d2h_done)
        e_end.record(es)
        torch.cuda.synchronize()
        e2e_ms = e_start.elapsed_time(e_end)
        e2e = {"value": e2e_pairs / (e2e_ms / 1000.0), "unit": UNIT, "steps": e2e_steps,
               "timed": "per step: H2D copies of the inputs + hydro_step + D2H copies of the state, "
                        "pipelined: the inputs arrive in a device staging copy on a copy es "
                        "during the previous step and the state leaves from one during the next "
                        "(device-to-device copies into and out of the step's arrays); the first "
                        "H2D and the last D2H inside the timed region",
               "h2d_bytes_per_step": 8 * n * len(KEYS), "d2h_bytes_per_step": 8 * n * (len(KEYS) + 1),
               "ms_per_step": e2e_ms / e2e_steps,
               "sequential": {"value": seq_pairs / (seq_ms / 1000.0), "ms_per_step": seq_ms / e2e_steps},
               "one_sequential_step_ms": phases}
    del host, host_out, st2, stage, in_stage

    # ---- the mixed step once more from the initial state, dt fixed (outside
    # the timed region), for the comparison with the FP64 step
    st.clear()
    torch.cuda.empty_cache()
    mixed_cmp, _ = one_step_host(H, hydro, w, dt_cmp)
    H.close()
    torch.cuda.empty_cache()

    # ---- the same mixed step with the plain (Toro) guess, same starting state
    plain_guess = None
    if learned:
        Hp = hydro.Hydro(hydro.default_config(precision=args.precision, **common))
        Hp.set_boxes(*boxes_of(hydro, w))
        stp = hydro.to_device(w)
        if tuning:
            Hp.set_tuning(tuning)
        kp = 2 if big else max(2, min(args.steps, 5))
        rp = timed_steps(hydro, Hp, stp, kp, 1, restart, ok_status, flush, stream)
        plain_guess = {"value": rp["pairs"] / (rp["gf_ms"] / 1000.0),
                       "step_rate": rp["pairs"] / (rp["ms"] / 1000.0), "ms_per_step": rp["ms"] / kp,
                       "flux_stage_ms": rp["flux_ms"] / kp, "flux_kernel_ms": rp["kern_ms"] / kp,
                       "newton_iters_per_face": rp["iters"] / max(rp["flux_pairs"], 1)}
        Hp.close()
        del stp
        torch.cuda.empty_cache()

    # ---- plain FP64 step on the same starting state: its first (untimed)
    # step from the initial state with the comparison dt gives the error of
    # the mixed step at full size
    fp64 = None
    err64 = None
    if not args.no_fp64:
        H64 = hydro.Hydro(hydro.default_config(precision="fp64", **common))
        H64.set_boxes(*boxes_of(hydro, w))
        # the list radius and slots found for the mixed step; default kernels
        tuning64 = None if tuning is None else dict(tuning, grad_min_ctas=1, flux_min_ctas=4)
        if tuning64:
            H64.set_tuning(tuning64)
        fp64_cmp, _ = one_step_host(H64, hydro, w, dt_cmp)
        err64 = error_vs_fp64(w, mixed_cmp, fp64_cmp)
        del fp64_cmp
        st64 = hydro.to_device(w)
        k64 = 1 if big else max(2, min(args.steps, 5))
        r64 = timed_steps(hydro, H64, st64, k64, 0 if big else 1, restart, ok_status, flush,
                          stream)
        fp64 = {"value": r64["pairs"] / (r64["gf_ms"] / 1000.0),
                "step_rate": r64["pairs"] / (r64["ms"] / 1000.0), "ms_per_step": r64["ms"] / k64,
                "flux_kernel_ms": r64["flux_ms"] / k64, "timed_steps": k64,
                "tuning": None if tuning64 is None else {k: tuning64[k] for k in (
                    "search_margin", "nbr_slots", "grad_min_ctas")}}
        H64.close()
        del st64
        torch.cuda.empty_cache()

    # ---- roofline of the dominant kernel (pair fluxes): the oracle-counted
    # work of the faces it solves over its event-timed duration, against this
    # GPU's measured FP32 and special-function throughput
    peaks = measured_peaks()
    faces = r["flux_pairs"] / args.steps
    hard = r["hard"] / args.steps
    iters = r["iters"] / args.steps
    kern_ms = r["kern_ms"] / args.steps
    # hard faces deferred to the hard-face kernel are solved there; the
    # Newton iterations are counted together, so the flux kernel is credited
    # with the share of its own faces
    solved = faces - (hard if r["active"] else 0.0)
    iters_own = iters * solved / max(faces, 1.0)
    ops = FACE_OPS["lognormal" if args.workload == "batch" else args.workload]
    flop = solved * ops["flop_base"] + iters_own * ops["flop_per_iter"]
    mufu = solved * ops["mufu_base"] + iters_own * ops["mufu_per_iter"]
    sec = kern_ms / 1000.0
    comp = {"fp32": {"achieved": flop / sec / 1e12, "peak": peaks["fp32"], "unit": "TFLOP/s"},
            "mufu": {"achieved": mufu / sec / 1e12, "peak": peaks["mufu"], "unit": "Tops/s"}}
    for c in comp.values():
        c["frac"] = c["achieved"] / c["peak"]
    traffic_pf = FLUX_TRAFFIC_BYTES_PER_FACE.get(args.workload)
    # (measured for the register bound of 4 CTAs per SM with the bucket queue)
    traffic = traffic_pf * faces if traffic_pf and (
        tuning is None or (tuning["flux_min_ctas"] == 4 and tuning.get("flux_queue", 1) == 1)) else None
    hbm_peak = measured_hbm_gbs()
    if traffic and hbm_peak:
        comp["hbm"] = {"achieved": traffic / sec / 1e9, "peak": hbm_peak, "unit": "GB/s",
                       "frac": traffic / sec / 1e9 / hbm_peak}
    top = max(("fp32", "mufu"), key=lambda k: comp[k]["frac"])
    roof = {"bound": "alu", "achieved": comp[top]["achieved"], "peak": comp[top]["peak"],
            "unit": comp[top]["unit"] + (" (special-function unit)" if top == "mufu" else ""),
            "frac": comp[top]["frac"], "traffic": traffic,
            "kernel": f"k_fluxes<float,{riemann},{args.scheme}>", "kernel_ms": kern_ms,
            "work_per_face": {k: ops[k] for k in ("flop_base", "flop_per_iter", "mufu_base",
                                                 "mufu_per_iter")},
            "work_note": "operations of the oracle's face routine counted by its counting build "
                         "(oracle/face_work.py) on a sample of the same generator; each add, "
                         "mul, div, sqrt, pow one flop; special-function ops: div 1, sqrt 1, pow 2",
            "peak_note": "measured by hydro_probe_peak (burst, this GPU)", "components": comp,
            "fp64_peak_tflops": peaks["fp64"]}

    # ---- the other configurations at their full sizes (default workload only)
    others = None
    if (world == 1 and not args.no_others and args.workload == "lognormal" and n == DEFAULT_N["lognormal"]
            and args.precision == "mixed"):
        others = other_workloads(hydro, flush, stream)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu, _ = oracle_sample_rate(args.workload, args.cpu_n, args.cpu_reps)
        # the same sample on one core (one pass)
        one, _ = oracle_sample_rate(args.workload, args.cpu_n, 1, threads=1)
        cpu["single_core"] = {"value": one["value"], "cores": one["cores"], "sample": one["sample"]}
        # on a sample of the same generator the oracle also checks the GPU step
        cpu["gpu_parity_on_sample"] = oracle_sample_parity(args.workload, hydro)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "step_rate": step_rate,
        "grad_flux_ms_per_step": gf_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": wname, "particles": n,
                   "timed_steps": "each from the initial state (h: its converged smoothing lengths)" if restart else "consecutive",
                   "precision": args.precision, "scheme": args.scheme, "riemann": riemann,
                   "cuda_graph": bool(graph), "graph_steps": r["graph_steps"],
                   "tuning": tuning,
                   "kernel": "wendland_c2", "n_ngb": 32,
                   "l2": "flushed before every timed step (256 MB write)",
                   "particle_order": ("the library's Morton order, kept by sorted_output = 1 "
                                      "(the generator's order applied the step's permutation "
                                      "once, before timing)") if sorted_out else "the generator's",
                   "pairs_per_step": r["pairs"] / args.steps,
                   "grad_pairs": last["grad_pairs"], "flux_pairs": last["flux_pairs"],
                   "newton_iters_per_face": iters / max(faces, 1),
                   "learned_guess": learned, "riemann_polish": bool(args.riemann_polish),
                   "gravity": bool(args.gravity), "entropy_switch": bool(args.entropy),
                   "setup_s": setup_s},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": r["launches"],
        "clocks": clocks, "plain_fp64": fp64, "mixed_plain_guess": plain_guess,
        "error_vs_fp64": err64, "conservation": conservation, "other_workloads": others,
        "stage_ms": {k: last[k] for k in ("ms_neighbours", "ms_density", "ms_gradients",
                                          "ms_fluxes", "ms_flux_kernel", "ms_hard_faces",
                                          "ms_update")},
        "step_ms_each": [round(t, 3) for t in r["each_ms"]],
    }
    if learned:
        line["learned"] = dict(training, mode="adaptive (learned_guess = 1)",
                               active_steps=r["active"], hard_faces_per_step=hard,
                               learned_faces_per_step=r["learned"] / args.steps,
                               fallbacks_per_step=r["fallbacks"] / args.steps,
                               hard_kernel_ms=r["hard_ms"] / args.steps,
                               probe_ms_plain_learned=last["learned_probe_ms"])
        line["learned"].pop("theta")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def measured_hbm_gbs():
    """The measured HBM copy bandwidth of this machine's GPUs (GB/s), or None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError, TypeError):
        return None


def bench_rungs(args):
    """Individual timesteps: base steps of hydro_step_rungs, each from the
    initial state (dt0 = K CFL steps of it), L2 flushed before each."""
    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2211_12243_gb300 import build, hydro
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    kind = args.workload
    w, wname = make_workload(kind, args.n, seed=rank)
    n = w["x"].size
    riemann = args.riemann or ("hllc" if kind == "wave" else "exact")
    cfg = hydro.default_config(gamma=w["gamma"], scheme=args.scheme, riemann=riemann,
                               precision=args.precision, search_margin=1.15)
    H = hydro.Hydro(cfg)
    H.set_boxes(*boxes_of(hydro, w))
    H.reserve(n, 96)
    st = hydro.to_device(w)
    # the initial state's converged h and its CFL dt (one untimed step on a copy)
    tmp = {k: v.clone() for k, v in st.items()}
    s0 = H.step(tmp, -1.0, check=False)
    assert s0["status"] in (0, -5), s0
    st["h"].copy_(tmp["h"])
    del tmp
    dt0 = args.rungs * s0["dt"]
    saved = {k: v.clone() for k, v in st.items()}
    rung = torch.zeros(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        for k, v in saved.items():
            st[k].copy_(v)
        s = H.step_rungs(st, dt0, rung, check=False)
        assert s["status"] in (0, -5), s
    clk = ClockSampler(local)
    clk.start()
    ms, pairs, psteps, stats = 0.0, 0, 0, None
    launches0 = hydro.kernel_launches()
    for _ in range(args.steps):
        for k, v in saved.items():
            st[k].copy_(v)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats = H.step_rungs(st, dt0, rung, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        assert stats["status"] in (0, -5), stats
        ms += e0.elapsed_time(e1)
        pairs += stats["grad_pairs"] + stats["flux_pairs"]
        psteps += stats["active_steps"]
    launches = hydro.kernel_launches() - launches0
    clocks = clk.stop()
    pairs_all, ms_max, _ = aggregate(world, pairs, ms, ms, "cuda")
    hist = np.bincount(rung.cpu().numpy(), minlength=stats["rung_max"] + 1).tolist()
    line = {
        "metric": METRIC + " [individual timesteps: pairs over the whole base step]",
        "value": pairs_all / (ms_max / 1000.0), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": wname, "particles": n, "variant": "hydro_step_rungs",
                   "dt0_cfl_steps": args.rungs, "rung_histogram": hist,
                   "rung_max": stats["rung_max"], "substeps": stats["substeps"],
                   "particle_steps_per_base_step": psteps / args.steps,
                   "pairs_per_base_step": pairs / args.steps,
                   "precision": args.precision, "scheme": args.scheme, "riemann": riemann,
                   "timed_steps": "each from the initial state",
                   "l2": "flushed before every timed base step (256 MB write)"},
        "particle_steps_per_s": psteps * world / (ms_max / 1000.0),
        "gpu_launches": launches, "clocks": clocks, "roofline": None, "cpu_baseline": None,
        "e2e": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# Algorithmic work of one face, counted by the oracle's counting build on a
# sample of each generator (python -m oracle.face_work; tests check that
# these equal a fresh count): flops per face and per Newton iteration (each
# add, mul, div, sqrt, pow one flop) and special-function operations (div 1,
# sqrt 1, pow 2).  The batch of boxes takes the log-normal counts.
FACE_OPS = {
    "sod": {"flop_base": 481.469, "flop_per_iter": 44.0, "mufu_base": 84.65, "mufu_per_iter": 16.0},
    "sedov": {"flop_base": 504.363, "flop_per_iter": 44.0, "mufu_base": 77.628, "mufu_per_iter": 16.0},
    "lognormal": {"flop_base": 577.432, "flop_per_iter": 44.101, "mufu_base": 84.84,
                  "mufu_per_iter": 15.596},
    "wave": {"flop_base": 466.427, "flop_per_iter": 0.0, "mufu_base": 34.0, "mufu_per_iter": 0.0},
}
# DRAM bytes (read + write) per face of the flux kernel, from one ncu capture
# of the current kernel on a small case of the workload (profiles/); a
# launch's traffic scales with its faces
FLUX_TRAFFIC_BYTES_PER_FACE = {"sod": 28.56, "lognormal": 32.59}

if __name__ == "__main__":
    sys.exit(main())
