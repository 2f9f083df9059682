"""Helpers shared by the GPU parity tests: the same seeded workload is run
through the CUDA library (via its C ABI) and through the FP64 oracle, stage
by stage, and the outputs are compared."""
import math

import numpy as np

OPTS = ("kernel", "scheme", "riemann", "limiter", "time_extrap")


def oracle_cfg(orc, gamma, **kw):
    return orc.config(gamma=gamma, **kw)


def gpu_cfg(hydro, gamma, precision="fp64", **kw):
    return hydro.default_config(gamma=gamma, precision=precision, **kw)


def oracle_stages(orc, cfg, w, dt):
    x, y, z, L = w["x"], w["y"], w["z"], w["L"]
    h, om, it, st = orc.density(cfg, x, y, z, L, w["h"])
    assert st == 0
    prims = orc.primitives(cfg, w["m"], w["px"], w["py"], w["pz"], w["E"], w["U"], om)
    B6, E6, nc = orc.matrices(cfg, x, y, z, L, h, om)
    grad, alpha, vsig = orc.gradients(cfg, x, y, z, L, h, om, prims, B6, nc)
    dQ, fst, _, dQabs = orc.fluxes(cfg, x, y, z, L, h, om, B6, prims, grad, alpha, dt,
                                   want_abs=True)
    return dict(h=h, omega=om, B=B6, grad=grad, alpha=alpha, ncond=nc, dQ=dQ, dQabs=dQabs,
                prims=prims, vsig=vsig, flux=fst, gamma=cfg.gamma)


def gpu_stages(hydro, H, w, dt, search=1.3, boxes=None):
    import torch
    st = hydro.to_device(w)
    if boxes is None:
        boxes = hydro.single_box(w)
    H.set_boxes(*boxes)
    hs = st["h"] * search
    H.build_neighbours(st, hs, export=False)
    H.density(st)
    B, G, A, N = H.gradients(st)
    dQ = H.fluxes(st, B, G, A, dt)
    torch.cuda.synchronize()
    c = lambda t: t.detach().cpu().numpy()
    return dict(h=c(st["h"]), omega=c(st["omega"]), B=c(B), grad=c(G), alpha=c(A), ncond=c(N),
                dQ=c(dQ))


def flux_scale(o, gamma=None):
    """Per-particle, per-component scale of the flux sums: the oracle's sum
    over the particle's faces of |c| (the net can cancel).  A component that
    vanishes identically on every face (the mass flux of a fluid at rest,
    the energy flux of a static pressure field) takes the scale it would
    have from the momentum flux through the sound speed: mass ~ |c_P| / c_s,
    energy ~ |c_P| c_s."""
    a = o["dQabs"]
    rho, vx, vy, vz, p = o["prims"]
    g = o.get("gamma", 5.0 / 3.0) if gamma is None else gamma
    cs = np.sqrt(g * p / rho)
    pm = a[:, 1] + a[:, 2] + a[:, 3]
    sc = np.empty_like(a)
    sc[:, 0] = np.maximum(a[:, 0], pm / cs)
    sc[:, 1] = sc[:, 2] = sc[:, 3] = pm
    sc[:, 4] = np.maximum(a[:, 4], pm * cs)
    return sc + 1e-300


def rel_err(a, b, scale):
    return np.max(np.abs(a - b) / scale)


def compare(g, o, tol, what=("h", "omega", "B", "grad", "ncond", "dQ")):
    """Worst normalised error per quantity.  Scales: h, omega, N_cond: the
    value; B: the row's largest entry; limited gradients alpha*grad: |grad| +
    |f_i|/h_i (a gradient's natural size); dQ: the particle's sum of |c| over
    its faces (the net can cancel)."""
    errs = {}
    if "h" in what:
        errs["h"] = rel_err(g["h"], o["h"], np.abs(o["h"]))
    if "omega" in what:
        errs["omega"] = rel_err(g["omega"], o["omega"], np.abs(o["omega"]))
    if "B" in what:
        sc = np.abs(o["B"]).max(1, keepdims=True)
        errs["B"] = rel_err(g["B"], o["B"], sc)
    if "ncond" in what:
        errs["ncond"] = rel_err(g["ncond"], o["ncond"], np.abs(o["ncond"]))
    if "grad" in what:
        lg_g = g["alpha"][:, :, None] * g["grad"]
        lg_o = o["alpha"][:, :, None] * o["grad"]
        f = np.stack(o["prims"], 1)
        sc = np.abs(lg_o) + (np.abs(f) / o["h"][:, None])[:, :, None] + 1e-300
        errs["grad"] = rel_err(lg_g, lg_o, sc)
    if "dQ" in what:
        errs["dQ"] = rel_err(g["dQ"][:, :5], o["dQ"][:, :5], flux_scale(o))
    bad = {k: v for k, v in errs.items() if not (v <= tol)}
    return errs, bad


def conservation(before, after, gamma):
    """Relative drift of total mass, momentum (per axis, scaled by
    sum m (|v| + c_s)) and energy between two states (dicts of numpy)."""
    m0 = before["m"]
    v = np.stack([before["px"], before["py"], before["pz"]], 1) / m0[:, None]
    cs = np.sqrt(np.maximum(gamma * (gamma - 1) * before["U"] / m0, 0))
    out = {}
    out["M"] = abs(math.fsum(after["m"]) - math.fsum(before["m"])) / math.fsum(np.abs(before["m"]))
    out["E"] = abs(math.fsum(after["E"]) - math.fsum(before["E"])) / math.fsum(np.abs(before["E"]))
    ps = math.fsum(m0 * (np.linalg.norm(v, axis=1) + cs))
    for k in ("px", "py", "pz"):
        out[k] = abs(math.fsum(after[k]) - math.fsum(before[k])) / ps
    return out


def well_conditioned(orc, w, o, crit=100.0):
    """Particles whose own E and whose neighbours' E are well conditioned
    (N_cond <= crit): the staged calls run without the N_cond guard, and for
    a (near-)singular E the inverse is rounding noise in any precision."""
    ok = o["ncond"] <= crit
    off, idx = orc.neighbours(w["x"], w["y"], w["z"], w["L"], o["h"] * 1.0000001)
    good = ok.copy()
    for i in np.nonzero(ok)[0]:
        good[i] = ok[idx[off[i]:off[i + 1]]].all()
    return ok, good


def mask_conditioned(o, g, ok, good):
    o2, g2 = dict(o), dict(g)
    for k in ("B", "grad", "alpha", "ncond"):
        o2[k], g2[k] = o[k][ok], g[k][ok]
    o2["prims"] = tuple(p[ok] for p in o["prims"])
    o2["h_m"] = o["h"][ok]
    for k in ("dQ", "dQabs"):
        o2[k] = o[k][good]
    g2["dQ"] = g["dQ"][good]
    o2["prims_g"] = tuple(p[good] for p in o["prims"])
    return o2, g2


def compare_masked(orc, w, o, g, tol, what):
    ok, good = well_conditioned(orc, w, o)
    assert good.mean() > 0.9
    o2, g2 = mask_conditioned(o, g, ok, good)
    errs, bad = {}, {}
    e, b = compare(g, o, tol, what=tuple(k for k in what if k in ("h", "omega")))
    errs.update(e); bad.update(b)
    oh = dict(o2, h=o2["h_m"])
    e, b = compare(g2, oh, tol, what=tuple(k for k in what if k in ("B", "grad", "ncond")))
    errs.update(e); bad.update(b)
    if "dQ" in what:
        od = dict(o2, prims=o2["prims_g"])
        e, b = compare(g2, od, tol, what=("dQ",))
        errs.update(e); bad.update(b)
    return errs, bad
