"""The paper's hydro validation problems (§3.1), run as multi-step
simulations on the GPU through the C ABI:

* sound waves (§3.1.1): gamma = 1.4, c_s = sqrt(gamma), cubic spline,
  N_NGB = 32, one wavelength along x, a few particle planes across; the L1
  norm of the density after one crossing time converges at second order
  (limiter off, as in the paper) up to 128 particles per wavelength;
* Sod shock tube (§3.1.2): (1, 0, 1) | (0.25, 0, 0.1795), gamma = 1.4,
  N_NGB = 64, cubic-spline kernel, t = 0.13, against the exact solution
  (the oracle's exact Riemann sampler); the L1 errors fall with resolution
  and transverse velocities stay negligible;
* Gresho-Chan vortex (§3.1.3): triangular v_phi profile in pressure balance,
  rho = 1, gamma = 1.4, p(0) = 5, 64^2 particles per plane of side 2 on a
  Cartesian lattice, to t = 3: the profile is kept up to a small decay.

Densities are set through the particle masses on a uniform lattice (a
reading: the paper sets them through the number density for the tube).
Printed figures: pytest -s."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hyd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_12243_gb300 import build, hydro
    build.build()
    return hydro


def _lattice(nx, ny, nz, a):
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    return ((i.ravel() + 0.5) * a, (j.ravel() + 0.5) * a, (k.ravel() + 0.5) * a)


def _pack(x, y, z, L, rho, vx, vy, vz, p, a, gamma, n_ngb, kernel_kn):
    vol = a ** 3
    m = rho * vol
    U = p * vol / (gamma - 1.0)
    E = U + 0.5 * m * (vx * vx + vy * vy + vz * vz)
    # h from the lattice number density: (4 pi / 3) h^3 / a^3 = N_NGB
    h = np.full(x.size, (3.0 * n_ngb / (4.0 * math.pi)) ** (1.0 / 3.0) * a)
    return dict(x=x, y=y, z=z, m=m, px=m * vx, py=m * vy, pz=m * vz, E=E, U=U, h=h,
                L=np.asarray(L, dtype=np.float64), gamma=gamma)


def _evolve(hyd, w, cfg, t_end):
    """Steps of the CFL timestep, the last one cut to land on t_end."""
    import torch
    H = hyd.Hydro(cfg)
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    t = 0.0
    dt_next = None
    while t < t_end * (1.0 - 1e-12):
        dt = -1.0
        if dt_next is not None and t + dt_next >= t_end:
            dt = t_end - t
        s = H.step(st, dt)
        assert s["status"] == 0, s
        t += s["dt"]
        dt_next = s["dt_next"]
    torch.cuda.synchronize()
    # volumes at the final positions
    H.build_neighbours(st, st["h"] * 1.3, export=False)
    H.density(st)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in st.items()}
    H.close()
    return out, t


def _soundwave(n, planes=8, A=1e-3, gamma=1.4):
    a = 1.0 / n
    x, y, z = _lattice(n, planes, planes, a)
    cs = math.sqrt(gamma)
    ph = np.cos(2.0 * math.pi * x)
    rho = 1.0 + A * ph
    p = 1.0 + A * gamma * ph
    vx = A * cs * ph
    zero = np.zeros_like(x)
    return _pack(x, y, z, (1.0, planes * a, planes * a), rho, vx, zero, zero, p, a, gamma,
                 32.0, None), cs


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
def test_soundwave_converges_at_second_order(hyd, scheme):
    """The paper's setup (cubic spline, N_NGB = 32, limiter off) at
    amplitude 1e-5 (at the paper's 1e-3 the wave's nonlinear steepening over
    one crossing, O(A^2), is reached by N = 64) for N = 16 ... 128."""
    A, gamma = 1e-5, 1.4
    l1 = {}
    for n in (16, 32, 64, 128):
        w, cs = _soundwave(n, A=A, gamma=gamma)
        cfg = hyd.default_config(gamma=gamma, precision="fp64", scheme=scheme, limiter=0,
                                 c_cfl=0.1, kernel="cubic")
        out, t = _evolve(hyd, w, cfg, 1.0 / cs)
        # the kernel estimate of the density of a lattice carries a uniform
        # bias of a few per cent (the discrete sum of W is not 1/a^3): the
        # perturbation is measured against the mean estimate
        rho = out["m"] / out["omega"]
        delta = rho / np.mean(rho) - 1.0
        exact = A * np.cos(2.0 * math.pi * out["x"] - 2.0 * math.pi * cs * t)
        l1[n] = float(np.mean(np.abs(delta - exact)))
        vt = np.sqrt(np.mean((out["py"] / out["m"]) ** 2 + (out["pz"] / out["m"]) ** 2))
        assert vt < 1e-12, (n, vt)   # no transverse motion grows
    orders = [math.log2(l1[a] / l1[b]) for a, b in ((16, 32), (32, 64), (64, 128))]
    print(f"soundwave {scheme}: L1 {l1}, orders {[round(o, 2) for o in orders]}")
    # second order (the paper: both schemes); measured MFV 1.77 / 2.01 / 2.00,
    # MFM 2.24 / 2.09 / 2.03 with the FP64 oracle
    assert orders[0] > 1.6 and orders[1] > 1.8 and orders[2] > 1.8, (l1, orders)
    assert l1[128] < 2e-3 * A, l1


def _sod(n, planes=8, gamma=1.4):
    """Periodic tube [0, 2): left half (1, 0, 1), right half (0.25, 0, 0.1795);
    n particles per unit length."""
    a = 1.0 / n
    x, y, z = _lattice(2 * n, planes, planes, a)
    left = x < 1.0
    rho = np.where(left, 1.0, 0.25)
    p = np.where(left, 1.0, 0.1795)
    zero = np.zeros_like(x)
    return _pack(x, y, z, (2.0, planes * a, planes * a), rho, zero, zero, zero, p, a, gamma,
                 64.0, None)


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
def test_sod_gamma_1_4_follows_exact_solution(orc, hyd, scheme):
    gamma, t_end = 1.4, 0.13
    r = orc.riemann_star(1.0, 0.0, 1.0, 0.25, 0.0, 0.1795, gamma)
    errs = {}
    for n in (100, 200):
        w = _sod(n, gamma=gamma)
        cfg = hyd.default_config(gamma=gamma, precision="mixed", scheme=scheme, kernel="cubic",
                                 n_ngb=64.0)
        out, t = _evolve(hyd, w, cfg, t_end)
        x = out["x"]
        sel = (x > 0.6) & (x < 1.4)
        ex = []
        for xi in x[sel]:
            c = (xi - 1.0) / t
            rr, uu, pp, _ = orc.riemann_sample(1.0, -c, 1.0, 0.25, -c, 0.1795, gamma, r["p"],
                                               r["u"] - c)
            ex.append((rr, uu + c, pp))
        ex = np.array(ex)
        m, om = out["m"][sel], out["omega"][sel]
        rho = m / om
        vx = out["px"][sel] / m
        vy, vz = out["py"][sel] / m, out["pz"][sel] / m
        ekin = 0.5 * m * (vx * vx + vy * vy + vz * vz)
        p = (out["E"][sel] - ekin) * (gamma - 1.0) / om
        errs[n] = [float(np.mean(np.abs(f - ex[:, k]))) for k, f in enumerate((rho, vx, p))]
        # transverse motion negligible (the paper's check)
        assert np.abs(vy).max() < 1e-2 and np.abs(vz).max() < 1e-2, n
    print(f"sod gamma 1.4 {scheme}: L1 (rho, vx, p) {errs}")
    for k in range(3):
        # shocks converge at first order: doubling n must lower every error
        assert errs[200][k] < 0.8 * errs[100][k], (k, errs)
    # at n = 200 the profiles follow the exact solution closely
    assert errs[200][0] < 0.03 and errs[200][1] < 0.05 and errs[200][2] < 0.03, errs


def _gresho(n=64, planes=8, gamma=1.4):
    a = 2.0 / n
    x, y, z = _lattice(n, n, planes, a)
    dx, dy = x - 1.0, y - 1.0
    r = np.sqrt(dx * dx + dy * dy)
    vphi = np.where(r <= 0.2, 5.0 * r, np.where(r < 0.4, 2.0 - 5.0 * r, 0.0))
    rs = np.maximum(r, 1e-300)
    p = np.where(r <= 0.2, 5.0 + 12.5 * r * r,
                 np.where(r < 0.4, 9.0 + 12.5 * r * r - 20.0 * r + 4.0 * np.log(rs / 0.2),
                          3.0 + 4.0 * math.log(2.0)))
    vx, vy = -vphi * dy / rs, vphi * dx / rs
    rho = np.ones_like(x)
    return _pack(x, y, z, (2.0, 2.0, planes * a), rho, vx, vy, np.zeros_like(x), p, a, gamma,
                 32.0, None)


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
def test_gresho_vortex_keeps_its_profile(hyd, scheme):
    gamma = 1.4
    w = _gresho(gamma=gamma)
    cfg = hyd.default_config(gamma=gamma, precision="mixed", scheme=scheme)
    out, t = _evolve(hyd, w, cfg, 3.0)
    m = out["m"]
    dx, dy = out["x"] - 1.0, out["y"] - 1.0
    r = np.sqrt(dx * dx + dy * dy)
    vx, vy = out["px"] / m, out["py"] / m
    vphi = (-vx * dy + vy * dx) / np.maximum(r, 1e-300)
    want = np.where(r <= 0.2, 5.0 * r, np.where(r < 0.4, 2.0 - 5.0 * r, 0.0))
    sel = r < 0.5
    l1 = float(np.mean(np.abs(vphi[sel] - want[sel])))
    # the binned profile's peak (1 at r = 0.2 initially)
    edges = np.linspace(0.0, 0.5, 26)
    idx = np.digitize(r, edges) - 1
    prof = np.array([vphi[idx == k].mean() for k in range(25)])
    rc = 0.5 * (edges[1:] + edges[:-1])
    kpk = int(np.argmax(prof))
    # angular momentum about the vortex axis (not conserved to rounding by the
    # scheme, only approximately)
    lz0 = np.sum(w["m"] * ((w["x"] - 1.0) * w["py"] / w["m"] - (w["y"] - 1.0) * w["px"] / w["m"]))
    lz1 = np.sum(m * (dx * vy - dy * vx))
    print(f"gresho {scheme}: t = {t:.3f}, L1(v_phi) = {l1:.4f}, peak {prof[kpk]:.3f} at "
          f"r = {rc[kpk]:.2f}, Lz {lz0:.6f} -> {lz1:.6f}")
    # the profile keeps its shape and position with a decay of its peak over
    # the 2.4 orbits (measured: peak 0.72 at r = 0.19, L1 0.085-0.09, Lz
    # within 4%), momentum is conserved to rounding
    assert prof[kpk] > 0.65 and 0.15 < rc[kpk] < 0.25, (prof, rc)
    assert l1 < 0.12, l1
    assert abs(lz1 - lz0) < 0.06 * abs(lz0), (lz0, lz1)
    # linear momentum is conserved by construction
    assert abs(np.sum(out["px"])) < 1e-12 * np.sum(np.abs(w["px"])) + 1e-15


def _evolve_rungs(hyd, w, cfg, t_end, mult=4.0):
    """Base steps of hydro_step_rungs of mult CFL steps each (the CFL dt of
    the base step's start, from a global step on a copy), the last cut to
    land on t_end."""
    import torch
    H = hyd.Hydro(cfg)
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    rung = torch.zeros(w["x"].size, dtype=torch.int32, device="cuda")
    t, rungs = 0.0, set()
    while t < t_end * (1.0 - 1e-12):
        probe = {k: v.clone() for k, v in st.items()}
        dt_cfl = H.step(probe, -1.0)["dt"]
        dt0 = min(mult * dt_cfl, t_end - t)
        s = H.step_rungs(st, dt0, rung)
        assert s["status"] == 0, s
        rungs |= set(np.unique(rung.cpu().numpy()).tolist())
        t += dt0
    torch.cuda.synchronize()
    H.build_neighbours(st, st["h"] * 1.3, export=False)
    H.density(st)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in st.items()}
    H.close()
    return out, t, rungs


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
def test_sod_with_individual_timesteps_follows_exact_solution(orc, hyd, scheme):
    """The gamma = 1.4 tube at n = 100 run with individual timesteps (base
    steps of four CFL steps, §2.3.4, §2.3.10) stays as close to the exact
    solution as the global CFL-stepped run."""
    gamma, t_end = 1.4, 0.13
    r = orc.riemann_star(1.0, 0.0, 1.0, 0.25, 0.0, 0.1795, gamma)
    w = _sod(100, gamma=gamma)
    cfg = hyd.default_config(gamma=gamma, precision="mixed", scheme=scheme, kernel="cubic",
                             n_ngb=64.0)
    errs = {}
    outs = {"global": _evolve(hyd, w, cfg, t_end)[:2]}
    o, t, rungs = _evolve_rungs(hyd, w, cfg, t_end)
    outs["rungs"] = (o, t)
    assert len(rungs) >= 2, rungs
    for mode, (out, t) in outs.items():
        x = out["x"]
        sel = (x > 0.6) & (x < 1.4)
        ex = np.array([orc.riemann_sample(1.0, -(xi - 1.0) / t, 1.0, 0.25, -(xi - 1.0) / t, 0.1795,
                                          gamma, r["p"], r["u"] - (xi - 1.0) / t)[0]
                       for xi in x[sel]])
        errs[mode] = float(np.mean(np.abs(out["m"][sel] / out["omega"][sel] - ex)))
    print(f"sod rungs {scheme}: L1(rho) {errs}, rungs {sorted(rungs)}")
    assert errs["rungs"] < 1.3 * errs["global"] + 2e-3, errs
    assert errs["rungs"] < 0.03, errs
