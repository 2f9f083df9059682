"""Pins of the FP64 oracle against facts that do not come from the oracle:
closed forms, textbook values, library routines, symmetries and invariants
of the method (arXiv:2211.12243 §2.3).  CPU only."""
import math
import os

import numpy as np
import pytest
from scipy import integrate, optimize
from scipy.spatial import cKDTree

from paper_2211_12243_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# kernel (§2.3.2): unit normalisation and compact support
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kernel", ["wendland", "cubic"])
@pytest.mark.parametrize("H", [1.0, 0.37, 2.5])
def test_kernel_unit_integral(orc, kernel, H):
    f = lambda r: 4.0 * math.pi * r * r * float(orc.kernel_W(r, H, kernel))
    val, err = integrate.quad(f, 0.0, H, epsabs=1e-14, epsrel=1e-13, points=[0.5 * H])
    assert abs(val - 1.0) < 1e-12


def test_kernel_central_values_and_support(orc):
    # Wendland C2: W(0,H) = 21/(2 pi H^3); cubic M4: 8/(pi H^3)
    assert float(orc.kernel_W(0.0, 1.0, "wendland")) == pytest.approx(21 / (2 * math.pi), rel=1e-15)
    assert float(orc.kernel_W(0.0, 2.0, "cubic")) == pytest.approx(8 / (math.pi * 8), rel=1e-15)
    for k in ("wendland", "cubic"):
        assert float(orc.kernel_W(1.0, 1.0, k)) == 0.0
        assert float(orc.kernel_W(1.3, 1.0, k)) == 0.0
        # continuity of the cubic spline at q = 1/2
    a = float(orc.kernel_W(0.5 - 1e-12, 1.0, "cubic"))
    b = float(orc.kernel_W(0.5 + 1e-12, 1.0, "cubic"))
    assert abs(a - b) < 1e-10


@pytest.mark.parametrize("kernel", ["wendland", "cubic"])
def test_kernel_dWdH_matches_difference_quotient(orc, kernel):
    for r in (0.05, 0.3, 0.49, 0.51, 0.8, 0.97):
        H, e = 1.0, 1e-6
        fd = (float(orc.kernel_W(r, H + e, kernel)) - float(orc.kernel_W(r, H - e, kernel))) / (2 * e)
        assert float(orc.kernel_dWdH(r, H, kernel)) == pytest.approx(fd, rel=1e-6, abs=1e-9)


# --------------------------------------------------------------------------
# neighbour search (§2.2.3): brute force, the cell grid and scipy agree
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L", [(1.0, 1.0, 1.0), (4.0, 1.0, 1.0), (1.0, 2.0, 0.5)])
def test_neighbours_match_kdtree_and_brute_force(orc, L):
    rng = np.random.default_rng(7)
    n = 1500
    L = np.array(L)
    pos = rng.random((n, 3)) * L
    hs = rng.uniform(0.05, 0.2, n) * L.min()
    off_b, idx_b = orc.neighbours(pos[:, 0], pos[:, 1], pos[:, 2], L, hs, use_grid=False)
    off_g, idx_g = orc.neighbours(pos[:, 0], pos[:, 1], pos[:, 2], L, hs, use_grid=True)
    assert np.array_equal(off_b, off_g) and np.array_equal(idx_b, idx_g)
    tree = cKDTree(pos, boxsize=L)
    for i in range(n):
        ref = sorted(tree.query_ball_point(pos[i], hs[i]))
        got = idx_b[off_b[i]:off_b[i + 1]].tolist()
        assert got == ref
        assert i in got  # self included


@pytest.mark.parametrize("L", [(1.0, 1.0, 1.0), (1.0, 0.5, 2.0)])
def test_flux_pairs_match_brute_force(orc, L):
    """The faces of §2.3.3: every unordered pair {i, j} with r_ij < max(h_i, h_j)
    (periodic minimum image) exactly once, against an O(N^2) enumeration;
    with unequal h most pairs are seen from one side only."""
    rng = np.random.default_rng(13)
    n = 400
    L = np.array(L)
    pos = rng.random((n, 3)) * L
    h = rng.uniform(0.05, 0.25, n) * L.min()
    pairs = orc.flux_pairs(pos[:, 0], pos[:, 1], pos[:, 2], L, h)
    got = {(min(a, b), max(a, b)) for a, b in pairs.tolist()}
    assert len(got) == pairs.shape[0]             # each pair once
    d = pos[None, :, :] - pos[:, None, :]
    d -= np.round(d / L) * L
    r = np.sqrt(np.sum(d * d, 2))
    i, j = np.nonzero(np.triu(r < np.maximum(h[:, None], h[None, :]), 1))
    ref = set(zip(i.tolist(), j.tolist()))
    assert got == ref
    one_sided = np.sum((r[i, j] < np.maximum(h[i], h[j])) & (r[i, j] >= np.minimum(h[i], h[j])))
    assert one_sided > 0.2 * len(ref)


# --------------------------------------------------------------------------
# density and smoothing length (§2.3.2, §2.3.5 Eq. 18)
# --------------------------------------------------------------------------
def _lattice_shells(rmax):
    """(distance/a, multiplicity) of simple-cubic lattice shells below rmax*a."""
    k = int(math.ceil(rmax)) + 1
    g = np.arange(-k, k + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    r2 = (X * X + Y * Y + Z * Z).ravel()
    vals, counts = np.unique(r2, return_counts=True)
    keep = np.sqrt(vals) < rmax
    return np.sqrt(vals[keep]), counts[keep]


def test_density_on_perfect_lattice_matches_shell_sum(orc):
    # perfect lattice: h solves (4 pi/3) h^3 sum_shells c_s W(r_s, h) = N_NGB,
    # computed here by counting lattice shells, independently of the search
    n = 10
    w = W.lattice_wave(n, jitter=0.0)
    cfg = orc.config()
    h, om, it, st = orc.density(cfg, w["x"], w["y"], w["z"], w["L"], w["h"])
    assert st == 0
    a = 1.0 / n
    r, c = _lattice_shells(4.0)

    def g(hh):
        q = r * a / hh
        t = np.clip(1 - q, 0, None)
        Wsum = np.sum(c * 21 / (2 * math.pi * hh ** 3) * t ** 4 * (1 + 4 * q))
        return 4 * math.pi / 3 * hh ** 3 * Wsum - 32.0

    href = optimize.brentq(g, 1.2 * a, 3.0 * a, xtol=1e-16, rtol=1e-15)
    assert np.allclose(h, href, rtol=1e-12, atol=0)
    assert np.ptp(h) / href < 1e-12 and np.ptp(om) / om.mean() < 1e-12


def test_density_partition_of_unity_volume(orc):
    # Eq. 7 with f = 1: sum_i V_i approximates the box volume to O(h^2)
    w = W.lattice_wave(12)
    cfg = orc.config()
    h, om, it, st = orc.density(cfg, w["x"], w["y"], w["z"], w["L"], w["h"])
    assert st == 0
    assert abs(om.sum() - 1.0) < 0.05


def test_density_residual_and_monotone_bracket(orc):
    # the returned h is a root: moving h by +-1e-9 relative flips the sign of
    # (4 pi/3) h^3 n(h) - N, evaluated on an independent KD-tree neighbour set
    w = W.lognormal(3000, seed=1, grid=16, contrast=100.0)
    cfg = orc.config()
    h, om, it, st = orc.density(cfg, w["x"], w["y"], w["z"], w["L"], w["h"])
    assert st == 0 and it.max() < 40
    pos = np.stack([w["x"], w["y"], w["z"]], 1)
    tree = cKDTree(pos, boxsize=w["L"])
    for i in range(0, 3000, 97):
        for s, sign in ((1 - 1e-9, -1), (1 + 1e-9, 1)):
            hh = h[i] * s
            js = tree.query_ball_point(pos[i], hh)
            d = pos[js] - pos[i]
            d -= np.round(d / w["L"]) * w["L"]
            q = np.linalg.norm(d, axis=1) / hh
            t = np.clip(1 - q, 0, None)
            val = 4 * math.pi / 3 * hh ** 3 * np.sum(21 / (2 * math.pi * hh ** 3) * t ** 4 * (1 + 4 * q)) - 32
            assert np.sign(val) == sign
        # omega is 1/sum_j W at the converged h (independent neighbour set)
        js = tree.query_ball_point(pos[i], h[i])
        d = pos[js] - pos[i]
        d -= np.round(d / w["L"]) * w["L"]
        q = np.linalg.norm(d, axis=1) / h[i]
        t = np.clip(1 - q, 0, None)
        Wsum = np.sum(21 / (2 * math.pi * h[i] ** 3) * t ** 4 * (1 + 4 * q))
        assert om[i] == pytest.approx(1 / Wsum, rel=1e-12)


# --------------------------------------------------------------------------
# E matrix, B = E^-1, N_cond (Eqs. 11, 19)
# --------------------------------------------------------------------------
def _b9(B6):
    xx, xy, xz, yy, yz, zz = B6.T
    return np.stack([np.stack([xx, xy, xz], -1), np.stack([xy, yy, yz], -1),
                     np.stack([xz, yz, zz], -1)], -2)


def test_matrices_inverse_and_isotropic_lattice(orc):
    n = 10
    w = W.lattice_wave(n, jitter=0.0)
    cfg = orc.config()
    h, om, _, _ = orc.density(cfg, w["x"], w["y"], w["z"], w["L"], w["h"])
    B6, E6, nc = orc.matrices(cfg, w["x"], w["y"], w["z"], w["L"], h, om)
    B, E = _b9(B6), _b9(E6)
    I = np.einsum("nij,njk->nik", B, E)
    assert np.abs(I - np.eye(3)).max() < 1e-12
    # cubic symmetry: E proportional to I, so N_cond = 1 (§2.3.5)
    assert np.abs(nc - 1.0).max() < 1e-12
    # value of E_xx from lattice shells: sum_s omega W(r_s,h) * sum_{d in shell} d_x^2
    a = 1.0 / n
    r, c = _lattice_shells(h[0] / a)
    # sum over a shell of d_x^2 = c_s r_s^2 a^2 / 3 by cubic symmetry
    q = r * a / h[0]
    t = np.clip(1 - q, 0, None)
    Wr = 21 / (2 * math.pi * h[0] ** 3) * t ** 4 * (1 + 4 * q)
    Exx = np.sum(om[0] * Wr * c * (r * a) ** 2 / 3.0)
    assert E6[:, 0] == pytest.approx(Exx, rel=1e-12)
    assert np.abs(E6[:, 1]).max() < 1e-12 * Exx


def test_ncond_detects_planar_neighbourhood(orc):
    # all particles in one plane z = const: E is singular -> N_cond = inf
    n = 12
    a = 1.0 / n
    g = (np.arange(n) + 0.5) * a
    X, Y = np.meshgrid(g, g, indexing="ij")
    x, y = X.ravel(), Y.ravel()
    z = np.full(x.size, 0.5)
    L = np.array([1.0, 1.0, 1.0])
    h = np.full(x.size, 3.1 * a)
    om = np.full(x.size, a * a)
    cfg = orc.config()
    B6, E6, nc = orc.matrices(cfg, x, y, z, L, h, om)
    assert np.all(~np.isfinite(nc) | (nc > 1e8))


# --------------------------------------------------------------------------
# gradient estimator (Eq. 10): linear exactness, quadratic on a lattice
# --------------------------------------------------------------------------
def _state_with_primitives(orc, cfg, w, rho, v, p):
    h, om, _, st = orc.density(cfg, w["x"], w["y"], w["z"], w["L"], w["h"])
    assert st == 0
    m = rho * om
    U = p * om / (cfg.gamma - 1.0)
    P = v * m[:, None]
    E = U + 0.5 * m * np.sum(v * v, 1)
    return h, om, m, P, E, U


def test_gradients_exact_for_linear_fields(orc):
    w = W.lattice_wave(12, jitter=0.05)
    cfg = orc.config()
    x = np.stack([w["x"], w["y"], w["z"]], 1)
    g = np.array([[0.3, -0.2, 0.1], [0.05, 0.02, -0.04], [-0.01, 0.03, 0.02],
                  [0.02, 0.0, 0.01], [0.2, 0.1, -0.3]])
    c0 = np.array([2.0, 0.1, -0.2, 0.05, 3.0])
    f = c0 + (x - 0.5) @ g.T   # linear inside the box
    rho, v, p = f[:, 0], f[:, 1:4], f[:, 4]
    h, om, m, P, E, U = _state_with_primitives(orc, cfg, w, rho, v, p)
    prims = orc.primitives(cfg, m, P[:, 0], P[:, 1], P[:, 2], E, U, om)
    assert np.allclose(prims[0], rho, rtol=1e-13) and np.allclose(prims[4], p, rtol=1e-12)
    B6, E6, nc = orc.matrices(cfg, w["x"], w["y"], w["z"], w["L"], h, om)
    grad, alpha, vsig = orc.gradients(cfg, w["x"], w["y"], w["z"], w["L"], h, om, prims, B6, nc)
    inner = np.all((x > h.max() + 1e-3) & (x < 1 - h.max() - 1e-3), axis=1)
    assert inner.sum() > 50
    assert np.abs(grad[inner] - g[None]).max() < 1e-10
    # linear fields create no new extrema: the limiter leaves them alone
    assert np.all(alpha[inner] == 1.0)


def test_gradients_exact_for_quadratic_on_perfect_lattice(orc):
    # odd moments of a cubic lattice neighbourhood vanish, so the LV estimator
    # is exact for quadratics at lattice points (second order, §2.3.3)
    n = 12
    w = W.lattice_wave(n, jitter=0.0)
    cfg = orc.config(limiter=False)
    x = np.stack([w["x"], w["y"], w["z"]], 1) - 0.5
    Hq = np.array([[0.4, 0.1, -0.2], [0.1, -0.3, 0.05], [-0.2, 0.05, 0.2]])
    f = 5.0 + 0.5 * np.einsum("ni,ij,nj->n", x, Hq, x) + x @ np.array([0.1, 0.2, 0.3])
    v = np.zeros((x.shape[0], 3))
    h, om, m, P, E, U = _state_with_primitives(orc, cfg, w, f, v, np.full(x.shape[0], 1.0))
    prims = orc.primitives(cfg, m, P[:, 0], P[:, 1], P[:, 2], E, U, om)
    B6, E6, nc = orc.matrices(cfg, w["x"], w["y"], w["z"], w["L"], h, om)
    grad, alpha, vsig = orc.gradients(cfg, w["x"], w["y"], w["z"], w["L"], h, om, prims, B6, nc)
    inner = np.all(np.abs(x) < 0.5 - h.max() - 1e-3, axis=1)
    exact = x @ Hq.T + np.array([0.1, 0.2, 0.3])
    assert np.abs(grad[inner, 0] - exact[inner]).max() < 1e-10


def test_limiter_bounds(orc):
    # conditioned BJ: after limiting, every midpoint extrapolation stays within
    # beta * (f_max - f_i) and beta * (f_min - f_i), beta in [1, 2]; a step
    # function is limited (alpha < 1) next to the jump
    w = W.lattice_wave(10, jitter=0.1)
    cfg = orc.config()
    x = np.stack([w["x"], w["y"], w["z"]], 1)
    rho = np.where(x[:, 0] < 0.5, 1.0, 4.0)
    p = np.where(x[:, 0] < 0.5, 1.0, 0.5)
    v = np.zeros_like(x)
    h, om, m, P, E, U = _state_with_primitives(orc, cfg, w, rho, v, p)
    prims = orc.primitives(cfg, m, P[:, 0], P[:, 1], P[:, 2], E, U, om)
    B6, E6, nc = orc.matrices(cfg, w["x"], w["y"], w["z"], w["L"], h, om)
    grad, alpha, vsig = orc.gradients(cfg, w["x"], w["y"], w["z"], w["L"], h, om, prims, B6, nc)
    assert np.all(alpha <= 1.0) and np.all(alpha >= 0.0)
    near = np.abs(x[:, 0] - 0.5) < 0.5 / 10
    assert np.all(alpha[near, 0] < 1.0)
    off, idx = orc.neighbours(w["x"], w["y"], w["z"], w["L"], h)
    for i in range(0, x.shape[0], 37):
        js = idx[off[i]:off[i + 1]]
        d = x[js] - x[i]
        d -= np.round(d) * 1.0
        for f in range(5):
            vals = prims[f][js]
            fmax, fmin = vals.max(), vals.min()
            ext = 0.5 * d @ (alpha[i, f] * grad[i, f])
            assert ext.max() <= 2.0 * (fmax - prims[f][i]) + 1e-12
            assert ext.min() >= 2.0 * (fmin - prims[f][i]) - 1e-12


@pytest.mark.parametrize("k", [0.3, -0.3, 0.0])
def test_signal_velocity_closed_form(orc, k):
    """The signal velocity of the CFL condition (Eqs. 31-32): at rest or in
    a uniform expansion every pair carries 2c; a uniform compression
    v = -k x adds the approach speed k r_ij, largest for the farthest
    neighbour within h (found by brute force)."""
    n = 12
    w = W.lattice_wave(n, jitter=0.0)
    cfg = orc.config()
    x = np.stack([w["x"], w["y"], w["z"]], 1) - 0.5
    N = x.shape[0]
    v = -k * x
    h, om, m, P, E, U = _state_with_primitives(orc, cfg, w, np.full(N, 1.0), v, np.full(N, 1.0))
    prims = orc.primitives(cfg, m, P[:, 0], P[:, 1], P[:, 2], E, U, om)
    B6, E6, nc = orc.matrices(cfg, w["x"], w["y"], w["z"], w["L"], h, om)
    _, _, vsig = orc.gradients(cfg, w["x"], w["y"], w["z"], w["L"], h, om, prims, B6, nc)
    c = math.sqrt(cfg.gamma)
    inner = np.flatnonzero(np.all(np.abs(x) < 0.5 - h.max() - 1e-3, axis=1))
    assert inner.size > 50
    for i in inner[::7]:
        r = np.sqrt(np.sum((x - x[i]) ** 2, 1))
        rmax = r[(r < h[i]) & (np.arange(N) != i)].max()
        expect = 2 * c + max(k, 0.0) * rmax
        assert vsig[i] == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("frac,beta_min,beta_max,ncrit",
                         [(0.9, 1.0, 2.0, 100.0), (-0.8, 1.0, 2.0, 100.0), (0.7, 1.0, 1.0, 100.0),
                          (0.2, 1.0, 2.0, 100.0), (0.9, 0.3, 2.0, 0.5), (0.9, 0.8, 2.0, 0.5)])
def test_limiter_closed_form_on_a_spike(orc, frac, beta_min, beta_max, ncrit):
    """The conditioned Barth-Jespersen limiter (§2.3.6) in closed form: on a
    perfect lattice (N_cond = 1, so beta = max(beta_min, beta_max
    min(1, ncrit^2))) a linear pressure p = p0 + a x with a spike
    delta = frac M at one particle i (M = max_j a dx_j over i's neighbours).
    The neighbourhood is point-symmetric, so the gradient at i is a exactly
    (the spike cancels), the midpoint extrapolations reach +-M/2, and the
    neighbour extremes are +-M - delta:
    alpha = min(1, beta min((M - delta) / (M/2), (M + delta) / (M/2)))."""
    n = 12
    w = W.lattice_wave(n, jitter=0.0)
    cfg = orc.config(beta_min=beta_min, beta_max=beta_max, ncond_crit=ncrit)
    x = np.stack([w["x"], w["y"], w["z"]], 1)
    N = x.shape[0]
    i = int(np.argmin(np.sum((x - 0.5 + 0.5 / n) ** 2, 1)))   # a central particle
    a = 0.3
    h0, _, _, _ = orc.density(cfg, w["x"], w["y"], w["z"], w["L"], w["h"])[:4]
    d = x - x[i]
    r = np.sqrt(np.sum(d * d, 1))
    nb = (r < h0[i]) & (np.arange(N) != i)          # i's neighbours, by brute force
    M = a * d[nb, 0].max()
    assert M > 0 and np.isclose(d[nb, 0].min(), -d[nb, 0].max())
    p = 3.0 + a * (x[:, 0] - x[i, 0])
    p[i] += frac * M
    rho = np.full(N, 1.5)
    v = np.zeros((N, 3))
    h, om, m, P, E, U = _state_with_primitives(orc, cfg, w, rho, v, p)
    prims = orc.primitives(cfg, m, P[:, 0], P[:, 1], P[:, 2], E, U, om)
    B6, E6, nc = orc.matrices(cfg, w["x"], w["y"], w["z"], w["L"], h, om)
    assert nc[i] == pytest.approx(1.0, rel=1e-12)
    grad, alpha, vsig = orc.gradients(cfg, w["x"], w["y"], w["z"], w["L"], h, om, prims, B6, nc)
    assert np.abs(grad[i, 4] - np.array([a, 0.0, 0.0])).max() < 1e-10
    delta = frac * M
    beta = max(beta_min, beta_max * min(1.0, ncrit ** 2))
    expect = min(1.0, beta * min((M - delta) / (0.5 * M), (M + delta) / (0.5 * M)))
    assert alpha[i, 4] == pytest.approx(expect, rel=1e-9)
    assert np.all(alpha[i, :4] == 1.0)   # uniform density and velocity


# --------------------------------------------------------------------------
# Riemann solvers (§2.3.3): Toro's tables, jump conditions, invariants
# --------------------------------------------------------------------------
def _toro_rows():
    rows = []
    for line in open(os.path.join(GOLDEN, "toro_2009_table_4_2.txt")):
        if line.startswith("#") or not line.strip():
            continue
        a, b, c = line.split("|")
        rows.append((list(map(float, a.split())), list(map(float, b.split())), float(c)))
    return rows


def _star_densities(orc, d, g, ps, us):
    rl, ul, pl, rr, ur, pr = d
    out = []
    for eps in (-1e-9, 1e-9):
        V = us + eps
        out.append(orc.riemann_sample(rl, ul - V, pl, rr, ur - V, pr, g, ps, us - V)[0])
    return out


@pytest.mark.parametrize("row", range(5))
def test_exact_riemann_matches_toro_table(orc, row):
    d, star, tol = _toro_rows()[row]
    r = orc.riemann_star(*d, 1.4)
    assert r["vacuum"] == 0 and r["bisect"] == 0
    assert r["p"] == pytest.approx(star[0], rel=tol)
    assert r["u"] == pytest.approx(star[1], rel=tol, abs=1e-9)
    rl_s, rr_s = _star_densities(orc, d, 1.4, r["p"], r["u"])
    assert rl_s == pytest.approx(star[2], rel=tol)
    assert rr_s == pytest.approx(star[3], rel=tol)


@pytest.mark.parametrize("d", [(1.0, 0.0, 1.0, 0.125, 0.0, 0.1), (1.0, 0.3, 5.0, 0.2, -0.4, 0.1),
                               (0.5, -1.0, 0.1, 2.0, 1.0, 3.0), (1.0, 0.0, 1e-6, 1.0, 0.0, 1e4)])
@pytest.mark.parametrize("g", [1.4, 5.0 / 3.0])
def test_exact_riemann_jump_conditions(orc, d, g):
    """Shock side: Rankine-Hugoniot (mass, momentum, energy) with the shock
    speed from mass conservation.  Rarefaction side: isentrope and the
    Riemann invariant u +- 2c/(g-1)."""
    rl, ul, pl, rr, ur, pr = d
    r = orc.riemann_star(*d, g)
    ps, us = r["p"], r["u"]
    rls, rrs = _star_densities(orc, d, g, ps, us)
    for (rk, uk, pk, rs, sgn) in ((rl, ul, pl, rls, -1), (rr, ur, pr, rrs, 1)):
        if ps > pk:
            S = (rs * us - rk * uk) / (rs - rk)
            ek = pk / ((g - 1) * rk) + 0.5 * uk * uk
            es = ps / ((g - 1) * rs) + 0.5 * us * us
            mom_k = rk * uk * (uk - S) + pk
            mom_s = rs * us * (us - S) + ps
            assert mom_s == pytest.approx(mom_k, rel=1e-9, abs=1e-12 * max(pk, ps))
            en_k = rk * ek * (uk - S) + pk * uk
            en_s = rs * es * (us - S) + ps * us
            assert en_s == pytest.approx(en_k, rel=1e-8, abs=1e-10 * max(pk, ps) * (abs(us) + 1))
        else:
            assert ps / rs ** g == pytest.approx(pk / rk ** g, rel=1e-10)
            ck, cs = math.sqrt(g * pk / rk), math.sqrt(g * ps / rs)
            assert us - sgn * 2 * cs / (g - 1) == pytest.approx(uk - sgn * 2 * ck / (g - 1), rel=1e-10, abs=1e-10)


def test_exact_riemann_special_cases(orc):
    g = 5.0 / 3.0
    # pure contact: equal p and u, any density jump -> p* = p, u* = u
    r = orc.riemann_star(1.0, 0.3, 2.0, 0.1, 0.3, 2.0, g)
    assert r["p"] == pytest.approx(2.0, rel=1e-15) and r["u"] == pytest.approx(0.3, rel=1e-15)
    # mirror-symmetric data -> u* = 0
    r = orc.riemann_star(1.0, 0.7, 1.0, 1.0, -0.7, 1.0, g)
    assert abs(r["u"]) < 1e-15
    # Galilean shift of both velocities shifts u*, leaves p*
    a = orc.riemann_star(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, g)
    b = orc.riemann_star(1.0, 2.5, 1.0, 0.125, 2.5, 0.1, g)
    assert b["p"] == pytest.approx(a["p"], rel=1e-13) and b["u"] == pytest.approx(a["u"] + 2.5, rel=1e-13)
    # vacuum generation is flagged
    r = orc.riemann_star(1.0, -20.0, 0.1, 1.0, 20.0, 0.1, g)
    assert r["vacuum"] == 1
    # the root does not depend on the starting guess
    for p0 in (1e-8, 0.01, 0.5, 3.0, 100.0):
        c = orc.riemann_star(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, g, p0=p0)
        assert c["p"] == pytest.approx(a["p"], rel=1e-14)


_SAMPLE_CASES = [(1.0, 0.0, 1.0, 0.125, 0.0, 0.1),      # rarefaction | shock
                 (1.0, -2.0, 0.4, 1.0, 2.0, 0.4),      # two rarefactions
                 (1.0, 1.5, 1.0, 0.5, -1.0, 2.0),      # two shocks
                 (0.3, 0.2, 5.0, 1.0, 0.1, 0.2),       # strong left rarefaction
                 (1.0, 0.75, 1.0, 0.125, 0.0, 0.1)]    # sonic left rarefaction


@pytest.mark.parametrize("d", _SAMPLE_CASES)
@pytest.mark.parametrize("g", [1.4, 5.0 / 3.0])
def test_exact_riemann_sampling_is_mirror_symmetric(orc, d, g):
    """Euler's equations are invariant under x -> -x, u -> -u: the problem
    with its sides swapped and its velocities negated has the mirrored
    solution.  Sampled at x/t = 0 in frames moving with V across every wave
    (head, fan, tail, star regions, shocks), the mirrored problem's state is
    the original's with u negated, the side flag swapped, so the oracle's
    right-side branches agree with its left-side ones, which the star-state
    and jump-condition pins above fix."""
    rl, ul, pl, rr, ur, pr = d
    r = orc.riemann_star(*d, g)
    assert r["vacuum"] == 0
    ps, us = r["p"], r["u"]
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    lo, hi = min(ul - cl, us) - 1.0, max(ur + cr, us) + 1.0
    for V in np.linspace(lo, hi, 97) + 1e-7:
        a = orc.riemann_sample(rl, ul - V, pl, rr, ur - V, pr, g, ps, us - V)
        b = orc.riemann_sample(rr, -(ur - V), pr, rl, -(ul - V), pl, g, ps, -(us - V))
        assert b[0] == pytest.approx(a[0], rel=1e-13)
        assert b[1] == pytest.approx(-a[1], rel=1e-13, abs=1e-13)
        assert b[2] == pytest.approx(a[2], rel=1e-13)
        assert b[3] == -a[3]


@pytest.mark.parametrize("g", [1.4, 5.0 / 3.0])
def test_exact_riemann_fan_interior(orc, g):
    """Inside a rarefaction fan the state at x/t = 0 is the sonic point of
    the characteristic through the origin: u - c = 0 for a left fan (u + c
    = 0 for a right one), with the entropy p / rho^g and the Riemann
    invariant u + 2c/(g-1) (u - 2c/(g-1)) of the unperturbed side."""
    rl, ul, pl, rr, ur, pr = 1.0, -2.0, 0.4, 1.0, 2.0, 0.4   # two rarefactions
    r = orc.riemann_star(rl, ul, pl, rr, ur, pr, g)
    ps, us = r["p"], r["u"]
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
    csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
    for sgn, (head, tail), (rk, uk, pk, ck) in (
            (-1, (ul - cl, us - csl), (rl, ul, pl, cl)),
            (1, (us + csr, ur + cr), (rr, ur, pr, cr))):
        assert head < tail
        for f in (0.2, 0.5, 0.8):
            V = head + f * (tail - head)
            rho, u, p, side = orc.riemann_sample(rl, ul - V, pl, rr, ur - V, pr, g, ps, us - V)
            assert side == sgn
            c = math.sqrt(g * p / rho)
            assert u + sgn * c == pytest.approx(0.0, abs=1e-12)
            assert p / rho ** g == pytest.approx(pk / rk ** g, rel=1e-12)
            assert (u + V) - sgn * 2 * c / (g - 1) == pytest.approx(uk - sgn * 2 * ck / (g - 1),
                                                                     rel=1e-12, abs=1e-12)


def test_hllc_consistency(orc):
    g = 1.4
    n = np.array([0.6, 0.8, 0.0])
    w = np.array([0.8, -0.6, 0.5]) * 0.3
    # identical states: HLLC returns the physical flux
    rho, u, p = 1.3, 0.4, 2.0
    F, ps, ss = orc.hllc(rho, u, p, w, rho, u, p, w, n, g)
    E = p / (g - 1) + 0.5 * rho * (u * u + w @ w)
    assert F[0] == pytest.approx(rho * u, rel=1e-14)
    assert np.allclose(F[1:4], rho * u * (u * n + w) + p * n, rtol=1e-14)
    assert F[4] == pytest.approx(u * (E + p), rel=1e-14)
    # isolated contact is resolved exactly: S* = u, p* = p, upwind mass flux
    F, ps, ss = orc.hllc(1.0, 0.2, 1.0, w, 0.1, 0.2, 1.0, -w, n, g)
    assert ss == pytest.approx(0.2, rel=1e-14) and ps == pytest.approx(1.0, rel=1e-14)
    assert F[0] == pytest.approx(1.0 * 0.2, rel=1e-14)


def _phys_flux(rho, u, p, w, n, g):
    E = p / (g - 1) + 0.5 * rho * (u * u + w @ w)
    return np.concatenate([[rho * u], rho * u * (u * n + w) + p * n, [u * (E + p)]])


def test_hllc_upwinds_supersonic_flow_and_is_mirror_symmetric(orc):
    """Toro (2009) ch. 10, the solver §2.3.3 allows besides the exact one:
    when every wave moves right (left) the flux at x/t = 0 is the left
    (right) state's physical flux; and the problem mirrored through the
    face (sides swapped, normal velocities negated) has the mirrored flux:
    mass, energy and tangential momentum flux negated, the normal momentum
    flux, p* unchanged, S* negated."""
    g = 1.4
    n = np.array([0.6, 0.8, 0.0])
    wl, wr = np.array([0.8, -0.6, 0.5]) * 0.3, np.array([-0.4, 0.3, 0.2]) * 0.2
    rl, pl, rr, pr = 1.0, 1.0, 0.6, 0.7
    for ul, ur, side in ((5.0, 6.0, -1), (-6.0, -5.5, 1)):
        F, ps, ss = orc.hllc(rl, ul, pl, wl, rr, ur, pr, wr, n, g)
        ref = _phys_flux(rl, ul, pl, wl, n, g) if side < 0 else _phys_flux(rr, ur, pr, wr, n, g)
        assert np.allclose(F, ref, rtol=1e-13, atol=1e-13)
    for (ul, ur) in ((0.3, -0.2), (-0.5, 1.1), (2.0, 1.0), (0.0, 0.0)):
        F, ps, ss = orc.hllc(rl, ul, pl, wl, rr, ur, pr, wr, n, g)
        G, ps2, ss2 = orc.hllc(rr, -ur, pr, wr, rl, -ul, pl, wl, n, g)
        assert ps2 == pytest.approx(ps, rel=1e-13) and ss2 == pytest.approx(-ss, rel=1e-13, abs=1e-14)
        scale = np.abs(F).max()
        assert abs(G[0] + F[0]) < 1e-13 * scale and abs(G[4] + F[4]) < 1e-13 * scale
        Fm, Gm = F[1:4], G[1:4]
        assert abs(Gm @ n - Fm @ n) < 1e-13 * scale
        assert np.abs((Gm - (Gm @ n) * n) + (Fm - (Fm @ n) * n)).max() < 1e-13 * scale


def test_pair_limiter_bounds(orc):
    rng = np.random.default_rng(3)
    for _ in range(2000):
        a, b = rng.uniform(-2, 2, 2)
        e = rng.uniform(-4, 4)
        out = orc.pair_limit(e, a, b)
        d = abs(a - b)
        lo, hi = min(a, b), max(a, b)
        # never beyond the neighbour bracket widened by psi1 d
        assert lo - 0.5 * d - 1e-15 <= out <= hi + 0.5 * d + 1e-15
        # never past the mean by more than psi2 d towards the far side
        if a < b:
            assert out <= 0.5 * (a + b) + 0.25 * d + 1e-15
        elif a > b:
            assert out >= 0.5 * (a + b) - 0.25 * d - 1e-15
        # values inside [own, mean] are untouched
        if min(a, 0.5 * (a + b)) <= e <= max(a, 0.5 * (a + b)):
            assert out == e
    # the ends of the allowed range are reached: an extrapolation far past the
    # neighbour stops at mean + psi2 d (mean - psi2 d), one far behind the own
    # value at own - psi1 d (own + psi1 d); in between the result does not
    # decrease with the extrapolation
    for _ in range(500):
        a, b = rng.uniform(-2, 2, 2)
        d = abs(a - b)
        if d < 1e-6:
            continue
        s = 1.0 if a < b else -1.0
        mean = 0.5 * (a + b)
        assert orc.pair_limit(b + s * 10 * d, a, b) == pytest.approx(mean + s * 0.25 * d, rel=1e-14, abs=1e-14)
        assert orc.pair_limit(a - s * 10 * d, a, b) == pytest.approx(a - s * 0.5 * d, rel=1e-14, abs=1e-14)
        es = np.sort(rng.uniform(-4, 4, 64))
        outs = np.array([orc.pair_limit(e, a, b) for e in es])
        assert np.all(np.diff(outs) >= -1e-15)
    # positive quantities stay positive
    assert orc.pair_limit(-1.0, 0.1, 5.0, positive=True) > 0.0
    for _ in range(500):
        a, b = rng.uniform(1e-3, 2, 2)
        assert orc.pair_limit(rng.uniform(-4, 4), a, b, positive=True) > 0.0


# --------------------------------------------------------------------------
# full step: conservation (Eq. 15), MFM masses, Galilean invariance, mirror
# --------------------------------------------------------------------------
def _moving(w, seed=5, amp=0.3):
    rng = np.random.default_rng(seed)
    n = w["x"].size
    v = rng.normal(0, amp, (n, 3))
    w = dict(w)
    w["px"], w["py"], w["pz"] = w["m"] * v[:, 0], w["m"] * v[:, 1], w["m"] * v[:, 2]
    w["E"] = w["U"] + 0.5 * w["m"] * np.sum(v * v, 1)
    return w


def _cons_drift(orc, cfg, w, dt):
    s, out, info = orc.step(cfg, w, dt)
    assert info["status"] == 0
    v = np.stack([w["px"], w["py"], w["pz"]], 1) / w["m"][:, None]
    cs = np.sqrt(cfg.gamma * (cfg.gamma - 1) * w["U"] / w["m"])
    res = {}
    res["M"] = abs(math.fsum(s["m"]) - math.fsum(w["m"])) / math.fsum(np.abs(w["m"]))
    res["E"] = abs(math.fsum(s["E"]) - math.fsum(w["E"])) / math.fsum(np.abs(w["E"]))
    pscale = math.fsum(w["m"] * (np.linalg.norm(v, axis=1) + cs))
    for k in ("px", "py", "pz"):
        res[k] = abs(math.fsum(s[k]) - math.fsum(w[k])) / pscale
    return s, out, info, res


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
@pytest.mark.parametrize("riemann", ["exact", "hllc"])
def test_step_conserves_mass_momentum_energy(orc, scheme, riemann):
    w = _moving(W.lattice_wave(10, jitter=0.05))
    cfg = orc.config(scheme=scheme, riemann=riemann)
    s, out, info, res = _cons_drift(orc, cfg, w, dt=-1.0)
    assert info["dt"] > 0 and info["flux"]["pairs"] > 0
    for k, v in res.items():
        assert v < 1e-13, (k, v)
    if scheme == "mfm":
        assert np.array_equal(s["m"], w["m"])   # zero mass flux, bitwise
        assert np.all(out["dQ"][:, 0] == 0.0)
    # the flux really moved something
    assert np.abs(out["dQ"][:, 1:5]).max() > 0


def test_step_sod_conserves(orc):
    w = W.sod(8)
    cfg = orc.config()
    s, out, info, res = _cons_drift(orc, cfg, w, dt=-1.0)
    for k, v in res.items():
        assert v < 1e-13, (k, v)


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
def test_flux_galilean_invariance(orc, scheme):
    """Boosting every velocity by V leaves dm unchanged and transforms
    dP -> dP + dm V, dE -> dE + dP.V + dm V^2/2 (the boost/de-boost of §2.3.3)."""
    w = _moving(W.lattice_wave(8, jitter=0.05), amp=0.2)
    V = np.array([0.7, -0.4, 0.25])
    wb = dict(w)
    wb["px"], wb["py"], wb["pz"] = w["px"] + w["m"] * V[0], w["py"] + w["m"] * V[1], w["pz"] + w["m"] * V[2]
    wb["E"] = w["E"] + (w["px"] * V[0] + w["py"] * V[1] + w["pz"] * V[2]) + 0.5 * w["m"] * (V @ V)
    cfg = orc.config(scheme=scheme, alpha1=0.0)
    dt = 2e-3
    _, o1, _ = orc.step(cfg, w, dt)
    _, o2, _ = orc.step(cfg, wb, dt)
    d1, d2 = o1["dQ"], o2["dQ"]
    scale = np.abs(d1).max(0) + 1e-300
    assert np.allclose(d2[:, 0], d1[:, 0], atol=1e-11 * scale[0] + 1e-300)
    dP = d1[:, 1:4] + d1[:, :1] * V
    assert np.abs(d2[:, 1:4] - dP).max() < 1e-10 * scale[1:4].max()
    dE = d1[:, 4] + d1[:, 1:4] @ V + 0.5 * d1[:, 0] * (V @ V)
    assert np.abs(d2[:, 4] - dE).max() < 1e-10 * scale[4]
    # the internal-energy change (Eq. 24) is frame independent
    assert np.abs(d2[:, 5] - d1[:, 5]).max() < 1e-10 * scale[5]


def test_flux_mirror_symmetry(orc):
    """Reflecting x -> L - x and v_x -> -v_x mirrors the update."""
    w = _moving(W.lattice_wave(8, jitter=0.05), amp=0.2)
    wm = dict(w)
    xm = 1.0 - w["x"]
    xm[xm >= 1.0] -= 1.0
    wm["x"] = xm
    wm["px"] = -w["px"]
    cfg = orc.config()
    dt = 2e-3
    _, o1, _ = orc.step(cfg, w, dt)
    _, o2, _ = orc.step(cfg, wm, dt)
    sgn = np.array([1, -1, 1, 1, 1, 1])
    scale = np.abs(o1["dQ"]).max(0)
    assert np.all(np.abs(o2["dQ"] - o1["dQ"] * sgn) <= 1e-10 * scale + 1e-300)


def test_uniform_state_is_stationary(orc):
    # perfect lattice, uniform rho, p, v: every particle is in equilibrium;
    # sum_j A_ij = 0 by symmetry, so the update vanishes to round-off
    w = W.lattice_wave(8, jitter=0.0)
    w = dict(w)
    w["m"] = np.full(w["x"].size, 1.0 / 512)
    w["U"] = w["m"] * 1.0 / (w["gamma"] - 1)
    w["E"] = w["U"].copy()
    cfg = orc.config()
    s, out, info = orc.step(cfg, w, 1e-3)
    assert np.abs(out["dQ"][:, 1:5]).max() < 1e-15 * 1e-3 * 10


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
def test_uniform_flow_is_carried_unchanged(orc, scheme):
    """A uniform state moving with v0 (Galilean invariance of §2.3.4's
    update): nothing is exchanged, every particle drifts by v0 dt (modulo
    the periodic box) and keeps its mass, momentum and energy."""
    w = dict(W.lattice_wave(8, jitter=0.0))
    N = w["x"].size
    v0 = np.array([0.7, -0.4, 0.25])
    w["m"] = np.full(N, 1.0 / N)
    w["px"], w["py"], w["pz"] = (w["m"] * v0[a] for a in range(3))
    w["U"] = w["m"] * 1.0 / (w["gamma"] - 1)
    w["E"] = w["U"] + 0.5 * w["m"] * (v0 @ v0)
    cfg = orc.config(scheme=scheme)
    dt = 1e-3
    s, out, info = orc.step(cfg, w, dt)
    assert np.abs(out["dQ"][:, :5]).max() < 1e-15
    for a, k in enumerate("xyz"):
        moved = (w[k] + v0[a] * dt) % 1.0
        dx = (s[k] - moved + 0.5) % 1.0 - 0.5
        assert np.abs(dx).max() < 1e-15
    for k in ("m", "px", "py", "pz", "E"):
        assert np.allclose(s[k], w[k], rtol=1e-13, atol=0.0)


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
def test_sod_tube_follows_exact_solution(orc, scheme):
    """Multi-step 3D Sod tube (§3.1.2 setup family; gamma = 5/3, rho_R = 1/8):
    the density near the x = 2 interface approaches the exact Riemann
    solution (pinned above by Toro's tables) far better than the frozen
    initial state does."""
    g = 5.0 / 3.0
    s = W.sod(16)
    cfg = orc.config(scheme=scheme)
    t = 0.0
    while t < 0.4:
        s, out, info = orc.step(cfg, s, -1.0)
        assert info["status"] == 0
        t += info["dt"]
    r = orc.riemann_star(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, g)
    x = s["x"]
    sel = (x > 1.3) & (x < 3.0)

    def exact(xx):
        out = []
        for xi in xx:
            c = (xi - 2.0) / t
            rr, uu, pp, _ = orc.riemann_sample(1.0, -c, 1.0, 0.125, -c, 0.1, g, r["p"], r["u"] - c)
            out.append((rr, uu + c, pp))
        return np.array(out)

    ex = exact(x[sel])
    prims = orc.primitives(cfg, s["m"], s["px"], s["py"], s["pz"], s["E"], s["U"], s["omega"])
    rho, vx, p = prims[0][sel], prims[1][sel], prims[4][sel]
    frozen = np.stack([np.where(x[sel] < 2.0, 1.0, 0.125), np.zeros(sel.sum()),
                       np.where(x[sel] < 2.0, 1.0, 0.1)], 1)
    for k, f in enumerate((rho, vx, p)):
        l1 = np.mean(np.abs(f - ex[:, k]))
        l1_frozen = np.mean(np.abs(frozen[:, k] - ex[:, k]))
        assert l1 < (0.6, 0.3, 0.5)[k] * l1_frozen, (k, l1, l1_frozen)
        # and in absolute terms at this resolution (n = 16: 16 particles per unit
        # length on the dense side; measured MFV 0.094 / 0.075 / 0.096, MFM 0.099 /
        # 0.078 / 0.099 for rho / v / p over 1.3 < x < 3 at t = 0.4)
        assert l1 < (0.11, 0.09, 0.11)[k], (k, l1)
    # transverse motion stays negligible (§3.1.2)
    assert np.abs(prims[2][sel]).max() < 1e-2 and np.abs(prims[3][sel]).max() < 1e-2


# --------------------------------------------------------------------------
# half-step predictor (§2.3.4, Eq. 16: face states advanced by dt/2)
# --------------------------------------------------------------------------
def _lattice_faces(orc, cfg, w, rho, v, p, dt):
    """Face states (rho, u, p on both sides, normal velocities in the frame
    of the pair's mean velocity) of every flux pair, from the oracle's full
    pipeline: density, E and B, limited gradients, face reconstruction."""
    h, om, m, P, E, U = _state_with_primitives(orc, cfg, w, rho, v, p)
    prims = orc.primitives(cfg, m, P[:, 0], P[:, 1], P[:, 2], E, U, om)
    B6, E6, nc = orc.matrices(cfg, w["x"], w["y"], w["z"], w["L"], h, om)
    grad, alpha, _ = orc.gradients(cfg, w["x"], w["y"], w["z"], w["L"], h, om, prims, B6, nc)
    pairs = orc.flux_pairs(w["x"], w["y"], w["z"], w["L"], h)
    _, _, faces = orc.fluxes(cfg, w["x"], w["y"], w["z"], w["L"], h, om, B6, prims, grad,
                             alpha, dt, pairs=pairs, want_faces=True)
    return h, alpha, pairs, faces


def test_predictor_accelerates_by_the_pressure_gradient(orc):
    """Perfect lattice at rest, linear density and pressure fields: Euler's
    momentum equation gives each side's velocity after half a step as
    -dt/2 grad p / rho (the particle's own rho).  The face moves with the
    mean of the two half-step velocities, so in its frame the normal
    velocities are equal and opposite, u_L - u_R = -dt/2 (grad p . n)
    (1/rho_i - 1/rho_j); with div v = 0 density and pressure only take
    their midpoint values.  On a cubic lattice B is isotropic, so the face
    normal is the separation's direction."""
    n = 12
    w = W.lattice_wave(n, jitter=0.0)
    cfg = orc.config()
    x = np.stack([w["x"], w["y"], w["z"]], 1) - 0.5
    g_p = np.array([0.3, -0.2, 0.15])
    g_rho = np.array([0.4, 0.1, -0.3])
    rho, p = 2.5 + x @ g_rho, 3.0 + x @ g_p
    dt = 0.01
    h, alpha, pairs, F = _lattice_faces(orc, cfg, w, rho, np.zeros_like(x), p, dt)
    inner = np.all(np.abs(x) < 0.5 - h.max() - 1e-3, axis=1)   # away from the periodic seam
    assert np.all(alpha[inner] == 1.0)
    sel = inner[pairs[:, 0]] & inner[pairs[:, 1]]
    assert sel.sum() > 1000
    i, j = pairs[sel, 0], pairs[sel, 1]
    F = F[sel]
    d = x[j] - x[i]
    nh = d / np.linalg.norm(d, axis=1)[:, None]
    xm = x[i] + 0.5 * d
    scale = 0.5 * dt * np.linalg.norm(g_p) / rho.min()
    rel = -0.5 * dt * (nh @ g_p) * (1.0 / rho[i] - 1.0 / rho[j])
    assert np.abs(rel).max() > 1e-3 * scale
    assert np.abs((F[:, 1] - F[:, 4]) - rel).max() < 1e-12 * scale
    assert np.abs(F[:, 1] + F[:, 4]).max() < 1e-12 * scale
    for k in (0, 3):
        assert np.abs(F[:, k] - (2.5 + xm @ g_rho)).max() < 1e-13 * 2.5
    for k in (2, 5):
        assert np.abs(F[:, k] - (3.0 + xm @ g_p)).max() < 1e-13 * 3.0


def test_predictor_compresses_with_the_velocity_divergence(orc):
    """Uniform density and pressure, linear velocity v = K x: continuity and
    the adiabatic pressure equation give the face states after half a step
    as rho (1 - dt/2 tr K) and p (1 - dt/2 gamma tr K) on both sides, and
    the extrapolated velocities equal the pair's mean velocity at the
    midpoint (zero normal velocity in its frame)."""
    n = 12
    w = W.lattice_wave(n, jitter=0.0)
    cfg = orc.config()
    x = np.stack([w["x"], w["y"], w["z"]], 1) - 0.5
    K = np.array([[0.3, 0.1, -0.05], [0.02, -0.1, 0.04], [0.0, 0.07, 0.2]])
    v = x @ K.T
    N = x.shape[0]
    dt = 0.01
    h, alpha, pairs, F = _lattice_faces(orc, cfg, w, np.full(N, 2.5), v, np.full(N, 3.0), dt)
    inner = np.all(np.abs(x) < 0.5 - h.max() - 1e-3, axis=1)
    sel = inner[pairs[:, 0]] & inner[pairs[:, 1]]
    assert sel.sum() > 1000
    F = F[sel]
    tr = np.trace(K)
    for k in (0, 3):
        assert np.abs(F[:, k] - 2.5 * (1.0 - 0.5 * dt * tr)).max() < 1e-13 * 2.5
    for k in (2, 5):
        assert np.abs(F[:, k] - 3.0 * (1.0 - 0.5 * dt * cfg.gamma * tr)).max() < 1e-13 * 3.0
    vscale = np.abs(v).max()
    assert np.abs(F[:, 1]).max() < 1e-13 * vscale and np.abs(F[:, 4]).max() < 1e-13 * vscale


def test_rung_predictor_advances_each_side_over_its_own_time(orc):
    """Individual timesteps (§2.3.4): a face exchanges over dt_ij =
    min(dt_i, dt_j) and each side is predicted from the state its particle
    last took, over the time since then plus dt_ij / 2.  With uniform density
    and pressure and a linear velocity v = K x, Euler's equations give each
    side's state after a time t as rho (1 - t tr K) and p (1 - t gamma tr K)
    (first order, as the predictor), whatever the other side's time."""
    n = 12
    w = W.lattice_wave(n, jitter=0.0)
    cfg = orc.config()
    x = np.stack([w["x"], w["y"], w["z"]], 1) - 0.5
    K = np.array([[0.3, 0.1, -0.05], [0.02, -0.1, 0.04], [0.0, 0.07, 0.2]])
    v = x @ K.T
    N = x.shape[0]
    h, om, m, P, E, U = _state_with_primitives(orc, cfg, w, np.full(N, 2.5), v, np.full(N, 3.0))
    prims = orc.primitives(cfg, m, P[:, 0], P[:, 1], P[:, 2], E, U, om)
    B6, E6, nc = orc.matrices(cfg, w["x"], w["y"], w["z"], w["L"], h, om)
    grad, alpha, _ = orc.gradients(cfg, w["x"], w["y"], w["z"], w["L"], h, om, prims, B6, nc)
    pairs = orc.flux_pairs(w["x"], w["y"], w["z"], w["L"], h)
    rng = np.random.default_rng(11)
    dt0 = 0.02
    dtp = dt0 * 2.0 ** -rng.integers(0, 3, N)          # rungs 0, 1, 2
    toff = dtp * rng.integers(0, 4, N) / 4.0           # time since the state was taken
    _, st, F = orc.fluxes_rung(cfg, w["x"], w["y"], w["z"], w["L"], h, om, B6, prims, grad,
                               alpha, dtp, toff, pairs)
    inner = np.all(np.abs(x) < 0.5 - h.max() - 1e-3, axis=1)
    sel = inner[pairs[:, 0]] & inner[pairs[:, 1]]
    assert sel.sum() > 1000
    i, j = pairs[sel, 0], pairs[sel, 1]
    F = F[sel]
    dtij = np.minimum(dtp[i], dtp[j])
    tl, tr = toff[i] + 0.5 * dtij, toff[j] + 0.5 * dtij
    assert np.unique(np.round(tl / dt0, 6)).size >= 4   # several distinct side times
    trK = np.trace(K)
    assert np.abs(F[:, 0] - 2.5 * (1.0 - tl * trK)).max() < 1e-13 * 2.5
    assert np.abs(F[:, 3] - 2.5 * (1.0 - tr * trK)).max() < 1e-13 * 2.5
    assert np.abs(F[:, 2] - 3.0 * (1.0 - tl * cfg.gamma * trK)).max() < 1e-13 * 3.0
    assert np.abs(F[:, 5] - 3.0 * (1.0 - tr * cfg.gamma * trK)).max() < 1e-13 * 3.0


# --------------------------------------------------------------------------
# Sedov-Taylor blast (§3.1): shock radius of the self-similar solution
# --------------------------------------------------------------------------
def test_sedov_similarity_constant():
    """The similarity integration (tests/sedov_similarity.py) reproduces the
    textbook shock constants of the 3D blast, xi0 = 1.1517 at gamma = 5/3
    and 1.0328 at gamma = 1.4, independently of its grid."""
    import sedov_similarity as S
    assert S.xi0(5.0 / 3.0) == pytest.approx(1.1517, abs=2e-4)
    assert S.xi0(1.4) == pytest.approx(1.0328, abs=2e-4)
    assert abs(S.xi0(5.0 / 3.0, n=4000) - S.xi0(5.0 / 3.0)) < 2e-5
    # the profile starts from the strong-shock jump: rho = (g+1)/(g-1) rho1
    pr = S.profile(5.0 / 3.0, n=2000)
    assert pr[0, 1] == 4.0 and np.all(np.diff(pr[:, 1]) < 0)


def _sedov_run(orc, n, t_end):
    w = W.sedov(n)
    cfg = orc.config(gamma=w["gamma"])
    s, t = dict(w), 0.0
    while t < t_end:
        s, _, info = orc.step(cfg, s, -1.0)
        assert info["status"] == 0
        t += info["dt"]
    return w, s, t


def test_oracle_sedov_blast_follows_similarity_solution(orc):
    """Sedov blast (the config-3 generator: energy 1 on the central 32
    particles of a unit lattice, rho = 1) run by the oracle to t ~ 0.018:
    the density-weighted radius of the shell (particles denser than halfway
    between the ambient and the peak density) lies within 4 % of
    R = xi0 (E t^2 / rho)^(1/5); total energy is conserved to 1e-13 (the
    paper reports machine precision); the peak density rises with
    resolution and stays below the strong-shock limit 4."""
    import sedov_similarity as S
    peaks = []
    for n in (24, 32):
        w, s, t = _sedov_run(orc, n, 0.0184)
        R = S.shock_radius(1.0, t)
        r = np.sqrt((s["x"] - 0.5) ** 2 + (s["y"] - 0.5) ** 2 + (s["z"] - 0.5) ** 2)
        rho = s["m"] / s["omega"]
        shell = rho > 0.5 * (1.0 + rho.max())
        r_shell = np.average(r[shell], weights=rho[shell])
        assert abs(r_shell / R - 1.0) < 0.04, (n, r_shell, R)
        e0, e1 = math.fsum(w["E"]), math.fsum(s["E"])
        assert abs(e1 - e0) < 1e-13 * e0
        assert abs(math.fsum(s["m"]) - math.fsum(w["m"])) < 1e-13 * math.fsum(w["m"])
        for k in ("px", "py", "pz"):
            assert abs(math.fsum(s[k])) < 1e-13 * math.fsum(np.abs(s[k]))
        peaks.append(rho.max())
    assert 1.5 < peaks[0] < peaks[1] < 4.0, peaks


# --------------------------------------------------------------------------
# sound wave (§3.1): second-order convergence of the linear solution
# --------------------------------------------------------------------------
def _soundwave(n, A, gamma=1.4, planes=8, n_ngb=32.0):
    """One wavelength along x of a unit box, `planes` lattice planes across;
    rho = 1 + A cos(2 pi x), p = 1 + gamma A cos(2 pi x), v_x = A c_s cos(2 pi x)
    (through the masses and energies of a uniform lattice)."""
    a = 1.0 / n
    i, j, k = np.meshgrid(np.arange(n), np.arange(planes), np.arange(planes), indexing="ij")
    x, y, z = (i.ravel() + 0.5) * a, (j.ravel() + 0.5) * a, (k.ravel() + 0.5) * a
    cs = math.sqrt(gamma)
    ph = np.cos(2.0 * math.pi * x)
    rho, p, vx = 1.0 + A * ph, 1.0 + gamma * A * ph, A * cs * ph
    m = rho * a ** 3
    U = p * a ** 3 / (gamma - 1.0)
    h = np.full(x.size, (3.0 * n_ngb / (4.0 * math.pi)) ** (1.0 / 3.0) * a)
    return dict(x=x, y=y, z=z, m=m, px=m * vx, py=0.0 * x, pz=0.0 * x, E=U + 0.5 * m * vx * vx,
                U=U, h=h, L=np.array([1.0, planes * a, planes * a]), gamma=gamma), cs


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
def test_oracle_soundwave_converges_at_second_order(orc, scheme):
    """The paper's sound-wave test (§3.1: gamma = 1.4, c_s = sqrt(gamma),
    N_NGB = 32, cubic spline, limiter off) run by the oracle for one
    crossing time at N = 16, 32, 64 particles per wavelength: the L1 error of
    the density against the linear solution falls at second order (the paper
    finds both schemes second order).  The amplitude is 1e-5, not the
    paper's 1e-3: at 1e-3 the wave's own nonlinear steepening over one
    crossing (an O(A^2) departure from the linear solution) is reached by
    N = 64, which the paper notes as the floor of the L1 norm.  Transverse
    velocities stay at rounding level."""
    A, gamma = 1e-5, 1.4
    l1 = {}
    for n in (16, 32, 64):
        w, cs = _soundwave(n, A, gamma)
        cfg = orc.config(gamma=gamma, kernel="cubic", scheme=scheme, limiter=False, c_cfl=0.1)
        t_end = 1.0 / cs
        s, t, dt_next = w, 0.0, None
        while t < t_end * (1.0 - 1e-12):
            dt = -1.0 if dt_next is None or t + dt_next < t_end else t_end - t
            s, _, info = orc.step(cfg, s, dt)
            assert info["status"] == 0
            t += info["dt"]
            dt_next = info["dt_next"]
        _, om, _, _ = orc.density(cfg, s["x"], s["y"], s["z"], s["L"], s["h"])
        rho = s["m"] / om
        # the kernel estimate of a lattice's density is uniformly biased by a
        # few per cent: the perturbation is measured against its mean
        delta = rho / rho.mean() - 1.0
        exact = A * np.cos(2.0 * math.pi * s["x"] - 2.0 * math.pi * cs * t)
        l1[n] = float(np.mean(np.abs(delta - exact)))
        vt = np.sqrt(np.mean((s["py"] / s["m"]) ** 2 + (s["pz"] / s["m"]) ** 2))
        assert vt < 1e-12, (n, vt)
    assert math.log2(l1[16] / l1[32]) > 1.7, l1
    assert math.log2(l1[32] / l1[64]) > 1.9, l1
    assert l1[64] < 1e-2 * A, l1


# --------------------------------------------------------------------------
# external acceleration (§2.3.8) integrated by the rule of §2.3.4
# --------------------------------------------------------------------------
def _uniform_moving(v0, n=8):
    w = dict(W.lattice_wave(n, jitter=0.0))
    m = np.full(w["x"].size, 1.0 / n ** 3)
    w["m"] = m
    w["px"], w["py"], w["pz"] = m * v0[0], m * v0[1], m * v0[2]
    w["U"] = m * 1.0 / (w["gamma"] - 1)
    w["E"] = w["U"] + 0.5 * m * float(np.dot(v0, v0))
    return w


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
def test_gravity_on_a_uniform_state_closed_form(orc, scheme):
    """A uniform lattice moving with v0 in a uniform acceleration a: the
    fluxes vanish (Galilean-invariant uniform state), so the step is the
    source rule alone: P += m a dt, E += dt P.a (the trapezoid between the
    start state and the flux-updated state, which equals the start state
    here), U unchanged, x += dt v0 + a dt^2 / 2 (the mean of the old and new
    velocity), masses unchanged."""
    v0 = np.array([0.3, -0.2, 0.1])
    a = np.array([0.5, 1.5, -2.0])
    w = _uniform_moving(v0)
    n = w["x"].size
    dt = 1e-3
    cfg = orc.config(scheme=scheme)
    s, out, info = orc.step(cfg, w, dt, acc=np.tile(a, (n, 1)))
    assert info["status"] == 0
    m = w["m"]
    assert np.array_equal(s["m"], m)
    for q, k in enumerate(("px", "py", "pz")):
        want = w[k] + m * a[q] * dt
        assert np.allclose(s[k], want, rtol=1e-13, atol=1e-16 * np.abs(want).max()), k
    dE = dt * m * float(np.dot(v0, a))
    assert np.allclose(s["E"] - w["E"], dE, rtol=1e-9, atol=1e-18)
    assert np.allclose(s["U"], w["U"], rtol=1e-13)
    for q, k in enumerate(("x", "y", "z")):
        d = s[k] - w[k] - (dt * v0[q] + 0.5 * a[q] * dt * dt)
        d -= np.round(d)          # unit periodic box
        assert np.abs(d).max() < 1e-14, k


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
def test_gravity_momentum_and_exchange_term(orc, scheme):
    """A pressure bump in the middle of a tube at rest (uniform state at the
    periodic seam, so no face across it carries mass): the flux conserves
    momentum, so the total momentum changes by exactly sum_i dt/2 (m^n + m^{n+1})
    a_i for any field a_i; the exchange sums sum_j dm_ij r_ij over all
    particles equal twice the change of sum_k m_k x_k that the mass exchange
    alone makes (each face moves c_m from x_i to x_j), and vanish for MFM."""
    rng = np.random.default_rng(7)
    w = _uniform_moving(np.zeros(3), n=12)
    x = w["x"]
    bump = np.exp(-((x - 0.5) / 0.08) ** 2)     # 1e-17 at the seam
    w["U"] = w["m"] * (1.0 + 2.0 * bump) / (w["gamma"] - 1)
    w["E"] = w["U"].copy()
    n = x.size
    acc = rng.normal(0.0, 0.5, (n, 3))
    cfg = orc.config(scheme=scheme)
    s, out, info = orc.step(cfg, w, 1e-3, acc=acc)
    assert info["status"] == 0
    dt = info["dt"]
    w_ = 0.5 * dt * (w["m"] + s["m"])
    for q, k in enumerate(("px", "py", "pz")):
        want = math.fsum(w_ * acc[:, q])
        got = math.fsum(s[k]) - math.fsum(w[k])
        assert abs(got - want) < 1e-12 * math.fsum(np.abs(w_ * acc[:, q])), k
    # exchange sums from the oracle's flux routine on the same start state
    co = cfg
    h, om, _, _ = orc.density(co, w["x"], w["y"], w["z"], w["L"], w["h"])
    prims = orc.primitives(co, w["m"], w["px"], w["py"], w["pz"], w["E"], w["U"], om)
    B6, _, nc = orc.matrices(co, w["x"], w["y"], w["z"], w["L"], h, om)
    grad, alpha, _ = orc.gradients(co, w["x"], w["y"], w["z"], w["L"], h, om, prims, B6, nc)
    dQ, _, _, dM = orc.fluxes(co, w["x"], w["y"], w["z"], w["L"], h, om, B6, prims, grad,
                              alpha, dt, want_dM=True)
    if scheme == "mfm":
        assert np.all(dM == 0.0)
        return
    moved = np.array([math.fsum(dQ[:, 0] * c) for c in (w["x"], w["y"], w["z"])])
    total = np.array([math.fsum(dM[:, q]) for q in range(3)])
    assert np.abs(moved[0]) > 0
    assert np.allclose(total, 2.0 * moved, rtol=1e-9, atol=1e-12 * np.abs(dQ[:, 0]).sum())


# --------------------------------------------------------------------------
# entropy switch (§2.3.7)
# --------------------------------------------------------------------------
def test_entropy_switch_regimes(orc):
    """The three pressure routes: total energy when U > alpha1 (E_grav +
    E_kin); else the entropic function (p = A rho^gamma) when U < alpha2
    (E_kin^max + U) or U < alpha3 E_grav; else the internal energy."""
    g = 5.0 / 3.0
    m = np.ones(6)
    om = np.full(6, 0.5)                     # rho = 2
    v = np.array([0.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    px, py, pz = m * v, np.zeros(6), np.zeros(6)
    U = np.array([1.0, 1e-6, 5e-3, 1e-6, 5e-3, 5e-3])
    E = U + 0.5 * m * v * v
    ekmax = np.array([0.0, 1.0, 1.0, 1.0, 1e-3, 1e-3])
    A = np.array([0.3, 0.3, 0.3, -1.0, 0.3, 0.3])
    h = np.ones(6)
    acc = np.zeros((6, 3))
    acc[5, 2] = 10.0                          # E_grav = 10 > U / alpha3 = 5
    cfg = orc.config(gamma=g, entropy=True)
    rho, _, _, _, p, src = orc.primitives(cfg, m, px, py, pz, E, U, om, h=h, acc=acc, A=A,
                                          ekmax=ekmax, want_src=True)
    # 0: hot; 1: cold, large relative motion; 2: cold, relative motion small
    # vs U / alpha2; 3: entropy route but A unset; 4: U > alpha2 (ekmax + U);
    # 5: E_grav large: the first test fails (U < alpha1 (E_grav + E_kin)),
    # the entropy route through U < alpha3 E_grav
    assert list(src) == [0, 1, 2, 2, 2, 1]
    assert p[0] == pytest.approx((E[0] - 0.0) * (g - 1) / 0.5, rel=1e-15)
    assert p[1] == pytest.approx(0.3 * 2.0 ** g, rel=1e-15)
    assert p[2] == pytest.approx(5e-3 * (g - 1) / 0.5, rel=1e-15)
    assert p[5] == pytest.approx(0.3 * 2.0 ** g, rel=1e-15)
    # switched off: never the entropy route
    cfg0 = orc.config(gamma=g, entropy=False)
    *_, src0 = orc.primitives(cfg0, m, px, py, pz, E, U, om, h=h, acc=acc, A=A, ekmax=ekmax,
                              want_src=True)
    assert 1 not in list(src0)


def test_ekin_max_brute_force(orc):
    rng = np.random.default_rng(4)
    n = 300
    x, y, z = rng.random(n), rng.random(n), rng.random(n)
    L = np.array([1.0, 1.0, 1.0])
    h = rng.uniform(0.1, 0.2, n)
    m = rng.uniform(0.5, 1.5, n)
    vel = rng.normal(0, 1, (n, 3))
    got = orc.ekin_max(x, y, z, L, h, m, m * vel[:, 0], m * vel[:, 1], m * vel[:, 2])
    for i in range(0, n, 7):
        d = np.stack([x - x[i], y - y[i], z - z[i]], 1)
        d -= np.round(d)
        r2 = (d[:, 0] ** 2 + d[:, 1] ** 2) + d[:, 2] ** 2
        sel = (r2 < h[i] ** 2) & (np.arange(n) != i)
        want = (0.5 * m[i] * np.sum((vel[sel] - vel[i]) ** 2, 1)).max() if sel.any() else 0.0
        assert got[i] == pytest.approx(want, rel=1e-14), i


def _cold_streams(n=10):
    """Two cold streams colliding along x (|v| = 2, c_s ~ 0.03): the relative
    kinetic energy of neighbours dwarfs U."""
    w = dict(W.lattice_wave(n, jitter=0.0))
    m = np.full(w["x"].size, 1.0 / n ** 3)
    vx = np.where(w["x"] < 0.5, 2.0, -2.0)
    w["m"] = m
    w["px"], w["py"], w["pz"] = m * vx, 0.0 * m, 0.0 * m
    w["U"] = m * 1e-3 / (w["gamma"] - 1)
    w["E"] = w["U"] + 0.5 * m * vx * vx
    w["A"] = np.zeros(w["x"].size)
    return w


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
def test_entropy_constant_in_mfm_and_carried_in_mfv(orc, scheme):
    """The entropic function follows the pressure used at the start of the
    step (re-set from the energies where they gave the pressure); MFM keeps it
    constant along the particles, MFV carries m A with the mass fluxes, so
    sum m A is conserved to rounding."""
    w = _cold_streams()
    cfg = orc.config(gamma=w["gamma"], scheme=scheme, entropy=True)
    # two steps: the first sets A from the energies, the second may use it
    s1, _, i1 = orc.step(cfg, w, 1e-3)
    assert i1["status"] == 0 and np.all(s1["A"] > 0)
    s2, _, i2 = orc.step(cfg, s1, 1e-3)
    assert i2["status"] == 0
    # the A the second step started from: re-set where the energies gave p
    h, om = s2["h"], s2["omega"]
    ek = orc.ekin_max(s1["x"], s1["y"], s1["z"], s1["L"], h, s1["m"], s1["px"], s1["py"], s1["pz"])
    rho, _, _, _, p, src = orc.primitives(cfg, s1["m"], s1["px"], s1["py"], s1["pz"], s1["E"],
                                          s1["U"], om, h=h, A=s1["A"], ekmax=ek, want_src=True)
    assert (src == 1).sum() > 0           # the cold streams take the entropy route
    A_used = np.where(src == 1, s1["A"], p / rho ** w["gamma"])
    if scheme == "mfm":
        assert np.allclose(s2["A"], A_used, rtol=1e-14, atol=0.0)   # (numpy vs C pow: ulps)
    else:
        before = math.fsum(s1["m"] * A_used)
        after = math.fsum(s2["m"] * s2["A"])
        assert abs(after - before) < 1e-13 * math.fsum(np.abs(s1["m"] * A_used))


# --------------------------------------------------------------------------
# individual timesteps (§2.3.4 hierarchy, §2.3.10 criteria)
# --------------------------------------------------------------------------

def test_rung_select_closed_form(orc):
    """The smallest r >= 0 with min(dt_cfl, dt_acc) > 2^-r dt0: 0 above dt0,
    floor(log2(dt0 / t)) + 1 below it (strict at the powers of two), capped."""
    dt0 = 0.37
    cases = [(2 * dt0, np.inf, 0), (dt0, np.inf, 1), (dt0 * (1 + 1e-12), np.inf, 0),
             (dt0 / 2, np.inf, 2), (np.inf, dt0 / 4, 3), (dt0 / 3, dt0, 2), (dt0, dt0 / 3, 2),
             (np.inf, np.inf, 0)]
    for dtc, dta, want in cases:
        assert orc.rung_select(dtc, dta, dt0, 12) == (want, False), (dtc, dta)
    assert orc.rung_select(dt0 * 2.0 ** -13, np.inf, dt0, 12) == (12, True)
    assert orc.rung_select(dt0 * 2.0 ** -12 * 1.5, np.inf, dt0, 12) == (12, False)
    rng = np.random.default_rng(11)
    for t in dt0 * np.exp(rng.uniform(-8.0, 1.0, 400)):
        e = math.log2(dt0 / t)
        if abs(e - round(e)) < 1e-9:
            continue
        want = 0 if t > dt0 else math.floor(e) + 1
        assert orc.rung_select(t, np.inf, dt0, 20)[0] == want, t


def test_rung_limiter_is_graph_distance_bound(orc):
    """Limited rungs r_i = max_j (r0_j - 2 d(i, j)), d the hop distance in
    the interaction graph (breadth-first search from every particle)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import shortest_path
    rng = np.random.default_rng(12)
    n = 300
    pairs = set()
    while len(pairs) < 500:
        i, j = rng.integers(0, n, 2)
        if i != j:
            pairs.add((min(i, j), max(i, j)))
    pairs = np.array(sorted(pairs), dtype=np.int64)
    r0 = rng.integers(0, 12, n).astype(np.int32)
    r0[rng.random(n) < 0.7] = 0
    got, sweeps = orc.rung_limit(pairs, r0)
    g = coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(n, n))
    d = shortest_path(g, directed=False, unweighted=True)
    want = np.max(np.where(np.isfinite(d), r0[None, :] - 2 * d, -np.inf), axis=1)
    assert np.array_equal(got, want.astype(np.int32))
    assert sweeps >= 2
    for i, j in pairs:
        assert abs(int(got[i]) - int(got[j])) <= 2


def test_rungs_reduce_to_the_global_step(orc):
    """A base step no particle's criteria subdivide (every rung 0) is the
    global step with dt = dt0, to the last bit."""
    w = W.sod(8)
    co = orc.config(gamma=w["gamma"])
    _, _, i0 = orc.step(co, w, -1.0)
    dt0 = 0.5 * i0["dt"]
    sr, rung, ir = orc.step_rungs(co, w, dt0, c_acc=1e9)
    sg, _, _ = orc.step(co, w, dt0)
    assert ir["status"] == 0 and ir["rung_max"] == 0 and not rung.any()
    for k in ("x", "y", "z", "m", "px", "py", "pz", "E", "U", "h", "omega"):
        assert np.array_equal(sr[k], sg[k]), k


def test_rung_criteria_and_assignment(orc):
    """At the start: dt_cfl is the global step's per-particle CFL value (its
    minimum is the global CFL dt, Eq. 31); dt_acc = c_acc sqrt(h rho / |grad
    p|) for a linear pressure field (exact gradients away from the periodic
    seam, limiter off); the rungs are rung_select of the two, limited."""
    n = 12
    w = dict(W.lattice_wave(n, jitter=0.0))
    eps = 0.3
    x = w["x"]
    p = 1.0 + eps * x
    N = x.size
    m = np.full(N, 1.0 / n ** 3)
    w["m"] = m
    w["px"], w["py"], w["pz"] = 0.0 * m, 0.0 * m, 0.0 * m
    w["U"] = p * m / (w["gamma"] - 1.0)   # volume = 1 / n^3 = m at rho = 1
    w["E"] = w["U"].copy()
    co = orc.config(gamma=w["gamma"], limiter=False)
    _, _, i0 = orc.step(co, w, -1.0)
    c_acc = 0.2
    sr, rung, ir = orc.step_rungs(co, w, 4.0 * i0["dt"], c_acc=c_acc)
    assert ir["status"] == 0
    assert ir["dt_cfl"].min() == pytest.approx(i0["dt"], rel=1e-14)
    # interior: every neighbour within h on the same side of the seam
    h0 = orc.step(co, w, -1.0)[0]["h"]   # (the step's solved h at the start)
    inner = (x > 1.5 * h0.max()) & (x < 1.0 - 1.5 * h0.max())
    assert inner.sum() > N // 3
    # p_i = U_i (gamma - 1) / omega_i and rho_i = m_i / omega_i with the
    # lattice's uniform omega, so |grad p| / rho = eps exactly
    want = c_acc * np.sqrt(h0 / eps)
    assert np.allclose(ir["dt_acc"][inner], want[inner], rtol=1e-9, atol=0)
    r0 = np.array([orc.rung_select(a, b, 4.0 * i0["dt"], 12)[0]
                   for a, b in zip(ir["dt_cfl"], ir["dt_acc"])], dtype=np.int32)
    pairs = []
    L = w["L"]
    for i in range(N):
        d = np.stack([x - x[i], w["y"] - w["y"][i], w["z"] - w["z"][i]], 1)
        d -= np.round(d / L) * L
        r2 = (d[:, 0] ** 2 + d[:, 1] ** 2) + d[:, 2] ** 2
        hm = np.maximum(h0, h0[i])
        for j in np.nonzero((r2 < hm * hm) & (np.arange(N) > i))[0]:
            pairs.append((i, j))
    limited, _ = orc.rung_limit(np.array(pairs), r0)
    assert np.array_equal(rung, limited)
    assert len(set(rung.tolist())) >= 2


def test_rung_step_conserves_and_counts(orc):
    """Several rungs (Sod tube, dt0 = 8 CFL steps): mass, momentum and energy
    are conserved to rounding (every face applies min(dt_i, dt_j) to both
    sides); each particle takes 2^r_i steps."""
    w = W.sod(8)
    co = orc.config(gamma=w["gamma"])
    _, _, i0 = orc.step(co, w, -1.0)
    sr, rung, ir = orc.step_rungs(co, w, 8.0 * i0["dt"], c_acc=0.2)
    assert ir["status"] == 0
    assert len(set(rung.tolist())) >= 2 and ir["substeps"] == 2 ** ir["rung_max"]
    assert ir["active_steps"] == int(np.sum(2 ** rung.astype(np.int64)))
    for k in ("m", "E"):
        assert abs(math.fsum(sr[k]) - math.fsum(w[k])) < 1e-13 * math.fsum(np.abs(w[k]))
    scale = math.fsum(w["m"] * (np.abs(w["px"] / w["m"]) + np.sqrt(w["gamma"] * (w["gamma"] - 1)
                                                                   * w["U"] / w["m"])))
    for k in ("px", "py", "pz"):
        assert abs(math.fsum(sr[k]) - math.fsum(w[k])) < 1e-13 * scale, k


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
def test_rung_steps_follow_the_sod_solution(orc, scheme):
    """A gamma = 1.4 Sod tube run with individual timesteps (base steps of
    four CFL steps) stays as close to the exact solution as the global
    CFL-stepped run over the same time."""
    gamma, t_end = 1.4, 0.1
    n = 24
    a = 1.0 / n
    i, j, k = np.meshgrid(np.arange(2 * n), np.arange(4), np.arange(4), indexing="ij")
    x, y, z = (i.ravel() + 0.5) * a, (j.ravel() + 0.5) * a, (k.ravel() + 0.5) * a
    left = x < 1.0
    rho = np.where(left, 1.0, 0.25)
    p = np.where(left, 1.0, 0.1795)
    m = rho * a ** 3
    U = p * a ** 3 / (gamma - 1.0)
    zero = 0.0 * m
    w = dict(x=x, y=y, z=z, m=m, px=zero, py=zero, pz=zero, E=U.copy(), U=U,
             h=np.full(x.size, 2.0 * a), L=np.array([2.0, 4 * a, 4 * a]), gamma=gamma)
    co = orc.config(gamma=gamma, scheme=scheme)
    r = orc.riemann_star(1.0, 0.0, 1.0, 0.25, 0.0, 0.1795, gamma)

    def l1(s, t):
        sel = (s["x"] > 0.6) & (s["x"] < 1.4)
        ex = np.array([orc.riemann_sample(1.0, -(xi - 1.0) / t, 1.0, 0.25, -(xi - 1.0) / t,
                                          0.1795, gamma, r["p"], r["u"] - (xi - 1.0) / t)[0]
                       for xi in s["x"][sel]])
        return float(np.mean(np.abs(s["m"][sel] / s["omega"][sel] - ex)))

    errs, rungs = {}, set()
    for mode in ("global", "rungs"):
        s, t = dict(w), 0.0
        while t < t_end * (1 - 1e-12):
            _, _, i0 = orc.step(co, s, -1.0)
            if mode == "global":
                dt = min(i0["dt"], t_end - t)
                s, _, info = orc.step(co, s, dt)
            else:
                dt = min(4.0 * i0["dt"], t_end - t)
                s, rung, info = orc.step_rungs(co, s, dt, c_acc=0.2)
                rungs |= set(rung.tolist())
            assert info["status"] == 0
            t += dt
        # volumes at the final positions
        s["omega"] = orc.step(co, s, 1e-300)[0]["omega"]
        errs[mode] = l1(s, t)
    assert len(rungs) >= 2, rungs
    assert errs["rungs"] < 1.3 * errs["global"] + 2e-3, errs
    assert errs["rungs"] < 0.06, errs


def test_entropy_is_carried_upwind_by_mfv(orc):
    """A cold, nearly pressureless lattice with random velocities and a step
    in A (1e-8 on [0, 1/2), 2e-8 on [1/2, 1)).  The MFV mass fluxes (relative
    to the faces, which move with the particles' mean velocity) run both ways
    across the step; with the donor's A each particle's new A is a weighted
    mean of its own and its donors' values, so A stays within [1e-8, 2e-8]
    and particles farther than h from the step keep theirs (§2.3.7, the MFV
    transport of m A).  A receiver's or a central A would leave that range."""
    n = 16
    w = dict(W.lattice_wave(n, jitter=0.0))
    N = w["x"].size
    rng = np.random.default_rng(21)
    m = np.full(N, 1.0 / n ** 3)
    v = rng.normal(0.0, 0.3, (N, 3))
    w["m"] = m
    w["px"], w["py"], w["pz"] = m * v[:, 0], m * v[:, 1], m * v[:, 2]
    w["U"] = 1e-7 * m
    w["E"] = w["U"] + 0.5 * m * np.sum(v * v, 1)
    x = w["x"]
    w["A"] = np.where(x < 0.5, 1e-8, 2e-8)
    co = orc.config(gamma=w["gamma"], scheme="mfv", entropy=True)
    s1, _, info = orc.step(co, w, 0.01)
    assert info["status"] == 0
    # every particle took the entropy route (cold, E_kin^max >> U / alpha2)
    ek = orc.ekin_max(w["x"], w["y"], w["z"], w["L"], s1["h"], m, w["px"], w["py"], w["pz"])
    src = orc.primitives(co, m, w["px"], w["py"], w["pz"], w["E"], w["U"], s1["omega"],
                         h=s1["h"], A=w["A"], ekmax=ek, want_src=True)[-1]
    assert np.all(src == 1), np.bincount(src)
    A = s1["A"]
    assert A.min() >= 1e-8 * (1 - 1e-12) and A.max() <= 2e-8 * (1 + 1e-12), (A.min(), A.max())
    # mixing happened at both steps (x = 1/2 and the periodic x = 0)
    mixed = (A > 1e-8 * (1 + 1e-6)) & (A < 2e-8 * (1 - 1e-6))
    assert mixed.sum() > N // 20, mixed.sum()
    h = float(np.max(s1["h"]))
    d = np.minimum(np.abs(x - 0.5), np.minimum(x, 1.0 - x))   # distance to a step
    far = d > 1.5 * h
    assert far.sum() > N // 10
    assert np.allclose(A[far], w["A"][far], rtol=1e-12, atol=0)
