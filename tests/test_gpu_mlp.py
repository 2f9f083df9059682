"""The learned starting pressure on the GPU, through the C ABI, against the
FP64 reference network of oracle/mlp.py and the oracle's exact Riemann
solver: features, the training gradient (exact and bf16-rounded forward),
tensor-core inference within a bound derived from bf16 rounding, training
on faces the method records, the flux with the learned guess against the
flux without it, and the iterations it saves (judged by the oracle)."""
import numpy as np
import pytest

from oracle import mlp
from paper_2211_12243_gb300 import workloads as W

from parity_util import compare_masked, gpu_stages, oracle_stages

pytestmark = pytest.mark.gpu

GAMMA = 5.0 / 3.0


@pytest.fixture(scope="module")
def hyd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_12243_gb300 import build, hydro
    build.build()
    return hydro


def _random_faces(orc, n, seed, gamma=GAMMA):
    """Face problems over several decades of density and pressure ratio,
    away from vacuum, with p* from the oracle's exact solver.  float32 [7, n]."""
    rng = np.random.default_rng(seed)
    out = np.zeros((7, n), dtype=np.float32)
    k = 0
    while k < n:
        rl, rr = np.exp(rng.uniform(-3, 3, 2))
        pl, pr = np.exp(rng.uniform(-5, 5, 2))
        cl, cr = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
        ul, ur = rng.normal(0, 1.5, 2) * np.array([cl, cr])
        f = np.array([rl, ul, pl, rr, ur, pr], dtype=np.float32).astype(np.float64)
        c2 = np.sqrt(gamma * f[2] / f[0]) + np.sqrt(gamma * f[5] / f[3])
        if 2.0 / (gamma - 1.0) * c2 <= (f[4] - f[1]) * 1.05:
            continue
        r = orc.riemann_star(*f, gamma)
        if r["vacuum"] or not r["p"] > 0:
            continue
        out[:6, k] = f
        out[6, k] = r["p"]
        k += 1
    return out


def _theta(x, seed, out_scale=1.0):
    """Float32-representable parameters with the standardisation of x."""
    p = mlp.unpack(mlp.init(seed))
    rng = np.random.default_rng(seed + 100)
    p["b1"] = rng.normal(0, 0.1, mlp.NH)
    p["b2"] = rng.normal(0, 0.1, mlp.NH)
    p["w3"] = p["w3"] * out_scale
    p["b3"] = np.array([0.05])
    p["mean"] = x.mean(0)
    p["scale"] = x.std(0) + 1e-3
    p["xmin"], p["xmax"] = x.min(0) - 1.0, x.max(0) + 1.0
    return mlp.pack(p).astype(np.float32).astype(np.float64)


def _feature_tol(f64, gamma=GAMMA):
    """Per-face, per-feature bound on |float features - FP64 features|: a
    relative 2e-4 (fast float log, power and division), plus, for the three
    features built on a difference (PVRS, two-rarefaction numerator,
    two-shock numerator), eight float ulps of the terms relative to the
    difference itself, floored as the feature is (1e-6 p_a)."""
    rl, ul, pl, rr, ur, pr = f64[:6]
    eps = 8 * 2.0 ** -23
    pa, du = 0.5 * (pl + pr), ur - ul
    cl, cr = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
    t_pv = 0.125 * np.abs(du) * (rl + rr) * (cl + cr)
    ppv = pa - 0.125 * du * (rl + rr) * (cl + cr)
    fl = 1e-6 * pa
    num = cl + cr - 0.5 * (gamma - 1) * du
    p0 = np.maximum(ppv, 0.0)
    gl = np.sqrt((2.0 / ((gamma + 1.0) * rl)) / ((gamma - 1.0) / (gamma + 1.0) * pl + p0))
    gr = np.sqrt((2.0 / ((gamma + 1.0) * rr)) / ((gamma - 1.0) / (gamma + 1.0) * pr + p0))
    pts_n = gl * pl + gr * pr - du
    tol = np.zeros((f64.shape[1], 12))
    tol[:, 7] = eps * (pa + t_pv) / np.maximum(np.abs(ppv), fl)
    tol[:, 8] = 2 * gamma / (gamma - 1) * eps * (cl + cr + 0.5 * (gamma - 1) * np.abs(du)) / np.abs(num)
    tol[:, 9] = eps * (gl * pl + gr * pr + np.abs(du)) / np.maximum(np.abs(pts_n), fl * (gl + gr))
    # the two-shock value also inherits the PVRS error through gl, gr
    tol[:, 9] += tol[:, 7]
    return tol


def test_features_match_oracle(orc, hyd):
    import torch
    f = _random_faces(orc, 3000, 1)
    H = hyd.Hydro(hyd.default_config(gamma=GAMMA, precision="mixed"))
    x, t = H.mlp_features(torch.as_tensor(f, device="cuda"))
    x, t = x.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64)
    f64 = f.astype(np.float64)
    xo, pa = mlp.features(*f64[:6], GAMMA)
    to = mlp.target(xo, pa, f64[6])
    ftol = _feature_tol(f64)
    # fast float logs / powers: a few 1e-6 relative; the two-rarefaction
    # power (exponent 2 gamma / (gamma - 1) = 5) amplifies it five-fold
    assert np.all(np.abs(x - xo) <= 2e-4 * (1.0 + np.abs(xo)) + ftol)
    # the target subtracts the two-shock feature
    assert np.all(np.abs(t - to) <= 1e-4 * (1.0 + np.abs(to)) + 2e-4 * (1.0 + np.abs(xo[:, 9]))
                  + ftol[:, 9])


@pytest.mark.parametrize("quant", [False, True])
def test_gradient_matches_oracle(orc, hyd, quant):
    import torch
    f = _random_faces(orc, 1500, 2)
    xo, pa = mlp.features(*f.astype(np.float64)[:6], GAMMA)
    x32 = xo.astype(np.float32)
    x = x32.astype(np.float64)
    t = np.random.default_rng(3).normal(0, 1, x.shape[0]).astype(np.float32)
    theta = _theta(x, 4)
    H = hyd.Hydro(hyd.default_config(gamma=GAMMA, precision="mixed"))
    H.mlp_load(theta)
    g, loss = H.mlp_gradient(torch.as_tensor(x32, device="cuda"),
                             torch.as_tensor(t, device="cuda"), quant=quant)
    g = g.cpu().numpy().astype(np.float64)
    go = mlp.backward(theta, x, t.astype(np.float64), quant=quant)
    lo = mlp.loss(theta, x, t.astype(np.float64), quant=quant)
    assert float(loss.item()) == pytest.approx(lo, rel=1e-4)
    # per parameter block, relative to the block's largest entry: float
    # accumulation over 1500 samples, and with bf16 rounding the odd
    # activation whose float and double values round to neighbouring bf16s
    # (b3's gradient is the mean residual, which cancels: its scale is the
    # mean absolute residual)
    tol = 1e-3 if quant else 1e-4
    yo, _ = mlp.forward(theta, x, quant=quant)
    k = 0
    for name, shp in mlp.SIZES:
        m = int(np.prod(shp))
        a, b = g[k:k + m], go[k:k + m]
        k += m
        if name in mlp.FIXED:
            assert np.all(a == 0.0)
            continue
        scale = np.mean(np.abs(yo - t)) if name == "b3" else np.max(np.abs(b))
        assert np.max(np.abs(a - b)) <= tol * scale + 1e-12, name


def _predict_bound(theta, x, ftol):
    """Bound on |y_gpu - y_oracle(quant)| from the float features (the
    feature bound above), one bf16 ulp of every rounded input and activation
    that can round the other way, and float accumulation."""
    p = mlp.unpack(theta)
    _, (xs, a1, h1, a2, h2, W1, W2) = mlp.forward(theta, x, quant=True)
    ulp = lambda v: 2.0 ** (np.floor(np.log2(np.maximum(np.abs(v), 1e-30))) - 7)
    dxs = (2e-4 * (1.0 + np.abs(x)) + ftol) / p["scale"] + ulp(xs)
    da1 = dxs @ np.abs(W1).T + 1e-6 * (np.abs(xs) @ np.abs(W1).T + np.abs(p["b1"]))
    dh1 = np.where(a1 > -da1, da1 + ulp(h1), 0.0)
    da2 = dh1 @ np.abs(W2).T + 1e-6 * (np.abs(h1) @ np.abs(W2).T + np.abs(p["b2"]))
    dy = np.where(a2 > -da2, da2, 0.0) @ np.abs(p["w3"]) + 1e-6 * (np.abs(h2) @ np.abs(p["w3"]))
    return dy + 1e-5


def test_tensor_core_inference_matches_oracle(orc, hyd):
    import torch
    f = _random_faces(orc, 1000, 5)   # 8 tiles of 128 and a ragged tail
    f64 = f.astype(np.float64)
    xo, pa = mlp.features(*f64[:6], GAMMA)
    theta = _theta(xo, 6, out_scale=0.2)   # corrections |y| mostly below the limit of 2
    H = hyd.Hydro(hyd.default_config(gamma=GAMMA, precision="mixed"))
    H.mlp_load(theta)
    pg = H.mlp_predict(torch.as_tensor(f, device="cuda")).cpu().numpy().astype(np.float64)
    yo, _ = mlp.forward(theta, xo, quant=True)
    ftol = _feature_tol(f64)
    bound = _predict_bound(theta, xo, ftol)
    inrange = np.abs(yo) + bound <= 2.0   # the feature box holds every face
    assert inrange.sum() > 900
    ok = pg > 0
    assert np.all(ok[inrange])
    # y_gpu = ln(p_guess / p_TS); the oracle's p_TS differs from the
    # kernel's by the feature bound of x_9
    y = np.log(pg[inrange] / pa[inrange]) - xo[inrange, 9]
    err = np.abs(y - yo[inrange])
    lim = bound[inrange] + 2e-4 * (1.0 + np.abs(xo[inrange, 9])) + ftol[inrange, 9]
    assert np.all(err <= lim), (err.max(), np.argmax(err - lim))
    # the typical error is far inside the bound (most rows round alike)
    assert np.median(err) < 1e-3


def test_out_of_range_faces_keep_the_plain_guess(orc, hyd):
    import torch
    f = _random_faces(orc, 256, 7)
    f64 = f.astype(np.float64)
    xo, _ = mlp.features(*f64[:6], GAMMA)
    theta = _theta(xo, 8, out_scale=0.2)
    # a feature box of the middle half of the data on two features
    p = mlp.unpack(theta)
    q = np.quantile(xo, [0.25, 0.75], axis=0)
    p["xmin"][[0, 4]], p["xmax"][[0, 4]] = q[0, [0, 4]], q[1, [0, 4]]
    theta = mlp.pack(p).astype(np.float32).astype(np.float64)
    H = hyd.Hydro(hyd.default_config(gamma=GAMMA, precision="mixed"))
    H.mlp_load(theta)
    pg = H.mlp_predict(torch.as_tensor(f, device="cuda")).cpu().numpy()
    p = mlp.unpack(theta)
    tol = 2e-4 * (1.0 + np.abs(xo)) + _feature_tol(f64)
    out = np.any((xo + tol < p["xmin"]) | (xo - tol > p["xmax"]), 1)
    inside = np.all((xo - tol >= p["xmin"]) & (xo + tol <= p["xmax"]), 1)
    yo, _ = mlp.forward(theta, xo, quant=True)
    assert out.sum() > 100 and inside.sum() > 30
    assert np.all(pg[out] == -1.0)
    assert np.all(pg[inside & (np.abs(yo) < 1.9)] > 0)


def test_mlp_calls_reject_bad_state(hyd):
    import torch
    H = hyd.Hydro(hyd.default_config(gamma=GAMMA, precision="mixed"))
    f = torch.ones((7, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(hyd.HydroError) as e:
        H.mlp_predict(f)
    assert e.value.code == -9            # no network yet
    bad = np.ones(hyd.MLP_NPARAM, dtype=np.float32)
    bad[-1] = 0.0                        # a zero feature scale
    with pytest.raises(hyd.HydroError):
        H.mlp_load(bad)
    H.set_config(learned_guess=1)
    w = W.sod(4)
    st = hyd.to_device(w)
    H.set_boxes(*hyd.single_box(w))
    assert H.step(st, check=False, stats=False) == -9


def _record(hyd, w, steps, cap=1 << 20, keep=1.0):
    """Hard faces of `steps` plain mixed steps of workload w (GPU)."""
    import torch
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision="mixed"))
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    buf = torch.zeros((7, cap), dtype=torch.float32, device="cuda")
    H.record_faces(buf, keep=keep, hard_only=True)
    for _ in range(steps):
        H.step(st)
    n = min(H.recorded_faces(), cap)
    return buf[:, :n].contiguous()


@pytest.fixture(scope="module")
def trained(hyd):
    """A network trained on the GPU by the library's own kernels on the hard
    faces of Sedov blasts (16^3 and 20^3 lattices, 6 steps each) and of a
    log-normal field -- other lattices and fields than the test cases."""
    import torch
    faces = torch.cat([_record(hyd, W.sedov(16), 6), _record(hyd, W.sedov(20), 6),
                       _record(hyd, W.lognormal(8192, seed=5, grid=16), 2)], 1).contiguous()
    H = hyd.Hydro(hyd.default_config(gamma=GAMMA, precision="mixed"))
    loss = H.mlp_train(faces, steps=10000, batch=1024, lr=2e-3, seed=11).cpu().numpy()
    return dict(theta=H.mlp_get().astype(np.float64), loss=loss, n=faces.shape[1], faces=faces)


def test_training_reduces_the_loss(trained):
    loss = trained["loss"]
    assert trained["n"] > 2000
    assert np.all(np.isfinite(loss))
    assert loss[-200:].mean() < 0.1 * loss[:50].mean()


def _hard_mask(fc, gamma):
    """Faces whose adaptive guess (Toro 2009, §9.5.1) is the two-shock value."""
    rl, ul, pl, rr, ur, pr = fc[:, 0], fc[:, 1], fc[:, 2], fc[:, 3], fc[:, 4], fc[:, 5]
    cl, cr = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
    ppv = np.maximum(0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr), 0.0)
    pmin, pmax = np.minimum(pl, pr), np.maximum(pl, pr)
    pvrs = (pmax <= 2 * pmin) & (ppv >= pmin) & (ppv <= pmax)
    return ~pvrs & (ppv >= pmin)


@pytest.mark.parametrize("p_tol", [2e-6, 1e-12])
def test_learned_guess_saves_oracle_iterations(orc, trained, p_tol):
    """The oracle's own faces of a different Sedov lattice (12^3, first step):
    its exact solver started from the trained network's guess (where in
    range, as on the GPU) reaches the same fluxes in fewer Newton iterations
    than from the adaptive guess, at the mixed path's tolerance and at the
    FP64 one."""
    w = W.sedov(12)
    cfg = orc.config(gamma=w["gamma"], p_tol=p_tol)
    x, y, z, L = w["x"], w["y"], w["z"], w["L"]
    h, om, _, _ = orc.density(cfg, x, y, z, L, w["h"])
    prims = orc.primitives(cfg, w["m"], w["px"], w["py"], w["pz"], w["E"], w["U"], om)
    B6, _, nc = orc.matrices(cfg, x, y, z, L, h, om)
    grad, alpha, vsig = orc.gradients(cfg, x, y, z, L, h, om, prims, B6, nc)
    dt = 0.2 * np.min(h / vsig)
    pairs = orc.flux_pairs(x, y, z, L, h)
    dQ0, st0, fc = orc.fluxes(cfg, x, y, z, L, h, om, B6, prims, grad, alpha, dt, pairs=pairs,
                              want_faces=True)
    hard = _hard_mask(fc, w["gamma"]) & (fc[:, 6] > 0)
    assert hard.sum() > 100
    xo, pa = mlp.features(*fc[hard, :6].T, w["gamma"])
    yq, _ = mlp.forward(trained["theta"], xo, quant=True)
    use = mlp.use_learned(trained["theta"], xo, yq)
    assert use.mean() > 0.5
    guess = np.full(pairs.shape[0], -1.0)
    guess[np.nonzero(hard)[0][use]] = mlp.guess(xo, pa, yq)[use]
    dQ1, st1, fc1 = orc.fluxes(cfg, x, y, z, L, h, om, B6, prims, grad, alpha, dt, pairs=pairs,
                               pair_guess=guess, want_faces=True)
    # same star pressures and fluxes: the iteration converges either way, and
    # the last step squares the remaining error (below p_tol^2 relative)
    same = 1e-11 if p_tol < 1e-6 else 1e-9
    assert np.max(np.abs(fc1[:, 6] - fc[:, 6]) / np.maximum(fc[:, 6], 1e-300)) < same
    scale = np.abs(dQ0).max(0) + 1e-300
    assert np.max(np.abs(dQ1 - dQ0) / scale) < same
    it0, it1 = fc[hard, 8].mean(), fc1[hard, 8].mean()
    assert it1 < it0 - 0.5, (it0, it1)


@pytest.mark.parametrize("name", ["sedov12", "lognormal"])
def test_learned_flux_matches_oracle(orc, hyd, trained, name):
    """Staged mixed-precision fluxes with and without the learned guess
    against the FP64 oracle, per particle within the mixed path's 1e-5; the
    learned run solves the hard faces from the network and iterates less."""
    if name == "sedov12":
        w, dt, search = W.sedov(12), 1e-6, 1.3
    else:
        w, dt, search = W.lognormal(4096, seed=2, grid=16), 1e-3, 2.5
    o = oracle_stages(orc, orc.config(gamma=w["gamma"]), w, dt)
    res = {}
    for learned in (0, 1):
        H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision="mixed",
                                          learned_guess=learned))
        H.mlp_load(trained["theta"].astype(np.float32))
        g = gpu_stages(hyd, H, w, dt, search=search)
        # particles with (near-)singular E are masked as in the staged parity
        errs, bad = compare_masked(orc, w, o, g, 1e-5, ("dQ",))
        assert not bad, (learned, errs)
        res[learned] = H.get_stats()
    s0, s1 = res[0], res[1]
    # the plain kernel does not classify faces; the learned path defers the
    # hard ones and solves each from the network or, out of range, Toro's guess
    assert s0["hard_faces"] == 0 and s0["learned_faces"] == 0
    assert s1["hard_faces"] > 0
    assert s1["learned_faces"] > 0.2 * s1["hard_faces"]
    assert s1["learned_faces"] + s1["guess_fallbacks"] == s1["hard_faces"]
    assert s1["flux_pairs"] == s0["flux_pairs"]
    assert s1["newton_iters"] < s0["newton_iters"], (s0, s1)


def test_adaptive_learned_path_pauses_when_unused(hyd):
    """learned_guess = 1: a learned probe call, a plain probe call, then 15
    calls with the winner, then the probes again.  A network whose
    corrections all fall below 1e-3 starts no face, so the plain guess wins
    whatever the times; learned_guess = 2 never pauses."""
    p = mlp.unpack(mlp.init(1))
    p["w3"][:] = 0.0                     # y = t_mean + t_scale b3 = 0
    p["xmin"], p["xmax"] = np.full(mlp.NF, -1e30), np.full(mlp.NF, 1e30)
    theta = mlp.pack(p).astype(np.float32)
    w = W.sod(12)
    for mode, want in ((1, [1, 0] + [0] * 15 + [1, 0]), (2, [1] * 19)):
        H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision="mixed", learned_guess=mode))
        H.mlp_load(theta)
        H.set_boxes(*hyd.single_box(w))
        st = hyd.to_device(w)
        seen = []
        for _ in range(19):
            s = H.step(st)
            seen.append(s["learned_active"])
            if s["learned_active"]:
                assert s["hard_faces"] > 0 and s["learned_faces"] == 0
                assert s["guess_fallbacks"] == s["hard_faces"]
        assert seen == want, (mode, seen)
