"""Pins of the FP64 star-pressure network reference (oracle/mlp.py): the
analytic gradient against central finite differences, and the physics-based
features against the exact solver on problems where they are exact."""
import numpy as np
import pytest

from oracle import mlp


def _data(n=64, seed=0):
    rng = np.random.default_rng(seed)
    rl = np.exp(rng.uniform(-2, 2, n))
    rr = np.exp(rng.uniform(-2, 2, n))
    pl = np.exp(rng.uniform(-4, 4, n))
    pr = np.exp(rng.uniform(-4, 4, n))
    ul = rng.normal(0, 1, n)
    ur = rng.normal(0, 1, n)
    x, pa = mlp.features(rl, ul, pl, rr, ur, pr, 5.0 / 3.0)
    t = rng.normal(0, 1, n)
    return x, t


def test_backward_matches_finite_differences():
    x, t = _data()
    theta = mlp.init(3)
    p = mlp.unpack(theta)
    p["mean"] = x.mean(0)
    p["scale"] = x.std(0) + 1e-3
    p["b1"] = np.random.default_rng(4).normal(0, 0.1, mlp.NH)
    p["tmean"], p["tscale"] = np.array([0.3]), np.array([0.7])
    theta = mlp.pack(p)
    g = mlp.backward(theta, x, t)
    rng = np.random.default_rng(5)
    n_train = mlp.NPARAM - 4 * mlp.NF - 2
    for idx in rng.choice(n_train, 60, replace=False):
        e = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[idx] += e
        tm[idx] -= e
        fd = (mlp.loss(tp, x, t) - mlp.loss(tm, x, t)) / (2 * e)
        assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), idx
    # standardisation parameters are fixed
    assert np.all(g[n_train:] == 0.0)


def test_two_rarefaction_feature_is_exact_for_two_rarefactions(orc):
    # Toro's test 2 (strong double rarefaction) and a mild one: the
    # two-rarefaction value is the exact star pressure
    for d in [(1.0, -2.0, 0.4, 1.0, 2.0, 0.4), (1.0, -0.3, 1.0, 0.5, 0.2, 0.7)]:
        g = 1.4
        x, pa = mlp.features(*[np.array([v]) for v in d], g)
        r = orc.riemann_star(*d, g)
        assert pa[0] * np.exp(x[0, 8]) == pytest.approx(r["p"], rel=1e-10)


def test_two_shock_and_pvrs_features_on_a_contact(orc):
    # equal pressures and velocities: p* = p; PVRS and two-shock give it exactly
    x, pa = mlp.features(np.array([1.0]), np.array([0.3]), np.array([2.0]), np.array([0.125]),
                         np.array([0.3]), np.array([2.0]), 5.0 / 3.0)
    assert x[0, 7] == pytest.approx(0.0, abs=1e-15)
    assert x[0, 9] == pytest.approx(0.0, abs=1e-14)
    assert x[0, 0] == 0.0 and x[0, 1] == 0.0 and x[0, 4] == 0.0


def test_bf16_rounding_ties_to_even():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa (1)
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    # just above a tie rounds up; just below rounds down
    assert mlp.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert mlp.bf16(1.0 + 2.0 ** -8 - 2.0 ** -20) == 1.0
    assert mlp.bf16(-3.0) == -3.0 and mlp.bf16(0.0) == 0.0
    # 8 significant bits: 257 is not representable, 256 and 258 are
    assert mlp.bf16(257.0) == 256.0 and mlp.bf16(258.0) == 258.0
    assert mlp.bf16(1e-30) == pytest.approx(1e-30, rel=2 ** -8)


def test_quantised_forward_equals_exact_on_representable_values():
    # every operand already a bf16 value (small dyadic numbers): rounding is a no-op
    rng = np.random.default_rng(7)
    p = mlp.unpack(mlp.init(0))
    p["W1"] = rng.integers(-8, 9, p["W1"].shape) / 8.0
    p["W2"] = rng.integers(-8, 9, p["W2"].shape) / 64.0
    p["mean"] = np.zeros(mlp.NF)
    p["scale"] = np.ones(mlp.NF)
    theta = mlp.pack(p)
    x = rng.integers(-4, 5, (16, mlp.NF)) / 4.0
    y0, _ = mlp.forward(theta, x)
    # the hidden activations are sums of few dyadic terms: exact in 8 bits here
    y1, _ = mlp.forward(theta, x, quant=True)
    _, inter = mlp.forward(theta, x)
    assert np.all(mlp.bf16(inter[2]) == inter[2])
    assert np.array_equal(y0, y1)


def test_quantised_backward_matches_finite_differences_of_the_surrogate():
    # straight-through: the gradient equals the exact gradient of the network
    # whose weights are the rounded ones (rounding held fixed)
    x, t = _data(32, seed=3)
    theta = mlp.init(5)
    p = mlp.unpack(theta)
    p["mean"] = x.mean(0)
    p["scale"] = x.std(0) + 1e-3
    theta = mlp.pack(p)
    g = mlp.backward(theta, x, t, quant=True)
    _, (xs, a1, h1, a2, h2, W1, W2) = mlp.forward(theta, x, quant=True)
    # surrogate: unquantised network on the rounded inputs/weights, with h1
    # replaced by its rounded value through a fixed offset
    q = dict(p)
    q["W1"], q["W2"] = W1, W2
    q["mean"], q["scale"] = np.zeros(mlp.NF), np.ones(mlp.NF)
    q["tmean"], q["tscale"] = np.zeros(1), np.ones(1)
    q["xmin"], q["xmax"] = np.full(mlp.NF, -1e30), np.full(mlp.NF, 1e30)
    off = h1 - np.maximum(xs @ W1.T + p["b1"], 0.0)

    def surrogate_loss(th):
        r = mlp.unpack(th)
        hh = np.maximum(xs @ r["W1"].T + r["b1"], 0.0) + off
        aa = hh @ r["W2"].T + r["b2"]
        yy = np.maximum(aa, 0.0) @ r["w3"] + r["b3"][0]
        return 0.5 * np.mean((yy - t) ** 2)

    th0 = mlp.pack(q)
    rng = np.random.default_rng(9)
    n_train = mlp.NPARAM - 4 * mlp.NF - 2
    for idx in rng.choice(n_train, 40, replace=False):
        e = 1e-6
        tp, tm = th0.copy(), th0.copy()
        tp[idx] += e
        tm[idx] -= e
        fd = (surrogate_loss(tp) - surrogate_loss(tm)) / (2 * e)
        assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), idx
