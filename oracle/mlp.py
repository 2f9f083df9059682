"""FP64 reference of the star-pressure network (TEST INFRASTRUCTURE ONLY).

The learned guess feeds the exact Riemann solver of §2.3.3 (Toro 2009) a
starting pressure; the solver still iterates to its tolerance, so the
network changes the iteration count, not the answer.

Features (12) of a face problem (rho_L, u_L, p_L, rho_R, u_R, p_R; gamma),
with p_a = (p_L + p_R)/2, rho_a = (rho_L + rho_R)/2, c_a = sqrt(gamma p_a / rho_a):
  0 ln(p_L/p_a)     1 ln(p_R/p_a)     2 ln(rho_L/rho_a)   3 ln(rho_R/rho_a)
  4 (u_R - u_L)/c_a clipped to [-8, 8]
  5 c_L/c_a         6 c_R/c_a
  7 ln(max(p_PVRS, 1e-6 p_a)/p_a)   (primitive-variable linearisation)
  8 ln(p_TR/p_a)    (two-rarefaction value)
  9 ln(p_TS/p_a)    (two-shock value)
 10 |ln(p_L/p_R)|   11 (p_L - p_R)/(p_L + p_R)
Target: ln(p*/p_TS), the correction of the two-shock value (feature 9:
p_TS = p_a exp(x_9)); the learned guess is p_TS exp(y).  Network:
x -> relu(W1 x + b1) -> relu(W2 h + b2) -> y = t_mean + t_scale (w3.h + b3),
after a per-feature standardisation (x - mean) / scale.  The feature and
target standardisations and the box [xmin, xmax] of the training features
are fixed (set from the training data), the rest is trained.

Packed parameter order (float32 on the device side): W1[64][12], b1[64],
W2[64][64], b2[64], w3[64], b3, mean[12], scale[12], t_mean, t_scale,
xmin[12], xmax[12].
"""
from __future__ import annotations

import numpy as np

NF, NH = 12, 64
SIZES = [("W1", (NH, NF)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)),
         ("b3", (1,)), ("mean", (NF,)), ("scale", (NF,)), ("tmean", (1,)), ("tscale", (1,)),
         ("xmin", (NF,)), ("xmax", (NF,))]
FIXED = ("mean", "scale", "tmean", "tscale", "xmin", "xmax")
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def features(rl, ul, pl, rr, ur, pr, g):
    """Feature matrix [n, 12] (float64) of the face problems."""
    rl, ul, pl, rr, ur, pr = (np.asarray(v, dtype=np.float64) for v in (rl, ul, pl, rr, ur, pr))
    pa = 0.5 * (pl + pr)
    ra = 0.5 * (rl + rr)
    ca = np.sqrt(g * pa / ra)
    cl = np.sqrt(g * pl / rl)
    cr = np.sqrt(g * pr / rr)
    du = ur - ul
    ppv = 0.5 * (pl + pr) - 0.125 * du * (rl + rr) * (cl + cr)
    z = (g - 1.0) / (2.0 * g)
    # two-rarefaction value (exact for two rarefactions)
    num = cl + cr - 0.5 * (g - 1.0) * du
    num = np.maximum(num, 1e-12 * (cl + cr))
    ptr = (num / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    # two-shock value around max(0, p_PVRS)
    p0 = np.maximum(ppv, 0.0)
    gl = np.sqrt((2.0 / ((g + 1.0) * rl)) / ((g - 1.0) / (g + 1.0) * pl + p0))
    gr = np.sqrt((2.0 / ((g + 1.0) * rr)) / ((g - 1.0) / (g + 1.0) * pr + p0))
    pts = (gl * pl + gr * pr - du) / (gl + gr)
    floor = 1e-6 * pa
    x = np.stack([
        np.log(pl / pa), np.log(pr / pa), np.log(rl / ra), np.log(rr / ra),
        np.clip(du / ca, -8.0, 8.0), cl / ca, cr / ca,
        np.log(np.maximum(ppv, floor) / pa), np.log(np.maximum(ptr, floor) / pa),
        np.log(np.maximum(pts, floor) / pa), np.abs(np.log(pl / pr)), (pl - pr) / (pl + pr),
    ], axis=1)
    return x, pa


def target(x, pa, pstar):
    """Training target ln(p*/p_TS) of faces with features x."""
    return np.log(np.asarray(pstar, dtype=np.float64) / pa) - x[:, 9]


def guess(x, pa, y):
    """Starting pressure p_TS exp(y) from the network output y."""
    return pa * np.exp(x[:, 9] + y)


def in_range(theta, x, y):
    """Faces where the learned guess is used: every feature inside the box
    [xmin, xmax] of the training data and a correction |y| <= 2; elsewhere
    the solver keeps its plain guess."""
    p = unpack(theta)
    inside = np.all((x >= p["xmin"]) & (x <= p["xmax"]), axis=1)
    return inside & (np.abs(y) <= 2.0)


def use_learned(theta, x, y):
    """Faces that start the solver from the learned value: in range and a
    correction |y| >= 1e-3 (a smaller one keeps the two-shock value, which
    then starts within 1e-3 of p* anyway)."""
    return in_range(theta, x, y) & (np.abs(y) >= 1e-3)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, k = {}, 0
    for name, shp in SIZES:
        m = int(np.prod(shp))
        out[name] = theta[k:k + m].reshape(shp)
        k += m
    return out


def pack(params):
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel() for name, _ in SIZES])


def init(seed=0):
    rng = np.random.default_rng(seed)
    p = {
        "W1": rng.normal(0, np.sqrt(2.0 / NF), (NH, NF)),
        "b1": np.zeros(NH),
        "W2": rng.normal(0, np.sqrt(2.0 / NH), (NH, NH)),
        "b2": np.zeros(NH),
        "w3": rng.normal(0, np.sqrt(1.0 / NH), NH),
        "b3": np.zeros(1),
        "mean": np.zeros(NF),
        "scale": np.ones(NF),
        "tmean": np.zeros(1),
        "tscale": np.ones(1),
        "xmin": np.full(NF, -1e30),
        "xmax": np.full(NF, 1e30),
    }
    return pack(p)


def bf16(a):
    """Round to bfloat16 (8 significant bits, round to nearest, ties to even),
    applied to the float32 value as the device does; returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def forward(theta, x, quant=False):
    """Prediction [n] and the intermediates (for backward).  quant=True rounds
    the standardised inputs, W1, the first hidden activations and W2 to
    bf16, the operands of the tensor-core products; sums stay exact here."""
    p = unpack(theta)
    q = bf16 if quant else (lambda v: v)
    xs = q((x - p["mean"]) / p["scale"])
    W1, W2 = q(p["W1"]), q(p["W2"])
    a1 = xs @ W1.T + p["b1"]
    h1 = q(np.maximum(a1, 0.0))
    a2 = h1 @ W2.T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = p["tmean"][0] + p["tscale"][0] * (h2 @ p["w3"] + p["b3"][0])
    return y, (xs, a1, h1, a2, h2, W1, W2)


def loss(theta, x, t, quant=False):
    y, _ = forward(theta, x, quant)
    return 0.5 * np.mean((y - t) ** 2)


def backward(theta, x, t, quant=False):
    """Gradient of the mean squared error 0.5 mean((y - t)^2) with respect to
    the trainable parameters (W1, b1, W2, b2, w3, b3); the standardisations
    (mean, scale, t_mean, t_scale) are fixed and get zero gradient.  With quant=True the
    forward pass rounds as in forward(quant=True) and the backward pass
    treats each rounding as the identity (straight-through), using the
    rounded values in every product."""
    p = unpack(theta)
    y, (xs, a1, h1, a2, h2, W1, W2) = forward(theta, x, quant)
    n = x.shape[0]
    dy = p["tscale"][0] * (y - t) / n
    g = {name: np.zeros(shp) for name, shp in SIZES}
    g["w3"] = h2.T @ dy
    g["b3"] = np.array([dy.sum()])
    dh2 = np.outer(dy, p["w3"])
    da2 = dh2 * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    dh1 = da2 @ W2
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ xs
    g["b1"] = da1.sum(0)
    return pack(g)
