"""Seeded synthetic initial conditions for the hydro step.

These generators only lay particles down and fill in their conserved
quantities from a prescribed (rho, v, P) field; they hold none of the hydro
method's arithmetic.  Both the GPU library's tests and the CPU oracle's tests
draw their inputs from here.

Every generator returns a dict of float64 numpy arrays in structure-of-arrays
form (x, y, z, m, px, py, pz, E, U, h) plus the periodic box lengths ``L`` and
the adiabatic index.  ``h`` is a first guess of the compact-support radius
from the prescribed number density, (4 pi / 3) n h^3 = N_NGB (§2.3.5, Eq. 18).

Workloads (the problems of §3.1 of the paper, in the sizes used here):
  * ``lattice_wave``: jittered cubic lattice, rho = 1 + 0.1 sin(2 pi x) set by
    the particle masses, uniform P = 1, v = 0.
  * ``sod``: 3D shock tube in a 4 x 1 x 1 periodic box, left lattice
    rho = 1, P = 1 (spacing a), right lattice rho = 0.125, P = 0.1 (spacing 2a),
    equal particle masses, interfaces at x = 0 and x = 2.
  * ``lognormal``: clustered box from a lognormal density field with contrast
    1e4, P proportional to rho^gamma, Gaussian velocities of 0.1 sound speeds.
  * ``sedov``: uniform lattice, rho = 1, P = 1e-6, unit energy deposited
    kernel-weighted on the 32 particles nearest the box centre.
  * ``batch``: many independent periodic boxes of mixed sizes and generators.
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 20221122
N_NGB = 32.0


def _h_guess(number_density, n_ngb=N_NGB):
    return np.cbrt(3.0 * n_ngb / (4.0 * math.pi * number_density))


def _pack(x, y, z, m, vx, vy, vz, u_spec, h, L, gamma, name, **meta):
    m = np.ascontiguousarray(m, dtype=np.float64)
    px, py, pz = m * vx, m * vy, m * vz
    U = m * u_spec
    E = U + 0.5 * m * (vx * vx + vy * vy + vz * vz)
    out = dict(
        x=np.ascontiguousarray(x, dtype=np.float64),
        y=np.ascontiguousarray(y, dtype=np.float64),
        z=np.ascontiguousarray(z, dtype=np.float64),
        m=m,
        px=np.ascontiguousarray(px), py=np.ascontiguousarray(py),
        pz=np.ascontiguousarray(pz),
        E=np.ascontiguousarray(E), U=np.ascontiguousarray(U),
        h=np.ascontiguousarray(h, dtype=np.float64),
        L=np.asarray(L, dtype=np.float64), gamma=float(gamma), name=name,
    )
    out.update(meta)
    return out


def _lattice(nx, ny, nz, a, x0=0.0):
    i = (np.arange(nx) + 0.5) * a + x0
    j = (np.arange(ny) + 0.5) * a
    k = (np.arange(nz) + 0.5) * a
    X, Y, Z = np.meshgrid(i, j, k, indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def _wrap(v, L):
    v = np.mod(v, L)
    v[v >= L] -= L  # np.mod can round up to L
    return v


def lattice_wave(n=32, seed=0, gamma=5.0 / 3.0, jitter=1e-3):
    """n^3 jittered lattice in the unit box: rho = 1 + 0.1 sin(2 pi x) through
    the masses, P = 1, v = 0.  Jitter uniform in +-jitter*a per axis."""
    rng = np.random.default_rng(BASE_SEED + 0 + 1000 * seed)
    a = 1.0 / n
    x, y, z = _lattice(n, n, n, a)
    N = x.size
    x = _wrap(x + rng.uniform(-jitter * a, jitter * a, N), 1.0)
    y = _wrap(y + rng.uniform(-jitter * a, jitter * a, N), 1.0)
    z = _wrap(z + rng.uniform(-jitter * a, jitter * a, N), 1.0)
    rho = 1.0 + 0.1 * np.sin(2.0 * math.pi * x)
    m = rho * a ** 3
    P = np.ones(N)
    zero = np.zeros(N)
    h = _h_guess(np.full(N, 1.0 / a ** 3))
    return _pack(x, y, z, m, zero, zero, zero, P / ((gamma - 1.0) * rho), h,
                 (1.0, 1.0, 1.0), gamma, f"lattice_wave_{n}")


def sod(n=78, gamma=5.0 / 3.0, rho_l=1.0, p_l=1.0, rho_r=0.125, p_r=0.1):
    """3D Sod tube, box 4 x 1 x 1: left x in [0,2) lattice of spacing 1/n
    (2n x n x n particles), right x in [2,4) lattice of spacing 2/n
    (n x n/2 x n/2).  Equal masses m = rho_l / n^3, so rho_r = rho_l / 8.
    n = 78 gives 1,067,742 particles."""
    assert n % 2 == 0
    a = 1.0 / n
    xl, yl, zl = _lattice(2 * n, n, n, a)
    xr, yr, zr = _lattice(n, n // 2, n // 2, 2 * a, x0=2.0)
    x = np.concatenate([xl, xr])
    y = np.concatenate([yl, yr])
    z = np.concatenate([zl, zr])
    N = x.size
    m = np.full(N, rho_l * a ** 3)
    left = np.arange(N) < xl.size
    rho = np.where(left, rho_l, rho_l / 8.0)
    P = np.where(left, p_l, p_r)
    zero = np.zeros(N)
    nd = np.where(left, 1.0 / a ** 3, 1.0 / (2 * a) ** 3)
    h = _h_guess(nd)
    return _pack(x, y, z, m, zero, zero, zero, P / ((gamma - 1.0) * rho), h,
                 (4.0, 1.0, 1.0), gamma, f"sod_{n}", rho_r=rho_l / 8.0, p_r=p_r,
                 rho_l=rho_l, p_l=p_l, n_left=int(xl.size))


def _gaussian_field(G, seed, slope=-2.0):
    rng = np.random.default_rng(seed)
    k = np.fft.fftfreq(G) * G
    kx, ky, kz = np.meshgrid(k, k, k[: G // 2 + 1], indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** (slope / 2.0)
    noise = rng.standard_normal((G, G, G))
    f = np.fft.irfftn(np.fft.rfftn(noise) * amp, s=(G, G, G), axes=(0, 1, 2))
    f -= f.mean()
    f /= f.std()
    return f


def lognormal(N=1 << 24, seed=0, gamma=5.0 / 3.0, contrast=1e4, grid=None, vel_frac=0.1):
    """Clustered unit box: density delta = exp(s g - s^2/2) from a Gaussian
    field g (P(k) ~ k^-2) on grid^3 cells, s chosen so max/min = contrast;
    N particles drawn multinomially over cells, uniform within a cell.
    Equal masses 1/N; P = K rho^gamma with K such that the particle-mean
    sound speed is 1; velocities N(0, (vel_frac c_s)^2) per axis."""
    rng = np.random.default_rng(BASE_SEED + 2 + 1000 * seed)
    if grid is None:
        grid = int(min(256, max(16, 2 ** round(math.log2(N ** (1.0 / 3.0))))))
    g = _gaussian_field(grid, BASE_SEED + 2 + 1000 * seed + 7)
    s = math.log(contrast) / (g.max() - g.min())
    delta = np.exp(s * g - 0.5 * s * s)
    prob = (delta / delta.sum()).ravel()
    counts = rng.multinomial(N, prob)
    cell = np.repeat(np.arange(prob.size), counts)
    ci, cj, ck = np.unravel_index(cell, (grid, grid, grid))
    a = 1.0 / grid
    x = _wrap((ci + rng.random(N)) * a, 1.0)
    y = _wrap((cj + rng.random(N)) * a, 1.0)
    z = _wrap((ck + rng.random(N)) * a, 1.0)
    perm = rng.permutation(N)
    x, y, z, cell = x[perm], y[perm], z[perm], cell[perm]
    mean_delta = delta.mean()
    rho = (delta.ravel() / mean_delta)[cell]
    m = np.full(N, 1.0 / N)
    cs_shape = rho ** ((gamma - 1.0) / 2.0)
    K = 1.0 / (gamma * cs_shape.mean() ** 2)
    P = K * rho ** gamma
    cs = np.sqrt(gamma * P / rho)
    vx = rng.standard_normal(N) * vel_frac * cs
    vy = rng.standard_normal(N) * vel_frac * cs
    vz = rng.standard_normal(N) * vel_frac * cs
    h = _h_guess(rho * N)
    return _pack(x, y, z, m, vx, vy, vz, P / ((gamma - 1.0) * rho), h,
                 (1.0, 1.0, 1.0), gamma, f"lognormal_{N}")


def _wendland(r, H):
    q = r / H
    return np.where(q < 1.0, 21.0 / (2.0 * math.pi * H ** 3) * (1 - q) ** 4 * (1 + 4 * q), 0.0)


def sedov(n=128, gamma=5.0 / 3.0, p0=1e-6, e_blast=1.0):
    """n^3 lattice (n even) in the unit box, rho = 1, P = p0, v = 0; energy
    e_blast added as internal energy to the 32 particles of the two lattice
    shells nearest the box centre (8 at r^2 = 3/4 a^2, 24 at 11/4 a^2), with
    weights W(r, H), H = sqrt(19)/2 a (the third shell gets zero)."""
    assert n % 2 == 0
    a = 1.0 / n
    x, y, z = _lattice(n, n, n, a)
    N = x.size
    m = np.full(N, a ** 3)
    r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
    H = math.sqrt(19.0) / 2.0 * a
    w = _wendland(r, H)
    u_spec = np.full(N, p0 / ((gamma - 1.0) * 1.0))
    w_sum = w.sum()
    u_spec = u_spec + e_blast * (w / w_sum) / m
    zero = np.zeros(N)
    h = _h_guess(np.full(N, 1.0 / a ** 3))
    return _pack(x, y, z, m, zero, zero, zero, u_spec, h, (1.0, 1.0, 1.0), gamma,
                 f"sedov_{n}", n_hot=int((w > 0).sum()))


def batch(nbox=512, seed=0, nmin=4096, nmax=65536):
    """nbox independent periodic boxes, sizes log-uniform in [nmin, nmax],
    generators cycling lattice_wave / sod / lognormal (box k uses the
    generator k % 3).  Returns the concatenation with box_off[nbox+1] and
    box_len[3 nbox]."""
    rng = np.random.default_rng(BASE_SEED + 4 + 1000 * seed)
    sizes = np.exp(rng.uniform(math.log(nmin), math.log(nmax), nbox)).astype(np.int64)
    parts = []
    for k in range(nbox):
        kind = k % 3
        if kind == 0:
            n = max(4, int(round(sizes[k] ** (1.0 / 3.0))))
            p = lattice_wave(n, seed=seed * 100003 + k)
        elif kind == 1:
            # sod(n): 2n^3 + n^3/4 particles
            n = max(4, 2 * int(round((sizes[k] / 2.25) ** (1.0 / 3.0) / 2.0)))
            p = sod(n)
        else:
            p = lognormal(int(sizes[k]), seed=seed * 100003 + k, grid=16)
        parts.append(p)
    keys = ["x", "y", "z", "m", "px", "py", "pz", "E", "U", "h"]
    out = {k: np.concatenate([p[k] for p in parts]) for k in keys}
    counts = np.array([p["x"].size for p in parts], dtype=np.int64)
    out["box_off"] = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    out["box_len"] = np.concatenate([p["L"] for p in parts]).astype(np.float64)
    out["gamma"] = 5.0 / 3.0
    out["name"] = f"batch_{nbox}"
    out["L"] = None
    return out


def config_workload(k, small=False):
    """The five benchmark problems by index: 0 lattice_wave(32),
    1 sod(78), 2 lognormal(2^24), 3 sedov(128), 4 batch(512).  small=True
    gives a reduced size of the same generator."""
    if k == 0:
        return lattice_wave(16 if small else 32)
    if k == 1:
        return sod(16 if small else 78)
    if k == 2:
        return lognormal(1 << 14 if small else 1 << 24)
    if k == 3:
        return sedov(16 if small else 128)
    if k == 4:
        return batch(8 if small else 512, nmin=512 if small else 4096,
                     nmax=4096 if small else 65536)
    raise ValueError(k)
