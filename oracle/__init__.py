"""ctypes front end of the FP64 CPU oracle (``hydro_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the GPU library never does.

``build()`` compiles ``hydro_oracle.c`` with gcc (-O2, -ffp-contract=off,
OpenMP) into ``liboracle.so`` next to it.  Every wrapper takes and returns
float64 numpy arrays in the caller's particle order.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hydro_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


_CNT_SRC = os.path.join(_HERE, "flopcount.cpp")
_CNT_LIB = os.path.join(_HERE, "libflopcount.so")
_cnt = None


def _fresh(lib, *srcs):
    return os.path.exists(lib) and all(os.path.getmtime(lib) >= os.path.getmtime(s) for s in srcs)


def build(force=False):
    """Compile the oracle shared library and its operation-counting build
    (seconds)."""
    if force or not _fresh(_LIB, _SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    if force or not _fresh(_CNT_LIB, _SRC, _CNT_SRC):
        tmp = _CNT_LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-w", "-o", tmp, _CNT_SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _CNT_LIB)
    return _LIB


class Config(C.Structure):
    _fields_ = [
        ("gamma", C.c_double), ("kernel", C.c_int), ("n_ngb", C.c_double),
        ("scheme", C.c_int), ("riemann", C.c_int), ("limiter", C.c_int),
        ("time_extrap", C.c_int), ("ncond_crit", C.c_double), ("ngb_grow", C.c_double),
        ("max_ngb_grow", C.c_int), ("psi1", C.c_double), ("psi2", C.c_double),
        ("beta_min", C.c_double), ("beta_max", C.c_double), ("c_cfl", C.c_double),
        ("alpha1", C.c_double), ("h_tol", C.c_double), ("p_tol", C.c_double),
        ("max_h_iter", C.c_int), ("max_newton", C.c_int), ("entropy", C.c_int),
        ("alpha2", C.c_double), ("alpha3", C.c_double),
    ]


class FluxStats(C.Structure):
    _fields_ = [("newton_iters", C.c_int64), ("faces", C.c_int64), ("vacuum", C.c_int64),
                ("bisect_fallback", C.c_int64), ("first_order", C.c_int64),
                ("pairs", C.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class StepInfo(C.Structure):
    _fields_ = [("dt", C.c_double), ("dt_next", C.c_double), ("ngb_rounds", C.c_int),
                ("ncond_fail", C.c_int64), ("grad_pairs", C.c_int64), ("flux", FluxStats)]


class RungInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("rung_max", C.c_int), ("substeps", C.c_int64),
                ("active_steps", C.c_int64), ("faces", C.c_int64), ("capped", C.c_int64),
                ("limiter_sweeps", C.c_int)]


def config(gamma=5.0 / 3.0, kernel="wendland", n_ngb=32.0, scheme="mfv", riemann="exact",
           limiter=True, time_extrap=True, ncond_crit=100.0, ngb_grow=1.2, max_ngb_grow=5,
           psi1=0.5, psi2=0.25, beta_min=1.0, beta_max=2.0, c_cfl=0.2, alpha1=0.01,
           h_tol=1e-10, p_tol=1e-12, max_h_iter=60, max_newton=100, entropy=False,
           alpha2=1e-3, alpha3=1e-3):
    return Config(gamma, {"wendland": 0, "cubic": 1}[kernel], n_ngb,
                  {"mfv": 0, "mfm": 1}[scheme], {"exact": 0, "hllc": 1}[riemann],
                  int(bool(limiter)), int(bool(time_extrap)), ncond_crit, ngb_grow,
                  max_ngb_grow, psi1, psi2, beta_min, beta_max, c_cfl, alpha1, h_tol, p_tol,
                  max_h_iter, max_newton, int(bool(entropy)), alpha2, alpha3)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        d, i64, i32, vp = C.c_double, C.c_int64, C.c_int, C.c_void_p
        P = C.POINTER
        L.orc_kernel_W.restype = d
        L.orc_kernel_W.argtypes = [i32, d, d]
        L.orc_kernel_dWdH.restype = d
        L.orc_kernel_dWdH.argtypes = [i32, d, d]
        L.orc_neighbours.restype = i64
        L.orc_neighbours.argtypes = [i64, vp, vp, vp, vp, vp, i32, i64, vp, vp]
        L.orc_density.restype = i32
        L.orc_density.argtypes = [P(Config), i64, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_primitives.restype = None
        L.orc_primitives.argtypes = [P(Config), i64] + [vp] * 17
        L.orc_matrices.restype = None
        L.orc_matrices.argtypes = [P(Config), i64, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_gradients.restype = None
        L.orc_gradients.argtypes = [P(Config), i64] + [vp] * 16
        L.orc_flux_pairs.restype = i64
        L.orc_flux_pairs.argtypes = [i64, vp, vp, vp, vp, vp, i64, vp]
        L.orc_fluxes.restype = None
        L.orc_fluxes.argtypes = ([P(Config), i64] + [vp] * 14 + [d, i64, vp, vp, vp,
                                 P(FluxStats), vp, vp, vp, vp, vp])
        L.orc_fluxes_rung.restype = None
        L.orc_fluxes_rung.argtypes = ([P(Config), i64] + [vp] * 16 + [i64, vp, vp,
                                      P(FluxStats), vp])
        L.orc_riemann_guess.restype = d
        L.orc_riemann_guess.argtypes = [d] * 7
        L.orc_riemann_star.restype = i32
        L.orc_riemann_star.argtypes = [d] * 9 + [i32, P(d), P(d), P(i32), P(i32)]
        L.orc_riemann_sample.restype = None
        L.orc_riemann_sample.argtypes = [d] * 9 + [P(d), P(d), P(d), P(i32)]
        L.orc_hllc.restype = None
        L.orc_hllc.argtypes = [d, d, d, vp, d, d, d, vp, vp, d, vp, P(d), P(d)]
        L.orc_pair_limit.restype = d
        L.orc_pair_limit.argtypes = [d] * 5 + [i32]
        L.orc_step.restype = i32
        L.orc_step.argtypes = ([P(Config), i64] + [vp] * 14 + [d] + [vp] * 5 + [P(StepInfo)])
        L.orc_ekin_max.restype = None
        L.orc_rung_select.restype = i32
        L.orc_rung_select.argtypes = [d, d, d, i32, P(i32)]
        L.orc_rung_limit.restype = i32
        L.orc_rung_limit.argtypes = [i64, vp, vp]
        L.orc_step_rungs.restype = i32
        L.orc_step_rungs.argtypes = ([P(Config), i64] + [vp] * 12 + [d, d, i32, vp, vp, vp,
                                                                    P(RungInfo)])
        L.orc_ekin_max.argtypes = [i64] + [vp] * 10
        L.orc_num_threads.restype = i32
        L.orc_set_num_threads.argtypes = [i32]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(t):
    lib().orc_set_num_threads(int(t))


def kernel_W(r, H, kernel="wendland"):
    k = {"wendland": 0, "cubic": 1}[kernel]
    f = lib().orc_kernel_W
    return np.vectorize(lambda rr: f(k, float(rr), float(H)))(r)


def kernel_dWdH(r, H, kernel="wendland"):
    k = {"wendland": 0, "cubic": 1}[kernel]
    f = lib().orc_kernel_dWdH
    return np.vectorize(lambda rr: f(k, float(rr), float(H)))(r)


def neighbours(x, y, z, L, hs, use_grid=True):
    """Gather lists {j : r_ij < hs_i} (self included), rows ascending: (off, idx)."""
    x, y, z, L, hs = map(_f64, (x, y, z, L, hs))
    n = x.size
    off = np.zeros(n + 1, dtype=np.int64)
    tot = lib().orc_neighbours(n, _p(x), _p(y), _p(z), _p(L), _p(hs), int(use_grid), 0,
                               _p(off), None)
    idx = np.zeros(max(tot, 1), dtype=np.int32)
    tot2 = lib().orc_neighbours(n, _p(x), _p(y), _p(z), _p(L), _p(hs), int(use_grid), tot,
                                _p(off), _p(idx))
    assert tot2 == tot
    return off, idx[:tot]


def density(cfg, x, y, z, L, h_guess, n_ngb=None, active=None):
    """Solve Eq. 18 for h; returns (h, omega, iters, status)."""
    x, y, z, L = map(_f64, (x, y, z, L))
    h = _f64(h_guess).copy()
    n = x.size
    om = np.zeros(n)
    it = np.zeros(n, dtype=np.int32)
    nn = None if n_ngb is None else _f64(n_ngb)
    act = None if active is None else np.ascontiguousarray(active, dtype=np.int32)
    st = lib().orc_density(C.byref(cfg), n, _p(x), _p(y), _p(z), _p(L), _p(nn), _p(act),
                           _p(h), _p(om), _p(it))
    return h, om, it, st


def primitives(cfg, m, px, py, pz, E, U, omega, h=None, acc=None, A=None, ekmax=None,
               want_src=False):
    """rho, vx, vy, vz, p (§2.3.7); acc[n,3] (with h) enters the pressure
    switch through E_grav = m |a| h; with the entropy switch (cfg.entropy),
    A (entropic function) and ekmax (E_kin^max) select the entropy route.
    want_src appends the pressure source per particle (0 total energy,
    1 entropy, 2 internal energy)."""
    arrs = list(map(_f64, (m, px, py, pz, E, U, omega)))
    n = arrs[0].size
    out = [np.zeros(n) for _ in range(5)]
    hh = None if h is None else _f64(h)
    aa = None if acc is None else _f64(acc).reshape(n, 3)
    AA = None if A is None else _f64(A)
    ek = None if ekmax is None else _f64(ekmax)
    src = np.zeros(n, dtype=np.int32) if want_src else None
    lib().orc_primitives(C.byref(cfg), n, *[_p(a) for a in arrs], _p(hh), _p(aa), _p(AA), _p(ek),
                         _p(src), *[_p(o) for o in out])
    return tuple(out) + ((src,) if want_src else ())  # rho, vx, vy, vz, p[, src]


def ekin_max(x, y, z, L, h, m, px, py, pz):
    """max_j (1/2) m_i |v_j - v_i|^2 over j != i with r_ij < h_i (§2.3.7)."""
    arrs = list(map(_f64, (x, y, z, L, h, m, px, py, pz)))
    out = np.zeros(arrs[0].size)
    lib().orc_ekin_max(arrs[0].size, *[_p(a) for a in arrs], _p(out))
    return out


def matrices(cfg, x, y, z, L, h, omega):
    """(B6, E6, ncond) per Eqs. 11, 19; 6 unique entries xx, xy, xz, yy, yz, zz."""
    x, y, z, L, h, omega = map(_f64, (x, y, z, L, h, omega))
    n = x.size
    B6 = np.zeros((n, 6))
    E6 = np.zeros((n, 6))
    nc = np.zeros(n)
    lib().orc_matrices(C.byref(cfg), n, _p(x), _p(y), _p(z), _p(L), _p(h), _p(omega), _p(B6),
                       _p(E6), _p(nc))
    return B6, E6, nc


def gradients(cfg, x, y, z, L, h, omega, prims, B6, ncond):
    """(grad[n,5,3], alpha[n,5], vsig[n]) per Eq. 10 and the limiter of §2.3.6."""
    x, y, z, L, h, omega, B6, ncond = map(_f64, (x, y, z, L, h, omega, B6, ncond))
    rho, vx, vy, vz, p = map(_f64, prims)
    n = x.size
    grad = np.zeros((n, 5, 3))
    alpha = np.zeros((n, 5))
    vsig = np.zeros(n)
    lib().orc_gradients(C.byref(cfg), n, _p(x), _p(y), _p(z), _p(L), _p(h), _p(omega),
                        _p(rho), _p(vx), _p(vy), _p(vz), _p(p), _p(B6), _p(ncond), _p(grad),
                        _p(alpha), _p(vsig))
    return grad, alpha, vsig


def flux_pairs(x, y, z, L, h):
    x, y, z, L, h = map(_f64, (x, y, z, L, h))
    n = x.size
    np_ = lib().orc_flux_pairs(n, _p(x), _p(y), _p(z), _p(L), _p(h), 0, None)
    pairs = np.zeros((max(np_, 1), 2), dtype=np.int64)
    np2 = lib().orc_flux_pairs(n, _p(x), _p(y), _p(z), _p(L), _p(h), np_, _p(pairs))
    assert np2 == np_
    return pairs[:np_]


def fluxes(cfg, x, y, z, L, h, omega, B6, prims, grad, alpha, dt, pairs=None,
           pair_guess=None, want_faces=False, want_abs=False, want_dM=False, A=None):
    """dQ[n,6] = (dm, dpx, dpy, dpz, dE, dU) of Eqs. 16 and 24; (dQ, stats, faces)
    or, with want_abs, (dQ, stats, faces, dQabs[n,5] = sum over faces of |c|);
    with want_dM then dM[n,3] = sum_j dm_ij r_ij (§2.3.8); with A (entropic
    function) last dS[n], the upwind entropy the mass fluxes carry (§2.3.7)."""
    x, y, z, L, h, omega, B6 = map(_f64, (x, y, z, L, h, omega, B6))
    grad, alpha = _f64(grad), _f64(alpha)
    rho, vx, vy, vz, p = map(_f64, prims)
    if pairs is None:
        pairs = flux_pairs(x, y, z, L, h)
    pairs = np.ascontiguousarray(pairs, dtype=np.int64)
    n = x.size
    npairs = pairs.shape[0]
    dQ = np.zeros((n, 6))
    st = FluxStats()
    faces = np.zeros((npairs, 9)) if want_faces else None
    pg = None if pair_guess is None else _f64(pair_guess)
    dQabs = np.zeros((n, 5)) if want_abs else None
    dM = np.zeros((n, 3)) if want_dM else None
    AA = None if A is None else _f64(A)
    dS = np.zeros(n) if A is not None else None
    lib().orc_fluxes(C.byref(cfg), n, _p(x), _p(y), _p(z), _p(L), _p(h), _p(omega), _p(B6),
                     _p(rho), _p(vx), _p(vy), _p(vz), _p(p), _p(grad), _p(alpha), float(dt),
                     npairs, _p(pairs), _p(pg), _p(dQ), C.byref(st), _p(faces), _p(dQabs),
                     _p(dM), _p(AA), _p(dS))
    out = (dQ, st.as_dict(), faces) + ((dQabs,) if want_abs else ()) + ((dM,) if want_dM else ())
    return out + ((dS,) if A is not None else ())


def fluxes_rung(cfg, x, y, z, L, h, omega, B6, prims, grad, alpha, dtp, toff, pairs):
    """The face arithmetic of an individual-timestep sub-step (§2.3.4): the
    face (i, j) exchanges over dt_ij = min(dtp_i, dtp_j) and predicts each
    side over toff + dt_ij / 2.  Returns (dQ[n,6], stats, faces[npairs,9]) as
    fluxes(..., want_faces=True)."""
    x, y, z, L, h, omega, B6 = map(_f64, (x, y, z, L, h, omega, B6))
    grad, alpha, dtp, toff = map(_f64, (grad, alpha, dtp, toff))
    rho, vx, vy, vz, p = map(_f64, prims)
    pairs = np.ascontiguousarray(pairs, dtype=np.int64)
    n = x.size
    dQ = np.zeros((n, 6))
    st = FluxStats()
    faces = np.zeros((pairs.shape[0], 9))
    lib().orc_fluxes_rung(C.byref(cfg), n, _p(x), _p(y), _p(z), _p(L), _p(h), _p(omega),
                          _p(B6), _p(rho), _p(vx), _p(vy), _p(vz), _p(p), _p(grad), _p(alpha),
                          _p(dtp), _p(toff), pairs.shape[0], _p(pairs), _p(dQ), C.byref(st),
                          _p(faces))
    return dQ, st.as_dict(), faces


OP_KEYS = ("add", "mul", "div", "sqrt", "pow", "cmp", "fabs", "faces", "newton_iters")


def count_face_ops(cfg, x, y, z, L, h, omega, B6, prims, grad, alpha, dt, pairs):
    """Operations of the oracle's per-face arithmetic over the given pairs
    (flopcount.cpp: the oracle compiled with a counting scalar type), as a
    dict of OP_KEYS totals.  Single-threaded."""
    global _cnt
    if _cnt is None:
        build()
        _cnt = C.CDLL(_CNT_LIB)
        _cnt.orc_count_faces.restype = None
        _cnt.orc_count_faces.argtypes = [C.POINTER(Config), C.c_int64] + [C.c_void_p] * 14 + [
            C.c_double, C.c_int64, C.c_void_p, C.c_void_p]
    x, y, z, L, h, omega, B6 = map(_f64, (x, y, z, L, h, omega, B6))
    grad, alpha = _f64(grad), _f64(alpha)
    rho, vx, vy, vz, p = map(_f64, prims)
    pairs = np.ascontiguousarray(pairs, dtype=np.int64)
    out = np.zeros(9, dtype=np.int64)
    _cnt.orc_count_faces(C.byref(cfg), x.size, _p(x), _p(y), _p(z), _p(L), _p(h), _p(omega),
                         _p(B6), _p(rho), _p(vx), _p(vy), _p(vz), _p(p), _p(grad), _p(alpha),
                         float(dt), pairs.shape[0], _p(pairs), _p(out))
    return {k: int(v) for k, v in zip(OP_KEYS, out)}


def riemann_guess(rl, ul, pl, rr, ur, pr, g):
    return lib().orc_riemann_guess(rl, ul, pl, rr, ur, pr, g)


def riemann_star(rl, ul, pl, rr, ur, pr, g, p0=-1.0, tol=1e-12, max_newton=100):
    ps, us = C.c_double(), C.c_double()
    it, bis = C.c_int(), C.c_int()
    vac = lib().orc_riemann_star(rl, ul, pl, rr, ur, pr, g, p0, tol, max_newton,
                                 C.byref(ps), C.byref(us), C.byref(it), C.byref(bis))
    return dict(p=ps.value, u=us.value, iters=it.value, bisect=bis.value, vacuum=vac)


def riemann_sample(rl, ul, pl, rr, ur, pr, g, ps, us):
    r, u, p = C.c_double(), C.c_double(), C.c_double()
    side = C.c_int()
    lib().orc_riemann_sample(rl, ul, pl, rr, ur, pr, g, ps, us, C.byref(r), C.byref(u),
                             C.byref(p), C.byref(side))
    return r.value, u.value, p.value, side.value


def hllc(rl, ul, pl, wl, rr, ur, pr, wr, nhat, g):
    wl, wr, nhat = _f64(wl), _f64(wr), _f64(nhat)
    F = np.zeros(5)
    ps, ss = C.c_double(), C.c_double()
    lib().orc_hllc(rl, ul, pl, _p(wl), rr, ur, pr, _p(wr), _p(nhat), g, _p(F), C.byref(ps),
                   C.byref(ss))
    return F, ps.value, ss.value


def pair_limit(e, a, b, psi1=0.5, psi2=0.25, positive=False):
    return lib().orc_pair_limit(e, a, b, psi1, psi2, int(bool(positive)))


def step(cfg, state, dt=-1.0, acc=None):
    """One full step on a copy of ``state`` (workload dict).  Returns
    (new_state, outputs, info) where outputs has B6, grad, alpha, ncond, dQ.
    acc[n,3]: an external acceleration held over the step (§2.3.8).  With
    cfg.entropy the entropic function state["A"] (entries <= 0 unset) is
    evolved and returned in new_state["A"] (§2.3.7)."""
    s = {k: _f64(state[k]).copy() for k in ("x", "y", "z", "m", "px", "py", "pz", "E", "U", "h")}
    L = _f64(state["L"])
    n = s["x"].size
    s["omega"] = np.zeros(n)
    if cfg.entropy:
        s["A"] = _f64(state["A"]).copy() if "A" in state else np.zeros(n)
    out = dict(B6=np.zeros((n, 6)), grad=np.zeros((n, 5, 3)), alpha=np.zeros((n, 5)),
               ncond=np.zeros(n), dQ=np.zeros((n, 6)))
    info = StepInfo()
    st = lib().orc_step(C.byref(cfg), n, _p(s["x"]), _p(s["y"]), _p(s["z"]), _p(L), _p(s["m"]),
                        _p(s["px"]), _p(s["py"]), _p(s["pz"]), _p(s["E"]), _p(s["U"]),
                        _p(s["h"]), _p(s["omega"]),
                        _p(None if acc is None else _f64(acc).reshape(n, 3)),
                        _p(s["A"] if cfg.entropy else None), float(dt),
                        _p(out["B6"]), _p(out["grad"]),
                        _p(out["alpha"]), _p(out["ncond"]), _p(out["dQ"]), C.byref(info))
    inf = dict(status=st, dt=info.dt, dt_next=info.dt_next, ngb_rounds=info.ngb_rounds,
               ncond_fail=info.ncond_fail, grad_pairs=info.grad_pairs, flux=info.flux.as_dict())
    s["L"] = L
    s["gamma"] = state.get("gamma", cfg.gamma)
    return s, out, inf


def rung_select(dt_cfl, dt_acc, dt0, max_rung=12):
    """Rung of one particle (§2.3.10): (r, capped)."""
    cap = C.c_int32(0)
    r = lib().orc_rung_select(float(dt_cfl), float(dt_acc), float(dt0), int(max_rung),
                              C.byref(cap))
    return r, bool(cap.value)


def rung_limit(pairs, rung):
    """Neighbour limiter |r_i - r_j| <= 2 over the pairs [k, 2] (§2.3.10);
    returns (rungs, sweeps)."""
    pr = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
    r = np.ascontiguousarray(rung, dtype=np.int32).copy()
    sweeps = lib().orc_rung_limit(pr.shape[0], _p(pr), _p(r))
    return r, sweeps


def step_rungs(cfg, state, dt0, c_acc=0.2, max_rung=12):
    """One base step dt0 with individual timesteps (§2.3.4, §2.3.10) on a
    copy of ``state``.  Returns (new_state, rung, info); info["dt_cfl"],
    info["dt_acc"]: the two timestep criteria of every particle at the start."""
    s = {k: _f64(state[k]).copy() for k in ("x", "y", "z", "m", "px", "py", "pz", "E", "U", "h")}
    L = _f64(state["L"])
    n = s["x"].size
    s["omega"] = np.zeros(n)
    rung = np.zeros(n, dtype=np.int32)
    dtc, dta = np.zeros(n), np.zeros(n)
    info = RungInfo()
    st = lib().orc_step_rungs(C.byref(cfg), n, _p(s["x"]), _p(s["y"]), _p(s["z"]), _p(L),
                              _p(s["m"]), _p(s["px"]), _p(s["py"]), _p(s["pz"]), _p(s["E"]),
                              _p(s["U"]), _p(s["h"]), _p(s["omega"]), float(dt0), float(c_acc),
                              int(max_rung), _p(rung), _p(dtc), _p(dta), C.byref(info))
    inf = {k: getattr(info, k) for k, _ in RungInfo._fields_}
    inf["dt_cfl"], inf["dt_acc"] = dtc, dta
    inf["status"] = st
    s["L"] = L
    s["gamma"] = state.get("gamma", cfg.gamma)
    return s, rung, inf
