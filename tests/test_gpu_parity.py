"""GPU parity: the CUDA library, called through its C ABI, against the FP64
oracle on the same seeded inputs.  FP64 results within 1e-12 (normalised
as in parity_util.compare), neighbour lists bit-exact, the mixed-precision
path within 1e-5, global conservation within 1e-12."""
import math

import numpy as np
import pytest

from paper_2211_12243_gb300 import workloads as W

from parity_util import (compare, compare_masked as _compare_masked, conservation, flux_scale,
                         gpu_stages, oracle_stages)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hyd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_12243_gb300 import build, hydro
    build.build()
    return hydro


def _moving(w, seed=3, amp=0.2):
    rng = np.random.default_rng(seed)
    n = w["x"].size
    v = rng.normal(0, amp, (n, 3))
    w = dict(w)
    w["px"], w["py"], w["pz"] = w["m"] * v[:, 0], w["m"] * v[:, 1], w["m"] * v[:, 2]
    w["E"] = w["U"] + 0.5 * w["m"] * np.sum(v * v, 1)
    return w


CASES = {
    # name: (workload factory, oracle/GPU options)
    "wave_hllc": (lambda: W.lattice_wave(12), dict(riemann="hllc")),
    "wave_moving_exact": (lambda: _moving(W.lattice_wave(10, jitter=0.05)), dict()),
    "sod_exact": (lambda: W.sod(8), dict()),
    "sod_mfm": (lambda: W.sod(8), dict(scheme="mfm")),
    "lognormal_exact": (lambda: W.lognormal(4096, seed=2, grid=16), dict(search=2.5)),
    "sedov_exact": (lambda: W.sedov(12), dict()),
    # the paper's cubic-spline kernel (§2.3.2; the configs use Wendland C2)
    "wave_moving_cubic": (lambda: _moving(W.lattice_wave(10, jitter=0.05)), dict(kernel="cubic")),
    "sod_cubic": (lambda: W.sod(8), dict(kernel="cubic")),
    "sod_cubic_mfm": (lambda: W.sod(8), dict(kernel="cubic", scheme="mfm")),
}


def _cfgs(orc, hyd, w, opts, precision="fp64"):
    opts = {k: v for k, v in opts.items() if k != "search"}
    co = orc.config(gamma=w["gamma"], **opts)
    cg = hyd.default_config(gamma=w["gamma"], precision=precision, **opts)
    return co, cg


@pytest.mark.parametrize("name", ["wave_hllc", "sod_exact", "lognormal_exact", "sedov_exact"])
def test_neighbour_lists_bit_exact(orc, hyd, name):
    w = CASES[name][0]()
    import torch
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"]))
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    hs = w["h"] * 1.37
    off, idx = H.build_neighbours(st, torch.as_tensor(hs, device="cuda"))
    off_o, idx_o = orc.neighbours(w["x"], w["y"], w["z"], w["L"], hs)
    assert np.array_equal(off.cpu().numpy(), off_o)
    assert np.array_equal(idx.cpu().numpy(), idx_o)


@pytest.mark.parametrize("name", list(CASES))
def test_stages_fp64_match_oracle(orc, hyd, name):
    factory, opts = CASES[name]
    w = factory()
    co, cg = _cfgs(orc, hyd, w, opts)
    dt = 1e-3 if "sedov" not in name else 1e-6
    o = oracle_stages(orc, co, w, dt)
    g = gpu_stages(hyd, hyd.Hydro(cg), w, dt, search=opts.get("search", 1.3))
    errs, bad = _compare_masked(orc, w, o, g, 1e-12, ("h", "omega", "B", "grad", "ncond", "dQ"))
    assert not bad, errs


@pytest.mark.parametrize("name", list(CASES))
def test_stages_mixed_match_oracle(orc, hyd, name):
    factory, opts = CASES[name]
    w = factory()
    co, cg = _cfgs(orc, hyd, w, opts, precision="mixed")
    dt = 1e-3 if "sedov" not in name else 1e-6
    o = oracle_stages(orc, co, w, dt)
    g = gpu_stages(hyd, hyd.Hydro(cg), w, dt, search=opts.get("search", 1.3))
    errs, bad = _compare_masked(orc, w, o, g, 1e-5, ("h", "omega", "dQ"))
    assert not bad, errs
    # h refined to double-class accuracy despite the float iteration
    assert errs["h"] < 1e-12, errs


def _step_both(orc, hyd, w, opts, precision, dt):
    import torch
    co, cg = _cfgs(orc, hyd, w, opts, precision)
    so, out_o, info_o = orc.step(co, w, dt)
    info_o["_out"] = out_o
    H = hyd.Hydro(cg)
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    stats = H.step(st, dt)
    torch.cuda.synchronize()
    sg = {k: v.cpu().numpy() for k, v in st.items()}
    return so, info_o, sg, stats


@pytest.mark.parametrize("name", ["wave_moving_exact", "sod_exact", "sod_mfm", "lognormal_exact",
                                  "wave_moving_cubic", "sod_cubic", "sod_cubic_mfm"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_full_step_matches_oracle(orc, hyd, name, precision, tol):
    factory, opts = CASES[name]
    w = factory()
    so, info_o, sg, stats = _step_both(orc, hyd, w, opts, precision, dt=-1.0)
    assert stats["status"] == 0
    # CFL timestep (Eqs. 31-32)
    assert stats["dt"] == pytest.approx(info_o["dt"], rel=tol)
    assert stats["grad_pairs"] == info_o["grad_pairs"]
    assert stats["flux_pairs"] == info_o["flux"]["pairs"]
    for k in ("h", "omega"):
        assert np.max(np.abs(sg[k] - so[k]) / np.abs(so[k])) < tol, k
    # conserved quantities: compare the change, normalised by its scale
    for k in ("m", "px", "py", "pz", "E", "U"):
        d_o = so[k] - w[k]
        d_g = sg[k] - w[k]
        scale = np.abs(d_o).max() + 1e-300
        assert np.max(np.abs(d_g - d_o)) < max(tol, 1e-12) * scale * 10 + 1e-300, k
    # positions moved by dt * mean velocity (periodic wrap)
    L = w["L"]
    for a, k in enumerate(("x", "y", "z")):
        d = sg[k] - so[k]
        d -= np.round(d / L[a]) * L[a]
        assert np.max(np.abs(d)) < tol * np.max(w["h"]) + 1e-15
    cons = conservation(w, sg, w["gamma"])
    assert max(cons.values()) < 1e-12, cons
    # per-particle flux error, normalised by the particle's sum of |c| over
    # its faces (recomputed by the oracle from its own step outputs)
    co, _ = _cfgs(orc, hyd, w, opts, precision)
    out_o = info_o["_out"]
    prims = orc.primitives(co, w["m"], w["px"], w["py"], w["pz"], w["E"], w["U"], so["omega"])
    dQ, _, _, dQabs = orc.fluxes(co, w["x"], w["y"], w["z"], w["L"], so["h"], so["omega"],
                                 out_o["B6"], prims, out_o["grad"], out_o["alpha"], info_o["dt"],
                                 want_abs=True)
    assert np.allclose(dQ, out_o["dQ"], rtol=0, atol=1e-300 + 1e-14 * np.abs(dQ).max())
    sc = flux_scale(dict(dQabs=dQabs, prims=prims, gamma=w["gamma"]))
    d_g = np.stack([sg[k] - w[k] for k in ("m", "px", "py", "pz", "E")], 1)
    d_o = np.stack([so[k] - w[k] for k in ("m", "px", "py", "pz", "E")], 1)
    qscale = np.abs(np.stack([w[k] for k in ("m", "px", "py", "pz", "E")], 1)) * 4e-16
    err = np.max(np.abs(d_g - d_o) / (sc + qscale))
    assert err < tol, err


@pytest.mark.parametrize("crit", [4.0, 3.0])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_guard_rounds_match_oracle(orc, hyd, crit, precision, tol):
    """The N_cond guard (§2.3.5) with a low threshold takes all five growth
    rounds (crit 4: every particle passes in the end; crit 3: seven still
    fail, status ENCOND).  A round re-solves the grown particles' densities
    and recomputes only the gradients those change; the step must end where
    the oracle, which recomputes every particle each round, ends."""
    import torch
    w = W.lognormal(4096, seed=2, grid=16)
    co, cg = _cfgs(orc, hyd, w, dict(ncond_crit=crit), precision)
    so, _, info_o = orc.step(co, w, -1.0)
    assert info_o["ngb_rounds"] == 5
    H = hyd.Hydro(cg)
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    stats = H.step(st, -1.0, check=False)
    torch.cuda.synchronize()
    sg = {k: v.cpu().numpy() for k, v in st.items()}
    assert stats["status"] == info_o["status"]
    assert stats["ngb_rounds"] == info_o["ngb_rounds"]
    assert stats["ncond_fail"] == info_o["ncond_fail"]
    assert stats["grad_pairs"] == info_o["grad_pairs"]
    assert stats["flux_pairs"] == info_o["flux"]["pairs"]
    assert stats["dt"] == pytest.approx(info_o["dt"], rel=tol)
    for k in ("h", "omega"):
        assert np.max(np.abs(sg[k] - so[k]) / np.abs(so[k])) < tol, k
    # the mixed path refines every root in double-float arithmetic, the grown
    # particles' (N_NGB = 32 * 1.2^k) included: h to double-class accuracy
    assert np.max(np.abs(sg["h"] - so["h"]) / so["h"]) < 1e-12
    for k in ("m", "px", "py", "pz", "E", "U"):
        d_o = so[k] - w[k]
        d_g = sg[k] - w[k]
        scale = np.abs(d_o).max() + 1e-300
        assert np.max(np.abs(d_g - d_o)) < max(tol, 1e-12) * scale * 10 + 1e-300, k


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("graph", [0, 1])
def test_guard_rounds_2e16_match_oracle(orc, hyd, precision, tol, graph):
    """The default threshold on 2^16 particles of the clustered generator:
    the first growth round grows 249 particles, more than n / 1024, and the
    recomputed particles are marked by a scan of every list; the second
    grows 22 and the third 2, marked by tree walks from them (the counts are
    the oracle's rounds at this seed).  Host-driven and graph steps."""
    import torch
    w = W.lognormal(1 << 16, seed=0)
    co = orc.config(gamma=w["gamma"])
    cg = hyd.default_config(gamma=w["gamma"], precision=precision, graph=graph)
    so, _, info_o = orc.step(co, w, -1.0)
    assert info_o["ngb_rounds"] == 3 and info_o["ncond_fail"] == 0
    H = hyd.Hydro(cg)
    H.set_boxes(*hyd.single_box(w))
    for rep in range(2):            # the context's first step is host-driven, the second a graph
        st = hyd.to_device(w)
        stats = H.step(st, -1.0, check=False)
        torch.cuda.synchronize()
        sg = {k: v.cpu().numpy() for k, v in st.items()}
        assert stats["status"] == info_o["status"]
        assert stats["ngb_rounds"] == 3 and stats["ncond_fail"] == 0
        assert stats["grad_pairs"] == info_o["grad_pairs"]
        assert stats["flux_pairs"] == info_o["flux"]["pairs"]
        for k in ("h", "omega"):
            assert np.max(np.abs(sg[k] - so[k]) / np.abs(so[k])) < tol, k
        for k in ("m", "px", "py", "pz", "E", "U"):
            d_o = so[k] - w[k]
            d_g = sg[k] - w[k]
            scale = np.abs(d_o).max() + 1e-300
            assert np.max(np.abs(d_g - d_o)) < max(tol, 1e-12) * scale * 10 + 1e-300, k
        cons = conservation(w, sg, w["gamma"])
        assert max(cons.values()) < 1e-12, cons


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_conserves_and_reports(hyd, precision):
    import torch
    w = _moving(W.lognormal(20000, seed=4, grid=32), amp=0.3)
    cg = hyd.default_config(gamma=w["gamma"], precision=precision)
    H = hyd.Hydro(cg)
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    for _ in range(3):
        before = {k: v.cpu().numpy() for k, v in st.items()}
        stats = H.step(st, -1.0)
        assert stats["status"] == 0
        after = {k: v.cpu().numpy() for k, v in st.items()}
        cons = conservation(before, after, w["gamma"])
        assert max(cons.values()) < 1e-12, cons
        assert stats["flux_pairs"] > 0 and stats["grad_pairs"] > 0
    assert np.all(np.isfinite(after["E"]))


def test_mfm_keeps_masses_bitwise(hyd):
    import torch
    w = _moving(W.lattice_wave(10, jitter=0.05))
    for precision in ("fp64", "mixed"):
        H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision=precision, scheme="mfm"))
        H.set_boxes(*hyd.single_box(w))
        st = hyd.to_device(w)
        H.step(st, 1e-3)
        assert np.array_equal(st["m"].cpu().numpy(), w["m"])


def test_batched_boxes_match_single_boxes(orc, hyd):
    """Several independent periodic boxes in one launch give what each box
    gives alone (oracle per box)."""
    import torch
    parts = [W.lattice_wave(8), W.sod(6), W.lognormal(1500, seed=9, grid=16)]
    keys = ["x", "y", "z", "m", "px", "py", "pz", "E", "U", "h"]
    w = {k: np.concatenate([p[k] for p in parts]) for k in keys}
    counts = [p["x"].size for p in parts]
    box_off = np.concatenate([[0], np.cumsum(counts)])
    box_len = np.concatenate([p["L"] for p in parts])
    H = hyd.Hydro(hyd.default_config(gamma=5.0 / 3.0))
    H.set_boxes(box_off, box_len)
    st = hyd.to_device(w)
    dt = 1e-3
    stats = H.step(st, dt)
    assert stats["status"] == 0
    sg = {k: v.cpu().numpy() for k, v in st.items()}
    co = orc.config()
    for b, p in enumerate(parts):
        so, _, _ = orc.step(co, p, dt)
        sl = slice(box_off[b], box_off[b + 1])
        for k in ("h", "omega"):
            assert np.max(np.abs(sg[k][sl] - so[k]) / so[k]) < 1e-12
        for k in ("m", "px", "E"):
            d_o = so[k] - p[k]
            d_g = sg[k][sl] - p[k]
            assert np.max(np.abs(d_g - d_o)) <= 1e-10 * (np.abs(d_o).max() + 1e-300), k


def test_degenerate_inputs_report_status(hyd):
    import torch
    H = hyd.Hydro(hyd.default_config())
    # empty boxes are rejected
    with pytest.raises(hyd.HydroError):
        H.set_boxes(np.array([0, 0]), np.array([1.0, 1.0, 1.0]))
    # too few particles for N_NGB = 32 in the box: the h root would exceed
    # the periodic half-box; the step reports it instead of looping
    rng = np.random.default_rng(1)
    n = 8
    w = dict(x=rng.random(n), y=rng.random(n), z=rng.random(n), m=np.full(n, 1.0 / n),
             px=np.zeros(n), py=np.zeros(n), pz=np.zeros(n), E=np.full(n, 1.0),
             U=np.full(n, 1.0), h=np.full(n, 0.3), L=np.array([1.0, 1.0, 1.0]))
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    rc = H.step(st, 1e-3, stats=False, check=False)
    assert rc == -10  # HYDRO_ESEARCH
    # bad config
    with pytest.raises(hyd.HydroError):
        hyd.Hydro(hyd.default_config(gamma=0.5))


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_gravity_step_matches_oracle(orc, hyd, scheme, precision, tol):
    """hydro_set_gravity (§2.3.8): a random acceleration field on a Sod tube;
    the host-driven and the graph step end where the oracle's step ends."""
    import torch
    w = W.sod(8)
    n = w["x"].size
    acc = np.random.default_rng(3).normal(0.0, 0.5, (n, 3))
    co = orc.config(gamma=w["gamma"], scheme=scheme)
    so, _, info_o = orc.step(co, w, -1.0, acc=acc)
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision=precision, scheme=scheme))
    H.set_boxes(*hyd.single_box(w))
    acc_d = torch.as_tensor(acc, device="cuda").contiguous()
    H.set_gravity(acc_d)
    st = hyd.to_device(w)
    init = {k: v.clone() for k, v in st.items()}
    for graph in (0, 1):
        for k, v in init.items():
            st[k].copy_(v)
        stats = H.step(st, -1.0)
        torch.cuda.synchronize()
        assert stats["status"] == 0 and stats["graph"] == graph, stats
        assert stats["dt"] == pytest.approx(info_o["dt"], rel=tol)
        sg = {k: v.cpu().numpy() for k, v in st.items()}
        for k in ("h", "omega"):
            assert np.max(np.abs(sg[k] - so[k]) / np.abs(so[k])) < tol, (graph, k)
        for k in ("m", "px", "py", "pz", "E", "U"):
            d_o = so[k] - w[k]
            d_g = sg[k] - w[k]
            scale = np.abs(d_o).max() + 1e-300
            assert np.max(np.abs(d_g - d_o)) < max(tol, 1e-12) * scale * 10 + 1e-300, (graph, k)
        # the step's totals are those of the state before and after it: their
        # change is the external impulse and work (the fluxes conserve)
        for q, (key, k) in enumerate((("mass", "m"), ("mom", "px"), ("mom", "py"),
                                      ("mom", "pz"), ("energy", "E"))):
            before = stats[key][0] if key != "mom" else stats[key][0][q - 1]
            after = stats[key][1] if key != "mom" else stats[key][1][q - 1]
            assert before == pytest.approx(math.fsum(w[k]), rel=1e-13, abs=1e-15), (graph, k)
            assert after == pytest.approx(math.fsum(sg[k]), rel=1e-13, abs=1e-15), (graph, k)
            ch_o = math.fsum(so[k]) - math.fsum(w[k])
            if k != "m":
                assert abs(ch_o) > 1e-6 * math.fsum(np.abs(w[k])) + 1e-12   # the source acted
            tot = math.fsum(np.abs(w[k])) + math.fsum(np.abs(w["m"]))
            assert abs((after - before) - ch_o) < 10 * max(tol, 1e-12) * tot, (graph, k)
    H.set_gravity(None)


def _entropy_mix(n=10, seed=5):
    """Cold streams colliding along x (|v| = 2, U/m = 2.5e-3) with a hot
    slab (U/m = 2.5, z < 0.3) and a little transverse noise: the hot slab
    takes the total-energy route, stream particles near the two interfaces
    the entropy route (E_kin^max ~ 8 m >> U / alpha2) where A > 0, the
    interiors the internal-energy route (§2.3.7).  A: random, a fifth unset
    (zero)."""
    rng = np.random.default_rng(seed)
    w = dict(W.lattice_wave(n, jitter=0.0))
    N = w["x"].size
    m = np.full(N, 1.0 / n ** 3)
    vx = np.where(w["x"] < 0.5, 2.0, -2.0)
    vy = rng.normal(0.0, 1e-3, N)
    w["m"] = m
    w["px"], w["py"], w["pz"] = m * vx, m * vy, 0.0 * m
    u = np.where(w["z"] < 0.3, 2.5, 2.5e-3)
    w["U"] = m * u
    w["E"] = w["U"] + 0.5 * m * (vx * vx + vy * vy)
    w["A"] = np.where(rng.random(N) < 0.2, 0.0, rng.uniform(5e-3, 2e-2, N))
    return w


@pytest.mark.parametrize("scheme", ["mfv", "mfm"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_entropy_switch_step_matches_oracle(orc, hyd, scheme, precision, tol):
    """hydro_set_entropy with cfg.entropy_switch (§2.3.7): the pressure
    routes, the re-set of A where the energies gave the pressure, the MFV
    entropy flux and the MFM constant A; the host-driven and the graph step
    end where the oracle's step ends."""
    import torch
    w = _entropy_mix()
    co = orc.config(gamma=w["gamma"], scheme=scheme, entropy=True)
    so, _, info_o = orc.step(co, w, -1.0)
    assert info_o["status"] == 0
    # every route is taken
    ek = orc.ekin_max(w["x"], w["y"], w["z"], w["L"], so["h"], w["m"], w["px"], w["py"], w["pz"])
    _, _, _, _, _, src = orc.primitives(co, w["m"], w["px"], w["py"], w["pz"], w["E"], w["U"],
                                        so["omega"], h=so["h"], A=w["A"], ekmax=ek, want_src=True)
    assert all((src == r).sum() > 0 for r in (0, 1, 2)), np.bincount(src)
    cg = hyd.default_config(gamma=w["gamma"], precision=precision, scheme=scheme,
                            entropy_switch=1)
    H = hyd.Hydro(cg)
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    with pytest.raises(hyd.HydroError):
        H.step(st, -1.0)             # the switch is on and no A is held
    init = {k: v.clone() for k, v in st.items()}
    A0 = torch.as_tensor(w["A"], device="cuda").clone()
    A = A0.clone()
    H.set_entropy(A)
    for graph in (0, 1):
        for k, v in init.items():
            st[k].copy_(v)
        A.copy_(A0)
        stats = H.step(st, -1.0)
        torch.cuda.synchronize()
        assert stats["status"] == 0 and stats["graph"] == graph, stats
        assert stats["dt"] == pytest.approx(info_o["dt"], rel=tol)
        sg = {k: v.cpu().numpy() for k, v in st.items()}
        for k in ("h", "omega"):
            assert np.max(np.abs(sg[k] - so[k]) / np.abs(so[k])) < tol, (graph, k)
        for k in ("m", "px", "py", "pz", "E", "U"):
            d_o = so[k] - w[k]
            d_g = sg[k] - w[k]
            scale = np.abs(d_o).max() + 1e-300
            assert np.max(np.abs(d_g - d_o)) < max(tol, 1e-12) * scale * 10 + 1e-300, (graph, k)
        Ag = A.cpu().numpy()
        assert np.all(Ag > 0)
        assert np.max(np.abs(Ag - so["A"]) / so["A"]) < tol * 10, (graph, scheme)
    H.set_entropy(None)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_entropy_switch_with_guard_rounds(orc, hyd, precision, tol):
    """The entropy route of re-solved particles in the N_cond guard rounds
    (§2.3.5, §2.3.7): a log-normal box with a low threshold (all five growth
    rounds) and cold random velocities, the switch on, A set for most
    particles; the step ends where the oracle's ends."""
    import torch
    w = dict(W.lognormal(4096, seed=2, grid=16))
    n = w["x"].size
    rng = np.random.default_rng(9)
    v = rng.normal(0.0, 3.0, (n, 3))
    w["px"], w["py"], w["pz"] = w["m"] * v[:, 0], w["m"] * v[:, 1], w["m"] * v[:, 2]
    w["U"] = 1e-4 * w["U"]
    w["E"] = w["U"] + 0.5 * w["m"] * np.sum(v * v, 1)
    w["A"] = np.where(rng.random(n) < 0.1, 0.0, rng.uniform(0.5, 2.0, n))
    co = orc.config(gamma=w["gamma"], ncond_crit=4.0, entropy=True)
    so, _, info_o = orc.step(co, w, 1e-4)
    assert info_o["ngb_rounds"] == 5 and info_o["status"] == 0
    ek = orc.ekin_max(w["x"], w["y"], w["z"], w["L"], so["h"], w["m"], w["px"], w["py"], w["pz"])
    _, _, _, _, _, src = orc.primitives(co, w["m"], w["px"], w["py"], w["pz"], w["E"], w["U"],
                                        so["omega"], h=so["h"], A=w["A"], ekmax=ek, want_src=True)
    assert (src == 1).sum() > n // 2 and (src == 2).sum() > 0, np.bincount(src)
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision=precision, ncond_crit=4.0,
                                     entropy_switch=1))
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    A = torch.as_tensor(w["A"], device="cuda").clone()
    H.set_entropy(A)
    stats = H.step(st, 1e-4, check=False)
    torch.cuda.synchronize()
    assert stats["status"] == 0 and stats["ngb_rounds"] == 5, stats
    sg = {k: v.cpu().numpy() for k, v in st.items()}
    for k in ("h", "omega"):
        assert np.max(np.abs(sg[k] - so[k]) / np.abs(so[k])) < tol, k
    for k in ("m", "px", "py", "pz", "E", "U"):
        d_o = so[k] - w[k]
        d_g = sg[k] - w[k]
        scale = np.abs(d_o).max() + 1e-300
        assert np.max(np.abs(d_g - d_o)) < max(tol, 1e-12) * scale * 10 + 1e-300, k
    Ag = A.cpu().numpy()
    assert np.max(np.abs(Ag - so["A"]) / so["A"]) < tol * 10
