"""The step as one captured CUDA graph (hydro_config.graph = 1, the default):
its re-search and N_cond loops run as device-side WHILE nodes.  A graph
step must end where the host-driven step (graph = 0) and the FP64 oracle
end, including steps that take re-search rounds and every N_cond growth
round (§2.3.5)."""
import numpy as np
import pytest

from paper_2211_12243_gb300 import workloads as W

from parity_util import conservation

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "z", "m", "px", "py", "pz", "E", "U", "h")


@pytest.fixture(scope="module")
def hyd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_12243_gb300 import build, hydro
    build.build()
    return hydro


def _batch():
    parts = [W.lattice_wave(8), W.sod(6), W.lognormal(1500, seed=9, grid=16)]
    w = {k: np.concatenate([p[k] for p in parts]) for k in KEYS}
    counts = [p["x"].size for p in parts]
    w["box_off"] = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    w["box_len"] = np.concatenate([p["L"] for p in parts])
    w["gamma"] = 5.0 / 3.0
    return w


CASES = {
    "sod": (lambda: W.sod(8), {}),
    "wave_hllc": (lambda: W.lattice_wave(10, jitter=0.05), dict(riemann="hllc")),
    # N_cond threshold 4: five growth rounds in every step
    "lognormal_guard": (lambda: W.lognormal(4096, seed=2, grid=16), dict(ncond_crit=4.0)),
    "batch": (_batch, {}),
}


def _boxes(hyd, w):
    if "box_off" in w:
        return w["box_off"], w["box_len"]
    return hyd.single_box(w)


def _run(hyd, w, cfg, nstep, restart, dt):
    """nstep steps; restart: every step from the initial state (rough h, so
    every step re-searches)."""
    import torch
    H = hyd.Hydro(cfg)
    H.set_boxes(*_boxes(hyd, w))
    st = hyd.to_device(w)
    init = {k: v.clone() for k, v in st.items()}
    out = []
    for _ in range(nstep):
        if restart:  # (same tensors: the graph's pointers stay valid)
            for k, v in init.items():
                st[k].copy_(v)
        s = H.step(st, dt, check=False)
        torch.cuda.synchronize()
        out.append((s, {k: v.cpu().numpy() for k, v in st.items()}))
    H.close()
    return out


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("restart", [False, True])
def test_graph_steps_match_host_steps(hyd, name, precision, tol, restart):
    factory, opts = CASES[name]
    w = factory()
    dt = -1.0 if name != "batch" else 1e-4
    runs = {}
    for graph in (1, 0):
        cfg = hyd.default_config(gamma=w["gamma"], precision=precision, graph=graph, **opts)
        runs[graph] = _run(hyd, w, cfg, 6, restart, dt)
    how = [s["graph"] for s, _ in runs[1]]
    # graph steps from the second on; a step may hand over to the host path
    # to grow a buffer (2: the overflow region of the lists, which the guard
    # rounds' rebuilt lists fill, or the fixed list slots), after which the
    # graph runs again
    assert how[0] == 0 and how[-1] == 1 and all(g in (1, 2) for g in how[1:]), how
    assert how.count(2) <= 2, how
    for k, ((sg, xg), (sh, xh)) in enumerate(zip(runs[1], runs[0])):
        assert sh["graph"] == 0
        for key in ("status", "grad_pairs", "flux_pairs", "ngb_rounds", "ncond_fail",
                    "list_rebuilds"):
            assert sg[key] == sh[key], (k, key, sg[key], sh[key])
        assert sg["dt"] == pytest.approx(sh["dt"], rel=tol)
        for key in ("h", "omega"):
            assert np.max(np.abs(xg[key] - xh[key]) / np.abs(xh[key])) < tol, (k, key)
        ref_h = runs[0][k - 1][1] if (k > 0 and not restart) else w
        ref_g = runs[1][k - 1][1] if (k > 0 and not restart) else w
        for key in ("m", "px", "py", "pz", "E", "U"):
            d_h = xh[key] - ref_h[key]
            d_g = xg[key] - ref_g[key]
            scale = np.abs(d_h).max() + 1e-300
            assert np.max(np.abs(d_g - d_h)) <= 10 * tol * scale + 1e-300, (k, key)
    if restart and name == "lognormal_guard":
        # the rough initial h of this box takes re-search rounds on the device
        assert runs[1][-1][0]["list_rebuilds"] > 0
    if name == "lognormal_guard":
        assert runs[1][-1][0]["ngb_rounds"] == 5


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_graph_step_matches_oracle(orc, hyd, precision, tol):
    """A graph step (the second step of the context) from the initial state
    of a log-normal box, with re-search rounds and all five N_cond growth
    rounds on the device, against the oracle's step."""
    import torch
    w = W.lognormal(4096, seed=2, grid=16)
    co = orc.config(gamma=w["gamma"], ncond_crit=4.0)
    so, _, info_o = orc.step(co, w, -1.0)
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision=precision, ncond_crit=4.0))
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    init = {k: v.clone() for k, v in st.items()}
    H.step(st, -1.0, check=False)          # host-driven first step
    for attempt in range(3):
        # graph steps from the same state; the first may hand over to the
        # host path once to grow the overflow region of the lists (graph 2)
        for k, v in init.items():
            st[k].copy_(v)
        stats = H.step(st, -1.0, check=False)
        torch.cuda.synchronize()
        if stats["graph"] == 1:
            break
    assert stats["graph"] == 1
    assert stats["list_rebuilds"] > 0
    sg = {k: v.cpu().numpy() for k, v in st.items()}
    assert stats["status"] == info_o["status"]
    assert stats["ngb_rounds"] == info_o["ngb_rounds"] == 5
    assert stats["ncond_fail"] == info_o["ncond_fail"]
    assert stats["grad_pairs"] == info_o["grad_pairs"]
    assert stats["flux_pairs"] == info_o["flux"]["pairs"]
    assert stats["dt"] == pytest.approx(info_o["dt"], rel=tol)
    for k in ("h", "omega"):
        assert np.max(np.abs(sg[k] - so[k]) / np.abs(so[k])) < tol, k
    for k in ("m", "px", "py", "pz", "E", "U"):
        d_o = so[k] - w[k]
        d_g = sg[k] - w[k]
        scale = np.abs(d_o).max() + 1e-300
        assert np.max(np.abs(d_g - d_o)) < max(tol, 1e-12) * scale * 10 + 1e-300, k
    cons = conservation(w, sg, w["gamma"])
    assert max(cons.values()) < 1e-12, cons


def test_graph_step_that_cannot_finish_leaves_the_state(hyd):
    """Too few particles for N_NGB in the box: every re-search round fails;
    the graph step reports HYDRO_ESEARCH like the host-driven step and leaves
    the caller's state as it was."""
    import torch
    rng = np.random.default_rng(1)
    n = 8
    w = dict(x=rng.random(n), y=rng.random(n), z=rng.random(n), m=np.full(n, 1.0 / n),
             px=np.zeros(n), py=np.zeros(n), pz=np.zeros(n), E=np.full(n, 1.0),
             U=np.full(n, 1.0), h=np.full(n, 0.3), L=np.array([1.0, 1.0, 1.0]))
    ok = W.lattice_wave(6)   # a box that steps, to get past the first (host-driven) step
    H = hyd.Hydro(hyd.default_config())
    H.set_boxes(*hyd.single_box(ok))
    st = hyd.to_device(ok)
    assert H.step(st, 1e-3)["status"] == 0
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    before = {k: v.cpu().numpy().copy() for k, v in st.items()}
    rc = H.step(st, 1e-3, stats=False, check=False)
    torch.cuda.synchronize()
    assert rc == -10  # HYDRO_ESEARCH
    for k, v in st.items():
        assert np.array_equal(v.cpu().numpy(), before[k]), k
