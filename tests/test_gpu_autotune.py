"""hydro_autotune: the launch-parameter candidates (list radius factor, fixed
list slots, register bounds of the gradient and flux kernels) are timed on
the caller's particles, which stay untouched; every variant computes the
same step (FP64 oracle within the parity tolerances)."""
import numpy as np
import pytest

from paper_2211_12243_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hyd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_12243_gb300 import build, hydro
    build.build()
    return hydro


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_autotune_chooses_and_leaves_the_state(hyd, precision):
    import torch
    w = W.sod(12)
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision=precision))
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    before = {k: v.cpu().numpy().copy() for k, v in st.items()}
    t = H.autotune(st)
    torch.cuda.synchronize()
    for k, v in st.items():
        assert np.array_equal(v.cpu().numpy(), before[k]), k
    assert t["search_margin"] in (1.05, 1.1, 1.15, 1.25)
    assert t["nbr_slots"] in (64, 96, 128)
    assert t["grad_min_ctas"] in (1, 4, 5, 6)
    assert t["flux_min_ctas"] in (4, 5, 6)
    assert min(min(r) for r in t["front_ms"]) > 0 and min(t["grad_ms"]) > 0
    if precision == "mixed":
        assert min(t["flux_ms"]) > 0
    # the chosen front is the fastest measured
    i = (1.05, 1.1, 1.15, 1.25).index(t["search_margin"])
    j = (64, 96, 128).index(t["nbr_slots"])
    assert t["front_ms"][i][j] == min(min(r) for r in t["front_ms"])
    s = H.step(st, 1e-3)
    assert s["status"] == 0
    with pytest.raises(hyd.HydroError):
        H.set_tuning(dict(t, flux_min_ctas=7))
    with pytest.raises(hyd.HydroError):
        H.set_tuning(dict(t, nbr_slots=8))


@pytest.mark.parametrize("variant", [
    dict(search_margin=1.05, nbr_slots=64, grad_min_ctas=5, flux_min_ctas=5),
    dict(search_margin=1.25, nbr_slots=128, grad_min_ctas=6, flux_min_ctas=6),
    dict(search_margin=1.1, nbr_slots=96, grad_min_ctas=1, flux_min_ctas=4),
    dict(search_margin=1.05, nbr_slots=128, grad_min_ctas=4, flux_min_ctas=4, grad_rank=2),
])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("name", ["sod_exact", "lognormal_hllc", "lognormal_exact"])
def test_every_variant_computes_the_same_step(orc, hyd, variant, precision, tol, name):
    import torch
    if name == "sod_exact":
        w, opts = W.sod(8), {}
    elif name == "lognormal_exact":
        w, opts = W.lognormal(4096, seed=2, grid=16), {}
    else:
        w, opts = W.lognormal(4096, seed=2, grid=16), dict(riemann="hllc")
    co = orc.config(gamma=w["gamma"], **opts)
    so, _, info_o = orc.step(co, w, -1.0)
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision=precision, **opts))
    H.set_tuning(variant)
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    for step in range(2):        # a host-driven step, then a graph step
        if step:
            for k in ("x", "y", "z", "m", "px", "py", "pz", "E", "U", "h"):
                st[k].copy_(torch.as_tensor(w[k], device="cuda"))
        s = H.step(st, -1.0)
        torch.cuda.synchronize()
        assert s["status"] == info_o["status"]
        assert s["grad_pairs"] == info_o["grad_pairs"]
        assert s["flux_pairs"] == info_o["flux"]["pairs"]
        sg = {k: v.cpu().numpy() for k, v in st.items()}
        for k in ("h", "omega"):
            assert np.max(np.abs(sg[k] - so[k]) / np.abs(so[k])) < tol, (step, k)
        for k in ("m", "px", "py", "pz", "E", "U"):
            d_o = so[k] - w[k]
            d_g = sg[k] - w[k]
            scale = np.abs(d_o).max() + 1e-300
            assert np.max(np.abs(d_g - d_o)) < max(tol, 1e-12) * scale * 10 + 1e-300, (step, k)


def test_ranked_tiles_reproduce_the_unranked_stages(hyd):
    """The density and gradient kernels rank tiles of 128 consecutive
    particles by list length (the gradient kernel also tiles of 128 R, R = 8
    at 2^21 particles); each particle is still computed by one thread in one
    order, so h, omega, B, the limited gradients and N_cond equal the
    unranked kernels' bit for bit."""
    import torch
    w = W.lognormal(1 << 21, seed=3)
    # converged smoothing lengths to start from (one short step solves them,
    # with the re-searches the staged density call does not make)
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision="mixed"))
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    s = H.step(st, 1e-9, check=False)
    assert s["status"] in (0, -5)   # (HYDRO_ENCOND: a few stay ill-conditioned)
    torch.cuda.synchronize()
    w = dict(w, **{k: st[k].cpu().numpy() for k in st})
    H.close()
    out = []
    for rank in (0, 1, 2):
        H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision="mixed"))
        H.set_tuning(dict(search_margin=1.1, nbr_slots=128, grad_min_ctas=1, flux_min_ctas=4,
                          grad_rank=rank))
        H.set_boxes(*hyd.single_box(w))
        st = hyd.to_device(w)
        H.build_neighbours(st, st["h"] * 1.3, export=False)
        H.density(st)
        B, G, A, N = H.gradients(st)
        torch.cuda.synchronize()
        c = lambda t: t.detach().cpu().numpy()
        out.append(dict(h=c(st["h"]), omega=c(st["omega"]), B=c(B), G=c(G), A=c(A), N=c(N)))
        H.close()
    for r in (1, 2):
        for k in out[0]:
            assert np.array_equal(out[0][k], out[r][k], equal_nan=True), (r, k)
