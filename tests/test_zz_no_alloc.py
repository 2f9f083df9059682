"""The allocation-free totals entry point (hydro_totals_noalloc), for callers
that cannot call cudaMalloc (a host application that owns every device
allocation through its own pool, or a plugin that must keep the device
memory footprint fixed).  Its output must agree with the totals the regular
hydro_step reports, on two calls in a row.  Kept in a file of its own that
pytest collects last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_totals_noalloc_match_step_totals():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_12243_gb300 import build, hydro, workloads
    build.build()
    w = workloads.sod(12)
    rng = np.random.default_rng(11)
    v = rng.normal(0, 0.3, (w["x"].size, 3))
    w["px"], w["py"], w["pz"] = w["m"] * v[:, 0], w["m"] * v[:, 1], w["m"] * v[:, 2]
    w["E"] = w["U"] + 0.5 * w["m"] * np.sum(v * v, 1)
    H = hydro.Hydro(hydro.default_config(gamma=w["gamma"]))
    H.set_boxes(*hydro.single_box(w))
    st = hydro.to_device(w)
    before = {k: t.clone() for k, t in st.items()}
    stats = H.step(st, 1e-3)
    ref_before = np.array([stats["mass"][0]] + list(stats["mom"][0]) + [stats["energy"][0]])
    ref_after = np.array([stats["mass"][1]] + list(stats["mom"][1]) + [stats["energy"][1]])
    scale = np.array([np.abs(w["m"]).sum(), np.abs(w["px"]).sum(), np.abs(w["py"]).sum(),
                      np.abs(w["pz"]).sum(), np.abs(w["E"]).sum()])
    for _ in range(2):   # two calls in a row share the static scratch
        got_b = hydro.totals_noalloc(before).cpu().numpy()
        got_a = hydro.totals_noalloc(st).cpu().numpy()
        torch.cuda.synchronize()
        assert np.all(np.abs(got_b - ref_before) <= 1e-12 * scale), (got_b, ref_before)
        assert np.all(np.abs(got_a - ref_after) <= 1e-12 * scale), (got_a, ref_after)
    # sizes beyond the static scratch are refused
    lib = hydro._load()
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    p = before["m"].data_ptr()
    assert lib.hydro_totals_noalloc((1 << 26) + 1, p, p, p, p, p, out.data_ptr(), None) == -1
