"""The allocation-free totals entry point (hydro_totals_noalloc), for callers
that cannot call cudaMalloc (a host application that owns every device
allocation through its own pool, or a plugin that must keep the device
memory footprint fixed).  Its output must agree with the totals the regular
hydro_step reports, and with exactly rounded sums of the host arrays, on two
calls in a row.  Kept in a file of its own that pytest collects last."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hyd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_12243_gb300 import build, hydro
    build.build()
    return hydro


def test_totals_noalloc_match_step_totals(hyd):
    import torch
    from paper_2211_12243_gb300 import workloads
    w = workloads.sod(12)
    rng = np.random.default_rng(11)
    v = rng.normal(0, 0.3, (w["x"].size, 3))
    w["px"], w["py"], w["pz"] = w["m"] * v[:, 0], w["m"] * v[:, 1], w["m"] * v[:, 2]
    w["E"] = w["U"] + 0.5 * w["m"] * np.sum(v * v, 1)
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"]))
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    before = {k: t.clone() for k, t in st.items()}
    stats = H.step(st, 1e-3)
    ref_before = np.array([stats["mass"][0]] + list(stats["mom"][0]) + [stats["energy"][0]])
    ref_after = np.array([stats["mass"][1]] + list(stats["mom"][1]) + [stats["energy"][1]])
    scale = np.array([np.abs(w["m"]).sum(), np.abs(w["px"]).sum(), np.abs(w["py"]).sum(),
                      np.abs(w["pz"]).sum(), np.abs(w["E"]).sum()])
    for _ in range(2):   # two calls in a row share the static scratch
        got_b = hyd.totals_noalloc(before).cpu().numpy()
        got_a = hyd.totals_noalloc(st).cpu().numpy()
        torch.cuda.synchronize()
        assert np.all(np.abs(got_b - ref_before) <= 1e-12 * scale), (got_b, ref_before)
        assert np.all(np.abs(got_a - ref_after) <= 1e-12 * scale), (got_a, ref_after)
    H.close()


@pytest.mark.parametrize("n", [0, 1, 4096, 4097, 300_001])
def test_totals_noalloc_match_exact_sums(hyd, n):
    """Against math.fsum (the correctly rounded sum) of the host arrays:
    values spread over sixteen decades with both signs, so that plain
    summation would lose digits; one row of partial sums per 4096 values
    (n = 300,001: 74 rows, the last one ragged).  Two calls in a row, the
    second on different data, so a row left from the first would show."""
    import torch
    rng = np.random.default_rng(n + 5)
    keys = ("m", "px", "py", "pz", "E")
    for call in range(2):
        host = {k: rng.normal(0.0, 1.0, n) * 10.0 ** rng.uniform(-8, 8, n) for k in keys}
        host["m"] = np.abs(host["m"])
        dev = {k: torch.as_tensor(v, device="cuda") for k, v in host.items()}
        got = hyd.totals_noalloc(dev).cpu().numpy()
        for q, k in enumerate(keys):
            exact = math.fsum(host[k])
            bound = 1e-15 * math.fsum(np.abs(host[k])) + 1e-300
            assert abs(got[q] - exact) <= bound, (call, k, got[q], exact, bound)


def test_totals_noalloc_rejects_sizes_beyond_the_scratch(hyd):
    import torch
    lib = hyd._load()
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    assert lib.hydro_totals_noalloc((1 << 26) + 1, p, p, p, p, p, out.data_ptr(), None) == -1
    assert lib.hydro_totals_noalloc(-1, p, p, p, p, p, out.data_ptr(), None) == -1
    assert lib.hydro_totals_noalloc(4, p, p, p, p, p, None, None) == -1
