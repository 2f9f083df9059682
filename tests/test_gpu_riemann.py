"""The mixed path's exact Riemann solver (§2.3.3, Toro 2009) on the faces a
step actually solves: the flux kernel records each face's float states and
its star pressure; the FP64 oracle solves the same (float) states to 1e-14.
The float Newton iteration stops at a relative change of 2e-6 and lands
within a few float ulps of the root; with hydro_config.riemann_polish one
more Newton step in FP64 makes p* the correctly rounded root."""
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


def _recorded(hyd, w, polish, hard_only):
    import torch
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision="mixed",
                                     riemann_polish=int(polish)))
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    cap = 1 << 20
    buf = torch.zeros((7, cap), dtype=torch.float32, device="cuda")
    H.record_faces(buf, keep=1.0, hard_only=hard_only)
    stats = H.step(st, -1.0)
    n = min(H.recorded_faces(), cap)
    H.close()
    return buf[:, :n].cpu().numpy().astype(np.float64), stats


@pytest.mark.parametrize("name", ["sod", "lognormal"])
def test_star_pressure_against_the_fp64_root(orc, hyd, name):
    w = W.sod(8) if name == "sod" else W.lognormal(4096, seed=2, grid=16)
    g = w["gamma"]
    res = {}
    for polish in (False, True):
        f, stats = _recorded(hyd, w, polish, hard_only=True)
        assert stats["status"] in (0, -5) and f.shape[1] > 50, (stats["status"], f.shape)
        err = np.empty(f.shape[1])
        for k in range(f.shape[1]):
            rl, ul, pl, rr, ur, pr, ps = f[:, k]
            r = orc.riemann_star(rl, ul, pl, rr, ur, pr, g, tol=1e-14)
            err[k] = abs(ps / r["p"] - 1.0)
        res[polish] = err
    # the float iteration's own tolerance; the polished value within one
    # float ulp (2^-23) of the root of the recorded states
    assert res[False].max() < 2e-6, res[False].max()
    assert res[True].max() <= 2.0 ** -23, res[True].max()
    assert np.median(res[True]) <= np.median(res[False]) + 1e-12
