"""sorted_output: hydro_step writes the particles back in its own (Morton)
order and hydro_get_order reports the permutation.  The reordered state is
the caller-order step's state permuted (the same arithmetic: the FP64 path
to its flux-accumulation rounding, 1e-12); the next steps from the sorted
state reorder it only locally and still agree with the caller-order run; the rung path refuses the mode; the order query needs a
completed step."""
import numpy as np
import pytest

from paper_2211_12243_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "z", "m", "px", "py", "pz", "E", "U", "h", "omega")


@pytest.fixture(scope="module")
def hyd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_12243_gb300 import build, hydro
    build.build()
    return hydro


def _close(a, b, tol):
    scale = np.maximum(np.abs(b), np.abs(b).max() * 1e-6) + 1e-300
    return float(np.max(np.abs(a - b) / scale)) <= tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
@pytest.mark.parametrize("graph", [0, 1])
def test_sorted_output_is_the_caller_order_step_permuted(hyd, precision, tol, graph):
    import torch
    w = W.lognormal(1 << 14, seed=5, grid=16)
    ctx = []
    for so in (0, 1):
        H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision=precision, graph=graph,
                                         sorted_output=so))
        H.set_boxes(*hyd.single_box(w))
        ctx.append(H)
    H0, H1 = ctx
    with pytest.raises(hyd.HydroError) as e:
        H1.get_order()   # no step yet
    assert e.value.code == -9
    st0, st1 = hyd.to_device(w), hyd.to_device(w)
    dt = None
    for step in range(3):
        s0 = H0.step(st0, dt if dt else -1.0, check=False)
        s1 = H1.step(st1, s0["dt"], check=False)
        dt = s0["dt"]
        assert s0["status"] == s1["status"] and s0["status"] in (0, -5)
        torch.cuda.synchronize()
        perm = H1.get_order().long()
        p = perm.cpu().numpy()
        assert np.array_equal(np.sort(p), np.arange(p.size))
        if step == 0:
            order = p.copy()          # caller index of each sorted slot
        else:
            order = order[p]          # compose: slot <- previous slot <- caller index
            # the state was already in the previous step's order: the drift
            # reorders particles only locally (a random order would put
            # about 3 % of them within 256 places of their slot)
            assert np.mean(np.abs(p - np.arange(p.size)) <= 256) > 0.9
        for k in KEYS:
            a = st1[k].cpu().numpy()
            b = st0[k].cpu().numpy()[order]
            assert _close(a, b, tol), (step, k)


def test_rungs_refuse_sorted_output(hyd):
    import torch
    w = W.sod(8)
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], sorted_output=1))
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    rung = torch.zeros(w["x"].size, dtype=torch.int32, device="cuda")
    with pytest.raises(hyd.HydroError) as e:
        H.step_rungs(st, 1e-3, rung)
    assert e.value.code == -9   # HYDRO_ESTATE
