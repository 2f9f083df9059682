"""Error paths of the C ABI, each made on the host side -- no GPU fault, trap
or hang is caused: a non-finite value in the caller's state, a caller
neighbour-list buffer one entry too small, a smoothing-length iteration
capped at one Newton step, and the learned guess's tensor-core wait run out
through the test hook (the weight copy is never issued, so nothing is in
flight when the bounded wait gives up).  Each call returns its status and
leaves the caller's state exactly as it was; the context keeps working
afterwards.  Host-driven steps (a context's first) and captured-graph steps
(its later ones) are both covered."""
import ctypes as C

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


def _snap(st):
    return {k: v.clone() for k, v in st.items()}


def _unchanged(st, snap):
    import torch
    torch.cuda.synchronize()
    # bitwise, NaNs included
    return all(torch.equal(st[k].view(torch.int64), snap[k].view(torch.int64)) for k in snap)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("key", ["x", "E", "h"])
def test_nonfinite_input_leaves_the_state(hyd, precision, key):
    w = W.sod(8)
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision=precision))
    H.set_boxes(*hyd.single_box(w))
    good = hyd.to_device(w)
    for attempt in range(2):   # the context's first call, then after a good step
        st = _snap(good)
        st[key][37] = float("nan") if attempt == 0 else float("inf")
        snap = _snap(st)
        stats = H.step(st, -1.0, check=False)
        assert stats["status"] == -7, stats   # HYDRO_ENONFINITE
        assert _unchanged(st, snap)
        ok = _snap(good)
        s2 = H.step(ok, -1.0, check=False)
        assert s2["status"] == 0, s2
    # the rung step checks the same way
    st = _snap(good)
    st[key][5] = float("nan")
    snap = _snap(st)
    import torch
    rung = torch.zeros(st["x"].numel(), dtype=torch.int32, device="cuda")
    s3 = H.step_rungs(st, 1e-3, rung, check=False)
    assert s3["status"] == -7 and _unchanged(st, snap)
    H.close()


def test_undersized_neighbour_list_reports_capacity(hyd):
    import torch
    w = W.sod(8)
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"]))
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    snap = _snap(st)
    hs = (st["h"] * 1.2).contiguous()
    off, idx = H.build_neighbours(st, hs)
    need = idx.numel()
    lib = hyd._load()
    p = hyd.particles_struct(st)
    off2 = torch.zeros_like(off)
    guard = 64
    buf = torch.full((need - 1 + guard,), -7, dtype=torch.int32, device="cuda")
    nl = hyd.NbrList(off2.data_ptr(), buf.data_ptr(), need - 1, 0)
    rc = lib.hydro_build_neighbours(H.h, C.byref(p), hs.data_ptr(), C.byref(nl), None)
    torch.cuda.synchronize()
    assert rc == -3   # HYDRO_ECAPACITY
    assert nl.needed == need
    assert torch.all(buf == -7)   # nothing written, the guard region included
    assert torch.equal(off2, off)   # the row offsets still describe the lists
    assert _unchanged(st, snap)
    # exactly enough room: the same lists
    buf2 = torch.full((need,), -7, dtype=torch.int32, device="cuda")
    nl2 = hyd.NbrList(off2.data_ptr(), buf2.data_ptr(), need, 0)
    rc = lib.hydro_build_neighbours(H.h, C.byref(p), hs.data_ptr(), C.byref(nl2), None)
    torch.cuda.synchronize()
    assert rc == 0 and nl2.needed == need and torch.equal(buf2, idx)
    H.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_h_iteration_cap_reports_noconv(hyd, precision):
    w = W.lattice_wave(12, jitter=0.1)
    w = dict(w)
    w["h"] = w["h"] * 1.3   # a start one Newton step cannot settle
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision=precision, max_h_iter=1))
    H.set_boxes(*hyd.single_box(w))
    st = hyd.to_device(w)
    snap = _snap(st)
    graphs = []
    for _ in range(2):   # host-driven, then the captured graph
        stats = H.step(st, -1.0, check=False)
        assert stats["status"] == -4, stats   # HYDRO_ENOCONV_H
        assert _unchanged(st, snap)
        graphs.append(stats["graph"])
    assert graphs == [0, 1], graphs
    # with the default cap the same context steps normally
    H.set_config(max_h_iter=60)
    stats = H.step(st, -1.0, check=False)
    assert stats["status"] == 0, stats
    H.close()


def test_mlp_wait_runs_out_reports_emlp(hyd):
    import torch
    from oracle import mlp
    w = W.sod(8)
    theta = mlp.init(3).astype(np.float32)
    H = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision="mixed", learned_guess=2))
    H.set_boxes(*hyd.single_box(w))
    H.mlp_load(theta)
    H.test_mlp_stall(1)
    st = hyd.to_device(w)
    snap = _snap(st)
    graphs = []
    for _ in range(2):   # host-driven, then the captured graph
        stats = H.step(st, -1.0, check=False)
        assert stats["status"] == -11, stats   # HYDRO_EMLP
        assert _unchanged(st, snap)
        graphs.append(stats["graph"])
    assert graphs == [0, 1], graphs
    # standalone inference: the status comes with the next synchronisation
    faces = torch.rand((6, 300), dtype=torch.float32, device="cuda") + 0.5
    H.mlp_predict(faces)
    assert H.sync_status() == -11
    # hook off: the learned path runs and the step matches a plain-guess step
    H.test_mlp_stall(0)
    stats = H.step(st, -1.0, check=False)
    assert stats["status"] == 0 and stats["learned_active"] == 1, stats
    Hp = hyd.Hydro(hyd.default_config(gamma=w["gamma"], precision="mixed"))
    Hp.set_boxes(*hyd.single_box(w))
    sp = _snap(snap)
    Hp.step(sp, -1.0)
    torch.cuda.synchronize()
    for k in ("px", "E"):
        d_l = (st[k] - snap[k]).cpu().numpy()
        d_p = (sp[k] - snap[k]).cpu().numpy()
        assert np.max(np.abs(d_l - d_p)) <= 1e-5 * np.abs(d_p).max(), k
    H.close()
    Hp.close()
