"""Thin ctypes binding of ``libhydro.so`` (the C ABI of ``include/hydro.h``).

Argument marshalling only: every step of the hydro path runs in the CUDA
kernels of the library.  PyTorch provides the device memory and the stream.
If the library has not been built, loading fails with an error -- there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhydro.so")
_lib = None

KERNELS = {"wendland": 0, "cubic": 1}
SCHEMES = {"mfv": 0, "mfm": 1}
RIEMANN = {"exact": 0, "hllc": 1}
PRECISION = {"fp64": 0, "mixed": 1}

STATUS = {0: "HYDRO_OK", -1: "HYDRO_EINVAL", -2: "HYDRO_ENOMEM", -3: "HYDRO_ECAPACITY",
          -4: "HYDRO_ENOCONV_H", -5: "HYDRO_ENCOND", -6: "HYDRO_ERIEMANN",
          -7: "HYDRO_ENONFINITE", -8: "HYDRO_ECUDA", -9: "HYDRO_ESTATE", -10: "HYDRO_ESEARCH",
          -11: "HYDRO_EMLP"}

MLP_NPARAM = 12 * 64 + 64 + 64 * 64 + 64 + 64 + 1 + 24 + 2 + 24


class HydroError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _load().hydro_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {STATUS.get(code, code)} ({msg})")


class Config(C.Structure):
    _fields_ = [
        ("gamma", C.c_double), ("kernel", C.c_int), ("n_ngb", C.c_double),
        ("scheme", C.c_int), ("riemann", C.c_int), ("precision", C.c_int),
        ("learned_guess", C.c_int), ("limiter", C.c_int), ("time_extrap", C.c_int),
        ("ncond_crit", C.c_double), ("ngb_grow", C.c_double), ("max_ngb_grow", C.c_int),
        ("psi1", C.c_double), ("psi2", C.c_double), ("beta_min", C.c_double),
        ("beta_max", C.c_double), ("c_cfl", C.c_double), ("alpha1", C.c_double),
        ("h_tol", C.c_double), ("p_tol", C.c_double), ("max_h_iter", C.c_int),
        ("max_newton", C.c_int), ("search_margin", C.c_double), ("graph", C.c_int),
        ("entropy_switch", C.c_int), ("alpha2", C.c_double), ("alpha3", C.c_double),
        ("c_acc", C.c_double), ("max_rung", C.c_int), ("riemann_polish", C.c_int),
        ("sorted_output", C.c_int),
    ]


class Particles(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, C.c_void_p) for k in
                ("x", "y", "z", "mass", "px", "py", "pz", "etot", "eint", "h", "omega")]


class NbrList(C.Structure):
    _fields_ = [("off", C.c_void_p), ("idx", C.c_void_p), ("capacity", C.c_int64),
                ("needed", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("dt", C.c_double), ("dt_next", C.c_double),
        ("grad_pairs", C.c_int64), ("flux_pairs", C.c_int64), ("newton_iters", C.c_int64),
        ("guess_fallbacks", C.c_int64), ("learned_faces", C.c_int64),
        ("hard_faces", C.c_int64), ("learned_active", C.c_int), ("vacuum_faces", C.c_int64),
        ("first_order_faces", C.c_int64), ("ngb_rounds", C.c_int), ("ncond_fail", C.c_int64),
        ("list_rebuilds", C.c_int), ("mass", C.c_double * 2), ("mom", (C.c_double * 3) * 2),
        ("energy", C.c_double * 2), ("ms_sort", C.c_float), ("ms_neighbours", C.c_float),
        ("ms_density", C.c_float), ("ms_gradients", C.c_float), ("ms_fluxes", C.c_float),
        ("ms_update", C.c_float), ("ms_flux_kernel", C.c_float), ("ms_hard_faces", C.c_float),
        ("graph", C.c_int), ("learned_probe_ms", C.c_float * 2),
        ("rung_max", C.c_int), ("substeps", C.c_int64), ("active_steps", C.c_int64),
        ("rung_capped", C.c_int64), ("rung_sparse", C.c_int64),
    ]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            if k == "mom":
                v = [[v[w][a] for a in range(3)] for w in range(2)]
            elif k in ("mass", "energy", "learned_probe_ms"):
                v = [v[0], v[1]]
            d[k] = v
        return d


class Tuning(C.Structure):
    _fields_ = [
        ("search_margin", C.c_double), ("nbr_slots", C.c_int), ("grad_min_ctas", C.c_int),
        ("flux_min_ctas", C.c_int), ("front_ms", (C.c_float * 3) * 4), ("grad_ms", C.c_float * 4),
        ("flux_ms", C.c_float * 3), ("flux_queue", C.c_int), ("flux_queue_ms", C.c_float * 2),
        ("grad_rank", C.c_int), ("grad_rank_ms", C.c_float * 3),
    ]

    def as_dict(self):
        return {"search_margin": self.search_margin, "nbr_slots": self.nbr_slots,
                "grad_min_ctas": self.grad_min_ctas, "flux_min_ctas": self.flux_min_ctas,
                "front_ms": [[self.front_ms[i][j] for j in range(3)] for i in range(4)],
                "grad_ms": list(self.grad_ms), "flux_ms": list(self.flux_ms),
                "flux_queue": self.flux_queue, "flux_queue_ms": list(self.flux_queue_ms),
                "grad_rank": self.grad_rank, "grad_rank_ms": list(self.grad_rank_ms)}


EXPORTS = ["hydro_config_default", "hydro_create", "hydro_destroy", "hydro_set_config",
           "hydro_set_boxes", "hydro_reserve", "hydro_build_neighbours", "hydro_density",
           "hydro_gradients", "hydro_fluxes", "hydro_step", "hydro_sync_status",
           "hydro_get_stats", "hydro_mlp_load", "hydro_mlp_get", "hydro_mlp_predict",
           "hydro_mlp_features", "hydro_mlp_gradient", "hydro_mlp_train", "hydro_record_faces",
           "hydro_recorded_faces", "hydro_totals_noalloc", "hydro_kernel_launches",
           "hydro_strerror", "hydro_autotune", "hydro_set_tuning", "hydro_set_gravity",
           "hydro_set_entropy", "hydro_step_rungs", "hydro_test_mlp_stall",
           "hydro_probe_peak", "hydro_get_order"]


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2211_12243_gb300.build.build() (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        vp, i64, P = C.c_void_p, C.c_int64, C.POINTER
        L.hydro_config_default.argtypes = [P(Config)]
        L.hydro_config_default.restype = None
        L.hydro_create.argtypes = [P(vp), P(Config)]
        L.hydro_destroy.argtypes = [vp]
        L.hydro_destroy.restype = None
        L.hydro_set_config.argtypes = [vp, P(Config)]
        L.hydro_set_boxes.argtypes = [vp, i64, vp, vp]
        L.hydro_reserve.argtypes = [vp, i64, C.c_int]
        L.hydro_build_neighbours.argtypes = [vp, P(Particles), vp, P(NbrList), vp]
        L.hydro_density.argtypes = [vp, P(Particles), vp]
        L.hydro_gradients.argtypes = [vp, P(Particles), vp, vp, vp, vp, vp]
        L.hydro_fluxes.argtypes = [vp, P(Particles), vp, vp, vp, C.c_double, vp, vp]
        L.hydro_step.argtypes = [vp, P(Particles), C.c_double, P(Stats), vp]
        L.hydro_step_rungs.argtypes = [vp, P(Particles), C.c_double, vp, P(Stats), vp]
        L.hydro_sync_status.argtypes = [vp, vp]
        L.hydro_get_stats.argtypes = [vp, P(Stats), vp]
        L.hydro_mlp_load.argtypes = [vp, vp, C.c_size_t]
        L.hydro_mlp_get.argtypes = [vp, vp, C.c_size_t]
        L.hydro_mlp_predict.argtypes = [vp, vp, i64, vp, vp]
        L.hydro_mlp_features.argtypes = [vp, vp, i64, vp, vp, vp]
        L.hydro_mlp_gradient.argtypes = [vp, vp, vp, i64, C.c_int, vp, vp, vp]
        L.hydro_mlp_train.argtypes = [vp, vp, i64, i64, i64, C.c_double, C.c_uint64, vp, vp]
        L.hydro_record_faces.argtypes = [vp, vp, i64, C.c_double, C.c_int]
        L.hydro_recorded_faces.argtypes = [vp, P(i64), vp]
        L.hydro_totals_noalloc.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp]
        L.hydro_autotune.argtypes = [vp, P(Particles), P(Tuning), vp]
        L.hydro_set_tuning.argtypes = [vp, P(Tuning)]
        L.hydro_set_gravity.argtypes = [vp, vp]
        L.hydro_set_entropy.argtypes = [vp, vp]
        L.hydro_test_mlp_stall.argtypes = [vp, C.c_int]
        L.hydro_probe_peak.argtypes = [C.c_int, C.POINTER(C.c_double), vp]
        L.hydro_kernel_launches.argtypes = []
        L.hydro_kernel_launches.restype = C.c_int64
        L.hydro_strerror.argtypes = [C.c_int]
        L.hydro_strerror.restype = C.c_char_p
        _lib = L
    return _lib


def totals_noalloc(st, out=None, stream=None):
    """Totals of (m, px, py, pz, E) of a state dict of CUDA tensors through
    hydro_totals_noalloc (no allocation inside the library); returns the
    device tensor of 5 doubles."""
    import torch
    if out is None:
        out = torch.empty(5, dtype=torch.float64, device=st["m"].device)
    n = st["m"].numel()
    rc = _load().hydro_totals_noalloc(n, _ptr(st["m"]), _ptr(st["px"]), _ptr(st["py"]),
                                      _ptr(st["pz"]), _ptr(st["E"]), _ptr(out), _stream(stream))
    if rc:
        raise HydroError(rc, "hydro_totals_noalloc")
    return out


PROBES = {"fp32": 0, "fp64": 1, "mufu": 2}


def probe_peak(unit, stream=None):
    """Measured throughput of one arithmetic unit of the current GPU
    (hydro_probe_peak): TFLOP/s for "fp32" and "fp64", Tops/s for "mufu"."""
    v = C.c_double(0.0)
    rc = _load().hydro_probe_peak(PROBES[unit], C.byref(v), _stream(stream))
    if rc:
        raise HydroError(rc, "hydro_probe_peak")
    return v.value


def kernel_launches():
    """Kernels launched by the library in this process so far."""
    return int(_load().hydro_kernel_launches())


def default_config(**kw):
    cfg = Config()
    _load().hydro_config_default(C.byref(cfg))
    for k, v in kw.items():
        if k == "kernel":
            v = KERNELS[v] if isinstance(v, str) else v
        elif k == "scheme":
            v = SCHEMES[v] if isinstance(v, str) else v
        elif k == "riemann":
            v = RIEMANN[v] if isinstance(v, str) else v
        elif k == "precision":
            v = PRECISION[v] if isinstance(v, str) else v
        elif isinstance(v, bool):
            v = int(v)
        setattr(cfg, k, v)
    return cfg


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    return None if stream is None else C.c_void_p(stream.cuda_stream)


FIELDS = ("x", "y", "z", "m", "px", "py", "pz", "E", "U", "h", "omega")


def particles_struct(st):
    """Particles struct from a dict of float64 CUDA tensors (keys FIELDS)."""
    n = st["x"].numel()
    p = Particles()
    p.n = n
    names = dict(x="x", y="y", z="z", mass="m", px="px", py="py", pz="pz", etot="E",
                 eint="U", h="h", omega="omega")
    for cf, k in names.items():
        t = st.get(k)
        if t is not None:
            assert t.dtype.itemsize == 8 and t.is_cuda and t.is_contiguous() and t.numel() == n, k
        setattr(p, cf, None if t is None else t.data_ptr())
    return p


class Hydro:
    """One library context.  ``boxes``: (box_off, box_len) host arrays or the
    box lengths of a single box."""

    def __init__(self, config=None, **kw):
        self.lib = _load()
        self.cfg = config if config is not None else default_config(**kw)
        h = C.c_void_p()
        rc = self.lib.hydro_create(C.byref(h), C.byref(self.cfg))
        if rc:
            raise HydroError(rc, "hydro_create")
        self.h = h

    def close(self):
        if self.h:
            self.lib.hydro_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_config(self, **kw):
        for k, v in kw.items():
            if k == "scheme" and isinstance(v, str):
                v = SCHEMES[v]
            if k == "riemann" and isinstance(v, str):
                v = RIEMANN[v]
            if k == "precision" and isinstance(v, str):
                v = PRECISION[v]
            if k == "kernel" and isinstance(v, str):
                v = KERNELS[v]
            setattr(self.cfg, k, int(v) if isinstance(v, bool) else v)
        rc = self.lib.hydro_set_config(self.h, C.byref(self.cfg))
        if rc:
            raise HydroError(rc, "hydro_set_config")

    def set_boxes(self, box_off, box_len):
        box_off = np.ascontiguousarray(box_off, dtype=np.int64)
        box_len = np.ascontiguousarray(box_len, dtype=np.float64).ravel()
        nbox = box_off.size - 1
        rc = self.lib.hydro_set_boxes(self.h, nbox, box_off.ctypes.data_as(C.c_void_p),
                                      box_len.ctypes.data_as(C.c_void_p))
        if rc:
            raise HydroError(rc, "hydro_set_boxes")
        self.n_particles = int(box_off[-1])

    def reserve(self, n, per_particle=0):
        rc = self.lib.hydro_reserve(self.h, int(n), int(per_particle))
        if rc:
            raise HydroError(rc, "hydro_reserve")

    def build_neighbours(self, st, h_search, export=True, stream=None):
        import torch
        p = particles_struct(st)
        if not export:
            rc = self.lib.hydro_build_neighbours(self.h, C.byref(p), _ptr(h_search), None,
                                                 _stream(stream))
            if rc:
                raise HydroError(rc, "hydro_build_neighbours")
            return None
        n = p.n
        off = torch.zeros(n + 1, dtype=torch.int64, device=st["x"].device)
        nl = NbrList(off.data_ptr(), None, 0, 0)
        rc = self.lib.hydro_build_neighbours(self.h, C.byref(p), _ptr(h_search), C.byref(nl),
                                             _stream(stream))
        if rc not in (0, -3):
            raise HydroError(rc, "hydro_build_neighbours")
        idx = torch.zeros(max(nl.needed, 1), dtype=torch.int32, device=st["x"].device)
        nl2 = NbrList(off.data_ptr(), idx.data_ptr(), idx.numel(), 0)
        rc = self.lib.hydro_build_neighbours(self.h, C.byref(p), _ptr(h_search), C.byref(nl2),
                                             _stream(stream))
        if rc:
            raise HydroError(rc, "hydro_build_neighbours")
        return off, idx[: nl2.needed]

    def density(self, st, stream=None):
        p = particles_struct(st)
        rc = self.lib.hydro_density(self.h, C.byref(p), _stream(stream))
        if rc:
            raise HydroError(rc, "hydro_density")

    def gradients(self, st, stream=None):
        import torch
        n = st["x"].numel()
        dev = st["x"].device
        B = torch.empty((n, 6), dtype=torch.float64, device=dev)
        G = torch.empty((n, 5, 3), dtype=torch.float64, device=dev)
        A = torch.empty((n, 5), dtype=torch.float64, device=dev)
        N = torch.empty(n, dtype=torch.float64, device=dev)
        p = particles_struct(st)
        rc = self.lib.hydro_gradients(self.h, C.byref(p), _ptr(B), _ptr(G), _ptr(A), _ptr(N),
                                      _stream(stream))
        if rc:
            raise HydroError(rc, "hydro_gradients")
        return B, G, A, N

    def fluxes(self, st, B, G, A, dt, stream=None):
        import torch
        n = st["x"].numel()
        dQ = torch.empty((n, 6), dtype=torch.float64, device=st["x"].device)
        p = particles_struct(st)
        rc = self.lib.hydro_fluxes(self.h, C.byref(p), _ptr(B.contiguous()), _ptr(G.contiguous()),
                                   _ptr(A.contiguous()), float(dt), _ptr(dQ), _stream(stream))
        if rc:
            raise HydroError(rc, "hydro_fluxes")
        return dQ

    def step(self, st, dt=-1.0, stats=True, stream=None, check=True):
        p = particles_struct(st)
        s = Stats() if stats else None
        rc = self.lib.hydro_step(self.h, C.byref(p), float(dt), C.byref(s) if stats else None,
                                 _stream(stream))
        if rc and check:
            raise HydroError(rc, "hydro_step")
        return s.as_dict() if stats else rc

    def step_rungs(self, st, dt0, rung, stats=True, stream=None, check=True):
        """One base step dt0 with individual timesteps (hydro_step_rungs);
        rung: CUDA int32 tensor [n] receiving the rungs used."""
        p = particles_struct(st)
        s = Stats() if stats else None
        rc = self.lib.hydro_step_rungs(self.h, C.byref(p), float(dt0), _ptr(rung),
                                       C.byref(s) if stats else None, _stream(stream))
        if rc and check:
            raise HydroError(rc, "hydro_step_rungs")
        return s.as_dict() if stats else rc

    def autotune(self, st, stream=None):
        """Time the launch-parameter candidates on the state st and keep the
        fastest (hydro_autotune); returns the choices and times."""
        p = particles_struct(st)
        t = Tuning()
        rc = self.lib.hydro_autotune(self.h, C.byref(p), C.byref(t), _stream(stream))
        if rc:
            raise HydroError(rc, "hydro_autotune")
        return t.as_dict()

    def set_gravity(self, acc):
        """acc: CUDA float64 tensor [n, 3] (caller order) kept alive by the
        caller, or None (hydro_set_gravity)."""
        self._grav = acc
        rc = self.lib.hydro_set_gravity(self.h, _ptr(acc) if acc is not None else None)
        if rc:
            raise HydroError(rc, "hydro_set_gravity")

    def get_order(self, stream=None):
        """The last step's order (hydro_get_order): int32 CUDA tensor [n],
        entry i the input index of the particle at sorted position i."""
        import torch
        perm = torch.empty(self.n_particles, dtype=torch.int32, device="cuda")
        rc = self.lib.hydro_get_order(self.h, _ptr(perm), _stream(stream))
        if rc:
            raise HydroError(rc, "hydro_get_order")
        return perm

    def test_mlp_stall(self, on):
        """Error-path test hook: the network's weight copy is not issued, so
        its kernels' first wait runs out (hydro_test_mlp_stall)."""
        rc = self.lib.hydro_test_mlp_stall(self.h, int(on))
        if rc:
            raise HydroError(rc, "hydro_test_mlp_stall")

    def set_entropy(self, A):
        """A: CUDA float64 tensor [n] (caller order), the entropic function
        that hydro_step reads and rewrites with cfg.entropy_switch = 1; kept
        alive by the caller, or None (hydro_set_entropy)."""
        self._entA = A
        rc = self.lib.hydro_set_entropy(self.h, _ptr(A) if A is not None else None)
        if rc:
            raise HydroError(rc, "hydro_set_entropy")

    def set_tuning(self, d):
        t = Tuning()
        t.search_margin = d["search_margin"]
        t.nbr_slots = d["nbr_slots"]
        t.grad_min_ctas = d["grad_min_ctas"]
        t.flux_min_ctas = d["flux_min_ctas"]
        t.flux_queue = d.get("flux_queue", 1)
        t.grad_rank = d.get("grad_rank", 1)
        rc = self.lib.hydro_set_tuning(self.h, C.byref(t))
        if rc:
            raise HydroError(rc, "hydro_set_tuning")

    def sync_status(self, stream=None):
        return self.lib.hydro_sync_status(self.h, _stream(stream))

    def mlp_load(self, weights):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        rc = self.lib.hydro_mlp_load(self.h, w.ctypes.data_as(C.c_void_p), w.nbytes)
        if rc:
            raise HydroError(rc, "hydro_mlp_load")

    def mlp_get(self):
        w = np.zeros(MLP_NPARAM, dtype=np.float32)
        rc = self.lib.hydro_mlp_get(self.h, w.ctypes.data_as(C.c_void_p), w.nbytes)
        if rc:
            raise HydroError(rc, "hydro_mlp_get")
        return w

    @staticmethod
    def _faces(faces, rows):
        assert faces.dtype.itemsize == 4 and faces.is_cuda and faces.is_contiguous()
        assert faces.dim() == 2 and faces.shape[0] >= rows
        return faces.shape[1]

    def mlp_predict(self, faces, stream=None):
        """faces: float32 CUDA tensor [6 (or 7), n] -> p_guess [n] (-1: out of range)."""
        import torch
        n = self._faces(faces, 6)
        out = torch.empty(n, dtype=torch.float32, device=faces.device)
        rc = self.lib.hydro_mlp_predict(self.h, _ptr(faces), n, _ptr(out), _stream(stream))
        if rc:
            raise HydroError(rc, "hydro_mlp_predict")
        return out

    def mlp_features(self, faces, stream=None):
        import torch
        n = self._faces(faces, 7)
        x = torch.empty((n, 12), dtype=torch.float32, device=faces.device)
        t = torch.empty(n, dtype=torch.float32, device=faces.device)
        rc = self.lib.hydro_mlp_features(self.h, _ptr(faces), n, _ptr(x), _ptr(t),
                                         _stream(stream))
        if rc:
            raise HydroError(rc, "hydro_mlp_features")
        return x, t

    def mlp_gradient(self, x, t, quant=False, stream=None):
        import torch
        assert x.dtype == torch.float32 and x.is_contiguous() and x.shape[1] == 12
        assert t.dtype == torch.float32 and t.is_contiguous() and t.numel() == x.shape[0]
        g = torch.empty(MLP_NPARAM, dtype=torch.float32, device=x.device)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        rc = self.lib.hydro_mlp_gradient(self.h, _ptr(x), _ptr(t), x.shape[0], int(quant),
                                         _ptr(g), _ptr(loss), _stream(stream))
        if rc:
            raise HydroError(rc, "hydro_mlp_gradient")
        return g, loss

    def mlp_train(self, faces, steps, batch=1024, lr=1e-3, seed=0, stream=None):
        """Train on recorded faces [7, n]; returns the per-step loss tensor."""
        import torch
        n = self._faces(faces, 7)
        loss = torch.zeros(max(int(steps), 1), dtype=torch.float32, device=faces.device)
        rc = self.lib.hydro_mlp_train(self.h, _ptr(faces), n, int(steps), int(batch), float(lr),
                                      int(seed), _ptr(loss), _stream(stream))
        if rc:
            raise HydroError(rc, "hydro_mlp_train")
        return loss[: int(steps)]

    def record_faces(self, buf, keep=1.0, hard_only=False):
        """Record solved faces of the next flux calls into buf (float32 CUDA
        tensor [7, capacity]); buf=None stops recording."""
        cap = 0 if buf is None else self._faces(buf, 7)
        rc = self.lib.hydro_record_faces(self.h, _ptr(buf), cap, float(keep), int(hard_only))
        if rc:
            raise HydroError(rc, "hydro_record_faces")

    def recorded_faces(self, stream=None):
        v = C.c_int64()
        rc = self.lib.hydro_recorded_faces(self.h, C.byref(v), _stream(stream))
        if rc:
            raise HydroError(rc, "hydro_recorded_faces")
        return v.value

    def get_stats(self, stream=None):
        s = Stats()
        rc = self.lib.hydro_get_stats(self.h, C.byref(s), _stream(stream))
        if rc:
            raise HydroError(rc, "hydro_get_stats")
        return s.as_dict()


def to_device(w, device="cuda", keys=("x", "y", "z", "m", "px", "py", "pz", "E", "U", "h")):
    """Workload dict (numpy) -> dict of contiguous float64 CUDA tensors (+ omega)."""
    import torch
    out = {k: torch.as_tensor(np.ascontiguousarray(w[k], dtype=np.float64), device=device)
           for k in keys}
    out["omega"] = torch.zeros_like(out["x"])
    return out


def single_box(w):
    n = w["x"].size
    return np.array([0, n], dtype=np.int64), np.asarray(w["L"], dtype=np.float64)
