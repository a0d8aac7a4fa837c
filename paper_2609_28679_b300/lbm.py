"""Python binding of the C ABI in ``include/lbm.h`` (ctypes).

Argument marshalling only: every step of the method runs in the CUDA library
``liblbm.so``.  The functions keep the C names; pointers may be numpy arrays
(host, on_device=0) or CUDA torch tensors (device, on_device=1).  Importing
this module does not touch the GPU; the first call loads the library and
raises if it is missing or if no CUDA device is present.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_OK, LBM_E_INVALID, LBM_E_NOMEM, LBM_E_CUDA, LBM_E_UNSUPPORTED, LBM_E_STATE = 0, -1, -2, -3, -4, -5
LBM_F64, LBM_F32, LBM_BF16, LBM_F16 = 0, 1, 2, 3
LBM_IDEAL, LBM_VDW, LBM_PR = 0, 1, 2
LBM_T_NEWTON, LBM_T_MLP = 0, 1
LBM_PHI_UPWIND, LBM_PHI_CENTRAL = 0, 1
LBM_KERNEL_AUTO, LBM_KERNEL_SPLIT, LBM_KERNEL_FUSED, LBM_KERNEL_ZMARCH, LBM_KERNEL_ZGATHER = 0, 1, 2, 3, 4
LBM_KERNEL_YMARCH = 5
LBM_FACE_INLET_TOTAL, LBM_FACE_INLET_STATIC, LBM_FACE_OUTLET_P, LBM_FACE_OUTLET_EXTRAP, LBM_FACE_INLET_PT = 1, 2, 3, 4, 5

STORAGE = {"f64": LBM_F64, "f32": LBM_F32, "bf16": LBM_BF16, "f16": LBM_F16}
EOS = {"ideal": LBM_IDEAL, "vdw": LBM_VDW, "pr": LBM_PR}


class LbmError(RuntimeError):
    pass


class lbm_lattice(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("zwalls", ctypes.c_int), ("storage", ctypes.c_int), ("phi_scheme", ctypes.c_int)]


class lbm_eos(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("R", ctypes.c_double), ("cv", ctypes.c_double),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("Tc", ctypes.c_double), ("Pc", ctypes.c_double),
                ("omega", ctypes.c_double), ("kappa", ctypes.c_double), ("eta_over_mu", ctypes.c_double),
                ("k_over_mu", ctypes.c_double), ("t_solver", ctypes.c_int), ("mu", ctypes.c_double),
                ("isothermal", ctypes.c_int)]


class lbm_force(ctypes.Structure):
    _fields_ = [("accel", ctypes.c_double * 3), ("friction", ctypes.c_double), ("throttle_K", ctypes.c_double),
                ("throttle_sigma", ctypes.c_double), ("field", ctypes.c_void_p)]


class lbm_heat(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("zmask_lo", ctypes.c_int), ("zmask_hi", ctypes.c_int),
                ("field", ctypes.c_void_p)]


_lib = None

_SIGS = {
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(lbm_lattice), ctypes.POINTER(lbm_eos), ctypes.c_double,
                                  ctypes.c_double, ctypes.POINTER(lbm_force), ctypes.POINTER(lbm_heat),
                                  ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_create_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(lbm_lattice), ctypes.POINTER(lbm_eos),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(lbm_force), ctypes.POINTER(lbm_heat),
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_destroy": (None, [ctypes.c_void_p]),
    "lbm_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_set_force": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_set_walls": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                                     ctypes.c_double, ctypes.c_int]),
    "lbm_set_face": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_double,
                                    ctypes.c_double]),
    "lbm_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "lbm_init_f32": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "lbm_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbm_moments": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "lbm_moments_f32": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "lbm_populations": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "lbm_invariants": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_diagnostics": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_step_timed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "lbm_fp64_peak": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_set_kernel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "lbm_get_kernel": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 4),
    "lbm_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "lbm_set_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbm_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 4 +
                     [ctypes.POINTER(ctypes.c_double)]),
    "lbm_mlp_nparams": (ctypes.c_int, []),
    "lbm_mlp_train": (ctypes.c_int, [ctypes.POINTER(lbm_eos), ctypes.POINTER(ctypes.c_double), ctypes.c_longlong,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_ulonglong, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_mlp_grad": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_mlp_predict": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_longlong, ctypes.c_void_p]),
    "lbm_mlp_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_step_static": (ctypes.c_int, [ctypes.POINTER(lbm_lattice), ctypes.POINTER(lbm_eos), ctypes.c_double,
                                       ctypes.c_double, ctypes.POINTER(lbm_force), ctypes.POINTER(lbm_heat),
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblbm.so (no GPU work).  Raises if the library is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise LbmError(f"CUDA library not built: {path} is missing (run paper_2609_28679_b300.build)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _lib_gpu() -> ctypes.CDLL:
    lib = load_library()
    import torch

    if not torch.cuda.is_available():
        raise LbmError("no CUDA device: the library has no CPU path")
    torch.cuda.init()
    return lib


def _check(rc: int, h) -> None:
    if rc != LBM_OK:
        msg = _lib.lbm_last_error(h)
        raise LbmError(f"rc={rc}: {msg.decode() if msg else ''}")


def _ptr(a, single: bool = False):
    """Data pointer of a numpy array or torch tensor (None -> NULL), float64
    or, with single, float32."""
    if a is None:
        return None
    want = "float32" if single else "float64"
    if isinstance(a, np.ndarray):
        if not (a.dtype == np.dtype(want) and a.flags.c_contiguous):
            raise LbmError(f"host arrays must be C-contiguous {want}")
        return a.ctypes.data_as(ctypes.c_void_p)
    import torch

    if isinstance(a, torch.Tensor):
        if a.dtype != getattr(torch, want) or not a.is_contiguous():
            raise LbmError(f"tensors must be contiguous {want}")
        return ctypes.c_void_p(a.data_ptr())
    raise LbmError(f"unsupported buffer type {type(a)}")


# -- thin wrappers with the C names -------------------------------------------------

def lbm_create(lattice: lbm_lattice, eos: lbm_eos, tau_f: float, tau_g: float, force=None, heat=None):
    lib = _lib_gpu()
    h = ctypes.c_void_p()
    rc = lib.lbm_create(ctypes.byref(lattice), ctypes.byref(eos), tau_f, tau_g,
                        ctypes.byref(force) if force is not None else None,
                        ctypes.byref(heat) if heat is not None else None, ctypes.byref(h))
    _check(rc, None)
    return h


def lbm_create_batch(lattices, eos, tau_f, tau_g, force=None, heat=None):
    lib = _lib_gpu()
    n = len(lattices)
    La = (lbm_lattice * n)(*lattices)
    Ea = (lbm_eos * n)(*eos)
    tf = (ctypes.c_double * n)(*tau_f)
    tg = (ctypes.c_double * n)(*tau_g)
    Fa = (lbm_force * n)(*force) if force is not None else None
    Ha = (lbm_heat * n)(*heat) if heat is not None else None
    h = ctypes.c_void_p()
    rc = lib.lbm_create_batch(n, La, Ea, tf, tg, Fa, Ha, ctypes.byref(h))
    _check(rc, None)
    return h


def lbm_destroy(h) -> None:
    if h:
        load_library().lbm_destroy(h)


def lbm_set_stream(h, stream) -> None:
    _check(_lib.lbm_set_stream(h, ctypes.c_void_p(stream)), h)


def lbm_init(h, rho, u, T, on_device: int) -> None:
    _check(_lib.lbm_init(h, _ptr(rho), _ptr(u), _ptr(T), int(on_device)), h)


def lbm_init_f32(h, rho, u, T, on_device: int) -> None:
    _check(_lib.lbm_init_f32(h, _ptr(rho, True), _ptr(u, True), _ptr(T, True), int(on_device)), h)


def lbm_set_force(h, accel) -> None:
    a = np.ascontiguousarray(np.asarray(accel, dtype=np.float64).reshape(-1)[:3])
    if a.size < 3:
        a = np.concatenate([a, np.zeros(3 - a.size)])
    _check(_lib.lbm_set_force(h, a.ctypes.data), h)


def lbm_set_walls(h, u_lo, T_lo: float, u_hi, T_hi: float, wall_rho: int = 0) -> None:
    lo = np.zeros(3)
    hi = np.zeros(3)
    lo[:len(u_lo)] = u_lo
    hi[:len(u_hi)] = u_hi
    _check(_lib.lbm_set_walls(h, lo.ctypes.data, float(T_lo), hi.ctypes.data, float(T_hi), int(wall_rho)), h)


def lbm_set_face(h, face: int, kind: int, u=None, T: float = 0.0, P: float = 0.0) -> None:
    uu = np.zeros(3)
    if u is not None:
        uu[:len(u)] = u
    _check(_lib.lbm_set_face(h, int(face), int(kind), uu.ctypes.data, float(T), float(P)), h)


def lbm_step(h, n: int) -> None:
    _check(_lib.lbm_step(h, int(n)), h)


def lbm_moments(h, rho, u, T, on_device: int) -> None:
    _check(_lib.lbm_moments(h, _ptr(rho), _ptr(u), _ptr(T), int(on_device)), h)


def lbm_moments_f32(h, rho, u, T, on_device: int) -> None:
    _check(_lib.lbm_moments_f32(h, _ptr(rho, True), _ptr(u, True), _ptr(T, True), int(on_device)), h)


def lbm_populations(h, f, g, on_device: int) -> None:
    _check(_lib.lbm_populations(h, _ptr(f), _ptr(g), int(on_device)), h)


def lbm_invariants(h, out: np.ndarray) -> None:
    _check(_lib.lbm_invariants(h, _ptr(out)), h)


def lbm_diagnostics(h) -> np.ndarray:
    out = np.zeros(4, dtype=np.int64)
    _check(_lib.lbm_diagnostics(h, out.ctypes.data_as(ctypes.c_void_p)), h)
    return out


def lbm_step_timed(h, n: int) -> np.ndarray:
    """Mean device ms per step of passes 1, 2, 3 and of the whole step over n steps."""
    out = np.zeros(4, dtype=np.float64)
    _check(_lib.lbm_step_timed(h, int(n), out.ctypes.data_as(ctypes.c_void_p)), h)
    return out


def lbm_fp64_peak(stream=None) -> tuple:
    """(TFLOP/s, ms of the timed launch) of the float64 FMA probe."""
    lib = _lib_gpu()
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib.lbm_fp64_peak(ctypes.byref(tf), ctypes.byref(ms), ctypes.c_void_p(stream or 0)), None)
    return tf.value, ms.value


def lbm_set_kernel(h, variant: int, tx: int = 0, ty: int = 0, tz: int = 0) -> None:
    _check(_lib.lbm_set_kernel(h, variant, tx, ty, tz), h)


def lbm_set_graph(h, steps_per_graph: int) -> None:
    _check(_lib.lbm_set_graph(h, int(steps_per_graph)), h)


def lbm_autotune(h, trial_steps: int = 5):
    v = [ctypes.c_int() for _ in range(4)]
    ms = ctypes.c_double()
    _check(_lib.lbm_autotune(h, int(trial_steps), *[ctypes.byref(x) for x in v], ctypes.byref(ms)), h)
    return tuple(x.value for x in v), ms.value


def lbm_get_kernel(h):
    v = [ctypes.c_int() for _ in range(4)]
    _check(_lib.lbm_get_kernel(h, *[ctypes.byref(x) for x in v]), h)
    return tuple(x.value for x in v)


def lbm_step_static(lattice: lbm_lattice, eos: lbm_eos, tau_f: float, tau_g: float, force, heat,
                    f_in, g_in, f_out, g_out, stream: int | None = None) -> None:
    """One float64 step of caller-owned device populations without any
    allocation (see include/lbm.h); tensors are CUDA float64 [Q*N]."""
    lib = _lib_gpu()
    rc = lib.lbm_step_static(ctypes.byref(lattice), ctypes.byref(eos), tau_f, tau_g,
                             ctypes.byref(force) if force is not None else None,
                             ctypes.byref(heat) if heat is not None else None,
                             _ptr(f_in), _ptr(g_in), _ptr(f_out), _ptr(g_out),
                             ctypes.c_void_p(stream) if stream else None)
    _check(rc, None)


def lbm_mlp_nparams() -> int:
    return int(load_library().lbm_mlp_nparams())


def _f32(a: np.ndarray):
    if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous):
        raise LbmError("parameter arrays must be C-contiguous float32")
    return a.ctypes.data_as(ctypes.c_void_p)


def lbm_mlp_train(eos: lbm_eos, box, nsamples: int, steps: int, batch: int, lr: float, seed: int,
                  init: bool, params: np.ndarray, loss_hist: np.ndarray | None = None, stream: int | None = None):
    lib = _lib_gpu()
    b = (ctypes.c_double * 4)(*box)
    rc = lib.lbm_mlp_train(ctypes.byref(eos), b, int(nsamples), int(steps), int(batch), float(lr), int(seed),
                           int(bool(init)), _f32(params), _ptr(loss_hist) if loss_hist is not None else None,
                           ctypes.c_void_p(stream) if stream else None)
    _check(rc, None)


def lbm_mlp_grad(params: np.ndarray, rho, e, T):
    lib = _lib_gpu()
    g = np.zeros(lbm_mlp_nparams(), dtype=np.float32)
    loss = ctypes.c_double()
    rc = lib.lbm_mlp_grad(_f32(params), _ptr(rho), _ptr(e), _ptr(T), len(rho), _f32(g), ctypes.byref(loss))
    _check(rc, None)
    return loss.value, g


def lbm_mlp_predict(params: np.ndarray, rho, e) -> np.ndarray:
    lib = _lib_gpu()
    out = np.zeros(len(rho))
    _check(lib.lbm_mlp_predict(_f32(params), _ptr(rho), _ptr(e), len(rho), _ptr(out)), None)
    return out


def lbm_mlp_load(h, params: np.ndarray) -> None:
    _check(_lib.lbm_mlp_load(h, _f32(params)), h)


def lbm_last_error(h) -> str:
    msg = load_library().lbm_last_error(h)
    return msg.decode() if msg else ""


# -- convenience: structs from a workload case ---------------------------------------

def structs_from_case(case):
    lat = lbm_lattice(case.dim, case.nx, case.ny, case.nz, case.zwalls, STORAGE[case.storage],
                      LBM_PHI_CENTRAL if case.phi_central else LBM_PHI_UPWIND)
    eos = lbm_eos(EOS[case.eos], case.R, case.cv, case.a, case.b, case.Tc, case.Pc, case.omega, case.kappa,
                  case.eta_over_mu, case.k_over_mu, getattr(case, "t_solver", LBM_T_NEWTON), getattr(case, "mu", 0.0),
                  getattr(case, "isothermal", 0))
    force = lbm_force((ctypes.c_double * 3)(*case.accel), getattr(case, "friction", 0.0),
                      getattr(case, "throttle_K", 0.0), getattr(case, "throttle_sigma", 0.0))
    heat = lbm_heat(case.q, case.zlo, case.zhi)
    return lat, eos, force, heat


class Simulation:
    """One handle (a single case, or a list of cases stepped as a batch)."""

    def __init__(self, cases, variant: int | None = None, tile=None):
        self.cases = list(cases) if isinstance(cases, (list, tuple)) else [cases]
        self.dim = self.cases[0].dim
        self.Q = 3 ** self.dim
        parts = [structs_from_case(c) for c in self.cases]
        if len(self.cases) == 1:
            lat, eos, force, heat = parts[0]
            self.h = lbm_create(lat, eos, self.cases[0].tau_f, self.cases[0].tau_g, force, heat)
        else:
            self.h = lbm_create_batch([p[0] for p in parts], [p[1] for p in parts],
                                      [c.tau_f for c in self.cases], [c.tau_g for c in self.cases],
                                      [p[2] for p in parts], [p[3] for p in parts])
        self.N = sum(c.ncell for c in self.cases)
        c0 = self.cases[0]
        if any(c.zwalls == 2 for c in self.cases):
            lbm_set_walls(self.h, c0.uw_lo, c0.Tw_lo, c0.uw_hi, c0.Tw_hi, getattr(c0, "wall_rho", 0))
            for face, kind in enumerate(getattr(c0, "face_kind", (0, 0))):
                if kind:
                    lbm_set_face(self.h, face, kind, c0.uw_lo if face == 0 else c0.uw_hi,
                                 c0.Tw_lo if face == 0 else c0.Tw_hi, c0.face_P[face])
        if variant is not None:
            t = tile or (0, 0, 0)
            lbm_set_kernel(self.h, variant, *t)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, fields=None):
        if fields is None:
            fs = [c.fields() for c in self.cases]
            rho = np.concatenate([f[0] for f in fs])
            u = np.concatenate([f[1].ravel() for f in fs])
            T = np.concatenate([f[2] for f in fs])
        else:
            rho, u, T = fields
        lbm_init(self.h, np.ascontiguousarray(rho, dtype=np.float64), np.ascontiguousarray(u, dtype=np.float64).ravel(),
                 np.ascontiguousarray(T, dtype=np.float64), 0)

    def step(self, n: int = 1):
        lbm_step(self.h, n)

    def moments(self):
        rho = np.zeros(self.N)
        u = np.zeros(self.dim * self.N)
        T = np.zeros(self.N)
        lbm_moments(self.h, rho, u, T, 0)
        return rho, u, T

    def populations(self):
        f = np.zeros(self.Q * self.N)
        g = np.zeros(self.Q * self.N)
        lbm_populations(self.h, f, g, 0)
        return f, g

    def invariants(self) -> np.ndarray:
        out = np.zeros(len(self.cases) * (2 * self.dim + 3))
        lbm_invariants(self.h, out)
        return out.reshape(len(self.cases), 2 * self.dim + 3)

    def diagnostics(self) -> np.ndarray:
        return lbm_diagnostics(self.h)

    def kernel(self):
        return lbm_get_kernel(self.h)

    def autotune(self, trial_steps: int = 5):
        return lbm_autotune(self.h, trial_steps)

    def use_graphs(self, steps_per_graph: int, stream) -> None:
        """Step through CUDA graphs on `stream` (a torch.cuda.Stream)."""
        lbm_set_stream(self.h, stream.cuda_stream)
        lbm_set_graph(self.h, steps_per_graph)
