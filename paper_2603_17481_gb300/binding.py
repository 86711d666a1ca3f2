"""ctypes binding of the C ABI in include/lbm.h (same function names; argument marshalling only).

Every computation runs in liblbm.so. Host arrays are FP64 and may be numpy arrays or CPU torch
tensors (e.g. pinned buffers); they are checked for dtype, size and contiguity and passed by
pointer. Errors raise :class:`LbmError` carrying the library's status code. If the library is
missing, :func:`load` raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_UNSTABLE, LBM_ERR_STATE = 0, -1, -2, -3, -4, -5
LBM_STORE_F32, LBM_STORE_F16, LBM_STORE_BF16, LBM_STORE_MOMENTS = 0, 1, 2, 3
STORES = {"f32": LBM_STORE_F32, "f16": LBM_STORE_F16, "bf16": LBM_STORE_BF16, "mom": LBM_STORE_MOMENTS}
KERNEL_KINDS = ("nci", "hydro", "phase", "reduce", "convert")
NO_PARTNER = np.iinfo(np.int32).min


class LbmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {lbm_strerror(code)} ({code})")


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("Q", ctypes.c_int), ("store", ctypes.c_int),
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("nu_l", ctypes.c_double), ("nu_g", ctypes.c_double),
        ("sigma", ctypes.c_double), ("eps", ctypes.c_double), ("D", ctypes.c_double),
        ("nci_on", ctypes.c_int), ("w", ctypes.c_int),
        ("A_rep", ctypes.c_double), ("h0", ctypes.c_double), ("p", ctypes.c_double),
        ("q_th", ctypes.c_double), ("eta", ctypes.c_double), ("cos_opp", ctypes.c_double),
        ("eps_q", ctypes.c_double), ("eps_n", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("mass_check_every", ctypes.c_int), ("mass_tol", ctypes.c_double),
    ]


_lib = None
_VP = ctypes.c_void_p


def load():
    """Loads liblbm.so (built by ``paper_2603_17481_gb300.build``); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2603_17481_gb300.build.build() "
                           "(nvcc, sm_103a); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER(lbm_params)
    L.lbm_params_default.argtypes = [P]
    L.lbm_params_default.restype = None
    L.lbm_create.argtypes = [P, ctypes.POINTER(_VP)]
    L.lbm_destroy.argtypes = [_VP]
    L.lbm_destroy.restype = None
    L.lbm_set_stream.argtypes = [_VP, _VP]
    L.lbm_init_fields.argtypes = [_VP, _VP, _VP, _VP]
    L.lbm_set_state.argtypes = [_VP, _VP, _VP]
    L.lbm_get_state.argtypes = [_VP, _VP, _VP]
    L.lbm_step.argtypes = [_VP, ctypes.c_int]
    L.lbm_set_overlap.argtypes = [_VP, ctypes.c_int]
    L.lbm_get_overlap.argtypes = [_VP, _VP]
    L.lbm_read_fields.argtypes = [_VP, _VP, _VP, _VP]
    L.lbm_mass.argtypes = [_VP, _VP, _VP]
    L.lbm_read_nci.argtypes = [_VP, _VP, _VP]
    L.lbm_mass_noalloc.argtypes = [_VP, _VP, _VP]
    L.lbm_nci_diagnostics.argtypes = [_VP, _VP]
    L.lbm_curvature.argtypes = [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_int, _VP, _VP]
    L.lbm_energy_spectrum.argtypes = [_VP, ctypes.c_int, _VP]
    L.lbm_batch_create.argtypes = [_VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.POINTER(_VP)]
    L.lbm_batch_create_ex.argtypes = [_VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int, ctypes.POINTER(_VP)]
    L.lbm_batch_config.argtypes = [_VP, _VP, _VP]
    L.lbm_batch_step.argtypes = [_VP, ctypes.c_int]
    L.lbm_batch_synchronize.argtypes = [_VP]
    L.lbm_batch_destroy.argtypes = [_VP]
    L.lbm_batch_destroy.restype = None
    L.lbm_synchronize.argtypes = [_VP]
    L.lbm_profile.argtypes = [_VP, ctypes.c_int]
    L.lbm_profile_kinds.argtypes = [_VP, ctypes.c_uint]
    L.lbm_profile_sample.argtypes = [_VP, ctypes.c_int]
    L.lbm_profile_read.argtypes = [_VP, _VP, _VP]
    L.lbm_lattice.argtypes = [ctypes.c_int, ctypes.c_int, _VP, _VP]
    L.lbm_strerror.argtypes = [ctypes.c_int]
    L.lbm_strerror.restype = ctypes.c_char_p
    L.lbm_kernel_name.argtypes = [ctypes.c_int]
    L.lbm_kernel_name.restype = ctypes.c_char_p
    for name in ("lbm_create", "lbm_set_stream", "lbm_init_fields", "lbm_set_state", "lbm_get_state",
                 "lbm_step", "lbm_set_overlap", "lbm_get_overlap", "lbm_read_fields", "lbm_mass", "lbm_mass_noalloc", "lbm_read_nci", "lbm_synchronize",
                 "lbm_profile", "lbm_profile_kinds", "lbm_profile_sample", "lbm_profile_read", "lbm_lattice", "lbm_batch_create", "lbm_batch_step",
                 "lbm_batch_create_ex", "lbm_batch_config",
                 "lbm_nci_diagnostics", "lbm_curvature", "lbm_energy_spectrum",
                 "lbm_batch_synchronize"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int, where: str):
    if rc != LBM_OK:
        raise LbmError(rc, where)


def _ptr(a, n: int, dtype, name: str, writable: bool = False):
    """Pointer to a host buffer of n elements of dtype (numpy array or CPU torch tensor)."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if a.is_cuda or not a.is_contiguous() or a.numel() != n or a.element_size() != np.dtype(dtype).itemsize:
            raise ValueError(f"{name}: need a contiguous CPU tensor of {n} x {np.dtype(dtype).name}")
        return a.data_ptr(), a
    arr = np.asarray(a)
    if arr.dtype != dtype or not arr.flags["C_CONTIGUOUS"] or (writable and not arr.flags["WRITEABLE"]):
        if writable:
            raise ValueError(f"{name}: need a writable C-contiguous {np.dtype(dtype).name} array")
        arr = np.ascontiguousarray(arr, dtype=dtype)
    if arr.size != n:
        raise ValueError(f"{name}: expected {n} elements, got {arr.size}")
    return arr.ctypes.data, arr


def lbm_strerror(code: int) -> str:
    return load().lbm_strerror(int(code)).decode()


def lbm_kernel_name(kind: int) -> str:
    return load().lbm_kernel_name(int(kind)).decode()


def lbm_params_default() -> lbm_params:
    p = lbm_params()
    load().lbm_params_default(ctypes.byref(p))
    return p


def params_from_config(cfg: dict, store="f32", mass_check_every=0, mass_tol=1e-9) -> lbm_params:
    """lbm_params from a workload configuration dict (keys as in workloads.base_config)."""
    p = lbm_params_default()
    for k in ("dim", "nx", "ny", "nz", "Q", "nci_on", "w"):
        setattr(p, k, int(cfg[k]))
    for k in ("rho_l", "rho_g", "nu_l", "nu_g", "sigma", "eps", "D", "A_rep", "h0", "p", "q_th", "eta",
              "cos_opp", "eps_q", "eps_n"):
        setattr(p, k, float(cfg[k]))
    p.g = (ctypes.c_double * 3)(*[float(v) for v in cfg.get("g", (0.0, 0.0, 0.0))])
    p.store = STORES[store] if isinstance(store, str) else int(store)
    p.mass_check_every = int(mass_check_every)
    p.mass_tol = float(mass_tol)
    return p


def lbm_create(params: lbm_params) -> int:
    h = _VP()
    _check(load().lbm_create(ctypes.byref(params), ctypes.byref(h)), "lbm_create")
    return h.value


def lbm_destroy(ctx: int) -> None:
    if ctx:
        load().lbm_destroy(_VP(ctx))


def lbm_set_stream(ctx: int, stream: int) -> None:
    _check(load().lbm_set_stream(_VP(ctx), _VP(stream or 0)), "lbm_set_stream")


def lbm_init_fields(ctx: int, N: int, phi, u, pstar=None) -> None:
    pp, _a = _ptr(phi, N, np.float64, "phi")
    pu, _b = _ptr(u, 3 * N, np.float64, "u")
    ps, _c = _ptr(pstar, N, np.float64, "pstar")
    _check(load().lbm_init_fields(_VP(ctx), pp, pu, ps), "lbm_init_fields")


def lbm_set_state(ctx: int, N: int, Q: int, f, phi) -> None:
    pf, _a = _ptr(f, Q * N, np.float64, "f")
    pp, _b = _ptr(phi, N, np.float64, "phi")
    _check(load().lbm_set_state(_VP(ctx), pf, pp), "lbm_set_state")


def lbm_get_state(ctx: int, N: int, Q: int):
    f = np.empty((Q, N))
    phi = np.empty(N)
    _check(load().lbm_get_state(_VP(ctx), f.ctypes.data, phi.ctypes.data), "lbm_get_state")
    return f, phi


def lbm_step(ctx: int, n: int) -> None:
    _check(load().lbm_step(_VP(ctx), int(n)), "lbm_step")


def lbm_set_overlap(ctx: int, blocks: int) -> None:
    _check(load().lbm_set_overlap(_VP(ctx), int(blocks)), "lbm_set_overlap")


def lbm_get_overlap(ctx: int) -> int:
    b = ctypes.c_int(0)
    _check(load().lbm_get_overlap(_VP(ctx), ctypes.byref(b)), "lbm_get_overlap")
    return b.value


def lbm_read_fields(ctx: int, N: int, phi=None, u=None, pstar=None, want=("phi", "u", "pstar")):
    """Reads phi (N), u (3, N), p* (N); pre-allocated outputs may be passed (numpy or CPU tensors)."""
    if phi is None and "phi" in want:
        phi = np.empty(N)
    if u is None and "u" in want:
        u = np.empty((3, N))
    if pstar is None and "pstar" in want:
        pstar = np.empty(N)
    p1, _a = _ptr(phi, N, np.float64, "phi", True)
    p2, _b = _ptr(u, 3 * N, np.float64, "u", True)
    p3, _c = _ptr(pstar, N, np.float64, "pstar", True)
    _check(load().lbm_read_fields(_VP(ctx), p1, p2, p3), "lbm_read_fields")
    return phi, u, pstar


def lbm_mass(ctx: int):
    m = ctypes.c_double()
    mom = (ctypes.c_double * 3)()
    _check(load().lbm_mass(_VP(ctx), ctypes.addressof(m), ctypes.addressof(mom)), "lbm_mass")
    return m.value, np.array(list(mom))


def lbm_mass_noalloc(ctx: int):
    """lbm_mass without device allocation (static scratch; see include/lbm.h for its limits)."""
    m = ctypes.c_double()
    mom = (ctypes.c_double * 3)()
    _check(load().lbm_mass_noalloc(_VP(ctx), ctypes.addressof(m), ctypes.addressof(mom)), "lbm_mass_noalloc")
    return m.value, np.array(list(mom))


def lbm_read_nci(ctx: int, N: int):
    part = np.empty((N, 3), dtype=np.int32)
    frep = np.empty((3, N))
    _check(load().lbm_read_nci(_VP(ctx), part.ctypes.data, frep.ctypes.data), "lbm_read_nci")
    return part, frep


DIAG_KEYS = ("V_film", "sum_rep_n", "sum_cap_n", "max_rep", "sum_rep", "R_n", "mean_rep")


def lbm_nci_diagnostics(ctx: int) -> dict:
    out = np.zeros(7)
    _check(load().lbm_nci_diagnostics(_VP(ctx), out.ctypes.data_as(_VP)), "lbm_nci_diagnostics")
    return dict(zip(DIAG_KEYS, (float(v) for v in out)))


def lbm_curvature(ctx: int, kmin: float, kmax: float, nbins: int) -> dict:
    hist = np.zeros(max(nbins, 0), dtype=np.int64)
    out = np.zeros(2)
    _check(load().lbm_curvature(_VP(ctx), float(kmin), float(kmax), int(nbins),
                                hist.ctypes.data_as(_VP) if nbins > 0 else None, out.ctypes.data_as(_VP)),
           "lbm_curvature")
    return {"band_cells": float(out[0]), "mean": float(out[1]), "hist": hist}


def lbm_energy_spectrum(ctx: int, nshells: int) -> np.ndarray:
    E = np.zeros(int(nshells))
    _check(load().lbm_energy_spectrum(_VP(ctx), int(nshells), E.ctypes.data_as(_VP)), "lbm_energy_spectrum")
    return E


def lbm_synchronize(ctx: int) -> None:
    _check(load().lbm_synchronize(_VP(ctx)), "lbm_synchronize")


def lbm_profile(ctx: int, enable: bool) -> None:
    _check(load().lbm_profile(_VP(ctx), int(bool(enable))), "lbm_profile")


def lbm_profile_kinds(ctx: int, kinds) -> None:
    """Times only the named kernel kinds (names of KERNEL_KINDS); an empty list stops the profiler."""
    mask = 0
    for k in kinds:
        mask |= 1 << KERNEL_KINDS.index(k)
    _check(load().lbm_profile_kinds(_VP(ctx), mask), "lbm_profile_kinds")


def lbm_profile_sample(ctx: int, every: int) -> None:
    _check(load().lbm_profile_sample(_VP(ctx), int(every)), "lbm_profile_sample")


def lbm_profile_read(ctx: int):
    ms = np.zeros(len(KERNEL_KINDS))
    n = np.zeros(len(KERNEL_KINDS), dtype=np.int64)
    _check(load().lbm_profile_read(_VP(ctx), ms.ctypes.data, n.ctypes.data), "lbm_profile_read")
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_KINDS)}


def lbm_lattice(dim: int, Q: int):
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    _check(load().lbm_lattice(int(dim), int(Q), c.ctypes.data, w.ctypes.data), "lbm_lattice")
    return c, w


LBM_BATCH_PER_CASE, LBM_BATCH_NO_TUNE, LBM_BATCH_HYDRO_TY2, LBM_BATCH_HYDRO_TY8, LBM_BATCH_PHASE_ROWS2 = 1, 2, 4, 8, 16


def lbm_batch_create(ctxs, nstreams: int = 8, stream: int = 0) -> int:
    arr = (_VP * len(ctxs))(*[_VP(c) for c in ctxs])
    h = _VP()
    _check(load().lbm_batch_create(arr, len(ctxs), int(nstreams), _VP(stream or None), ctypes.byref(h)),
           "lbm_batch_create")
    return h.value


def lbm_batch_create_ex(ctxs, nstreams: int = 8, stream: int = 0, flags: int = 0) -> int:
    arr = (_VP * len(ctxs))(*[_VP(c) for c in ctxs])
    h = _VP()
    _check(load().lbm_batch_create_ex(arr, len(ctxs), int(nstreams), _VP(stream or None), int(flags),
                                      ctypes.byref(h)), "lbm_batch_create_ex")
    return h.value


def lbm_batch_config(batch: int) -> dict:
    cfg = np.zeros(8, dtype=np.int32)
    ms = np.zeros(7)
    _check(load().lbm_batch_config(_VP(batch), cfg.ctypes.data_as(_VP), ms.ctypes.data_as(_VP)), "lbm_batch_config")
    keys = ("fused", "hydro_ty", "hydro_tz", "phase_rows", "branches", "hydro_blocks", "phase_blocks", "hydro_items")
    d = {k: int(v) for k, v in zip(keys, cfg)}
    d["tune_ms"] = {"hydro_ty4": float(ms[0]), "hydro_ty2": float(ms[1]), "hydro_ty8": float(ms[2]),
                    "phase_rows4": float(ms[3]), "phase_rows2": float(ms[4]),
                    "step_fused": float(ms[5]), "step_per_case": float(ms[6])}
    return d


def lbm_batch_step(batch: int, n: int) -> None:
    _check(load().lbm_batch_step(_VP(batch), int(n)), "lbm_batch_step")


def lbm_batch_synchronize(batch: int) -> None:
    _check(load().lbm_batch_synchronize(_VP(batch)), "lbm_batch_synchronize")


def lbm_batch_destroy(batch: int) -> None:
    if batch:
        load().lbm_batch_destroy(_VP(batch))


class LbmBatch:
    """Independent contexts advanced together through one CUDA graph (keeps the contexts alive)."""

    def __init__(self, sims, nstreams: int = 8, stream: int = 0, flags: int = 0):
        self.sims = list(sims)
        self.h = lbm_batch_create_ex([s.ctx for s in self.sims], nstreams, stream, flags)

    def config(self) -> dict:
        return lbm_batch_config(self.h)

    def step(self, n: int = 2, sync: bool = True):
        """Advances every context by n steps; with ``sync`` waits for the work (so that the
        contexts' own reads may follow)."""
        lbm_batch_step(self.h, n)
        if sync:
            lbm_batch_synchronize(self.h)

    def synchronize(self):
        lbm_batch_synchronize(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lbm:
    """One simulation context (owns its device memory; destroyed with the object)."""

    def __init__(self, cfg: dict, store="f32", mass_check_every=0, mass_tol=1e-9, stream=None):
        self.cfg = dict(cfg)
        self.params = params_from_config(cfg, store, mass_check_every, mass_tol)
        self.N = cfg["nx"] * cfg["ny"] * cfg["nz"]
        self.Q = cfg["Q"]
        self.ctx = lbm_create(self.params)
        if stream is not None:
            lbm_set_stream(self.ctx, stream)

    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: int):
        lbm_set_stream(self.ctx, stream)

    def init_fields(self, phi, u, pstar=None):
        lbm_init_fields(self.ctx, self.N, phi, u, pstar)

    def set_state(self, f, phi):
        lbm_set_state(self.ctx, self.N, self.Q, f, phi)

    def get_state(self):
        return lbm_get_state(self.ctx, self.N, self.Q)

    def step(self, n: int = 1):
        lbm_step(self.ctx, n)

    def set_overlap(self, blocks: int):
        lbm_set_overlap(self.ctx, blocks)

    def overlap(self) -> int:
        return lbm_get_overlap(self.ctx)

    def read_fields(self, **kw):
        return lbm_read_fields(self.ctx, self.N, **kw)

    def mass(self):
        return lbm_mass(self.ctx)

    def mass_noalloc(self):
        return lbm_mass_noalloc(self.ctx)

    def read_nci(self):
        return lbm_read_nci(self.ctx, self.N)

    def synchronize(self):
        lbm_synchronize(self.ctx)

    def nci_diagnostics(self):
        return lbm_nci_diagnostics(self.ctx)

    def curvature(self, kmin: float, kmax: float, nbins: int):
        return lbm_curvature(self.ctx, kmin, kmax, nbins)

    def energy_spectrum(self, nshells: int):
        return lbm_energy_spectrum(self.ctx, nshells)

    def profile(self, enable=True):
        lbm_profile(self.ctx, enable)

    def profile_kinds(self, kinds):
        lbm_profile_kinds(self.ctx, kinds)

    def profile_sample(self, every: int):
        lbm_profile_sample(self.ctx, every)

    def profile_read(self):
        return lbm_profile_read(self.ctx)
