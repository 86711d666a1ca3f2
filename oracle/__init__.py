"""FP64 CPU oracle of the per-time-step lattice update of arXiv 2603.17481 (ctypes wrapper).

TEST INFRASTRUCTURE. This package is the correctness reference of the CUDA library, not part of
the product. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it. It shares no code with ``paper_2603_17481_gb300``: the C source
(``lbm_oracle.c``) restates the paper's equations in plain FP64 loops and this module only
marshals numpy arrays in and out of it.

Array conventions: cell index ``n = x + nx*(y + ny*z)``; populations ``f[i, n]`` (shape ``(Q, N)``),
vectors ``v[a, n]`` (shape ``(3, N)``, z row zero in 2D).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_HDR = os.path.join(_HERE, "lbm_oracle.h")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

NO_PARTNER = np.iinfo(np.int32).min


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liborc.so`` with gcc (portable flags, no FMA contraction)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("Q", ctypes.c_int),
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("nu_l", ctypes.c_double), ("nu_g", ctypes.c_double),
        ("sigma", ctypes.c_double), ("eps", ctypes.c_double), ("D", ctypes.c_double),
        ("nci_on", ctypes.c_int), ("w", ctypes.c_int),
        ("A_rep", ctypes.c_double), ("h0", ctypes.c_double), ("p", ctypes.c_double),
        ("q_th", ctypes.c_double), ("eta", ctypes.c_double), ("cos_opp", ctypes.c_double),
        ("eps_q", ctypes.c_double), ("eps_n", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("rho_bar", ctypes.c_double),
        ("decide_f32", ctypes.c_int),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_P = ctypes.POINTER(OrcParams)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_lattice.argtypes = [ctypes.c_int, ctypes.c_int, _I, _D]
            L.orc_feq.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _D, _D]
            L.orc_guo.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D]
            L.orc_regularized.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D]
            L.orc_hydro_cell.argtypes = [_P, _D, ctypes.c_double, _D, ctypes.c_double, _D, _D, _D, _D]
            L.orc_grad_iso.argtypes = [_P, _D, _D]
            L.orc_lap_iso.argtypes = [_P, _D, _D]
            L.orc_minmod.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_minmod.restype = ctypes.c_double
            L.orc_h_of_q.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_h_of_q.restype = ctypes.c_double
            L.orc_w_h.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.orc_w_h.restype = ctypes.c_double
            L.orc_nci.argtypes = [_P, _D, _I, _D, _D]
            L.orc_phi_update.argtypes = [_P, _D, _D, _D]
            L.orc_init.argtypes = [_P, _D, _D, _D, _D]
            L.orc_mean_density.argtypes = [_P, _D]
            L.orc_mean_density.restype = ctypes.c_double
            L.orc_moments.argtypes = [_P, _D, _D, _D, _D]
            L.orc_step.argtypes = [_P, _D, _D, ctypes.c_int, _D]
            L.orc_step.restype = ctypes.c_int
            L.orc_nci_diagnostics.argtypes = [_P, _D, _D]
            L.orc_nci_diagnostics.restype = ctypes.c_int
            L.orc_curvature.argtypes = [_P, _D, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_longlong), _D]
            L.orc_curvature.restype = ctypes.c_int
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


_FIELDS = [f[0] for f in OrcParams._fields_]


def make_params(cfg: dict) -> OrcParams:
    """Build the oracle's parameter struct from a plain configuration dict."""
    P = OrcParams()
    for k in _FIELDS:
        if k == "g":
            g = tuple(cfg.get("g", (0.0, 0.0, 0.0)))
            P.g = (ctypes.c_double * 3)(*[float(v) for v in g])
        elif k in ("rho_bar", "decide_f32"):
            continue
        else:
            setattr(P, k, type(getattr(P, k))(cfg[k]))
    P.rho_bar = float(cfg.get("rho_bar", 0.0))
    P.decide_f32 = int(cfg.get("decide_f32", 1))
    return P


def ncells(P: OrcParams) -> int:
    return P.nx * P.ny * P.nz


def lattice(dim: int, Q: int):
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q, dtype=np.float64)
    rc = lib().orc_lattice(dim, Q, c.ctypes.data_as(_I), _d(w))
    if rc:
        raise ValueError(f"unsupported lattice D{dim}Q{Q}")
    return c, w


def feq(dim: int, Q: int, pstar: float, u) -> np.ndarray:
    u = _f64(u, (3,))
    out = np.zeros(Q)
    lib().orc_feq(dim, Q, float(pstar), _d(u), _d(out))
    return out


def guo(dim: int, Q: int, u, Fr) -> np.ndarray:
    u = _f64(u, (3,))
    Fr = _f64(Fr, (3,))
    out = np.zeros(Q)
    lib().orc_guo(dim, Q, _d(u), _d(Fr), _d(out))
    return out


def regularized(dim: int, Q: int, u, A2) -> np.ndarray:
    u = _f64(u, (3,))
    A2 = _f64(A2, (9,))
    out = np.zeros(Q)
    lib().orc_regularized(dim, Q, _d(u), _d(A2), _d(out))
    return out


def hydro_cell(P: OrcParams, f, phi: float, gphi, lphi: float, frep=(0.0, 0.0, 0.0)):
    f = _f64(f, (P.Q,))
    g = _f64(gphi, (3,))
    fr = _f64(frep, (3,))
    fpost = np.zeros(P.Q)
    u = np.zeros(3)
    ps = np.zeros(1)
    lib().orc_hydro_cell(ctypes.byref(P), _d(f), float(phi), _d(g), float(lphi), _d(fr),
                         _d(fpost), _d(u), _d(ps))
    return fpost, u, float(ps[0])


def grad_iso(P: OrcParams, psi) -> np.ndarray:
    psi = _f64(psi, (ncells(P),))
    out = np.zeros((3, ncells(P)))
    lib().orc_grad_iso(ctypes.byref(P), _d(psi), _d(out))
    return out


def lap_iso(P: OrcParams, psi) -> np.ndarray:
    psi = _f64(psi, (ncells(P),))
    out = np.zeros(ncells(P))
    lib().orc_lap_iso(ctypes.byref(P), _d(psi), _d(out))
    return out


def minmod(a: float, b: float) -> float:
    return lib().orc_minmod(float(a), float(b))


def h_of_q(q: float, eps: float) -> float:
    return lib().orc_h_of_q(float(q), float(eps))


def w_h(h: float, h0: float = 1.0, p: float = 4.0) -> float:
    return lib().orc_w_h(float(h), float(h0), float(p))


def nci(P: OrcParams, phi):
    """Returns (partner (N,3) int32 with NO_PARTNER where chi = 0, frep (3,N), margin (N,))."""
    N = ncells(P)
    phi = _f64(phi, (N,))
    part = np.zeros((N, 3), dtype=np.int32)
    frep = np.zeros((3, N))
    marg = np.zeros(N)
    lib().orc_nci(ctypes.byref(P), _d(phi), part.ctypes.data_as(_I), _d(frep), _d(marg))
    return part, frep, marg


def nci_diagnostics(P: OrcParams, phi) -> dict:
    """Film statistics of Sec. 3.3 on phi: V_film, sum |F_rep.n|, sum |F_cap.n|, max |F_rep|,
    sum |F_rep|, and from them R_n (Eq. 74; 0 when there is no film) and the film mean of |F_rep|."""
    N = ncells(P)
    phi = _f64(phi, (N,))
    out = np.zeros(5)
    if lib().orc_nci_diagnostics(ctypes.byref(P), _d(phi), _d(out)):
        raise MemoryError("oracle diagnostics failed to allocate")
    v, srn, scn, fmax, sabs = (float(x) for x in out)
    return {"V_film": v, "sum_rep_n": srn, "sum_cap_n": scn, "max_rep": fmax, "sum_rep": sabs,
            "R_n": srn / scn if scn > 0 else 0.0, "mean_rep": sabs / v if v > 0 else 0.0}


def curvature(P: OrcParams, phi, kmin: float, kmax: float, nbins: int):
    """Band cells, mean curvature and the histogram of kappa = div n (Eq. 78) on [kmin, kmax)."""
    N = ncells(P)
    phi = _f64(phi, (N,))
    hist = np.zeros(nbins, dtype=np.int64)
    out = np.zeros(2)
    if lib().orc_curvature(ctypes.byref(P), _d(phi), float(kmin), float(kmax), int(nbins),
                           hist.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), _d(out)):
        raise MemoryError("oracle curvature failed")
    n = float(out[0])
    return {"band_cells": n, "mean": float(out[1]) / n if n > 0 else 0.0, "hist": hist}


def energy_spectrum(P: OrcParams, phi, u, nshells: int) -> np.ndarray:
    """Carrier-phase kinetic-energy spectrum (Sec. 3.4), numpy FFT as the transform.

    The carrier phase is the liquid, chi = 1 where phi >= 1/2 (reading R23). The fluctuation is
    u' = chi (u - <u>_liquid) and u_hat(k) = (1/N) sum_x u'(x) exp(-i k.x) per component, so that
    sum_k |u_hat|^2 = <|u'|^2> (Parseval). With k_a = 2 pi m_a / n_a and the shell width
    2 pi / max(n_a), E(K) = sum over k with floor(|k| / width + 1/2) = K of |u_hat(k)|^2 / 2.
    Returns E for K = 0 .. nshells - 1 (energy beyond the last shell is not returned).
    """
    nx, ny, nz = P.nx, P.ny, P.nz
    N = nx * ny * nz
    phi = _f64(phi, (N,))
    u = _f64(u, (3, N))
    chi = (phi >= 0.5).astype(np.float64)
    ubar = (u * chi).sum(axis=1) / max(chi.sum(), 1.0)
    up = chi * (u - ubar[:, None])
    # |k| in units of the shell width: m_a M / n_a with M = max(n_a), exact for the half-integer
    # ties of boxes such as 96 x 64, which round up
    M = max(nx, ny, nz)
    m = [np.fft.fftfreq(n, 1.0 / n) for n in (nz, ny, nx)]
    kk = np.sqrt(sum((mm * M / n)[tuple(slice(None) if i == j else None for j in range(3))] ** 2
                     for i, (mm, n) in enumerate(zip(m, (nz, ny, nx)))))
    shell = np.floor(kk + 0.5).astype(np.int64)
    E = np.zeros(nshells)
    for a in range(3):
        uh = np.fft.fftn(up[a].reshape(nz, ny, nx)) / N
        e = 0.5 * (uh.real ** 2 + uh.imag ** 2)
        ok = shell < nshells
        E += np.bincount(shell[ok], weights=e[ok], minlength=nshells)[:nshells]
    return E


def phi_update(P: OrcParams, phi, u) -> np.ndarray:
    N = ncells(P)
    phi = _f64(phi, (N,))
    u = _f64(u, (3, N))
    out = np.zeros(N)
    lib().orc_phi_update(ctypes.byref(P), _d(phi), _d(u), _d(out))
    return out


def mean_density(P: OrcParams, phi) -> float:
    phi = _f64(phi, (ncells(P),))
    return lib().orc_mean_density(ctypes.byref(P), _d(phi))


def init(P: OrcParams, phi, u, pstar=None) -> np.ndarray:
    """Equilibrium initial populations; also sets ``P.rho_bar`` from phi."""
    N = ncells(P)
    phi = _f64(phi, (N,))
    u = _f64(u, (3, N))
    f = np.zeros((P.Q, N))
    ps = None if pstar is None else _f64(pstar, (N,))
    P.rho_bar = mean_density(P, phi)
    lib().orc_init(ctypes.byref(P), _d(phi), _d(u), None if ps is None else _d(ps), _d(f))
    return f


def moments(P: OrcParams, f, phi):
    N = ncells(P)
    f = _f64(f, (P.Q, N))
    phi = _f64(phi, (N,))
    ps = np.zeros(N)
    u = np.zeros((3, N))
    lib().orc_moments(ctypes.byref(P), _d(f), _d(phi), _d(ps), _d(u))
    return ps, u


def step(P: OrcParams, f, phi, nsteps: int):
    """Advance in place on copies; returns (f, phi, u_last)."""
    N = ncells(P)
    f = np.array(f, dtype=np.float64, order="C").reshape(P.Q, N)
    phi = np.array(phi, dtype=np.float64, order="C").reshape(N)
    u = np.zeros((3, N))
    rc = lib().orc_step(ctypes.byref(P), _d(f), _d(phi), int(nsteps), _d(u))
    if rc:
        raise MemoryError("oracle step failed to allocate")
    return f, phi, u
