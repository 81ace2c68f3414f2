"""ctypes wrapper of the plain FP64 CPU oracle (``ns3d_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``, and by
nothing else.  It shares no code with the CUDA path (``paper_2211_16718_gb300``)
and never imports it.

Every function takes and returns NumPy float64 arrays.  The state layout is
``u[5, nz, ny, nx]`` (rho, rho*u, rho*v, rho*w, e), x fastest, on the triply
periodic grid x_i = i*dx, dx = lx/nx (arXiv 2211.16718, Sec. 2.1-2.2).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ns3d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBPATH = os.path.join(_BUILD, "libns3d_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, OpenMP if available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIBPATH) and os.path.getmtime(_LIBPATH) >= os.path.getmtime(_SRC):
        return _LIBPATH
    base = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    tmp = _LIBPATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


class _CParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("weno_p", ctypes.c_int), ("weno_linear", ctypes.c_int), ("roe_state", ctypes.c_int),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
        ("gamma", ctypes.c_double), ("mu_eff", ctypes.c_double), ("prandtl", ctypes.c_double),
        ("weno_eps", ctypes.c_double), ("harten_delta", ctypes.c_double),
    ]


@dataclasses.dataclass
class Params:
    """Oracle parameters (defaults: the paper's gamma, Pr and eps; Sec. 2.1-2.2)."""
    nx: int
    ny: int
    nz: int
    lx: float = 2.0 * math.pi
    ly: float = 2.0 * math.pi
    lz: float = 2.0 * math.pi
    gamma: float = 1.4
    mu_eff: float = 0.0
    prandtl: float = 0.72
    weno_eps: float = 1e-6
    weno_p: int = 2
    weno_linear: int = 0
    roe_state: int = 0
    harten_delta: float = 0.1

    def c(self) -> _CParams:
        return _CParams(self.nx, self.ny, self.nz, self.weno_p, self.weno_linear, self.roe_state,
                        self.lx, self.ly, self.lz, self.gamma, self.mu_eff, self.prandtl,
                        self.weno_eps, self.harten_delta)

    @property
    def shape(self):
        return (5, self.nz, self.ny, self.nx)


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_L = ctypes.c_long
RHS_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            pp = ctypes.POINTER(_CParams)
            sig = {
                "orc_set_threads": (None, [_I]),
                "orc_get_threads": (_I, []),
                "orc_has_openmp": (_I, []),
                "orc_flux": (None, [_P, _I, _D, _P]),
                "orc_weno5_candidates": (None, [_P, _P]),
                "orc_weno5_beta": (None, [_P, _P]),
                "orc_weno5_weights": (None, [_P, _D, _I, _I, _P]),
                "orc_weno5": (_D, [_P, _D, _I, _I]),
                "orc_weno5_line": (None, [_P, _I, _D, _I, _I, _P, _P]),
                "orc_roe_matrix": (None, [_P, _P, _I, _D, _I, _D, _P]),
                "orc_roe_eigensystem": (None, [_P, _P, _I, _D, _P, _P, _P]),
                "orc_interface_flux": (None, [pp, _I, _P, _P]),
                "orc_rhs": (None, [pp, _P, _P]),
                "orc_rhs_hyp": (None, [pp, _P, _P]),
                "orc_rhs_visc": (None, [pp, _P, _P]),
                "orc_rhs_points": (None, [pp, _P, _L, _P, _P]),
                "orc_rk_generic": (None, [_L, _P, _D, _I, RHS_FN, _P]),
                "orc_rk_step": (None, [pp, _P, _D, _I, _I]),
                "orc_stats": (None, [pp, _P, _P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def has_openmp() -> bool:
    return bool(lib().orc_has_openmp())


# ---- pointwise building blocks (for pins) -----------------------------------
def flux(U, d: int, gamma: float = 1.4) -> np.ndarray:
    U = _f64(U)
    F = np.zeros(5)
    lib().orc_flux(_ptr(U), d, gamma, _ptr(F))
    return F


def weno5_candidates(q) -> np.ndarray:
    q = _f64(q)
    out = np.zeros(3)
    lib().orc_weno5_candidates(_ptr(q), _ptr(out))
    return out


def weno5_beta(q) -> np.ndarray:
    q = _f64(q)
    out = np.zeros(3)
    lib().orc_weno5_beta(_ptr(q), _ptr(out))
    return out


def weno5_weights(q, eps: float = 1e-6, p: int = 2, linear: bool = False) -> np.ndarray:
    q = _f64(q)
    out = np.zeros(3)
    lib().orc_weno5_weights(_ptr(q), eps, p, int(linear), _ptr(out))
    return out


def weno5(q, eps: float = 1e-6, p: int = 2, linear: bool = False) -> float:
    q = _f64(q)
    return float(lib().orc_weno5(_ptr(q), eps, p, int(linear)))


def weno5_line(q, eps: float = 1e-6, p: int = 2, linear: bool = False):
    q = _f64(q)
    qL = np.zeros_like(q)
    qR = np.zeros_like(q)
    lib().orc_weno5_line(_ptr(q), q.size, eps, p, int(linear), _ptr(qL), _ptr(qR))
    return qL, qR


def roe_matrix(UL, UR, d: int, gamma: float = 1.4, absval: bool = False, harten_delta: float = 0.0):
    UL, UR = _f64(UL), _f64(UR)
    A = np.zeros(25)
    lib().orc_roe_matrix(_ptr(UL), _ptr(UR), d, gamma, int(absval), harten_delta, _ptr(A))
    return A.reshape(5, 5)


def roe_eigensystem(UL, UR, d: int, gamma: float = 1.4):
    UL, UR = _f64(UL), _f64(UR)
    X, Xi, lam = np.zeros(25), np.zeros(25), np.zeros(5)
    lib().orc_roe_eigensystem(_ptr(UL), _ptr(UR), d, gamma, _ptr(X), _ptr(Xi), _ptr(lam))
    return X.reshape(5, 5), Xi.reshape(5, 5), lam


def interface_flux(P: Params, d: int, us) -> np.ndarray:
    """Roe/WENO5 flux at interface i+1/2 from the 6 point states i-2..i+3 (6x5)."""
    us = _f64(us).reshape(6, 5)
    out = np.zeros(5)
    cp = P.c()
    lib().orc_interface_flux(ctypes.byref(cp), d, _ptr(us), _ptr(out))
    return out


# ---- whole-grid operators ---------------------------------------------------
def _check_state(P: Params, u) -> np.ndarray:
    u = _f64(u)
    if u.shape != P.shape:
        raise ValueError(f"state shape {u.shape} != {P.shape}")
    return u


def rhs(P: Params, u) -> np.ndarray:
    u = _check_state(P, u)
    r = np.empty_like(u)
    cp = P.c()
    lib().orc_rhs(ctypes.byref(cp), _ptr(u), _ptr(r))
    return r


def rhs_hyp(P: Params, u) -> np.ndarray:
    u = _check_state(P, u)
    r = np.empty_like(u)
    cp = P.c()
    lib().orc_rhs_hyp(ctypes.byref(cp), _ptr(u), _ptr(r))
    return r


def rhs_visc(P: Params, u) -> np.ndarray:
    u = _check_state(P, u)
    r = np.empty_like(u)
    cp = P.c()
    lib().orc_rhs_visc(ctypes.byref(cp), _ptr(u), _ptr(r))
    return r


def rhs_points(P: Params, u, flat_idx) -> np.ndarray:
    """RHS at selected flat point indices (k*ny + j)*nx + i; returns [npts, 5]."""
    u = _check_state(P, u)
    idx = np.ascontiguousarray(flat_idx, dtype=np.int64)
    out = np.zeros((idx.size, 5))
    cp = P.c()
    lib().orc_rhs_points(ctypes.byref(cp), _ptr(u), idx.size, idx.ctypes.data_as(ctypes.c_void_p), _ptr(out))
    return out


def rk_step(P: Params, u, dt: float, nsteps: int = 1, scheme: str = "rk4") -> np.ndarray:
    u = _check_state(P, u).copy()
    cp = P.c()
    lib().orc_rk_step(ctypes.byref(cp), _ptr(u), dt, nsteps, 0 if scheme == "rk4" else 1)
    return u


def rk_generic(u, dt: float, fn, scheme: str = "rk4") -> np.ndarray:
    """One RK step of du/dt = fn(u) for an arbitrary Python right-hand side."""
    u = _f64(u).copy()
    n = u.size

    def cb(_ctx, up, rp):
        uin = np.ctypeslib.as_array(up, shape=(n,))
        rout = np.ctypeslib.as_array(rp, shape=(n,))
        rout[:] = fn(uin.copy())

    cfn = RHS_FN(cb)
    lib().orc_rk_generic(n, _ptr(u), dt, 0 if scheme == "rk4" else 1, cfn, None)
    return u


STATS_FIELDS = ("mass", "momx", "momy", "momz", "energy", "ke", "enstrophy", "rho_min", "p_min",
                "max_wavespeed_over_dx")


def stats(P: Params, u) -> dict:
    u = _check_state(P, u)
    out = np.zeros(10)
    cp = P.c()
    lib().orc_stats(ctypes.byref(cp), _ptr(u), _ptr(out))
    return dict(zip(STATS_FIELDS, out.tolist()))


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
