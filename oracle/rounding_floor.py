"""FP64 rounding floor of the discrete operator, measured on the oracle itself.

TEST INFRASTRUCTURE ONLY.  Builds a copy of ns3d_oracle.c with every ``double``
promoted to ``long double`` (80-bit on x86-64, IEEE binary128 on aarch64) and
compares the FP64 oracle's right-hand side with it.  The difference is the
rounding error of one FP64 evaluation of the method; two independent FP64
implementations (oracle and CUDA path) cannot agree more closely than about
this.  At low Mach number the convective fluxes carry the O(1) background
pressure while the right-hand side is O(Mach^2 / L), so the floor of the
relative max-norm grows like 1 / (Mach^2 * dx).
"""
from __future__ import annotations

import ctypes
import math
import os
import re
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libns3d_oracle_ld.so")
_lib = None


def build() -> str:
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "ns3d_oracle.c")
    if os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    text = open(src).read()
    text = re.sub(r"\bdouble\b", "long double", text)
    text = re.sub(r"\bsqrt\(", "sqrtl(", text)
    text = re.sub(r"\bfabs\(", "fabsl(", text)
    c = os.path.join(_BUILD, "ns3d_oracle_ld.c")
    with open(c, "w") as f:
        f.write(text)
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", c, "-o", _LIB, "-lm"],
                   check=True, capture_output=True)
    return _LIB


class _CParamsLD(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("weno_p", ctypes.c_int),
                ("weno_linear", ctypes.c_int), ("roe_state", ctypes.c_int)] + \
               [(n, ctypes.c_longdouble) for n in ("lx", "ly", "lz", "gamma", "mu_eff", "prandtl", "weno_eps",
                                                   "harten_delta")]


def rhs_extended(u: np.ndarray, mu_eff: float, lengths=(2 * math.pi,) * 3) -> np.ndarray:
    """Right-hand side evaluated in long double (result rounded to float64)."""
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
    nz, ny, nx = u.shape[1:]
    p = _CParamsLD(nx, ny, nz, 2, 0, 0, lengths[0], lengths[1], lengths[2], 1.4, mu_eff, 0.72, 1e-6, 0.1)
    ul = np.ascontiguousarray(u, dtype=np.longdouble)
    rl = np.zeros_like(ul)
    _lib.orc_rhs(ctypes.byref(p), ul.ctypes.data_as(ctypes.c_void_p), rl.ctypes.data_as(ctypes.c_void_p))
    return rl.astype(np.float64)
