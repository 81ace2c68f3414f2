"""Forward-mode (dual-number) build of the CPU oracle: exact Jacobian-vector products of
the oracle's discrete operator, and from them its discrete adjoint.

TEST INFRASTRUCTURE ONLY.  The same source ns3d_oracle.c is compiled as C++ with every
floating-point ``double`` replaced by a dual number (value, derivative); the parameter
struct keeps plain doubles so the ctypes layout is unchanged.  Derivative rules: the
usual ones for + - * / and sqrt; |x| has derivative sign(x) with sign(0) = 0 (the
subgradient used at the kink of the eigenvalue magnitudes).  Branches (Harten's fix,
minima) follow the value part.

  rhs_jvp(P, u, w)            -> (R(u), J(u) w)
  rk_step_jvp(P, u, w, dt, n) -> (Phi(u), dPhi(u) w) for n RK steps
  rhs_jacobian(P, u)          -> dense J(u) (small grids only)
  rhs_vjp_dense(P, u, lam)    -> J(u)^T lam (small grids only)
  stats_jvp(P, u, w)          -> statistics and their directional derivatives
  functional_grad_dense(...)  -> gradient of final-time KE / enstrophy (small grids only)
"""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libns3d_oracle_dual.so")
_lib = None

_DUAL = r"""
#include <cmath>
#include <cstring>
struct dual {
  double v, d;
  dual() : v(0.0), d(0.0) {}
  dual(double x) : v(x), d(0.0) {}
  dual(double x, double y) : v(x), d(y) {}
  dual& operator+=(const dual& o) { v += o.v; d += o.d; return *this; }
  dual& operator-=(const dual& o) { v -= o.v; d -= o.d; return *this; }
  dual& operator*=(const dual& o) { d = d * o.v + v * o.d; v *= o.v; return *this; }
  dual& operator/=(const dual& o) { d = (d * o.v - v * o.d) / (o.v * o.v); v /= o.v; return *this; }
};
static inline dual operator+(dual a, const dual& b) { return a += b; }
static inline dual operator-(dual a, const dual& b) { return a -= b; }
static inline dual operator*(dual a, const dual& b) { return a *= b; }
static inline dual operator/(dual a, const dual& b) { return a /= b; }
static inline dual operator-(const dual& a) { return dual(-a.v, -a.d); }
static inline bool operator<(const dual& a, const dual& b) { return a.v < b.v; }
static inline bool operator>(const dual& a, const dual& b) { return a.v > b.v; }
static inline bool operator<=(const dual& a, const dual& b) { return a.v <= b.v; }
static inline bool operator>=(const dual& a, const dual& b) { return a.v >= b.v; }
static inline bool operator==(const dual& a, const dual& b) { return a.v == b.v; }
static inline bool operator!=(const dual& a, const dual& b) { return a.v != b.v; }
static inline dual sqrt(const dual& a) { double s = std::sqrt(a.v); return dual(s, a.d / (2.0 * s)); }
static inline dual fabs(const dual& a) { return dual(std::fabs(a.v), a.v > 0 ? a.d : (a.v < 0 ? -a.d : 0.0)); }
typedef double PREAL;
"""


def build() -> str:
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "ns3d_oracle.c")
    me = os.path.abspath(__file__)
    if os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(os.path.getmtime(src), os.path.getmtime(me)):
        return _LIB
    text = open(src).read()
    # keep the parameter struct in plain doubles
    a = text.index("typedef struct {")
    b = text.index("} orc_params;")
    text = text[:a] + text[a:b].replace("double", "PREAL") + text[b:]
    text = re.sub(r"\bdouble\b", "dual", text)
    text = text.replace("#include <math.h>", "")
    text = text.replace("sizeof(dual[5])", "sizeof(dual) * 5")
    text = _DUAL + 'extern "C" {\n' + text + "\n}\n"
    # C -> C++: malloc results need casts
    text = re.sub(r"(dual \(\*(\w+)\)\[5\]) = malloc\(", r"\1 = (dual (*)[5])malloc(", text)
    text = re.sub(r"(dual \*(\w+)) = malloc\(", r"\1 = (dual *)malloc(", text)
    text = text.replace("dual *k1 = malloc(sizeof(dual) * n), *k2 = malloc(sizeof(dual) * n);",
                        "dual *k1 = (dual *)malloc(sizeof(dual) * n), *k2 = (dual *)malloc(sizeof(dual) * n);")
    text = text.replace("INFINITY", "HUGE_VAL")
    cpp = os.path.join(_BUILD, "ns3d_oracle_dual.cpp")
    with open(cpp, "w") as f:
        f.write(text)
    base = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fpermissive", "-w", "-fPIC",
            "-shared"]
    tmp = _LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", cpp, "-o", tmp], check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError:
        r = subprocess.run(base + [cpp, "-o", tmp], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("dual oracle build failed:\n" + r.stderr[-4000:])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


class Dual(ctypes.Structure):
    """A dual number passed by value (the C++ struct is two doubles)."""
    _fields_ = [("v", ctypes.c_double), ("d", ctypes.c_double)]


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def _pack(u, w) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.empty(u.shape + (2,), dtype=np.float64)
    out[..., 0] = u
    out[..., 1] = w
    return out


def rhs_jvp(P, u, w):
    """(R(u), J(u) w) of the oracle's right-hand side.  P: oracle.Params."""
    x = _pack(u, w)
    r = np.zeros_like(x)
    cp = P.c()
    lib().orc_rhs(ctypes.byref(cp), x.ctypes.data_as(ctypes.c_void_p), r.ctypes.data_as(ctypes.c_void_p))
    return r[..., 0].copy(), r[..., 1].copy()


def rk_step_jvp(P, u, w, dt: float, nsteps: int = 1, scheme: str = "rk4"):
    """(Phi(u), dPhi(u) w) of nsteps Runge-Kutta steps."""
    x = _pack(u, w)
    cp = P.c()
    f = lib().orc_rk_step
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, Dual, ctypes.c_int, ctypes.c_int]
    f(ctypes.byref(cp), x.ctypes.data_as(ctypes.c_void_p), Dual(float(dt), 0.0), int(nsteps),
      0 if scheme == "rk4" else 1)
    return x[..., 0].copy(), x[..., 1].copy()


def stats_jvp(P, u, w):
    """(stats(u), d stats(u) w): the ten statistics of the oracle and their directional
    derivatives (index 5 = mean kinetic energy, 6 = mean enstrophy)."""
    x = _pack(u, w)
    out = np.zeros((10, 2))
    cp = P.c()
    lib().orc_stats(ctypes.byref(cp), x.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p))
    return out[:, 0].copy(), out[:, 1].copy()


def flux_jvp(U, w, d: int, gamma: float = 1.4):
    """(f_d(U), df_d(U) w) of the convective flux of one state."""
    x = _pack(np.asarray(U, dtype=np.float64).reshape(5), np.asarray(w, dtype=np.float64).reshape(5))
    out = np.zeros((5, 2))
    f = lib().orc_flux
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, Dual, ctypes.c_void_p]
    f(x.ctypes.data_as(ctypes.c_void_p), int(d), Dual(float(gamma), 0.0), out.ctypes.data_as(ctypes.c_void_p))
    return out[:, 0].copy(), out[:, 1].copy()


def rhs_jacobian(P, u) -> np.ndarray:
    """Dense Jacobian dR/du (5N x 5N) column by column (for small grids)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    n = u.size
    J = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        J[:, j] = rhs_jvp(P, u, e.reshape(u.shape))[1].ravel()
        e[j] = 0.0
    return J


def rhs_vjp_dense(P, u, lam) -> np.ndarray:
    """J(u)^T lam from the dense Jacobian (the oracle's discrete adjoint; small grids)."""
    J = rhs_jacobian(P, u)
    return (J.T @ np.ascontiguousarray(lam, dtype=np.float64).ravel()).reshape(np.shape(u))


def functional_grad_dense(P, u0, dt: float, nsteps: int, scheme: str = "rk4", which: str = "ke") -> np.ndarray:
    """Gradient of the mean kinetic energy (which='ke') or enstrophy ('enstrophy') after
    nsteps Runge-Kutta steps with respect to the initial state, one forward-mode sweep per
    component (small grids)."""
    k = {"ke": 5, "enstrophy": 6}[which]
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    g = np.zeros(u0.size)
    e = np.zeros(u0.size)
    for j in range(u0.size):
        e[j] = 1.0
        uN, dN = rk_step_jvp(P, u0, e.reshape(u0.shape), dt, nsteps, scheme)
        g[j] = stats_jvp(P, uN, dN)[1][k]
        e[j] = 0.0
    return g.reshape(u0.shape)
