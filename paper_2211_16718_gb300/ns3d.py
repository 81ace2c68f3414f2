"""Thin ctypes binding of libns3d.so (include/ns3d.h): argument marshalling only.

Every step of the right-hand side, the Runge-Kutta update and the statistics
runs in the library's CUDA kernels; this module only passes torch tensors'
device pointers and the current torch stream.  If the library is missing or
cannot be loaded, every call raises ``RuntimeError`` (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(PKG, "libns3d.so")

NS3D_OK, NS3D_EINVAL, NS3D_ENOMEM, NS3D_ECUDA, NS3D_ENONPHYSICAL, NS3D_ETIMEOUT = 0, -1, -2, -3, -4, -5
NS3D_ERANGE = -6
NS3D_RK4, NS3D_SSPRK3 = 0, 1
NS3D_FP64, NS3D_FP32_BULK, NS3D_FP64_STRICT = 0, 1, 2
NS3D_STORAGE_AUTO, NS3D_STORAGE_FULL, NS3D_STORAGE_LEAN = 0, 1, 2
NS3D_STATS_NDOUBLE = 12
KERNELS = ("prim", "visc", "dir_x", "dir_y", "dir_z", "stats", "stats_final", "adj_visc", "adj_dir", "adj_misc")
NS3D_FUNC_KE, NS3D_FUNC_ENSTROPHY = 0, 1
FUNCTIONALS = {"ke": NS3D_FUNC_KE, "enstrophy": NS3D_FUNC_ENSTROPHY}
EXPORTS = ("ns3d_default_params", "ns3d_init", "ns3d_free", "ns3d_set_stream", "ns3d_rhs", "ns3d_rk_step",
           "ns3d_stats", "ns3d_stats_async", "ns3d_step_host", "ns3d_check", "ns3d_strerror", "ns3d_last_error",
           "ns3d_timing_enable", "ns3d_timing_read", "ns3d_alu_probe", "ns3d_rhs_vjp", "ns3d_rk_step_vjp",
           "ns3d_functional", "ns3d_traj_forward", "ns3d_traj_vjp", "ns3d_storage_info", "ns3d_dt_from_cfl")


class Ns3dError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ns3d error {code}: {msg}")
        self.code = code


class NonPhysicalError(Ns3dError):
    pass


class CParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("rk", ctypes.c_int), ("precision", ctypes.c_int), ("weno_p", ctypes.c_int),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
        ("gamma", ctypes.c_double), ("mu_eff", ctypes.c_double), ("prandtl", ctypes.c_double),
        ("weno_eps", ctypes.c_double), ("harten_delta", ctypes.c_double),
        ("storage", ctypes.c_int),
    ]


class CStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("mass", "momx", "momy", "momz", "energy", "ke", "enstrophy",
                                                 "rho_min", "p_min", "max_wavespeed_over_dx")] + \
               [("status", ctypes.c_int), ("reserved", ctypes.c_int)]


STATS_FIELDS = tuple(n for n, _ in CStats._fields_[:10])

_lock = threading.Lock()
_lib = None


def lib():
    """Load libns3d.so once; raise RuntimeError if it is absent (no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIBPATH):
                raise RuntimeError(f"{LIBPATH} is missing: build it with paper_2211_16718_gb300.build.build() "
                                   "(nvcc for sm_103a); there is no CPU fallback")
            L = ctypes.CDLL(LIBPATH)
            P, D, I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
            pp = ctypes.POINTER(CParams)
            sigs = {
                "ns3d_default_params": (None, [pp, I, I, I]),
                "ns3d_init": (I, [pp, P, ctypes.POINTER(P)]),
                "ns3d_free": (None, [P]),
                "ns3d_set_stream": (I, [P, P]),
                "ns3d_rhs": (I, [P, P, P]),
                "ns3d_rk_step": (I, [P, P, D, I]),
                "ns3d_stats": (I, [P, P, ctypes.POINTER(CStats)]),
                "ns3d_stats_async": (I, [P, P, P]),
                "ns3d_step_host": (I, [P, P, D, I, ctypes.POINTER(CStats)]),
                "ns3d_check": (I, [P]),
                "ns3d_strerror": (ctypes.c_char_p, [I]),
                "ns3d_last_error": (ctypes.c_char_p, [P]),
                "ns3d_timing_enable": (I, [P, I]),
                "ns3d_timing_read": (I, [P, P, P, I]),
                "ns3d_alu_probe": (I, [P]),
                "ns3d_rhs_vjp": (I, [P, P, P, P]),
                "ns3d_rk_step_vjp": (I, [P, P, P, D]),
                "ns3d_functional": (I, [P, P, I, P, P]),
                "ns3d_traj_forward": (I, [P, P, D, I, I]),
                "ns3d_traj_vjp": (I, [P, P]),
                "ns3d_storage_info": (I, [P, P, P]),
                "ns3d_dt_from_cfl": (I, [P, P, D, P]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def default_params(nx: int, ny: int, nz: int, **kw) -> CParams:
    p = CParams()
    lib().ns3d_default_params(ctypes.byref(p), nx, ny, nz)
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def _stream_handle():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t, n: int):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError("expected a CUDA float64 tensor")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"expected a contiguous tensor of {n} elements, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One ns3d context (library-owned scratch) for a fixed grid and parameters."""

    def __init__(self, nx: int, ny: int, nz: int, **kw):
        self.params = default_params(nx, ny, nz, **kw)
        self.N = nx * ny * nz
        self.shape = (5, nz, ny, nx)
        self._ctx = ctypes.c_void_p()
        self.traj_generation = 0  # counts ns3d_traj_forward calls: which recording the library holds
        rc = lib().ns3d_init(ctypes.byref(self.params), _stream_handle(), ctypes.byref(self._ctx))
        if rc != NS3D_OK:
            raise Ns3dError(rc, lib().ns3d_strerror(rc).decode())

    def _check(self, rc: int):
        if rc == NS3D_OK:
            return
        msg = lib().ns3d_last_error(self._ctx).decode() or lib().ns3d_strerror(rc).decode()
        if rc == NS3D_ENONPHYSICAL:
            raise NonPhysicalError(rc, msg)
        raise Ns3dError(rc, msg)

    def _sync_stream(self):
        self._check(lib().ns3d_set_stream(self._ctx, _stream_handle()))

    def rhs(self, u, out=None):
        import torch
        if out is None:
            out = torch.empty_like(u)
        self._sync_stream()
        self._check(lib().ns3d_rhs(self._ctx, _dptr(u, 5 * self.N), _dptr(out, 5 * self.N)))
        return out

    def rk_step(self, u, dt: float, nsteps: int = 1):
        self._sync_stream()
        self._check(lib().ns3d_rk_step(self._ctx, _dptr(u, 5 * self.N), float(dt), int(nsteps)))
        return u

    def stats(self, u) -> dict:
        self._sync_stream()
        s = CStats()
        rc = lib().ns3d_stats(self._ctx, _dptr(u, 5 * self.N), ctypes.byref(s))
        if rc not in (NS3D_OK, NS3D_ENONPHYSICAL, NS3D_ERANGE):
            self._check(rc)
        d = {n: getattr(s, n) for n in STATS_FIELDS}
        d["status"] = s.status
        return d

    def stats_async(self, u, out):
        """Write NS3D_STATS_NDOUBLE doubles of statistics into the device tensor out (no sync)."""
        self._sync_stream()
        self._check(lib().ns3d_stats_async(self._ctx, _dptr(u, 5 * self.N), _dptr(out, NS3D_STATS_NDOUBLE)))
        return out

    def step_host(self, u_host, dt: float, nsteps: int = 1) -> dict:
        """End to end with a host numpy array (float64, C-contiguous, 5*N): copied in, stepped, copied back.
        On grids with nz >= 64 the copies overlap with the first and last RK stages (in z-slabs) when
        u_host is pinned, e.g. torch.empty(..., pin_memory=True).numpy()."""
        import numpy as np
        if not (isinstance(u_host, np.ndarray) and u_host.dtype == np.float64 and u_host.flags.c_contiguous
                and u_host.size == 5 * self.N):
            raise ValueError("expected a C-contiguous float64 numpy array of 5*N elements")
        self._sync_stream()
        s = CStats()
        rc = lib().ns3d_step_host(self._ctx, ctypes.c_void_p(u_host.ctypes.data), float(dt), int(nsteps),
                                  ctypes.byref(s))
        if rc not in (NS3D_OK, NS3D_ENONPHYSICAL, NS3D_ERANGE):
            self._check(rc)
        d = {n: getattr(s, n) for n in STATS_FIELDS}
        d["status"] = s.status
        return d

    def check(self):
        self._sync_stream()
        self._check(lib().ns3d_check(self._ctx))

    # ---- adjoint -----------------------------------------------------------------
    def rhs_vjp(self, u, lam, out=None):
        """out = J(u)^T lam with J = dR/du (ns3d_rhs_vjp)."""
        import torch
        if out is None:
            out = torch.empty_like(u)
        self._sync_stream()
        self._check(lib().ns3d_rhs_vjp(self._ctx, _dptr(u, 5 * self.N), _dptr(lam, 5 * self.N),
                                       _dptr(out, 5 * self.N)))
        return out

    def rk_step_vjp(self, u, ubar, dt: float):
        """ubar <- (d step(u)/du)^T ubar for one step from u (ns3d_rk_step_vjp); u is unchanged."""
        self._sync_stream()
        self._check(lib().ns3d_rk_step_vjp(self._ctx, _dptr(u, 5 * self.N), _dptr(ubar, 5 * self.N), float(dt)))
        return ubar

    def functional(self, u, which: str = "ke", grad=None, value: bool = True):
        """(value, grad) of the mean kinetic energy ("ke") or enstrophy ("enstrophy") of u;
        grad: a tensor like u to receive the gradient, True to allocate one, or None."""
        import torch
        if grad is True:
            grad = torch.empty_like(u)
        v = ctypes.c_double()
        self._sync_stream()
        self._check(lib().ns3d_functional(self._ctx, _dptr(u, 5 * self.N), FUNCTIONALS[which],
                                          ctypes.byref(v) if value else None,
                                          _dptr(grad, 5 * self.N) if grad is not None else None))
        return (v.value if value else None), grad

    def traj_forward(self, u, dt: float, nsteps: int, every: int = 16):
        """Advance u by nsteps steps, recording checkpoints every `every` steps (ns3d_traj_forward)."""
        self._sync_stream()
        self.traj_generation += 1
        self._check(lib().ns3d_traj_forward(self._ctx, _dptr(u, 5 * self.N), float(dt), int(nsteps), int(every)))
        return u

    def traj_vjp(self, ubar):
        """ubar (adjoint of the final state) <- adjoint of the initial state (ns3d_traj_vjp)."""
        self._sync_stream()
        self._check(lib().ns3d_traj_vjp(self._ctx, _dptr(ubar, 5 * self.N)))
        return ubar

    def storage_info(self) -> dict:
        """{"storage": NS3D_STORAGE_FULL | NS3D_STORAGE_LEAN, "device_bytes": library-owned bytes}"""
        st, nb = ctypes.c_int(), ctypes.c_size_t()
        self._check(lib().ns3d_storage_info(self._ctx, ctypes.byref(st), ctypes.byref(nb)))
        return {"storage": st.value, "device_bytes": nb.value}

    def timing_enable(self, on: bool = True):
        self._check(lib().ns3d_timing_enable(self._ctx, int(bool(on))))

    def timing_read(self) -> dict:
        n = len(KERNELS)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        self._check(lib().ns3d_timing_read(self._ctx, ctypes.cast(ms, ctypes.c_void_p),
                                           ctypes.cast(cnt, ctypes.c_void_p), n))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNELS)}

    def close(self):
        if self._ctx:
            lib().ns3d_free(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dt_from_cfl(self, u, cfl: float) -> float:
        """dt = CFL / max over points and directions of (|u_d| + c)/dx_d (ns3d_dt_from_cfl)."""
        dt = ctypes.c_double()
        self._sync_stream()
        self._check(lib().ns3d_dt_from_cfl(self._ctx, _dptr(u, 5 * self.N), float(cfl), ctypes.byref(dt)))
        return dt.value


def alu_probe() -> dict:
    """Measured arithmetic throughput of the current device, G lane-ops/s."""
    out = (ctypes.c_double * 5)()
    rc = lib().ns3d_alu_probe(ctypes.cast(out, ctypes.c_void_p))
    if rc != NS3D_OK:
        raise Ns3dError(rc, lib().ns3d_strerror(rc).decode())
    return dict(zip(("dfma", "dadd", "ddiv", "dsqrt", "ffma"), list(out)))


def stats_noalloc(params: CParams, u, out):
    """Statistics of the device state u into the device tensor out (NS3D_STATS_NDOUBLE
    float64) through ns3d_stats_noalloc, which allocates no device memory: for callers that
    own all GPU memory through their own pool or must not perturb another code's memory
    footprint.  No context is needed; the work goes on the current torch stream without
    synchronising.  Calls that overlap on the GPU share the library's fixed scratch array
    and race; serialise them."""
    fn = lib().ns3d_stats_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(CParams), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    n = params.nx * params.ny * params.nz
    rc = fn(ctypes.byref(params), _dptr(u, 5 * n), _dptr(out, NS3D_STATS_NDOUBLE), _stream_handle())
    if rc != NS3D_OK:
        raise Ns3dError(rc, lib().ns3d_strerror(rc).decode())
    return out


# ---- ensembles of independent grids -------------------------------------------------
NS3D_BATCH_SEQUENTIAL, NS3D_BATCH_GRAPH, NS3D_BATCH_PERSISTENT = 0, 1, 2
SCHEDULES = {"sequential": NS3D_BATCH_SEQUENTIAL, "graph": NS3D_BATCH_GRAPH, "persistent": NS3D_BATCH_PERSISTENT}


def _batch_fn(name, res, args):
    fn = getattr(lib(), name)
    fn.restype = res
    fn.argtypes = args
    return fn


class Batch:
    """An ensemble of independent grids (ns3d_batch_*): per-instance parameters, states
    (caller-owned CUDA float64 tensors) and time steps; three schedules of the same
    arithmetic: "sequential", "graph" (batched launches in one CUDA graph) and
    "persistent" (one cooperative kernel for all steps)."""

    def __init__(self, params: list):
        P = ctypes.c_void_p
        self.count = len(params)
        arr = (CParams * self.count)(*params)
        self.params = list(params)
        self._b = ctypes.c_void_p()
        rc = _batch_fn("ns3d_batch_init", ctypes.c_int, [ctypes.POINTER(CParams), ctypes.c_int, P, ctypes.POINTER(P)])(
            arr, self.count, _stream_handle(), ctypes.byref(self._b))
        if rc != NS3D_OK:
            raise Ns3dError(rc, lib().ns3d_strerror(rc).decode())
        self._states = None

    def _err(self, rc):
        if rc == NS3D_OK:
            return
        msg = _batch_fn("ns3d_batch_last_error", ctypes.c_char_p, [ctypes.c_void_p])(self._b).decode()
        if rc == NS3D_ENONPHYSICAL:
            raise NonPhysicalError(rc, msg or "non-physical state")
        raise Ns3dError(rc, msg or lib().ns3d_strerror(rc).decode())

    def set_states(self, tensors):
        if len(tensors) != self.count:
            raise ValueError("one state per instance")
        ptrs = (ctypes.c_void_p * self.count)()
        for i, (t, p) in enumerate(zip(tensors, self.params)):
            ptrs[i] = _dptr(t, 5 * p.nx * p.ny * p.nz).value
        self._states = list(tensors)
        self._err(_batch_fn("ns3d_batch_set_states", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p])(self._b, ptrs))

    def set_dt(self, dts):
        arr = (ctypes.c_double * self.count)(*[float(d) for d in dts])
        self._err(_batch_fn("ns3d_batch_set_dt", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p])(self._b, arr))

    def set_dt_from_cfl(self, cfl: float):
        """Each instance's dt from its own current state at one CFL number
        (ns3d_batch_set_dt_from_cfl); returns the time steps."""
        arr = (ctypes.c_double * self.count)()
        self._err(_batch_fn("ns3d_batch_set_dt_from_cfl", ctypes.c_int,
                            [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p])(self._b, float(cfl), arr))
        return list(arr)

    def set_variant(self, v: int):
        self._err(_batch_fn("ns3d_batch_set_variant", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int])(self._b, int(v)))

    def step(self, nsteps: int = 1, schedule: str = "graph"):
        self._err(_batch_fn("ns3d_batch_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int])(
            self._b, int(nsteps), SCHEDULES[schedule]))

    def stats(self):
        import torch
        out = torch.zeros((self.count, NS3D_STATS_NDOUBLE), dtype=torch.float64, device="cuda")
        self._err(_batch_fn("ns3d_batch_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p])(
            self._b, ctypes.c_void_p(out.data_ptr())))
        return out

    def check(self):
        self._err(_batch_fn("ns3d_batch_check", ctypes.c_int, [ctypes.c_void_p])(self._b))

    def set_instance_variant(self, i: int, v: int):
        self._err(_batch_fn("ns3d_batch_set_instance_variant", ctypes.c_int,
                            [ctypes.c_void_p, ctypes.c_int, ctypes.c_int])(self._b, int(i), int(v)))

    def set_branches(self, nb: int):
        self._err(_batch_fn("ns3d_batch_set_branches", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int])(self._b, int(nb)))

    def autotune(self, cache_path=None) -> dict:
        """Per grid size the tile shape, then the graph's branch count (ns3d_batch_autotune).
        Returns {"variants": per instance, "branches": n, "ms_variants": per instance [3],
        "ms_branches": [8]} (-1: not timed)."""
        ms = (ctypes.c_double * (3 * self.count + 8))()
        path = cache_path.encode() if cache_path else None
        self._err(_batch_fn("ns3d_batch_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p])(
            self._b, path, ms))
        out = self.schedule_info()
        out["ms_variants"] = [list(ms[3 * i: 3 * i + 3]) for i in range(self.count)]
        out["ms_branches"] = list(ms[3 * self.count:])
        return out

    def schedule_info(self) -> dict:
        v = (ctypes.c_int * self.count)()
        nb = ctypes.c_int()
        self._err(_batch_fn("ns3d_batch_schedule_info", ctypes.c_int, [ctypes.c_void_p] * 3)(
            self._b, v, ctypes.byref(nb)))
        return {"variants": list(v), "branches": nb.value}

    def info(self) -> dict:
        v, c, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._err(_batch_fn("ns3d_batch_info", ctypes.c_int, [ctypes.c_void_p] * 4)(
            self._b, ctypes.byref(v), ctypes.byref(c), ctypes.byref(g)))
        return {"variant": v.value, "persistent_ctas_per_sm": c.value, "persistent_in_graph": g.value}

    def close(self):
        if self._b:
            _batch_fn("ns3d_batch_free", None, [ctypes.c_void_p])(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_solver_variant(solver: Solver, v: int):
    rc = _batch_fn("ns3d_set_variant", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int])(solver._ctx, int(v))
    solver._check(rc)


def set_solver_zorder(solver: Solver, order: int):
    """CTA order of the z pass (ns3d_set_zorder): 0 tiles along z first, 1 line groups first, -1 by size."""
    rc = _batch_fn("ns3d_set_zorder", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int])(solver._ctx, int(order))
    solver._check(rc)
