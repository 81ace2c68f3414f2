"""ns3d_stats_noalloc: statistics without any device allocation.

Callers that own all GPU memory through their own pool, or that run inside another
code's time loop and must not change its memory footprint, cannot let the library call
cudaMalloc (creating a context allocates scratch).  This entry point keeps its only
scratch in a fixed file-scope device array.  The test calls it through the C ABI and
compares it with the context-based statistics (ns3d_stats_async) within the tolerance
the parity tests use for statistics (1e-12 relative), on two calls in a row with
different grids, compares one call directly with the CPU oracle's statistics, then
checks that a non-physical flag (negative or infinite density) does not carry over.
This file is collected last; it passes alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest

from paper_2211_16718_gb300 import inputs as I

pytestmark = pytest.mark.gpu

STATS_TOL = 1e-12


@pytest.fixture(scope="module")
def ns3d():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2211_16718_gb300 import build as B
    B.build()
    from paper_2211_16718_gb300 import ns3d as N
    N.lib()
    return N


def _call_c_abi(ns3d, params, u, out):
    import torch
    fn = ns3d.lib().ns3d_stats_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(ns3d.CParams), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return fn(ctypes.byref(params), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(out.data_ptr()),
              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _reference(ns3d, u_np, **kw):
    import torch
    nz, ny, nx = u_np.shape[1:]
    s = ns3d.Solver(nx, ny, nz, **kw)
    out = torch.zeros(ns3d.NS3D_STATS_NDOUBLE, dtype=torch.float64, device="cuda")
    s.stats_async(torch.from_numpy(u_np).cuda(), out)
    ref = out.cpu().numpy()
    s.close()
    return ref


def _compare(got, ref):
    mass = ref[0]
    for k in range(10):
        if k in (1, 2, 3):  # momentum sums are cancellation residues: compare against the mass
            assert abs(got[k] - ref[k]) <= STATS_TOL * abs(mass), k
        else:
            assert got[k] == pytest.approx(ref[k], rel=STATS_TOL, abs=0.0), k


def test_noalloc_stats_match_context_stats_two_calls(ns3d):
    import torch
    cases = [
        (I.isotropic_turbulence(32, seed=3), dict()),
        (I.random_smooth(24, 20, 16, seed=4, amp=0.1, mach=0.4, lx=3.0, ly=2.0, lz=1.5),
         dict(lx=3.0, ly=2.0, lz=1.5)),
    ]
    for u_np, kw in cases:
        ref = _reference(ns3d, u_np, **kw)
        nz, ny, nx = u_np.shape[1:]
        p = ns3d.default_params(nx, ny, nz, **kw)
        u = torch.from_numpy(u_np).cuda()
        out = torch.full((ns3d.NS3D_STATS_NDOUBLE,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call_c_abi(ns3d, p, u, out) == ns3d.NS3D_OK
        got = out.cpu().numpy()
        _compare(got, ref)
        assert got[10] == 0.0 and ref[10] == 0.0


def test_noalloc_stats_match_oracle(ns3d):
    """One call compared directly with the FP64 CPU oracle's statistics (Sec. 2.3 reading:
    sums times the cell volume, volume means of KE and enstrophy, minima, CFL wave speed)."""
    import torch
    from oracle import oracle as O
    O.build()
    u_np = I.isotropic_turbulence(32, seed=6)
    so = O.stats(O.Params(32, 32, 32), u_np)
    p = ns3d.default_params(32, 32, 32)
    out = torch.full((ns3d.NS3D_STATS_NDOUBLE,), float("nan"), dtype=torch.float64, device="cuda")
    assert _call_c_abi(ns3d, p, torch.from_numpy(u_np).cuda(), out) == ns3d.NS3D_OK
    got = out.cpu().numpy()
    for k, name in enumerate(ns3d.STATS_FIELDS):
        if name.startswith("mom"):
            assert abs(got[k] - so[name]) <= STATS_TOL * so["mass"], name
        else:
            assert got[k] == pytest.approx(so[name], rel=STATS_TOL, abs=0.0), name
    assert got[10] == 0.0


@pytest.mark.parametrize("rho_bad", [-0.5, float("inf")], ids=["negative_rho", "infinite_rho"])
def test_noalloc_flags_nonphysical_without_carry_over(ns3d, rho_bad):
    import torch
    bad = I.random_smooth(16, 16, 16, seed=5, amp=0.1)
    bad[0, 2, 3, 4] = rho_bad
    good = I.random_smooth(16, 16, 16, seed=5, amp=0.1)
    p = ns3d.default_params(16, 16, 16)
    out = torch.zeros(ns3d.NS3D_STATS_NDOUBLE, dtype=torch.float64, device="cuda")
    ns3d.stats_noalloc(p, torch.from_numpy(bad).cuda(), out)
    assert out[10].item() == 1.0
    ns3d.stats_noalloc(p, torch.from_numpy(good).cuda(), out)
    assert out[10].item() == 0.0
    _compare(out.cpu().numpy(), _reference(ns3d, good))


def test_noalloc_rejects_bad_arguments(ns3d):
    import torch
    p = ns3d.default_params(8, 8, 8)
    u = torch.from_numpy(I.uniform(8, 8, 8)).cuda()
    out = torch.zeros(ns3d.NS3D_STATS_NDOUBLE, dtype=torch.float64, device="cuda")
    big = ns3d.default_params(2048, 2048, 2048)  # 2^33 points: beyond the supported maximum
    assert _call_c_abi(ns3d, big, u, out) == ns3d.NS3D_EINVAL
    p.nx = 0
    assert _call_c_abi(ns3d, p, u, out) == ns3d.NS3D_EINVAL
    fn = ns3d.lib().ns3d_stats_noalloc
    assert fn(None, None, None, None) == ns3d.NS3D_EINVAL
