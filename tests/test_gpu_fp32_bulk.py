"""FP32-bulk mode (NS3D_FP32_BULK): smoothness indicators, weights, interface values and
Roe flux in FP32; state, conservative difference, viscous terms, RK and reductions FP64.

Tolerance, derived from the arithmetic: each interface flux carries a relative FP32
rounding error of order c * 2^-24 (c ~ 10-30 for the WENO + Roe evaluation), and the
RHS is a difference of two fluxes over dx.  So the RHS error is bounded by ~2c 2^-24 of
the flux scale S_F = max|f| / dx_min; the tests assert ||r32 - r64||_inf <= 1e-5 S_F
(about 170 * 2^-24).  After K RK steps of size dt the state error is bounded by
K dt times that.  What FP32 cannot change, it must keep exactly: free-stream
preservation and discrete conservation (the fluxes are widened to FP64 before the
difference, so the sums telescope to FP64 rounding).
"""
import math
import os

import numpy as np
import pytest

from paper_2211_16718_gb300 import inputs as I

from tests._util import flux_scale

pytestmark = pytest.mark.gpu

FLUX_TOL = 1e-5


@pytest.fixture(scope="module")
def ns3d():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2211_16718_gb300 import build as B
    B.build()
    from paper_2211_16718_gb300 import ns3d as N
    N.lib()
    return N


@pytest.fixture(scope="module")
def orc(oracle):
    oracle.set_threads(os.cpu_count() or 1)
    return oracle


def _gpu(u):
    import torch
    return torch.from_numpy(np.ascontiguousarray(u)).cuda()


CASES = [
    ("hit64", lambda: I.isotropic_turbulence(64, seed=1), dict(mu_eff=I.hit_mu_eff())),
    ("tgv32", lambda: I.taylor_green(32), dict(mu_eff=6.25e-5)),
    ("ragged_37x29x23", lambda: I.random_smooth(37, 29, 23, seed=2, amp=0.1, mach=0.4, lx=3.0, ly=2.0, lz=1.5),
     dict(mu_eff=3e-3, lx=3.0, ly=2.0, lz=1.5)),
    ("shock_tube_y", lambda: I.shock_tube(12, 40, 10, axis=1), dict(mu_eff=1e-3)),
    ("near_sonic", lambda: I.random_smooth(24, 20, 16, seed=6, amp=0.1, mach=1.1), dict(mu_eff=1e-3)),
]


@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_fp32_bulk_rhs_within_fp32_bound(ns3d, orc, name, make, kw):
    u = make()
    nz, ny, nx = u.shape[1:]
    s = ns3d.Solver(nx, ny, nz, precision=ns3d.NS3D_FP32_BULK, **kw)
    r32 = s.rhs(_gpu(u)).cpu().numpy()
    okw = {k: v for k, v in kw.items() if k in ("lx", "ly", "lz", "mu_eff")}
    r64 = orc.rhs(orc.Params(nx, ny, nz, **okw), u)
    L = (kw.get("lx", 2 * math.pi), kw.get("ly", 2 * math.pi), kw.get("lz", 2 * math.pi))
    err = np.abs(r32 - r64).max() / flux_scale(u, L)
    assert err <= FLUX_TOL, f"{name}: {err:.3e}"
    # and it is not the FP64 result (the mode really runs in FP32)
    assert not np.array_equal(r32, r64)


def test_fp32_bulk_free_stream_and_conservation(ns3d):
    u = I.uniform(20, 12, 9, rho=1.2, u=0.3, v=-0.4, w=0.1, p=0.9)
    s = ns3d.Solver(20, 12, 9, mu_eff=1e-2, precision=ns3d.NS3D_FP32_BULK)
    assert np.all(s.rhs(_gpu(u)).cpu().numpy() == 0.0)
    u = I.random_smooth(40, 36, 28, seed=7, amp=0.2, mach=0.5)
    s = ns3d.Solver(40, 36, 28, mu_eff=2e-2, precision=ns3d.NS3D_FP32_BULK)
    r = s.rhs(_gpu(u)).cpu().numpy().reshape(5, -1)
    scale = np.abs(r).max(axis=1)
    assert np.all(np.abs(r.sum(axis=1)) <= 64 * np.finfo(float).eps * scale * r.shape[1])


def test_fp32_bulk_rk4_ten_steps(ns3d, orc):
    """10 RK4 steps of the 32^3 isotropic-turbulence field: state error <= 10 dt FLUX_TOL S_F."""
    n = 32
    u0 = I.isotropic_turbulence(n, seed=4)
    mu = I.hit_mu_eff()
    P = orc.Params(n, n, n, mu_eff=mu)
    dt = 0.4 / orc.stats(P, u0)["max_wavespeed_over_dx"]
    s = ns3d.Solver(n, n, n, mu_eff=mu, precision=ns3d.NS3D_FP32_BULK)
    ud = _gpu(u0)
    s.rk_step(ud, dt, 10)
    err = np.abs(ud.cpu().numpy() - orc.rk_step(P, u0, dt, 10)).max()
    bound = 10 * dt * FLUX_TOL * flux_scale(u0, (2 * math.pi,) * 3)
    assert err <= bound, (err, bound)


@pytest.mark.parametrize("n", [(32, 32, 32), (33, 20, 18)], ids=["nx_even_paired_epilogue", "nx_odd"])
def test_fp32_bulk_ssprk3_steps(ns3d, orc, n):
    """5 SSP-RK3 steps (every SSP stage epilogue) on a grid whose nx is even (the y and z passes
    move their epilogue operands as 16-byte pairs) and odd (one point per thread): state error
    <= 5 dt FLUX_TOL S_F against the oracle."""
    u0 = I.random_smooth(*n, seed=8, amp=0.15, mach=0.5)
    mu = 2e-3
    P = orc.Params(*n, mu_eff=mu)
    dt = 0.4 / orc.stats(P, u0)["max_wavespeed_over_dx"]
    s = ns3d.Solver(*n, mu_eff=mu, rk=ns3d.NS3D_SSPRK3, precision=ns3d.NS3D_FP32_BULK)
    ud = _gpu(u0)
    s.rk_step(ud, dt, 5)
    s.check()
    err = np.abs(ud.cpu().numpy() - orc.rk_step(P, u0, dt, 5, scheme="ssprk3")).max()
    bound = 5 * dt * FLUX_TOL * flux_scale(u0, (2 * math.pi,) * 3)
    assert err <= bound, (err, bound)
    s.close()


def test_fp32_bulk_tile_variants_bitwise_identical(ns3d):
    """The FP32-bulk passes have one tile shape: setting another variant on the context changes
    nothing (the same bits), on a grid with nx even (the y and z passes' paired epilogue)."""
    import torch
    n = (20, 36, 18)
    u = I.random_smooth(*n, seed=6, amp=0.1, mach=0.5)
    outs = []
    for v in range(3):
        s = ns3d.Solver(*n, mu_eff=3e-3, precision=ns3d.NS3D_FP32_BULK)
        ns3d.set_solver_variant(s, v)
        ud = torch.from_numpy(u.copy()).cuda()
        r = s.rhs(ud).cpu().numpy()
        s.rk_step(ud, 0.01, 2)
        outs.append((r, ud.cpu().numpy()))
        s.close()
    for v in (1, 2):
        assert np.array_equal(outs[v][0], outs[0][0]) and np.array_equal(outs[v][1], outs[0][1])


def test_fp32_bulk_hit256_sampled_points(ns3d, orc):
    """256^3 decaying turbulence (the tile shape leaves ragged tiles at 256): the FP32-bulk
    RHS at 2048 sampled points, including the periodic seams and tile edges, against the
    oracle's local evaluation, within the FP32 bound."""
    import torch
    n = 256
    u = I.isotropic_turbulence(n, seed=0)
    mu = I.hit_mu_eff()
    s = ns3d.Solver(n, n, n, mu_eff=mu, precision=ns3d.NS3D_FP32_BULK)
    r = s.rhs(_gpu(u))
    rng = np.random.default_rng(3)
    edges = [0, 1, 26, 27, 28, 53, 54, 242, 243, 255]
    extra = [(k * n + j) * n + i for i in edges for j in (0, 27, 255) for k in (0, 128, 255)]
    idx = np.unique(np.concatenate([rng.choice(n ** 3, size=2048, replace=False), extra]))
    r32 = r.reshape(5, -1)[:, torch.from_numpy(idx).cuda()].cpu().numpy()
    del r
    s.close()
    r64 = orc.rhs_points(orc.Params(n, n, n, mu_eff=mu), u, idx).T
    err = np.abs(r32 - r64).max() / flux_scale(u, (2 * math.pi,) * 3)
    assert err <= FLUX_TOL, err
