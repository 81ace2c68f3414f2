"""Storage modes: viscous fluxes one direction at a time (NS3D_STORAGE_LEAN) give the same
bits as all three at once; stage buffers are allocated on the first step; and a 1024^3
grid with SSP-RK3 fits on one GPU, its right-hand side checked against the oracle on
sampled 11^3 windows."""
import numpy as np
import pytest

from paper_2211_16718_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ns3d():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2211_16718_gb300 import build as B
    B.build()
    from paper_2211_16718_gb300 import ns3d as N
    N.lib()
    return N


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("rk", [0, 1])
def test_lean_storage_is_bitwise_identical(ns3d, precision, rk):
    import torch
    n = (20, 18, 16)
    u = I.random_smooth(*n, seed=3, amp=0.1, mach=0.5)
    out = {}
    for storage in (ns3d.NS3D_STORAGE_FULL, ns3d.NS3D_STORAGE_LEAN):
        s = ns3d.Solver(*n, mu_eff=4e-3, rk=rk, precision=precision, storage=storage)
        assert s.storage_info()["storage"] == storage
        ud = torch.from_numpy(u.copy()).cuda()
        r = s.rhs(ud).cpu().numpy()
        s.rk_step(ud, 0.02, 3)
        s.check()
        out[storage] = (r, ud.cpu().numpy())
        s.close()
    for a, b in zip(out[ns3d.NS3D_STORAGE_FULL], out[ns3d.NS3D_STORAGE_LEAN]):
        assert np.array_equal(a, b)


def test_lean_storage_adjoint_is_bitwise_identical(ns3d):
    import torch
    n = (16, 12, 10)
    u = I.random_smooth(*n, seed=4, amp=0.1, mach=0.5)
    lam = np.random.default_rng(0).normal(size=u.shape)
    res = []
    for storage in (ns3d.NS3D_STORAGE_FULL, ns3d.NS3D_STORAGE_LEAN):
        s = ns3d.Solver(*n, mu_eff=4e-3, storage=storage)
        ub = torch.from_numpy(lam.copy()).cuda()
        s.rk_step_vjp(torch.from_numpy(u.copy()).cuda(), ub, 0.02)
        res.append(ub.cpu().numpy())
        s.close()
    assert np.array_equal(res[0], res[1])


def test_stage_buffers_are_allocated_on_the_first_step(ns3d):
    import torch
    n = 16
    for rk, extra in ((0, 3), (1, 2)):  # RK4: two stage states + accumulator; SSP-RK3: two states
        s = ns3d.Solver(n, n, n, mu_eff=1e-3, rk=rk, storage=ns3d.NS3D_STORAGE_LEAN)
        b0 = s.storage_info()["device_bytes"]
        ud = torch.from_numpy(I.random_smooth(n, n, n, seed=1)).cuda()
        s.rhs(ud)
        assert s.storage_info()["device_bytes"] == b0
        s.rk_step(ud, 0.01, 1)
        assert s.storage_info()["device_bytes"] - b0 == extra * 5 * 8 * n ** 3
        s.close()


def test_bad_storage_mode_is_rejected(ns3d):
    with pytest.raises(ns3d.Ns3dError):
        ns3d.Solver(8, 8, 8, storage=7)


def test_1024_cubed_ssprk3_fits_and_matches_the_oracle_on_windows(ns3d, oracle):
    import torch
    free_b, _ = torch.cuda.mem_get_info()
    if free_b < 275e9:
        pytest.skip(f"needs ~270 GB of free device memory, {free_b / 1e9:.0f} GB free")
    import bench
    n = 1024
    u = I.isotropic_turbulence_device(n, seed=0)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    mu = I.hit_mu_eff()
    s = ns3d.Solver(n, n, n, mu_eff=mu, rk=ns3d.NS3D_SSPRK3)
    assert s.storage_info()["storage"] == ns3d.NS3D_STORAGE_LEAN
    rhs = torch.empty_like(u)
    s.rhs(u, rhs)
    s.check()
    chk = bench.window_oracle_check(u, rhs, mu, n_sample=8, seed=1)
    assert chk["max_rel_err"] <= 1e-12, chk
    del rhs
    torch.cuda.empty_cache()
    st0 = s.stats(u)
    s.rk_step(u, s.dt_from_cfl(u, 0.4), 1)
    st1 = s.stats(u)
    assert st1["status"] == 0
    assert abs(st1["mass"] - st0["mass"]) <= 1e-13 * st0["mass"]
    assert abs(st1["energy"] - st0["energy"]) <= 1e-13 * st0["energy"]
    s.close()
