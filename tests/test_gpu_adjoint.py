"""The hand-written adjoint (ns3d_rhs_vjp, ns3d_rk_step_vjp, ns3d_functional,
ns3d_traj_forward / ns3d_traj_vjp and the torch.autograd Functions) against the
oracle's own discrete adjoint: J^T lam from the dense forward-mode Jacobian on tiny
grids, and dot-product identities <lam, J w> = <J^T lam, w> with the oracle's exact
forward-mode derivatives on grids that span several tiles with ragged edges."""
import numpy as np
import pytest

from paper_2211_16718_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_DENSE = 1e-11   # vector relative max-norm, J^T lam vs the dense oracle adjoint
TOL_DOT = 1e-11     # relative difference of the two sides of a dot-product identity


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
def dual(oracle):
    from oracle import dual_oracle as D
    D.build()
    D.set_threads(8)
    return D


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _scaled_noise(u, seed):
    return np.random.default_rng(seed).normal(size=u.shape) * np.abs(u).max(axis=(1, 2, 3), keepdims=True)


def _case(name):
    """(state, oracle-params kwargs, grid)"""
    if name == "viscous_ragged":
        n = (7, 6, 5)
        return I.random_smooth(*n, seed=31, amp=0.12, mach=0.5), dict(mu_eff=2e-2), n
    if name == "inviscid_8":
        n = (8, 8, 8)
        return I.random_smooth(*n, seed=32, amp=0.1, mach=0.6), dict(mu_eff=0.0), n
    if name == "shock_tube":
        n = (12, 4, 4)
        return I.shock_tube(*n, axis=0), dict(mu_eff=0.0), n
    if name == "shock_tube_z":
        n = (4, 4, 12)
        return I.shock_tube(*n, axis=2), dict(mu_eff=1e-3), n
    if name == "hit_8":
        return I.isotropic_turbulence(8, seed=3), dict(mu_eff=I.hit_mu_eff()), (8, 8, 8)
    raise KeyError(name)


@pytest.mark.parametrize("name", ["viscous_ragged", "inviscid_8", "shock_tube", "shock_tube_z", "hit_8"])
@pytest.mark.parametrize("precision", [0, 2])
def test_rhs_vjp_equals_dense_oracle_adjoint(ns3d, oracle, dual, name, precision):
    u, kw, n = _case(name)
    P = oracle.Params(*n, **kw)
    lam = _scaled_noise(u, 5)[::-1].copy()  # any adjoint field
    ref = dual.rhs_vjp_dense(P, u, lam)
    s = ns3d.Solver(*n, precision=precision, **kw)
    got = s.rhs_vjp(_dev(u), _dev(lam)).cpu().numpy()
    s.check()
    s.close()
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err <= TOL_DENSE, err


# The grids put one, two and three adjoint tiles (32 points in the NS3D_FP64 form, 16 in the
# strict one) along each pencil, with ragged last tiles: the tile seams and the halos that cross
# them are exercised in every direction.
@pytest.mark.parametrize("n,kw,seed", [((20, 16, 12), dict(mu_eff=5e-3), 1),
                                       ((33, 18, 17), dict(mu_eff=0.0), 2),
                                       ((12, 40, 9), dict(mu_eff=1e-3, harten_delta=0.4), 3),
                                       ((10, 12, 72), dict(mu_eff=2e-3), 4),
                                       ((70, 9, 10), dict(mu_eff=2e-3), 5)])
def test_rhs_vjp_dot_product_identity(ns3d, oracle, dual, n, kw, seed):
    u = I.random_smooth(*n, seed=seed, amp=0.15, mach=0.6)
    P = oracle.Params(*n, **kw)
    s = ns3d.Solver(*n, **kw)
    lam = np.random.default_rng(seed + 10).normal(size=u.shape)
    jtl = s.rhs_vjp(_dev(u), _dev(lam)).cpu().numpy()
    for k in range(2):
        w = _scaled_noise(u, seed + 20 + k)
        _, jw = dual.rhs_jvp(P, u, w)
        lhs, rhs = float((lam * jw).sum()), float((jtl * w).sum())
        assert abs(lhs - rhs) <= TOL_DOT * (np.abs(lam * jw).sum()), (lhs, rhs)
    s.close()


def test_rhs_vjp_is_deterministic_and_bitwise_repeatable(ns3d):
    n = (24, 20, 18)
    u = I.random_smooth(*n, seed=4, amp=0.1)
    lam = np.random.default_rng(1).normal(size=u.shape)
    s = ns3d.Solver(*n, mu_eff=3e-3)
    a = s.rhs_vjp(_dev(u), _dev(lam)).cpu().numpy()
    b = s.rhs_vjp(_dev(u), _dev(lam)).cpu().numpy()
    assert np.array_equal(a, b)
    s.close()


@pytest.mark.parametrize("rk", [0, 1])
def test_rk_step_vjp_dot_product_identity(ns3d, oracle, dual, rk):
    n = (16, 12, 10)
    u = I.random_smooth(*n, seed=7, amp=0.12, mach=0.5)
    kw = dict(mu_eff=4e-3)
    P = oracle.Params(*n, **kw)
    dt = 0.02
    s = ns3d.Solver(*n, rk=rk, **kw)
    ub = np.random.default_rng(3).normal(size=u.shape)
    ubd = _dev(ub)
    ud = _dev(u)
    s.rk_step_vjp(ud, ubd, dt)
    got = ubd.cpu().numpy()
    assert np.array_equal(ud.cpu().numpy(), u)  # the state is not modified
    scheme = "rk4" if rk == 0 else "ssprk3"
    for k in range(2):
        w = _scaled_noise(u, 40 + k)
        _, dphi = dual.rk_step_jvp(P, u, w, dt, 1, scheme)
        lhs, rhs = float((ub * dphi).sum()), float((got * w).sum())
        assert abs(lhs - rhs) <= TOL_DOT * np.abs(ub * dphi).sum(), (lhs, rhs)
    s.close()


@pytest.mark.parametrize("which", ["ke", "enstrophy"])
def test_functional_gradient_equals_oracle(ns3d, oracle, dual, which):
    n = (7, 6, 5)
    u = I.random_smooth(*n, seed=12, amp=0.2, mach=0.6)
    P = oracle.Params(*n)
    s = ns3d.Solver(*n)
    val, g = s.functional(_dev(u), which, grad=True)
    st = oracle.stats(P, u)
    assert abs(val - st[which]) <= 1e-13 * abs(st[which])
    k = 5 if which == "ke" else 6
    ref = np.zeros(u.size)
    e = np.zeros(u.size)
    for j in range(u.size):
        e[j] = 1.0
        ref[j] = dual.stats_jvp(P, u, e.reshape(u.shape))[1][k]
        e[j] = 0.0
    ref = ref.reshape(u.shape)
    got = g.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    s.close()


@pytest.mark.parametrize("rk,which", [(0, "ke"), (1, "enstrophy")])
def test_trajectory_gradient_matches_oracle_directional_derivatives(ns3d, oracle, dual, rk, which):
    """Gradient of a final-time functional through 11 steps with checkpoints every 4
    (a ragged last segment), against the oracle's forward-mode derivative along seeded
    directions."""
    n = (16, 14, 12)
    u = I.random_smooth(*n, seed=21, amp=0.1, mach=0.4)
    kw = dict(mu_eff=5e-3)
    P = oracle.Params(*n, **kw)
    dt, nsteps = 0.02, 11
    s = ns3d.Solver(*n, rk=rk, **kw)
    ud = _dev(u)
    s.traj_forward(ud, dt, nsteps, 4)
    uN = ud.cpu().numpy()
    ref_uN = oracle.rk_step(P, u, dt, nsteps, "rk4" if rk == 0 else "ssprk3")
    assert np.abs(uN - ref_uN).max() / np.abs(ref_uN).max() <= 1e-10
    _, g = s.functional(ud, which, grad=True)
    s.traj_vjp(g)
    got = g.cpu().numpy()
    k = 5 if which == "ke" else 6
    for j in range(2):
        w = _scaled_noise(u, 60 + j)
        xN, dN = dual.rk_step_jvp(P, u, w, dt, nsteps, "rk4" if rk == 0 else "ssprk3")
        dref = dual.stats_jvp(P, xN, dN)[1][k]
        dgot = float((got * w).sum())
        assert abs(dgot - dref) <= 1e-9 * abs(dref), (dgot, dref)
    s.close()


def test_autograd_functions_agree_with_the_c_calls(ns3d):
    import torch
    from paper_2211_16718_gb300 import autograd as A
    n = (12, 10, 8)
    u = I.random_smooth(*n, seed=2, amp=0.1, mach=0.4)
    s = ns3d.Solver(*n, mu_eff=2e-3)
    dt = 0.03
    u0 = _dev(u).requires_grad_()
    ke = A.functional(A.trajectory(u0, s, dt, 7, every=3), s, "ke")
    ke.backward()
    ud = _dev(u)
    s.traj_forward(ud, dt, 7, 3)
    val, g = s.functional(ud, "ke", grad=True)
    assert abs(ke.item() - val) == 0.0
    s.traj_vjp(g)
    assert torch.equal(u0.grad, g)
    # one RK step and the RHS
    u1 = _dev(u).requires_grad_()
    lam = torch.randn_like(u1)
    (A.rk_step(u1, s, dt) * lam).sum().backward()
    ref = lam.clone()
    s.rk_step_vjp(_dev(u), ref, dt)
    assert torch.equal(u1.grad, ref)
    u2 = _dev(u).requires_grad_()
    (A.rhs(u2, s) * lam).sum().backward()
    assert torch.equal(u2.grad, s.rhs_vjp(_dev(u), lam))
    s.close()


def test_autograd_chained_trajectories_on_one_solver(ns3d):
    """A trajectory followed by a multi-step rk_step on the same Solver: the rk_step's
    backward runs first and records its own trajectory in the library, so the trajectory's
    backward must not reverse that recording.  The gradient equals the C-call path (each
    recording reversed in turn), and two trajectories recorded before one backward give
    the gradient of the one they belong to."""
    import torch
    from paper_2211_16718_gb300 import autograd as A
    n = (12, 10, 8)
    u = I.random_smooth(*n, seed=3, amp=0.1, mach=0.4)
    s = ns3d.Solver(*n, mu_eff=2e-3)
    dt = 0.03
    u0 = _dev(u).requires_grad_()
    ke = A.functional(A.rk_step(A.trajectory(u0, s, dt, 5, every=2), s, dt, nsteps=3), s, "ke")
    ke.backward()
    ua = _dev(u)
    s.traj_forward(ua, dt, 5, 2)
    ub = ua.clone()
    s.traj_forward(ub, dt, 3, 3)
    val, g = s.functional(ub, "ke", grad=True)
    assert ke.item() == val
    s.traj_vjp(g)                   # reverse of the 3 steps
    s.traj_forward(_dev(u), dt, 5, 2)
    s.traj_vjp(g)                   # reverse of the first 5 steps
    assert torch.equal(u0.grad, g)
    # two recordings before one backward: the first trajectory's gradient is its own
    u1 = _dev(u).requires_grad_()
    y1 = A.trajectory(u1, s, dt, 4, every=2)
    y2 = A.trajectory(_dev(u), s, dt, 2, every=1)  # records over the first one
    A.functional(y1, s, "ke").backward()
    uc = _dev(u)
    s.traj_forward(uc, dt, 4, 2)
    _, g1 = s.functional(uc, "ke", grad=True)
    s.traj_vjp(g1)
    assert torch.equal(u1.grad, g1)
    del y2
    s.close()


def test_gradient_matches_central_differences_of_the_gpu_path(ns3d):
    """d KE(u_N)/d u_0 along seeded directions against central differences of the GPU
    forward path itself (relative step 1e-6 of each field's scale)."""
    n = (24, 24, 24)
    u = I.taylor_green(24, v0=0.1)
    u = u + 1e-3 * _scaled_noise(u, 9)  # off the symmetry planes of the vortex
    s = ns3d.Solver(*n, mu_eff=2.5e-4)
    dt, nsteps = 0.05, 20
    ud = _dev(u)
    s.traj_forward(ud, dt, nsteps, 8)
    _, g = s.functional(ud, "ke", grad=True)
    s.traj_vjp(g)
    got = g.cpu().numpy()

    def ke_of(x):
        xd = _dev(x)
        s.rk_step(xd, dt, nsteps)
        return s.functional(xd, "ke")[0]

    for j in range(3):
        w = _scaled_noise(u, 80 + j)
        h = 1e-6
        fd = (ke_of(u + h * w) - ke_of(u - h * w)) / (2 * h)
        ad = float((got * w).sum())
        assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)
    s.close()


def test_adjoint_rejects_bad_use(ns3d):
    import torch
    n = (8, 8, 8)
    u = _dev(I.random_smooth(*n, seed=1))
    s = ns3d.Solver(*n)
    with pytest.raises(ns3d.Ns3dError):
        s.traj_vjp(torch.zeros_like(u))  # nothing recorded
    with pytest.raises(ns3d.Ns3dError):
        s.rhs_vjp(u, u, out=u)  # aliasing
    s.close()
    s32 = ns3d.Solver(*n, precision=ns3d.NS3D_FP32_BULK)
    with pytest.raises(ns3d.Ns3dError):
        s32.rhs_vjp(u, torch.ones_like(u))
    s32.close()


@pytest.mark.parametrize("rk", [0, 1])
def test_trajectory_reversal_equals_stepwise_vjps_bitwise(ns3d, rk):
    """The checkpointed reverse sweep (stage states kept from the segment recompute) gives the
    same bits as reversing the steps one by one with ns3d_rk_step_vjp."""
    import torch
    n = (12, 10, 8)
    u = I.random_smooth(*n, seed=5, amp=0.1, mach=0.4)
    s = ns3d.Solver(*n, mu_eff=3e-3, rk=rk)
    dt, nsteps = 0.02, 7
    states = [torch.from_numpy(u.copy()).cuda()]
    for _ in range(nsteps):
        x = states[-1].clone()
        s.rk_step(x, dt, 1)
        states.append(x)
    lam = torch.from_numpy(np.random.default_rng(2).normal(size=u.shape)).cuda()
    g1 = lam.clone()
    for k in range(nsteps - 1, -1, -1):
        s.rk_step_vjp(states[k], g1, dt)
    x = states[0].clone()
    s.traj_forward(x, dt, nsteps, 3)
    assert torch.equal(x, states[-1])
    g2 = lam.clone()
    s.traj_vjp(g2)
    assert torch.equal(g1, g2)
    s.close()


@pytest.mark.parametrize("precision", [0, 2])
def test_rhs_vjp_on_grids_smaller_than_the_stencil(ns3d, oracle, dual, precision):
    """Dimensions of 1-3 points: every stencil wraps around the periodic box several times."""
    n = (3, 2, 1)
    u = I.random_smooth(*n, seed=14, amp=0.1, mach=0.5)
    kw = dict(mu_eff=1e-2)
    P = oracle.Params(*n, **kw)
    lam = np.random.default_rng(8).normal(size=u.shape)
    ref = dual.rhs_vjp_dense(P, u, lam)
    s = ns3d.Solver(*n, precision=precision, **kw)
    got = s.rhs_vjp(_dev(u), _dev(lam)).cpu().numpy()
    s.check()
    s.close()
    assert np.abs(got - ref).max() <= TOL_DENSE * np.abs(ref).max()


def test_adjoint_double_float_range_is_reported(ns3d):
    """Data differences far beyond ~1e9 exceed the double-float range of the NS3D_FP64
    adjoint: it reports NS3D_ERANGE; the strict form handles them.  Adjoint inputs of any
    scale are fine (each tile works relative to the power of two of its largest |lambda|)."""
    import torch
    n = 16
    x = I.grid(n)
    shp = (n, n, n)
    p = 1e25 * (1.0 + 0.1 * np.sin(x))[None, None, :] * np.ones(shp)
    zero = np.zeros(shp)
    u = _dev(I.to_conserved(np.ones(shp), zero, zero, zero, p))
    lam = torch.ones_like(u) * torch.linspace(0.0, 1.0, n, dtype=torch.float64, device="cuda")
    s = ns3d.Solver(n, n, n, precision=ns3d.NS3D_FP64_STRICT)
    ref = s.rhs_vjp(u, lam)
    s.check()
    assert bool(torch.isfinite(ref).all())
    s.close()
    s = ns3d.Solver(n, n, n, precision=ns3d.NS3D_FP64)
    s.rhs_vjp(u, lam)
    with pytest.raises(ns3d.Ns3dError) as ei:
        s.check()
    assert ei.value.code == ns3d.NS3D_ERANGE
    # ordinary data, adjoint scaled by 1e-200 and 1e+200: the same result scaled exactly
    v = _dev(I.random_smooth(12, 12, 12, seed=3, amp=0.1))
    lam = torch.from_numpy(np.random.default_rng(0).normal(size=(5, 12, 12, 12))).cuda()
    s2 = ns3d.Solver(12, 12, 12, mu_eff=1e-3)
    a = s2.rhs_vjp(v, lam)
    for scale in (2.0 ** -660, 2.0 ** 660):
        b = s2.rhs_vjp(v, lam * scale)
        s2.check()
        assert torch.equal(b, a * scale)
    s2.close()
