"""Pins of the oracle's whole right-hand side, Runge-Kutta update and statistics
(arXiv 2211.16718, Sec. 2.1-2.3) against closed forms, invariants and exact solutions."""
import math

import numpy as np
import pytest

from paper_2211_16718_gb300 import inputs as I

GAMMA = 1.4


def _P(oracle, nx, ny, nz, **kw):
    return oracle.Params(nx, ny, nz, **kw)


def test_free_stream_is_exactly_preserved(oracle):
    for (nx, ny, nz) in [(8, 8, 8), (9, 7, 5), (12, 1, 3)]:
        u = I.uniform(nx, ny, nz, rho=1.3, u=0.31, v=-0.2, w=0.07, p=0.8)
        r = oracle.rhs(_P(oracle, nx, ny, nz, mu_eff=3e-3), u)
        assert np.all(r == 0.0)


@pytest.mark.parametrize("shape", [(16, 12, 10), (9, 13, 7)])
def test_discrete_conservation(oracle, shape):
    """Central and conservative differences telescope: sum over the grid of each RHS
    component vanishes up to rounding (mass, momentum, energy)."""
    nx, ny, nz = shape
    u = I.random_smooth(nx, ny, nz, seed=2, amp=0.2, mach=0.5)
    r = oracle.rhs(_P(oracle, nx, ny, nz, mu_eff=2e-2), u)
    scale = np.abs(r).reshape(5, -1).max(axis=1)
    sums = r.reshape(5, -1).sum(axis=1)
    assert np.all(np.abs(sums) <= 64 * np.finfo(float).eps * scale * r[0].size)


def test_entropy_wave_reduces_to_scalar_weno(oracle):
    """rho = 1 + 0.2 sin x, u = 1, v = w = 0, p const: the jump of the reconstructed
    state is an entropy eigenvector (optimal weights), so the mass flux is the
    left-biased WENO5 value of rho and d(rho)/dt = -(rhoL_{i+1/2} - rhoL_{i-1/2})/dx."""
    n = 32
    x = I.grid(n)
    rho1 = 1.0 + 0.2 * np.sin(x)
    shp = (4, 3, n)
    rho = np.broadcast_to(rho1, shp).copy()
    u = I.to_conserved(rho, np.ones(shp), np.zeros(shp), np.zeros(shp), np.full(shp, 1 / GAMMA))
    P = _P(oracle, n, 3, 4, weno_linear=1)
    r = oracle.rhs(P, u)
    qL, _ = oracle.weno5_line(rho1, linear=True)
    expect = -(qL - np.roll(qL, 1)) / (2 * math.pi / n)
    np.testing.assert_allclose(r[0, 1, 2], expect, rtol=0, atol=1e-13)
    # and the exact solution rho(x - t): the RHS approximates -rho' with 5th-order error
    assert np.abs(r[0, 1, 2] + 0.2 * np.cos(x)).max() < 5e-5


def _s(theta):
    """Symbol of the 4th-order central first derivative: D sin(kx) = s(k h)/h cos(kx)."""
    return (8 * np.sin(theta) - np.sin(2 * theta)) / 6


def _mode_state(field, axis, amp, n, comp):
    """Uniform rho = 1, p = 1/gamma, with one velocity component = amp sin(x_axis)."""
    shp = (n, n, n)
    xs = I.grid(n)
    prof = amp * np.sin(xs)
    vel = [np.zeros(shp), np.zeros(shp), np.zeros(shp)]
    sl = [None, None, None]
    sl[2 - axis] = slice(None)
    vel[comp] = np.broadcast_to(prof[tuple(sl)], shp).copy()
    return I.to_conserved(np.ones(shp), vel[0], vel[1], vel[2], np.full(shp, 1 / GAMMA))


@pytest.mark.parametrize("axis,comp,factor", [(1, 0, 1.0), (2, 1, 1.0), (0, 0, 4.0 / 3.0), (2, 2, 4.0 / 3.0),
                                              (0, 2, 1.0)])
def test_viscous_single_mode_multiplier(oracle, axis, comp, factor):
    """Velocity component `comp` = A sin(x_axis): the viscous momentum term is
    factor * mu * D(D u) = -factor * mu * (s(h)/h)^2 A sin; factor 1 for shear,
    4/3 for compression (tau_ii = mu (2 - 2/3) du_i/dx_i, the symmetric-stress reading)."""
    n, A, mu = 16, 0.05, 0.01
    u = _mode_state(None, axis, A, n, comp)
    r = oracle.rhs_visc(_P(oracle, n, n, n, mu_eff=mu), u)
    h = 2 * math.pi / n
    xs = I.grid(n)
    prof = -factor * mu * (_s(h) / h) ** 2 * A * np.sin(xs)
    sl = [None, None, None]
    sl[2 - axis] = slice(None)
    expect = np.broadcast_to(prof[tuple(sl)], (n, n, n))
    np.testing.assert_allclose(r[1 + comp], expect, rtol=0, atol=1e-15)
    assert np.all(r[0] == 0)
    for other in range(3):
        if other != comp:
            assert np.abs(r[1 + other]).max() < 1e-18


def test_heat_conduction_single_mode(oracle):
    """T = 1 + A sin z at rest with p uniform: energy RHS = kappa D(D T) with
    kappa = mu/((gamma-1) Pr), i.e. -kappa (s(h)/h)^2 A sin z (Sec. 2.1 heat flux)."""
    n, A, mu, pr = 16, 0.02, 0.01, 0.72
    shp = (n, n, n)
    z = I.grid(n)[:, None, None] * np.ones(shp)
    T = 1.0 + A * np.sin(z)
    p = np.full(shp, 1 / GAMMA)
    rho = GAMMA * p / T
    zero = np.zeros(shp)
    u = I.to_conserved(rho, zero, zero, zero, p)
    r = oracle.rhs_visc(_P(oracle, n, n, n, mu_eff=mu, prandtl=pr), u)
    h = 2 * math.pi / n
    kappa = mu / ((GAMMA - 1) * pr)
    np.testing.assert_allclose(r[4], -kappa * (_s(h) / h) ** 2 * A * np.sin(z), rtol=0, atol=1e-14)
    assert np.abs(r[1:4]).max() == 0.0


def test_translation_symmetry_bitwise(oracle):
    nx, ny, nz = 10, 9, 8
    u = I.random_smooth(nx, ny, nz, seed=4, amp=0.1)
    P = _P(oracle, nx, ny, nz, mu_eff=5e-3)
    r = oracle.rhs(P, u)
    for ax in (1, 2, 3):
        rs = oracle.rhs(P, np.roll(u, 1, axis=ax))
        assert np.array_equal(rs, np.roll(r, 1, axis=ax))


def test_axis_permutation_symmetry(oracle):
    """Swapping x and y (and the u, v components) swaps the RHS the same way."""
    n = 10
    u = I.random_smooth(n, n, 7, seed=5, amp=0.1)
    P = _P(oracle, n, n, 7, mu_eff=5e-3)
    r = oracle.rhs(P, u)
    us = np.swapaxes(u, 2, 3)[[0, 2, 1, 3, 4]].copy()
    rs = oracle.rhs(P, us)
    expect = np.swapaxes(r, 2, 3)[[0, 2, 1, 3, 4]]
    np.testing.assert_allclose(rs, expect, rtol=0, atol=1e-13 * np.abs(r).max())


def test_reflection_symmetry(oracle):
    """x -> -x with u -> -u maps the solution to itself: the RHS mirrors, with the sign
    of the x-momentum component flipped (left- and right-biased roles swap)."""
    nx, ny, nz = 12, 6, 5
    u = I.random_smooth(nx, ny, nz, seed=6, amp=0.1)
    P = _P(oracle, nx, ny, nz, mu_eff=5e-3)
    r = oracle.rhs(P, u)

    def mirror(a):
        m = np.roll(a[..., ::-1], 1, axis=-1).copy()   # x_i -> x_{-i}
        m[1] = -m[1]
        return m

    np.testing.assert_allclose(oracle.rhs(P, mirror(u)), mirror(r), rtol=0, atol=1e-13 * np.abs(r).max())


def test_rhs_points_equals_full_rhs(oracle):
    nx, ny, nz = 11, 9, 7
    u = I.random_smooth(nx, ny, nz, seed=8, amp=0.1)
    P = _P(oracle, nx, ny, nz, mu_eff=1e-2)
    r = oracle.rhs(P, u).reshape(5, -1)
    idx = np.random.default_rng(0).choice(nx * ny * nz, size=40, replace=False)
    assert np.array_equal(oracle.rhs_points(P, u, idx), r[:, idx].T)


# ---- Runge-Kutta (Sec. 2.2: classical RK4 and three-stage TVD RK) -------------
@pytest.mark.parametrize("scheme,order", [("rk4", 4), ("ssprk3", 3)])
def test_rk_stability_polynomial(oracle, scheme, order):
    """On du/dt = A u one step multiplies by the truncated exponential sum_{j<=order} (dt A)^j/j!
    (both schemes are exact for linear problems up to their order)."""
    a, b, dt = -0.3, 1.7, 0.4
    A = np.array([[a, -b], [b, a]])
    u0 = np.array([0.7, -0.2])
    got = oracle.rk_generic(u0, dt, lambda v: A @ v, scheme=scheme)
    M = np.eye(2)
    term = np.eye(2)
    for j in range(1, order + 1):
        term = term @ (dt * A) / j
        M = M + term
    np.testing.assert_allclose(got, M @ u0, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("scheme,order", [("rk4", 4), ("ssprk3", 3)])
def test_rk_temporal_order_full_operator(oracle, scheme, order):
    """dt-halving at a fixed grid.  The operator uses the optimal WENO weights: with the
    Jiang-Shu weights and eps = 1e-6 the RHS has very large higher derivatives wherever
    beta ~ eps, so the asymptotic temporal regime starts only at much smaller dt."""
    nx, ny, nz = 12, 10, 8
    u0 = I.random_smooth(nx, ny, nz, seed=9, amp=0.1, mach=0.3)
    P = _P(oracle, nx, ny, nz, mu_eff=1e-2, weno_linear=1)
    T = 0.4

    def run(n):
        return oracle.rk_step(P, u0, T / n, n, scheme)

    ref = run(128)
    e = [np.abs(run(n) - ref).max() for n in (4, 8)]
    assert math.log2(e[0] / e[1]) == pytest.approx(order, abs=0.3)


def test_isentropic_vortex_converges_to_exact_solution(oracle):
    """Euler (mu = 0) advection of an isentropic vortex (z-independent, nz = 1): after
    t = 2 the error against the exact translated vortex falls with the grid."""
    L, T = 16.0, 2.0
    errs = []
    for n in (32, 64, 128):
        u0 = I.isentropic_vortex(n, n, 1, t=0.0, length=L)
        P = _P(oracle, n, n, 1, lx=L, ly=L, lz=1.0)
        dt = 0.4 / oracle.stats(P, u0)["max_wavespeed_over_dx"]
        m = int(math.ceil(T / dt))
        u = oracle.rk_step(P, u0, T / m, m)
        ue = I.isentropic_vortex(n, n, 1, t=T, length=L)
        errs.append(np.abs(u - ue).max())
    assert errs[2] < 1e-4
    assert math.log2(errs[0] / errs[1]) > 3.0 and math.log2(errs[1] / errs[2]) > 3.0


# ---- statistics -------------------------------------------------------------------
def test_tgv_statistics_closed_forms(oracle):
    """Taylor-Green with rho = 1 at t = 0: KE = V0^2/8 and, with the 4th-order derivative,
    enstrophy <|omega|^2>/2 = (3/8) V0^2 (s(h)/h)^2 (discrete orthogonality)."""
    n, v0 = 16, 0.1
    u = I.taylor_green(n, v0=v0, isothermal=False)
    P = _P(oracle, n, n, n)
    st = oracle.stats(P, u)
    h = 2 * math.pi / n
    vol = (2 * math.pi) ** 3
    assert st["ke"] == pytest.approx(v0 * v0 / 8, rel=1e-13)
    assert st["enstrophy"] == pytest.approx(3 / 8 * v0 * v0 * (_s(h) / h) ** 2, rel=1e-12)
    assert st["mass"] == pytest.approx(vol, rel=1e-14)
    assert abs(st["momx"]) < 1e-14 and abs(st["momy"]) < 1e-14 and st["momz"] == 0.0
    assert st["energy"] == pytest.approx(vol * (1 / (GAMMA * (GAMMA - 1)) + v0 * v0 / 8), rel=1e-13)
    assert st["rho_min"] == 1.0
    assert st["p_min"] == pytest.approx(1 / GAMMA - 3 * v0 * v0 / 8, rel=1e-13)


def test_tgv_isothermal_extremes_and_wave_speed(oracle):
    """Isothermal Taylor-Green (rho = gamma p, so p/rho = 1/gamma and c = 1 at every point) on
    a grid holding x, y = pi/2 and z = 0: p_min = 1/gamma - 3 V0^2/8 where
    (cos 2x + cos 2y)(cos 2z + 2) = -6, rho_min = gamma p_min at the same point, the largest
    (|u_d| + c)/dx_d is (V0 + 1)/h (|u| = V0 at x = pi/2, y = z = 0), and the total mass is the
    box volume (the cosines sum to zero over the grid)."""
    n, v0 = 16, 0.1
    u = I.taylor_green(n, v0=v0, isothermal=True)
    st = oracle.stats(_P(oracle, n, n, n), u)
    h = 2 * math.pi / n
    pmin = 1 / GAMMA - 3 * v0 * v0 / 8
    assert st["p_min"] == pytest.approx(pmin, rel=1e-13)
    assert st["rho_min"] == pytest.approx(GAMMA * pmin, rel=1e-13)
    assert st["max_wavespeed_over_dx"] == pytest.approx((v0 + 1) / h, rel=1e-13)
    assert st["mass"] == pytest.approx((2 * math.pi) ** 3, rel=1e-13)


def test_uniform_state_wave_speed(oracle):
    u = I.uniform(8, 6, 4, rho=2.0, u=0.3, v=-0.5, w=0.1, p=0.7)
    P = _P(oracle, 8, 6, 4, lx=1.0, ly=2.0, lz=3.0)
    c = math.sqrt(GAMMA * 0.7 / 2.0)
    expect = max((0.3 + c) * 8 / 1.0, (0.5 + c) * 6 / 2.0, (0.1 + c) * 4 / 3.0)
    assert oracle.stats(P, u)["max_wavespeed_over_dx"] == pytest.approx(expect, rel=1e-14)


def test_cfl_reading_matches_paper_128_dt(oracle):
    """Sec. 2.3: the 128^3 decay run used dt = 0.025 at CFL about 1.  With
    CFL = dt max(|u_d| + c)/dx_d on the synthetic initial field the CFL is within 30 %."""
    n = 128
    u = I.isotropic_turbulence(n, seed=0)
    st = oracle.stats(oracle.Params(n, n, n), u)
    cfl = 0.025 * st["max_wavespeed_over_dx"]
    assert 0.7 < cfl < 1.3


def test_rhs_at_a_point_is_local_to_an_11_cube_window(oracle):
    """The right-hand side at a point depends only on the state within 4 points along
    the axes, so evaluating it on the 11^3 periodic window centred on the point gives the
    full-grid value bitwise (the basis of the sampled parity checks on grids the oracle
    cannot hold)."""
    import numpy as np
    from paper_2211_16718_gb300 import inputs as I
    n = 20
    u = I.isotropic_turbulence(n, seed=4)
    mu = I.hit_mu_eff()
    P = oracle.Params(n, n, n, mu_eff=mu)
    full = oracle.rhs(P, u)
    r, w = 5, 11
    h = 2 * np.pi / n
    Pw = oracle.Params(w, w, w, lx=w * h, ly=w * h, lz=w * h, mu_eff=mu)
    for (i, j, k) in [(0, 0, 0), (3, 17, 9), (19, 5, 12)]:
        iz, iy, ix = [(np.arange(-r, r + 1) + c) % n for c in (k, j, i)]
        win = np.ascontiguousarray(u[:, iz][:, :, iy][:, :, :, ix])
        got = oracle.rhs_points(Pw, win, [(r * w + r) * w + r])[0]
        assert np.array_equal(got, full[:, k, j, i])
