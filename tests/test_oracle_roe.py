"""Pins of the oracle's convective flux and Roe upwinding (arXiv 2211.16718, Sec. 2.1
flux vectors, Sec. 2.2 Eq. Roe) against the mathematics of the Euler equations."""
import numpy as np
import pytest

GAMMA = 1.4


def _state(rho, u, v, w, p, gamma=GAMMA):
    return np.array([rho, rho * u, rho * v, rho * w, p / (gamma - 1) + 0.5 * rho * (u * u + v * v + w * w)])


def _random_state(rng, mach=0.8):
    rho = rng.uniform(0.5, 2.0)
    p = rng.uniform(0.3, 1.5)
    c = np.sqrt(GAMMA * p / rho)
    u, v, w = rng.uniform(-mach, mach, size=3) * c
    return _state(rho, u, v, w, p)


def _fd_jacobian(oracle, U, d, h=1e-6):
    J = np.zeros((5, 5))
    for m in range(5):
        e = np.zeros(5)
        e[m] = h * max(1.0, abs(U[m]))
        J[:, m] = (oracle.flux(U + e, d) - oracle.flux(U - e, d)) / (2 * e[m])
    return J


def test_flux_at_rest_is_pressure_only(oracle):
    U = _state(1.3, 0.0, 0.0, 0.0, 0.9)
    for d in range(3):
        F = oracle.flux(U, d)
        expect = np.zeros(5)
        expect[1 + d] = 0.9
        np.testing.assert_allclose(F, expect, atol=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_flux_jacobian_has_euler_characteristic_speeds(oracle, seed):
    """Eigenvalues of df/du are u_d - c, u_d (x3), u_d + c with c^2 = gamma p/rho."""
    rng = np.random.default_rng(seed)
    U = _random_state(rng)
    rho = U[0]
    vel = U[1:4] / rho
    p = (GAMMA - 1) * (U[4] - 0.5 * rho * vel @ vel)
    c = np.sqrt(GAMMA * p / rho)
    for d in range(3):
        ev = np.sort(np.linalg.eigvals(_fd_jacobian(oracle, U, d)).real)
        np.testing.assert_allclose(ev, np.sort([vel[d] - c, vel[d], vel[d], vel[d], vel[d] + c]), atol=2e-6)


def test_flux_rotation_covariance(oracle):
    """Permuting the axes together with the velocity components permutes the flux."""
    rng = np.random.default_rng(11)
    U = _random_state(rng)
    perm = [1, 2, 0]  # new axis a holds old axis perm[a]
    Up = np.array([U[0], U[1 + perm[0]], U[1 + perm[1]], U[1 + perm[2]], U[4]])
    for a in range(3):
        F = oracle.flux(U, perm[a])
        Fp = oracle.flux(Up, a)
        np.testing.assert_allclose(Fp, [F[0], F[1 + perm[0]], F[1 + perm[1]], F[1 + perm[2]], F[4]], rtol=1e-15, atol=1e-16)


@pytest.mark.parametrize("seed", range(6))
def test_eigenvectors_are_inverse_and_diagonalise_jacobian(oracle, seed):
    rng = np.random.default_rng(20 + seed)
    U = _random_state(rng)
    for d in range(3):
        X, Xi, lam = oracle.roe_eigensystem(U, U, d)
        np.testing.assert_allclose(Xi @ X, np.eye(5), atol=1e-13)
        A = oracle.roe_matrix(U, U, d)
        np.testing.assert_allclose(A, X @ np.diag(lam) @ Xi, atol=1e-13)
        np.testing.assert_allclose(A, _fd_jacobian(oracle, U, d), atol=5e-7)


@pytest.mark.parametrize("seed", range(10))
def test_roe_property(oracle, seed):
    """Roe's average makes A~ (U_R - U_L) = f(U_R) - f(U_L) exactly (Roe 1981)."""
    rng = np.random.default_rng(40 + seed)
    UL, UR = _random_state(rng), _random_state(rng)
    for d in range(3):
        A = oracle.roe_matrix(UL, UR, d)
        lhs = A @ (UR - UL)
        rhs = oracle.flux(UR, d) - oracle.flux(UL, d)
        np.testing.assert_allclose(lhs, rhs, atol=1e-13 * max(1.0, np.abs(rhs).max()))


def test_dissipation_matrix_eigenvalues_with_harten_fix(oracle):
    """|A| has eigenvalues |lambda_k|; Harten's fix lifts |u-c| < delta to (l^2+d^2)/(2d)."""
    rho, p = 1.0, 1.0 / GAMMA  # c = 1
    for un, fix in [(0.3, 0.1), (0.97, 0.1), (1.02, 0.2), (-0.99, 0.1)]:
        U = _state(rho, un, 0.1, -0.05, p)
        vel = np.array([un, 0.1, -0.05])
        q2 = vel @ vel
        H = (U[4] + p) / rho
        c = np.sqrt((GAMMA - 1) * (H - 0.5 * q2))
        lam = np.array([un - c, un, un, un, un + c])
        delta = fix * c
        absl = np.abs(lam)
        for k in (0, 4):
            if absl[k] < delta:
                absl[k] = (lam[k] ** 2 + delta ** 2) / (2 * delta)
        A = oracle.roe_matrix(U, U, 0, absval=True, harten_delta=fix)
        ev = np.sort(np.linalg.eigvals(A).real)
        np.testing.assert_allclose(ev, np.sort(absl), atol=1e-12)


def test_harten_fix_inactive_below_mach_09(oracle):
    """With |u| < 0.9 c the fix (delta = 0.1 c) never triggers: bitwise equal fluxes."""
    rng = np.random.default_rng(5)
    from oracle.oracle import Params
    for _ in range(20):
        us = np.array([_random_state(rng, mach=0.85) for _ in range(6)])
        for d in range(3):
            a = oracle.interface_flux(Params(8, 8, 8, harten_delta=0.1), d, us)
            b = oracle.interface_flux(Params(8, 8, 8, harten_delta=0.0), d, us)
            assert np.array_equal(a, b)


def test_interface_flux_consistency(oracle):
    """A uniform stencil gives the exact physical flux f(U) (consistency of Eq. Roe)."""
    from oracle.oracle import Params
    rng = np.random.default_rng(9)
    U = _random_state(rng)
    for d in range(3):
        F = oracle.interface_flux(Params(8, 8, 8), d, np.tile(U, (6, 1)))
        np.testing.assert_allclose(F, oracle.flux(U, d), rtol=1e-14, atol=1e-15)


def test_upwinding_selects_upwind_state_for_supersonic_flow(oracle):
    """All eigenvalues positive: F = f(uL) when uL, uR come from smooth linear data with
    optimal weights, i.e. the dissipation term equals (f^R - f^L)/2 exactly for a
    linear flux; here checked for a supersonic uniform-gradient density wave."""
    from oracle.oracle import Params
    P = Params(8, 8, 8, weno_linear=1, harten_delta=0.0)
    us = np.array([_state(1.0 + 0.01 * m, 2.0, 0.0, 0.0, 1.0 / GAMMA) for m in range(6)])
    F = oracle.interface_flux(P, 0, us)
    # left-biased reconstruction of each flux component, independently through weno5
    fl = np.array([oracle.flux(s, 0) for s in us])
    expect = np.array([oracle.weno5(fl[0:5, m], linear=True) for m in range(5)])
    np.testing.assert_allclose(F, expect, rtol=1e-9, atol=1e-12)


def _smooth_line(n):
    """A smooth x-dependent state (density, velocity and pressure all varying) on an n x 1 x 1 grid."""
    x = np.arange(n) * 2 * np.pi / n
    rho = 1 + 0.2 * np.sin(x) + 0.1 * np.cos(2 * x)
    u = 0.3 + 0.1 * np.sin(x + 0.4)
    p = 1 / GAMMA + 0.05 * np.cos(x)
    U = np.zeros((5, 1, 1, n))
    U[:, 0, 0, :] = _state(rho, u, 0.0 * x, 0.0 * x, p)
    return U


def test_roe_average_of_reconstructed_states_satisfies_the_roe_property(oracle):
    """Sec. 2.2 does not say which two states enter the Roe average at an interface: the grid
    points on either side (the reading taken) or the two WENO5 reconstructions (oracle switch
    roe_state=1).  With the average taken of the reconstructions, Roe's property
    A(u~)(u^R - u^L) = f(u^R) - f(u^L) holds for them; in supersonic flow every eigenvalue is
    positive, |A| = A, and the interface flux must then be exactly
    (f^L + f^R)/2 - (f(u^R) - f(u^L))/2, with f^L, f^R the reconstructions of the point fluxes
    and u^L, u^R those of the states (each through the pinned scalar WENO5, mirrored for the
    right-biased value).  The grid-point average does not satisfy it for these states."""
    from oracle.oracle import Params
    rng = np.random.default_rng(23)
    for d in range(3):
        for _ in range(5):
            us = []
            for _j in range(6):
                rho = rng.uniform(0.8, 1.3)
                p = rng.uniform(0.6, 0.9)
                vel = rng.uniform(-0.1, 0.1, size=3)
                vel[d] += 2.5 * np.sqrt(GAMMA * p / rho)  # Mach ~2.5 along d: all eigenvalues > 0
                us.append(_state(rho, *vel, p))
            us = np.array(us)
            fl = np.array([oracle.flux(s, d) for s in us])
            uL = np.array([oracle.weno5(us[0:5, m]) for m in range(5)])
            uR = np.array([oracle.weno5(us[5:0:-1, m]) for m in range(5)])
            fL = np.array([oracle.weno5(fl[0:5, m]) for m in range(5)])
            fR = np.array([oracle.weno5(fl[5:0:-1, m]) for m in range(5)])
            expect = 0.5 * (fL + fR) - 0.5 * (oracle.flux(uR, d) - oracle.flux(uL, d))
            F1 = oracle.interface_flux(Params(8, 8, 8, roe_state=1), d, us)
            np.testing.assert_allclose(F1, expect, rtol=1e-12, atol=1e-12 * np.abs(expect).max())
            F0 = oracle.interface_flux(Params(8, 8, 8, roe_state=0), d, us)
            assert np.abs(F0 - expect).max() > 1e-9 * np.abs(expect).max()


def test_roe_state_readings_agree_to_high_order_on_smooth_data(oracle):
    """On smooth data the two readings of the Roe-average states give right-hand sides that
    differ far below the RHS itself and shrink fast under refinement: the states only enter
    the dissipation, which multiplies the O(h^5) jump of the reconstructions."""
    from oracle.oracle import Params
    prev = None
    for n in (32, 64, 128, 256):
        U = _smooth_line(n)
        r0 = oracle.rhs(Params(n, 1, 1, mu_eff=0.0), U)
        r1 = oracle.rhs(Params(n, 1, 1, mu_eff=0.0, roe_state=1), U)
        d = np.abs(r0 - r1).max()
        assert d > 0.0  # the switch does change the arithmetic
        if prev is not None:
            assert prev / d >= 20.0, (n, prev, d)
        prev = d
    assert prev <= 1e-11 * np.abs(r0).max()


def test_roe_average_of_reconstructed_states_keeps_free_stream_and_conservation(oracle):
    """The alternative reading is still a conservative, consistent scheme: a uniform state
    in motion gives an exactly zero RHS, and the RHS sums to zero over the periodic grid."""
    from oracle.oracle import Params
    P = Params(12, 10, 8, mu_eff=0.0, roe_state=1)
    U = np.zeros((5, 8, 10, 12))
    U[:] = _state(1.3, 0.4, -0.2, 0.1, 0.9)[:, None, None, None]
    assert not np.any(oracle.rhs(P, U))
    rng = np.random.default_rng(17)
    x = np.arange(12) * 2 * np.pi / 12
    y = np.arange(10) * 2 * np.pi / 10
    z = np.arange(8) * 2 * np.pi / 8
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    rho = 1 + 0.2 * np.sin(X + 2 * Y) + 0.1 * rng.uniform() * np.cos(Z)
    u, v, w = 0.3 * np.sin(Y), 0.2 * np.cos(X + Z), 0.1 * np.sin(Z - X)
    p = 1 / GAMMA + 0.05 * np.cos(X - Y)
    W = _state(rho, u, v, w, p)
    R = oracle.rhs(P, W)
    scale = np.abs(R).max()
    for m in range(5):
        assert abs(R[m].sum()) <= 1e-13 * scale * R[m].size


def test_roe_average_of_the_two_grid_points_satisfies_the_roe_property(oracle):
    """The reading taken for Sec. 2.2's Roe average: the grid points i, i+1 on either side of the
    interface.  Pin: with linear weights and a stencil U_j = U_a + phi_j dU (every component
    varying along one state-space direction), each reconstruction is U_a + phi^ dU, so the jump
    u^R - u^L = kappa (U_{i+1} - U_i) with kappa = (phi^R - phi^L)/(phi_{i+1} - phi_i).  Roe's
    property for the pair (U_i, U_{i+1}) then makes the supersonic (|A| = A) interface flux
    exactly (f^L + f^R)/2 - kappa (f(U_{i+1}) - f(U_i))/2, with f^L, f^R the reconstructions of
    the point fluxes.  Another pair of states for the average breaks the identity."""
    from oracle.oracle import Params
    rng = np.random.default_rng(29)
    P = Params(8, 8, 8, weno_linear=1, harten_delta=0.0)
    for d in range(3):
        for _ in range(5):
            rho, p = rng.uniform(0.8, 1.2), rng.uniform(0.6, 0.9)
            vel = rng.uniform(-0.1, 0.1, size=3)
            vel[d] += 2.5 * np.sqrt(GAMMA * p / rho)  # Mach ~2.5 along d
            Ua = _state(rho, *vel, p)
            dU = _state(1.0, *rng.uniform(-0.5, 0.5, size=3), 1.0) * rng.uniform(-0.05, 0.05, size=5)
            phi = rng.uniform(-1.0, 1.0, size=6)
            phi[3] = phi[2] + rng.uniform(0.3, 0.8)  # a well-conditioned kappa
            us = np.array([Ua + phi[j] * dU for j in range(6)])
            fl = np.array([oracle.flux(s, d) for s in us])
            fL = np.array([oracle.weno5(fl[0:5, m], linear=True) for m in range(5)])
            fR = np.array([oracle.weno5(fl[5:0:-1, m], linear=True) for m in range(5)])
            kappa = (oracle.weno5(phi[5:0:-1], linear=True) - oracle.weno5(phi[0:5], linear=True)) / (phi[3] - phi[2])
            expect = 0.5 * (fL + fR) - 0.5 * kappa * (oracle.flux(us[3], d) - oracle.flux(us[2], d))
            F = oracle.interface_flux(P, d, us)
            np.testing.assert_allclose(F, expect, rtol=1e-11, atol=1e-11 * np.abs(expect).max())
