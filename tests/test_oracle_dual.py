"""Pins of the forward-mode (dual-number) oracle, the reference for the hand-written adjoint.

The dual build must (i) reproduce the plain oracle's values bitwise, (ii) give the exact
derivative of the discrete operator.  (ii) is pinned against things the dual arithmetic
does not produce itself: the textbook Euler flux Jacobian, the Fourier symbol of the
operator linearised about a uniform state (optimal WENO5 weights, Roe dissipation |A|
from an eigendecomposition of the textbook Jacobian, 4th-order central viscous terms),
and Richardson-extrapolated central differences of the plain oracle on non-uniform states."""
import math

import numpy as np
import pytest

from paper_2211_16718_gb300 import inputs as I

G = 1.4


@pytest.fixture(scope="module")
def dual(oracle):
    from oracle import dual_oracle as D
    D.build()
    D.set_threads(4)
    return D


def flux_jacobian(U, d, gamma=G):
    """Textbook Jacobian dF_d/dU of the 3D Euler flux in conservative variables."""
    rho = U[0]
    V = np.array(U[1:4]) / rho
    q2 = V @ V
    p = (gamma - 1) * (U[4] - 0.5 * rho * q2)
    H = (U[4] + p) / rho
    phi = 0.5 * (gamma - 1) * q2
    n = np.zeros(3)
    n[d] = 1.0
    un = V[d]
    A = np.zeros((5, 5))
    A[0, 1:4] = n
    A[1:4, 0] = phi * n - V * un
    A[1:4, 1:4] = np.outer(V, n) - (gamma - 1) * np.outer(n, V) + un * np.eye(3)
    A[1:4, 4] = (gamma - 1) * n
    A[4, 0] = un * (phi - H)
    A[4, 1:4] = H * n - (gamma - 1) * un * V
    A[4, 4] = gamma * un
    return A


def test_values_bitwise_equal_plain_oracle(oracle, dual):
    u = I.random_smooth(10, 9, 7, seed=3, amp=0.1, mach=0.4)
    P = oracle.Params(10, 9, 7, mu_eff=3e-3)
    w = np.random.default_rng(1).normal(size=u.shape)
    r, _ = dual.rhs_jvp(P, u, w)
    assert np.array_equal(r, oracle.rhs(P, u))
    for scheme in ("rk4", "ssprk3"):
        x, _ = dual.rk_step_jvp(P, u, w, 0.01, 2, scheme)
        assert np.array_equal(x, oracle.rk_step(P, u, 0.01, 2, scheme))
    s, _ = dual.stats_jvp(P, u, w)
    assert np.array_equal(s, np.array(list(oracle.stats(P, u).values())))


def test_flux_jvp_is_textbook_jacobian(dual):
    rng = np.random.default_rng(7)
    for _ in range(6):
        rho = rng.uniform(0.5, 2.0)
        vel = rng.normal(size=3)
        p = rng.uniform(0.5, 2.0)
        U = np.array([rho, *(rho * vel), p / (G - 1) + 0.5 * rho * vel @ vel])
        w = rng.normal(size=5)
        for d in range(3):
            _, jw = dual.flux_jvp(U, w, d, G)
            ref = flux_jacobian(U, d) @ w
            assert np.abs(jw - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


def _uniform_state(n, rho, vel, p):
    e = p / (G - 1) + 0.5 * rho * float(np.dot(vel, vel))
    u = np.empty((5,) + n[::-1])
    vals = [rho, rho * vel[0], rho * vel[1], rho * vel[2], e]
    for v in range(5):
        u[v] = vals[v]
    return u


@pytest.mark.parametrize("d", [0, 1, 2])
def test_linearisation_about_uniform_state_is_fourier_symbol(oracle, dual, d):
    """JVP of a single Fourier mode about a uniform state, against the closed-form symbol:
    hyperbolic part -(1 - e^{-i th})/h [A (S_L + S_R)/2 - |A| (S_R - S_L)/2] with the
    optimal fifth-order interpolation symbols S_L, S_R, and viscous part -(s(th)/h)^2 times
    the linearised stress / heat-flux operator, s(t) = (8 sin t - sin 2t)/6."""
    n = (12, 10, 8)
    nd = n[d]
    h = 2 * math.pi / nd
    mu, pr = 2e-2, 0.72
    kappa = mu / ((G - 1) * pr)
    rho, p = 1.3, 0.9
    c = math.sqrt(G * p / rho)
    vel = np.array([0.25, -0.35, 0.15]) * c
    u0 = _uniform_state(n, rho, vel, p)
    P = oracle.Params(*n, mu_eff=mu, prandtl=pr)
    rng = np.random.default_rng(11 + d)
    what = rng.normal(size=5) + 1j * rng.normal(size=5)
    k = 2
    idx = np.arange(nd)
    phase = np.exp(1j * k * idx * h)
    shape = [1, 1, 1]
    shape[2 - d] = nd
    mode = phase.reshape(shape)
    w = np.real(what.reshape(5, 1, 1, 1) * mode[None])
    w = np.broadcast_to(w, u0.shape).copy()
    _, jw = dual.rhs_jvp(P, u0, w)

    th = k * h
    cL = np.array([2, -13, 47, 27, -3]) / 60.0
    SL = sum(cL[t] * np.exp(1j * th * (t - 2)) for t in range(5))
    SR = sum(cL[t] * np.exp(1j * th * (3 - t)) for t in range(5))
    A = flux_jacobian(u0[:, 0, 0, 0], d)
    lam, R = np.linalg.eig(A)
    absA = np.real(R @ np.diag(np.abs(lam)) @ np.linalg.inv(R))
    M = A * (SL + SR) / 2 - absA * (SR - SL) / 2
    hyp = -(1 - np.exp(-1j * th)) / h * (M @ what)
    # linearised primitives (u, v, w, T) of the perturbation
    E = u0[4, 0, 0, 0]
    m = rho * vel
    dvel = (what[1:4] - vel * what[0]) / rho
    dT = G * (G - 1) * (what[4] / rho - E * what[0] / rho**2 - (m @ what[1:4]) / rho**2
                        + (m @ m) * what[0] / rho**3)
    s = (8 * math.sin(th) - math.sin(2 * th)) / 6
    dd = -(s / h) ** 2   # symbol of the 4th-order central first derivative applied twice
    visc = np.zeros(5, dtype=complex)
    tau = np.array([mu * dvel[mm] for mm in range(3)], dtype=complex)
    tau[d] = (4.0 / 3.0) * mu * dvel[d]
    visc[1:4] = dd * tau
    visc[4] = dd * (vel @ tau + kappa * dT)
    ref = np.real((hyp + visc).reshape(5, 1, 1, 1) * mode[None])
    ref = np.broadcast_to(ref, u0.shape)
    assert np.abs(jw - ref).max() <= 1e-12 * np.abs(ref).max()


def _richardson(f, u, w, h):
    d1 = (f(u + h * w) - f(u - h * w)) / (2 * h)
    d2 = (f(u + 0.5 * h * w) - f(u - 0.5 * h * w)) / h
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("case", ["smooth_viscous", "shock_tube", "hit"])
def test_rhs_jvp_matches_richardson_differences(oracle, dual, case):
    if case == "smooth_viscous":
        u = I.random_smooth(12, 10, 8, seed=5, amp=0.12, mach=0.5)
        P = oracle.Params(12, 10, 8, mu_eff=5e-3)
    elif case == "shock_tube":
        u = I.shock_tube(16, 4, 4, axis=0)
        P = oracle.Params(16, 4, 4, mu_eff=0.0)
    else:
        u = I.isotropic_turbulence(12, seed=2)
        P = oracle.Params(12, 12, 12, mu_eff=I.hit_mu_eff())
    w = np.random.default_rng(3).normal(size=u.shape) * np.abs(u).max(axis=(1, 2, 3), keepdims=True)
    _, jw = dual.rhs_jvp(P, u, w)
    # the nonlinear weights have curvature ~1/(eps + beta)^3 where the data are flat, so
    # the step must be small; 1e-6 of the field scale sits between that and roundoff
    fd = _richardson(lambda x: oracle.rhs(P, x), u, w, 1e-6)
    err = np.abs(fd - jw).max() / np.abs(jw).max()
    assert err <= 1e-8, err


@pytest.mark.parametrize("scheme", ["rk4", "ssprk3"])
def test_rk_and_functional_jvp_match_differences(oracle, dual, scheme):
    # (not the Taylor-Green field: its symmetry planes carry velocities of ~1e-17 whose Roe
    # averages sit on the kink of |u_n|, which any finite difference step straddles)
    u = I.random_smooth(12, 12, 12, seed=8, amp=0.15, mach=0.5)
    P = oracle.Params(12, 12, 12, mu_eff=1e-2)
    w = np.random.default_rng(4).normal(size=u.shape) * np.abs(u).max(axis=(1, 2, 3), keepdims=True)
    dt = 0.05
    _, dx = dual.rk_step_jvp(P, u, w, dt, 3, scheme)
    fd = _richardson(lambda x: oracle.rk_step(P, x, dt, 3, scheme), u, w, 1e-6)
    assert np.abs(fd - dx).max() / np.abs(dx).max() <= 1e-8
    uN, dN = dual.rk_step_jvp(P, u, w, dt, 3, scheme)
    _, ds = dual.stats_jvp(P, uN, dN)
    ke = lambda x: oracle.stats(P, oracle.rk_step(P, x, dt, 3, scheme))["ke"]
    h = 1e-6
    fd_ke = (4 * (ke(u + 0.5 * h * w) - ke(u - 0.5 * h * w)) / h - (ke(u + h * w) - ke(u - h * w)) / (2 * h)) / 3
    assert abs(fd_ke - ds[5]) <= 5e-8 * abs(ds[5])


def test_kinetic_energy_derivative_closed_form(oracle, dual):
    u = I.random_smooth(8, 6, 5, seed=9, amp=0.2, mach=0.6)
    P = oracle.Params(8, 6, 5)
    w = np.random.default_rng(2).normal(size=u.shape)
    _, ds = dual.stats_jvp(P, u, w)
    V = u[1:4] / u[0]
    ref = np.mean((V * w[1:4]).sum(0) - 0.5 * (V * V).sum(0) * w[0])
    assert abs(ds[5] - ref) <= 1e-14 * abs(ref) + 1e-17
