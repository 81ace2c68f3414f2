"""Pins of the oracle's WENO5 reconstruction (arXiv 2211.16718, Sec. 2.2) against
exact arithmetic, the paper's printed coefficients and the behaviour the paper states."""
import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_stencils():
    rows = {}
    with open(os.path.join(GOLDEN, "weno5_stencils.txt")) as f:
        for line in f:
            line = line.split("#")[0].split()
            if line:
                rows[line[0]] = [Fr(t) for t in line[1:]]
    return rows


def _quadratic_through_cell_averages(cells, avgs):
    """Exact coefficients (a0, a1, a2) of P(x) = a0 + a1 x + a2 x^2 whose averages over the
    unit cells [m - 1/2, m + 1/2], m in cells, equal avgs (Gaussian elimination in Q)."""
    def avg_row(m):
        lo, hi = Fr(2 * m - 1, 2), Fr(2 * m + 1, 2)
        return [hi - lo, (hi ** 2 - lo ** 2) / 2, (hi ** 3 - lo ** 3) / 3]
    A = [avg_row(m) + [Fr(a)] for m, a in zip(cells, avgs)]
    n = 3
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [x - f * y for x, y in zip(A[r], A[c])]
    return [A[i][3] / A[i][i] for i in range(n)]


STENCILS = {0: (-2, -1, 0), 1: (-1, 0, 1), 2: (0, 1, 2)}  # cells of candidate k relative to j


def test_candidates_equal_polynomial_reconstruction(oracle):
    """Candidate k is the quadratic with the cell averages of its 3 cells, evaluated at
    x_{j+1/2}; derived here in exact arithmetic, compared with the oracle and the paper."""
    gold = _golden_stencils()
    for k, cells in STENCILS.items():
        exact = []
        for unit in range(5):  # coefficient of f_{j-2+unit}
            avgs = [Fr(1) if (m + 2) == unit else Fr(0) for m in cells]
            a = _quadratic_through_cell_averages(cells, avgs)
            xh = Fr(1, 2)
            exact.append(a[0] + a[1] * xh + a[2] * xh * xh)
        assert exact == gold[f"cand{k + 1}"], f"paper's candidate {k + 1} differs from its definition"
        for unit in range(5):
            q = np.zeros(5)
            q[unit] = 1.0
            got = oracle.weno5_candidates(q)[k]
            assert got == pytest.approx(float(exact[unit]), abs=1e-15)


def test_optimal_weights_give_printed_fifth_order_stencil(oracle):
    gold = _golden_stencils()
    c = gold["weights"]
    combo = [sum(c[k] * gold[f"cand{k + 1}"][u] for k in range(3)) for u in range(5)]
    assert combo == gold["optimal"]
    assert sum(c) == 1
    for unit in range(5):
        q = np.zeros(5)
        q[unit] = 1.0
        got = oracle.weno5(q, linear=True)
        assert got == pytest.approx(float(gold["optimal"][unit]), abs=1e-15)


def _cell_averages_of_poly(coeffs, centers, h):
    """Exact cell averages of sum_n coeffs[n] x^n over [x_c - h/2, x_c + h/2]."""
    out = []
    for xc in centers:
        lo, hi = xc - h / 2, xc + h / 2
        out.append(sum(cn * (hi ** (n + 1) - lo ** (n + 1)) / (n + 1) for n, cn in enumerate(coeffs)) / h)
    return np.array(out)


@pytest.mark.parametrize("seed", range(5))
def test_candidates_exact_for_quadratics_optimal_for_quartics(oracle, seed):
    """Each candidate reproduces cell averages of a degree-2 polynomial exactly at the
    interface; the optimal combination does so up to degree 4 (Sec. 2.2)."""
    rng = np.random.default_rng(seed)
    h = 0.37
    centers = (np.arange(5) - 2) * h + 0.11
    xi = centers[2] + h / 2
    c2 = rng.normal(size=3)
    q2 = _cell_averages_of_poly(c2, centers, h)
    exact2 = np.polynomial.polynomial.polyval(xi, c2)
    cand = oracle.weno5_candidates(q2)
    np.testing.assert_allclose(cand, exact2, rtol=0, atol=1e-13)
    c4 = rng.normal(size=5)
    q4 = _cell_averages_of_poly(c4, centers, h)
    exact4 = np.polynomial.polynomial.polyval(xi, c4)
    assert oracle.weno5(q4, linear=True) == pytest.approx(exact4, abs=1e-13)
    # a cubic is not reproduced by a single candidate (the pin has power)
    c3 = np.array([0.0, 0.0, 0.0, 1.0])
    q3 = _cell_averages_of_poly(c3, centers, h)
    assert abs(oracle.weno5_candidates(q3)[0] - np.polynomial.polynomial.polyval(xi, c3)) > 1e-4


def _beta_from_definition(q, k):
    """Jiang-Shu smoothness indicator of candidate k: sum over l = 1, 2 of
    h^{2l-1} * integral over cell j of (d^l P/dx^l)^2, with h = 1 (exact rationals)."""
    cells = STENCILS[k]
    a = _quadratic_through_cell_averages(cells, [q[m + 2] for m in cells])
    # P' = a1 + 2 a2 x, P'' = 2 a2 on [-1/2, 1/2]
    lo, hi = Fr(-1, 2), Fr(1, 2)
    i1 = (a[1] ** 2) * (hi - lo) + 2 * a[1] * 2 * a[2] * (hi ** 2 - lo ** 2) / 2 + (2 * a[2]) ** 2 * (hi ** 3 - lo ** 3) / 3
    i2 = (2 * a[2]) ** 2 * (hi - lo)
    return i1 + i2


@pytest.mark.parametrize("seed", range(8))
def test_smoothness_indicators_equal_their_definition(oracle, seed):
    rng = np.random.default_rng(100 + seed)
    qi = [int(v) for v in rng.integers(-50, 51, size=5)]
    beta = oracle.weno5_beta(np.array(qi, dtype=float))
    for k in range(3):
        assert beta[k] == pytest.approx(float(_beta_from_definition(qi, k)), rel=1e-14, abs=1e-14)


@pytest.mark.parametrize("slope", [0.0, 1e-4, 0.3, -7.0])
def test_linear_data_gives_optimal_weights(oracle, slope):
    q = 2.5 + slope * np.arange(5)
    beta = oracle.weno5_beta(q)
    # the stencil differences cancel the offset 2.5: relative rounding grows like 2.5/|slope|
    rtol = 1e-14 * max(1.0, 2.5 / abs(slope)) if slope else 0.0
    np.testing.assert_allclose(beta, slope * slope, rtol=rtol, atol=0.0)
    w = oracle.weno5_weights(q)
    np.testing.assert_allclose(w, [0.1, 0.6, 0.3], rtol=max(1e-14, 4 * rtol))


def test_weights_sum_to_one_and_avoid_discontinuity(oracle):
    rng = np.random.default_rng(7)
    for _ in range(50):
        q = rng.normal(size=5) * rng.choice([1e-3, 1.0, 1e3])
        w = oracle.weno5_weights(q)
        assert abs(w.sum() - 1.0) < 1e-14 and (w >= 0).all()
    # a jump between f_j and f_{j+1}: only candidate 1 (cells j-2..j) is smooth
    w = oracle.weno5_weights(np.array([0.0, 0.0, 0.0, 1.0, 1.0]))
    assert w[0] > 0.999 and w[1] < 1e-3 and w[2] < 1e-3
    # a jump between f_{j-1} and f_j: candidate 3 (cells j..j+2) is the smooth one
    w = oracle.weno5_weights(np.array([0.0, 0.0, 1.0, 1.0, 1.0]))
    assert w[2] > 0.999


def _convergence(oracle, linear, Ns):
    errs = []
    for N in Ns:
        x = np.arange(N) * 2 * np.pi / N
        h = 2 * np.pi / N
        q = np.exp(np.sin(x))
        dq = np.cos(x) * q
        qL, qR = oracle.weno5_line(q, linear=linear)
        errs.append((np.abs((qL - np.roll(qL, 1)) / h - dq).max(), np.abs((qR - np.roll(qR, 1)) / h - dq).max()))
    return [(math.log2(a[0] / b[0]), math.log2(a[1] / b[1])) for a, b in zip(errs, errs[1:])]


def test_fifth_order_convergence_optimal_weights(oracle):
    """Conservative difference of interface values approximates q' to order 5 (Sec. 2.2)."""
    for oL, oR in _convergence(oracle, True, (32, 64, 128, 256)):
        assert 4.85 < oL < 5.15 and 4.85 < oR < 5.15


def test_fifth_order_convergence_nonlinear_weights(oracle):
    """With the nonlinear weights on smooth data, omega -> c and the order tends to 5."""
    orders = _convergence(oracle, False, (64, 128, 256))
    for oL, oR in orders:
        assert oL > 4.7 and oR > 4.7


def test_right_biased_is_mirror_of_left(oracle):
    rng = np.random.default_rng(3)
    q = rng.normal(size=17)
    qL, qR = oracle.weno5_line(q)
    # mirroring the line maps interface i+1/2 to interface (n-2-i)+1/2 and swaps L and R
    rL, rR = oracle.weno5_line(q[::-1].copy())
    n = q.size
    for i in range(n):
        j = (n - 2 - i) % n
        assert qL[i] == rR[j] and qR[i] == rL[j]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_weight_exponent_acts_on_eps_plus_beta(oracle, seed):
    """Reading of Sec. 2.2's nonlinear weights: alpha_k = c_k / (eps + beta_k)^p.  Whatever the
    indicators are, the ratio (omega_j / omega_k) / (c_j / c_k) = ((eps + beta_k) / (eps + beta_j))^p,
    so the p = 2 ratio is the square and the p = 3 ratio the cube of the p = 1 ratio.  A
    misplaced exponent (eps + beta_k^p) or a dropped one breaks these relations."""
    rng = np.random.default_rng(seed)
    c = np.array([0.1, 0.6, 0.3])
    for _ in range(20):
        q = rng.normal(size=5) * rng.uniform(1e-2, 1.0)
        w = {p: oracle.weno5_weights(q, eps=1e-6, p=p) for p in (1, 2, 3)}
        for j, k in ((0, 1), (2, 1), (0, 2)):
            r = {p: (w[p][j] / w[p][k]) / (c[j] / c[k]) for p in (1, 2, 3)}
            assert r[2] == pytest.approx(r[1] ** 2, rel=1e-12)
            assert r[3] == pytest.approx(r[1] ** 3, rel=1e-12)
