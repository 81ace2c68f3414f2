"""Checks of the seeded initial conditions (arXiv 2211.16718, Sec. 2.3) and of the paper
constants used as defaults (golden fixture with citations)."""
import math
import os

import numpy as np
import pytest

from paper_2211_16718_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _constants():
    out = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as f:
        for line in f:
            line = line.split("#")[0].split()
            if line:
                out[line[0]] = float(line[1])
    return out


def test_paper_constants_are_the_defaults(oracle):
    c = _constants()
    P = oracle.Params(8, 8, 8)
    assert P.gamma == c["gamma"] and P.prandtl == c["prandtl"] and P.weno_eps == c["weno_eps"]
    assert I.GAMMA == c["gamma"]
    assert I.hit_mu_eff() == pytest.approx(c["hit_rho"] * c["hit_u0"] * (2 / c["hit_k0"]) / c["hit_re_lambda"])


def test_spectrum_integrals():
    """The model spectrum integrates to (3/2) u0^2 and gives the Taylor microscale
    lambda = sqrt(15 u0^2 / (2 int k^2 E)) = 2/k0 used for mu_eff = rho u0 lambda / Re_lambda."""
    from scipy.integrate import quad
    u0, k0 = 0.3, 4.0
    e_tot = quad(lambda k: I.hit_spectrum(k, u0, k0), 0, np.inf)[0]
    assert e_tot == pytest.approx(1.5 * u0 * u0, rel=1e-10)
    k2e = quad(lambda k: k * k * I.hit_spectrum(k, u0, k0), 0, np.inf)[0]
    lam = math.sqrt(15 * u0 * u0 / (2 * k2e))
    assert lam == pytest.approx(2 / k0, rel=1e-10)
    assert I.hit_mu_eff(u0, k0, 50.0) == pytest.approx(u0 * lam / 50.0, rel=1e-12)


@pytest.mark.parametrize("n", [16, 32])
def test_hit_velocity_solenoidal_with_model_shell_energies(n):
    u0, k0 = 0.3, 4.0
    u, v, w = I.hit_velocity(n, seed=3, u0=u0, k0=k0)
    assert (u * u + v * v + w * w).mean() / 3 == pytest.approx(u0 * u0, rel=1e-12)
    k = np.fft.fftfreq(n, d=1.0 / n)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    uh, vh, wh = (np.fft.fftn(a) for a in (u, v, w))
    div = KX * uh + KY * vh + KZ * wh
    assert np.abs(div).max() < 1e-10 * np.abs(uh).max()
    e_mode = 0.5 * (np.abs(uh) ** 2 + np.abs(vh) ** 2 + np.abs(wh) ** 2) / float(n) ** 6
    shell = np.rint(np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)).astype(int)
    e_shell = np.bincount(shell.ravel(), weights=e_mode.ravel())
    s = np.arange(1, n // 2)
    ratio = e_shell[s] / I.hit_spectrum(s, u0, k0)
    np.testing.assert_allclose(ratio, ratio[0], rtol=1e-9)  # shape of E(k) exactly, one global factor
    assert ratio[0] == pytest.approx(1.0, rel=0.05)
    assert e_shell[0] < 1e-25 and e_shell[n // 2:].sum() < 1e-25


def test_hit_is_seeded_and_uniform_thermo():
    a = I.isotropic_turbulence(16, seed=5)
    b = I.isotropic_turbulence(16, seed=5)
    c = I.isotropic_turbulence(16, seed=6)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.all(a[0] == 1.0)
    p = (I.GAMMA - 1) * (a[4] - 0.5 * (a[1] ** 2 + a[2] ** 2 + a[3] ** 2) / a[0])
    np.testing.assert_allclose(p, 1 / I.GAMMA, rtol=1e-14)


def test_taylor_green_is_divergence_free_and_isothermal():
    n = 16
    u = I.taylor_green(n)
    vel = u[1:4] / u[0]
    p = (I.GAMMA - 1) * (u[4] - 0.5 * (u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / u[0])
    np.testing.assert_allclose(I.GAMMA * p / u[0], 1.0, rtol=1e-14)
    k = np.fft.fftfreq(n, d=1.0 / n)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    div = KX * np.fft.fftn(vel[0]) + KY * np.fft.fftn(vel[1]) + KZ * np.fft.fftn(vel[2])
    assert np.abs(div).max() < 1e-10


def test_vortex_is_periodic_to_roundoff():
    """Core radius 1 in a box of 16: the field at the box edge differs from the
    free stream by less than 1e-13 (the periodic truncation is negligible)."""
    u = I.isentropic_vortex(64, 64, 1, length=16.0)
    edge = u[:, :, :, 0]
    free = I.uniform(1, 64, 1, rho=1.0, u=0.5, v=0.25)[:, :, :, 0]
    assert np.abs(edge - free).max() < 1e-13


def test_device_turbulence_is_the_spectral_interpolant_of_the_base_grid():
    """The n^3 field built on the device (here on the CPU) takes the base-grid field's values
    at the coincident points and keeps its RMS and zero divergence."""
    import numpy as np
    torch = pytest.importorskip("torch")
    from paper_2211_16718_gb300 import inputs as I
    u = I.isotropic_turbulence_device(48, seed=5, nbase=16, device="cpu").numpy()
    base = I.isotropic_turbulence(16, seed=5)
    assert np.abs(u[:, ::3, ::3, ::3] - base).max() <= 1e-14
    rms = np.sqrt((u[1] ** 2 + u[2] ** 2 + u[3] ** 2).mean() / 3)
    assert abs(rms - 0.3) <= 1e-14
    k = np.fft.fftfreq(48, d=1.0 / 48)
    div = sum(np.fft.ifftn(1j * k.reshape(sh) * np.fft.fftn(u[1 + c])).real
              for c, sh in enumerate([(1, 1, 48), (1, 48, 1), (48, 1, 1)]))
    assert np.abs(div).max() <= 1e-12


def test_turbulence_planes_equal_the_device_field():
    """The host-side planes generator gives the same planes as the device generator (run on
    the CPU here), including planes across the periodic wrap."""
    import numpy as np
    pytest.importorskip("torch")
    from paper_2211_16718_gb300 import inputs as I
    full = I.isotropic_turbulence_device(48, seed=5, nbase=16, device="cpu").numpy()
    planes = I.isotropic_turbulence_planes(48, seed=5, z0=44, count=9, nbase=16)
    zs = [(44 + j) % 48 for j in range(9)]
    assert np.abs(planes - full[:, zs]).max() <= 1e-14
