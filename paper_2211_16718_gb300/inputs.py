"""Seeded synthetic initial conditions for the triply periodic compressible solver.

This module feeds both the CUDA path and the CPU oracle.  It holds no part of
the discretization (no reconstruction, upwinding, viscous operator or time
integration); it only turns the initial conditions named by arXiv 2211.16718
(Sec. 2.3, isotropic turbulence decay) and by the textbook test problems into
conserved-variable arrays ``u[5, nz, ny, nx]`` (rho, rho*u, rho*v, rho*w, e),
x fastest, on the grid x_i = i*dx, dx = L/N.

The conversion from primitive to conserved variables uses the definition of
the total energy per unit volume given with the governing equations
(Sec. 2.1): e = p/(gamma-1) + rho*(u^2+v^2+w^2)/2.

Nondimensionalisation: rho = 1, p = 1/gamma, so T = gamma*p/rho = 1 and the
sound speed is 1; velocities are Mach numbers.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4


def grid(n: int, length: float = 2.0 * math.pi) -> np.ndarray:
    """Grid point coordinates x_i = i*L/n, i = 0..n-1."""
    return np.arange(n, dtype=np.float64) * (length / n)


def to_conserved(rho, u, v, w, p, gamma: float = GAMMA) -> np.ndarray:
    """Stack primitive fields into the conserved state u[5, nz, ny, nx]."""
    rho = np.asarray(rho, dtype=np.float64)
    out = np.empty((5,) + rho.shape, dtype=np.float64)
    out[0] = rho
    out[1] = rho * u
    out[2] = rho * v
    out[3] = rho * w
    out[4] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return out


def _mesh(nx, ny, nz, lx, ly, lz):
    x, y, z = grid(nx, lx), grid(ny, ly), grid(nz, lz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def uniform(nx, ny, nz, rho=1.0, u=0.0, v=0.0, w=0.0, p=1.0 / GAMMA, gamma=GAMMA) -> np.ndarray:
    """Uniform (free-stream) state."""
    shp = (nz, ny, nx)
    f = lambda a: np.full(shp, a, dtype=np.float64)  # noqa: E731
    return to_conserved(f(rho), f(u), f(v), f(w), f(p), gamma)


def taylor_green(n: int, v0: float = 0.1, gamma: float = GAMMA, isothermal: bool = True,
                 ny: int | None = None, nz: int | None = None) -> np.ndarray:
    """Taylor-Green vortex on [0, 2pi)^3 with rho0 = 1, p0 = 1/gamma.

    u = V0 sin x cos y cos z, v = -V0 cos x sin y cos z, w = 0,
    p = p0 + V0^2/16 (cos 2x + cos 2y)(cos 2z + 2);
    isothermal: rho = gamma p (T = 1), else rho = 1.
    """
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    X, Y, Z = _mesh(n, ny, nz, 2 * math.pi, 2 * math.pi, 2 * math.pi)
    u = v0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -v0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    p = 1.0 / gamma + (v0 * v0 / 16.0) * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    rho = gamma * p if isothermal else np.ones_like(p)
    return to_conserved(rho, u, v, w, p, gamma)


def random_smooth(nx: int, ny: int, nz: int, seed: int, amp: float = 0.05, kmax: int = 3,
                  mach: float = 0.3, lx: float = 2 * math.pi, ly: float = 2 * math.pi,
                  lz: float = 2 * math.pi, gamma: float = GAMMA) -> np.ndarray:
    """Sum of a few random low-wavenumber Fourier modes per primitive field."""
    rng = np.random.default_rng(seed)
    X, Y, Z = _mesh(nx, ny, nz, lx, ly, lz)

    def field():
        f = np.zeros_like(X)
        for _ in range(6):
            k = rng.integers(-kmax, kmax + 1, size=3)
            a, ph = rng.normal(), rng.uniform(0, 2 * math.pi)
            f += a * np.sin(2 * math.pi * (k[0] * X / lx + k[1] * Y / ly + k[2] * Z / lz) + ph)
        return f / 6.0

    rho = 1.0 + amp * field()
    u, v, w = (mach * field() for _ in range(3))
    p = (1.0 + amp * field()) / gamma
    return to_conserved(rho, u, v, w, p, gamma)


def isentropic_vortex(nx: int, ny: int, nz: int, t: float = 0.0, length: float = 10.0,
                      strength: float = 1.0, radius: float = 1.0, u_inf: float = 0.5,
                      v_inf: float = 0.25, lz: float = 1.0, gamma: float = GAMMA) -> np.ndarray:
    """Isentropic vortex advected by (u_inf, v_inf), z-independent; exact Euler solution.

    Centre starts at (L/2, L/2) and moves to (L/2 + u_inf t, L/2 + v_inf t) (periodic).
    With r = distance/radius: perturbation velocity (strength/2pi) e^{(1-r^2)/2} (-dy, dx)/radius,
    theta = gamma p / rho = 1 - (gamma-1) strength^2/(8 pi^2) e^{1-r^2}, rho = theta^{1/(gamma-1)},
    p = rho theta / gamma (radial momentum balance of a steady isentropic vortex).
    """
    X, Y, _ = _mesh(nx, ny, nz, length, length, lz)
    xc = (0.5 * length + u_inf * t) % length
    yc = (0.5 * length + v_inf * t) % length
    dx = (X - xc + 0.5 * length) % length - 0.5 * length
    dy = (Y - yc + 0.5 * length) % length - 0.5 * length
    r2 = (dx * dx + dy * dy) / (radius * radius)
    g = (strength / (2 * math.pi)) * np.exp(0.5 * (1.0 - r2))
    u = u_inf - g * dy / radius
    v = v_inf + g * dx / radius
    w = np.zeros_like(u)
    theta = 1.0 - (gamma - 1.0) * strength ** 2 / (8.0 * math.pi ** 2) * np.exp(1.0 - r2)
    rho = theta ** (1.0 / (gamma - 1.0))
    p = rho * theta / gamma
    return to_conserved(rho, u, v, w, p, gamma)


def shock_tube(nx: int, ny: int, nz: int, axis: int = 0, gamma: float = GAMMA) -> np.ndarray:
    """Periodic Sod-type shock tube along `axis`: (rho, p) = (1, 1/gamma) on the first half
    and (0.125, 0.1/gamma) on the second, at rest (two discontinuities through the wrap)."""
    shp = (nz, ny, nx)
    n = shp[2 - axis]
    left = (np.arange(n) < n // 2)
    sl = [None, None, None]
    sl[2 - axis] = slice(None)
    mask = np.broadcast_to(left[tuple(sl)], shp)
    rho = np.where(mask, 1.0, 0.125)
    p = np.where(mask, 1.0 / gamma, 0.1 / gamma)
    zero = np.zeros(shp)
    return to_conserved(rho, zero, zero, zero, p, gamma)


# ---- decaying isotropic turbulence (Sec. 2.3) --------------------------------
def hit_spectrum(k, u0: float = 0.3, k0: float = 4.0):
    """Model spectrum E(k) = 16 sqrt(2/pi) u0^2/k0 (k/k0)^4 exp(-2 (k/k0)^2)."""
    k = np.asarray(k, dtype=np.float64)
    return 16.0 * math.sqrt(2.0 / math.pi) * u0 * u0 / k0 * (k / k0) ** 4 * np.exp(-2.0 * (k / k0) ** 2)


def hit_velocity(n: int, seed: int, u0: float = 0.3, k0: float = 4.0):
    """Solenoidal random velocity on [0,2pi)^3 whose shell energies follow E(k).

    Steps: Gaussian white noise per component (seeded) -> FFT (Hermitian by
    construction) -> projection P(k) = I - k k^T/|k|^2 -> every integer shell
    s = round(|k|), 1 <= s < n/2, rescaled to carry E(s) (Nyquist and k = 0 set
    to zero) -> inverse FFT -> one global factor so that <u_i u_i>/3 = u0^2.
    Returns (u, v, w) arrays of shape (n, n, n), indexed [z, y, x].
    """
    rng = np.random.default_rng(seed)
    half = n // 2
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kr = np.fft.rfftfreq(n, d=1.0 / n)
    KZ, KY, KX = np.meshgrid(k1, k1, kr, indexing="ij")
    kk = KX * KX + KY * KY + KZ * KZ
    uh = [np.fft.rfftn(rng.standard_normal((n, n, n))) for _ in range(3)]
    kdotu = KX * uh[0] + KY * uh[1] + KZ * uh[2]
    with np.errstate(invalid="ignore", divide="ignore"):
        inv = np.where(kk > 0, 1.0 / kk, 0.0)
    uh = [uh[0] - KX * kdotu * inv, uh[1] - KY * kdotu * inv, uh[2] - KZ * kdotu * inv]
    del kdotu
    nyq = (np.abs(KX) == half) | (np.abs(KY) == half) | (np.abs(KZ) == half)
    shell = np.rint(np.sqrt(kk)).astype(np.int64)
    keep = (~nyq) & (shell >= 1) & (shell < half)
    # rfft half-space: every kx in 1..n/2-1 stands for itself and its mirror
    mult = np.where((KX > 0) & (KX < half), 2.0, 1.0)
    e_mode = 0.5 * (np.abs(uh[0]) ** 2 + np.abs(uh[1]) ** 2 + np.abs(uh[2]) ** 2) / float(n) ** 6 * mult
    nsh = half
    e_shell = np.bincount(shell[keep].ravel(), weights=e_mode[keep].ravel(), minlength=nsh)
    target = hit_spectrum(np.arange(nsh, dtype=np.float64), u0, k0)
    with np.errstate(invalid="ignore", divide="ignore"):
        fac = np.where(e_shell > 0, np.sqrt(target / np.where(e_shell > 0, e_shell, 1.0)), 0.0)
    scale = np.where(keep, fac[np.minimum(shell, nsh - 1)], 0.0)
    vel = [np.fft.irfftn(c * scale, s=(n, n, n), axes=(0, 1, 2)) for c in uh]
    rms2 = (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2).mean() / 3.0
    g = u0 / math.sqrt(rms2)
    return vel[0] * g, vel[1] * g, vel[2] * g


def isotropic_turbulence(n: int, seed: int, u0: float = 0.3, k0: float = 4.0,
                         gamma: float = GAMMA) -> np.ndarray:
    """Decaying isotropic turbulence initial state: rho = 1, p = 1/gamma, hit_velocity."""
    u, v, w = hit_velocity(n, seed, u0, k0)
    rho = np.ones_like(u)
    p = np.full_like(u, 1.0 / gamma)
    return to_conserved(rho, u, v, w, p, gamma)


def hit_mu_eff(u0: float = 0.3, k0: float = 4.0, re_lambda: float = 50.0, rho: float = 1.0) -> float:
    """mu_eff = rho u0 lambda / Re_lambda with the Taylor microscale of E(k): lambda = 2/k0."""
    return rho * u0 * (2.0 / k0) / re_lambda


def isotropic_turbulence_device(n: int, seed: int, nbase: int = 64, u0: float = 0.3, k0: float = 4.0,
                                gamma: float = GAMMA, device: str = "cuda"):
    """The decaying-turbulence initial state on an n^3 grid built directly in device
    memory (a torch float64 tensor [5, n, n, n]), for grids whose host-side generation
    would take too long or too much host memory (1024^3: 43 GB per state).

    The velocity is hit_velocity(nbase, seed) interpolated spectrally to n^3: its
    Fourier coefficients (all shells below nbase/2, Nyquist zero) are zero-padded and
    inverse-transformed on the device, so the n^3 field is the same band-limited field
    sampled more finely.  The spectrum E(k) of Sec. 2.3 carries a fraction below
    exp(-2 (nbase/(2 k0))^2) (~1e-56 for nbase = 64, k0 = 4) of its energy beyond
    shell nbase/2, so this is the n^3 realisation up to that truncation.  The RMS
    normalisation of hit_velocity carries over exactly (Parseval on both grids).
    torch (FFT on the device) is used for input generation only."""
    import torch
    if n < nbase:
        raise ValueError("n must be >= nbase")
    vel = hit_velocity(nbase, seed, u0, k0)
    scale = (n / nbase) ** 3
    h = nbase // 2
    out = torch.empty((5, n, n, n), dtype=torch.float64, device=device)
    out[0].fill_(1.0)
    for c in range(3):
        small = torch.fft.rfftn(torch.from_numpy(np.ascontiguousarray(vel[c])).to(device))  # [nb, nb, nb/2+1]
        big = torch.zeros((n, n, n // 2 + 1), dtype=torch.complex128, device=device)
        # fftfreq order: indices 0..h-1 are k = 0..h-1, h..nb-1 are k = -h..-1 (k = -h is Nyquist, zero)
        for zs, zd in ((slice(0, h), slice(0, h)), (slice(h, nbase), slice(n - h, n))):
            for ys, yd in ((slice(0, h), slice(0, h)), (slice(h, nbase), slice(n - h, n))):
                big[zd, yd, : h + 1] = small[zs, ys, : h + 1] * scale
        del small
        out[1 + c] = torch.fft.irfftn(big, s=(n, n, n))
        del big
    p = 1.0 / gamma
    out[4] = p / (gamma - 1.0) + 0.5 * (out[1] * out[1] + out[2] * out[2] + out[3] * out[3])
    return out


def isotropic_turbulence_planes(n: int, seed: int, z0: int, count: int, nbase: int = 64, u0: float = 0.3,
                                k0: float = 4.0, gamma: float = GAMMA) -> np.ndarray:
    """The z-planes z0, z0 + 1, ..., z0 + count - 1 (periodic) of the state that
    isotropic_turbulence_device(n, seed, nbase) builds, computed on the host without the
    whole n^3 field: the band-limited velocity is summed over its base-grid wavenumbers
    along z at the requested planes only, then inverse-transformed in x and y plane by
    plane.  Equal to the device field up to rounding.  Returns u[5, count, n, n]."""
    if n < nbase:
        raise ValueError("n must be >= nbase")
    vel = hit_velocity(nbase, seed, u0, k0)
    h = nbase // 2
    zs = (z0 + np.arange(count)) % n
    kz = np.fft.fftfreq(nbase, d=1.0 / nbase)
    E = np.exp(2j * math.pi * np.outer(zs, kz) / n)  # [count, nbase]
    out = np.empty((5, count, n, n), dtype=np.float64)
    out[0] = 1.0
    for c in range(3):
        small = np.fft.rfftn(vel[c])  # [nbase (kz), nbase (ky), h + 1 (kx)]
        a = np.tensordot(E, small, axes=(1, 0))  # [count, nbase (ky), h + 1]
        big = np.zeros((count, n, n // 2 + 1), dtype=np.complex128)
        big[:, :h, : h + 1] = a[:, :h]
        big[:, n - h:, : h + 1] = a[:, h:]
        out[1 + c] = np.fft.irfft2(big, s=(n, n), axes=(1, 2)) * (float(n) ** 2 / float(nbase) ** 3)
    p = 1.0 / gamma
    out[4] = p / (gamma - 1.0) + 0.5 * (out[1] * out[1] + out[2] * out[2] + out[3] * out[3])
    return out
