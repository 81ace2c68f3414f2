"""Shared helpers of the test-suite (no method arithmetic)."""
import numpy as np


def rel_err(x, y) -> float:
    """Relative max-norm of the whole vector: ||x - y||_inf / ||y||_inf (all 5 variables)."""
    x = np.asarray(x)
    y = np.asarray(y)
    return float(np.abs(x - y).max() / np.abs(y).max())


def rel_err_var(x, y) -> float:
    """Per-variable normalised max-norm, max over the 5 conserved variables:
    ||x_v - y_v||_inf / max(||y_v||_inf, 1e-3 max_w ||y_w||_inf).  Stricter than rel_err for
    components that are small cancellation residues (e.g. the mass RHS of a solenoidal
    field), whose absolute rounding is ~eps |f| / dx."""
    x = np.asarray(x).reshape(5, -1)
    y = np.asarray(y).reshape(5, -1)
    scale = np.abs(y).max(axis=1)
    floor = 1e-3 * scale.max()
    return float((np.abs(x - y).max(axis=1) / np.maximum(scale, floor)).max())


def inc_rel_err(x, y, u0) -> float:
    """Relative max-norm error of the increment: ||(x - u0) - (y - u0)||_inf / ||y - u0||_inf."""
    x = np.asarray(x)
    y = np.asarray(y)
    d = y - np.asarray(u0)
    return float(np.abs(x - y).max() / np.abs(d).max())


def flux_scale(u, lengths, gamma: float = 1.4) -> float:
    """max over points, components and directions of |f_d(u)|, divided by the smallest grid
    spacing: the scale of the right-hand side that FP32 rounding of the interface fluxes acts on."""
    rho = u[0]
    vel = u[1:4] / rho
    p = (gamma - 1) * (u[4] - 0.5 * rho * (vel ** 2).sum(axis=0))
    fmax = 0.0
    for d in range(3):
        un = vel[d]
        comps = [u[1 + d], u[1] * un, u[2] * un, u[3] * un, (u[4] + p) * un]
        comps[1 + d] = comps[1 + d] + p
        fmax = max(fmax, max(float(np.abs(c).max()) for c in comps))
    nz, ny, nx = u.shape[1:]
    dx = min(lengths[0] / nx, lengths[1] / ny, lengths[2] / nz)
    return fmax / dx
