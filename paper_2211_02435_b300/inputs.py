"""Seeded synthetic input fields (density and velocity) for the LBM step.

This module only draws initial flow fields; it holds none of the lattice
Boltzmann method's arithmetic.  The same arrays feed the CUDA path and the
CPU oracle.  All generators run on the host in float64 with numpy's PCG64.

Fields are returned as ``rho[Nz, Ny, Nx]`` and ``u[d, Nz, Ny, Nx]`` (x fastest),
with lattice coordinates x = 0..Nx-1 at the cell positions.
"""
from __future__ import annotations

import numpy as np


def _grid(dims):
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return nx, ny, nz, x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def taylor_green(dims, u0, nu=None, t=0.0, d=3):
    """Taylor-Green vortex of Eq. 5.1 at time t (z-invariant, u_z = 0).

    The wavenumber along each axis is 2 pi / N_axis (kappa = 2 pi / L on the
    square domains of the paper).  ``nu`` is only needed for t > 0.
    """
    nx, ny, nz, x, y, _ = _grid(dims)
    kx, ky = 2 * np.pi / nx, 2 * np.pi / ny
    a = 1.0
    b = 1.0
    if t:
        a = np.exp(-nu * (kx * kx + ky * ky) * t)
        b = np.exp(-2 * nu * (kx * kx + ky * ky) * t)
    u = np.zeros((d, nz, ny, nx))
    u[0] = u0 * np.cos(kx * x) * np.sin(ky * y) * a
    u[1] = -u0 * np.sin(kx * x) * np.cos(ky * y) * a
    rho = 1.0 - 0.75 * u0 * u0 * (np.cos(2 * kx * x) + np.cos(2 * ky * y)) * b
    return rho, u


def add_uniform_noise(u, amplitude, seed):
    """Add seeded uniform noise in [-amplitude, amplitude] to every velocity
    component, shifted to zero mean per component (returns a new array)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = u.copy()
    for c in range(u.shape[0]):
        n = rng.uniform(-amplitude, amplitude, size=u.shape[1:])
        out[c] += n - n.mean()
    return out


def fourier_modes(dims, n_modes=8, umax=0.08, kmax=4, seed=3):
    """Sum of ``n_modes`` divergence-free random-phase Fourier modes,
    u = sum_k a_k e_k cos(2 pi k.x / L + phi_k), k integer in [-kmax, kmax]^3
    without 0, e_k a random unit vector orthogonal to k, a_k ~ U[0.5, 1],
    rescaled so that max |u| = umax; rho = 1."""
    nx, ny, nz, x, y, z = _grid(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    u = np.zeros((3, nz, ny, nx))
    for _ in range(n_modes):
        while True:
            k = rng.integers(-kmax, kmax + 1, size=3)
            if np.any(k):
                break
        r = rng.standard_normal(3)
        e = r - k * (r @ k) / (k @ k)
        e /= np.linalg.norm(e)
        amp = rng.uniform(0.5, 1.0)
        phi = rng.uniform(0.0, 2 * np.pi)
        ph = 2 * np.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz) + phi
        c = np.cos(ph)
        for dd in range(3):
            u[dd] += amp * e[dd] * c
    u *= umax / np.sqrt((u * u).sum(0)).max()
    return np.ones((nz, ny, nx)), u


def random_deviations(q, ncells, scale, seed):
    """Seeded random zero-centered populations [q, ncells] (collision tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.standard_normal((q, ncells))


def shear_viscosity_rate(nu):
    """Shear relaxation rate for kinematic viscosity nu with c_s^2 = 1/3:
    nu = (1/omega - 1/2) / 3."""
    return 1.0 / (3.0 * nu + 0.5)


def batch_ensemble(n=4096, edges=(16, 24, 32, 48, 64, 96), nu_range=(1e-4, 1e-1),
                   u0_range=(0.01, 0.08), seed=4):
    """Parameters of an ensemble of cubic periodic Taylor-Green domains: edge
    lengths drawn uniformly from ``edges``, viscosity log-uniform in
    ``nu_range``, amplitude uniform in ``u0_range``.  Returns (dims[n][3],
    nu[n], u0[n])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    e = rng.choice(np.asarray(edges), size=n)
    lo, hi = np.log(nu_range[0]), np.log(nu_range[1])
    nu = np.exp(rng.uniform(lo, hi, size=n))
    u0 = rng.uniform(u0_range[0], u0_range[1], size=n)
    dims = np.stack([e, e, e], axis=1).astype(np.int64)
    return dims, nu, u0
