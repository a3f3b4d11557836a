"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no lattice-Boltzmann arithmetic: it only draws numbers and
evaluates the analytic initial fields (density, velocity, phase profile) of
the synthetic workloads.  Turning them into moments is left to each side
(the library's ``llb_init_equilibrium`` on the GPU, ``oracle.lb.equilibrium_moments``
on the CPU), so neither side's arithmetic leaks into the other.

Arrays are float64, shaped (nz, ny, nx) for scalars and (3, nz, ny, nx)
for vectors, x fastest.  Random numbers come from numpy's PCG64 generator
seeded with the given seed, drawn in x-fastest order.
"""
from __future__ import annotations

import numpy as np


def _grid(nx: int, ny: int, nz: int):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def taylor_green_3d(nx: int, ny: int, nz: int, u0: float = 0.05, rho0: float = 1.0,
                    noise: float = 0.0, seed: int = 2301):
    """3D Taylor-Green vortex with optional uniform velocity noise.

    u = u0 sin(kx x) cos(ky y) cos(kz z), v = -u0 cos(kx x) sin(ky y) cos(kz z),
    w = 0, k_a = 2 pi / n_a, rho = rho0; plus U(-noise, noise) added to each
    velocity component when ``noise`` > 0.
    """
    x, y, z = _grid(nx, ny, nz)
    kx, ky, kz = 2 * np.pi / nx, 2 * np.pi / ny, 2 * np.pi / nz
    u = np.empty((3, nz, ny, nx), dtype=np.float64)
    u[0] = u0 * np.sin(kx * x) * np.cos(ky * y) * np.cos(kz * z)
    u[1] = -u0 * np.cos(kx * x) * np.sin(ky * y) * np.cos(kz * z)
    u[2] = 0.0
    if noise > 0.0:
        rng = np.random.default_rng(seed)
        u += rng.uniform(-noise, noise, size=u.shape)
    rho = np.full((nz, ny, nx), rho0, dtype=np.float64)
    return rho, u


def shear_wave_2d(nx: int, ny: int, nz: int, u0: float = 0.01, rho0: float = 1.0):
    """Two-dimensional Taylor-Green cell, uniform along z.

    u = u0 sin(k x) cos(k y), v = -u0 cos(k x) sin(k y), w = 0 with k = 2 pi / nx
    (requires nx == ny).  An exact incompressible Navier-Stokes solution whose
    velocity decays as exp(-2 nu k^2 t).
    """
    if nx != ny:
        raise ValueError("shear_wave_2d needs nx == ny")
    x, y, _ = _grid(nx, ny, nz)
    k = 2 * np.pi / nx
    u = np.zeros((3, nz, ny, nx), dtype=np.float64)
    u[0] = u0 * np.sin(k * x) * np.cos(k * y)
    u[1] = -u0 * np.cos(k * x) * np.sin(k * y)
    rho = np.full((nz, ny, nx), rho0, dtype=np.float64)
    return rho, u


def random_moments(nx: int, ny: int, nz: int, seed: int = 1, nfields: int = 10,
                   rho_spread: float = 0.05, j_amp: float = 0.03,
                   p_diag=(0.30, 0.37), p_off: float = 0.01):
    """Random moment field in canonical order, independent at every node.

    nfields=10: (rho, j_x, j_y, j_z, P_xx, P_yy, P_zz, P_xy, P_xz, P_yz).
    nfields=11: (rho1, rho2, j, P) with rho1 + rho2 spread like rho and
    rho1 / (rho1 + rho2) drawn from U(0, 1).
    rho ~ U(1 - rho_spread, 1 + rho_spread), j ~ U(-j_amp, j_amp),
    diagonal P ~ U(p_diag), off-diagonal P ~ U(-p_off, p_off).
    """
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    rho = rng.uniform(1.0 - rho_spread, 1.0 + rho_spread, size=shape)
    j = rng.uniform(-j_amp, j_amp, size=(3,) + shape)
    pd = rng.uniform(p_diag[0], p_diag[1], size=(3,) + shape)
    po = rng.uniform(-p_off, p_off, size=(3,) + shape)
    if nfields == 10:
        return np.concatenate([rho[None], j, pd, po]).astype(np.float64)
    if nfields == 11:
        frac = rng.uniform(0.0, 1.0, size=shape)
        return np.concatenate([(rho * frac)[None], (rho * (1.0 - frac))[None], j, pd, po]).astype(np.float64)
    raise ValueError("nfields must be 10 or 11")


def random_moments_device(nx: int, ny: int, nz: int, seed: int = 1, rho_spread: float = 0.05,
                          j_amp: float = 0.03, p_diag=(0.30, 0.37), p_off: float = 0.01):
    """The random_moments recipe (one component) drawn on the GPU with a seeded
    torch generator, as a float32 device tensor of shape (10, nz, ny, nx): for
    boxes whose inputs are too large to build on the host."""
    import torch

    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    m = torch.empty((10, nz, ny, nx), dtype=torch.float32, device="cuda")
    ranges = [(1.0 - rho_spread, 1.0 + rho_spread)] + [(-j_amp, j_amp)] * 3 + [tuple(p_diag)] * 3 + \
             [(-p_off, p_off)] * 3
    for f, (lo, hi) in enumerate(ranges):
        torch.rand(m[f].shape, generator=g, device="cuda", out=m[f])
        m[f].mul_(hi - lo).add_(lo)
    return m


def point_perturbation(nx: int, ny: int, nz: int, at=(0, 0, 0), delta: float = 0.1, rho0: float = 1.0):
    """Fluid at rest with rho = rho0 everywhere except rho0 + delta at node ``at`` = (x, y, z)."""
    rho = np.full((nz, ny, nx), rho0, dtype=np.float64)
    rho[at[2], at[1], at[0]] += delta
    return rho, np.zeros((3, nz, ny, nx), dtype=np.float64)


def droplets(nx: int, ny: int, nz: int, centres, radii, velocities, width: float = 2.0):
    """Droplets of fluid 1 in a matrix of fluid 2, with a tanh interface.

    Each droplet d contributes phi_d = tanh((R_d - r_d) / xi) with xi = width / 2
    and r_d the periodic (minimum-image) distance to its centre; phi = max_d phi_d
    (phi = +1 inside, -1 outside).  rho1 = (1 + phi) / 2, rho2 = (1 - phi) / 2
    (total density 1), u = sum_d u_d (1 + phi_d) / 2.
    Returns (rho1, rho2, u) with u of shape (3, nz, ny, nx).
    """
    x, y, z = _grid(nx, ny, nz)
    xi = width / 2.0
    phi = np.full((nz, ny, nx), -1.0)
    u = np.zeros((3, nz, ny, nx))
    for (cx, cy, cz), r0, vel in zip(centres, radii, velocities):
        dx = (x - cx + nx / 2) % nx - nx / 2
        dy = (y - cy + ny / 2) % ny - ny / 2
        dz = (z - cz + nz / 2) % nz - nz / 2
        r = np.sqrt(dx * dx + dy * dy + dz * dz)
        phid = np.tanh((r0 - r) / xi)
        phi = np.maximum(phi, phid)
        for a in range(3):
            u[a] += vel[a] * (1.0 + phid) / 2.0
    return (1.0 + phi) / 2.0, (1.0 - phi) / 2.0, u


def droplet_pair(nx: int, ny: int, nz: int, radius: float, speed: float, impact: float, width: float = 2.0):
    """Two equal droplets approaching along x: centres (Lx/2 -+ 2R, Ly/2 -+ b/2, Lz/2),
    velocities (+-speed, 0, 0), impact parameter b = ``impact``."""
    c1 = (nx / 2 - 2 * radius, ny / 2 - impact / 2, nz / 2)
    c2 = (nx / 2 + 2 * radius, ny / 2 + impact / 2, nz / 2)
    return droplets(nx, ny, nz, [c1, c2], [radius, radius], [(speed, 0.0, 0.0), (-speed, 0.0, 0.0)], width)
