"""Seeded synthetic initial conditions for the structured-grid Euler solver.

This module is shared by the CPU oracle's tests, the GPU parity tests and the
benchmark.  It only builds input states: it holds no part of the finite-volume
method itself (no reconstruction, flux, residual, time step or update).  The
only arithmetic here converts primitive fields (rho, velocity, p) into the
conserved vector of Eq. (2), Q = (rho, rho*u, rho*v[, rho*w], rho*e_t), with
rho*e_t = p/(gamma-1) + rho*|u|^2/2 for an ideal gas.

Layout of every state: float64, C-contiguous, struct-of-arrays (the SoA layout
of Sec. 3.1), shape (nvar, ny, nx) in 2D (nvar = 4) and (nvar, nz, ny, nx) in
3D (nvar = 5); x varies fastest.  Cell centres sit at (i + 1/2) * dx.

Workloads (the paper's supersonic-inlet case of Sec. 3.2 has no published grid,
so these seeded states stand in for it):
  * isentropic vortex (strength 5, centre of [0,10]^2, free stream M = 0.5)
    plus uniform +-1e-3 density noise, periodic;
  * Kelvin-Helmholtz shear layer on [0,1]^2 (density 2/1, velocity +-0.5,
    8 random-phase transverse modes of total amplitude 0.01), periodic;
  * Taylor-Green vortex on [0,2pi]^3 at M = 0.1 with 1e-4 relative pressure
    noise, periodic;
  * Sod shock tube along x, and rotated 2D Sod problems with transmissive
    boundaries, for the batched workload (sizes log-uniform in [64, 2048]).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Sequence, Tuple

import numpy as np

GAMMA = 1.4

BC_PERIODIC = 0
BC_TRANSMISSIVE = 1


@dataclass(frozen=True)
class GridSpec:
    """A uniform Cartesian single-block grid.

    dim: 2 or 3.  n: cells per axis (nx, ny, nz); nz = 1 in 2D.
    length: domain extent per axis; spacing = length / n.
    bc: per axis (low side, high side), BC_PERIODIC or BC_TRANSMISSIVE.
    """

    dim: int
    n: Tuple[int, int, int]
    length: Tuple[float, float, float]
    bc: Tuple[Tuple[int, int], Tuple[int, int], Tuple[int, int]] = (
        (BC_PERIODIC, BC_PERIODIC), (BC_PERIODIC, BC_PERIODIC), (BC_PERIODIC, BC_PERIODIC))

    @property
    def nvar(self) -> int:
        return self.dim + 2

    @property
    def ncells(self) -> int:
        return self.n[0] * self.n[1] * (self.n[2] if self.dim == 3 else 1)

    @property
    def shape(self) -> Tuple[int, ...]:
        if self.dim == 2:
            return (self.nvar, self.n[1], self.n[0])
        return (self.nvar, self.n[2], self.n[1], self.n[0])

    @property
    def spacing(self) -> Tuple[float, float, float]:
        return tuple(self.length[d] / self.n[d] for d in range(3))


def grid2d(nx: int, ny: int, lx: float, ly: float, bc=BC_PERIODIC) -> GridSpec:
    bcs = bc if isinstance(bc, tuple) else ((bc, bc), (bc, bc), (BC_PERIODIC, BC_PERIODIC))
    return GridSpec(2, (nx, ny, 1), (lx, ly, 1.0), bcs)


def grid3d(nx: int, ny: int, nz: int, lx: float, ly: float, lz: float, bc=BC_PERIODIC) -> GridSpec:
    bcs = bc if isinstance(bc, tuple) else ((bc, bc), (bc, bc), (bc, bc))
    return GridSpec(3, (nx, ny, nz), (lx, ly, lz), bcs)


def conserved(rho, vel: Sequence[np.ndarray], p, gamma: float = GAMMA) -> np.ndarray:
    """Stack primitives into the conserved SoA vector of Eq. (2)."""
    rho = np.asarray(rho, dtype=np.float64)
    comps = [rho]
    ke = np.zeros_like(rho)
    for u in vel:
        u = np.broadcast_to(np.asarray(u, dtype=np.float64), rho.shape)
        comps.append(rho * u)
        ke = ke + u * u
    comps.append(np.broadcast_to(np.asarray(p, dtype=np.float64), rho.shape) / (gamma - 1.0) + 0.5 * rho * ke)
    return np.ascontiguousarray(np.stack(comps, axis=0))


def cell_centres(g: GridSpec):
    h = g.spacing
    return [(np.arange(g.n[d], dtype=np.float64) + 0.5) * h[d] for d in range(g.dim)]


# ----------------------------------------------------------------------------- 2D states

def isentropic_vortex(n: int = 128, beta: float = 5.0, mach: float = 0.5, noise: float = 1e-3,
                      seed: int = 0, t: float = 0.0, length: float = 10.0, gamma: float = GAMMA):
    """Shu's isentropic vortex on [0, L]^2 (L = 10), centre at the middle.

    Free stream rho = p = 1 moving along +x at u = mach * sqrt(gamma).  With
    noise > 0 the density gets an additive uniform perturbation
    noise * (2 xi - 1), xi ~ U[0, 1) from numpy default_rng(seed), holding
    u, v, p.  With t > 0 (and noise = 0) this is the exact solution at time t:
    the initial vortex translated by u_inf * t on the periodic domain.
    Returns (GridSpec, U).
    """
    g = grid2d(n, n, length, length)
    x, y = cell_centres(g)
    X, Y = np.meshgrid(x, y, indexing="xy")
    uinf = mach * np.sqrt(gamma)
    xc = 0.5 * length + uinf * t
    # periodic minimum-image distance to the (translated) centre
    dx = (X - xc + 0.5 * length) % length - 0.5 * length
    dy = Y - 0.5 * length
    r2 = dx * dx + dy * dy
    amp = beta / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    u = uinf - amp * dy
    v = amp * dx
    T = 1.0 - (gamma - 1.0) * beta * beta / (8.0 * gamma * np.pi * np.pi) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    if noise:
        xi = np.random.default_rng(seed).random(rho.shape)
        rho = rho + noise * (2.0 * xi - 1.0)
    return g, conserved(rho, (u, v), p, gamma)


def kelvin_helmholtz(n: int = 4096, seed: int = 1, amplitude: float = 0.01, modes: int = 8,
                     sigma: float = 0.05, gamma: float = GAMMA):
    """Kelvin-Helmholtz shear layer on the periodic unit square.

    rho = 2, u = +0.5 in the band |y - 1/2| < 1/4, else rho = 1, u = -0.5;
    p = 2.5.  Transverse velocity: (amplitude / modes) * sum_m sin(2 pi m x + phi_m)
    times two Gaussians (width sigma) centred on the shear lines y = 1/4, 3/4,
    phi_m ~ U[0, 2 pi) from default_rng(seed).
    """
    g = grid2d(n, n, 1.0, 1.0)
    x, y = cell_centres(g)
    phi = np.random.default_rng(seed).random(modes) * 2.0 * np.pi
    sx = np.zeros_like(x)
    for m in range(1, modes + 1):
        sx += np.sin(2.0 * np.pi * m * x + phi[m - 1])
    sx *= amplitude / modes
    gy = np.exp(-((y - 0.25) ** 2) / (2 * sigma * sigma)) + np.exp(-((y - 0.75) ** 2) / (2 * sigma * sigma))
    band = np.abs(y - 0.5) < 0.25
    rho = np.where(band, 2.0, 1.0)[:, None] * np.ones((1, n))
    u = np.where(band, 0.5, -0.5)[:, None] * np.ones((1, n))
    v = gy[:, None] * sx[None, :]
    return g, conserved(rho, (u, v), 2.5, gamma)


def sod_tube(nx: int, ny: int = 4, x0: float = 0.5, axis: int = 0, gamma: float = GAMMA,
             bc=BC_TRANSMISSIVE):
    """Sod's shock tube along x (axis 0) or y (axis 1) on the unit square.

    Left (rho, u, p) = (1, 0, 1), right (0.125, 0, 0.1), diaphragm at x0.
    """
    if axis == 0:
        g = grid2d(nx, ny, 1.0, 1.0, bc)
        x = cell_centres(g)[0][None, :] * np.ones((ny, 1))
    else:
        g = grid2d(ny, nx, 1.0, 1.0, bc)
        x = cell_centres(g)[1][:, None] * np.ones((1, ny))
    left = x < x0
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    return g, conserved(rho, (np.zeros_like(rho), np.zeros_like(rho)), p, gamma)


def sod_rotated(n: int, theta: float, gamma: float = GAMMA):
    """Sod problem on the unit square across the line through the centre with
    normal (cos theta, sin theta); transmissive boundaries on all sides."""
    g = grid2d(n, n, 1.0, 1.0, BC_TRANSMISSIVE)
    x, y = cell_centres(g)
    X, Y = np.meshgrid(x, y, indexing="xy")
    left = (X - 0.5) * np.cos(theta) + (Y - 0.5) * np.sin(theta) < 0.0
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    z = np.zeros_like(rho)
    return g, conserved(rho, (z, z), p, gamma)


def batched_sod(count: int = 96, seed: int = 3, nmin: int = 64, nmax: int = 2048):
    """Sizes and angles of the batched rotated-Sod workload.

    N_i = round(exp(U[ln nmin, ln nmax])) per problem (square grids),
    theta_i ~ U[0, 2 pi), both from default_rng(seed).
    Returns a list of (n, theta).
    """
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), count))).astype(int)
    angles = rng.uniform(0.0, 2.0 * np.pi, count)
    return [(int(s), float(a)) for s, a in zip(sizes, angles)]


def uniform_state(g: GridSpec, rho=1.0, vel=(0.3, -0.2, 0.1), p=0.9, gamma: float = GAMMA):
    """A uniform (free-stream) state on grid g."""
    shape = g.shape[1:]
    return conserved(np.full(shape, rho), tuple(np.full(shape, vel[d]) for d in range(g.dim)),
                     np.full(shape, p), gamma)


def random_smooth(g: GridSpec, seed: int = 0, amp: float = 0.2, gamma: float = GAMMA):
    """A positive, smooth-plus-noise state for parity and invariance tests:
    rho, p around 1 and velocities around (0.3, -0.2, 0.1) with a few random
    Fourier modes of relative size amp and 1e-3 white noise."""
    rng = np.random.default_rng(seed)
    cc = cell_centres(g)
    grids = np.meshgrid(*cc[::-1], indexing="ij")[::-1]  # x, y[, z] broadcast to (z,) y, x
    L = g.length

    def field(base, scale):
        f = np.full(g.shape[1:], base, dtype=np.float64)
        for _ in range(3):
            ph = rng.random() * 2 * np.pi
            k = rng.integers(1, 4, size=g.dim)
            arg = ph + sum(2 * np.pi * k[d] * grids[d] / L[d] for d in range(g.dim))
            f += scale * amp * np.sin(arg) / 3.0
        f += 1e-3 * scale * (2 * rng.random(f.shape) - 1)
        return f

    rho = field(1.0, 1.0)
    p = field(1.0, 1.0)
    vel = tuple(field(b, 1.0) for b in (0.3, -0.2, 0.1)[: g.dim])
    return conserved(rho, vel, p, gamma)


# ----------------------------------------------------------------------------- 3D states

def taylor_green(n: int = 384, mach: float = 0.1, noise: float = 1e-4, seed: int = 2,
                 gamma: float = GAMMA):
    """Taylor-Green vortex on the periodic cube [0, 2 pi]^3.

    rho = 1, V0 = 1, u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
    p = p0 + (cos 2x + cos 2y)(cos 2z + 2) / 16 with p0 = 1 / (gamma M^2);
    then p <- p (1 + noise (2 xi - 1)), xi ~ U[0, 1) from default_rng(seed).
    """
    L = 2.0 * np.pi
    g = grid3d(n, n, n, L, L, L)
    x, y, z = cell_centres(g)
    sx, cx = np.sin(x), np.cos(x)
    sy, cy = np.sin(y), np.cos(y)
    cz = np.cos(z)
    p0 = 1.0 / (gamma * mach * mach)
    nvar = 5
    U = np.empty((nvar, n, n, n), dtype=np.float64)
    rng = np.random.default_rng(seed)
    c2x, c2y, c2z = np.cos(2 * x), np.cos(2 * y), np.cos(2 * z)
    for k in range(n):  # plane by plane keeps the temporaries small
        u = (cy * cz[k])[:, None] * sx[None, :]      # (y, x)
        v = -(sy * cz[k])[:, None] * cx[None, :]
        p = p0 + (c2x[None, :] + c2y[:, None]) * (c2z[k] + 2.0) / 16.0
        if noise:
            p = p * (1.0 + noise * (2.0 * rng.random(p.shape) - 1.0))
        U[0, k] = 1.0
        U[1, k] = u
        U[2, k] = v
        U[3, k] = 0.0
        U[4, k] = p / (gamma - 1.0) + 0.5 * (u * u + v * v)
    return g, U
