"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds no step of the solver: it only draws the initial distributions and
wall data of the workloads below from numpy's seeded generator. Both the CUDA path and
the oracle receive the identical arrays.

Initial state: the continuum Maxwellian rho/(2 pi T)^{3/2} exp(-|v|^2/(2T)) sampled at
the velocity nodes v = (i - N/2 + 1) 2L/N, multiplied by (1 + a U[-1, 1]) per (cell, node),
with rho = 1, zero velocity and amplitude a = 1e-3.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MAXWELL_B0 = 1.0 / (4.0 * np.pi)


def _nodes(N: int, L: float) -> np.ndarray:
    return (np.arange(N) - N // 2 + 1) * (2.0 * L / N)


def sampled_maxwellian(N: int, L: float, rho: float = 1.0, u=(0.0, 0.0, 0.0), T: float = 1.0) -> np.ndarray:
    """Continuum Maxwellian sampled at the velocity nodes, shape (N, N, N)."""
    v = _nodes(N, L)
    d1 = (v - u[0])[:, None, None]
    d2 = (v - u[1])[None, :, None]
    d3 = (v - u[2])[None, None, :]
    return rho / (2.0 * np.pi * T) ** 1.5 * np.exp(-(d1 * d1 + d2 * d2 + d3 * d3) / (2.0 * T))


def initial_state(J: int, N: int, L: float, T: float = 1.5, rho: float = 1.0, noise: float = 1e-3,
                  seed: int = 0) -> np.ndarray:
    """f0[j] = M(rho, 0, T) (1 + noise U[-1, 1]), shape (J, N, N, N), float64."""
    rng = np.random.default_rng(seed)
    M = sampled_maxwellian(N, L, rho, (0.0, 0.0, 0.0), T)
    u = rng.uniform(-1.0, 1.0, size=(J, N, N, N))
    return np.ascontiguousarray(M[None] * (1.0 + noise * u))


@dataclass
class Workload:
    """A 1-D planar heat-transfer problem between diffuse walls."""

    name: str
    J: int
    N: int
    L: float
    eps: float
    T_left: float
    T_right: float
    x_lo: float = 0.0
    x_hi: float = 1.0
    b0: float = MAXWELL_B0
    T_init: float = 1.5
    seed: int = 0
    iterations: int = 0        # fixed SGS iteration count (0: run to tolerance)
    tol: float = 1e-8
    precision: str = "fp64"

    @property
    def total_mass(self) -> float:
        # noise-free initial density 1 times the domain length
        return 1.0 * (self.x_hi - self.x_lo)

    def initial_state(self) -> np.ndarray:
        return initial_state(self.J, self.N, self.L, T=self.T_init, seed=self.seed)


def heat_16cells_16v() -> Workload:
    """16 cells on [0, 1], 16^3 velocities on [-6, 6]^3, eps = 1, walls T = 1 and 2, 20 SGS iterations."""
    return Workload("heat1d_J16_N16_eps1", J=16, N=16, L=6.0, eps=1.0, T_left=1.0, T_right=2.0, T_init=1.5,
                    iterations=20)


def heat_64cells_32v(seed: int = 0) -> Workload:
    """64 cells on [0, 1], 32^3 velocities on [-8, 8]^3, eps = 0.01, seeded wall temperatures
    T_L ~ U[0.8, 1.2], T_R ~ U[1.5, 2.5]; initial temperature (T_L + T_R)/2; to residual 1e-8."""
    rng = np.random.default_rng(seed)
    TL = float(rng.uniform(0.8, 1.2))
    TR = float(rng.uniform(1.5, 2.5))
    return Workload("heat1d_J64_N32_eps0.01", J=64, N=32, L=8.0, eps=0.01, T_left=TL, T_right=TR,
                    T_init=0.5 * (TL + TR), seed=seed, tol=1e-8)


def heat_batch(n: int = 64, seed: int = 0, J_range=(32, 256), N_choices=(24, 32), eps_range=(1e-3, 1.0),
               L: float = 8.0) -> list:
    """Independent heat-transfer instances of a batch: cells uniform in J_range (inclusive),
    velocity grid drawn from N_choices, eps log-uniform in eps_range, wall temperatures
    T_L ~ U[0.8, 1.2], T_R ~ U[1.5, 2.5], box [-L, L]^3; each instance's initial state has its
    own seed (seed * 1000 + index)."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n):
        J = int(rng.integers(J_range[0], J_range[1] + 1))
        N = int(N_choices[int(rng.integers(0, len(N_choices)))])
        eps = float(np.exp(rng.uniform(np.log(eps_range[0]), np.log(eps_range[1]))))
        TL = float(rng.uniform(0.8, 1.2))
        TR = float(rng.uniform(1.5, 2.5))
        out.append(Workload(f"heat1d_batch{q}_J{J}_N{N}", J=J, N=N, L=L, eps=eps, T_left=TL, T_right=TR,
                            T_init=0.5 * (TL + TR), seed=seed * 1000 + q, tol=1e-8))
    return out


def rankine_hugoniot(mach: float = 2.0, rho1: float = 1.0, T1: float = 1.0, gamma: float = 5.0 / 3.0):
    """Upstream and downstream states (rho, u, T) of a stationary normal shock of a
    monatomic gas (the Maxwellian exp(-|v-u|^2 / (2T)) has sound speed sqrt(gamma T))."""
    u1 = mach * np.sqrt(gamma * T1)
    m2 = mach * mach
    r = (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    t = (2.0 * gamma * m2 - (gamma - 1.0)) * ((gamma - 1.0) * m2 + 2.0) / ((gamma + 1.0) ** 2 * m2)
    return (rho1, u1, T1), (rho1 * r, u1 / r, T1 * t)


@dataclass
class ShockWorkload:
    """1-D stationary normal shock between Rankine-Hugoniot inflow Maxwellians."""

    name: str
    J: int
    N: int
    L: float
    eps: float
    up: tuple
    down: tuple
    x_lo: float = -20.0
    x_hi: float = 20.0
    width: float = 1.0
    tol: float = 1e-8

    def initial_state(self) -> np.ndarray:
        """Maxwellians of a tanh profile centred at x = 0: density and temperature blend the
        two states, the velocity keeps the mass flux rho u of the upstream state."""
        (r1, u1, T1), (r2, u2, T2) = self.up, self.down
        dx = (self.x_hi - self.x_lo) / self.J
        out = np.empty((self.J, self.N, self.N, self.N))
        for j in range(self.J):
            x = self.x_lo + (j + 0.5) * dx
            s = 0.5 * (1.0 + np.tanh(x / self.width))
            rho = r1 + (r2 - r1) * s
            T = T1 + (T2 - T1) * s
            out[j] = sampled_maxwellian(self.N, self.L, rho, (r1 * u1 / rho, 0.0, 0.0), T)
        return out


def shock_128cells_32v(mach: float = 2.0) -> ShockWorkload:
    """Mach-2 normal shock: 128 cells on [-20, 20], 32^3 velocities on [-10, 10]^3, hard
    spheres, eps = 0.1, Rankine-Hugoniot inflow data on both sides."""
    up, down = rankine_hugoniot(mach)
    return ShockWorkload(f"shock1d_M{mach:g}_J128_N32_eps0.1", J=128, N=32, L=10.0, eps=0.1, up=up, down=down)


@dataclass
class CavityWorkload:
    """2-D lid-driven cavity on [0, 1]^2: diffuse walls at temperature T_wall, the top wall
    (y = 1) moving with speed lid along x; initial state the Maxwellian M(1, 0, T_wall)
    sampled at the nodes in every cell."""

    name: str
    nx: int
    ny: int
    N: int
    L: float
    eps: float
    lid: float = 0.5
    T_wall: float = 1.0
    tol: float = 1e-8

    @property
    def J(self) -> int:
        return self.nx * self.ny

    @property
    def total_mass(self) -> float:
        return 1.0  # density 1 on the unit square

    def initial_state(self) -> np.ndarray:
        M = sampled_maxwellian(self.N, self.L, 1.0, (0.0, 0.0, 0.0), self.T_wall)
        return np.ascontiguousarray(np.repeat(M[None], self.J, 0))


def cavity_64x64_24v() -> CavityWorkload:
    """64 x 64 cells, 24^3 velocities on [-6, 6]^3, Maxwell molecules, eps = 0.05, lid speed
    0.5, walls at T = 1."""
    return CavityWorkload("cavity2d_64x64_N24_eps0.05", nx=64, ny=64, N=24, L=6.0, eps=0.05)


@dataclass
class CavityHeatWorkload:
    """2-D heat transfer in a cavity with the BGK operator: the square (-1/2, 1/2)^2, all
    walls at rest, the top wall (y = 1/2) at temperature T_top and the others at T_wall,
    penalty frequency nu = 4 pi rho (b0 = 1), initial state M(1, 0, T_wall) in every cell."""

    name: str
    nx: int
    ny: int
    N: int
    L: float
    eps: float
    T_wall: float = 1.0
    T_top: float = 2.0
    b0: float = 1.0
    tol: float = 1e-5

    @property
    def J(self) -> int:
        return self.nx * self.ny

    @property
    def total_mass(self) -> float:
        return 1.0  # density 1 on the unit square

    def initial_state(self) -> np.ndarray:
        M = sampled_maxwellian(self.N, self.L, 1.0, (0.0, 0.0, 0.0), self.T_wall)
        return np.ascontiguousarray(np.repeat(M[None], self.J, 0))


def cavity_heat_bgk_40x40_20v(eps: float) -> CavityHeatWorkload:
    """The BGK heat-transfer cavity of the paper's 2-D BGK example: 40 x 40 cells, 20^3
    velocities on [-6, 6]^3, top wall at T = 2, the other walls at T = 1."""
    return CavityHeatWorkload(f"cavity2d_heat_bgk_40x40_N20_eps{eps:g}", nx=40, ny=40, N=20, L=6.0, eps=eps)
