"""Pins of the oracle's macroscopic quantities: density, bulk velocity and temperature as
the moments define them (d = 3), and the heat flux q = 1/2 int (v - U)|v - U|^2 f dv of the
lid-driven cavity study (Section 4.2.2).

- A sampled Maxwellian with given (rho, U, T) returns them, with q = 0.
- A Grad-type distribution M (1 + 2 q.c (|c|^2 / (2T) - 5/2) / (5 rho T^2)), c = v - U,
  leaves rho, U and T unchanged and has heat flux exactly q (Gaussian moment identities
  int |c|^4 M = 15 rho T^2, int |c|^6 M = 105 rho T^3): a dropped 1/2, a sign, v in place of
  c or a wrong dimension in T fails it.
- A shift of the distribution by whole grid cells in velocity moves U by the shift and leaves
  T and q unchanged (Galilean invariance of the central moments)."""
import numpy as np
import pytest


def maxwellian(v, rho, U, T):
    c2 = (v[:, None, None] - U[0]) ** 2 + (v[None, :, None] - U[1]) ** 2 + (v[None, None, :] - U[2]) ** 2
    return rho / (2 * np.pi * T) ** 1.5 * np.exp(-c2 / (2 * T))


def grad_heat(v, rho, U, T, q):
    c = [v[:, None, None] - U[0], v[None, :, None] - U[1], v[None, None, :] - U[2]]
    c2 = c[0] ** 2 + c[1] ** 2 + c[2] ** 2
    qc = q[0] * c[0] + q[1] * c[1] + q[2] * c[2]
    return maxwellian(v, rho, U, T) * (1 + 2 * qc / (5 * rho * T * T) * (c2 / (2 * T) - 2.5))


@pytest.mark.parametrize("rho,U,T", [(1.0, (0.0, 0.0, 0.0), 1.0), (1.7, (0.3, -0.2, 0.1), 1.4),
                                     (0.6, (-0.5, 0.25, 0.0), 0.8)])
def test_maxwellian_moments_and_zero_heat_flux(oracle, rho, U, T):
    N, L = 32, 10.0
    v = oracle.velocity_nodes(N, L)
    out = oracle.macroscopic(maxwellian(v, rho, np.array(U), T), L)
    assert abs(out[0] - rho) <= 1e-12 * rho
    assert np.abs(out[1:4] - U).max() <= 1e-12
    assert abs(out[4] - T) <= 1e-12 * T
    assert np.abs(out[5:8]).max() <= 1e-12


@pytest.mark.parametrize("q", [(0.05, 0.0, 0.0), (0.02, -0.03, 0.01), (-0.04, 0.01, 0.03)])
def test_grad_distribution_has_its_heat_flux(oracle, q):
    N, L = 32, 10.0
    rho, U, T = 1.3, np.array([0.2, -0.1, 0.35]), 1.2
    v = oracle.velocity_nodes(N, L)
    out = oracle.macroscopic(grad_heat(v, rho, U, T, np.array(q)), L)
    assert abs(out[0] - rho) <= 1e-12 * rho
    assert np.abs(out[1:4] - U).max() <= 1e-12
    assert abs(out[4] - T) <= 1e-12 * T
    assert np.abs(out[5:8] - np.array(q)).max() <= 1e-12


def test_shift_by_grid_cells_moves_only_the_velocity(oracle):
    N, L = 32, 10.0
    dv = 2 * L / N
    v = oracle.velocity_nodes(N, L)
    f = grad_heat(v, 1.0, np.zeros(3), 0.7, np.array([0.03, -0.02, 0.01]))
    base = oracle.macroscopic(f, L)
    g = np.roll(f, (3, -2, 1), axis=(0, 1, 2))  # compact support: nothing wraps
    out = oracle.macroscopic(g, L)
    assert abs(out[0] - base[0]) <= 1e-13
    assert np.abs(out[1:4] - base[1:4] - dv * np.array([3, -2, 1])).max() <= 1e-12
    assert abs(out[4] - base[4]) <= 1e-12
    assert np.abs(out[5:8] - base[5:8]).max() <= 1e-12
