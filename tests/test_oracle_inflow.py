"""Pins of inflow boundaries (the normal-shock workload) in the oracle.

- The Rankine-Hugoniot inflow data conserve the Euler fluxes of mass, momentum and energy
  across the shock (closed form of the jump conditions for gamma = 5/3).
- Free-molecular limit with inflow on both sides: one SGS iteration carries the left
  Maxwellian on v1 > 0 and the right one on v1 < 0 through every cell (exact upwind
  propagation, no wall-density coupling).
- A converged steady state with inflow data has the same discrete mass flux through every
  face (the collision operator conserves mass exactly).
"""
import numpy as np
import pytest

from paper_2409_01910_gb300 import inputs as I


def grid(N, L):
    v = (np.arange(N) - N // 2 + 1) * (2 * L / N)
    return v, np.stack(np.meshgrid(v, v, v, indexing="ij"), -1)


def test_rankine_hugoniot_conserves_euler_fluxes():
    for mach in (1.2, 2.0, 3.0):
        (r1, u1, T1), (r2, u2, T2) = I.rankine_hugoniot(mach)
        flux = lambda r, u, T: (r * u, r * u * u + r * T, u * (0.5 * r * u * u + 1.5 * r * T + r * T))
        a, b = flux(r1, u1, T1), flux(r2, u2, T2)
        assert np.allclose(a, b, rtol=1e-13, atol=0), (mach, a, b)
        assert u1 / np.sqrt(5.0 / 3.0 * T1) == pytest.approx(mach, rel=1e-14)
        assert u2 < np.sqrt(5.0 / 3.0 * T2)  # subsonic downstream
    (r1, u1, T1), (r2, u2, T2) = I.rankine_hugoniot(2.0)
    assert (r2, u2, T2) == pytest.approx((16.0 / 7.0, 7.0 * u1 / 16.0, 133.0 / 64.0), rel=1e-14)


def inflow_problem(oracle, N, L, J, eps, up, down, **kw):
    return oracle.Problem(N=N, L=L, J=J, eps=eps, x_lo=-4.0, x_hi=4.0, kernel=oracle.HARD_SPHERE,
                          bc_kind=(oracle.INFLOW, oracle.INFLOW), bc_rho=(up[0], down[0]),
                          bc_u=((up[1], 0.0, 0.0), (down[1], 0.0, 0.0)), bc_T=(up[2], down[2]), total_mass=0.0,
                          **kw)


def test_free_molecular_inflow_is_upwind_transport(oracle):
    N, L, J = 8, 8.0, 5
    up, down = I.rankine_hugoniot(2.0)
    prob = inflow_problem(oracle, N, L, J, 1e12, up, down)
    f = I.initial_state(J, N, L, T=1.5, seed=2)
    oracle.sgs_iteration(prob, f)
    v, V = grid(N, L)
    M1 = I.sampled_maxwellian(N, L, up[0], (up[1], 0, 0), up[2])
    M2 = I.sampled_maxwellian(N, L, down[0], (down[1], 0, 0), down[2])
    pos, neg = V[..., 0] > 0, V[..., 0] < 0
    scale = max(M1.max(), M2.max())
    assert abs(f[:, pos] - M1[pos]).max() <= 1e-10 * scale
    assert abs(f[:, neg] - M2[neg]).max() <= 1e-10 * scale


def test_converged_inflow_problem_has_constant_face_mass_flux(oracle):
    """BGK collisions (which conserve mass exactly and converge in a few SGS iterations) with
    different inflow states on the two sides: the converged discrete mass flux is the same
    through every face, including the two boundary faces fed by the inflow halves."""
    N, L, J = 8, 6.0, 6
    a, b = (1.0, 0.3, 1.0), (1.1, 0.3, 1.2)
    prob = oracle.Problem(N=N, L=L, J=J, eps=0.5, kernel=oracle.BGK, bc_kind=(oracle.INFLOW, oracle.INFLOW),
                          bc_rho=(a[0], b[0]), bc_u=((a[1], 0.0, 0.0), (b[1], 0.0, 0.0)), bc_T=(a[2], b[2]),
                          total_mass=0.0, inner_tol=1e-13)
    f = I.initial_state(J, N, L, T=1.1, seed=1)
    res = 1.0
    for it in range(60):
        oracle.sgs_iteration(prob, f)
        res = oracle.solve_residual(prob, f)
        if res < 1e-12:
            break
    assert res < 1e-12, res
    v, V = grid(N, L)
    wt = (2 * L / N) ** 3
    v1 = V[..., 0]
    Ma = I.sampled_maxwellian(N, L, a[0], (a[1], 0, 0), a[2])
    Mb = I.sampled_maxwellian(N, L, b[0], (b[1], 0, 0), b[2])
    cells = np.concatenate([np.where(v1 > 0, Ma, 0.0)[None], f, np.where(v1 < 0, Mb, 0.0)[None]])
    flux = [wt * (np.maximum(v1, 0) * cells[j] + np.minimum(v1, 0) * cells[j + 1]).sum() for j in range(J + 1)]
    assert np.ptp(flux) <= 1e-10 * abs(np.mean(flux)), flux
