"""Pins of the oracle's nonlinear multigrid V-cycle (eq. (30)).

- The FAS correction vanishes at a converged fine solution: a V-cycle leaves it unchanged
  (the coarse right-hand side equals R_H(I f), whose solution is I f).
- In the stiff regime (eps = 0.01, BGK mode) V-cycles reduce the residual far faster than
  the same number of SGS iterations, the behaviour reported in Section 4.
"""
import numpy as np

from paper_2409_01910_gb300 import inputs as I


def test_vcycle_fixed_point_at_converged_solution(oracle):
    N, L, J = 8, 6.0, 8
    prob = oracle.Problem(N=N, L=L, J=J, eps=0.1, bc_T=(1.0, 2.0), total_mass=1.0, inner_tol=1e-13,
                          kernel=oracle.BGK)
    f = I.initial_state(J, N, L, T=1.5)
    for _ in range(60):
        oracle.sgs_iteration(prob, f)
        if oracle.solve_residual(prob, f) < 1e-12:
            break
    assert oracle.solve_residual(prob, f) < 1e-12
    g = f.copy()
    oracle.vcycle(prob, g, 3, 1, 1, 4)
    assert abs(g - f).max() <= 1e-11 * f.max()


def test_vcycle_accelerates_stiff_case(oracle):
    N, L, J = 8, 6.0, 16
    prob = oracle.Problem(N=N, L=L, J=J, eps=0.01, bc_T=(1.0, 2.0), total_mass=1.0, inner_tol=1e-12,
                          kernel=oracle.BGK)
    f = I.initial_state(J, N, L, T=1.5)
    g = f.copy()
    for _ in range(6):
        oracle.sgs_iteration(prob, f)
        oracle.vcycle(prob, g, 3, 1, 1, 4)
    assert oracle.solve_residual(prob, g) < 0.01 * oracle.solve_residual(prob, f)
