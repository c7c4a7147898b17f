"""Pins of the oracle's source iteration (eq. (SI), the collision term split by the BGK
penalty of eq. (28) and lagged):
- one iteration against a dense linear solve (numpy) of the same upwind transport with
  absorption, node by node, with P, nu, M and the wall ghosts of the previous iterate;
- a converged SGS steady state is a fixed point of the source iteration;
- at small eps the source iteration converges far more slowly than SGS (Section 3.1:
  amplification 1 - O(eps^2) against 1 - O(eps))."""
import numpy as np
import pytest

from paper_2409_01910_gb300 import inputs as I


@pytest.mark.parametrize("kernel", [0, 2])
def test_si_matches_dense_transport_solve(oracle, kernel):
    N, J, L, eps = 8, 6, 6.0, 0.3
    prob = oracle.Problem(N=N, L=L, J=J, eps=eps, kernel=kernel, bc_T=(1.0, 1.6), total_mass=1.0)
    f0 = I.initial_state(J, N, L, T=1.3, seed=21)
    dx = prob.dx
    v = oracle.velocity_nodes(N, L)
    P = np.empty_like(f0)
    M = np.empty_like(f0)
    nu = np.empty(J)
    for j in range(J):
        Qj, P[j], nu[j], th = oracle.collide_cell(prob, f0[j])
        M[j] = oracle.eval_maxwellian(N, L, th)
    gl, gr = oracle.ghost(prob, 0, f0[0]), oracle.ghost(prob, 1, f0[-1])
    expect = np.empty_like(f0)
    a = nu / eps
    for i1 in range(N):
        c = abs(v[i1]) / dx
        A = np.diag(c + a)
        for j in range(J):
            if v[i1] > 0 and j > 0:
                A[j, j - 1] = -c
            if v[i1] < 0 and j < J - 1:
                A[j, j + 1] = -c
        rhs = P[:, i1] / eps + a[:, None, None] * M[:, i1]
        if v[i1] > 0:
            rhs[0] += c * gl[i1]
        if v[i1] < 0:
            rhs[-1] += c * gr[i1]
        expect[:, i1] = np.linalg.solve(A, rhs.reshape(J, -1)).reshape(J, N, N)
    f = f0.copy()
    oracle.si_iteration(prob, f, rescale=False)
    assert np.abs(f - expect).max() <= 1e-13 * np.abs(expect).max()
    if kernel == 2:
        assert np.abs(P).max() == 0.0


def test_si_fixed_point_is_the_steady_state(oracle):
    """From a state whose outer residual is r, one source iteration moves f by O(r): the
    steady state of the discrete equations is its fixed point (a wrong source or ghost would
    move a converged state by the size of P)."""
    N, J, L = 8, 4, 6.0
    prob = oracle.Problem(N=N, L=L, J=J, eps=1.0, bc_T=(1.0, 1.5), total_mass=1.0, inner_tol=1e-12)
    f = I.initial_state(J, N, L, T=1.25, seed=22)
    g = f.copy()
    oracle.si_iteration(prob, g)
    d_init = np.abs(g - f).max() / np.abs(f).max()
    for _ in range(40):
        oracle.sgs_iteration(prob, f)
    res = oracle.solve_residual(prob, f)
    assert res < 1e-6, res
    g = f.copy()
    oracle.si_iteration(prob, g)
    d = np.abs(g - f).max() / np.abs(f).max()
    assert d <= 30 * res and d <= 1e-4 * d_init, (d, res, d_init)


def test_si_is_slow_at_small_eps(oracle):
    N, J, L = 8, 8, 6.0
    prob = oracle.Problem(N=N, L=L, J=J, eps=0.01, bc_T=(1.0, 1.5), total_mass=1.0, inner_tol=1e-12)
    f0 = I.initial_state(J, N, L, T=1.25, seed=23)
    f_si, f_sgs = f0.copy(), f0.copy()
    for _ in range(30):
        oracle.si_iteration(prob, f_si)
        oracle.sgs_iteration(prob, f_sgs)
    r_si, r_sgs = oracle.solve_residual(prob, f_si), oracle.solve_residual(prob, f_sgs)
    assert r_si > 4 * r_sgs, (r_si, r_sgs)
