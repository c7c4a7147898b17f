"""Pins of the oracle's nonlinear multigrid V-cycle (eq. (30)).

- The FAS correction vanishes at a converged fine solution: a V-cycle leaves it unchanged
  (the coarse right-hand side equals R_H(I f), whose solution is I f).
- In the stiff regime (eps = 0.01, BGK mode) V-cycles reduce the residual far faster than
  the same number of SGS iterations, the behaviour reported in Section 4.
"""
import numpy as np
import pytest

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



@pytest.mark.parametrize("coarse_iters", [1, 2])
def test_fas_coarse_right_hand_side_on_a_nonconverged_state(oracle, coarse_iters):
    """The coarse right-hand side of eq. (30) on a state far from convergence, binary
    collisions, diffuse walls: with no smoothing (pre = post = 0) a two-grid cycle changes f
    only by the prolonged correction f_H - I f, the same on both children of a pair. The
    coarse iterate f_H is then coarse_iters SGS iterations on R_H(.) = b_H from I f. Here b_H =
    R_H(I f) - I R_h(f) is formed with numpy from the oracle's residual fields (I the mean of
    the two children), the same coarse iterations are run on it, and the result must equal
    the cycle's coarse iterate. A dropped term, a wrong sign or a wrong restriction in the
    cycle's b_H changes the coarse iterate by O(|I R_h|)."""
    N, L, J = 8, 6.0, 8
    prob = oracle.Problem(N=N, L=L, J=J, eps=0.5, bc_T=(1.0, 1.8), total_mass=1.0, inner_fixed=12,
                          kernel=oracle.MAXWELL)
    rng = np.random.default_rng(17)
    f = I.initial_state(J, N, L, T=1.2, seed=3)
    f *= 1.0 + 0.2 * rng.uniform(-1.0, 1.0, (J, 1, 1, 1))  # cell densities far from the steady state
    g = f.copy()
    oracle.vcycle(prob, g, 2, 0, 0, coarse_iters)
    d = g - f
    scale = np.abs(f).max()
    assert np.abs(d[0::2] - d[1::2]).max() <= 1e-15 * scale  # injection: one correction per pair
    dxH = 2.0 * prob.dx

    def field(x, dx):
        Q, _, _ = oracle.collide(prob, x)
        return oracle.residual(prob, x, Q, dx=dx, return_field=True)[1]

    Rh = field(f, prob.dx)
    If = 0.5 * (f[0::2] + f[1::2])
    IRh = 0.5 * (Rh[0::2] + Rh[1::2])
    bH = field(If, dxH) - IRh
    w = (2 * L / N) ** 3
    assert np.sqrt(dxH * w * (IRh * IRh).sum()) > 1e-2  # far from converged
    fH = If.copy()
    for _ in range(coarse_iters):
        oracle.sgs_iteration(prob, fH, b=bH, rescale=False, dx=dxH)
    corr = fH - If
    assert np.abs(corr).max() > 1e-3 * scale  # the coarse correction is not negligible
    assert np.abs(0.5 * (d[0::2] + d[1::2]) - corr).max() <= 1e-12 * np.abs(corr).max()
    # the plausible mistakes are far outside that bound
    for wrong in (field(If, dxH) + IRh, -IRh, field(If, dxH) - 2.0 * IRh):
        fw = If.copy()
        for _ in range(coarse_iters):
            oracle.sgs_iteration(prob, fw, b=wrong, rescale=False, dx=dxH)
        assert np.abs((fw - If) - corr).max() > 1e-6 * np.abs(corr).max()
