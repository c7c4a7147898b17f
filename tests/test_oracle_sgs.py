"""Pins of the oracle's SGS-PFP iteration (eqs. (20)-(29)), walls (eq. (31)), mass rescale
(eq. (32)) and outer residual, against closed forms and invariants.

- Equal wall temperatures: the uniform Maxwellian at the wall temperature is an exact
  fixed point (global equilibrium).
- Free-molecular limit (eps -> infinity): the steady state carries rho_L M_L on v1 > 0 and
  rho_R M_R on v1 < 0 in every cell, with zero net mass flux at the walls.
- PFP and FP solve the same cell equation (eq. (20)) to the same g.
- A converged solution has zero discrete mass flux through every face, and its moments
  do not depend on the inner method.
- The mass rescale restores the prescribed total mass; BGK mode has P = 0.
- Paper sanity (Section 4.1): PFP needs far fewer inner iterations than FP at small eps,
  and Newton for the discrete Maxwellian takes about five iterations.
"""
import numpy as np
import pytest

from paper_2409_01910_gb300 import inputs as I


def grid(N, L):
    v = (np.arange(N) - N // 2 + 1) * (2 * L / N)
    return v, np.stack(np.meshgrid(v, v, v, indexing="ij"), -1)


def fields(f, L):
    N = f.shape[-1]
    v, V = grid(N, L)
    w = (2 * L / N) ** 3
    rho = w * f.sum((1, 2, 3))
    U = w * np.einsum("jabc,abcd->jd", f, V) / rho[:, None]
    E = w * np.einsum("jabc,abc->j", f, (V**2).sum(-1))
    T = (E / rho - (U**2).sum(1)) / 3
    return rho, U, T


def test_equal_wall_temperature_fixed_point(oracle):
    N, L, J = 16, 8.0, 4
    M = I.sampled_maxwellian(N, L, 1.0, (0, 0, 0), 1.0)
    f = np.ascontiguousarray(np.repeat(M[None], J, 0))
    prob = oracle.Problem(N=N, L=L, J=J, eps=0.5, bc_T=(1.0, 1.0), total_mass=(2 * L / N) ** 3 * M.sum())
    f0 = f.copy()
    st = oracle.sgs_iteration(prob, f)
    assert abs(f - f0).max() <= 1e-13 * f0.max()
    assert st["inner_iters"] == 0


def test_free_molecular_limit(oracle):
    N, L, J = 8, 6.0, 4
    TL, TR = 1.0, 2.0
    prob = oracle.Problem(N=N, L=L, J=J, eps=1e12, bc_T=(TL, TR), total_mass=1.0)
    f = I.initial_state(J, N, L, T=1.5)
    for _ in range(3):
        oracle.sgs_iteration(prob, f)
    v, V = grid(N, L)
    ML = I.sampled_maxwellian(N, L, 1.0, (0, 0, 0), TL)
    MR = I.sampled_maxwellian(N, L, 1.0, (0, 0, 0), TR)
    pos, neg = V[..., 0] > 0, V[..., 0] < 0
    big_L = pos & (ML > 1e-3 * ML.max())
    big_R = neg & (MR > 1e-3 * MR.max())
    rho_L = np.mean(f[:, big_L] / ML[big_L])
    rho_R = np.mean(f[:, big_R] / MR[big_R])
    scale = f.max()
    assert abs(f[:, pos] - rho_L * ML[pos]).max() <= 1e-10 * scale
    assert abs(f[:, neg] - rho_R * MR[neg]).max() <= 1e-10 * scale
    # zero net mass flux at the walls: rho_L sum_{v1>0} v1 M_L = -rho_R sum_{v1<0} v1 M_R
    ratio = -(V[..., 0][neg] * MR[neg]).sum() / (V[..., 0][pos] * ML[pos]).sum()
    assert abs(rho_L / rho_R - ratio) <= 1e-10 * ratio


def _cell_problem(oracle, eps):
    N, L, J = 8, 6.0, 3
    prob = oracle.Problem(N=N, L=L, J=J, eps=eps, bc_T=(1.0, 2.0), inner_tol=1e-13, inner_max=5000)
    v, V = grid(N, L)
    rng = np.random.default_rng(7)
    f = np.stack([I.sampled_maxwellian(N, L, 1.0, (0.1 * j, 0, 0), 1.0 + 0.3 * j) for j in range(J)])
    f *= 1 + 0.05 * rng.uniform(-1, 1, f.shape)
    Q, P, nu = oracle.collide(prob, f)
    dx = prob.dx
    vp = np.maximum(V[..., 0], 0)
    vm = np.minimum(V[..., 0], 0)
    r = (-vp * f[0] + vm * f[2]) / dx - P[1] / eps
    return prob, dx, r, nu[1], f[1], V


@pytest.mark.parametrize("eps", [1.0, 0.01])
def test_pfp_and_fp_solve_the_same_cell_equation(oracle, eps):
    prob, dx, r, nu, g0, V = _cell_problem(oracle, eps)
    g_pfp, it_pfp, _ = oracle.cell_solve(prob, dx, r, nu, g0)
    prob.inner_method = oracle.FP
    g_fp, it_fp, _ = oracle.cell_solve(prob, dx, r, nu, g0)
    assert it_pfp < prob.inner_max and it_fp < prob.inner_max
    np.testing.assert_allclose(g_pfp, g_fp, rtol=0, atol=1e-11 * abs(g_fp).max())
    # the cell equation (eq. (20)) holds
    N, L = prob.N, prob.L
    th, _ = oracle.discrete_maxwellian(N, L, oracle.moments(g_pfp, L))
    M = oracle.eval_maxwellian(N, L, th)
    res = np.abs(V[..., 0]) / dx * g_pfp + r - nu / eps * (M - g_pfp)
    assert np.sqrt((2 * L / N) ** 3 * (res**2).sum()) < 1e-12
    if eps < 0.1:
        assert it_pfp < it_fp / 3  # the preconditioner pays off at small eps


def test_converged_solution_properties(oracle):
    """BGK mode (P = 0): SGS converges to round-off; the converged state has zero discrete
    mass flux through every face and the prescribed total mass."""
    N, L, J = 8, 6.0, 8
    prob = oracle.Problem(N=N, L=L, J=J, eps=1.0, bc_T=(1.0, 2.0), total_mass=1.0, inner_tol=1e-13,
                          kernel=oracle.BGK)
    f = I.initial_state(J, N, L, T=1.5)
    res = []
    for _ in range(40):
        oracle.sgs_iteration(prob, f)
        res.append(oracle.solve_residual(prob, f))
        if res[-1] < 1e-11:
            break
    assert res[-1] < 1e-11
    assert all(b < a for a, b in zip(res[:5], res[1:6]))
    dx = prob.dx
    v, V = grid(N, L)
    w = (2 * L / N) ** 3
    vp, vm = np.maximum(V[..., 0], 0), np.minimum(V[..., 0], 0)
    scale = w * (np.abs(V[..., 0]) * f[0]).sum()
    for j in range(J - 1):
        flux = w * (vp * f[j] + vm * f[j + 1]).sum()
        assert abs(flux) <= 1e-10 * scale, (j, flux)
    assert abs(dx * w * f.sum() - prob.total_mass) <= 1e-14


def test_outer_iterates_independent_of_inner_method(oracle):
    """With the cell equations solved exactly, SGS-FP and SGS-PFP produce the same outer
    iterates (Section 4.1 notes identical convergence plots)."""
    N, L, J = 8, 6.0, 6
    out = []
    for method in (oracle.PFP, oracle.FP):
        prob = oracle.Problem(N=N, L=L, J=J, eps=0.3, bc_T=(1.0, 2.0), total_mass=1.0, inner_tol=1e-13,
                              inner_max=5000, inner_method=method)
        f = I.initial_state(J, N, L, T=1.5)
        res = []
        for _ in range(6):
            oracle.sgs_iteration(prob, f)
            res.append(oracle.solve_residual(prob, f))
        out.append((f, res))
    (f1, r1), (f2, r2) = out
    assert all(b < a for a, b in zip(r1, r1[1:]))
    assert abs(f1 - f2).max() <= 1e-11 * f2.max()


def test_bgk_mode_has_no_penalty(oracle):
    N, L = 8, 6.0
    prob = oracle.Problem(N=N, L=L, J=2, kernel=oracle.BGK)
    f = I.initial_state(2, N, L, T=1.2)
    Q, P, nu = oracle.collide(prob, f)
    assert np.all(P == 0.0)
    for j in range(2):
        th, _ = oracle.discrete_maxwellian(N, L, oracle.moments(f[j], L))
        M = oracle.eval_maxwellian(N, L, th)
        np.testing.assert_allclose(Q[j], nu[j] * (M - f[j]), atol=1e-15)
        assert abs(nu[j] - oracle.moments(f[j], L)[0]) <= 1e-15  # 4 pi b0 rho with b0 = 1/(4 pi)


def test_paper_sanity_iteration_counts(oracle):
    N, L, J = 8, 6.0, 8
    counts = {}
    for method in (oracle.PFP, oracle.FP):
        prob = oracle.Problem(N=N, L=L, J=J, eps=1e-3, bc_T=(1.0, 2.0), inner_method=method, inner_max=2000)
        f = I.initial_state(J, N, L, T=1.5)
        st = {}
        for _ in range(2):
            s = oracle.sgs_iteration(prob, f)
            for k, v in s.items():
                st[k] = st.get(k, 0) + v
        counts[method] = st
    pfp, fp = counts[oracle.PFP], counts[oracle.FP]
    assert pfp["inner_iters"] / pfp["visits"] < 11
    assert fp["inner_iters"] / fp["visits"] > 5 * pfp["inner_iters"] / pfp["visits"]
    assert pfp["newton_iters"] / pfp["newton_solves"] < 8


def test_relaxed_step1_when_existence_fails(oracle):
    """A cell equation with a known solution g* (r = A M[g*] - (|v1|/dx + A) g*), started
    from two counter-moving beams at v1 = +-3 whose step-1 target violates eq. (26)
    (s0 < 0: the beams carry more |v1|-weighted mass than their Maxwellian). PFP with the
    fixed-point fallback, plain FP, and PFP with the relaxed step 1 of the remark after
    eq. (26) all reach g*; the relaxed form needs no fallback."""
    N, L, dx, eps, nu = 12, 6.0, 0.05, 1.0, 1.0
    A = nu / eps
    v = oracle.velocity_nodes(N, L)
    V = np.stack(np.meshgrid(v, v, v, indexing="ij"), -1)
    w = (2 * L / N) ** 3
    c = np.abs(V[..., 0]) / dx
    gstar = np.exp(-((V - [0.3, 0.0, 0.0]) ** 2).sum(-1) / 2.0) * (1.0 + 0.2 * np.cos(V[..., 1]))
    gstar /= w * gstar.sum()
    th, it = oracle.discrete_maxwellian(N, L, oracle.moments(gstar, L))
    assert it > 0
    r = A * oracle.eval_maxwellian(N, L, th) - (c + A) * gstar
    beam = lambda u: np.exp(-((V - [u, 0.0, 0.0]) ** 2).sum(-1) / (2 * 0.25))
    g0 = beam(3.0) + beam(-3.0)
    g0 /= w * g0.sum()
    th0, _ = oracle.discrete_maxwellian(N, L, oracle.moments(g0, L))
    M0 = oracle.eval_maxwellian(N, L, th0)
    e = w * (c * (M0 - g0) - r)
    s = [e.sum(), (e * V[..., 0]).sum(), (e * V[..., 1]).sum(), (e * V[..., 2]).sum(), (e * (V ** 2).sum(-1)).sum()]
    assert not (s[0] > 0 and s[0] * s[4] > s[1] ** 2 + s[2] ** 2 + s[3] ** 2)
    out = {}
    for method in (oracle.PFP, oracle.FP, oracle.PFP_RELAX):
        prob = oracle.Problem(N=N, L=L, eps=eps, inner_method=method, inner_tol=1e-12, inner_max=5000)
        g, its, st = oracle.cell_solve(prob, dx, r, nu, g0)
        assert np.abs(g - gstar).max() <= 1e-9 * gstar.max(), method
        out[method] = (its, st)
    assert out[oracle.PFP][1]["existence_fallbacks"] >= 1
    assert out[oracle.PFP_RELAX][1]["existence_fallbacks"] == 0
    assert out[oracle.PFP_RELAX][0] <= out[oracle.FP][0]
