"""Pins of the oracle's conservation projection of Q (an option, not in the paper).

The projection q -> q_c is fixed by two properties that together determine it uniquely
(q = q_c + d is the orthogonal split of q along span(phi) and its complement):
  (i)  sum_k phi_i(v_k) q_c,k = 0 for phi = (1, v1, v2, v3, |v|^2);
  (ii) d = q - q_c lies in span(phi), checked by a least-squares fit with numpy.
Both are checked on random inputs and on Q of a non-equilibrium distribution, whose
momentum and energy moments the spectral method leaves nonzero. The projected operator
keeps Q[M] = 0 and the penalty split P = Q - nu (M - f).
"""
import numpy as np
import pytest


def basis(N, L):
    v = (np.arange(N) - N // 2 + 1) * (2 * L / N)
    V = np.stack(np.meshgrid(v, v, v, indexing="ij"), -1).reshape(-1, 3)
    return np.column_stack([np.ones(len(V)), V, (V**2).sum(-1)])  # K x 5


def check_projection(q, qc, Phi, tol=1e-13):
    scale = (np.abs(Phi) * np.abs(q.reshape(-1, 1))).sum(0)
    mom = Phi.T @ qc.reshape(-1)
    assert np.all(np.abs(mom) <= tol * scale), (mom, scale)
    d = (q - qc).reshape(-1)
    coef, *_ = np.linalg.lstsq(Phi, d, rcond=None)
    assert np.abs(Phi @ coef - d).max() <= tol * max(np.abs(d).max(), np.abs(q).max())


@pytest.mark.parametrize("N,L,seed", [(8, 6.0, 0), (12, 8.0, 1), (16, 10.0, 2)])
def test_projection_of_random_vectors(oracle, N, L, seed):
    q = np.random.default_rng(seed).standard_normal((N, N, N))
    qc = oracle.conserve_project(q, L)
    check_projection(q, qc, basis(N, L))
    # a projection: applying it twice changes nothing
    assert np.abs(oracle.conserve_project(qc, L) - qc).max() <= 1e-13 * np.abs(q).max()


def test_projection_leaves_zero_moment_vectors(oracle):
    N, L = 8, 6.0
    Phi = basis(N, L)
    q = np.random.default_rng(5).standard_normal(N**3)
    q -= Phi @ np.linalg.lstsq(Phi, q, rcond=None)[0]  # remove the span by numpy's solver
    qc = oracle.conserve_project(q.reshape(N, N, N), L)
    assert np.abs(qc.reshape(-1) - q).max() <= 1e-13 * np.abs(q).max()


def bimodal(N, L):
    v = (np.arange(N) - N // 2 + 1) * (2 * L / N)
    V = np.stack(np.meshgrid(v, v, v, indexing="ij"), -1)
    return np.exp(-((V - [1.2, 0, 0]) ** 2).sum(-1) / 1.0) + 0.8 * np.exp(-((V + [0.5, 0.3, 0]) ** 2).sum(-1) / 2.5)


@pytest.mark.parametrize("kernel", [0, 1])
def test_projected_collision_conserves(oracle, kernel):
    N, L = 16, 8.0
    f = bimodal(N, L)
    plain = oracle.Problem(N=N, L=L, kernel=kernel)
    proj = oracle.Problem(N=N, L=L, kernel=kernel, conserve_proj=1)
    Q0, P0, nu0, _ = oracle.collide_cell(plain, f)
    Q1, P1, nu1, _ = oracle.collide_cell(proj, f)
    Phi = basis(N, L)
    scale = (np.abs(Phi) * np.abs(Q0.reshape(-1, 1))).sum(0)
    # the paper's operator leaves a momentum or energy moment at spectral-accuracy level
    assert np.max(np.abs(Phi.T @ Q0.reshape(-1))[1:] / scale[1:]) > 1e-12
    check_projection(Q0, Q1, Phi)
    assert nu0 == nu1
    # P = Q - nu (M - f) with the same M: the two P differ by exactly the Q correction
    assert np.abs((P1 - P0) - (Q1 - Q0)).max() <= 1e-14 * np.abs(Q0).max()


def test_projected_collision_of_maxwellian_vanishes(oracle):
    N, L = 16, 6.0
    v = (np.arange(N) - N // 2 + 1) * (2 * L / N)
    V = np.stack(np.meshgrid(v, v, v, indexing="ij"), -1)
    M = 0.9 / (2 * np.pi * 1.3) ** 1.5 * np.exp(-((V - [0.4, -0.1, 0.2]) ** 2).sum(-1) / (2 * 1.3))
    Q, P, nu, _ = oracle.collide_cell(oracle.Problem(N=N, L=L, conserve_proj=1), M)
    assert np.abs(Q).max() <= 1e-13 * nu * M.max()
    assert np.abs(P).max() <= 1e-13 * nu * M.max()


# Maxwellian-weighted variant (conserve_proj = 2): q_c = q - M (lambda . phi). It is fixed by
# (i) zero moments and (ii) q - q_c = M (phi . c) for some c, checked with numpy least squares.
def check_weighted(q, qc, M, Phi, tol=1e-13):
    scale = (np.abs(Phi) * np.abs(q.reshape(-1, 1))).sum(0)
    assert np.all(np.abs(Phi.T @ qc.reshape(-1)) <= tol * scale)
    d = (q - qc).reshape(-1)
    MPhi = M.reshape(-1, 1) * Phi
    coef, *_ = np.linalg.lstsq(MPhi, d, rcond=None)
    assert np.abs(MPhi @ coef - d).max() <= 1e-13 * np.abs(q).max()


@pytest.mark.parametrize("N,L,seed", [(8, 6.0, 0), (16, 10.0, 3)])
def test_weighted_projection_of_random_vectors(oracle, N, L, seed):
    rng = np.random.default_rng(seed)
    v = (np.arange(N) - N // 2 + 1) * (2 * L / N)
    V = np.stack(np.meshgrid(v, v, v, indexing="ij"), -1)
    M = 1.3 / (2 * np.pi * 1.7) ** 1.5 * np.exp(-((V - [0.8, 0.2, -0.3]) ** 2).sum(-1) / (2 * 1.7))
    q = rng.standard_normal((N, N, N)) * M
    qc = oracle.conserve_project_w(q, L, M)
    check_weighted(q, qc, M, basis(N, L))
    assert np.abs(oracle.conserve_project_w(qc, L, M) - qc).max() <= 1e-13 * np.abs(q).max()
    # far from the Maxwellian the correction vanishes with it (the tails are left alone)
    far = M < 1e-12 * M.max()
    assert np.abs((qc - q)[far]).max() <= 1e-10 * np.abs(q).max()


@pytest.mark.parametrize("kernel", [0, 1])
def test_weighted_projected_collision_conserves(oracle, kernel):
    N, L = 16, 8.0
    f = bimodal(N, L)
    Q0, P0, nu0, th = oracle.collide_cell(oracle.Problem(N=N, L=L, kernel=kernel), f)
    Q2, P2, nu2, th2 = oracle.collide_cell(oracle.Problem(N=N, L=L, kernel=kernel, conserve_proj=2), f)
    M = oracle.eval_maxwellian(N, L, th)
    check_weighted(Q0, Q2, M, basis(N, L))
    assert np.abs((P2 - P0) - (Q2 - Q0)).max() <= 1e-14 * np.abs(Q0).max()
    # the weighted and the plain projection both zero the moments, with different corrections
    Q1, _, _, _ = oracle.collide_cell(oracle.Problem(N=N, L=L, kernel=kernel, conserve_proj=1), f)
    assert np.abs(Q1 - Q2).max() > 1e-6 * np.abs(Q1 - Q0).max()
