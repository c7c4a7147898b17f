"""Pins of the oracle's discrete Maxwellian (eqs. (13)-(14)) and the PFP step-1 solve.

- A sampled Gaussian is its own discrete Maxwellian (theta recovered to round-off).
- Weighted moments of the solution match the target to round-off, for the plain weights
  and for the |v1|/dx weights of step 1 (eq. (24)).
- Newton converges in a handful of iterations from the continuum guess (the paper
  reports about five on average).
- The existence condition of step 1 (eq. (26)) holds for moments of a positive function.
"""
import numpy as np
import pytest


def grid(N, L):
    v = (np.arange(N) - N // 2 + 1) * (2 * L / N)
    return v, np.stack(np.meshgrid(v, v, v, indexing="ij"), -1)


def test_gaussian_is_its_own_discrete_maxwellian(oracle):
    N, L = 16, 6.0
    v, V = grid(N, L)
    U, T, rho = np.array([0.4, -0.3, 0.2]), 1.3, 0.8
    th_true = np.array([np.log(rho / (2 * np.pi * T) ** 1.5) - U @ U / (2 * T), *(U / T), 1 / (2 * T)])
    M = np.exp(th_true[0] + V @ th_true[1:4] - th_true[4] * (V**2).sum(-1))
    th, it = oracle.discrete_maxwellian(N, L, oracle.moments(M, L))
    assert 0 < it <= 8
    np.testing.assert_allclose(th, th_true, atol=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_moments_matched(oracle, seed):
    N, L = 16, 6.0
    v, V = grid(N, L)
    rng = np.random.default_rng(seed)
    f = np.exp(-((V - rng.uniform(-0.5, 0.5, 3)) ** 2).sum(-1) / (2 * rng.uniform(0.7, 1.8)))
    f *= 1 + 0.3 * rng.uniform(-1, 1, f.shape)
    m = oracle.moments(f, L)
    th, it = oracle.discrete_maxwellian(N, L, m)
    assert 0 < it <= 10
    M = oracle.eval_maxwellian(N, L, th)
    np.testing.assert_allclose(oracle.moments(M, L), m, rtol=0, atol=1e-14 * abs(m).max())
    # the discrete Maxwellian has the form exp(alpha + beta.v - gamma |v|^2)
    lm = np.log(M)
    np.testing.assert_allclose(lm, th[0] + V @ th[1:4] - th[4] * (V**2).sum(-1), atol=1e-12)


def test_weighted_step1_moments(oracle):
    N, L, dx = 16, 6.0, 1.0 / 16
    v, V = grid(N, L)
    wk = (2 * L / N) ** 3 * np.abs(V[..., 0]) / dx
    th_true = np.array([-2.0, 0.3, -0.1, 0.05, 0.45])
    Mt = np.exp(th_true[0] + V @ th_true[1:4] - th_true[4] * (V**2).sum(-1))
    phi = np.stack([np.ones_like(Mt), V[..., 0], V[..., 1], V[..., 2], (V**2).sum(-1)])
    s = (phi * wk * Mt).reshape(5, -1).sum(1)
    # existence condition (eq. (26)) for moments of a positive function
    assert s[0] > 0 and s[0] * s[4] > s[1] ** 2 + s[2] ** 2 + s[3] ** 2
    th, it = oracle.discrete_maxwellian(N, L, s, wk=wk, theta0=th_true + np.array([0.1, 0.05, 0.0, -0.05, 0.03]))
    assert it > 0
    np.testing.assert_allclose(th, th_true, atol=1e-12)


def test_newton_failure_reported(oracle):
    N, L = 8, 6.0
    # negative energy: no Maxwellian has these moments
    th, it = oracle.discrete_maxwellian(N, L, np.array([1.0, 0.0, 0.0, 0.0, -1.0]))
    assert it < 0
    th, it = oracle.discrete_maxwellian(N, L, np.array([1.0, 0.0, 0.0, 0.0, 3.0]), maxit=0)
    assert it < 0
