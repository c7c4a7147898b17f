"""Pins of the fast (Carleman-form) spectral oracle, hard spheres, 3-D velocity:
- the closed forms of the radial factors phi and Psi against adaptive quadrature of their
  definitions, and the half-circle reduction int_0^pi phi(t cos th) dth = Psi(t);
- the half-sphere rule against adaptive quadrature of beta(l, m), and beta(0, 0) against
  its closed form 8 pi^2 b0 T^4 from the direct double integral over the truncation balls;
- exact mass conservation; momentum and energy to spectral accuracy (decaying with N);
- convergence to the brute-force continuum operator (the same velocities and tolerances as
  the direct form's pin) and convergence in the number of sphere nodes."""
import numpy as np
import pytest
from scipy import integrate, special

from oracle import fast_spectral as F

B0 = 1.0 / (4.0 * np.pi)


def test_radial_factors_closed_forms():
    L = 8.0
    T = F.truncation_radius(L)
    for s in (0.0, 0.3, 1.0, 2.5, 7.0):
        ref = 2.0 * integrate.quad(lambda r: r * np.cos(np.pi * r * s / L), 0.0, T, limit=200)[0]
        assert F.phi(np.array([s]), T, L)[0] == pytest.approx(ref, rel=1e-10, abs=1e-12)
    for t in (0.0, 0.4, 1.5, 3.0, 9.0):
        ref = 2.0 * np.pi * integrate.quad(lambda r: r * special.j0(np.pi * r * t / L), 0.0, T, limit=200)[0]
        assert F.psi(np.array([t]), T, L)[0] == pytest.approx(ref, rel=1e-10, abs=1e-12)
        circle = integrate.quad(lambda th: F.phi(np.array([t * np.cos(th)]), T, L)[0], 0.0, np.pi, limit=200)[0]
        assert circle == pytest.approx(F.psi(np.array([t]), T, L)[0], rel=1e-9, abs=1e-11)


def test_half_sphere_rule_and_beta():
    L = 6.0
    T = F.truncation_radius(L)
    e, w = F.half_sphere_rule(24, 48)
    assert w.sum() == pytest.approx(2.0 * np.pi, rel=1e-14)
    assert np.all(e[:, 2] >= 0.0) and np.allclose((e * e).sum(1), 1.0)
    # beta(0, 0) = 4 b0 int int delta(x.y) dx dy over |x|, |y| <= T = 8 pi^2 b0 T^4
    assert F.beta_fast([[0, 0, 0]], [[0, 0, 0]], L, B0, (e, w))[0] == pytest.approx(
        8.0 * np.pi ** 2 * B0 * T ** 4, rel=1e-13)
    for l, m in (([1, 0, 2], [0, -1, 1]), ([2, 1, -1], [1, 1, 0]), ([0, 3, 0], [2, 0, 0])):
        l, m = np.array(l, float), np.array(m, float)

        def g(th, az):
            ev = np.array([np.sin(th) * np.cos(az), np.sin(th) * np.sin(az), np.cos(th)])
            mp = np.sqrt(max(m @ m - (m @ ev) ** 2, 0.0))
            return F.phi(np.array([l @ ev]), T, L)[0] * F.psi(np.array([mp]), T, L)[0] * np.sin(th)

        ref = 4.0 * B0 * integrate.dblquad(g, 0.0, 2.0 * np.pi, 0.0, np.pi / 2, epsabs=1e-11, epsrel=1e-10)[0]
        assert F.beta_fast([l], [m], L, B0, (e, w))[0] == pytest.approx(ref, rel=1e-7, abs=1e-9)


def test_fast_mass_is_exact(oracle):
    from test_oracle_collision import grid

    N, L = 16, 8.0
    v, V = grid(N, L)
    f = np.exp(-((V - [0.4, 0, 0]) ** 2).sum(-1) / 1.4) + 0.5 * np.exp(-((V + [0.3, 0.2, 0]) ** 2).sum(-1) / 0.9)
    q = F.qfsm_fast(f, L, B0, 8, 16)
    w = (2 * L / N) ** 3
    assert abs(w * q.sum()) <= 1e-14 * w * (np.abs(q) * (1 + (V ** 2).sum(-1))).sum()


def test_fast_momentum_energy_spectral(oracle):
    """Momentum and energy are conserved to spectral accuracy only: check the decay with N."""
    from test_oracle_collision import grid

    cons = []
    for N in (24, 32):
        L = 8.0
        v, V = grid(N, L)
        f = np.exp(-((V - [0.4, 0, 0]) ** 2).sum(-1) / 1.4) + 0.5 * np.exp(-((V + [0.3, 0.2, 0]) ** 2).sum(-1) / 0.9)
        q = F.qfsm_fast(f, L, B0, 8, 16)
        w = (2 * L / N) ** 3
        scale = w * (np.abs(q) * (1 + (V ** 2).sum(-1))).sum()
        cons.append(max([abs(w * (q * V[..., d]).sum()) for d in range(3)] +
                        [abs(w * (q * (V ** 2).sum(-1)).sum())]) / scale)
    assert cons[1] <= 1e-4 and cons[1] < 0.1 * cons[0], cons


def test_fast_converges_to_continuum(oracle):
    from test_oracle_collision import R_of, _mix, continuum_Q, grid

    errs = []
    for N, rule, tol in ((24, (12, 24), 2.5e-2), (32, (8, 16), 5e-3)):
        L = 8.0
        v, V = grid(N, L)
        q = F.qfsm_fast(_mix(V.reshape(-1, 3)).reshape(N, N, N), L, B0, *rule)
        e = 0.0
        for idx in ((N // 2 - 1,) * 3, (N // 2, N // 2 - 1, N // 2 + 1), (N // 2 + 1, N // 2 - 2, N // 2 - 1)):
            e = max(e, abs(continuum_Q(_mix, V[idx], 2 * R_of(L), 1) - q[idx]))
        errs.append(e / abs(q).max())
        assert errs[-1] <= tol, (N, errs)
    assert errs[1] < 0.5 * errs[0]


def test_fast_converges_in_sphere_nodes(oracle):
    from test_oracle_collision import _mix, grid

    N, L = 16, 8.0
    v, V = grid(N, L)
    f = _mix(V.reshape(-1, 3)).reshape(N, N, N)
    q = [F.qfsm_fast(f, L, B0, mt, 2 * mt) for mt in (4, 8, 16)]
    d1 = np.abs(q[0] - q[2]).max()
    d2 = np.abs(q[1] - q[2]).max()
    assert d2 < 0.2 * d1, (d1, d2)
