"""Fast Fourier-spectral collision operator in the Carleman form, hard spheres, 3-D
velocity: the oracle of the fast spectral method (the GEMM-shaped form of Q).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: tests import it; the CUDA library
and its binding never do.

Carleman representation of the collision integral (eq. (2)) with both variables truncated
to the ball of radius T = 2R, R the support radius of the velocity box (x = v' - v and
y = v'_* - v each span the support's diameter):

    Q(v) = int int Bt delta(x.y) [f(v + x) f(v + y) - f(v + x + y) f(v)] dx dy,
    |x|, |y| <= T,   Bt = 4 b0 for B = b0 |q| in three dimensions.

With f(v) = sum_k fhat_k exp(i pi k.v / L) (the oracle's transform, modes |k_i| <= N/2 - 1)
the Galerkin coefficients are

    Qhat_k = sum_{l+m=k} (beta(l, m) - beta(m, m)) fhat_l fhat_m,

and in polar coordinates (x = rho e, y = rho' e', delta(x.y) = delta(e.e') / (rho rho'))

    beta(l, m) = 4 b0 int_{S^2_+} phi(l.e) Psi(|m - (m.e) e|) de,
    phi(s)     = 2 int_0^T rho cos(pi rho s / L) drho,
    Psi(t)     = int_0^pi phi(t cos th) dth = 2 pi int_0^T rho J0(pi rho t / L) drho
               = 2 T L J1(pi T t / L) / t          (Psi(0) = pi T^2).

A product rule on the half sphere (Gauss-Legendre in cos(theta) on [0, 1], the trapezoidal
rule in the azimuth) turns the gain into one convolution per node e_p of the weighted
spectra phi(l.e_p) fhat_l and Psi(|m_perp|) fhat_m; the loss uses the same rule for
beta(m, m), which keeps mass conservation exact (beta(-m, m) = beta(m, m) because phi is
even). Convolutions are linear (zero padding), so no mode wraps around.
"""
from __future__ import annotations

import numpy as np
from scipy import special

from . import oracle as O


def support_radius(L: float) -> float:
    """R for the velocity box [-L, L]^3 (the relation L = (3 sqrt 2 + 1) R / 2)."""
    return 2.0 * L / (3.0 * np.sqrt(2.0) + 1.0)


def phi(s, R, L):
    """phi(s) = 2 int_0^R rho cos(a rho) drho, a = pi s / L (closed form; phi(0) = R^2); R is
    the truncation radius."""
    a = np.pi * np.asarray(s, dtype=float) / L
    out = np.full(a.shape, R * R)
    nz = np.abs(a) > 1e-12
    an = a[nz]
    out[nz] = 2.0 * (R * np.sin(an * R) / an + (np.cos(an * R) - 1.0) / (an * an))
    return out


def psi(t, R, L):
    """Psi(t) = 2 pi int_0^R rho J0(pi rho t / L) drho = 2 R L J1(pi R t / L) / t (Psi(0) = pi R^2);
    R is the truncation radius."""
    t = np.asarray(t, dtype=float)
    out = np.full(t.shape, np.pi * R * R)
    nz = t > 1e-12
    out[nz] = 2.0 * R * L * special.j1(np.pi * R * t[nz] / L) / t[nz]
    return out


def half_sphere_rule(m_theta: int, m_phi: int):
    """Nodes e_p (M x 3) and weights w_p on the upper half sphere: Gauss-Legendre in
    mu = cos(theta) on [0, 1], uniform azimuths. The weights sum to 2 pi."""
    x, wx = np.polynomial.legendre.leggauss(m_theta)
    mu, wmu = 0.5 * (x + 1.0), 0.5 * wx
    az = 2.0 * np.pi * np.arange(m_phi) / m_phi
    st = np.sqrt(1.0 - mu * mu)
    e = np.stack([np.outer(st, np.cos(az)), np.outer(st, np.sin(az)), np.outer(mu, np.ones(m_phi))], -1)
    w = np.outer(wmu, np.full(m_phi, 2.0 * np.pi / m_phi))
    return e.reshape(-1, 3), w.reshape(-1)


def mode_grid(N):
    h = N // 2 - 1
    k = np.arange(-h, h + 1)
    return np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).astype(float)  # (n, n, n, 3)


def convolve(a, b):
    """Linear convolution of two (n, n, n) mode arrays indexed -h..h, kept on -h..h."""
    n = a.shape[0]
    h = n // 2
    s = (2 * n - 1,) * 3
    ax = (0, 1, 2)
    c = np.fft.ifftn(np.fft.fftn(a, s, axes=ax) * np.fft.fftn(b, s, axes=ax), axes=ax)
    return c[h:h + n, h:h + n, h:h + n]


def truncation_radius(L: float) -> float:
    """T = 2R: the Carleman variables x, y span the diameter of the support."""
    return 2.0 * support_radius(L)


def beta_fast(lmodes, mmodes, L, b0, rule):
    """beta(l, m) for paired mode lists (P x 3 each) by the half-sphere rule."""
    R = truncation_radius(L)
    e, w = rule
    le = np.asarray(lmodes, float) @ e.T  # (P, M)
    mm = np.asarray(mmodes, float)
    me = mm @ e.T
    mperp = np.sqrt(np.maximum((mm * mm).sum(-1)[:, None] - me * me, 0.0))
    return 4.0 * b0 * (phi(le, R, L) * psi(mperp, R, L)) @ w


def qhat_fast(fhat, N, L, b0, rule):
    """Qhat_k = sum_p w_p 4 b0 [phi(l.e_p) fhat] * [Psi(|m_perp|) fhat] - fhat * (beta(m, m) fhat)."""
    R = truncation_radius(L)
    K = mode_grid(N)
    e, w = rule
    gain = np.zeros_like(fhat)
    bmm = np.zeros(fhat.shape)
    k2 = (K * K).sum(-1)
    for p in range(len(w)):
        ke = K @ e[p]
        kperp = np.sqrt(np.maximum(k2 - ke * ke, 0.0))
        ph, ps = phi(ke, R, L), psi(kperp, R, L)
        gain += w[p] * convolve(ph * fhat, ps * fhat)
        bmm += w[p] * ph * ps
    gain *= 4.0 * b0
    bmm *= 4.0 * b0
    return gain - convolve(fhat, bmm * fhat)


def qfsm_fast(f, L, b0=1.0 / (4.0 * np.pi), m_theta=8, m_phi=16):
    """The fast spectral operator at the velocity nodes of one cell, f (N, N, N)."""
    N = f.shape[0]
    return O.idft(qhat_fast(O.dft(f), N, L, b0, half_sphere_rule(m_theta, m_phi)), N)
