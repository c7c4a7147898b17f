"""Pins of the oracle's collision operator (Fourier spectral method, eq. (16)).

- The direct Galerkin sum against a naive Python double loop over all mode pairs with
  weights from scipy quadrature and coefficients from numpy's FFT (tiny grids).
- Exact mass conservation (the (l, -l) weights vanish), Hermitian symmetry.
- Q[M] = 0 for the discrete Maxwellian (steady-state-preserving form, eq. (16)) and
  Q^FSM[M, M] small for a resolved Maxwellian.
- The BKW closed-form relaxation for Maxwell molecules with B = 1/(4 pi):
  f = exp(-|v|^2/2K)/(2 (2 pi K)^{3/2}) ((5K-3)/K + (1-K)|v|^2/K^2), K = 1 - exp(-t/6),
  Q = df/dt. Its normalisation is itself checked against a brute-force quadrature of
  the continuum operator (eq. (2)).
- Hard spheres against brute-force quadrature of the truncated operator (|q| <= 2R):
  spectral convergence with N.
- Entropy dissipation sum w Q ln f <= 0 near equilibrium.
"""
import numpy as np
import pytest
from scipy import integrate

B0 = 1.0 / (4.0 * np.pi)


def R_of(L):
    return 2.0 * L / (3.0 * np.sqrt(2.0) + 1.0)


def G_scipy(L, kernel, a2, b2):
    R2 = 2.0 * R_of(L)
    c = np.pi / (2.0 * L)
    a, b = np.sqrt(a2), np.sqrt(b2)

    def f(r):
        B = B0 * r if kernel == 1 else B0
        return 16 * np.pi**2 * r * r * B * np.sinc(c * a * r / np.pi) * np.sinc(c * b * r / np.pi)

    return integrate.quad(f, 0.0, R2, epsabs=1e-15, epsrel=1e-14, limit=400)[0]


def fft_coeffs(f):
    N = f.shape[0]
    h = N // 2 - 1
    F = np.fft.fftn(f) / N**3
    k = np.arange(-h, h + 1)
    ph = np.exp(2j * np.pi * k * (N // 2 - 1) / N)
    return F[np.ix_(k % N, k % N, k % N)] * ph[:, None, None] * ph[None, :, None] * ph[None, None, :]


def grid(N, L):
    v = (np.arange(N) - N // 2 + 1) * (2 * L / N)
    V = np.stack(np.meshgrid(v, v, v, indexing="ij"), -1)
    return v, V


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
@pytest.mark.parametrize("N,kernel", [(4, 0), (6, 0), (6, 1)])
def test_direct_sum_matches_naive_galerkin(oracle, N, kernel):
    L = 6.0
    h = N // 2 - 1
    rng = np.random.default_rng(N)
    a = rng.random((N, N, N))
    b = rng.random((N, N, N))
    ah, bh = fft_coeffs(a), fft_coeffs(b)
    cacheG = {}

    def Gq(a2, b2):
        if (a2, b2) not in cacheG:
            cacheG[(a2, b2)] = G_scipy(L, kernel, a2, b2)
        return cacheG[(a2, b2)]

    rng_k = range(-h, h + 1)
    ref = np.zeros((2 * h + 1,) * 3, complex)
    for k in np.ndindex(*(2 * h + 1,) * 3):
        kk = np.array(k) - h
        acc = 0j
        for m in np.ndindex(*(2 * h + 1,) * 3):
            mm = np.array(m) - h
            ll = kk - mm
            if np.any(np.abs(ll) > h):
                continue
            beta = Gq(int(kk @ kk), int((ll - mm) @ (ll - mm))) - Gq(int(4 * mm @ mm), 0)
            acc += beta * ah[tuple(ll + h)] * bh[tuple(mm + h)]
        ref[k] = acc
    got = oracle.qhat_direct(N, L, kernel, B0, ah, bh)
    assert abs(got - ref).max() <= 1e-12 * abs(ref).max()
    del rng_k


def test_mass_conservation_and_hermitian(oracle):
    N, L = 16, 6.0
    f = np.random.default_rng(5).random((N, N, N))
    fh = oracle.dft(f)
    qh = oracle.qhat_direct(N, L, 0, B0, fh, fh)
    h = N // 2 - 1
    assert abs(qh[h, h, h]) <= 1e-15 * abs(qh).max()
    np.testing.assert_allclose(qh, np.conj(qh[::-1, ::-1, ::-1]), atol=1e-14 * abs(qh).max())
    q = oracle.qfsm(f, L)
    assert abs(q.sum()) <= 1e-14 * abs(q).sum()


def test_collision_of_discrete_maxwellian_vanishes(oracle):
    N, L = 16, 6.0
    prob = oracle.Problem(N=N, L=L)
    v, V = grid(N, L)
    U = np.array([0.3, -0.2, 0.1])
    M = 1.1 / (2 * np.pi * 1.2) ** 1.5 * np.exp(-((V - U) ** 2).sum(-1) / (2 * 1.2))
    Q, P, nu, th = oracle.collide_cell(prob, M)
    scale = nu * M.max()
    assert abs(Q).max() <= 1e-13 * scale
    assert abs(P).max() <= 1e-13 * scale
    # the unsubtracted spectral operator is only spectrally small on a resolved Maxwellian
    assert abs(oracle.qfsm(M, L)).max() <= 1e-5 * scale


def test_momentum_energy_spectral_conservation(oracle):
    """Momentum and energy are conserved to spectral accuracy only: check the decay with N."""
    errs = []
    for N in (24, 32):
        L = 8.0
        v, V = grid(N, L)
        f = np.exp(-((V - [0.4, 0, 0]) ** 2).sum(-1) / 1.4) + 0.5 * np.exp(-((V + [0.3, 0.2, 0]) ** 2).sum(-1) / 0.9)
        q = oracle.qfsm(f, L)
        w = (2 * L / N) ** 3
        scale = w * (np.abs(q) * (1 + (V**2).sum(-1))).sum()
        assert abs(w * q.sum()) <= 1e-14 * scale
        e = max([abs(w * (q * V[..., d]).sum()) for d in range(3)] + [abs(w * (q * (V**2).sum(-1)).sum())])
        errs.append(e / scale)
    assert errs[1] <= 1e-4 and errs[1] < 0.1 * errs[0], errs


def bkw(v2, K):
    return np.exp(-v2 / (2 * K)) / (2 * (2 * np.pi * K) ** 1.5) * ((5 * K - 3) / K + (1 - K) / K**2 * v2)


def bkw_dt(v2, K):
    # d/dK of the closed form, times dK/dt = (1 - K)/6
    e = np.exp(-v2 / (2 * K)) / (2 * (2 * np.pi * K) ** 1.5)
    poly = (5 * K - 3) / K + (1 - K) / K**2 * v2
    de = e * (v2 / (2 * K * K) - 1.5 / K)
    dpoly = 3 / K**2 + v2 * (K - 2) / K**3
    return (de * poly + e * dpoly) * (1 - K) / 6


def _sphere(nt=16, nph=32):
    ct, wt = np.polynomial.legendre.leggauss(nt)
    ph = 2 * np.pi * np.arange(nph) / nph
    st = np.sqrt(1 - ct * ct)
    u = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(ct, np.ones(nph))], -1).reshape(-1, 3)
    return u, np.outer(wt, np.full(nph, 2 * np.pi / nph)).reshape(-1)


def continuum_Q(f, v, Rq, kernel=0, nr=48):
    """Brute-force quadrature of eq. (2) with |v - v_*| <= Rq at one velocity v."""
    x, wx = np.polynomial.legendre.leggauss(nr)
    r = 0.5 * Rq * (x + 1)
    wr = 0.5 * Rq * wx
    u, wu = _sphere()
    fv = f(v[None, :])[0]
    acc = 0.0
    for i in range(nr):
        B = B0 * r[i] if kernel == 1 else B0
        q = r[i] * u
        vp = v - 0.5 * (q[:, None, :] - r[i] * u[None, :, :])
        vs = v - 0.5 * (q[:, None, :] + r[i] * u[None, :, :])
        g = (f(vp.reshape(-1, 3)) * f(vs.reshape(-1, 3))).reshape(len(u), len(u))
        gain = (wu[:, None] * wu[None, :] * g).sum()
        loss = fv * (wu * f(v - q)).sum() * wu.sum()
        acc += wr[i] * r[i] ** 2 * B * (gain - loss)
    return acc


def test_bkw_normalisation_by_bruteforce():
    K = 0.75

    def f(x):
        return bkw((x * x).sum(-1), K)

    for v in (np.zeros(3), np.array([1.0, 0.5, 0.0]), np.array([2.0, -1.0, 0.5])):
        q = continuum_Q(f, v, 12.0)
        ref = bkw_dt(v @ v, K)
        assert abs(q - ref) <= 1e-9 * f(v[None])[0]


def test_bkw_spectral(oracle):
    N, L, K = 32, 8.0, 0.75
    v, V = grid(N, L)
    V2 = (V**2).sum(-1)
    q = oracle.qfsm(bkw(V2, K), L)
    ref = bkw_dt(V2, K)
    assert abs(q - ref).max() <= 5e-5 * abs(ref).max()


def _mix(x):
    a = np.array([0.6, 0.0, 0.0])
    return np.exp(-((x - a) ** 2).sum(-1) / 0.7) + 0.7 * np.exp(-((x + a) ** 2).sum(-1) / 0.5)


@pytest.mark.parametrize("kernel", [0, 1])
def test_truncated_continuum_convergence(oracle, kernel):
    errs = []
    for N, tol in ((24, 2e-2), (32, 5e-3)):
        L = 8.0
        v, V = grid(N, L)
        q = oracle.qfsm(_mix(V.reshape(-1, 3)).reshape(N, N, N), L, kernel)
        R = R_of(L)
        e = 0.0
        for idx in ((N // 2 - 1,) * 3, (N // 2, N // 2 - 1, N // 2 + 1), (N // 2 + 1, N // 2 - 2, N // 2 - 1)):
            e = max(e, abs(continuum_Q(_mix, V[idx], 2 * R, kernel) - q[idx]))
        errs.append(e / abs(q).max())
        assert errs[-1] <= tol, (N, errs)
    assert errs[1] < 0.5 * errs[0]


@pytest.mark.parametrize("kernel", [0, 1])
def test_entropy_dissipation(oracle, kernel):
    N, L = 16, 6.0
    v, V = grid(N, L)
    M = np.exp(-(V**2).sum(-1) / 2.2)
    for amp in (0.05, 0.2):
        f = M * (1 + amp * np.sin(V[..., 0]) * np.cos(0.7 * V[..., 1]) + amp * 0.5 * np.cos(V[..., 2]))
        q = oracle.qfsm(f, L, kernel)
        assert (q * np.log(f)).sum() < 0.0
