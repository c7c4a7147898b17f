"""Pins of the oracle's quadrature, Fourier weights and DFT against independent references.

- Gauss-Legendre nodes/weights against numpy's leggauss (library routine).
- G(a, b) against scipy's adaptive quad and against the closed form of the radial
  integral for Maxwell molecules (products of sines integrate in closed form).
- The gain/loss Fourier weights of the collision integral (eq. (2)) evaluated by direct
  product quadrature over |q| <= 2R, the direction of q and the unit vector w, with no
  use of the sphere-average identity: this pins G's definition including 16 pi^2.
- DFT / inverse DFT against numpy's FFT.
"""
import numpy as np
import pytest
from scipy import integrate

B0 = 1.0 / (4.0 * np.pi)


def R_of(L):
    return 2.0 * L / (3.0 * np.sqrt(2.0) + 1.0)


def G_scipy(L, kernel, b0, a2, b2):
    R2 = 2.0 * R_of(L)
    c = np.pi / (2.0 * L)
    a, b = np.sqrt(a2), np.sqrt(b2)

    def f(r):
        B = b0 * r if kernel == 1 else b0
        return 16 * np.pi**2 * r * r * B * np.sinc(c * a * r / np.pi) * np.sinc(c * b * r / np.pi)

    pts = np.linspace(0, R2, 33)
    return sum(integrate.quad(f, pts[i], pts[i + 1], epsabs=1e-15, epsrel=1e-14, limit=200)[0] for i in range(32))


def G_closed_maxwell(L, b0, a2, b2):
    R2 = 2.0 * R_of(L)
    c = np.pi / (2.0 * L)
    a, b = np.sqrt(a2), np.sqrt(b2)
    K = 16 * np.pi**2 * b0
    if a == 0 and b == 0:
        return K * R2**3 / 3
    if b == 0 or a == 0:
        s = c * max(a, b)
        return K / s * (np.sin(s * R2) / s**2 - R2 * np.cos(s * R2) / s)
    if a == b:
        return K / (c * c * a * a) * (R2 / 2 - np.sin(2 * c * a * R2) / (4 * c * a))
    return K / (c * c * a * b) * 0.5 * (np.sin(c * (a - b) * R2) / (c * (a - b)) - np.sin(c * (a + b) * R2) / (c * (a + b)))


def test_gauss_legendre_matches_numpy(oracle):
    for n in (5, 20, 33):
        x, w = oracle.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        o = np.argsort(x)
        np.testing.assert_allclose(x[o], xr, atol=2e-15)
        np.testing.assert_allclose(w[o], wr, atol=2e-15)


@pytest.mark.parametrize("L", [6.0, 8.0, 10.0])
def test_G_maxwell_closed_form_and_quad(oracle, L):
    N = 32
    h = N // 2 - 1
    scale = G_closed_maxwell(L, B0, 0, 0)
    rng = np.random.default_rng(1)
    pairs = [(0, 0), (0, 5), (7, 0), (3, 3), (12 * h * h, 0), (3 * h * h, 12 * h * h), (674, 675), (2, 2700)]
    pairs += [(int(rng.integers(0, 3 * h * h + 1)), int(rng.integers(0, 12 * h * h + 1))) for _ in range(12)]
    for a2, b2 in pairs:
        g = oracle.G(N, L, 0, B0, a2, b2)
        assert abs(g - G_closed_maxwell(L, B0, a2, b2)) <= 1e-13 * scale, (a2, b2)
        assert abs(g - G_scipy(L, 0, B0, a2, b2)) <= 1e-12 * scale, (a2, b2)
        assert abs(g - oracle.G(N, L, 0, B0, b2, a2)) <= 1e-14 * scale  # symmetric in (a, b)


def test_G_hard_sphere_quad(oracle):
    L, N = 10.0, 32
    scale = abs(G_scipy(L, 1, B0, 0, 0))
    for a2, b2 in [(0, 0), (1, 0), (0, 9), (5, 17), (675, 2700), (300, 1000)]:
        g = oracle.G(N, L, 1, B0, a2, b2)
        assert abs(g - G_scipy(L, 1, B0, a2, b2)) <= 1e-12 * scale, (a2, b2)


def _sphere_rule(nt=24, nph=48):
    ct, wt = np.polynomial.legendre.leggauss(nt)
    ph = 2 * np.pi * np.arange(nph) / nph
    st = np.sqrt(1 - ct * ct)
    u = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)), np.outer(ct, np.ones(nph))], -1).reshape(-1, 3)
    w = np.outer(wt, np.full(nph, 2 * np.pi / nph)).reshape(-1)
    return u, w


def brute_weights(L, kernel, b0, l, m, nr=40):
    """Gain and loss Fourier weights of eq. (2) by product quadrature in (|q|, q/|q|, w)."""
    xi = np.pi / L
    R2 = 2 * R_of(L)
    x, wx = np.polynomial.legendre.leggauss(nr)
    r = 0.5 * R2 * (x + 1)
    wr = 0.5 * R2 * wx
    u, wu = _sphere_rule()
    l, m = np.asarray(l, float), np.asarray(m, float)
    B = b0 * r if kernel == 1 else b0 * np.ones_like(r)
    # gain: exp(-i xi [(l+m).q + |q| (l-m).w]/2) with q = r u
    Eu = (wu[None, :] * np.exp(-0.5j * xi * r[:, None] * (u @ (l + m))[None, :])).sum(1)
    Ew = (wu[None, :] * np.exp(-0.5j * xi * r[:, None] * (u @ (l - m))[None, :])).sum(1)
    gain = (wr * r * r * B * Eu * Ew).sum()
    # loss: mode l sits on f(v_*) = f(v - q): exp(-i xi l.q), w-integral gives 4 pi
    El = (wu[None, :] * np.exp(-1j * xi * r[:, None] * (u @ l)[None, :])).sum(1)
    loss = (wr * r * r * B * El * wu.sum()).sum()
    return gain, loss


@pytest.mark.parametrize("kernel", [0, 1])
def test_fourier_weights_bruteforce(oracle, kernel):
    L, N = 6.0, 8
    scale = abs(oracle.G(N, L, kernel, B0, 0, 0))
    for l, m in [((0, 0, 0), (0, 0, 0)), ((1, 0, 0), (0, 0, 0)), ((1, -1, 2), (0, 2, -1)), ((3, 1, 0), (-2, 1, 1)),
                 ((2, 2, 2), (-3, 0, 1))]:
        gain, loss = brute_weights(L, kernel, B0, l, m)
        lp = np.add(l, m)
        lm = np.subtract(l, m)
        g = oracle.G(N, L, kernel, B0, int(lp @ lp), int(lm @ lm))
        lo = oracle.G(N, L, kernel, B0, int(4 * np.dot(l, l)), 0)
        assert abs(gain.imag) < 1e-12 * scale and abs(loss.imag) < 1e-12 * scale
        assert abs(gain.real - g) <= 1e-11 * scale, (l, m, gain, g)
        assert abs(loss.real - lo) <= 1e-11 * scale, (l, m, loss, lo)


def _fft_reference(f):
    N = f.shape[0]
    h = N // 2 - 1
    F = np.fft.fftn(f) / N**3
    k = np.arange(-h, h + 1)
    ph = np.exp(2j * np.pi * k * (N // 2 - 1) / N)  # index i = j + N/2 - 1
    sub = F[np.ix_(k % N, k % N, k % N)]
    return sub * ph[:, None, None] * ph[None, :, None] * ph[None, None, :]


@pytest.mark.parametrize("N", [4, 8, 16])
def test_dft_matches_numpy_fft(oracle, N):
    f = np.random.default_rng(N).random((N, N, N))
    np.testing.assert_allclose(oracle.dft(f), _fft_reference(f), rtol=0, atol=1e-15 * abs(f).sum() / N**3 * 10)


@pytest.mark.parametrize("N", [4, 8, 16])
def test_idft_matches_numpy_ifft(oracle, N):
    h = N // 2 - 1
    rng = np.random.default_rng(N + 1)
    qh = rng.standard_normal((2 * h + 1,) * 3) + 1j * rng.standard_normal((2 * h + 1,) * 3)
    q = oracle.idft(qh, N)
    k = np.arange(-h, h + 1)
    ph = np.exp(-2j * np.pi * k * (N // 2 - 1) / N)
    full = np.zeros((N, N, N), complex)
    full[np.ix_(k % N, k % N, k % N)] = qh * ph[:, None, None] * ph[None, :, None] * ph[None, None, :]
    ref = np.real(np.fft.ifftn(full) * N**3)
    np.testing.assert_allclose(q, ref, atol=1e-12 * abs(qh).sum() / N)


def test_dft_inverse_roundtrip(oracle):
    N = 16
    h = N // 2 - 1
    rng = np.random.default_rng(3)
    # a real function band-limited to |k_i| <= h is reproduced exactly
    qh = rng.standard_normal((2 * h + 1,) * 3) + 1j * rng.standard_normal((2 * h + 1,) * 3)
    qh = 0.5 * (qh + np.conj(qh[::-1, ::-1, ::-1]))
    f = oracle.idft(qh, N)
    np.testing.assert_allclose(oracle.dft(f), qh, atol=1e-12)
