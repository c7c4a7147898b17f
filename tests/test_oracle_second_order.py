"""Pins of the oracle's second-order scheme (eq. (reconstruction), eq. (slope); the slopes
explicit in the scans, eq. (SGS_BGK)):
- on a smooth manufactured distribution the discrete transport operator applied to exact
  cell averages differs from the exact cell average of v1 df/dx, which is
  v1 (f(x_{j+1/2}) - f(x_{j-1/2})) / dx, by O(dx^2) in interior cells (O(dx) for the
  first-order scheme);
- between equal walls the uniform Maxwellian is a fixed point of the second-order SGS
  iteration;
- the second-order SGS iteration converges in the second-order residual, to a state that is
  not the first-order steady state."""
import numpy as np
import pytest

from paper_2409_01910_gb300 import inputs as I


def manufactured(oracle, N, L, J):
    """Cell averages (5-point Gauss-Legendre per cell) of f(x, v) = M(v; rho(x), 0, T(x)) and
    the exact cell averages of v1 df/dx."""
    v = oracle.velocity_nodes(N, L)
    V = np.stack(np.meshgrid(v, v, v, indexing="ij"), -1)
    v2 = (V ** 2).sum(-1)

    def f(x):
        rho = 1.0 + 0.2 * np.sin(2 * np.pi * x)
        T = 1.5 + 0.3 * np.cos(2 * np.pi * x)
        return rho / (2 * np.pi * T) ** 1.5 * np.exp(-v2 / (2 * T))

    dx = 1.0 / J
    xg, wg = np.polynomial.legendre.leggauss(5)
    fbar = np.empty((J, N, N, N))
    b = np.empty_like(fbar)
    for j in range(J):
        a, c = j * dx, (j + 1) * dx
        fbar[j] = sum(wk * f(0.5 * (a + c) + 0.5 * dx * xk) for xk, wk in zip(xg, wg)) / 2.0
        b[j] = V[..., 0] * (f(c) - f(a)) / dx
    return fbar, b


@pytest.mark.parametrize("order,rate", [(1, 1.0), (2, 2.0)])
def test_truncation_error_order(oracle, order, rate):
    N, L = 8, 6.0
    errs = []
    for J in (16, 32, 64):
        fbar, b = manufactured(oracle, N, L, J)
        prob = oracle.Problem(N=N, L=L, J=J, eps=1.0, bc_T=(1.5, 1.5), order=order)
        _, R = oracle.residual(prob, fbar, np.zeros_like(fbar), b=b, return_field=True)
        errs.append(np.abs(R[3:-3]).max())  # interior cells: central slopes on both sides
    observed = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(observed - rate) < 0.15), (errs, observed)


def test_uniform_maxwellian_fixed_point_second_order(oracle):
    N, L, J = 16, 8.0, 6
    M = I.sampled_maxwellian(N, L, 1.0, (0, 0, 0), 1.3)
    f = np.ascontiguousarray(np.repeat(M[None], J, 0))
    prob = oracle.Problem(N=N, L=L, J=J, eps=0.2, bc_T=(1.3, 1.3), total_mass=(2 * L / N) ** 3 * M.sum(), order=2)
    g = f.copy()
    st = oracle.sgs_iteration(prob, g)
    assert np.abs(g - f).max() <= 1e-13 * f.max()
    assert st["inner_iters"] == 0


def test_second_order_iteration_converges_to_its_own_steady_state(oracle):
    N, L, J = 8, 6.0, 8
    kw = dict(N=N, L=L, J=J, eps=1.0, bc_T=(1.0, 1.5), total_mass=1.0, inner_tol=1e-12)
    p2, p1 = oracle.Problem(order=2, **kw), oracle.Problem(order=1, **kw)
    f = I.initial_state(J, N, L, T=1.25, seed=24)
    r0 = oracle.solve_residual(p2, f)
    for _ in range(40):
        oracle.sgs_iteration(p2, f)
    r2 = oracle.solve_residual(p2, f)
    assert r2 < 1e-4 * r0, (r0, r2)
    # the first-order equations are not satisfied by the second-order steady state
    assert oracle.solve_residual(p1, f) > 100 * r2


# ----------------------------------------------------------------------------- 2-D space
def test_2d_second_order_reduces_to_1d(oracle):
    """One 2-D row (ny = 1, dy huge): the four orderings with slopes from the state before
    each are two 1-D second-order SGS iterations."""
    N, L, nx = 8, 6.0, 5
    base = oracle.Problem(N=N, L=L, J=nx, eps=0.5, bc_T=(1.0, 2.0), total_mass=0.0, inner_fixed=4, order=2)
    q = oracle.Problem2D(base=base, ny=1, y_lo=0.0, y_hi=1e12, bc_T_y=(1.5, 1.3))
    f0 = I.initial_state(nx, N, L, T=1.4, seed=3)
    f2 = f0.copy()
    oracle.sgs_iteration2d(q, f2)
    f1 = f0.copy()
    for _ in range(2):
        oracle.sgs_iteration(base, f1, rescale=False)
    assert np.abs(f2 - f1).max() <= 1e-10 * np.abs(f1).max()


def manufactured_2d(oracle, N, L, n):
    v = oracle.velocity_nodes(N, L)
    V = np.stack(np.meshgrid(v, v, v, indexing="ij"), -1)
    v2 = (V ** 2).sum(-1)

    def f(x, y):
        rho = 1.0 + 0.2 * np.sin(2 * np.pi * x) * np.cos(np.pi * y)
        T = 1.5 + 0.3 * np.cos(2 * np.pi * y + 0.5) + 0.1 * x
        return rho / (2 * np.pi * T) ** 1.5 * np.exp(-v2 / (2 * T))

    h = 1.0 / n
    xg, wg = np.polynomial.legendre.leggauss(5)
    fbar = np.empty((n * n, N, N, N))
    b = np.empty_like(fbar)
    for j in range(n):
        for i in range(n):
            xs, ys = (i + 0.5 + 0.5 * xg) * h, (j + 0.5 + 0.5 * xg) * h
            fbar[j * n + i] = sum(wa * wb * f(xa, yb) for xa, wa in zip(xs, wg) for yb, wb in zip(ys, wg)) / 4.0
            fx = sum(wb * (f((i + 1) * h, yb) - f(i * h, yb)) for yb, wb in zip(ys, wg)) / 2.0
            fy = sum(wa * (f(xa, (j + 1) * h) - f(xa, j * h)) for xa, wa in zip(xs, wg)) / 2.0
            b[j * n + i] = (V[..., 0] * fx + V[..., 1] * fy) / h
    return fbar, b


@pytest.mark.parametrize("order,rate", [(1, 1.0), (2, 2.0)])
def test_2d_truncation_error_order(oracle, order, rate):
    N, L = 8, 6.0
    errs = []
    for n in (16, 32):  # n = 8 leaves too few interior cells for the asymptotic rate
        fbar, b = manufactured_2d(oracle, N, L, n)
        base = oracle.Problem(N=N, L=L, J=n, eps=1.0, bc_T=(1.5, 1.5), order=order)
        q = oracle.Problem2D(base=base, ny=n, bc_T_y=(1.5, 1.5))
        _, R = oracle.residual2d(q, fbar, np.zeros_like(fbar), b=b, return_field=True)
        R = R.reshape(n, n, N, N, N)[3:-3, 3:-3]  # interior cells
        errs.append(np.abs(R).max())
    observed = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(observed - rate) < 0.2), (errs, observed)


def test_2d_uniform_maxwellian_fixed_point_second_order(oracle):
    N, L, n = 16, 8.0, 3
    M = I.sampled_maxwellian(N, L, 1.0, (0, 0, 0), 1.2)
    f = np.ascontiguousarray(np.repeat(M[None], n * n, 0))
    base = oracle.Problem(N=N, L=L, J=n, eps=0.3, bc_T=(1.2, 1.2), total_mass=(2 * L / N) ** 3 * M.sum(), order=2)
    q = oracle.Problem2D(base=base, ny=n, bc_T_y=(1.2, 1.2))
    g = f.copy()
    oracle.sgs_iteration2d(q, g)
    assert np.abs(g - f).max() <= 1e-13 * f.max()
