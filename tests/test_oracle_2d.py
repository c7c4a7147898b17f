"""Pins of the 2-D-space oracle (four-ordering SGS, four diffuse walls, 2 x 2 FAS).

- With one cell row and a huge cell height (dy = 1e12) the y-transport terms vanish and one
  2-D SGS iteration equals two 1-D SGS iterations (orderings SW->NE, NE->SW, NW->SE, SE->NW
  scan x forward, backward, forward, backward); with one cell column the same holds along
  y, against the 1-D oracle applied to the distribution with v1 and v2 exchanged. This
  pins the 2-D transport, ghosts and orderings to the pinned 1-D oracle in each direction.
- Global equilibrium: with all walls at rest at one temperature the uniform Maxwellian is
  an exact fixed point.
- A converged BGK cavity (moving lid) has zero net mass flux out of every cell and the
  prescribed total mass; a FAS V-cycle leaves it unchanged.
"""
import numpy as np
import pytest

from paper_2409_01910_gb300 import inputs as I


def grid(N, L):
    v = (np.arange(N) - N // 2 + 1) * (2 * L / N)
    return v, np.stack(np.meshgrid(v, v, v, indexing="ij"), -1)


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_reduces_to_1d_along_x(oracle):
    N, L, nx = 8, 6.0, 5
    base = oracle.Problem(N=N, L=L, J=nx, eps=0.5, bc_T=(1.0, 2.0), total_mass=0.0, inner_fixed=4)
    q = oracle.Problem2D(base=base, ny=1, y_lo=0.0, y_hi=1e12, bc_T_y=(1.5, 1.3))
    f0 = I.initial_state(nx, N, L, T=1.4, seed=3)
    f2 = f0.copy()
    oracle.sgs_iteration2d(q, f2)
    f1 = f0.copy()
    for _ in range(2):
        oracle.sgs_iteration(base, f1, rescale=False)
    assert rel(f2, f1) <= 1e-10


def test_reduces_to_1d_along_y(oracle):
    N, L, ny = 8, 6.0, 5
    base = oracle.Problem(N=N, L=L, J=1, x_lo=0.0, x_hi=1e12, eps=0.5, bc_T=(1.5, 1.3), total_mass=0.0,
                          inner_fixed=4)
    q = oracle.Problem2D(base=base, ny=ny, y_lo=0.0, y_hi=1.0, bc_T_y=(1.0, 2.0))
    f0 = I.initial_state(ny, N, L, T=1.4, seed=4)
    f2 = f0.copy()
    oracle.sgs_iteration2d(q, f2)
    # 1-D along y: exchange v1 and v2; orderings scan y forward, backward, backward, forward
    p1 = oracle.Problem(N=N, L=L, J=ny, eps=0.5, bc_T=(1.0, 2.0), total_mass=0.0, inner_fixed=4)
    f1 = np.ascontiguousarray(f0.transpose(0, 2, 1, 3))
    for d in (1, -1, -1, 1):
        Q, P, nu = oracle.collide(p1, f1)
        oracle.sweep(p1, f1, P, nu, d)
    assert rel(f2, np.ascontiguousarray(f1.transpose(0, 2, 1, 3))) <= 1e-10


def test_equilibrium_is_a_fixed_point(oracle):
    N, L, nx, ny = 16, 8.0, 3, 2
    M = I.sampled_maxwellian(N, L, 1.0, (0, 0, 0), 1.0)
    f = np.ascontiguousarray(np.repeat(M[None], nx * ny, 0))
    mass = (2 * L / N) ** 3 * M.sum()  # unit square
    base = oracle.Problem(N=N, L=L, J=nx, eps=0.5, bc_T=(1.0, 1.0), total_mass=mass)
    q = oracle.Problem2D(base=base, ny=ny, bc_T_y=(1.0, 1.0))
    f0 = f.copy()
    st = oracle.sgs_iteration2d(q, f)
    assert abs(f - f0).max() <= 1e-13 * f0.max()
    assert st["inner_iters"] == 0 and st["visits"] == 4 * nx * ny


def bgk_cavity(oracle, n=4):
    N, L = 8, 6.0
    base = oracle.Problem(N=N, L=L, J=n, eps=0.5, kernel=oracle.BGK, bc_T=(1.0, 1.0), total_mass=1.0,
                          inner_tol=1e-13)
    q = oracle.Problem2D(base=base, ny=n, bc_T_y=(1.0, 1.0), bc_u_y=((0.0, 0.0, 0.0), (0.3, 0.0, 0.0)))
    f = I.initial_state(n * n, N, L, T=1.0, seed=5)
    res = 1.0
    for it in range(200):
        oracle.sgs_iteration2d(q, f)
        res = oracle.solve_residual2d(q, f)
        if res < 1e-12:
            break
    return q, f, res


def test_converged_bgk_cavity_conserves_mass_cellwise(oracle):
    q, f, res = bgk_cavity(oracle)
    assert res < 1e-12, res
    N, L, n = 8, 6.0, 4
    v, V = grid(N, L)
    w = (2 * L / N) ** 3
    v1, v2 = V[..., 0], V[..., 1]
    dx = dy = 1.0 / n
    F = f.reshape(n, n, N, N, N)  # [j][i]

    def nb(i, j, s):
        ii, jj = i + (s == 1) - (s == 0), j + (s == 3) - (s == 2)
        if 0 <= ii < n and 0 <= jj < n:
            return F[jj, ii]
        return oracle.ghost2d(q, s, F[j, i])

    net = []
    for j in range(n):
        for i in range(n):
            c = F[j, i]
            flux = (np.maximum(v1, 0) * (c - nb(i, j, 0)) + np.minimum(v1, 0) * (nb(i, j, 1) - c)) / dx + \
                   (np.maximum(v2, 0) * (c - nb(i, j, 2)) + np.minimum(v2, 0) * (nb(i, j, 3) - c)) / dy
            net.append(w * flux.sum())
    assert np.abs(net).max() <= 1e-10
    assert w * f.sum() * dx * dy == pytest.approx(1.0, rel=1e-12)
    # the lid drags the gas: positive x-velocity in the top row, negative in the bottom row
    ux = [(w * (F[j] * v1).sum((1, 2, 3)) / (w * F[j].sum((1, 2, 3)))).mean() for j in range(n)]
    assert ux[-1] > 0 > ux[0]


def test_vcycle_keeps_the_converged_cavity(oracle):
    q, f, res = bgk_cavity(oracle)
    g = f.copy()
    oracle.vcycle2d(q, g, 2, 1, 1, 4)
    assert rel(g, f) <= 1e-10
    assert oracle.solve_residual2d(q, g) < 1e-11
