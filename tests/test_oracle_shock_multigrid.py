"""Why the Mach-2 shock does not converge with deep V-cycles: a property of the coarse
problems of eq. (30), shown with the oracle alone.

On the shock (128 cells on [-20, 20], hard spheres, eps = 0.1, Rankine-Hugoniot inflow; a
16^3 velocity grid keeps the oracle fast) the coarse grids of a 4-level cycle have 32 and 16
cells of width 1.25 and 2.5, 12.5 and 25 times eps: the shock lies inside one or two coarse
cells. The coarse right-hand side b_H = R_H(I f) - I R_h(f) then carries the large difference
between the fine and the coarse transport of the shock profile, the coarse correction drives
coarse distributions to non-positive moments, where the discrete Maxwellian of eq. (13) does
not exist, and the iterate becomes non-finite in the second cycle. Two-level cycles (64
coarse cells) stay finite. The GPU library flags the same cycle with its NONPOSITIVE,
NEWTON_FAIL and NONFINITE status bits; its first 4-level cycle agrees with the oracle's."""
import numpy as np
import pytest

from paper_2409_01910_gb300 import inputs as I

pytestmark = pytest.mark.slow


def shock(oracle, N=16):
    wl = I.shock_128cells_32v()
    (r1, u1, T1), (r2, u2, T2) = wl.up, wl.down
    o = oracle.Problem(N=N, L=wl.L, J=wl.J, x_lo=wl.x_lo, x_hi=wl.x_hi, eps=wl.eps, kernel=oracle.HARD_SPHERE,
                       bc_kind=(oracle.INFLOW, oracle.INFLOW), bc_rho=(r1, r2), bc_u=((u1, 0, 0), (u2, 0, 0)),
                       bc_T=(T1, T2), total_mass=0.0, inner_fixed=5)
    w = I.ShockWorkload("shock_N16", J=wl.J, N=N, L=wl.L, eps=wl.eps, up=wl.up, down=wl.down)
    return o, w.initial_state()


def test_deep_vcycles_break_down_on_the_shock_two_levels_do_not(oracle):
    o, f0 = shock(oracle)
    f4 = f0.copy()
    with np.errstate(all="ignore"):
        oracle.vcycle(o, f4, 4, 1, 1, 4)
        assert np.isfinite(f4).all()  # the first 4-level cycle is still finite
        oracle.vcycle(o, f4, 4, 1, 1, 4)
    assert not np.isfinite(f4).all()
    f2 = f0.copy()
    for _ in range(2):
        oracle.vcycle(o, f2, 2, 1, 1, 4)
    assert np.isfinite(f2).all()
    rho = f2.reshape(f2.shape[0], -1).sum(1) * (2 * o.L / o.N) ** 3
    assert rho.min() > 0.9  # upstream density 1, downstream 16/7
