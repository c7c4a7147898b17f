"""GPU parity of the second-order scheme (eq. (reconstruction), eq. (slope), explicit slopes
in the scans, eq. (SGS_BGK)) against the oracle: SGS iterations and the outer residual
(FP64, 1e-12), a double-float scan (1e-11), a 3-level FAS V-cycle (1e-12), and inflow sides
(1e-12), with fixed inner counts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2409_01910_gb300 import inputs as I
from paper_2409_01910_gb300 import sgs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sgs.lib()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).cuda()


def heat(oracle, precision=sgs.FP64, J=8, eps=0.1):
    N, L = 8, 6.0
    kw = dict(eps=eps, bc_T=(1.0, 1.7), total_mass=1.0, inner_fixed=6)
    g = sgs.Problem(nx=J, nv=N, v_max=L, precision=precision, order=2, **kw)
    o = oracle.Problem(N=N, L=L, J=J, order=2, **kw)
    return g, o, I.initial_state(J, N, L, T=1.4, seed=41)


def test_second_order_iterations_and_residual(oracle):
    g, o, f0 = heat(oracle)
    fo = f0.copy()
    s = sgs.Solver(g)
    f = dev(f0)
    Q, P = s.field(), s.field()
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    for it in range(3):
        oracle.sgs_iteration(o, fo)
        s.iterate(f, Q, P, flags=sgs.IT_EVAL | (sgs.IT_P_VALID if it else 0), res=res)
    assert s.read_status()["status"] == 0
    assert rel(f.cpu().numpy().reshape(f0.shape), fo) <= 1e-12
    ro = oracle.solve_residual(o, fo)
    assert abs(res.item() - ro) <= 1e-10 * ro, (res.item(), ro)


@pytest.mark.parametrize("direction", [1, -1])
def test_second_order_df64_scan(oracle, direction):
    g, o, f0 = heat(oracle, precision=sgs.FP32, eps=0.01)
    Qo, Po, nuo = oracle.collide(o, f0)
    fo = f0.copy()
    oracle.sweep(o, fo, Po, nuo, direction)
    s = sgs.Solver(g)
    f = dev(f0)
    Q, P = s.field(), s.field()
    s.collide(f, Q, P)
    (s.sweep_forward if direction > 0 else s.sweep_backward)(f, dev(Po))
    assert s.read_status()["status"] == 0
    assert rel(f.cpu().numpy().reshape(f0.shape), fo) <= 1e-11


def test_second_order_vcycle(oracle):
    g, o, f0 = heat(oracle, eps=0.05)
    fo = f0.copy()
    oracle.vcycle(o, fo, 3, 1, 1, 2)
    s = sgs.Solver(g)
    f = dev(f0)
    s.vcycle(f, 3, 1, 1, 2)
    assert s.read_status()["status"] == 0
    assert rel(f.cpu().numpy().reshape(f0.shape), fo) <= 1e-12


def test_second_order_inflow(oracle):
    N, L, J = 8, 8.0, 8
    up, down = I.rankine_hugoniot(2.0)
    kw = dict(eps=0.5, total_mass=0.0, inner_fixed=4)
    bc = dict(bc_rho=(up[0], down[0]), bc_u=((up[1], 0.0, 0.0), (down[1], 0.0, 0.0)), bc_T=(up[2], down[2]))
    g = sgs.Problem(nx=J, x_lo=-4.0, x_hi=4.0, nv=N, v_max=L, collision=sgs.HARD_SPHERE,
                    bc_kind=(sgs.INFLOW, sgs.INFLOW), order=2, **bc, **kw)
    o = oracle.Problem(N=N, L=L, J=J, x_lo=-4.0, x_hi=4.0, kernel=oracle.HARD_SPHERE,
                       bc_kind=(oracle.INFLOW, oracle.INFLOW), order=2, **bc, **kw)
    f0 = I.ShockWorkload("t", J=J, N=N, L=L, eps=0.5, up=up, down=down, x_lo=-4.0, x_hi=4.0).initial_state()
    fo = f0.copy()
    s = sgs.Solver(g)
    f = dev(f0)
    Q, P = s.field(), s.field()
    for it in range(2):
        oracle.sgs_iteration(o, fo)
        s.iterate(f, Q, P, flags=sgs.IT_EVAL | (sgs.IT_P_VALID if it else 0))
    assert s.read_status()["status"] == 0
    assert rel(f.cpu().numpy().reshape(f0.shape), fo) <= 1e-12
