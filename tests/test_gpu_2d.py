"""GPU parity in 2-D space (lid-driven cavity layout: four diffuse walls, moving lid) against
the oracle: single orderings, one full SGS iteration (four orderings, rescale), the outer
residual and the 2 x 2 FAS V-cycle, all at 1e-12 in FP64 with a fixed inner count; the
mixed-precision form tracks the FP64 iteration."""
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


def cavity(oracle, nx=4, ny=3, N=8, L=6.0, eps=0.5, inner_fixed=4, precision=sgs.FP64, total_mass=1.0,
           inner_tol=1e-8, order=1, collision=sgs.MAXWELL, b0=1.0 / (4 * np.pi)):
    Tx, Ty, lid = (1.0, 1.2), (1.1, 1.0), (0.3, 0.0, 0.0)
    g = sgs.Problem(space_dim=2, nx=nx, ny=ny, nv=N, v_max=L, eps=eps, bc_T=Tx, bc_T_y=Ty,
                    bc_u_y=((0.0, 0.0, 0.0), lid), total_mass=total_mass, inner_fixed=inner_fixed,
                    precision=precision, inner_tol=inner_tol, order=order, collision=collision, b0=b0)
    base = oracle.Problem(N=N, L=L, J=nx, eps=eps, bc_T=Tx, total_mass=total_mass, inner_fixed=inner_fixed,
                          inner_tol=inner_tol, order=order, kernel=collision, b0=b0)
    o = oracle.Problem2D(base=base, ny=ny, bc_T_y=Ty, bc_u_y=((0.0, 0.0, 0.0), lid))
    f0 = I.initial_state(nx * ny, N, L, T=1.1, seed=6)
    return g, o, f0


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).cuda()


@pytest.mark.parametrize("ordering", [0, 1, 2, 3])
def test_single_ordering_parity(oracle, ordering):
    g, o, f0 = cavity(oracle)
    Qo, Po, nuo = oracle.collide2d(o, f0)
    fo = f0.copy()
    oracle.sweep2d(o, fo, Po, nuo, ordering)
    s = sgs.Solver(g)
    f = dev(f0)
    Q, P = s.field(), s.field()
    s.collide(f, Q, P)  # device collision frequencies and Maxwellians of f0
    s.sweep_ordering(f, dev(Po), ordering)
    st = s.read_status()
    assert st["status"] == 0 and st["visits"] == 12 and st["inner_iters"] == 4 * 12
    assert rel(f.cpu().numpy().reshape(f0.shape), fo) <= 1e-12


def test_sgs_iteration_and_residual_parity(oracle):
    g, o, f0 = cavity(oracle)
    fo = f0.copy()
    oracle.sgs_iteration2d(o, fo)
    Qo, _, _ = oracle.collide2d(o, fo)
    res_o = oracle.residual2d(o, fo, Qo)
    s = sgs.Solver(g)
    f = dev(f0)
    Q, P = s.field(), s.field()
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.iterate(f, Q, P, flags=sgs.IT_EVAL, res=res)
    assert s.read_status()["status"] == 0
    assert rel(f.cpu().numpy().reshape(f0.shape), fo) <= 1e-12
    assert abs(res.item() - res_o) <= 1e-11 * res_o


def test_vcycle_parity(oracle):
    g, o, f0 = cavity(oracle, nx=4, ny=4)
    fo = f0.copy()
    oracle.vcycle2d(o, fo, 2, 1, 1, 2)
    s = sgs.Solver(g)
    assert s.max_levels() == 3
    f = dev(f0)
    s.vcycle(f, 2, 1, 1, 2)
    assert s.read_status()["status"] == 0
    assert rel(f.cpu().numpy().reshape(f0.shape), fo) <= 1e-12


def test_mixed_2d_tracks_fp64(oracle):
    """Mixed precision in 2-D (FP32 sums in increment form, double-float scans,
    double-float defect-correction evaluations) after the same iterations as FP64."""
    g64, o, f0 = cavity(oracle, nx=4, ny=4, inner_fixed=0, inner_tol=1e-11)
    s64 = sgs.Solver(g64)
    f64 = dev(f0)
    Q, P = s64.field(), s64.field()
    for it in range(12):
        s64.iterate(f64, Q, P, flags=sgs.IT_EVAL | (sgs.IT_P_VALID if it else 0))
    g32, _, _ = cavity(oracle, nx=4, ny=4, inner_fixed=0, inner_tol=1e-11, precision=sgs.FP32)
    s32 = sgs.Solver(g32)
    f32 = dev(f0)
    Q2, P2 = s32.field(), s32.field()
    for k in range(3):
        s32.dc_step(f32, Q2, P2, 4)
    assert s64.read_status()["status"] == 0 and s32.read_status()["status"] == 0
    assert rel(f32.cpu().numpy(), f64.cpu().numpy()) <= 2e-8


# ----------------------------------------------------------------------------- second order
@pytest.mark.parametrize("precision,tol", [(sgs.FP64, 1e-12), (sgs.FP32, 1e-11)])
@pytest.mark.parametrize("ordering", [0, 1, 2, 3])
def test_second_order_ordering_parity(oracle, ordering, precision, tol):
    """Second order in 2-D space (slopes of eq. (slope) along x and y, explicit in the
    ordering, face-value wall ghosts): one ordering against the oracle, FP64 and double-float
    scans; a 4 x 3 grid with a moving lid, fixed inner count."""
    g, o, f0 = cavity(oracle, order=2, precision=precision)
    Qo, Po, nuo = oracle.collide2d(o, f0)
    fo = f0.copy()
    oracle.sweep2d(o, fo, Po, nuo, ordering)
    s = sgs.Solver(g)
    f = dev(f0)
    Q, P = s.field(), s.field()
    s.collide(f, Q, P)
    s.sweep_ordering(f, dev(Po), ordering)
    st = s.read_status()
    assert st["status"] == 0 and st["visits"] == 12
    assert rel(f.cpu().numpy().reshape(f0.shape), fo) <= tol


def test_second_order_iteration_and_residual_parity(oracle):
    g, o, f0 = cavity(oracle, order=2)
    Q0, _, _ = oracle.collide2d(o, f0)
    res0 = oracle.residual2d(o, f0, Q0)
    fo = f0.copy()
    for _ in range(2):
        oracle.sgs_iteration2d(o, fo)
    Qo, _, _ = oracle.collide2d(o, fo)
    res_o = oracle.residual2d(o, fo, Qo)
    s = sgs.Solver(g)
    f = dev(f0)
    Q, P = s.field(), s.field()
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.collide(f, Q, P)
    s.residual(f, Q, res)
    assert abs(res.item() - res0) <= 1e-12 * res0
    for it in range(2):
        s.iterate(f, Q, P, flags=sgs.IT_EVAL | (sgs.IT_P_VALID if it else 0), res=res)
    assert s.read_status()["status"] == 0
    assert rel(f.cpu().numpy().reshape(f0.shape), fo) <= 1e-12
    assert abs(res.item() - res_o) <= 1e-11 * res0


def test_second_order_vcycle_with_the_papers_parameters(oracle):
    """The paper's second-order multigrid parameters (5 pre-smoothing, 1 post-smoothing
    iteration) on an 8 x 8 grid down to 4 x 4, against the oracle's V-cycle."""
    g, o, f0 = cavity(oracle, nx=8, ny=8, order=2, inner_fixed=3)
    fo = f0.copy()
    oracle.vcycle2d(o, fo, 2, 5, 1, 2)
    s = sgs.Solver(g)
    f = dev(f0)
    s.vcycle(f, 2, 5, 1, 2)
    assert s.read_status()["status"] == 0
    assert rel(f.cpu().numpy().reshape(f0.shape), fo) <= 1e-12


@pytest.mark.parametrize("order", [1, 2])
def test_bgk_2d_iterations_and_residual_parity(oracle, order):
    """The BGK operator (P = 0, nu = 4 pi b0 rho with b0 = 1, the paper's 2-D BGK example) in
    2-D space at first and second order: two SGS iterations and the residual against the
    oracle."""
    g, o, f0 = cavity(oracle, order=order, collision=sgs.BGK, b0=1.0, eps=0.1)
    Q0, _, _ = oracle.collide2d(o, f0)
    r0 = oracle.residual2d(o, f0, Q0)  # the residual is a difference of O(r0) terms: compare on that scale
    fo = f0.copy()
    for _ in range(2):
        oracle.sgs_iteration2d(o, fo)
    Qo, _, _ = oracle.collide2d(o, fo)
    res_o = oracle.residual2d(o, fo, Qo)
    s = sgs.Solver(g)
    f = dev(f0)
    Q, P = s.field(), s.field()
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    for it in range(2):
        s.iterate(f, Q, P, flags=sgs.IT_EVAL | (sgs.IT_P_VALID if it else 0), res=res)
    assert s.read_status()["status"] == 0
    assert rel(f.cpu().numpy().reshape(f0.shape), fo) <= 1e-12
    assert abs(res.item() - res_o) <= 1e-11 * r0
