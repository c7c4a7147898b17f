"""GPU parity of the source iteration (eq. (SI), the collision term split by the BGK
penalty of eq. (28) and lagged) against the oracle: three iterations (collision step,
per-node transport march, mass rescale) from the same state, diffuse walls (Maxwell
molecules and BGK) and inflow sides (hard spheres): 1e-12 with FP64 collision sums,
1e-5 with the FP32 sums of the mixed form."""
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


def case(oracle, kind, precision):
    N, J, L = 8, 6, 6.0
    if kind == "inflow":
        up, down = I.rankine_hugoniot(2.0)
        bc = dict(bc_rho=(up[0], down[0]), bc_u=((up[1], 0.0, 0.0), (down[1], 0.0, 0.0)), bc_T=(up[2], down[2]),
                  total_mass=0.0)
        g = sgs.Problem(nx=J, x_lo=-4.0, x_hi=4.0, nv=N, v_max=L, eps=0.5, collision=sgs.HARD_SPHERE,
                        bc_kind=(sgs.INFLOW, sgs.INFLOW), precision=precision, **bc)
        o = oracle.Problem(N=N, L=L, J=J, x_lo=-4.0, x_hi=4.0, eps=0.5, kernel=oracle.HARD_SPHERE,
                           bc_kind=(oracle.INFLOW, oracle.INFLOW), **bc)
        f0 = I.ShockWorkload("t", J=J, N=N, L=L, eps=0.5, up=up, down=down, x_lo=-4.0, x_hi=4.0).initial_state()
        return g, o, f0
    kernel = sgs.BGK if kind == "bgk" else sgs.MAXWELL
    g = sgs.Problem(nx=J, nv=N, v_max=L, eps=0.3, collision=kernel, bc_T=(1.0, 1.6), total_mass=1.0,
                    precision=precision)
    o = oracle.Problem(N=N, L=L, J=J, eps=0.3, kernel=kernel, bc_T=(1.0, 1.6), total_mass=1.0)
    return g, o, I.initial_state(J, N, L, T=1.3, seed=31)


@pytest.mark.parametrize("kind,precision,tol", [("maxwell", sgs.FP64, 1e-12), ("bgk", sgs.FP64, 1e-12),
                                                ("inflow", sgs.FP64, 1e-12), ("maxwell", sgs.FP32, 1e-5)])
def test_source_iterations_parity(oracle, kind, precision, tol):
    g, o, f0 = case(oracle, kind, precision)
    fo = f0.copy()
    s = sgs.Solver(g)
    f = torch.from_numpy(f0.reshape(-1)).cuda()
    P = s.field()
    for _ in range(3):
        oracle.si_iteration(o, fo)
        s.si_iteration(f, P)
    assert s.read_status()["status"] == 0
    assert rel(f.cpu().numpy().reshape(f0.shape), fo) <= tol


def test_source_iteration_rejects_2d():
    s = sgs.Solver(sgs.Problem(space_dim=2, nx=2, ny=2, nv=8))
    f, P = s.field(), s.field()
    with pytest.raises(Exception):
        s.si_iteration(f, P)
