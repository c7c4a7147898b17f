"""Device status bits, each provoked from the host with valid launches (no fault, no trap,
no unbounded wait): a cell solve stopped by a tiny inner_max sets INNER_CAP; a one-step
Newton cap sets NEWTON_FAIL in the collision step and in the scan, which then falls back to
the fixed-point step; a distribution with negative density sets NONPOSITIVE in the
collision step. Each case also checks that no unrelated bit is set and that the counters
still add up."""
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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).cuda()


@pytest.mark.parametrize("precision", [sgs.FP64, sgs.FP32])
def test_inner_cap_bit(precision):
    J, N, L = 5, 8, 6.0
    s = sgs.Solver(sgs.Problem(nx=J, nv=N, v_max=L, eps=0.01, inner_tol=1e-13, inner_max=1, precision=precision))
    f = dev(I.initial_state(J, N, L, T=1.5, seed=21))
    Q, P = s.field(), s.field()
    s.collide(f, Q, P)
    assert s.read_status()["status"] == 0
    s.sweep_forward(f, P)
    st = s.read_status()
    assert st["status"] == sgs.ST_INNER_CAP, st
    assert st["visits"] == J and st["inner_iters"] == J
    assert torch.isfinite(f).all()


def test_newton_fail_bit():
    J, N, L = 4, 8, 6.0
    s = sgs.Solver(sgs.Problem(nx=J, nv=N, v_max=L, eps=0.1, newton_max=1, inner_fixed=3))
    f = dev(I.initial_state(J, N, L, T=1.5, seed=22))
    Q, P = s.field(), s.field()
    s.collide(f, Q, P)
    # one Newton step from the continuum guess does not reach the discrete Maxwellian
    assert s.read_status()["status"] == sgs.ST_NEWTON_FAIL
    s.reset_stats()
    s.sweep_forward(f, P)
    st = s.read_status()
    assert st["status"] == sgs.ST_NEWTON_FAIL, st
    # failed step-1 solves fall back to the fixed-point step; the visit still completes
    assert st["visits"] == J and st["inner_iters"] == 3 * J and st["fallbacks"] >= 1
    assert torch.isfinite(f).all()


def test_nonpositive_bit():
    J, N, L = 3, 8, 6.0
    s = sgs.Solver(sgs.Problem(nx=J, nv=N, v_max=L))
    f0 = I.initial_state(J, N, L, T=1.5, seed=23)
    f0[1] *= -1.0  # cell 1 has negative density
    f = dev(f0)
    Q, P = s.field(), s.field()
    s.collide(f, Q, P)
    st = s.read_status()
    assert st["status"] & sgs.ST_NONPOSITIVE, st
    assert not st["status"] & (sgs.ST_NONFINITE | sgs.ST_INNER_CAP | sgs.ST_TIMEOUT), st
    # the other cells are untouched by the flag: their operator equals that of a clean run
    s2 = sgs.Solver(sgs.Problem(nx=1, nv=N, v_max=L))
    Q2, P2 = s2.field(), s2.field()
    s2.collide(dev(f0[0:1]), Q2, P2)
    q0, q1 = Q.view(J, -1)[0], Q2.view(1, -1)[0]
    assert ((q0 - q1).abs().max() <= 1e-14 * q1.abs().max()).item()
    assert s2.read_status()["status"] == 0
