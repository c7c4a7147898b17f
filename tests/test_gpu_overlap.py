"""Pipelined SGS iterations (scans in 32-cell segments on the handle's own stream, the
collision step of each lane group as soon as the scan has left it, the groups evaluated
before the mass rescale carried over to the rescaled state) against the sequential order of
whole-grid steps and against the oracle. A ragged last group (70 cells: 32 + 32 + 6) and
both arithmetics; fixed inner counts so that both orders take the same decisions."""
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


def problem(precision, J=70):
    return sgs.Problem(nx=J, nv=8, v_max=6.0, eps=0.05, bc_T=(1.0, 1.7), total_mass=1.3, inner_fixed=5,
                       precision=precision)


def run(p, overlap, iters, f0, mixed=False):
    s = sgs.Solver(p)
    s.set_overlap(overlap)
    f = torch.from_numpy(f0.reshape(-1)).cuda()
    Q, P = s.field(), s.field()
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    rs = []
    if mixed:
        s.dc_step(f, Q, P, iters, res=res)
        s.dc_step(f, Q, P, 0, res=res)
        rs.append(res.item())
    else:
        for it in range(iters):
            s.iterate(f, Q, P, flags=sgs.IT_EVAL | (sgs.IT_P_VALID if it else 0), res=res)
            rs.append(res.item())
    st = s.read_status()
    return s, f.cpu().numpy().reshape(f0.shape), rs, st


def test_overlap_eligibility():
    s = sgs.Solver(problem(sgs.FP64))
    assert s.overlap()
    s.set_overlap(False)
    assert not s.overlap()
    assert not sgs.Solver(problem(sgs.FP64, J=32)).overlap()  # one lane group: nothing to pipeline


def test_pipelined_fp64_iterations_match_sequential_and_oracle(oracle):
    p = problem(sgs.FP64)
    f0 = I.initial_state(p.nx, p.nv, p.v_max, T=1.3, seed=31)
    s1, f1, r1, st1 = run(p, True, 3, f0)
    s0, f0g, r0, st0 = run(p, False, 3, f0)
    assert st1["status"] == 0 and st0["status"] == 0
    assert st1["visits"] == st0["visits"] == 3 * 2 * p.nx
    assert rel(f1, f0g) <= 1e-13
    for a, b in zip(r1, r0):
        assert abs(a - b) <= 1e-12 * r0[0]
    o = oracle.Problem(N=p.nv, L=p.v_max, J=p.nx, eps=p.eps, bc_T=tuple(p.bc_T), total_mass=p.total_mass,
                       inner_fixed=p.inner_fixed)
    fo = f0.copy()
    for _ in range(3):
        oracle.sgs_iteration(o, fo)
    assert rel(f1, fo) <= 1e-12
    assert abs(r1[-1] - oracle.solve_residual(o, fo)) <= 1e-12 * r0[0]


def test_pipelined_mixed_iterations_match_sequential():
    """Mixed precision: the groups evaluated before the rescale are scaled afterwards, while
    the sequential order evaluates the rescaled state; both are the same operator in exact
    arithmetic, and their FP32 increment sums round differently, so the iterates agree to the
    mixed form's resolution (it tracks FP64 iterates to about 2e-8), not to the last bit."""
    p = problem(sgs.FP32)
    f0 = I.initial_state(p.nx, p.nv, p.v_max, T=1.3, seed=32)
    _, f1, r1, st1 = run(p, True, 4, f0, mixed=True)
    _, f0g, r0, st0 = run(p, False, 4, f0, mixed=True)
    assert st1["status"] == 0 and st0["status"] == 0
    assert rel(f1, f0g) <= 5e-8
    assert abs(r1[-1] - r0[-1]) <= 1e-3 * r0[-1]
