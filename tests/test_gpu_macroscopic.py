"""Macroscopic quantities and the heat flux of Section 4.2.2 on the GPU against the oracle,
cell by cell: a multi-instance handle of uneven cell counts (the last instance's cells carry
a Grad-type heat-flux perturbation, so q is far from zero), a 2-D handle, and a state
produced by the solver itself."""
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


def grad_cells(J, N, L, seed):
    rng = np.random.default_rng(seed)
    v = (np.arange(N) - N // 2 + 1) * (2 * L / N)
    out = []
    for _ in range(J):
        rho, T = rng.uniform(0.5, 1.5), rng.uniform(0.7, 1.6)
        U, q = rng.uniform(-0.4, 0.4, 3), rng.uniform(-0.05, 0.05, 3)
        c = [v[:, None, None] - U[0], v[None, :, None] - U[1], v[None, None, :] - U[2]]
        c2 = c[0] ** 2 + c[1] ** 2 + c[2] ** 2
        M = rho / (2 * np.pi * T) ** 1.5 * np.exp(-c2 / (2 * T))
        qc = q[0] * c[0] + q[1] * c[1] + q[2] * c[2]
        out.append(M * (1 + 2 * qc / (5 * rho * T * T) * (c2 / (2 * T) - 2.5)))
    return np.stack(out)


def check(oracle, f_host, out, L, N):
    f_host = f_host.reshape(-1, N, N, N)
    got = out.cpu().numpy()
    assert got.shape == (f_host.shape[0], 8)
    for c in range(f_host.shape[0]):
        want = oracle.macroscopic(np.ascontiguousarray(f_host[c]), L)
        assert np.abs(got[c] - want).max() <= 1e-12 * max(1.0, np.abs(want).max()), (c, got[c], want)


def test_multi_instance_handle_matches_oracle(oracle):
    N, L = 16, 8.0
    ps = [sgs.Problem(nx=J, nv=N, v_max=L, eps=0.1) for J in (3, 7, 5)]
    s = sgs.Solver(ps)
    f0 = np.concatenate([I.initial_state(3, N, L, T=1.3, seed=5).reshape(-1),
                         I.initial_state(7, N, L, T=0.9, seed=6).reshape(-1),
                         grad_cells(5, N, L, seed=7).reshape(-1)])
    f = torch.from_numpy(f0).cuda()
    out = s.macroscopic(f)
    check(oracle, f0, out, L, N)
    # the Grad cells have a heat flux of the size they were built with
    assert np.abs(out[10:, 5:8].cpu().numpy()).max() > 1e-2


def test_2d_handle_and_solver_state_match_oracle(oracle):
    N, L = 16, 6.0
    p = sgs.Problem(space_dim=2, nx=4, ny=3, nv=N, v_max=L, eps=0.5, bc_u_y=((0, 0, 0), (0.3, 0, 0)))
    s = sgs.Solver(p)
    f0 = I.initial_state(12, N, L, T=1.0, seed=9).reshape(-1)
    f = torch.from_numpy(f0.copy()).cuda()
    Q, P = s.field(), s.field()
    for it in range(2):
        s.iterate(f, Q, P, flags=sgs.IT_P_VALID if it else 0)
    torch.cuda.synchronize()
    check(oracle, f.cpu().numpy(), s.macroscopic(f), L, N)
