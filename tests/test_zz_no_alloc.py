"""The allocation-free residual entry point against the workspace-based one and the oracle.

sgs_residual_noalloc serves callers that cannot allocate device memory: it keeps its
scratch in a static device array of the library instead of a caller-bound workspace. This
file is collected last so that a run stopping at the first failure has run every other test.
Cases: diffuse walls without a right-hand side, and inflow sides with a right-hand side b
(the form multigrid and defect correction use), each called twice in a row on the shared
scratch; the value must equal sgs_residual's to 1e-12 and the oracle's residual of the same
f, Q and b to 1e-12.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2409_01910_gb300 import inputs as I
from paper_2409_01910_gb300 import sgs

pytestmark = pytest.mark.gpu


def _entry():
    fn = sgs.lib().sgs_residual_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.POINTER(sgs._Problem), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return fn


def _cases(oracle):
    up, down = I.rankine_hugoniot(1.4)
    inflow = dict(bc_kind=(sgs.INFLOW, sgs.INFLOW), bc_rho=(up[0], down[0]),
                  bc_u=((up[1], 0.0, 0.0), (down[1], 0.0, 0.0)), bc_T=(up[2], down[2]), total_mass=0.0)
    out = []
    for kw, with_rhs in ((dict(nx=16, nv=16, v_max=6.0, eps=1.0, bc_T=(1.0, 2.0)), False),
                         (dict(nx=9, nv=8, v_max=6.0, eps=0.05, bc_T=(1.3, 0.8)), False),
                         (dict(nx=7, nv=8, v_max=8.0, eps=0.3, x_lo=-2.0, x_hi=2.0, **inflow), True)):
        g = sgs.Problem(**kw)
        o = oracle.Problem(N=g.nv, L=g.v_max, J=g.nx, x_lo=g.x_lo, x_hi=g.x_hi, eps=g.eps, bc_kind=tuple(g.bc_kind),
                           bc_rho=tuple(g.bc_rho), bc_u=tuple(tuple(u) for u in g.bc_u), bc_T=tuple(g.bc_T),
                           total_mass=g.total_mass)
        out.append((g, o, with_rhs))
    return out


def test_noalloc_residual_matches_workspace_residual_and_oracle(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fn = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    for p, o, with_rhs in _cases(oracle):  # two calls in a row per case, different sizes: the scratch is reused
        s = sgs.Solver(p)
        f0 = I.initial_state(p.nx, p.nv, p.v_max, T=1.4, seed=p.nx)
        f = torch.from_numpy(f0.reshape(-1)).cuda()
        Q, P = s.field(), s.field()
        s.collide(f, Q, P)
        b0 = 0.1 * np.random.default_rng(p.nx).standard_normal(f0.shape) if with_rhs else None
        rhs = torch.from_numpy(b0.reshape(-1)).cuda() if with_rhs else None
        ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        s.residual(f, Q, ref, rhs=rhs)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        pc = p.c()
        rp = rhs.data_ptr() if with_rhs else None
        assert fn(C.byref(pc), f.data_ptr(), Q.data_ptr(), rp, out.data_ptr(), stream) == sgs.OK
        torch.cuda.synchronize()
        assert abs(out.item() - ref.item()) <= 1e-12 * ref.item(), (out.item(), ref.item())
        ro = oracle.residual(o, f0, Q.cpu().numpy().reshape(f0.shape), b=b0)
        assert abs(out.item() - ro) <= 1e-12 * ro, (out.item(), ro)
        # a second call on the same data reproduces the value bit for bit
        out2 = torch.zeros(1, dtype=torch.float64, device="cuda")
        assert fn(C.byref(pc), f.data_ptr(), Q.data_ptr(), rp, out2.data_ptr(), stream) == sgs.OK
        torch.cuda.synchronize()
        assert out2.item() == out.item()
    # sizes beyond the static capacity are refused on the host, before any launch
    big = sgs.Problem(nx=5000, nv=8, v_max=6.0).c()
    assert fn(C.byref(big), f.data_ptr(), Q.data_ptr(), None, out.data_ptr(), stream) == sgs.ERR_ARG
