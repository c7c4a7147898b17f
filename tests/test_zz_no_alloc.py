"""The allocation-free residual entry point against the workspace-based one.

sgs_residual_noalloc serves callers that cannot allocate device memory: it keeps its
scratch in a static device array of the library instead of a caller-bound workspace. This
file is collected last so that a run stopping at the first failure has run every other test.
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


def test_noalloc_residual_matches_workspace_residual():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fn = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [sgs.Problem(nx=16, nv=16, v_max=6.0, eps=1.0, bc_T=(1.0, 2.0)),
             sgs.Problem(nx=9, nv=8, v_max=6.0, eps=0.05, bc_T=(1.3, 0.8))]
    for p in cases:  # two calls in a row, different sizes: the static scratch is reused
        s = sgs.Solver(p)
        f = torch.from_numpy(I.initial_state(p.nx, p.nv, p.v_max, T=1.4, seed=p.nx).reshape(-1)).cuda()
        Q, P = s.field(), s.field()
        s.collide(f, Q, P)
        ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        s.residual(f, Q, ref)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        pc = p.c()
        assert fn(C.byref(pc), f.data_ptr(), Q.data_ptr(), None, out.data_ptr(), stream) == sgs.OK
        torch.cuda.synchronize()
        assert abs(out.item() - ref.item()) <= 1e-12 * ref.item(), (out.item(), ref.item())
        # a second call on the same data reproduces the value bit for bit
        out2 = torch.zeros(1, dtype=torch.float64, device="cuda")
        assert fn(C.byref(pc), f.data_ptr(), Q.data_ptr(), None, out2.data_ptr(), stream) == sgs.OK
        torch.cuda.synchronize()
        assert out2.item() == out.item()
    # sizes beyond the static capacity are refused on the host, before any launch
    big = sgs.Problem(nx=5000, nv=8, v_max=6.0).c()
    assert fn(C.byref(big), f.data_ptr(), Q.data_ptr(), None, out.data_ptr(), stream) == sgs.ERR_ARG
