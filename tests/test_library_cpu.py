"""Host-side checks of the C ABI (no GPU): the library builds and loads, exports every
function include/sgs.h declares, validates problems, and its closed-form Fourier weights
agree with the oracle's adaptive quadrature (two independent implementations)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2409_01910_gb300 import build, sgs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "sgs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sgs_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def L():
    return sgs.lib()


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_problem_validation_on_host(L):
    p = sgs.Problem()
    h = C.c_void_p()
    ws = C.c_size_t()
    arr = (sgs._Problem * 1)(p.c())
    assert L.sgs_setup(arr, 1, C.byref(h), C.byref(ws)) == sgs.OK
    assert ws.value > 0
    off, J, nv = C.c_size_t(), C.c_int(), C.c_int()
    assert L.sgs_layout(h, 0, C.byref(off), C.byref(J), C.byref(nv)) == sgs.OK
    assert (off.value, J.value, nv.value) == (0, p.nx, p.nv)
    assert L.sgs_field_elems(h) == p.nx * p.nv**3
    # compute calls before a workspace is bound are rejected on the host
    assert L.sgs_collide(h, None, None, None, None) == sgs.ERR_ARG
    assert L.sgs_rescale(h, C.c_void_p(16), None) == sgs.ERR_WORKSPACE
    L.sgs_destroy(h)
    for bad in (dict(nv=10), dict(nv=36), dict(eps=0.0), dict(nx=0), dict(x_hi=-1.0), dict(collision=7),
                dict(bc_T=(1.0, -1.0)), dict(precision=5), dict(newton_max=0), dict(conserve_proj=3), dict(inner_method=3)):
        q = sgs.Problem(**bad)
        arr = (sgs._Problem * 1)(q.c())
        assert L.sgs_setup(arr, 1, C.byref(h), C.byref(ws)) == sgs.ERR_ARG, bad
    # the second-order scheme: one order per handle, not in the no-allocation residual
    arr = (sgs._Problem * 1)(sgs.Problem(order=3).c())
    assert L.sgs_setup(arr, 1, C.byref(h), C.byref(ws)) == sgs.ERR_ARG
    arr = (sgs._Problem * 1)(sgs.Problem(space_dim=2, nx=4, ny=3, order=2).c())
    assert L.sgs_setup(arr, 1, C.byref(h), C.byref(ws)) == sgs.OK  # 2-D second order
    L.sgs_destroy(h)
    arr = (sgs._Problem * 2)(sgs.Problem().c(), sgs.Problem(order=2).c())
    assert L.sgs_setup(arr, 2, C.byref(h), C.byref(ws)) == sgs.ERR_UNSUPPORTED
    p2 = sgs.Problem(order=2).c()
    dummy = C.c_void_p(256)
    assert L.sgs_residual_noalloc(C.byref(p2), dummy, dummy, None, dummy, None) == sgs.ERR_UNSUPPORTED
    # the no-allocation residual refuses what sgs_setup refuses, with the same codes, before
    # any CUDA call (no GPU is needed to reach these returns)
    refused = (dict(bc_kind=(sgs.INFLOW, sgs.DIFFUSE), bc_rho=(0.0, 1.0)),
               dict(bc_u=((0.3, 0.0, 0.0), (0.0, 0.0, 0.0))), dict(nv=10), dict(eps=-1.0), dict(order=5),
               dict(space_dim=2, nx=4, ny=3), dict(nx=4097))
    for bad in refused:
        q = sgs.Problem(**bad)
        arr = (sgs._Problem * 1)(q.c())
        hq, wsq = C.c_void_p(), C.c_size_t()
        want = L.sgs_setup(arr, 1, C.byref(hq), C.byref(wsq))
        if want == sgs.OK:  # valid for a handle, outside what the no-allocation residual computes
            L.sgs_destroy(hq)
            want = sgs.ERR_ARG
        assert L.sgs_residual_noalloc(C.byref(q.c()), dummy, dummy, None, dummy, None) == want, bad
    # the conservation projection is a handle-wide choice; it enlarges the workspace
    arr = (sgs._Problem * 2)(sgs.Problem().c(), sgs.Problem(conserve_proj=1).c())
    assert L.sgs_setup(arr, 2, C.byref(h), C.byref(ws)) == sgs.ERR_UNSUPPORTED
    arr = (sgs._Problem * 1)(sgs.Problem(conserve_proj=1).c())
    ws1 = C.c_size_t()
    assert L.sgs_setup(arr, 1, C.byref(h), C.byref(ws1)) == sgs.OK and ws1.value > ws.value
    L.sgs_destroy(h)
    q = sgs.Problem(space_dim=3)
    arr = (sgs._Problem * 1)(q.c())
    assert L.sgs_setup(arr, 1, C.byref(h), C.byref(ws)) == sgs.ERR_ARG
    # 2-D: one instance per handle; y extent and y walls validated
    q2 = sgs.Problem(space_dim=2, nx=4, ny=3)
    arr = (sgs._Problem * 2)(q2.c(), q2.c())
    assert L.sgs_setup(arr, 2, C.byref(h), C.byref(ws)) == sgs.ERR_UNSUPPORTED
    for bad in (dict(ny=0), dict(y_hi=-1.0), dict(bc_T_y=(1.0, 0.0))):
        arr = (sgs._Problem * 1)(sgs.Problem(**{"space_dim": 2, "nx": 4, "ny": 3, **bad}).c())
        assert L.sgs_setup(arr, 1, C.byref(h), C.byref(ws)) == sgs.ERR_ARG, bad
    arr = (sgs._Problem * 1)(sgs.Problem(space_dim=2, nx=4, ny=3, bc_u_y=((0, 0, 0), (0, 0.2, 0))).c())
    assert L.sgs_setup(arr, 1, C.byref(h), C.byref(ws)) == sgs.ERR_UNSUPPORTED  # normal wall velocity
    arr = (sgs._Problem * 1)(sgs.Problem(space_dim=2, nx=4, ny=3).c())
    assert L.sgs_setup(arr, 1, C.byref(h), C.byref(ws)) == sgs.OK
    off, J, nv = C.c_size_t(), C.c_int(), C.c_int()
    assert L.sgs_layout(h, 0, C.byref(off), C.byref(J), C.byref(nv)) == sgs.OK and J.value == 12
    L.sgs_destroy(h)
    assert L.sgs_strerror(sgs.ERR_WORKSPACE).decode().startswith("workspace")


def test_multi_instance_layout(L):
    ps = [sgs.Problem(nx=J) for J in (3, 7, 5)]
    arr = (sgs._Problem * 3)(*[p.c() for p in ps])
    h, ws = C.c_void_p(), C.c_size_t()
    assert L.sgs_setup(arr, 3, C.byref(h), C.byref(ws)) == sgs.OK
    K = 16**3
    offs = []
    for q in range(3):
        off, J, nv = C.c_size_t(), C.c_int(), C.c_int()
        L.sgs_layout(h, q, C.byref(off), C.byref(J), C.byref(nv))
        offs.append(off.value)
    assert offs == [0, 3 * K, 10 * K]
    assert L.sgs_field_elems(h) == 15 * K
    L.sgs_destroy(h)


@pytest.mark.parametrize("kernel,L_", [(0, 6.0), (0, 8.0), (1, 10.0)])
def test_closed_form_weights_match_oracle_quadrature(oracle, kernel, L_):
    N = 32
    h = N // 2 - 1
    b0 = 1.0 / (4 * np.pi)
    scale = abs(oracle.G(N, L_, kernel, b0, 0, 0))
    rng = np.random.default_rng(11)
    pairs = [(0, 0), (0, 1), (1, 0), (4, 4), (675, 2700), (12 * h * h, 0), (1, 2700), (674, 675)]
    pairs += [(int(rng.integers(0, 3 * h * h + 1)), int(rng.integers(0, 12 * h * h + 1))) for _ in range(40)]
    for a2, b2 in pairs:
        g = sgs.host_weight(N, L_, kernel, b0, a2, b2)
        assert abs(g - oracle.G(N, L_, kernel, b0, a2, b2)) <= 2e-14 * scale, (a2, b2)


def test_batch_api_on_host(L):
    """Batch and tuning entry points: host-side validation and the default scan shape."""
    ps = [sgs.Problem(nx=J, nv=16) for J in (4, 9)]
    arr = (sgs._Problem * 2)(*[p.c() for p in ps])
    h, ws = C.c_void_p(), C.c_size_t()
    assert L.sgs_setup(arr, 2, C.byref(h), C.byref(ws)) == sgs.OK
    e, c, t = C.c_int(), C.c_int(), C.c_int()
    assert L.sgs_get_sweep_shape(h, C.byref(e), C.byref(c), C.byref(t)) == sgs.OK
    # every node of a cell has an owner thread; warps 0-4 exist for the Newton evaluations
    assert 16 % e.value == 0 and c.value in (1, 2, 4, 8, 16) and 160 <= t.value <= 256 and t.value % 32 == 0
    assert e.value * c.value * t.value >= 16**3
    assert L.sgs_get_sweep_shape(h, None, C.byref(c), C.byref(t)) == sgs.ERR_ARG
    # nothing is enqueued before a workspace is bound
    assert L.sgs_update_active(h, C.c_void_p(16), 1e-8, None) == sgs.ERR_WORKSPACE
    assert L.sgs_update_active(h, C.c_void_p(16), -1.0, None) == sgs.ERR_ARG
    assert L.sgs_activate_all(h, None) == sgs.ERR_WORKSPACE
    assert L.sgs_autotune(h, C.c_void_p(16), C.c_void_p(16), 1, None, None) == sgs.ERR_WORKSPACE
    assert L.sgs_autotune(h, C.c_void_p(16), C.c_void_p(16), 0, None, None) == sgs.ERR_ARG
    # shapes that leave nodes without an owner, or break the cluster/thread rules
    for bad in ((3, 4, 256), (8, 3, 256), (8, 16, 100), (4, 1, 256), (8, 32, 128)):
        assert L.sgs_set_sweep_shape(h, *bad) == sgs.ERR_ARG, bad
    L.sgs_destroy(h)


def test_batch_inputs_follow_their_distributions():
    from paper_2409_01910_gb300 import inputs as I

    b = I.heat_batch(64, seed=0)
    assert len(b) == 64
    assert all(32 <= w.J <= 256 and w.N in (24, 32) and 1e-3 <= w.eps <= 1.0 for w in b)
    assert all(0.8 <= w.T_left <= 1.2 and 1.5 <= w.T_right <= 2.5 and w.L == 8.0 for w in b)
    assert {w.N for w in b} == {24, 32}
    # log-uniform eps: about half the instances below sqrt(1e-3)
    below = sum(w.eps < 10**-1.5 for w in b)
    assert 16 <= below <= 48
    # reproducible, and distinct seeds per instance
    b2 = I.heat_batch(64, seed=0)
    assert [(w.J, w.N, w.eps) for w in b] == [(w.J, w.N, w.eps) for w in b2]
    assert len({w.seed for w in b}) == 64


def test_fast_operator_and_macroscopic_on_host(L):
    """Host-side validation of the fast operator's entry points and of sgs_macroscopic (no
    device work is reached): hard spheres only, rule sizes, workspace growing with the chunk
    of nodes, calls before binding refused."""
    hs = sgs.Problem(nx=4, nv=16, v_max=8.0, collision=sgs.HARD_SPHERE, eps=0.1)
    arr = (sgs._Problem * 1)(hs.c())
    h, ws = C.c_void_p(), C.c_size_t()
    assert L.sgs_setup(arr, 1, C.byref(h), C.byref(ws)) == sgs.OK
    x, xb = C.c_void_p(), C.c_size_t()
    assert L.sgs_fast_setup(h, 8, 16, 4, C.byref(x), C.byref(xb)) == sgs.OK and xb.value > 0
    x8, xb8 = C.c_void_p(), C.c_size_t()
    assert L.sgs_fast_setup(h, 8, 16, 8, C.byref(x8), C.byref(xb8)) == sgs.OK and xb8.value > xb.value
    L.sgs_fast_destroy(x8)
    dummy = C.c_void_p(256)
    assert L.sgs_fast_collide(x, h, dummy, dummy, 3, None) == sgs.ERR_WORKSPACE  # nothing bound
    assert L.sgs_fast_collide(x, h, dummy, dummy, 2, None) == sgs.ERR_ARG  # 1 or 3 products
    assert L.sgs_fast_bind(x, C.c_void_p(256), 16) == sgs.ERR_WORKSPACE  # too small
    L.sgs_fast_destroy(x)
    for bad in ((0, 16, 4), (8, 0, 4), (8, 16, 0), (64, 65, 4)):
        y = C.c_void_p()
        assert L.sgs_fast_setup(h, *bad, C.byref(y), C.byref(xb)) == sgs.ERR_ARG, bad
    assert L.sgs_macroscopic(h, dummy, dummy, None) == sgs.ERR_WORKSPACE
    assert L.sgs_macroscopic(h, None, dummy, None) == sgs.ERR_ARG
    L.sgs_destroy(h)
    mx = (sgs._Problem * 1)(sgs.Problem(nx=4, nv=16).c())
    assert L.sgs_setup(mx, 1, C.byref(h), C.byref(ws)) == sgs.OK
    y = C.c_void_p()
    assert L.sgs_fast_setup(h, 8, 16, 4, C.byref(y), C.byref(xb)) == sgs.ERR_UNSUPPORTED  # Maxwell molecules
    L.sgs_destroy(h)
