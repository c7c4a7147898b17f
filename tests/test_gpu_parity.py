"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances: relative L-infinity max|a - b| / max|b| of 1e-12 for FP64 arithmetic; 1e-5 on Q
for the FP32 collision sum. Oracle inputs never come from the CUDA path: P and nu fed to
both sweeps are the oracle's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2409_01910_gb300 import inputs as I
from paper_2409_01910_gb300 import sgs

pytestmark = pytest.mark.gpu

B0 = 1.0 / (4 * np.pi)


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sgs.lib()


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def spec(**kw):
    """One problem description for both sides."""
    d = dict(nx=8, nv=8, v_max=6.0, eps=1.0, T=(1.0, 2.0), collision=0, total_mass=1.0, inner_tol=1e-8,
             inner_max=200, inner_fixed=0, precision=sgs.FP64, inner_method=sgs.PFP)
    d.update(kw)
    return d


def gpu_problem(d):
    return sgs.Problem(nx=d["nx"], nv=d["nv"], v_max=d["v_max"], eps=d["eps"], bc_T=d["T"], collision=d["collision"],
                       total_mass=d["total_mass"], inner_tol=d["inner_tol"], inner_max=d["inner_max"],
                       inner_fixed=d["inner_fixed"], precision=d["precision"], inner_method=d["inner_method"])


def oracle_problem(O, d):
    return O.Problem(N=d["nv"], L=d["v_max"], J=d["nx"], eps=d["eps"], bc_T=d["T"], kernel=d["collision"],
                     total_mass=d["total_mass"], inner_tol=d["inner_tol"], inner_max=d["inner_max"],
                     inner_fixed=d["inner_fixed"], inner_method=d["inner_method"])


def varied_state(J, N, L, seed=0):
    """Cells far from equilibrium: two-Maxwellian mixtures with cell-dependent shifts."""
    rng = np.random.default_rng(seed)
    f = np.empty((J, N, N, N))
    for j in range(J):
        u = rng.uniform(-0.6, 0.6, 3)
        f[j] = I.sampled_maxwellian(N, L, rng.uniform(0.5, 1.5), u, rng.uniform(0.6, 1.6))
        f[j] += I.sampled_maxwellian(N, L, rng.uniform(0.2, 0.6), -u, rng.uniform(0.4, 1.0))
        f[j] *= 1 + 0.02 * rng.uniform(-1, 1, (N, N, N))
    return f


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).cuda()


@pytest.mark.parametrize("N,J,L", [(8, 40, 6.0), (16, 16, 6.0), (12, 3, 6.0)])
def test_collide_fp64_parity(oracle, N, J, L):
    d = spec(nx=J, nv=N, v_max=L)
    f = varied_state(J, N, L)
    s = sgs.Solver(gpu_problem(d))
    fd = to_dev(f)
    Q, P = s.field(), s.field()
    s.collide(fd, Q, P)
    torch.cuda.synchronize()
    Qo, Po, nuo = oracle.collide(oracle_problem(oracle, d), f)
    assert rel(Q.cpu().numpy().reshape(f.shape), Qo) <= 1e-12
    assert rel(P.cpu().numpy().reshape(f.shape), Po) <= 1e-12
    assert s.read_status()["status"] == 0


def test_collide_fp64_parity_full_size_sampled(oracle):
    """64 cells on the 32^3 grid (the eps = 0.01 heat-transfer size); two sampled cells."""
    N, J, L = 32, 64, 8.0
    d = spec(nx=J, nv=N, v_max=L, eps=0.01)
    f = varied_state(J, N, L, seed=3)
    s = sgs.Solver(gpu_problem(d))
    Q, P = s.field(), s.field()
    s.collide(to_dev(f), Q, P)
    Qg = Q.cpu().numpy().reshape(f.shape)
    po = oracle_problem(oracle, d)
    for j in (0, J - 1):
        Qo, Po, nu, th = oracle.collide_cell(po, f[j])
        assert rel(Qg[j], Qo) <= 1e-12, j


@pytest.mark.parametrize("N,J,L", [(8, 40, 6.0), (16, 16, 6.0)])
def test_collide_fp32_within_tolerance(oracle, N, J, L):
    d = spec(nx=J, nv=N, v_max=L, precision=sgs.FP32)
    f = varied_state(J, N, L, seed=1)
    s = sgs.Solver(gpu_problem(d))
    Q, P = s.field(), s.field()
    s.collide(to_dev(f), Q, P)
    Q64 = s.field()
    s.collide(to_dev(f), Q64, None, precision=sgs.FP64)
    Qo, Po, nuo = oracle.collide(oracle_problem(oracle, d), f)
    assert rel(Q.cpu().numpy().reshape(f.shape), Qo) <= 1e-5
    assert rel(Q64.cpu().numpy().reshape(f.shape), Qo) <= 1e-12


def test_bgk_mode_parity(oracle):
    N, J, L = 8, 5, 6.0
    d = spec(nx=J, nv=N, v_max=L, collision=2)
    f = varied_state(J, N, L, seed=2)
    s = sgs.Solver(gpu_problem(d))
    Q, P = s.field(), s.field()
    s.collide(to_dev(f), Q, P)
    Qo, Po, nuo = oracle.collide(oracle_problem(oracle, d), f)
    assert rel(Q.cpu().numpy().reshape(f.shape), Qo) <= 1e-12
    assert torch.count_nonzero(P).item() == 0


@pytest.mark.parametrize("N,J,eps,direction", [(8, 6, 1.0, 1), (8, 6, 0.01, -1), (16, 4, 0.1, 1)])
def test_sweep_parity_fixed_inner_count(oracle, N, J, eps, direction):
    L = 6.0
    d = spec(nx=J, nv=N, v_max=L, eps=eps, inner_fixed=6)
    f0 = I.initial_state(J, N, L, T=1.5, seed=4)
    po = oracle_problem(oracle, d)
    Qo, Po, nuo = oracle.collide(po, f0)
    fo = f0.copy()
    oracle.sweep(po, fo, Po, nuo, direction)
    s = sgs.Solver(gpu_problem(d))
    fd = to_dev(f0)
    Q, P = s.field(), s.field()
    s.collide(fd, Q, P)  # sets the device collision frequencies of f0
    Pd = to_dev(Po)
    if direction > 0:
        s.sweep_forward(fd, Pd)
    else:
        s.sweep_backward(fd, Pd)
    st = s.read_status()
    assert st["status"] == 0
    assert st["visits"] == J and st["inner_iters"] == 6 * J
    assert rel(fd.cpu().numpy().reshape(f0.shape), fo) <= 1e-12


def test_sweep_tolerance_mode_agrees(oracle):
    N, J, L = 8, 6, 6.0
    d = spec(nx=J, nv=N, v_max=L, eps=0.05, inner_tol=1e-11)
    f0 = I.initial_state(J, N, L, T=1.5, seed=5)
    po = oracle_problem(oracle, d)
    Qo, Po, nuo = oracle.collide(po, f0)
    fo = f0.copy()
    sto = oracle.sweep(po, fo, Po, nuo, 1)
    s = sgs.Solver(gpu_problem(d))
    fd = to_dev(f0)
    Q, P = s.field(), s.field()
    s.collide(fd, Q, P)
    s.sweep_forward(fd, to_dev(Po))
    st = s.read_status()
    # the iteration count depends on a threshold; the solutions agree to the inner tolerance
    assert abs(st["inner_iters"] - sto["inner_iters"]) <= J
    assert rel(fd.cpu().numpy().reshape(f0.shape), fo) <= 1e-9


def test_residual_and_rescale_parity(oracle):
    N, J, L = 8, 7, 6.0
    d = spec(nx=J, nv=N, v_max=L, eps=0.3, total_mass=1.3)
    f = I.initial_state(J, N, L, T=1.2, seed=6)
    po = oracle_problem(oracle, d)
    Qo, Po, nuo = oracle.collide(po, f)
    s = sgs.Solver(gpu_problem(d))
    fd = to_dev(f)
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.residual(fd, to_dev(Qo), res)
    assert abs(res.item() - oracle.residual(po, f, Qo)) <= 1e-12 * oracle.residual(po, f, Qo)
    s.rescale(fd)
    fo = f.copy()
    oracle.rescale(po, fo)
    assert rel(fd.cpu().numpy().reshape(f.shape), fo) <= 1e-14


def test_sgs_iterations_parity(oracle):
    """Ten full SGS iterations (collide, forward, collide, backward, rescale) with a fixed
    inner count on the 16-cell heat-transfer problem; the residual after each iteration."""
    wl = I.heat_16cells_16v()
    d = spec(nx=wl.J, nv=wl.N, v_max=wl.L, eps=wl.eps, T=(wl.T_left, wl.T_right), total_mass=wl.total_mass,
             inner_fixed=8)
    f0 = wl.initial_state()
    po = oracle_problem(oracle, d)
    s = sgs.Solver(gpu_problem(d))
    fd = to_dev(f0)
    Q, P = s.field(), s.field()
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    fo = f0.copy()
    flags = sgs.IT_EVAL
    r0 = None
    for it in range(10):
        s.iterate(fd, Q, P, flags=flags, res=res)
        flags = sgs.IT_EVAL | sgs.IT_P_VALID
        oracle.sgs_iteration(po, fo)
        ro = oracle.solve_residual(po, fo)
        r0 = ro if r0 is None else r0
        # the residual is a difference of O(r0) terms: compare on that scale
        assert abs(res.item() - ro) <= 1e-12 * r0, it
    assert rel(fd.cpu().numpy().reshape(f0.shape), fo) <= 1e-12
    assert s.read_status()["status"] == 0


def test_nonfinite_input_sets_status_and_returns():
    N, J = 8, 3
    d = spec(nx=J, nv=N, inner_max=20)
    f = I.initial_state(J, N, 6.0)
    f[1, 3, 3, 3] = np.nan
    s = sgs.Solver(gpu_problem(d))
    fd = to_dev(f)
    Q, P = s.field(), s.field()
    s.collide(fd, Q, P)
    s.sweep_forward(fd, P)
    st = s.read_status()
    assert st["status"] & (sgs.ST_NONFINITE | sgs.ST_NEWTON_FAIL | sgs.ST_NONPOSITIVE)


@pytest.mark.parametrize("N,J,eps,direction", [(8, 6, 0.01, 1), (16, 4, 0.1, -1)])
def test_sweep_df64_parity(oracle, N, J, eps, direction):
    """Mixed-precision handles scan in double-float on the FP32 pipes: FP64-class accuracy."""
    L = 6.0
    d = spec(nx=J, nv=N, v_max=L, eps=eps, inner_fixed=6, precision=sgs.FP32)
    f0 = I.initial_state(J, N, L, T=1.5, seed=7)
    po = oracle_problem(oracle, d)
    Qo, Po, nuo = oracle.collide(po, f0)
    fo = f0.copy()
    oracle.sweep(po, fo, Po, nuo, direction)
    s = sgs.Solver(gpu_problem(d))
    fd = to_dev(f0)
    Q, P = s.field(), s.field()
    s.collide(fd, Q, P)
    Pd = to_dev(Po)
    if direction > 0:
        s.sweep_forward(fd, Pd)
    else:
        s.sweep_backward(fd, Pd)
    assert s.read_status()["status"] == 0
    assert rel(fd.cpu().numpy().reshape(f0.shape), fo) <= 1e-11


@pytest.mark.parametrize("N,J,L", [(8, 40, 6.0), (16, 16, 6.0), (12, 3, 6.0)])
def test_collide_df64_parity(oracle, N, J, L):
    """Double-float spectral sums (pairs of FP32 values on the FP32 pipes) against the FP64
    oracle: about 2^-48 per term, far inside the FP32 form's 1e-5."""
    d = spec(nx=J, nv=N, v_max=L, precision=sgs.FP32)
    f = varied_state(J, N, L, seed=2)
    s = sgs.Solver(gpu_problem(d))
    fd = to_dev(f)
    Q, P = s.field(), s.field()
    s.collide(fd, Q, P, precision=sgs.DF64)
    Qo, Po, nuo = oracle.collide(oracle_problem(oracle, d), f)
    assert rel(Q.cpu().numpy().reshape(f.shape), Qo) <= 1e-11
    assert rel(P.cpu().numpy().reshape(f.shape), Po) <= 1e-11
    assert s.read_status()["status"] == 0


def test_collide_df64_parity_full_size_sampled(oracle):
    N, J, L = 32, 64, 8.0
    d = spec(nx=J, nv=N, v_max=L, eps=0.01, precision=sgs.FP32)
    f = varied_state(J, N, L, seed=3)
    s = sgs.Solver(gpu_problem(d))
    Q, P = s.field(), s.field()
    s.collide(to_dev(f), Q, P, precision=sgs.DF64)
    Qd = Q.cpu().numpy().reshape(f.shape)
    po = oracle_problem(oracle, d)
    for j in (0, 45):
        Qo, Po, nuo = oracle.collide(po, f[j:j + 1])
        assert rel(Qd[j], Qo[0]) <= 1e-11, j
    assert s.read_status()["status"] == 0


@pytest.mark.parametrize("dc_prec", [sgs.DF64, sgs.FP64])
def test_defect_correction_tracks_fp64_iteration(dc_prec):
    """Mixed solver (FP32 collision sums in increment form + double-float scans + FP64
    defect correction) against the FP64 solver after the same number of SGS iterations from
    the same state: the iterates agree far below the FP32 resolution of the sums."""
    wl = I.heat_16cells_16v()
    d = spec(nx=wl.J, nv=wl.N, v_max=wl.L, eps=0.1, T=(wl.T_left, wl.T_right), total_mass=wl.total_mass,
             inner_tol=1e-11)
    f0 = wl.initial_state()
    s64 = sgs.Solver(gpu_problem(dict(d, precision=sgs.FP64)))
    f64 = to_dev(f0)
    Q, P = s64.field(), s64.field()
    res64 = torch.zeros(1, dtype=torch.float64, device="cuda")
    for it in range(48):
        s64.iterate(f64, Q, P, flags=sgs.IT_EVAL | (sgs.IT_P_VALID if it else 0), res=res64)
    s32 = sgs.Solver(gpu_problem(dict(d, precision=sgs.FP32)))
    s32.set_dc_precision(dc_prec)
    fdc = to_dev(f0)
    Q2, P2 = s32.field(), s32.field()
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    for k in range(6):
        s32.dc_step(fdc, Q2, P2, 8, res=res)
    s32.dc_step(fdc, Q2, P2, 0, res=res)  # FP64 residual of the final iterate
    assert s32.read_status()["status"] == 0
    # FP32 rounding of the increments between refreshes leaves ~1e-8; FP32 resolution is 6e-8
    assert rel(fdc.cpu().numpy(), f64.cpu().numpy()) <= 2e-8
    assert abs(res.item() - res64.item()) <= 0.05 * res64.item() + 1e-11, (res.item(), res64.item())


@pytest.mark.parametrize("levels,pre,post,coarse", [(3, 1, 1, 2), (2, 2, 1, 3)])
def test_vcycle_parity(oracle, levels, pre, post, coarse):
    """FAS V-cycle (eq. (30)) on the GPU against the oracle's, fixed inner counts."""
    N, J, L = 8, 8, 6.0
    d = spec(nx=J, nv=N, v_max=L, eps=0.05, inner_fixed=5)
    f0 = I.initial_state(J, N, L, T=1.5, seed=9)
    po = oracle_problem(oracle, d)
    fo = f0.copy()
    oracle.vcycle(po, fo, levels, pre, post, coarse)
    s = sgs.Solver(gpu_problem(d))
    assert s.max_levels() == 4
    fd = to_dev(f0)
    s.vcycle(fd, levels, pre, post, coarse)
    assert s.read_status()["status"] == 0
    assert rel(fd.cpu().numpy().reshape(f0.shape), fo) <= 1e-12


def test_vcycle_fp32_parity(oracle):
    """Mixed-precision V-cycle (FP32 collision sums, coarse levels in increment form against
    the restricted iterate) against the oracle's FP64 V-cycle: the increment form is exact in
    exact arithmetic (Q_s is bilinear), so only FP32 rounding of the sums separates them."""
    N, J, L = 8, 8, 6.0
    d = spec(nx=J, nv=N, v_max=L, eps=0.05, inner_fixed=5)
    f0 = I.initial_state(J, N, L, T=1.5, seed=9)
    fo = f0.copy()
    oracle.vcycle(oracle_problem(oracle, d), fo, 3, 1, 1, 2)
    s = sgs.Solver(gpu_problem(dict(d, precision=sgs.FP32)))
    fd = to_dev(f0)
    s.vcycle(fd, 3, 1, 1, 2)
    assert s.read_status()["status"] == 0
    assert rel(fd.cpu().numpy().reshape(f0.shape), fo) <= 1e-5


def test_dc_vcycle_tracks_fp64_vcycle():
    """Defect correction + V-cycles with FP32 sums against FP64 V-cycles from the same state:
    with every level in increment form the iterates stay far below FP32 resolution apart."""
    wl = I.heat_16cells_16v()
    d = spec(nx=wl.J, nv=wl.N, v_max=wl.L, eps=0.1, T=(wl.T_left, wl.T_right), total_mass=wl.total_mass,
             inner_tol=1e-11)
    f0 = wl.initial_state()
    s64 = sgs.Solver(gpu_problem(dict(d, precision=sgs.FP64)))
    f64 = to_dev(f0)
    s32 = sgs.Solver(gpu_problem(dict(d, precision=sgs.FP32)))
    fdc = to_dev(f0)
    Q, P = s32.field(), s32.field()
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    for k in range(6):
        s64.vcycle(f64, 3, 1, 1, 4)
        s32.dc_step(fdc, Q, P, 0, res=res)
        s32.vcycle(fdc, 3, 1, 1, 4)
    assert s64.read_status()["status"] == 0 and s32.read_status()["status"] == 0
    err = rel(fdc.cpu().numpy(), f64.cpu().numpy())
    print("dc+vcycle vs fp64 vcycle rel", err)
    assert err <= 5e-8


@pytest.mark.parametrize("precision,tol", [(sgs.FP64, 1e-12), (sgs.FP32, 1e-11)])
@pytest.mark.parametrize("direction", [1, -1])
def test_sweep_plain_fixed_point_parity(oracle, precision, tol, direction):
    """SGS-FP (eq. (22): no step 1, the Maxwellian of the current iterate in step 2) with a
    fixed inner count, in the FP64 and the double-float scan."""
    N, J, L = 8, 6, 6.0
    d = spec(nx=J, nv=N, v_max=L, eps=0.5, inner_fixed=7, inner_method=sgs.FP, precision=precision)
    f0 = I.initial_state(J, N, L, T=1.5, seed=12)
    po = oracle_problem(oracle, d)
    Qo, Po, nuo = oracle.collide(po, f0)
    fo = f0.copy()
    oracle.sweep(po, fo, Po, nuo, direction)
    s = sgs.Solver(gpu_problem(d))
    fd = to_dev(f0)
    Q, P = s.field(), s.field()
    s.collide(fd, Q, P)
    if direction > 0:
        s.sweep_forward(fd, to_dev(Po))
    else:
        s.sweep_backward(fd, to_dev(Po))
    st = s.read_status()
    assert st["status"] == 0 and st["inner_iters"] == 7 * J and st["fallbacks"] == 0
    assert rel(fd.cpu().numpy().reshape(f0.shape), fo) <= tol


def test_sweep_plain_fixed_point_tolerance_mode(oracle):
    """SGS-FP to an inner tolerance: the cell equations are solved to that tolerance on both
    sides (the stopping test on the GPU uses the step-2 identity after the first update)."""
    N, J, L = 8, 6, 6.0
    d = spec(nx=J, nv=N, v_max=L, eps=1.0, inner_tol=1e-11, inner_method=sgs.FP)
    f0 = I.initial_state(J, N, L, T=1.5, seed=13)
    po = oracle_problem(oracle, d)
    Qo, Po, nuo = oracle.collide(po, f0)
    fo = f0.copy()
    sto = oracle.sweep(po, fo, Po, nuo, 1)
    s = sgs.Solver(gpu_problem(d))
    fd = to_dev(f0)
    Q, P = s.field(), s.field()
    s.collide(fd, Q, P)
    s.sweep_forward(fd, to_dev(Po))
    st = s.read_status()
    assert st["status"] == 0
    assert abs(st["inner_iters"] - sto["inner_iters"]) <= J
    assert rel(fd.cpu().numpy().reshape(f0.shape), fo) <= 1e-9


def relax_cell_case(oracle, inner_method, precision):
    """One cell between inflow sides whose cell equation has the known solution g*: P is
    chosen so that r = A M[g*] - (|v1|/dx + A) g*; the stored value (two counter-moving
    beams at v1 = +-3) violates eq. (26) at the first inner iteration."""
    N, L, eps = 12, 6.0, 1.0
    bc = dict(bc_kind=(oracle.INFLOW, oracle.INFLOW), bc_rho=(1.0, 1.0), bc_u=((0.3, 0.0, 0.0), (-0.2, 0.0, 0.0)),
              bc_T=(1.0, 1.2), total_mass=0.0, inner_fixed=8, inner_method=inner_method)
    po = oracle.Problem(N=N, L=L, J=1, x_lo=0.0, x_hi=0.05, eps=eps, **bc)
    gp = sgs.Problem(nx=1, x_lo=0.0, x_hi=0.05, nv=N, v_max=L, eps=eps, precision=precision, **bc)
    v = oracle.velocity_nodes(N, L)
    V = np.stack(np.meshgrid(v, v, v, indexing="ij"), -1)
    w = (2 * L / N) ** 3
    dx = 0.05
    beam = lambda u: np.exp(-((V - [u, 0.0, 0.0]) ** 2).sum(-1) / (2 * 0.25))
    g0 = beam(3.0) + beam(-3.0)
    g0 /= w * g0.sum()
    f0 = g0[None].copy()
    Qo, Po_unused, nuo = oracle.collide(po, f0)
    A = nuo[0] / eps
    c = np.abs(V[..., 0]) / dx
    gstar = np.exp(-((V - [0.3, 0.0, 0.0]) ** 2).sum(-1) / 2.0) * (1.0 + 0.2 * np.cos(V[..., 1]))
    gstar /= w * gstar.sum()
    th, _ = oracle.discrete_maxwellian(N, L, oracle.moments(gstar, L))
    r_want = A * oracle.eval_maxwellian(N, L, th) - (c + A) * gstar
    gl, gr = oracle.ghost(po, 0, g0), oracle.ghost(po, 1, g0)
    r_ghost = (-np.maximum(V[..., 0], 0.0) * gl + np.minimum(V[..., 0], 0.0) * gr) / dx
    P = (eps * (r_ghost - r_want))[None]
    return po, gp, f0, P, nuo, gstar


@pytest.mark.parametrize("precision,tol", [(sgs.FP64, 1e-12), (sgs.FP32, 1e-11)])
def test_relaxed_step1_parity_where_existence_fails(oracle, precision, tol):
    """PFP with the relaxed step 1 (the remark after eq. (26)) against the oracle on a cell
    where eq. (26) fails at the first iteration; the plain PFP form falls back to the
    fixed-point step there instead."""
    for method in (sgs.PFP_RELAX, sgs.PFP):
        po, gp, f0, P, nuo, gstar = relax_cell_case(oracle, method, precision)
        fo = f0.copy()
        sto = oracle.sweep(po, fo, P, nuo, 1)
        s = sgs.Solver(gp)
        fd = to_dev(f0)
        Q, Ps = s.field(), s.field()
        s.collide(fd, Q, Ps)  # the scan reads the collision frequency of f0 from this step
        s.sweep_forward(fd, to_dev(P))
        st = s.read_status()
        assert st["status"] == 0 and st["inner_iters"] == 8
        assert rel(fd.cpu().numpy().reshape(f0.shape), fo) <= tol, method
        if method == sgs.PFP_RELAX:
            assert st["fallbacks"] == 0 and sto["existence_fallbacks"] == 0
        else:
            assert st["fallbacks"] >= 1 and sto["existence_fallbacks"] >= 1
