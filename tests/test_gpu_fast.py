"""The fast (Carleman-form) spectral operator on the tensor cores.

First the tensor-core path itself: tcgen05.mma products of BF16 operands with FP32
accumulation in TMEM against the CUDA-core product of the same BF16 terms (the operand layout
and descriptors), for the shapes the operator uses."""
import pytest

torch = pytest.importorskip("torch")

from paper_2409_01910_gb300 import sgs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sgs.lib()


@pytest.mark.parametrize("K,N", [(32, 64), (64, 96), (64, 48), (32, 32)])
@pytest.mark.parametrize("terms", [1, 3])
def test_tensor_core_products_match_cuda_cores(K, N, terms):
    err, ref = sgs.tc_selftest(K, N, terms)
    assert err >= 0.0, "completion wait gave up"
    # the same BF16 terms summed in FP32 in a different order: a few FP32 ulps of the sum
    assert err <= 1e-5 * max(ref, 1.0), (err, ref)


def hs_states(J, N, L, seed):
    """Cells far from equilibrium: two-Maxwellian mixtures with cell-dependent shifts."""
    from paper_2409_01910_gb300 import inputs as I
    import numpy as np

    rng = np.random.default_rng(seed)
    f = np.empty((J, N, N, N))
    for j in range(J):
        u = rng.uniform(-0.8, 0.8, 3)
        f[j] = I.sampled_maxwellian(N, L, rng.uniform(0.6, 1.4), u, rng.uniform(0.7, 1.5))
        f[j] += I.sampled_maxwellian(N, L, rng.uniform(0.2, 0.6), -u, rng.uniform(0.5, 1.0))
    return f


@pytest.mark.parametrize("terms,tol", [(3, 1e-3), (1, 6e-2)])
def test_fast_operator_matches_the_fast_oracle(terms, tol):
    """The fast (Carleman-form) operator for hard spheres, three tensor-core DFT passes per
    node of the 8 x 16 half-sphere rule, against the oracle's fast operator (the same
    discretisation in FP64) cell by cell. Tolerances from the arithmetic (a numpy emulation
    of the same passes with BF16 rounding): split BF16 operands (hi hi + lo hi + hi lo) leave
    about 2e-4 of max |Q|, single BF16 operands about 2.4e-2."""
    import numpy as np
    from oracle import fast_spectral as F

    N, L, J = 16, 8.0, 4
    b0 = 1.0 / (4.0 * np.pi)
    f = hs_states(J, N, L, seed=5)
    s = sgs.Solver(sgs.Problem(nx=J, nv=N, v_max=L, collision=sgs.HARD_SPHERE, b0=b0, eps=0.1))
    fast = sgs.FastOperator(s, m_theta=8, m_phi=16, chunk=8)
    fd = torch.from_numpy(f.reshape(-1)).cuda()
    Q = s.field()
    fast.collide(fd, Q, terms=terms)
    torch.cuda.synchronize()
    assert s.read_status()["status"] & sgs.ST_TIMEOUT == 0
    Qg = Q.cpu().numpy().reshape(f.shape)
    for j in range(J):
        qo = F.qfsm_fast(f[j], L, b0, 8, 16)
        err = float(np.abs(Qg[j] - qo).max() / np.abs(qo).max())
        assert err <= tol, (j, err)
    # mass is conserved by the fast operator's discretisation; the tensor-core form keeps it to
    # its own precision
    w = (2 * L / N) ** 3
    assert abs(w * Qg.sum((1, 2, 3))).max() <= tol * w * np.abs(Qg).sum((1, 2, 3)).max()


@pytest.mark.parametrize("terms,tol", [(3, 1e-3), (1, 8e-2)])
def test_fast_operator_at_the_shock_grid(terms, tol):
    """The full-size grid of the hard-sphere workload (32^3 on [-10, 10]^3, P = 48, K = 64: the
    launch shapes the benchmark's fast case times), two cells against the fast oracle. Bounds
    from a numpy emulation of the same passes with BF16 rounding on these two states: single
    BF16 products 5.0e-2 and 6.0e-2 of max |Q| (the longer transforms of N = 32 round more
    than N = 16's 2.4e-2), split products 6e-5 and 9e-5; the bounds leave about 30 % and a
    factor 10 above them."""
    import numpy as np
    from oracle import fast_spectral as F

    N, L, J = 32, 10.0, 2
    b0 = 1.0 / (4.0 * np.pi)
    f = hs_states(J, N, L, seed=9)
    s = sgs.Solver(sgs.Problem(nx=J, nv=N, v_max=L, collision=sgs.HARD_SPHERE, b0=b0, eps=0.1))
    fast = sgs.FastOperator(s, m_theta=8, m_phi=16, chunk=8)
    fd = torch.from_numpy(f.reshape(-1)).cuda()
    Q = s.field()
    fast.collide(fd, Q, terms=terms)
    torch.cuda.synchronize()
    assert s.read_status()["status"] & sgs.ST_TIMEOUT == 0
    Qg = Q.cpu().numpy().reshape(f.shape)
    for j in range(J):
        qo = F.qfsm_fast(f[j], L, b0, 8, 16)
        err = float(np.abs(Qg[j] - qo).max() / np.abs(qo).max())
        assert err <= tol, (j, err)
