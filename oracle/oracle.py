"""ctypes view of the plain C FP64 oracle (``sgs_oracle.c``).

TEST INFRASTRUCTURE ONLY. Tests, the smoke check and the CPU-baseline leg of the
benchmark import this module; the CUDA library and its Python binding never do.

``build()`` compiles the C source with gcc into ``oracle/_build/liboracle.so``.
All arrays are numpy float64, C-contiguous; a distribution of one cell is a
(N, N, N) array indexed [i1, i2, i3] with v = (i - N/2 + 1) * 2L/N.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
SRC = os.path.join(HERE, "sgs_oracle.c")
SRC2D = os.path.join(HERE, "sgs_oracle2d.c")

MAXWELL, HARD_SPHERE, BGK = 0, 1, 2
DIFFUSE, INFLOW = 0, 1
PFP, FP, PFP_RELAX = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle (plain C17, -O2, OpenMP over cells in the collision step)."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
        os.path.getmtime(SRC), os.path.getmtime(SRC2D), os.path.getmtime(os.path.join(HERE, "sgs_oracle.h"))
    ):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-std=c17", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, SRC, SRC2D, "-lm"]
        )
        os.replace(tmp, LIB)
    return LIB


class _Problem(C.Structure):
    _fields_ = [
        ("N", C.c_int),
        ("L", C.c_double),
        ("kernel", C.c_int),
        ("b0", C.c_double),
        ("J", C.c_int),
        ("x_lo", C.c_double),
        ("x_hi", C.c_double),
        ("eps", C.c_double),
        ("bc_kind", C.c_int * 2),
        ("bc_rho", C.c_double * 2),
        ("bc_u", (C.c_double * 3) * 2),
        ("bc_T", C.c_double * 2),
        ("total_mass", C.c_double),
        ("inner_tol", C.c_double),
        ("inner_max", C.c_int),
        ("inner_fixed", C.c_int),
        ("newton_tol", C.c_double),
        ("newton_max", C.c_int),
        ("inner_method", C.c_int),
        ("conserve_proj", C.c_int),
        ("order", C.c_int),
    ]


class _Stats(C.Structure):
    _fields_ = [
        ("inner_iters", C.c_long),
        ("visits", C.c_long),
        ("newton_iters", C.c_long),
        ("newton_solves", C.c_long),
        ("existence_fallbacks", C.c_long),
        ("newton_failures", C.c_long),
    ]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


@dataclass
class Problem:
    """One 1-D steady problem; field meanings follow the oracle's C struct."""

    N: int = 16
    L: float = 6.0
    kernel: int = MAXWELL
    b0: float = 1.0 / (4.0 * np.pi)
    J: int = 16
    x_lo: float = 0.0
    x_hi: float = 1.0
    eps: float = 1.0
    bc_kind: tuple = (DIFFUSE, DIFFUSE)
    bc_rho: tuple = (1.0, 1.0)
    bc_u: tuple = ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0))
    bc_T: tuple = (1.0, 2.0)
    total_mass: float = 1.0
    inner_tol: float = 1e-8
    inner_max: int = 200
    inner_fixed: int = 0
    newton_tol: float = 1e-10
    newton_max: int = 50
    inner_method: int = PFP
    conserve_proj: int = 0
    order: int = 1

    @property
    def dx(self) -> float:
        return (self.x_hi - self.x_lo) / self.J

    def c(self) -> _Problem:
        p = _Problem()
        for name in ("N", "L", "kernel", "b0", "J", "x_lo", "x_hi", "eps", "total_mass", "inner_tol",
                     "inner_max", "inner_fixed", "newton_tol", "newton_max", "inner_method", "conserve_proj", "order"):
            setattr(p, name, getattr(self, name))
        for s in range(2):
            p.bc_kind[s] = self.bc_kind[s]
            p.bc_rho[s] = self.bc_rho[s]
            p.bc_T[s] = self.bc_T[s]
            for d in range(3):
                p.bc_u[s][d] = self.bc_u[s][d]
        return p


class _Problem2D(C.Structure):
    _fields_ = [
        ("p", _Problem),
        ("ny", C.c_int),
        ("y_lo", C.c_double),
        ("y_hi", C.c_double),
        ("bc_kind_y", C.c_int * 2),
        ("bc_rho_y", C.c_double * 2),
        ("bc_u_y", (C.c_double * 3) * 2),
        ("bc_T_y", C.c_double * 2),
    ]


@dataclass
class Problem2D:
    """A 2-D-space problem: nx = base.J cells on [base.x_lo, base.x_hi] with the x sides of
    base, ny cells on [y_lo, y_hi] with the y sides given here."""

    base: Problem
    ny: int = 16
    y_lo: float = 0.0
    y_hi: float = 1.0
    bc_kind_y: tuple = (DIFFUSE, DIFFUSE)
    bc_rho_y: tuple = (1.0, 1.0)
    bc_u_y: tuple = ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0))
    bc_T_y: tuple = (1.0, 1.0)

    @property
    def nx(self) -> int:
        return self.base.J

    @property
    def cells(self) -> int:
        return self.base.J * self.ny

    def c(self) -> _Problem2D:
        q = _Problem2D()
        q.p = self.base.c()
        q.ny, q.y_lo, q.y_hi = self.ny, self.y_lo, self.y_hi
        for s in range(2):
            q.bc_kind_y[s] = self.bc_kind_y[s]
            q.bc_rho_y[s] = self.bc_rho_y[s]
            q.bc_T_y[s] = self.bc_T_y[s]
            for d in range(3):
                q.bc_u_y[s][d] = self.bc_u_y[s][d]
        return q


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d = C.POINTER(C.c_double)
        P = C.POINTER(_Problem)
        P2 = C.POINTER(_Problem2D)
        S = C.POINTER(_Stats)
        sig = {
            "or_velocity_nodes": (None, [C.c_int, C.c_double, d]),
            "or_gauss_legendre": (None, [C.c_int, d, d]),
            "or_G": (C.c_double, [C.c_int, C.c_double, C.c_int, C.c_double, C.c_long, C.c_long]),
            "or_dft": (None, [C.c_int, d, d]),
            "or_idft": (None, [C.c_int, d, d]),
            "or_qhat_direct": (None, [C.c_int, C.c_double, C.c_int, C.c_double, d, d, d]),
            "or_qfsm": (None, [C.c_int, C.c_double, C.c_int, C.c_double, d, d]),
            "or_moments": (None, [C.c_int, C.c_double, d, d]),
            "or_macroscopic": (None, [C.c_int, C.c_double, d, d]),
            "or_conserve_project": (C.c_int, [C.c_int, C.c_double, d]),
            "or_conserve_project_w": (C.c_int, [C.c_int, C.c_double, d, d]),
            "or_discrete_maxwellian": (C.c_int, [C.c_int, C.c_double, d, d, d, C.c_int, C.c_double, C.c_int]),
            "or_eval_maxwellian": (None, [C.c_int, C.c_double, d, d]),
            "or_collision_frequency": (C.c_double, [P, d]),
            "or_collide_cell": (None, [P, d, d, d, d, d]),
            "or_collide": (None, [P, C.c_int, d, d, d, d]),
            "or_cell_solve": (C.c_int, [P, C.c_double, d, C.c_double, d, S]),
            "or_wall_density": (C.c_double, [P, C.c_int, d]),
            "or_ghost": (None, [P, C.c_int, d, d]),
            "or_sweep": (None, [P, C.c_int, C.c_double, C.c_int, d, d, d, d, S]),
            "or_rescale": (None, [P, C.c_int, C.c_double, d]),
            "or_residual": (C.c_double, [P, C.c_int, C.c_double, d, d, d, d]),
            "or_sgs_iteration": (None, [P, C.c_int, C.c_double, d, d, C.c_int, S]),
            "or_si_iteration": (None, [P, C.c_int, C.c_double, d, d, C.c_int]),
            "or_vcycle": (None, [P, d, C.c_int, C.c_int, C.c_int, C.c_int, S]),
            "or_cell_solve_c": (C.c_int, [P, d, d, C.c_double, d, S]),
            "or_ghost2d": (None, [P2, C.c_int, d, d]),
            "or_sweep2d": (None, [P2, C.c_int, d, d, d, d, S]),
            "or_rescale2d": (None, [P2, d]),
            "or_residual2d": (C.c_double, [P2, d, d, d, d]),
            "or_sgs_iteration2d": (None, [P2, d, d, C.c_int, S]),
            "or_vcycle2d": (None, [P2, d, C.c_int, C.c_int, C.c_int, C.c_int, S]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _arr(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------- wrappers
def velocity_nodes(N, L):
    out = np.empty(N)
    lib().or_velocity_nodes(N, L, _p(out))
    return out


def gauss_legendre(n):
    x, w = np.empty(n), np.empty(n)
    lib().or_gauss_legendre(n, _p(x), _p(w))
    return x, w


def G(N, L, kernel, b0, a2, b2):
    return lib().or_G(N, L, kernel, b0, int(a2), int(b2))


def dft(f):
    N = f.shape[0]
    n = N - 1
    out = np.empty((n, n, n, 2))
    lib().or_dft(N, _p(_arr(f)), _p(out))
    return out[..., 0] + 1j * out[..., 1]


def idft(qhat, N):
    q = np.empty((N, N, N))
    qa = _arr(np.stack([qhat.real, qhat.imag], axis=-1))
    lib().or_idft(N, _p(qa), _p(q))
    return q


def qhat_direct(N, L, kernel, b0, ahat, bhat):
    n = N - 1
    a = _arr(np.stack([ahat.real, ahat.imag], axis=-1))
    b = _arr(np.stack([bhat.real, bhat.imag], axis=-1))
    out = np.empty((n, n, n, 2))
    lib().or_qhat_direct(N, L, kernel, b0, _p(a), _p(b), _p(out))
    return out[..., 0] + 1j * out[..., 1]


def qfsm(f, L, kernel=MAXWELL, b0=1.0 / (4 * np.pi)):
    N = f.shape[0]
    q = np.empty((N, N, N))
    lib().or_qfsm(N, L, kernel, b0, _p(_arr(f)), _p(q))
    return q


def moments(f, L):
    m = np.empty(5)
    lib().or_moments(f.shape[0], L, _p(_arr(f)), _p(m))
    return m


def macroscopic(f, L):
    """(rho, U1, U2, U3, T, q1, q2, q3) of one cell (N, N, N): the moments' definitions with
    d = 3 and the heat flux q = 1/2 int (v - U)|v - U|^2 f dv of Section 4.2.2."""
    out = np.empty(8)
    lib().or_macroscopic(f.shape[0], L, _p(_arr(f)), _p(out))
    return out


def conserve_project(q, L):
    """Conservation projection of one cell's q (N, N, N); returns a new array."""
    out = _arr(q).copy()
    if lib().or_conserve_project(q.shape[0], L, _p(out)) != 0:
        raise ArithmeticError("singular Gram matrix")
    return out


def conserve_project_w(q, L, M):
    """Maxwellian-weighted conservation projection of one cell's q; returns a new array."""
    out = _arr(q).copy()
    if lib().or_conserve_project_w(q.shape[0], L, _p(_arr(M)), _p(out)) != 0:
        raise ArithmeticError("singular Gram matrix")
    return out


def discrete_maxwellian(N, L, target, wk=None, theta0=None, tol=1e-10, maxit=50):
    """Returns (theta, iterations); iterations < 0 means failure."""
    th = np.zeros(5) if theta0 is None else _arr(theta0).copy()
    it = lib().or_discrete_maxwellian(N, L, _p(None if wk is None else _arr(wk)), _p(_arr(target)), _p(th),
                                      0 if theta0 is None else 1, tol, maxit)
    return th, it


def eval_maxwellian(N, L, theta):
    M = np.empty((N, N, N))
    lib().or_eval_maxwellian(N, L, _p(_arr(theta)), _p(M))
    return M


def collision_frequency(prob: Problem, f):
    p = prob.c()
    return lib().or_collision_frequency(C.byref(p), _p(_arr(f)))


def collide_cell(prob: Problem, f):
    """Returns (Q, P, nu, theta) of one cell."""
    p = prob.c()
    N = prob.N
    Q, P, th = np.empty((N, N, N)), np.empty((N, N, N)), np.empty(5)
    nu = C.c_double()
    lib().or_collide_cell(C.byref(p), _p(_arr(f)), _p(Q), _p(P), C.cast(C.pointer(nu), C.POINTER(C.c_double)),
                          _p(th))
    return Q, P, nu.value, th


def collide(prob: Problem, f):
    """All cells of f (J, N, N, N): returns (Q, P, nu)."""
    p = prob.c()
    f = _arr(f)
    J = f.shape[0]
    Q, P, nu = np.empty_like(f), np.empty_like(f), np.empty(J)
    lib().or_collide(C.byref(p), J, _p(f), _p(Q), _p(P), _p(nu))
    return Q, P, nu


def cell_solve(prob: Problem, dx, r, nu, g0):
    p = prob.c()
    st = _Stats()
    g = _arr(g0).copy()
    it = lib().or_cell_solve(C.byref(p), dx, _p(_arr(r)), nu, _p(g), C.byref(st))
    return g, it, st.as_dict()


def wall_density(prob: Problem, side, f_adj):
    p = prob.c()
    return lib().or_wall_density(C.byref(p), side, _p(_arr(f_adj)))


def ghost(prob: Problem, side, f_adj):
    p = prob.c()
    out = np.empty((prob.N,) * 3)
    lib().or_ghost(C.byref(p), side, _p(_arr(f_adj)), _p(out))
    return out


def sweep(prob: Problem, f, P, nu, direction, b=None, dx=None):
    """In place on f (J, N, N, N)."""
    p = prob.c()
    st = _Stats()
    J = f.shape[0]
    dx = prob.dx if dx is None else dx
    lib().or_sweep(C.byref(p), J, dx, direction, _p(f), _p(_arr(P)), _p(_arr(nu)),
                   _p(None if b is None else _arr(b)), C.byref(st))
    return st.as_dict()


def rescale(prob: Problem, f, dx=None):
    p = prob.c()
    lib().or_rescale(C.byref(p), f.shape[0], prob.dx if dx is None else dx, _p(f))


def residual(prob: Problem, f, Q, b=None, dx=None, return_field=False):
    p = prob.c()
    J = f.shape[0]
    R = np.empty_like(_arr(f)) if return_field else None
    res = lib().or_residual(C.byref(p), J, prob.dx if dx is None else dx, _p(_arr(f)), _p(_arr(Q)),
                            _p(None if b is None else _arr(b)), _p(R))
    return (res, R) if return_field else res


def sgs_iteration(prob: Problem, f, b=None, rescale=True, dx=None):
    p = prob.c()
    st = _Stats()
    lib().or_sgs_iteration(C.byref(p), f.shape[0], prob.dx if dx is None else dx, _p(f),
                           _p(None if b is None else _arr(b)), 1 if rescale else 0, C.byref(st))
    return st.as_dict()


def si_iteration(prob: Problem, f, b=None, rescale=True, dx=None):
    """One source iteration (eq. (SI) with the lagged BGK-penalty source), in place."""
    p = prob.c()
    lib().or_si_iteration(C.byref(p), f.shape[0], prob.dx if dx is None else dx, _p(f),
                          _p(None if b is None else _arr(b)), 1 if rescale else 0)


def vcycle(prob: Problem, f, levels, pre=1, post=1, coarse_iters=10):
    p = prob.c()
    st = _Stats()
    lib().or_vcycle(C.byref(p), _p(f), levels, pre, post, coarse_iters, C.byref(st))
    return st.as_dict()


def solve_residual(prob: Problem, f):
    """Residual of f after a fresh collision evaluation (no rescale)."""
    Q, _, _ = collide(prob, f)
    return residual(prob, f, Q)


# ------------------------------------------------------------------------------ 2-D space
def collide2d(prob: Problem2D, f):
    """Collision step of every cell (cells are independent): (Q, P, nu)."""
    return collide(prob.base, f)


def ghost2d(prob: Problem2D, side, f_adj):
    q = prob.c()
    g = np.empty_like(_arr(f_adj))
    lib().or_ghost2d(C.byref(q), side, _p(_arr(f_adj)), _p(g))
    return g


def sweep2d(prob: Problem2D, f, P, nu, ordering, b=None):
    q = prob.c()
    st = _Stats()
    lib().or_sweep2d(C.byref(q), ordering, _p(f), _p(_arr(P)), _p(_arr(nu)), _p(None if b is None else _arr(b)),
                     C.byref(st))
    return st.as_dict()


def rescale2d(prob: Problem2D, f):
    q = prob.c()
    lib().or_rescale2d(C.byref(q), _p(f))


def residual2d(prob: Problem2D, f, Q, b=None, return_field=False):
    q = prob.c()
    R = np.empty_like(_arr(f)) if return_field else None
    res = lib().or_residual2d(C.byref(q), _p(_arr(f)), _p(_arr(Q)), _p(None if b is None else _arr(b)), _p(R))
    return (res, R) if return_field else res


def sgs_iteration2d(prob: Problem2D, f, b=None, rescale=True):
    q = prob.c()
    st = _Stats()
    lib().or_sgs_iteration2d(C.byref(q), _p(f), _p(None if b is None else _arr(b)), 1 if rescale else 0,
                             C.byref(st))
    return st.as_dict()


def vcycle2d(prob: Problem2D, f, levels, pre=1, post=1, coarse_iters=10):
    q = prob.c()
    st = _Stats()
    lib().or_vcycle2d(C.byref(q), _p(f), levels, pre, post, coarse_iters, C.byref(st))
    return st.as_dict()


def solve_residual2d(prob: Problem2D, f):
    Q, _, _ = collide2d(prob, f)
    return residual2d(prob, f, Q)
