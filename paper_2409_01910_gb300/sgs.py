"""Thin Python binding of the C ABI in include/sgs.h (argument marshalling only).

PyTorch provides device memory and streams; every step of the solver runs in the CUDA
library ``_build/libsgs.so``. There is no CPU fallback: if the library cannot be loaded
the calls raise.

Names follow the C entry points: ``setup``, ``collide``, ``sweep_forward``,
``sweep_backward``, ``rescale``, ``residual``, ``iterate``, ``vcycle``, ``read_status``.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

from . import build as _build

OK, ERR_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_WORKSPACE, ERR_NOMEM = 0, -1, -2, -3, -4, -5
ST_NEWTON_FAIL, ST_INNER_CAP, ST_NONPOSITIVE, ST_NONFINITE, ST_TIMEOUT = 1, 2, 4, 8, 16
MAXWELL, HARD_SPHERE, BGK = 0, 1, 2
DIFFUSE, INFLOW = 0, 1
FP64, FP32, DF64 = 0, 1, 2
PFP, FP, PFP_RELAX = 0, 1, 2
IT_P_VALID, IT_EVAL = 1, 2
PEAK_PACKED = 256  # sgs_peak_fma: the packed FP32 pair FMA (fma.rn.f32x2)
PROF_NAMES = ("moments", "dft", "sum", "reduce_idft", "sweep", "residual", "rescale", "sum_fp64", "sum_df64", "fast")
PROF_CLASSES = len(PROF_NAMES)


class _BC(C.Structure):
    _fields_ = [("kind", C.c_int), ("rho", C.c_double), ("u", C.c_double * 3), ("T", C.c_double)]


class _Problem(C.Structure):
    _fields_ = [
        ("space_dim", C.c_int),
        ("nx", C.c_int),
        ("x_lo", C.c_double),
        ("x_hi", C.c_double),
        ("ny", C.c_int),
        ("y_lo", C.c_double),
        ("y_hi", C.c_double),
        ("nv", C.c_int),
        ("v_max", C.c_double),
        ("collision", C.c_int),
        ("b0", C.c_double),
        ("eps", C.c_double),
        ("bc", _BC * 4),
        ("total_mass", C.c_double),
        ("precision", C.c_int),
        ("inner_tol", C.c_double),
        ("inner_max", C.c_int),
        ("inner_fixed", C.c_int),
        ("newton_tol", C.c_double),
        ("newton_max", C.c_int),
        ("inner_method", C.c_int),
        ("conserve_proj", C.c_int),
        ("order", C.c_int),
    ]


class _Tuning(C.Structure):
    _fields_ = [
        ("sweep_ept", C.c_int),
        ("sweep_cluster", C.c_int),
        ("sweep_threads", C.c_int),
        ("sweep_ms", C.c_float),
        ("candidates", C.c_int),
        ("sum_warps", C.c_int),
        ("sum_units", C.c_int),
        ("sum_blocks", C.c_int),
        ("sum_ms", C.c_float),
        ("sum_candidates", C.c_int),
    ]


class _Stats(C.Structure):
    _fields_ = [
        ("status", C.c_uint),
        ("visits", C.c_ulonglong),
        ("inner_iters", C.c_ulonglong),
        ("newton_iters", C.c_ulonglong),
        ("newton_solves", C.c_ulonglong),
        ("fallbacks", C.c_ulonglong),
    ]


@dataclass
class Problem:
    """Python mirror of sgs_problem (1-D space, 3-D velocity)."""

    nx: int = 16
    x_lo: float = 0.0
    x_hi: float = 1.0
    nv: int = 16
    v_max: float = 6.0
    collision: int = MAXWELL
    b0: float = 1.0 / (4.0 * 3.141592653589793)
    eps: float = 1.0
    bc_kind: Sequence[int] = (DIFFUSE, DIFFUSE)
    bc_rho: Sequence[float] = (1.0, 1.0)
    bc_u: Sequence[Sequence[float]] = ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0))
    bc_T: Sequence[float] = (1.0, 2.0)
    total_mass: float = 1.0
    precision: int = FP64
    inner_tol: float = 1e-8
    inner_max: int = 200
    inner_fixed: int = 0
    newton_tol: float = 1e-10
    newton_max: int = 50
    inner_method: int = PFP
    conserve_proj: int = 0  # 1: FP64 projection of Q onto the zero-moment subspace (not in the paper)
    order: int = 1          # spatial order of the 1-D scheme: 1, or 2 (linear reconstruction, eq. (slope))
    space_dim: int = 1
    ny: int = 1
    y_lo: float = 0.0
    y_hi: float = 1.0
    # y_lo, y_hi sides (2-D): kind, density, velocity, temperature
    bc_kind_y: Sequence[int] = (DIFFUSE, DIFFUSE)
    bc_rho_y: Sequence[float] = (1.0, 1.0)
    bc_u_y: Sequence[Sequence[float]] = ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0))
    bc_T_y: Sequence[float] = (1.0, 1.0)

    @property
    def cells(self) -> int:
        return self.nx * (self.ny if self.space_dim == 2 else 1)

    def c(self) -> _Problem:
        p = _Problem()
        for name in ("space_dim", "nx", "x_lo", "x_hi", "ny", "y_lo", "y_hi", "nv", "v_max", "collision", "b0",
                     "eps", "total_mass", "precision", "inner_tol", "inner_max", "inner_fixed", "newton_tol",
                     "newton_max", "inner_method", "conserve_proj", "order"):
            setattr(p, name, getattr(self, name))
        kinds = list(self.bc_kind) + list(self.bc_kind_y)
        rhos = list(self.bc_rho) + list(self.bc_rho_y)
        us = list(self.bc_u) + list(self.bc_u_y)
        Ts = list(self.bc_T) + list(self.bc_T_y)
        for s in range(4):
            p.bc[s].kind = kinds[s]
            p.bc[s].rho = rhos[s]
            p.bc[s].T = Ts[s]
            for d in range(3):
                p.bc[s].u[d] = us[s][d]
        return p


_lib = None


def lib(build: bool = True):
    """Loads the CUDA library (building it first if asked and needed). Raises if absent."""
    global _lib
    if _lib is None:
        path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not found at {path}; run paper_2409_01910_gb300.build.build()")
        L = C.CDLL(path)
        vp, d = C.c_void_p, C.POINTER(C.c_double)
        sig = {
            "sgs_setup": (C.c_int, [C.POINTER(_Problem), C.c_int, C.POINTER(vp), C.POINTER(C.c_size_t)]),
            "sgs_bind_workspace": (C.c_int, [vp, vp, C.c_size_t]),
            "sgs_layout": (C.c_int, [vp, C.c_int, C.POINTER(C.c_size_t), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "sgs_field_elems": (C.c_size_t, [vp]),
            "sgs_collide": (C.c_int, [vp, vp, vp, vp, vp]),
            "sgs_collide_prec": (C.c_int, [vp, vp, vp, vp, C.c_int, vp]),
            "sgs_sweep_forward": (C.c_int, [vp, vp, vp, vp, vp]),
            "sgs_si_iteration": (C.c_int, [vp, vp, vp, vp, vp]),
            "sgs_sweep_backward": (C.c_int, [vp, vp, vp, vp, vp]),
            "sgs_sweep_ordering": (C.c_int, [vp, vp, vp, vp, C.c_int, vp]),
            "sgs_rescale": (C.c_int, [vp, vp, vp]),
            "sgs_macroscopic": (C.c_int, [vp, vp, vp, vp]),
            "sgs_residual": (C.c_int, [vp, vp, vp, vp, vp, vp]),
            "sgs_iterate": (C.c_int, [vp, vp, vp, vp, vp, C.c_int, vp, vp]),
            "sgs_dc_step": (C.c_int, [vp, vp, vp, vp, C.c_int, vp, vp]),
            "sgs_dc_clear": (C.c_int, [vp]),
            "sgs_set_dc_precision": (C.c_int, [vp, C.c_int]),
            "sgs_profile": (C.c_int, [vp, C.c_int]),
            "sgs_profile_read": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_ulonglong), C.POINTER(C.c_double),
                                           C.c_int]),
            "sgs_launch_count": (C.c_ulonglong, [vp]),
            "sgs_vcycle": (C.c_int, [vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, vp]),
            "sgs_max_levels": (C.c_int, [vp]),
            "sgs_set_overlap": (C.c_int, [vp, C.c_int]),
            "sgs_get_overlap": (C.c_int, [vp]),
            "sgs_residual_noalloc": (C.c_int, [C.POINTER(_Problem), vp, vp, vp, vp, vp]),
            "sgs_update_active": (C.c_int, [vp, vp, C.c_double, vp]),
            "sgs_activate_all": (C.c_int, [vp, vp]),
            "sgs_read_active": (C.c_int, [vp, C.POINTER(C.c_int), vp]),
            "sgs_get_sweep_shape": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "sgs_set_sweep_shape": (C.c_int, [vp, C.c_int, C.c_int, C.c_int]),
            "sgs_autotune": (C.c_int, [vp, vp, vp, C.c_int, C.POINTER(_Tuning), vp]),
            "sgs_read_status": (C.c_int, [vp, C.POINTER(_Stats), vp]),
            "sgs_reset_stats": (C.c_int, [vp, vp]),
            "sgs_destroy": (None, [vp]),
            "sgs_strerror": (C.c_char_p, [C.c_int]),
            "sgs_host_weight": (C.c_double, [C.c_int, C.c_double, C.c_int, C.c_double, C.c_longlong, C.c_longlong]),
            "sgs_peak_fma": (C.c_int, [C.c_int, C.c_longlong, C.POINTER(C.c_double), C.POINTER(C.c_int),
                                       C.POINTER(C.c_float), vp]),
            "sgs_probe_scan": (C.c_int, [C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                         C.POINTER(C.c_float), vp]),
            "sgs_fast_setup": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.POINTER(vp), C.POINTER(C.c_size_t)]),
            "sgs_fast_bind": (C.c_int, [vp, vp, C.c_size_t]),
            "sgs_fast_collide": (C.c_int, [vp, vp, vp, vp, C.c_int, vp]),
            "sgs_fast_destroy": (None, [vp]),
            "sgs_tc_selftest": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_size_t, C.POINTER(C.c_double),
                                          C.POINTER(C.c_double), vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class SGSError(RuntimeError):
    pass


def _check(code: int, what: str):
    if code != OK:
        raise SGSError(f"{what}: {lib().sgs_strerror(code).decode()} ({code})")


def host_weight(nv, v_max, collision, b0, a2, b2) -> float:
    return lib().sgs_host_weight(nv, v_max, collision, b0, a2, b2)


def peak_fma(precision, iters=1 << 16, stream=None) -> dict:
    """Measured FMA throughput of the current device's CUDA cores (FP32, FP64, or
    FP32 | PEAK_PACKED for the packed pair instruction)."""
    t, n, ms = C.c_double(), C.c_int(), C.c_float()
    _check(lib().sgs_peak_fma(precision, iters, C.byref(t), C.byref(n), C.byref(ms), _stream(stream)),
           "sgs_peak_fma")
    return {"tflops": float(t.value), "sms": int(n.value), "ms": float(ms.value)}


def probe_scan(nv, v_max, precision, cluster, threads, mode, reps=2000, stream=None) -> float:
    """Microseconds per cluster reduction (mode 0), per Newton iteration (mode 1) or per
    hardware cluster barrier (mode 2) of the persistent scan in one cluster of the given
    shape."""
    us = C.c_float()
    _check(lib().sgs_probe_scan(nv, v_max, precision, cluster, threads, mode, reps, C.byref(us), _stream(stream)),
           "sgs_probe_scan")
    return float(us.value)


def tc_selftest(K, N, terms=3, swap=0, stream=None):
    """Tensor-core check: (max |D_tcgen05 - D_cuda_cores|, max |D|) for a 128 x K by K x N
    product of seeded BF16-split values."""
    import torch

    scratch = torch.empty(4 * (128 * K + N * K + 256 * N) + 1024, dtype=torch.uint8, device="cuda")
    me, mr = C.c_double(), C.c_double()
    _check(lib().sgs_tc_selftest(K, N, terms, swap, scratch.data_ptr(), scratch.numel(), C.byref(me), C.byref(mr),
                                 _stream(stream)), "sgs_tc_selftest")
    return float(me.value), float(mr.value)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    import torch

    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(), "fields are contiguous FP64 CUDA tensors"
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Solver:
    """Owns one library handle and its torch-allocated workspace."""

    def __init__(self, problems, device="cuda"):
        import torch

        if isinstance(problems, Problem):
            problems = [problems]
        self.problems = list(problems)
        arr = (_Problem * len(self.problems))(*[p.c() for p in self.problems])
        h = C.c_void_p()
        ws = C.c_size_t()
        _check(lib().sgs_setup(arr, len(self.problems), C.byref(h), C.byref(ws)), "sgs_setup")
        self.h = h
        self.workspace = torch.empty(max(int(ws.value), 256), dtype=torch.uint8, device=device)
        _check(lib().sgs_bind_workspace(self.h, self.workspace.data_ptr(), self.workspace.numel()),
               "sgs_bind_workspace")
        self.n_inst = len(self.problems)
        self.field_elems = int(lib().sgs_field_elems(self.h))
        self.device = device

    def layout(self, inst: int):
        off, J, nv = C.c_size_t(), C.c_int(), C.c_int()
        _check(lib().sgs_layout(self.h, inst, C.byref(off), C.byref(J), C.byref(nv)), "sgs_layout")
        return int(off.value), int(J.value), int(nv.value)

    def field(self):
        import torch

        return torch.zeros(self.field_elems, dtype=torch.float64, device=self.device)

    def view(self, fld, inst: int):
        off, J, N = self.layout(inst)
        return fld[off: off + J * N ** 3].view(J, N, N, N)

    def collide(self, f, Q=None, P=None, precision=None, stream=None):
        if precision is None:
            _check(lib().sgs_collide(self.h, _ptr(f), _ptr(Q), _ptr(P), _stream(stream)), "sgs_collide")
        else:
            _check(lib().sgs_collide_prec(self.h, _ptr(f), _ptr(Q), _ptr(P), precision, _stream(stream)),
                   "sgs_collide_prec")

    def sweep_forward(self, f, P, rhs=None, stream=None):
        _check(lib().sgs_sweep_forward(self.h, _ptr(f), _ptr(P), _ptr(rhs), _stream(stream)), "sgs_sweep_forward")

    def sweep_backward(self, f, P, rhs=None, stream=None):
        _check(lib().sgs_sweep_backward(self.h, _ptr(f), _ptr(P), _ptr(rhs), _stream(stream)), "sgs_sweep_backward")

    def sweep_ordering(self, f, P, ordering, rhs=None, stream=None):
        _check(lib().sgs_sweep_ordering(self.h, _ptr(f), _ptr(P), _ptr(rhs), ordering, _stream(stream)),
               "sgs_sweep_ordering")

    def si_iteration(self, f, P, rhs=None, stream=None):
        """One source iteration (eq. (SI)); P receives the penalty of the previous iterate."""
        _check(lib().sgs_si_iteration(self.h, _ptr(f), _ptr(P), _ptr(rhs), _stream(stream)), "sgs_si_iteration")

    def rescale(self, f, stream=None):
        _check(lib().sgs_rescale(self.h, _ptr(f), _stream(stream)), "sgs_rescale")

    def macroscopic(self, f, out=None, stream=None):
        """(cells, 8) FP64 device tensor: rho, U1, U2, U3, T, q1, q2, q3 of every cell."""
        import torch

        if out is None:
            cells = self.field_elems // self.problems[0].nv ** 3
            out = torch.empty((cells, 8), dtype=torch.float64, device=f.device)
        _check(lib().sgs_macroscopic(self.h, _ptr(f), _ptr(out), _stream(stream)), "sgs_macroscopic")
        return out

    def residual(self, f, Q, res, rhs=None, stream=None):
        _check(lib().sgs_residual(self.h, _ptr(f), _ptr(Q), _ptr(rhs), _ptr(res), _stream(stream)), "sgs_residual")

    def iterate(self, f, Q, P, flags=0, res=None, rhs=None, stream=None):
        _check(lib().sgs_iterate(self.h, _ptr(f), _ptr(Q), _ptr(P), _ptr(rhs), flags, _ptr(res), _stream(stream)),
               "sgs_iterate")

    def dc_step(self, f, Q, P, lo_iters, res=None, stream=None):
        _check(lib().sgs_dc_step(self.h, _ptr(f), _ptr(Q), _ptr(P), lo_iters, _ptr(res), _stream(stream)),
               "sgs_dc_step")

    def set_dc_precision(self, precision):
        _check(lib().sgs_set_dc_precision(self.h, precision), "sgs_set_dc_precision")

    def dc_clear(self):
        _check(lib().sgs_dc_clear(self.h), "sgs_dc_clear")

    def profile(self, enable=True):
        _check(lib().sgs_profile(self.h, 1 if enable else 0), "sgs_profile")

    def profile_read(self, with_work=False):
        """Per class: (milliseconds, bracketed launch groups), or with_work (ms, groups, cells
        processed: evaluated by the sums, visited by the scans)."""
        ms = (C.c_double * PROF_CLASSES)()
        n = (C.c_ulonglong * PROF_CLASSES)()
        wk = (C.c_double * PROF_CLASSES)()
        _check(lib().sgs_profile_read(self.h, ms, n, wk, PROF_CLASSES), "sgs_profile_read")
        if with_work:
            return {PROF_NAMES[i]: (float(ms[i]), int(n[i]), float(wk[i])) for i in range(PROF_CLASSES)}
        return {PROF_NAMES[i]: (float(ms[i]), int(n[i])) for i in range(PROF_CLASSES)}

    def launch_count(self) -> int:
        return int(lib().sgs_launch_count(self.h))

    def vcycle(self, f, levels, pre=1, post=1, coarse_iters=10, stream=None):
        _check(lib().sgs_vcycle(self.h, _ptr(f), levels, pre, post, coarse_iters, _stream(stream)), "sgs_vcycle")

    def max_levels(self) -> int:
        return int(lib().sgs_max_levels(self.h))

    def set_overlap(self, enable: bool):
        """Pipelined iterations (collision steps behind the scans) on or off."""
        _check(lib().sgs_set_overlap(self.h, 1 if enable else 0), "sgs_set_overlap")

    def overlap(self) -> bool:
        return bool(lib().sgs_get_overlap(self.h))

    def update_active(self, res, tol, stream=None):
        _check(lib().sgs_update_active(self.h, _ptr(res), tol, _stream(stream)), "sgs_update_active")

    def activate_all(self, stream=None):
        _check(lib().sgs_activate_all(self.h, _stream(stream)), "sgs_activate_all")

    def read_active(self, stream=None) -> list:
        a = (C.c_int * self.n_inst)()
        _check(lib().sgs_read_active(self.h, a, _stream(stream)), "sgs_read_active")
        return [int(x) for x in a]

    def sweep_shape(self):
        e, c, t = C.c_int(), C.c_int(), C.c_int()
        _check(lib().sgs_get_sweep_shape(self.h, C.byref(e), C.byref(c), C.byref(t)), "sgs_get_sweep_shape")
        return int(e.value), int(c.value), int(t.value)

    def set_sweep_shape(self, ept, cluster, threads):
        _check(lib().sgs_set_sweep_shape(self.h, ept, cluster, threads), "sgs_set_sweep_shape")

    def autotune(self, f, P, reps=1, stream=None) -> dict:
        t = _Tuning()
        _check(lib().sgs_autotune(self.h, _ptr(f), _ptr(P), reps, C.byref(t), _stream(stream)), "sgs_autotune")
        return {k: (float(getattr(t, k)) if k.endswith("_ms") else int(getattr(t, k))) for k, _ in _Tuning._fields_}

    def read_status(self, stream=None) -> dict:
        st = _Stats()
        _check(lib().sgs_read_status(self.h, C.byref(st), _stream(stream)), "sgs_read_status")
        return {k: int(getattr(st, k)) for k, _ in _Stats._fields_}

    def reset_stats(self, stream=None):
        _check(lib().sgs_reset_stats(self.h, _stream(stream)), "sgs_reset_stats")

    def close(self):
        if getattr(self, "h", None):
            lib().sgs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FastOperator:
    """The fast (Carleman-form) spectral operator of a hard-sphere Solver on the tensor cores:
    Q[f, f] of every cell (see sgs_fast_collide)."""

    def __init__(self, solver: "Solver", m_theta: int = 8, m_phi: int = 16, chunk: int = 8):
        import torch

        h = C.c_void_p()
        ws = C.c_size_t()
        _check(lib().sgs_fast_setup(solver.h, m_theta, m_phi, chunk, C.byref(h), C.byref(ws)), "sgs_fast_setup")
        self.h = h
        self.solver = solver
        self.workspace = torch.empty(max(int(ws.value), 256), dtype=torch.uint8, device=solver.device)
        _check(lib().sgs_fast_bind(self.h, self.workspace.data_ptr(), self.workspace.numel()), "sgs_fast_bind")

    def collide(self, f, Q, terms: int = 3, stream=None):
        _check(lib().sgs_fast_collide(self.h, self.solver.h, _ptr(f), _ptr(Q), terms, _stream(stream)),
               "sgs_fast_collide")

    def close(self):
        if getattr(self, "h", None):
            lib().sgs_fast_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent steady problems of mixed velocity grids solved together.

    Kernels are compiled per velocity grid, so the problems are grouped by nv: one handle
    (one persistent scan launch, one CTA cluster per instance) per group, each group on its
    own stream. A defect-correction cycle of every group is captured in one CUDA graph:
    FP64 collision and residual per instance, deactivation of the converged instances, then
    lo_iters mixed-precision SGS iterations."""

    def __init__(self, problems, device="cuda"):
        import torch

        self.problems = list(problems)
        self.groups = {}
        for i, p in enumerate(self.problems):
            self.groups.setdefault(p.nv, []).append(i)
        self.solvers, self.f, self.Q, self.P, self.res, self.streams = {}, {}, {}, {}, {}, {}
        for nv, idx in self.groups.items():
            s = Solver([self.problems[i] for i in idx], device=device)
            self.solvers[nv] = s
            self.f[nv], self.Q[nv], self.P[nv] = s.field(), s.field(), s.field()
            self.res[nv] = torch.zeros(len(idx), dtype=torch.float64, device=device)
            self.streams[nv] = torch.cuda.Stream(device=device)
        self.graph = None

    def view(self, i: int):
        """The cells of problem i inside its group's field."""
        nv = self.problems[i].nv
        return self.solvers[nv].view(self.f[nv], self.groups[nv].index(i))

    def load(self, states):
        """Copies the initial distribution of every problem (arrays of shape (nx, nv, nv, nv))."""
        import torch

        for i, x in enumerate(states):
            self.view(i).copy_(torch.as_tensor(x))
        for s in self.solvers.values():
            s.activate_all()

    def _cycle(self, lo_iters: int, tol: float):
        import torch

        cur = torch.cuda.current_stream()
        for nv, s in self.solvers.items():
            st = self.streams[nv]
            st.wait_stream(cur)
            with torch.cuda.stream(st):
                s.dc_step(self.f[nv], self.Q[nv], self.P[nv], 0, res=self.res[nv], stream=st)
                s.update_active(self.res[nv], tol, stream=st)
                for it in range(lo_iters):
                    s.iterate(self.f[nv], self.Q[nv], self.P[nv], flags=IT_P_VALID if it == 0 else 0, stream=st)
        for st in self.streams.values():
            cur.wait_stream(st)

    def autotune(self, reps: int = 1) -> dict:
        """Scan-shape autotuner per velocity grid (advances the iterates; see sgs_autotune)."""
        out = {}
        for nv, s in self.solvers.items():
            s.collide(self.f[nv], self.Q[nv], self.P[nv])
            out[nv] = s.autotune(self.f[nv], self.P[nv], reps=reps)
        return out

    def capture(self, lo_iters: int, tol: float = 1e-8):
        """Records one defect-correction cycle of all groups in a CUDA graph (after one eager
        warm-up cycle)."""
        import torch

        self._cycle(lo_iters, tol)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._cycle(lo_iters, tol)
        self.graph = g
        return g

    def step(self, lo_iters: int = 10, tol: float = 1e-8):
        """One cycle: replays the captured graph if there is one, else runs eagerly."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._cycle(lo_iters, tol)

    def residuals(self):
        """FP64 residual of every problem at the last evaluation, in problem order."""
        import torch

        torch.cuda.synchronize()
        out = [0.0] * len(self.problems)
        for nv, idx in self.groups.items():
            r = self.res[nv].cpu().tolist()
            for k, i in enumerate(idx):
                out[i] = r[k]
        return out

    def status(self) -> int:
        st = 0
        for s in self.solvers.values():
            st |= s.read_status()["status"]
        return st
