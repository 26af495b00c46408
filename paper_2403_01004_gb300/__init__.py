"""GB300 (sm_103a) solvers for the operator-split parabolic operators of a thermodynamic MHD model
under the practical time-step limit (PTL) of arXiv:2403.01004.

This package is a thin ctypes binding over the C ABI of `libparabolic.so` (declared in
`include/parabolic.h`): argument marshalling only -- every step of the computation runs in the
library's CUDA kernels.  PyTorch tensors supply device memory and the CUDA stream.  There is no
CPU fallback: if the library has not been built, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, byref, c_double, c_int32, c_int64, c_void_p

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libparabolic.so")

PB_OK, PB_EINVAL, PB_ENOMEM, PB_ECUDA, PB_ENOCONVERGE, PB_EMAXCYCLES, PB_ENONFINITE, PB_ETIMEOUT, PB_ENOTSUP = range(9)
PB_FP64, PB_FP32, PB_BF16_STORE = 0, 1, 2
PB_TC_ANISO, PB_VISC_ISO = 0, 1
PB_RKL2, PB_RKG2 = 0, 1

PB_FP64_STORE = 3
PRECISIONS = {"fp64": PB_FP64, "fp32": PB_FP32, "bf16": PB_BF16_STORE, "fp64s": PB_FP64_STORE}
SCHEMES = {"rkl2": PB_RKL2, "rkg2": PB_RKG2}
PB_PTL_FMAX, PB_PTL_FULL = 0, 1
PB_SPHERICAL, PB_CARTESIAN_PERIODIC = 0, 1
PTL_MODES = {"fmax": PB_PTL_FMAX, "full": PB_PTL_FULL}
C_TC = (5.0 / 3.0 - 1.0) / 2.0

# C function names exported by the library (kept in step with include/parabolic.h)
EXPORTS = ("pb_advance_opts_init", "pb_status_string", "pb_last_error", "parabolic_setup",
           "parabolic_update", "parabolic_destroy", "parabolic_state_size", "parabolic_dt_explicit", "parabolic_apply",
           "ptl_compute", "ptl_full_compute", "rkl2_advance", "rkl2_advance_async", "rkl2_advance_relag",
           "be_pcg_advance", "pb_profile_enable", "pb_profile_read",
           "pb_ptl_noalloc", "pb_tune_init", "pb_batch_create", "pb_batch_destroy", "pb_batch_last_error",
           "pb_batch_rkl2_advance", "pb_autotune", "pb_model_create", "pb_model_destroy", "pb_model_last_error",
           "pb_model_num_params", "pb_model_get_params", "pb_model_set_params", "pb_model_save", "pb_model_load",
           "pb_guess_features", "pb_model_forward", "pb_model_grad", "pb_model_train", "learned_guess",
           "pb_guess_smooth", "pb_guess_smooth_passes")


class PbGrid(ctypes.Structure):
    _fields_ = [("n_r", c_int32), ("n_theta", c_int32), ("n_phi", c_int32),
                ("r_face", POINTER(c_double)), ("t_face", POINTER(c_double)), ("geometry", c_int32)]


class PbOperator(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("C", c_double), ("T0", c_void_p), ("n", c_void_p),
                ("B", c_void_p * 3), ("rho", c_void_p * 3), ("nu", c_void_p * 3)]


class PbAdvanceOpts(ctypes.Structure):
    _fields_ = [("scheme", c_int32), ("use_ptl", c_int32), ("max_cycles", c_int32),
                ("ptl_floor", c_double), ("dt_cycles", POINTER(c_double)), ("n_forced", c_int32),
                ("rtol", c_double), ("max_iter", c_int32), ("fixed_iters", c_int32),
                ("check_every", c_int32), ("judge_guess", c_int32), ("mixed_precision", c_int32),
                ("inner_rtol", c_double), ("ptl_mode", c_int32), ("precond", c_int32), ("pc_degree", c_int32)]


class PbStats(ctypes.Structure):
    _fields_ = [("cycles", c_int32), ("status_cycle", c_int32), ("total_stages", c_int64),
                ("total_iters", c_int64), ("dt_explicit", c_double), ("last_dt_ptl", c_double),
                ("fmax", c_double), ("k_index", c_int64), ("final_rel_residual", c_double),
                ("cycle_capacity", c_int32), ("dt_cycle", POINTER(c_double)),
                ("work_cycle", POINTER(c_int32)), ("dt_ptl_cycle", POINTER(c_double)),
                ("k_cycle", POINTER(c_int64)), ("guess_used", c_int32),
                ("dt_full_cycle", POINTER(c_double))]


class PbKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", c_int64), ("timed_launches", c_int64),
                ("total_ms", c_double), ("bytes", c_double)]


class PbTune(ctypes.Structure):
    _fields_ = [("kchunk", c_int32), ("blocks_per_sm", c_int32), ("small_tiles", c_int32)]


class PbTrainOpts(ctypes.Structure):
    _fields_ = [("steps", c_int32), ("batch", c_int32), ("crop", c_int32), ("border", c_int32),
                ("lr", c_double), ("seed", ctypes.c_uint64)]


class ParabolicError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libparabolic.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    lib.pb_advance_opts_init.argtypes = [POINTER(PbAdvanceOpts)]
    lib.pb_advance_opts_init.restype = None
    lib.pb_status_string.argtypes = [c_int32]
    lib.pb_status_string.restype = ctypes.c_char_p
    lib.pb_last_error.argtypes = [c_void_p]
    lib.pb_last_error.restype = ctypes.c_char_p
    lib.parabolic_setup.argtypes = [POINTER(PbGrid), POINTER(PbOperator), c_int32, c_void_p, POINTER(c_void_p)]
    lib.parabolic_update.argtypes = [c_void_p, POINTER(PbOperator)]
    lib.parabolic_destroy.argtypes = [c_void_p]
    lib.parabolic_state_size.argtypes = [c_void_p, POINTER(c_int64), POINTER(c_int32)]
    lib.parabolic_dt_explicit.argtypes = [c_void_p, POINTER(c_double)]
    lib.parabolic_apply.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.ptl_compute.argtypes = [c_void_p, c_void_p, POINTER(c_double), POINTER(c_int64), POINTER(c_double)]
    lib.rkl2_advance.argtypes = [c_void_p, c_void_p, c_double, POINTER(PbAdvanceOpts), POINTER(PbStats)]
    lib.rkl2_advance_async.argtypes = [c_void_p, c_void_p, c_double, POINTER(PbAdvanceOpts)]
    lib.rkl2_advance_relag.argtypes = [c_void_p, c_void_p, c_double, POINTER(PbAdvanceOpts), POINTER(PbOperator),
                                       POINTER(PbStats)]
    lib.rkl2_advance_relag.restype = c_int32
    lib.ptl_full_compute.argtypes = [c_void_p, c_void_p, POINTER(c_double), POINTER(c_int64), POINTER(c_int32)]
    lib.be_pcg_advance.argtypes = [c_void_p, c_void_p, c_double, POINTER(PbAdvanceOpts), c_void_p, POINTER(PbStats)]
    lib.pb_ptl_noalloc.argtypes = [c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                   POINTER(c_double), POINTER(c_int64), POINTER(c_double), c_void_p]
    lib.pb_ptl_noalloc.restype = c_int32
    lib.pb_tune_init.argtypes = [POINTER(PbTune)]
    lib.pb_tune_init.restype = None
    lib.pb_batch_create.argtypes = [POINTER(c_void_p), c_int32, POINTER(PbTune), POINTER(c_void_p)]
    lib.pb_batch_destroy.argtypes = [c_void_p]
    lib.pb_batch_last_error.argtypes = [c_void_p]
    lib.pb_batch_last_error.restype = ctypes.c_char_p
    lib.pb_batch_rkl2_advance.argtypes = [c_void_p, POINTER(c_void_p), POINTER(c_double), c_int32, POINTER(PbStats)]
    lib.pb_autotune.argtypes = [c_void_p, POINTER(c_void_p), POINTER(c_double), c_int32, POINTER(PbTune),
                                POINTER(c_double)]
    for name in ("pb_batch_create", "pb_batch_destroy", "pb_batch_rkl2_advance", "pb_autotune"):
        getattr(lib, name).restype = c_int32
    lib.pb_model_create.argtypes = [ctypes.c_uint64, POINTER(c_void_p)]
    lib.pb_model_destroy.argtypes = [c_void_p]
    lib.pb_model_last_error.argtypes = [c_void_p]
    lib.pb_model_last_error.restype = ctypes.c_char_p
    lib.pb_model_num_params.argtypes = []
    lib.pb_model_get_params.argtypes = [c_void_p, POINTER(ctypes.c_float), c_int64]
    lib.pb_model_set_params.argtypes = [c_void_p, POINTER(ctypes.c_float), c_int64]
    lib.pb_model_save.argtypes = [c_void_p, ctypes.c_char_p]
    lib.pb_model_load.argtypes = [c_void_p, ctypes.c_char_p]
    lib.pb_guess_features.argtypes = [c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_void_p, POINTER(c_double)]
    lib.pb_model_forward.argtypes = [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p, c_void_p]
    lib.pb_model_grad.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32,
                                  POINTER(c_double), POINTER(ctypes.c_float), c_void_p]
    lib.pb_model_train.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32,
                                   POINTER(PbTrainOpts), POINTER(c_double), c_void_p]
    lib.learned_guess.argtypes = [c_void_p, c_void_p, c_void_p, c_double, c_void_p]
    lib.pb_guess_smooth.argtypes = [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_int32,
                                    c_void_p]
    lib.pb_guess_smooth.restype = c_int32
    lib.pb_guess_smooth_passes.argtypes = []
    lib.pb_guess_smooth_passes.restype = c_int32
    for name in ("pb_model_create", "pb_model_destroy", "pb_model_num_params", "pb_model_get_params",
                 "pb_model_set_params", "pb_model_save", "pb_model_load", "pb_guess_features", "pb_model_forward",
                 "pb_model_grad", "pb_model_train", "learned_guess"):
        getattr(lib, name).restype = c_int32
    lib.pb_profile_enable.argtypes = [c_void_p, c_int32]
    lib.pb_profile_read.argtypes = [c_void_p, POINTER(PbKernelStat), c_int32, POINTER(c_int32)]
    for name in ("pb_profile_enable", "pb_profile_read", "parabolic_setup", "parabolic_update", "parabolic_destroy", "parabolic_state_size", "parabolic_dt_explicit",
                 "parabolic_apply", "ptl_compute", "rkl2_advance", "be_pcg_advance"):
        getattr(lib, name).restype = c_int32
    _lib = lib
    return lib


def _check(status: int, ctx_handle=None):
    if status != PB_OK:
        lib = load_library()
        msg = lib.pb_last_error(ctx_handle).decode() if lib.pb_last_error(ctx_handle) else ""
        raise ParabolicError(status, f"{lib.pb_status_string(status).decode()}: {msg}")


def _torch():
    import torch
    return torch


def _ptr(t) -> int:
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream_handle(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Context:
    """An operator set up on a grid (owns the library context and its device workspace)."""

    def __init__(self, handle, kind, precision, stream, n, elem):
        self.handle = handle
        self.kind = kind
        self.precision = precision
        self.stream = stream
        self.n = n
        self.elem = elem

    @property
    def dtype(self):
        torch = _torch()
        return {PB_FP64: torch.float64, PB_FP32: torch.float32, PB_BF16_STORE: torch.bfloat16,
                PB_FP64_STORE: torch.float64}[self.precision]

    def close(self):
        if self.handle:
            load_library().parabolic_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def parabolic_setup(r_face, t_face, n_phi: int, kind: str, fields: dict, precision: str = "fp64",
                    C: float = C_TC, stream=None) -> Context:
    """Builds a context on the spherical shell.  kind = "tc" with fields T0, n, B (3 tensors at
    corners), or kind = "visc" with fields rho, nu (lists of 3 tensors); fields are float64 CUDA
    tensors."""
    rf = (c_double * len(r_face))(*[float(x) for x in r_face])
    tf = (c_double * len(t_face))(*[float(x) for x in t_face])
    g = PbGrid(len(r_face) - 1, len(t_face) - 1, int(n_phi), ctypes.cast(rf, POINTER(c_double)),
               ctypes.cast(tf, POINTER(c_double)), PB_SPHERICAL)
    return _setup(g, kind, fields, precision, C, stream)


def parabolic_setup_box(n_r: int, n_theta: int, n_phi: int, kind: str, fields: dict, precision: str = "fp64",
                        C: float = C_TC, stream=None) -> Context:
    """Builds a context on the periodic box of unit cells (PB_CARTESIAN_PERIODIC); fields as for
    the shell, every viscosity component on the full n_r x n_theta x n_phi grid."""
    g = PbGrid(int(n_r), int(n_theta), int(n_phi), None, None, PB_CARTESIAN_PERIODIC)
    return _setup(g, kind, fields, precision, C, stream)


def _setup(g, kind, fields, precision, C, stream) -> Context:
    lib = load_library()
    torch = _torch()
    op, keep = _operator(kind, fields, C)
    h = c_void_p()
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib.parabolic_setup(byref(g), byref(op), PRECISIONS[precision], c_void_p(_stream_handle(st)), byref(h)))
    n = c_int64()
    e = c_int32()
    _check(lib.parabolic_state_size(h, byref(n), byref(e)), h)
    ctx = Context(h, kind, PRECISIONS[precision], st, n.value, e.value)
    ctx.C = float(C)
    return ctx


def _operator(kind: str, fields: dict, C: float):
    torch = _torch()
    op = PbOperator()
    keep = []

    def dptr(t):
        if t.dtype != torch.float64:
            raise TypeError("operator fields must be float64")
        keep.append(t)
        return _ptr(t)

    if kind == "tc":
        op.kind = PB_TC_ANISO
        op.C = float(C)
        op.T0 = dptr(fields["T0"])
        op.n = dptr(fields["n"])
        for a in range(3):
            op.B[a] = dptr(fields["B"][a])
    elif kind == "visc":
        op.kind = PB_VISC_ISO
        for a in range(3):
            op.rho[a] = dptr(fields["rho"][a])
            op.nu[a] = dptr(fields["nu"][a])
    else:
        raise ValueError(kind)
    return op, keep


def parabolic_update(ctx: Context, fields: dict) -> None:
    """Recomputes the frozen coefficients and dt_E in place from new operator fields."""
    op, keep = _operator(ctx.kind, fields, getattr(ctx, "C", C_TC))
    _check(load_library().parabolic_update(ctx.handle, byref(op)), ctx.handle)


def parabolic_dt_explicit(ctx: Context) -> float:
    v = c_double()
    _check(load_library().parabolic_dt_explicit(ctx.handle, byref(v)), ctx.handle)
    return v.value


def _check_state(ctx: Context, u):
    if u.numel() != ctx.n or u.dtype != ctx.dtype:
        raise ValueError(f"state must have {ctx.n} elements of {ctx.dtype}")


def parabolic_apply(ctx: Context, u, F=None):
    """F = L u (device tensors of the context precision)."""
    _check_state(ctx, u)
    if F is None:
        F = _torch().empty_like(u)
    _check(load_library().parabolic_apply(ctx.handle, c_void_p(_ptr(u)), c_void_p(_ptr(F))), ctx.handle)
    return F


def ptl_compute(ctx: Context, u):
    """Returns (dt_PTL, k, |F_k|) for state u (Eq. 5)."""
    _check_state(ctx, u)
    dt, k, fm = c_double(), c_int64(), c_double()
    _check(load_library().ptl_compute(ctx.handle, c_void_p(_ptr(u)), byref(dt), byref(k), byref(fm)), ctx.handle)
    return dt.value, k.value, fm.value


def ptl_full_compute(ctx: Context, u):
    """Returns (dt, cell, direction): Eq. 4 over every pair of face neighbours of state u (the PTL
    without the F_max localisation); the pair is (cell, cell + e_direction), direction 0 r,
    1 theta, 2 phi; (inf, -1, -1) when no pair qualifies."""
    _check_state(ctx, u)
    dt, cell, d = c_double(), c_int64(), c_int32()
    _check(load_library().ptl_full_compute(ctx.handle, c_void_p(_ptr(u)), byref(dt), byref(cell), byref(d)),
           ctx.handle)
    return dt.value, cell.value, d.value


PRECONDS = {"jacobi": 0, "chebyshev": 1}


def _opts(scheme="rkl2", use_ptl=True, max_cycles=0, ptl_floor=1.0, forced=None, rtol=1e-10,
          max_iter=100000, fixed_iters=0, check_every=8, judge_guess=True, mixed=False, inner_rtol=1e-6,
          ptl_mode="fmax", precond="jacobi", pc_degree=3):
    lib = load_library()
    o = PbAdvanceOpts()
    lib.pb_advance_opts_init(byref(o))
    o.scheme = SCHEMES[scheme]
    o.use_ptl = 1 if use_ptl else 0
    o.max_cycles = int(max_cycles)
    o.ptl_floor = float(ptl_floor)
    keep = None
    if forced is not None:
        keep = (c_double * len(forced))(*[float(x) for x in forced])
        o.dt_cycles = ctypes.cast(keep, POINTER(c_double))
        o.n_forced = len(forced)
    o.rtol = float(rtol)
    o.max_iter = int(max_iter)
    o.fixed_iters = int(fixed_iters)
    o.check_every = int(check_every)
    o.judge_guess = 1 if judge_guess else 0
    o.mixed_precision = 1 if mixed else 0
    o.inner_rtol = float(inner_rtol)
    o.ptl_mode = PTL_MODES[ptl_mode]
    o.precond = PRECONDS[precond]
    o.pc_degree = int(pc_degree)
    return o, keep


class _StatsBuf:
    def __init__(self, cap: int, record_full: bool = False):
        self.cap = cap
        self.full = (c_double * cap)() if record_full else None
        self.dt = (c_double * cap)()
        self.work = (c_int32 * cap)()
        self.dtp = (c_double * cap)()
        self.k = (c_int64 * cap)()
        self.st = PbStats()
        self.st.cycle_capacity = cap
        self.st.dt_cycle = ctypes.cast(self.dt, POINTER(c_double))
        self.st.work_cycle = ctypes.cast(self.work, POINTER(c_int32))
        self.st.dt_ptl_cycle = ctypes.cast(self.dtp, POINTER(c_double))
        self.st.k_cycle = ctypes.cast(self.k, POINTER(c_int64))
        if self.full is not None:
            self.st.dt_full_cycle = ctypes.cast(self.full, POINTER(c_double))

    def as_dict(self) -> dict:
        s = self.st
        n = min(s.cycles, self.cap)
        return dict(cycles=s.cycles, total_stages=s.total_stages, total_iters=s.total_iters,
                    dt_explicit=s.dt_explicit, last_dt_ptl=s.last_dt_ptl, fmax=s.fmax, k_index=s.k_index,
                    final_rel_residual=s.final_rel_residual, status_cycle=s.status_cycle,
                    dt_cycle=list(self.dt[:n]), work_cycle=list(self.work[:n]),
                    dt_ptl_cycle=list(self.dtp[:n]), k_cycle=list(self.k[:n]), guess_used=s.guess_used,
                    dt_full_cycle=list(self.full[:n]) if self.full is not None else None)


def rkl2_advance(ctx: Context, u, dt: float, scheme: str = "rkl2", use_ptl: bool = True,
                 forced=None, max_cycles: int = 0, ptl_floor: float = 1.0, stats_capacity: int = 4096,
                 raise_on_error: bool = True, ptl_mode: str = "fmax", record_full: bool = False) -> dict:
    """Advances u in place over dt with RKL2 / RKG2 under PTL cycling; returns the statistics.
    ptl_mode "full" sets the cycles from Eq. 4 over every pair of neighbours instead of Eq. 5;
    record_full also evaluates that value before every cycle (stats "dt_full_cycle")."""
    _check_state(ctx, u)
    o, keep = _opts(scheme, use_ptl, max_cycles, ptl_floor, forced, ptl_mode=ptl_mode)
    sb = _StatsBuf(stats_capacity, record_full)
    rc = load_library().rkl2_advance(ctx.handle, c_void_p(_ptr(u)), float(dt), byref(o), byref(sb.st))
    d = sb.as_dict()
    d["status"] = rc
    if raise_on_error:
        _check(rc, ctx.handle)
    return d


def rkl2_advance_relag(ctx: Context, u, dt: float, fields: dict, scheme: str = "rkl2", use_ptl: bool = True,
                       forced=None, max_cycles: int = 0, ptl_floor: float = 1.0, stats_capacity: int = 4096,
                       raise_on_error: bool = True) -> dict:
    """Non-linear conduction: like rkl2_advance, with the coefficients recomputed before every
    cycle from kappa = max(T, 0)^{5/2} of the current state; fields gives n and B (float64 CUDA
    tensors; T0 is not read)."""
    _check_state(ctx, u)
    if ctx.kind != "tc":
        raise ValueError("the re-lag is for conduction contexts")
    f = dict(fields)
    f.setdefault("T0", f["n"])
    op, keep_op = _operator("tc", f, getattr(ctx, "C", C_TC))
    o, keep = _opts(scheme, use_ptl, max_cycles, ptl_floor, forced)
    sb = _StatsBuf(stats_capacity)
    rc = load_library().rkl2_advance_relag(ctx.handle, c_void_p(_ptr(u)), float(dt), byref(o), byref(op), byref(sb.st))
    d = sb.as_dict()
    d["status"] = rc
    if raise_on_error:
        _check(rc, ctx.handle)
    return d


def rkl2_advance_async(ctx: Context, u, dt: float, scheme: str = "rkl2", forced=None, use_ptl: bool = True) -> None:
    """Enqueues a forced schedule, or one cycle of dt with use_ptl=False, on the context's stream
    and returns at once: no host reads, no allocation, capturable in a CUDA graph.  The PTL
    (use_ptl without a forced schedule) is refused."""
    _check_state(ctx, u)
    o, keep = _opts(scheme, use_ptl, 0, 1.0, forced)
    _check(load_library().rkl2_advance_async(ctx.handle, c_void_p(_ptr(u)), float(dt), byref(o)), ctx.handle)


def be_pcg_advance(ctx: Context, u, dt: float, use_ptl: bool = True, forced=None, rtol: float = 1e-10,
                   max_iter: int = 100000, fixed_iters: int = 0, x0=None, max_cycles: int = 0,
                   ptl_floor: float = 1.0, check_every: int = 8, stats_capacity: int = 4096,
                   raise_on_error: bool = True, judge_guess: bool = True, mixed: bool = False,
                   inner_rtol: float = 1e-6, ptl_mode: str = "fmax", record_full: bool = False,
                   precond: str = "jacobi", pc_degree: int = 3) -> dict:
    """Advances u in place over dt with Backward Euler + PCG under PTL cycling, preconditioned by
    point-Jacobi (precond "jacobi", PC1) or by the degree-pc_degree Chebyshev polynomial in
    D^-1 S ("chebyshev").  With x0 (first cycle's initial guess) and judge_guess, the solve
    starts from whichever of x0 and u has the smaller initial residual."""
    _check_state(ctx, u)
    o, keep = _opts("rkl2", use_ptl, max_cycles, ptl_floor, forced, rtol, max_iter, fixed_iters, check_every,
                    judge_guess, mixed, inner_rtol, ptl_mode, precond, pc_degree)
    sb = _StatsBuf(stats_capacity, record_full)
    x0p = c_void_p(_ptr(x0)) if x0 is not None else c_void_p(0)
    rc = load_library().be_pcg_advance(ctx.handle, c_void_p(_ptr(u)), float(dt), byref(o), x0p, byref(sb.st))
    d = sb.as_dict()
    d["status"] = rc
    if raise_on_error:
        _check(rc, ctx.handle)
    return d


def pb_profile_enable(ctx: Context, on: bool = True) -> None:
    """Resets the context's kernel counters; on=True also times every launch with CUDA events."""
    _check(load_library().pb_profile_enable(ctx.handle, 1 if on else 0), ctx.handle)


def pb_profile_read(ctx: Context) -> list:
    """Per kernel class: name, launches, timed launches, total milliseconds, algorithmic bytes."""
    buf = (PbKernelStat * 16)()
    n = c_int32()
    _check(load_library().pb_profile_read(ctx.handle, buf, 16, byref(n)), ctx.handle)
    return [dict(name=buf[i].name.decode(), launches=buf[i].launches, timed_launches=buf[i].timed_launches,
                 total_ms=buf[i].total_ms, bytes=buf[i].bytes) for i in range(n.value)]


class Batch:
    """Many float32 conduction contexts advanced together by one persistent graph launch."""

    def __init__(self, handle, ctxs):
        self.handle = handle
        self.ctxs = list(ctxs)   # kept alive: the batch uses their buffers

    def close(self):
        if self.handle:
            load_library().pb_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _bcheck(status: int, handle):
    if status != PB_OK:
        lib = load_library()
        raise ParabolicError(status, f"{lib.pb_status_string(status).decode()}: "
                                     f"{lib.pb_batch_last_error(handle).decode()}")


def pb_batch_create(ctxs, tune: dict | None = None) -> Batch:
    lib = load_library()
    arr = (c_void_p * len(ctxs))(*[c.handle for c in ctxs])
    t = None
    if tune is not None:
        t = PbTune(int(tune["kchunk"]), int(tune["blocks_per_sm"]), int(tune["small_tiles"]))
    h = c_void_p()
    _bcheck(lib.pb_batch_create(arr, len(ctxs), byref(t) if t is not None else None, byref(h)), None)
    return Batch(h, ctxs)


def _uptrs(batch, us):
    if len(us) != len(batch.ctxs):
        raise ValueError("one state per context")
    for c, u in zip(batch.ctxs, us):
        _check_state(c, u)
    return (c_void_p * len(us))(*[_ptr(u) for u in us])


def pb_batch_rkl2_advance(batch: Batch, us, dts, scheme: str = "rkl2") -> list:
    """Advances every us[p] in place over dts[p] (one cycle each) in one graph launch."""
    lib = load_library()
    n = len(us)
    st = (PbStats * n)()
    d = (c_double * n)(*[float(x) for x in dts])
    _bcheck(lib.pb_batch_rkl2_advance(batch.handle, _uptrs(batch, us), d, SCHEMES[scheme], st), batch.handle)
    return [dict(cycles=st[p].cycles, total_stages=st[p].total_stages) for p in range(n)]


def pb_autotune(batch: Batch, us, dts, scheme: str = "rkl2"):
    """Times the candidate schedules on copies of the states; returns (tune, best ms)."""
    lib = load_library()
    n = len(us)
    d = (c_double * n)(*[float(x) for x in dts])
    t = PbTune()
    ms = c_double()
    _bcheck(lib.pb_autotune(batch.handle, _uptrs(batch, us), d, SCHEMES[scheme], byref(t), byref(ms)), batch.handle)
    return dict(kchunk=t.kchunk, blocks_per_sm=t.blocks_per_sm, small_tiles=t.small_tiles), ms.value


class Model:
    """The learned-guess network (device parameters owned by the library)."""

    def __init__(self, seed: int = 0):
        lib = load_library()
        h = c_void_p()
        _mcheck(lib.pb_model_create(int(seed), byref(h)), None)
        self.handle = h

    def close(self):
        if self.handle:
            load_library().pb_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def num_params() -> int:
        return load_library().pb_model_num_params()

    def get_params(self):
        import numpy as np
        out = np.empty(self.num_params(), dtype=np.float32)
        _mcheck(load_library().pb_model_get_params(self.handle, out.ctypes.data_as(POINTER(ctypes.c_float)), out.size),
                self.handle)
        return out

    def set_params(self, params):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        _mcheck(load_library().pb_model_set_params(self.handle, a.ctypes.data_as(POINTER(ctypes.c_float)), a.size),
                self.handle)

    def save(self, path: str):
        _mcheck(load_library().pb_model_save(self.handle, path.encode()), self.handle)

    def load(self, path: str):
        _mcheck(load_library().pb_model_load(self.handle, path.encode()), self.handle)


def _mcheck(status: int, handle):
    if status != PB_OK:
        lib = load_library()
        raise ParabolicError(status, f"{lib.pb_status_string(status).decode()}: "
                                     f"{lib.pb_model_last_error(handle).decode()}")


def pb_guess_features(ctx: Context, u, dt: float, x=None):
    """(features [n_phi, n_theta, n_r, 16] bf16, target or None, S) for state u and BE step dt;
    with the solved state x the training target (x - u)/S is returned too."""
    torch = _torch()
    _check_state(ctx, u)
    feats = torch.empty(ctx.n * 16, dtype=torch.bfloat16, device=u.device)
    target = torch.empty(ctx.n, dtype=torch.float32, device=u.device) if x is not None else None
    S = c_double()
    _check(load_library().pb_guess_features(ctx.handle, c_void_p(_ptr(u)), float(dt),
                                            c_void_p(_ptr(x)) if x is not None else c_void_p(0), c_void_p(_ptr(feats)),
                                            c_void_p(_ptr(target)) if target is not None else c_void_p(0), byref(S)),
           ctx.handle)
    return feats, target, S.value


def pb_model_forward(model: Model, feats, shape, wrap_d: bool = False):
    """Network output (float32) for feats of shape (samples, D, H, W) x 16 channels."""
    torch = _torch()
    S_, D, H, W = shape
    out = torch.empty(S_ * D * H * W, dtype=torch.float32, device=feats.device)
    _mcheck(load_library().pb_model_forward(model.handle, c_void_p(_ptr(feats)), S_, D, H, W, int(wrap_d),
                                            c_void_p(_ptr(out)), c_void_p(_stream_handle(None))), model.handle)
    return out


def pb_model_grad(model: Model, feats, target, mask, shape):
    """(loss, gradient wrt every parameter as a float32 numpy array)."""
    import numpy as np
    S_, D, H, W = shape
    g = np.empty(Model.num_params(), dtype=np.float32)
    L = c_double()
    _mcheck(load_library().pb_model_grad(model.handle, c_void_p(_ptr(feats)), c_void_p(_ptr(target)),
                                         c_void_p(_ptr(mask)), S_, D, H, W, byref(L),
                                         g.ctypes.data_as(POINTER(ctypes.c_float)), c_void_p(_stream_handle(None))),
            model.handle)
    return L.value, g


def pb_model_train(model: Model, feats, targets, shape, steps: int, batch: int = 8, crop: int = 24, border: int = 4,
                   lr: float = 1e-3, seed: int = 0) -> float:
    """Adam on random crops of the samples (feats (N, D, H, W, 16) bf16, targets (N, D, H, W))."""
    N, D, H, W = shape
    o = PbTrainOpts(int(steps), int(batch), int(crop), int(border), float(lr), int(seed))
    L = c_double()
    _mcheck(load_library().pb_model_train(model.handle, c_void_p(_ptr(feats)), c_void_p(_ptr(targets)), N, D, H, W,
                                          byref(o), byref(L), c_void_p(_stream_handle(None))), model.handle)
    return L.value


def learned_guess(ctx: Context, model: Model, u, dt: float, x0=None):
    """x0 = u + S model(features(u, dt)) for a conduction context."""
    _check_state(ctx, u)
    if x0 is None:
        x0 = _torch().empty_like(u)
    _check(load_library().learned_guess(ctx.handle, model.handle, c_void_p(_ptr(u)), float(dt), c_void_p(_ptr(x0))),
           ctx.handle)
    return x0


__all__ = ["Model", "pb_guess_features", "pb_model_forward", "pb_model_grad", "pb_model_train", "learned_guess", "Batch", "pb_batch_create", "pb_batch_rkl2_advance", "pb_autotune", "pb_profile_enable", "pb_profile_read", "parabolic_setup", "parabolic_update", "parabolic_dt_explicit", "parabolic_apply", "ptl_compute", "rkl2_advance",
           "be_pcg_advance", "Context", "ParabolicError", "load_library", "EXPORTS"]


def pb_guess_smooth(x, shape, wrap_d: bool = True, passes: int | None = None, stream=None):
    """x (float32 CUDA tensor of S x D x H x W values) smoothed as learned_guess smooths the network
    output (passes defaults to the library's); returns a new tensor."""
    torch = _torch()
    if x.dtype != torch.float32:
        raise TypeError("float32 fields")
    lib = load_library()
    S_, D, H, W = (int(v) for v in shape)
    out = torch.empty_like(x)
    tmp = torch.empty_like(x)
    n = lib.pb_guess_smooth_passes() if passes is None else int(passes)
    _check(lib.pb_guess_smooth(c_void_p(_ptr(x)), c_void_p(_ptr(out)), c_void_p(_ptr(tmp)), S_, D, H, W,
                               1 if wrap_d else 0, n, c_void_p(_stream_handle(stream))))
    return out
