"""Thin ctypes binding of libmm (include/mm.h).  Argument marshalling only.

Every computation runs in the CUDA library; this module converts torch tensors to pointers and
status codes to exceptions.  Importing it without a built libmm.so raises immediately: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libmm.so")

MM_OK, MM_EINVAL, MM_ENOMEM, MM_ENOTSPD, MM_EBREAKDOWN, MM_ENOTCONV, MM_ETIMEOUT, MM_EBUSY, \
    MM_ECUDA = range(9)
MM_FP64, MM_FP32, MM_DF64, MM_FP32_DF64 = 0, 1, 2, 3
MM_TPLZ_AUTO, MM_TPLZ_FFT, MM_TPLZ_GEMM, MM_TPLZ_DIRECT = 0, 1, 2, 3
MM_PREC_BD, MM_PREC_2LVL_POST = 0, 1
MM_ECG_ORTHOMIN, MM_ECG_ORTHODIR = 0, 1
STATUS_NAMES = {0: "MM_OK", 1: "MM_EINVAL", 2: "MM_ENOMEM", 3: "MM_ENOTSPD", 4: "MM_EBREAKDOWN",
                5: "MM_ENOTCONV", 6: "MM_ETIMEOUT", 7: "MM_EBUSY", 8: "MM_ECUDA"}

# the exported entry points of include/mm.h
EXPORTS = ("mm_plan", "mm_plan_query", "mm_plan_destroy", "mm_apply_P", "mm_apply_Pt",
           "mm_apply_Ninv", "mm_rhs", "mm_apply_A", "mm_precond", "mm_pcg_solve", "mm_last_error",
           "mm_apply_A_noalloc", "mm_block_cg_solve", "mm_ecg_solve", "mm_deflation_build", "mm_deflation_build_apriori", "mm_deflation_get",
           "mm_deflation_apply", "mm_server_create", "mm_submit", "mm_poll", "mm_wait",
           "mm_server_destroy", "mm_estimate_bands", "mm_templates_set", "mm_solve_tod", "mm_autotune")


class TemplatesDesc(ctypes.Structure):
    _fields_ = [("n_poly", ctypes.c_int32), ("n_az", ctypes.c_int32), ("n_hwp", ctypes.c_int32),
                ("az_interp", ctypes.c_int32), ("az", ctypes.c_void_p), ("hwp", ctypes.c_void_p),
                ("inputs_on_device", ctypes.c_int32)]


class ProblemDesc(ctypes.Structure):
    _fields_ = [("n_det", ctypes.c_int32), ("n_int", ctypes.c_int32),
                ("block_len", ctypes.POINTER(ctypes.c_int64)), ("n_pix", ctypes.c_int64),
                ("pix", ctypes.c_void_p), ("psi", ctypes.c_void_p), ("lambda_", ctypes.c_int32),
                ("band", ctypes.c_void_p), ("cond_max", ctypes.c_double),
                ("precision", ctypes.c_int32), ("toeplitz_algo", ctypes.c_int32),
                ("inputs_on_device", ctypes.c_int32), ("tile_steps", ctypes.c_int32),
                ("pt_sub", ctypes.c_int32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("reliable_every", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("deadline_us", ctypes.c_int64)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("rel_res", ctypes.c_double),
                ("true_rel_res", ctypes.c_double), ("t_ms", ctypes.c_double),
                ("n_true_res", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("t_apply32_ms", ctypes.c_double), ("t_apply64_ms", ctypes.c_double),
                ("n_apply32", ctypes.c_int32), ("n_apply64", ctypes.c_int32),
                ("n_kernels", ctypes.c_int64), ("t_queue_ms", ctypes.c_double),
                ("t_unpoint32_ms", ctypes.c_double), ("t_point32_ms", ctypes.c_double)]


class TuneInfo(ctypes.Structure):
    _fields_ = [("tile_steps", ctypes.c_int32), ("win_samples", ctypes.c_int32), ("block_width", ctypes.c_int32),
                ("n_steps", ctypes.c_int32), ("n_win", ctypes.c_int32), ("n_width", ctypes.c_int32),
                ("steps_cand", ctypes.c_int32 * 8), ("steps_ms", ctypes.c_double * 8),
                ("win_cand", ctypes.c_int32 * 8), ("win_ms", ctypes.c_double * 8),
                ("width_cand", ctypes.c_int32 * 8), ("width_ms_per_col", ctypes.c_double * 8),
                ("apply_ms", ctypes.c_double), ("big_tiles", ctypes.c_int32), ("big_tiles_ms", ctypes.c_double),
                ("max_rel_dev", ctypes.c_double), ("n_rejected", ctypes.c_int32),
                ("seg_sub", ctypes.c_int32), ("n_seg", ctypes.c_int32), ("seg_cand", ctypes.c_int32 * 4),
                ("seg_ms", ctypes.c_double * 4)]


class MMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libmm.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    lib.mm_plan.argtypes = [ctypes.POINTER(ProblemDesc), vp, ctypes.POINTER(vp)]
    lib.mm_plan_query.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(vp), ctypes.POINTER(i64),
                                  ctypes.POINTER(ctypes.c_size_t)]
    lib.mm_plan_destroy.argtypes = [vp]
    lib.mm_plan_destroy.restype = None
    for name in ("mm_apply_P", "mm_apply_Pt", "mm_apply_Ninv"):
        getattr(lib, name).argtypes = [vp, vp, vp, vp]
    lib.mm_rhs.argtypes = [vp, vp, i32, i32, vp, vp]
    lib.mm_apply_A.argtypes = [vp, vp, vp, i32, vp]
    lib.mm_apply_A_noalloc.argtypes = [vp, vp, vp, i32, vp]
    lib.mm_precond.argtypes = [vp, vp, vp, i32, vp]
    lib.mm_pcg_solve.argtypes = [vp, vp, vp, i32, ctypes.POINTER(SolveOpts),
                                 ctypes.POINTER(SolveInfo), vp]
    lib.mm_block_cg_solve.argtypes = [vp, vp, vp, i32, i32, ctypes.POINTER(SolveOpts),
                                      ctypes.POINTER(SolveInfo), vp]
    lib.mm_solve_tod.argtypes = [vp, vp, i32, vp, i32, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp]
    lib.mm_autotune.argtypes = [vp, i32, ctypes.POINTER(TuneInfo), vp]
    lib.mm_ecg_solve.argtypes = [vp, vp, vp, i32, i32, ctypes.POINTER(SolveOpts),
                                 ctypes.POINTER(SolveInfo), vp]
    lib.mm_deflation_build.argtypes = [vp, vp, i32, i32, vp]
    lib.mm_deflation_build_apriori.argtypes = [vp, i32, vp]
    lib.mm_estimate_bands.argtypes = [i32, i32, vp, vp, vp, i32, vp, vp, vp]
    lib.mm_templates_set.argtypes = [vp, ctypes.POINTER(TemplatesDesc), vp]
    lib.mm_deflation_get.argtypes = [vp, ctypes.POINTER(ctypes.c_int), vp, vp, vp]
    lib.mm_deflation_apply.argtypes = [vp, vp, vp, i32, vp]
    lib.mm_server_create.argtypes = [ctypes.c_size_t, i32, ctypes.POINTER(vp)]
    lib.mm_submit.argtypes = [vp, ctypes.POINTER(ProblemDesc), vp, ctypes.c_int, ctypes.POINTER(SolveOpts),
                              ctypes.POINTER(i64)]
    lib.mm_poll.argtypes = [vp, i64, ctypes.POINTER(SolveInfo)]
    lib.mm_wait.argtypes = [vp, i64, i64, vp, ctypes.POINTER(SolveInfo)]
    lib.mm_server_destroy.argtypes = [vp]
    lib.mm_server_destroy.restype = None
    lib.mm_last_error.restype = ctypes.c_char_p
    for n in EXPORTS:
        if n not in ("mm_plan_destroy", "mm_last_error", "mm_server_destroy"):
            getattr(lib, n).restype = ctypes.c_int
    return lib


_lib = _load()


def lib():
    return _lib


def mm_last_error() -> str:
    return _lib.mm_last_error().decode()


def _check(code: int):
    if code != MM_OK:
        raise MMError(code, mm_last_error())


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _dev(t: torch.Tensor, dtype: torch.dtype, name: str):
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    return t


@dataclass
class Plan:
    handle: int
    n_obs: int
    n_samples: int
    obs_to_global: torch.Tensor   # int32 [n_obs] (copy, on the plan's device)
    bytes: int

    def __del__(self):
        try:
            if self.handle:
                _lib.mm_plan_destroy(ctypes.c_void_p(self.handle))
                self.handle = 0
        except Exception:
            pass

    def destroy(self):
        if self.handle:
            _lib.mm_plan_destroy(ctypes.c_void_p(self.handle))
            self.handle = 0


def mm_plan(n_det: int, n_int: int, block_len: Sequence[int], n_pix: int, pix: torch.Tensor,
            psi: torch.Tensor, lam: int, band: torch.Tensor, cond_max: float = 1e3,
            precision: int = MM_FP64, toeplitz_algo: int = MM_TPLZ_AUTO, tile_steps: int = 0,
            pt_sub: int = 0, stream=None) -> Plan:
    """Build a plan.  pix/psi/band are either all CUDA tensors or all CPU tensors."""
    on_dev = pix.is_cuda
    if (psi.is_cuda != on_dev) or (band.is_cuda != on_dev):
        raise ValueError("pix, psi and band must all be on the device or all on the host")
    for t, dt, nm in ((pix, torch.int32, "pix"), (psi, torch.float32, "psi"),
                      (band, torch.float64, "band")):
        if t.dtype != dt or not t.is_contiguous():
            raise TypeError(f"{nm} must be a contiguous {dt} tensor")
    bl = (ctypes.c_int64 * len(block_len))(*[int(v) for v in block_len])
    d = ProblemDesc(n_det=n_det, n_int=n_int, block_len=bl, n_pix=n_pix, pix=_ptr(pix),
                    psi=_ptr(psi), lambda_=lam, band=_ptr(band), cond_max=cond_max,
                    precision=precision, toeplitz_algo=toeplitz_algo,
                    inputs_on_device=1 if on_dev else 0, tile_steps=tile_steps, pt_sub=pt_sub)
    h = ctypes.c_void_p()
    _check(_lib.mm_plan(ctypes.byref(d), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h)))
    n_obs = ctypes.c_int64()
    o2g = ctypes.c_void_p()
    ns = ctypes.c_int64()
    nb = ctypes.c_size_t()
    _check(_lib.mm_plan_query(h, ctypes.byref(n_obs), ctypes.byref(o2g), ctypes.byref(ns),
                              ctypes.byref(nb)))
    dev = torch.device("cuda", torch.cuda.current_device())
    o2g_t = torch.empty(n_obs.value, dtype=torch.int32, device=dev)
    if n_obs.value:
        cuda_copy_dtod(o2g_t.data_ptr(), o2g.value, 4 * n_obs.value)
    return Plan(handle=h.value, n_obs=n_obs.value, n_samples=ns.value, obs_to_global=o2g_t,
                bytes=nb.value)


def cuda_copy_dtod(dst: int, src: int, nbytes: int):
    """Device-to-device copy of raw pointers (marshalling of the plan's pixel map)."""
    class _Arr:
        def __init__(self, ptr, n):
            self.__cuda_array_interface__ = {"shape": (n,), "typestr": "|u1", "data": (ptr, False),
                                             "version": 3}
    d = torch.as_tensor(_Arr(dst, nbytes), device="cuda")
    s = torch.as_tensor(_Arr(src, nbytes), device="cuda")
    d.copy_(s)


def mm_apply_P(plan: Plan, x: torch.Tensor, t: torch.Tensor, stream=None):
    _dev(x, torch.float64, "x"); _dev(t, torch.float64, "t")
    _check(_lib.mm_apply_P(ctypes.c_void_p(plan.handle), _ptr(x), _ptr(t), _stream_ptr(stream)))


def mm_apply_Pt(plan: Plan, t: torch.Tensor, y: torch.Tensor, stream=None):
    _dev(t, torch.float64, "t"); _dev(y, torch.float64, "y")
    _check(_lib.mm_apply_Pt(ctypes.c_void_p(plan.handle), _ptr(t), _ptr(y), _stream_ptr(stream)))


def mm_apply_Ninv(plan: Plan, t: torch.Tensor, y: torch.Tensor, stream=None):
    _dev(t, torch.float64, "t"); _dev(y, torch.float64, "y")
    _check(_lib.mm_apply_Ninv(ctypes.c_void_p(plan.handle), _ptr(t), _ptr(y), _stream_ptr(stream)))


def mm_rhs(plan: Plan, d: torch.Tensor, b: torch.Tensor, stream=None):
    """b [nrhs, n_obs, 3] (or [n_obs, 3]) = P~^T N^-1 G d for d [nrhs, N] (or [N]).  d may be a CUDA
    tensor or a CPU tensor (pinned or pageable); a CPU d is copied by the library and the call
    returns once it has been read."""
    if d.dtype not in (torch.float64, torch.float32):
        raise TypeError("d must be float64 or float32")
    if not d.is_contiguous():
        raise ValueError("d must be contiguous")
    _dev(b, torch.float64, "b")
    nrhs = 1 if d.dim() == 1 else d.shape[0]
    _check(_lib.mm_rhs(ctypes.c_void_p(plan.handle), _ptr(d), 1 if d.dtype == torch.float32 else 0,
                       nrhs, _ptr(b), _stream_ptr(stream)))


def mm_apply_A(plan: Plan, x: torch.Tensor, y: torch.Tensor, stream=None):
    _dev(x, torch.float64, "x"); _dev(y, torch.float64, "y")
    nrhs = 1 if x.dim() <= 2 else x.shape[0]
    _check(_lib.mm_apply_A(ctypes.c_void_p(plan.handle), _ptr(x), _ptr(y), nrhs, _stream_ptr(stream)))


def mm_apply_A_noalloc(plan: Plan, x: torch.Tensor, y: torch.Tensor, stream=None):
    """y = A x without any device allocation by the library (working space is a fixed 32 MiB
    array inside libmm; see include/mm.h for the size limit and the no-overlap rule)."""
    _dev(x, torch.float64, "x"); _dev(y, torch.float64, "y")
    nrhs = 1 if x.dim() <= 2 else x.shape[0]
    _check(_lib.mm_apply_A_noalloc(ctypes.c_void_p(plan.handle), _ptr(x), _ptr(y), nrhs,
                                   _stream_ptr(stream)))


def mm_precond(plan: Plan, r: torch.Tensor, z: torch.Tensor, stream=None):
    _dev(r, torch.float64, "r"); _dev(z, torch.float64, "z")
    nrhs = 1 if r.dim() <= 2 else r.shape[0]
    _check(_lib.mm_precond(ctypes.c_void_p(plan.handle), _ptr(r), _ptr(z), nrhs, _stream_ptr(stream)))


def mm_pcg_solve(plan: Plan, b: torch.Tensor, x: torch.Tensor, tol: float = 1e-6,
                 max_iter: int = 10000, precision: int = MM_FP64, reliable_every: int = 0,
                 check_every: int = 0, deadline_us: int = 0, profile: bool = False, stream=None,
                 raise_on_error=True, precond: int = MM_PREC_BD):
    """Solve A x = b (b, x: [nrhs, n_obs, 3] or [n_obs, 3]); returns a list of SolveInfo."""
    _dev(b, torch.float64, "b"); _dev(x, torch.float64, "x")
    nrhs = 1 if b.dim() <= 2 else b.shape[0]
    opts = SolveOpts(tol=tol, max_iter=max_iter, precond=precond, precision=precision,
                     reliable_every=reliable_every, check_every=check_every,
                     profile=1 if profile else 0, deadline_us=deadline_us)
    infos = (SolveInfo * nrhs)()
    code = _lib.mm_pcg_solve(ctypes.c_void_p(plan.handle), _ptr(b), _ptr(x), nrhs,
                             ctypes.byref(opts), infos, _stream_ptr(stream))
    if raise_on_error and code not in (MM_OK,):
        raise MMError(code, mm_last_error())
    return list(infos)


def mm_solve_tod(plan: Plan, d: torch.Tensor, x: torch.Tensor, tol: float = 1e-6,
                 max_iter: int = 10000, precision: int = MM_FP64, reliable_every: int = 0,
                 check_every: int = 0, deadline_us: int = 0, profile: bool = False, stream=None,
                 raise_on_error=True, precond: int = MM_PREC_BD):
    """Solve the map-making problem from the TOD d ([nrhs, N] or [N], float64 or float32, CUDA or
    CPU) into x ([nrhs, n_obs, 3] or [n_obs, 3]); returns a list of SolveInfo."""
    if d.dtype not in (torch.float64, torch.float32):
        raise TypeError("d must be float64 or float32")
    if not d.is_contiguous():
        raise ValueError("d must be contiguous")
    _dev(x, torch.float64, "x")
    nrhs = 1 if d.dim() == 1 else d.shape[0]
    opts = SolveOpts(tol=tol, max_iter=max_iter, precond=precond, precision=precision,
                     reliable_every=reliable_every, check_every=check_every,
                     profile=1 if profile else 0, deadline_us=deadline_us)
    infos = (SolveInfo * nrhs)()
    code = _lib.mm_solve_tod(ctypes.c_void_p(plan.handle), _ptr(d), 1 if d.dtype == torch.float32 else 0, _ptr(x),
                             nrhs, ctypes.byref(opts), infos, _stream_ptr(stream))
    if raise_on_error and code not in (MM_OK,):
        raise MMError(code, mm_last_error())
    return list(infos)


def mm_autotune(plan: Plan, max_width: int = 64, stream=None) -> dict:
    """Time and keep the fastest FP32 A-application configuration of the plan; returns the choice and
    every timing."""
    t = TuneInfo()
    _check(_lib.mm_autotune(ctypes.c_void_p(plan.handle), max_width, ctypes.byref(t), _stream_ptr(stream)))
    return {"tile_steps": t.tile_steps, "win_samples": t.win_samples, "block_width": t.block_width,
            "apply_ms": t.apply_ms, "big_tiles": t.big_tiles, "big_tiles_ms": t.big_tiles_ms,
            "max_rel_dev": t.max_rel_dev, "n_rejected": t.n_rejected,
            "steps_ms": {t.steps_cand[i]: t.steps_ms[i] for i in range(t.n_steps)},
            "win_ms": {t.win_cand[i]: t.win_ms[i] for i in range(t.n_win)},
            "width_ms_per_col": {t.width_cand[i]: t.width_ms_per_col[i] for i in range(t.n_width)},
            "seg_sub": t.seg_sub, "seg_ms": {t.seg_cand[i]: t.seg_ms[i] for i in range(t.n_seg)}}


def mm_block_cg_solve(plan: Plan, b: torch.Tensor, x: torch.Tensor, block_width: int = 0,
                      tol: float = 1e-6, max_iter: int = 10000, precision: int = MM_FP32,
                      stream=None, raise_on_error=True):
    """Block CG on nrhs right-hand sides (b, x: [nrhs, n_obs, 3]); returns a list of SolveInfo."""
    _dev(b, torch.float64, "b"); _dev(x, torch.float64, "x")
    nrhs = 1 if b.dim() <= 2 else b.shape[0]
    opts = SolveOpts(tol=tol, max_iter=max_iter, precond=MM_PREC_BD, precision=precision)
    infos = (SolveInfo * nrhs)()
    code = _lib.mm_block_cg_solve(ctypes.c_void_p(plan.handle), _ptr(b), _ptr(x), nrhs, block_width,
                                  ctypes.byref(opts), infos, _stream_ptr(stream))
    if raise_on_error and code != MM_OK:
        raise MMError(code, mm_last_error())
    return list(infos)


def mm_ecg_solve(plan: Plan, b: torch.Tensor, x: torch.Tensor, t: int, variant: int = MM_ECG_ORTHOMIN,
                 tol: float = 1e-6, max_iter: int = 10000, precision: int = MM_FP32, stream=None,
                 raise_on_error=True):
    """Enlarged CG with enlarging factor t for one right-hand side (b, x: [n_obs, 3])."""
    _dev(b, torch.float64, "b"); _dev(x, torch.float64, "x")
    opts = SolveOpts(tol=tol, max_iter=max_iter, precond=MM_PREC_BD, precision=precision)
    info = SolveInfo()
    code = _lib.mm_ecg_solve(ctypes.c_void_p(plan.handle), _ptr(b), _ptr(x), t, variant,
                             ctypes.byref(opts), ctypes.byref(info), _stream_ptr(stream))
    if raise_on_error and code != MM_OK:
        raise MMError(code, mm_last_error())
    return info


def mm_deflation_build(plan: Plan, b: torch.Tensor, m: int, precision: int = MM_FP64, stream=None):
    """Two-level a-posteriori deflation space from m Lanczos steps started at b ([n_obs, 3])."""
    _dev(b, torch.float64, "b")
    _check(_lib.mm_deflation_build(ctypes.c_void_p(plan.handle), _ptr(b), m, precision,
                                   _stream_ptr(stream)))


def mm_templates_set(plan: Plan, n_poly: int = 0, n_az: int = 0, n_hwp: int = 0, az_interp: bool = False,
                     az: Optional[torch.Tensor] = None, hwp: Optional[torch.Tensor] = None, stream=None):
    """Attach template classes to a lambda = 0 plan (az, hwp: float32 [N] CUDA tensors)."""
    for name, v in (("az", az), ("hwp", hwp)):
        if v is not None:
            _dev(v, torch.float32, name)
    t = TemplatesDesc(n_poly=n_poly, n_az=n_az, n_hwp=n_hwp, az_interp=1 if az_interp else 0,
                      az=_ptr(az) if az is not None else None, hwp=_ptr(hwp) if hwp is not None else None,
                      inputs_on_device=1)
    _check(_lib.mm_templates_set(ctypes.c_void_p(plan.handle), ctypes.byref(t), _stream_ptr(stream)))


def mm_estimate_bands(n_det: int, n_int: int, block_len: Sequence[int], pix: torch.Tensor, d: torch.Tensor,
                      lam: int, stream=None):
    """Noise weights from the data: (bands [n_blocks, lam + 1] float64 CUDA tensor,
    params [n_blocks, 3] numpy: log sigma^2, log f_knee in cycles per sample, alpha)."""
    import numpy as np
    _dev(pix, torch.int32, "pix"); _dev(d, torch.float64, "d")
    nb = n_det * n_int
    bl = (ctypes.c_int64 * nb)(*[int(v) for v in block_len])
    bands = torch.empty(nb, lam + 1, dtype=torch.float64, device=d.device)
    params = np.zeros((nb, 3))
    _check(_lib.mm_estimate_bands(n_det, n_int, bl, _ptr(pix), _ptr(d), lam, _ptr(bands),
                                  params.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)))
    return bands, params


def mm_deflation_build_apriori(plan: Plan, precision: int = MM_FP64, stream=None):
    """Two-level a-priori deflation space: one column per stationary interval of the plan."""
    _check(_lib.mm_deflation_build_apriori(ctypes.c_void_p(plan.handle), precision, _stream_ptr(stream)))


def mm_deflation_get(plan: Plan, stream=None):
    """(k, Z [k, n_obs, 3] float64 CUDA tensor, Ritz values [k] numpy)."""
    import numpy as np
    k = ctypes.c_int()
    _check(_lib.mm_deflation_get(ctypes.c_void_p(plan.handle), ctypes.byref(k), None, None,
                                 _stream_ptr(stream)))
    if k.value == 0:
        return 0, None, None
    Z = torch.empty(k.value, plan.n_obs, 3, dtype=torch.float64, device="cuda")
    theta = np.zeros(k.value)
    _check(_lib.mm_deflation_get(ctypes.c_void_p(plan.handle), ctypes.byref(k), _ptr(Z),
                                 theta.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)))
    return k.value, Z, theta


def mm_deflation_apply(plan: Plan, r: torch.Tensor, z: torch.Tensor, stream=None):
    """z = M_2lvl r (Eq. 2lvlDef0) for r, z [nrhs, n_obs, 3] or [n_obs, 3]."""
    _dev(r, torch.float64, "r"); _dev(z, torch.float64, "z")
    nrhs = 1 if r.dim() <= 2 else r.shape[0]
    _check(_lib.mm_deflation_apply(ctypes.c_void_p(plan.handle), _ptr(r), _ptr(z), nrhs,
                                   _stream_ptr(stream)))


class Server:
    """mm_server_* : continuous-batching solve server on the current device (host inputs)."""

    def __init__(self, hbm_budget: int = 0, max_slots: int = 8):
        h = ctypes.c_void_p()
        _check(_lib.mm_server_create(hbm_budget, max_slots, ctypes.byref(h)))
        self.handle = h.value
        self._keep = {}

    def submit(self, n_det, n_int, block_len, n_pix, pix, psi, lam, band, d, tol=1e-6,
               max_iter=5000, cond_max=1e3, reliable_every=0, deadline_us=0,
               precision=MM_FP32, plan_precision=MM_DF64) -> int:
        """Queue a solve (host arrays).  d float32 is passed as FP32 TOD, anything else as float64.
        precision MM_FP32: batched FP32 iterations; MM_FP64: FP64-class iterations in the
        arithmetic of plan_precision (IEEE FP64 for MM_FP64 / MM_FP32, double-float otherwise)."""
        import numpy as np
        pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int32))
        psi = np.ascontiguousarray(np.asarray(psi, dtype=np.float32))
        band = np.ascontiguousarray(np.asarray(band, dtype=np.float64))
        d = np.asarray(d)
        d_is_fp32 = 1 if d.dtype == np.float32 else 0
        d = np.ascontiguousarray(d if d_is_fp32 else d.astype(np.float64, copy=False))
        bl = (ctypes.c_int64 * len(block_len))(*[int(v) for v in block_len])
        desc = ProblemDesc(n_det=n_det, n_int=n_int, block_len=bl, n_pix=n_pix,
                           pix=pix.ctypes.data, psi=psi.ctypes.data, lambda_=lam,
                           band=band.ctypes.data, cond_max=cond_max, precision=plan_precision,
                           toeplitz_algo=MM_TPLZ_AUTO, inputs_on_device=0, tile_steps=0)
        opts = SolveOpts(tol=tol, max_iter=max_iter, precond=MM_PREC_BD, precision=precision,
                         reliable_every=reliable_every, deadline_us=deadline_us)
        rid = ctypes.c_int64()
        _check(_lib.mm_submit(ctypes.c_void_p(self.handle), ctypes.byref(desc),
                              d.ctypes.data, d_is_fp32, ctypes.byref(opts), ctypes.byref(rid)))
        self._keep[rid.value] = n_pix
        return rid.value

    def poll(self, rid: int):
        info = SolveInfo()
        code = _lib.mm_poll(ctypes.c_void_p(self.handle), rid, ctypes.byref(info))
        if code == MM_EBUSY:
            return None
        _check(code)
        return info

    def wait(self, rid: int, timeout_us: int = -1, raise_on_error=True):
        import numpy as np
        n_pix = self._keep[rid]
        m = np.zeros((n_pix, 3))
        info = SolveInfo()
        code = _lib.mm_wait(ctypes.c_void_p(self.handle), rid, timeout_us,
                            m.ctypes.data, ctypes.byref(info))
        if code == MM_ETIMEOUT:
            raise MMError(code, mm_last_error())
        self._keep.pop(rid, None)
        if raise_on_error and code != MM_OK:
            raise MMError(code, mm_last_error())
        return m, info

    def close(self):
        if self.handle:
            _lib.mm_server_destroy(ctypes.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
