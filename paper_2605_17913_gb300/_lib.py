"""ctypes binding of libqpgpu (include/qp.h): argument marshalling only.

Every step of the solve and of the backward pass runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current stream.  If the
library is missing or cannot be loaded, every call raises; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqpgpu.so")

# return codes (qp.h)
QP_OK, QP_PENDING = 0, 1
QP_EINVAL, QP_ENOMEM, QP_ECUDA, QP_EAGAIN, QP_ETIMEOUT, QP_ENOTSUP, QP_ESTATE = (
    -1, -2, -3, -4, -5, -6, -7)
# per-instance status
QP_SOLVED, QP_MAX_ITER, QP_STALLED, QP_NUMERICAL, QP_BAD_INPUT = 0, 1, 2, 3, 4
QP_IMPLICIT, QP_STANDARD, QP_STANDARD_SCHUR = 0, 1, 2
QP_SIGMA_MEHROTRA, QP_SIGMA_CONSTANT = 0, 1
QP_NORM_SCALED, QP_NORM_ABS = 0, 1
QP_GWG_FP32, QP_GWG_TF32, QP_GWG_BF16 = 0, 1, 2
QP_STATIC_CACHE_BYTES = 16 * 1024 * 1024
QP_SERVE_LAUNCHES, QP_SERVE_PERSISTENT = 0, 1
SERVE_MODES = {"launches": QP_SERVE_LAUNCHES, "persistent": QP_SERVE_PERSISTENT}
# per-instance diagnostics word (qp_handle_set_diag)
QP_STAGE_MASK = 0xFF
QP_STAGE_NAMES = {0: "none", 1: "scaling", 2: "predictor", 3: "centering", 4: "corrector",
                  5: "line search", 6: "relax", 7: "backward", 8: "init"}
QP_DIAG_FACTOR_FAILED, QP_DIAG_TC_FALLBACK, QP_DIAG_STAGE_FALLBACK, QP_DIAG_ASYNC_LOST = (
    0x100, 0x200, 0x400, 0x800)


class QPError(RuntimeError):
    pass


class Dims(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("n", ctypes.c_int32), ("n_eq", ctypes.c_int32),
                ("n_ineq", ctypes.c_int32)]


class HandleInfo(ctypes.Structure):
    _fields_ = [("fwd_threads", ctypes.c_int32), ("fwd_blocks_per_sm", ctypes.c_int32),
                ("bwd_threads", ctypes.c_int32), ("max_active", ctypes.c_int32),
                ("large_variant", ctypes.c_int32), ("fwd_smem_bytes", ctypes.c_size_t)]


class Settings(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_float),
        ("max_iter", ctypes.c_int32),
        ("sigma_mode", ctypes.c_int32),
        ("sigma", ctypes.c_float),
        ("kappa_min", ctypes.c_float),
        ("kappa_relax", ctypes.c_float),
        ("relax_tol", ctypes.c_float),
        ("relax_max_iter", ctypes.c_int32),
        ("formulation", ctypes.c_int32),
        ("residual_norm", ctypes.c_int32),
        ("gwg_precision", ctypes.c_int32),
        ("refine_steps", ctypes.c_int32),
        ("warm_start", ctypes.c_int32),
        ("relax_chord", ctypes.c_int32),
        ("refine_forward", ctypes.c_int32),
    ]


class ServeConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("max_queue", ctypes.c_int32),
                ("settings", Settings), ("mode", ctypes.c_int32), ("idle_ms", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_eq", ctypes.c_int32), ("n_ineq", ctypes.c_int32),
                ("want_grad", ctypes.c_int32)] + [
        (k, ctypes.c_void_p) for k in ("Q", "q", "A", "b", "G", "h", "dl_dx", "x", "y", "z", "s",
                                       "dQ", "dq", "dA", "db", "dG", "dh")]


class Result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("kkt_res", ctypes.c_float),
                ("t_submit_ms", ctypes.c_double), ("t_launch_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libqpgpu.so (built by ``paper_2605_17913_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise QPError(f"libqpgpu.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    L.qp_settings_default.restype = None
    L.qp_settings_default.argtypes = [ctypes.POINTER(Settings)]
    L.qp_status_string.restype = ctypes.c_char_p
    L.qp_status_string.argtypes = [ctypes.c_int]
    L.qp_smem_bytes.restype = ctypes.c_size_t
    L.qp_smem_bytes.argtypes = [i32, i32, i32]
    L.qp_handle_create.restype = ctypes.c_int
    L.qp_handle_create.argtypes = [ctypes.POINTER(Dims), ctypes.POINTER(vp)]
    L.qp_handle_create_threads.restype = ctypes.c_int
    L.qp_handle_create_threads.argtypes = [ctypes.POINTER(Dims), i32, ctypes.POINTER(vp)]
    L.qp_grad_cache_bytes.restype = ctypes.c_size_t
    L.qp_grad_cache_bytes.argtypes = [ctypes.POINTER(Dims)]
    L.qp_workspace_bytes.restype = ctypes.c_size_t
    L.qp_workspace_bytes.argtypes = [ctypes.POINTER(Dims)]
    L.qp_handle_destroy.restype = ctypes.c_int
    L.qp_handle_destroy.argtypes = [vp]
    L.qp_handle_set_diag.restype = ctypes.c_int
    L.qp_handle_set_diag.argtypes = [vp, vp]
    L.qp_handle_query.restype = ctypes.c_int
    L.qp_handle_query.argtypes = [vp, ctypes.POINTER(HandleInfo)]
    L.qp_solve_batch.restype = ctypes.c_int
    L.qp_solve_batch.argtypes = [vp, ctypes.POINTER(Settings)] + [vp] * 14 + [vp]
    L.qp_backward_batch.restype = ctypes.c_int
    L.qp_backward_batch.argtypes = [vp] * 13
    L.qp_serve_config_default.restype = None
    L.qp_serve_config_default.argtypes = [ctypes.POINTER(ServeConfig)]
    L.qp_serve_footprint_bytes.restype = ctypes.c_size_t
    L.qp_serve_footprint_bytes.argtypes = [i32, i32, i32, i32]
    L.qp_serve_create.restype = ctypes.c_int
    L.qp_serve_create.argtypes = [ctypes.POINTER(ServeConfig), ctypes.POINTER(vp)]
    L.qp_serve_submit.restype = ctypes.c_int
    L.qp_serve_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    L.qp_serve_poll.restype = ctypes.c_int
    L.qp_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(Result)]
    L.qp_serve_poll_any.restype = ctypes.c_int
    L.qp_serve_poll_any.argtypes = [vp, ctypes.POINTER(Result)]
    L.qp_serve_wait.restype = ctypes.c_int
    L.qp_serve_wait.argtypes = [vp, ctypes.c_uint64, i32, ctypes.POINTER(Result)]
    L.qp_serve_destroy.restype = ctypes.c_int
    L.qp_serve_destroy.argtypes = [vp]
    L.qp_solve_backward_static.restype = ctypes.c_int
    L.qp_solve_backward_static.argtypes = [vp, ctypes.POINTER(Settings)] + [vp] * 21
    L.qp_fma_probe.restype = ctypes.c_int
    L.qp_fma_probe.argtypes = [i32, i32, i32, vp, vp]
    L.qp_solve_backward_host.restype = ctypes.c_int
    L.qp_solve_backward_host.argtypes = [vp, ctypes.POINTER(Settings)] + [vp] * 20
    _lib = L
    return L


def status_string(code: int) -> str:
    return lib().qp_status_string(int(code)).decode()


def check(rc: int, what: str) -> None:
    if rc != QP_OK:
        raise QPError(f"{what}: {status_string(rc)} ({rc})")


def default_settings(**overrides) -> Settings:
    s = Settings()
    lib().qp_settings_default(ctypes.byref(s))
    for k, v in overrides.items():
        if k == "formulation" and isinstance(v, str):
            v = {"implicit": QP_IMPLICIT, "standard": QP_STANDARD,
                 "standard_schur": QP_STANDARD_SCHUR}[v]
        if k == "residual_norm" and isinstance(v, str):
            v = {"scaled": QP_NORM_SCALED, "abs": QP_NORM_ABS}[v]
        if k == "sigma_mode" and isinstance(v, str):
            v = {"mehrotra": QP_SIGMA_MEHROTRA, "constant": QP_SIGMA_CONSTANT}[v]
        if k == "gwg_precision" and isinstance(v, str):
            v = {"fp32": QP_GWG_FP32, "tf32": QP_GWG_TF32, "bf16": QP_GWG_BF16}[v]
        if not hasattr(s, k):
            raise KeyError(f"unknown setting {k}")
        setattr(s, k, v)
    return s


def ptr(t) -> Optional[int]:
    """Device address of a tensor (or None)."""
    if t is None:
        return None
    return t.data_ptr() if t.numel() > 0 else None


def smem_bytes(n: int, n_eq: int, n_ineq: int) -> int:
    return int(lib().qp_smem_bytes(n, n_eq, n_ineq))
