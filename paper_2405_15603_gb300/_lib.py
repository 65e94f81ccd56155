"""ctypes declarations of the C-ABI in include/kfac_pinn.h (marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

KFAC_MAX_LAYERS = 16

STATUS = {0: "KFAC_OK", 1: "KFAC_BAD_ARG", 2: "KFAC_NOT_PD", 3: "KFAC_NONFINITE",
          4: "KFAC_TIMEOUT", 5: "KFAC_OOM", 6: "KFAC_CUDA_ERROR", 7: "KFAC_NOT_READY"}

EXPORTS = [
    "kfac_pinn_param_count", "kfac_pinn_status_string", "kfac_pinn_create", "kfac_pinn_destroy",
    "kfac_pinn_reset", "kfac_pinn_forward_laplacian", "kfac_pinn_factors", "kfac_pinn_invert",
    "kfac_pinn_precondition", "kfac_pinn_update", "kfac_pinn_step", "kfac_pinn_step_host",
    "kfac_pinn_get_factor", "kfac_pinn_set_factor", "kfac_pinn_get_gradient",
    "kfac_pinn_get_direction", "kfac_pinn_sync_status", "kfac_pinn_launch_count",
    "kfac_pinn_timing_enable", "kfac_pinn_timing_read", "kfac_pinn_timing_read_ex",
    "kfac_pinn_forward_laplacian_noalloc",
    "kfac_pinn_get_line_search_losses", "kfac_pinn_forward_laplacian_backward",
    "kfac_pinn_get_update_coefficients", "kfac_pinn_batch_create", "kfac_pinn_batch_destroy",
    "kfac_pinn_batch_step", "kfac_pinn_last_cuda_error", "kfac_pinn_last_cuda_error_string",
    "kfac_pinn_set_store_forward",
    "kfac_pinn_set_cta_pairs",
    "kfac_pinn_set_graph", "kfac_pinn_set_autotune", "kfac_pinn_get_tuning", "kfac_pinn_set_tuning",
    "kfac_pinn_check_wait_timeout", "kfac_pinn_inject_alloc_failure", "kfac_pinn_batch_set_grouped",
    "kfac_pinn_batch_launches",
]

KFAC_TUNE_CAP = 128
KFAC_MAX_RESIDUALS = 8

KERNEL_CLASSES = {0: "layer_gemm", 1: "adjoint_gemm", 2: "gram", 3: "elementwise", 4: "eig", 5: "precond"}


class KfacConfig(C.Structure):
    _fields_ = [
        ("d", C.c_int), ("L", C.c_int), ("widths", C.c_int * KFAC_MAX_LAYERS),
        ("op", C.c_int), ("kappa", C.c_double), ("precision", C.c_int), ("variant", C.c_int),
        ("beta", C.c_double), ("lambda_", C.c_double), ("damping_sqrt", C.c_int),
        ("factor_init_identity", C.c_int), ("lr", C.c_double), ("momentum", C.c_double),
        ("max_n_int", C.c_int), ("max_n_bdy", C.c_int), ("update", C.c_int), ("eig_sm_budget", C.c_int),
        ("op_coef", C.c_void_p), ("residual", C.c_void_p),
    ]


class KfacResidual(C.Structure):
    _fields_ = [("M", C.c_int), ("b", C.c_void_p), ("Q", C.c_void_p), ("W", C.c_void_p)]


TUNE_KINDS = {0: "gram", 1: "fwd_tan", 2: "bwd_tan"}


class KfacTuneEntry(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("P", C.c_int), ("Q", C.c_int), ("K", C.c_int), ("tiles", C.c_int),
        ("sym", C.c_int), ("split", C.c_int), ("chunk", C.c_int), ("model_chunk", C.c_int),
        ("us", C.c_float), ("model_us", C.c_float),
    ]


class KfacError(RuntimeError):
    def __init__(self, fn: str, code: int):
        msg = f"{fn} returned {STATUS.get(code, code)}"
        if code == 6 and _LIB is not None:      # KFAC_CUDA_ERROR: name the CUDA error behind it
            msg += f" ({_LIB.kfac_pinn_last_cuda_error_string().decode()})"
        super().__init__(msg)
        self.code = code
        self.status = STATUS.get(code, str(code))


_LIB = None


def lib_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "libkfacpinn.so")


def load() -> C.CDLL:
    """Load libkfacpinn.so; fails loudly when it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2405_15603_gb300.build.build()")
    lib = C.CDLL(path)
    P, I, D, H = C.c_void_p, C.c_int, C.c_double, C.c_void_p
    st = C.c_int
    sig = {
        "kfac_pinn_param_count": (C.c_int64, [C.POINTER(KfacConfig)]),
        "kfac_pinn_status_string": (C.c_char_p, [I]),
        "kfac_pinn_create": (st, [C.POINTER(KfacConfig), C.POINTER(H)]),
        "kfac_pinn_destroy": (st, [H]),
        "kfac_pinn_reset": (st, [H, P]),
        "kfac_pinn_forward_laplacian": (st, [H, P, P, P, I, P, P, P]),
        "kfac_pinn_forward_laplacian_backward": (st, [H, P, P, P, I, P, P, P, P, P]),
        "kfac_pinn_factors": (st, [H, P, P, P, I, P, P, I, P, P]),
        "kfac_pinn_invert": (st, [H, P]),
        "kfac_pinn_precondition": (st, [H, P, P, P]),
        "kfac_pinn_update": (st, [H, P, P]),
        "kfac_pinn_step": (st, [H, P, P, P, I, P, P, I, P, P]),
        "kfac_pinn_step_host": (st, [H, P, P, P, I, P, P, I, P, P]),
        "kfac_pinn_get_factor": (st, [H, P, I, I, P]),
        "kfac_pinn_set_factor": (st, [H, P, I, I, P]),
        "kfac_pinn_get_gradient": (st, [H, P, P]),
        "kfac_pinn_get_direction": (st, [H, P, P]),
        "kfac_pinn_get_line_search_losses": (st, [H, P, P]),
        "kfac_pinn_get_update_coefficients": (st, [H, P, P]),
        "kfac_pinn_last_cuda_error": (I, []),
        "kfac_pinn_set_store_forward": (st, [H, I]),
        "kfac_pinn_set_cta_pairs": (st, [H, I]),
        "kfac_pinn_set_graph": (st, [H, I]),
        "kfac_pinn_set_autotune": (st, [H, I]),
        "kfac_pinn_get_tuning": (st, [H, C.POINTER(KfacTuneEntry), I, C.POINTER(C.c_int)]),
        "kfac_pinn_set_tuning": (st, [H, C.POINTER(KfacTuneEntry), I]),
        "kfac_pinn_last_cuda_error_string": (C.c_char_p, []),
        "kfac_pinn_batch_create": (st, [P, I, I, C.POINTER(C.c_void_p)]),
        "kfac_pinn_batch_destroy": (st, [P]),
        "kfac_pinn_batch_step": (st, [P, P, P, P, P, P, P, P, P, P, I]),
        "kfac_pinn_batch_set_grouped": (st, [P, I]),
        "kfac_pinn_batch_launches": (st, [P, C.POINTER(C.c_longlong)]),
        "kfac_pinn_sync_status": (st, [H, C.POINTER(C.c_int)]),
        "kfac_pinn_launch_count": (C.c_int64, [H]),
        "kfac_pinn_timing_enable": (st, [H, I]),
        "kfac_pinn_check_wait_timeout": (st, [H, P, I, I]),
        "kfac_pinn_inject_alloc_failure": (st, [C.c_longlong]),
        "kfac_pinn_forward_laplacian_noalloc": (st, [C.POINTER(KfacConfig), P, P, P, I, P, P, P]),
        "kfac_pinn_timing_read": (st, [H, I, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                       C.POINTER(C.c_double)]),
        "kfac_pinn_timing_read_ex": (st, [H, I, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                          C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib
