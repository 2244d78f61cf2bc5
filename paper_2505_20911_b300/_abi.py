"""ctypes binding of libtgv.so (the C ABI in include/tgv.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Loading fails loudly if the library has not been built; there
is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtgv.so")

TGV_F64, TGV_F32, TGV_BF16, TGV_F16 = 0, 1, 2, 3
TGV_OK = 0
TGV_ERR_ARG, TGV_ERR_UNSUPPORTED, TGV_ERR_CUDA = -1, -2, -3
TGV_ERR_NONFINITE, TGV_ERR_UNSTABLE_DT, TGV_ERR_TIMEOUT, TGV_ERR_WORKSPACE = -4, -5, -6, -7
TGV_SPLIT_BLAISDELL, TGV_SPLIT_DIVERGENCE, TGV_SPLIT_KGP, TGV_SPLIT_KEEP = 0, 1, 2, 3
TGV_SPLIT_FEIEREISEN = 4
TGV_ENC_PLAIN, TGV_ENC_OFFSET = 0, 1
TGV_FLAG_ALLOW_UNSTABLE_DT = 1
TGV_FLAG_CHECK_FINITE = 2
TGV_FLAG_CELL_CENTERED = 4
TGV_FLAG_SYMMETRIC = 8
TGV_DIAG_COUNT = 10
TGV_ABI_VERSION = 1


class tgv_config(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("split_form", C.c_int32), ("q_storage", C.c_int32),
        ("qt_storage", C.c_int32), ("compute", C.c_int32), ("accumulate", C.c_int32),
        ("encoding", C.c_int32), ("tile", C.c_int32), ("zchunk", C.c_int32),
        ("flags", C.c_int32), ("length", C.c_double), ("gamma", C.c_double),
        ("mach", C.c_double), ("re", C.c_double), ("pr", C.c_double), ("mu", C.c_double),
    ]


class tgv_slab(C.Structure):
    _fields_ = [("z0", C.c_int32), ("nz", C.c_int32)]


class TGVError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


_lib = None

_P = C.c_void_p
_CFG = C.POINTER(tgv_config)
_SLAB = C.POINTER(tgv_slab)
# name -> (restype, argtypes)
SIGNATURES = {
    "tgv_abi_version": (C.c_int32, []),
    "tgv_strerror": (C.c_char_p, [C.c_int32]),
    "tgv_check_config": (C.c_int32, [_CFG]),
    "tgv_state_bytes": (C.c_size_t, [_CFG]),
    "tgv_qt_bytes": (C.c_size_t, [_CFG]),
    "tgv_tile_count": (C.c_int32, []),
    "tgv_tile_shape": (C.c_int32, [C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "tgv_dt_max": (C.c_double, [_CFG]),
    "tgv_init": (C.c_int32, [_CFG, _P, _P]),
    "rhs_eval": (C.c_int32, [_CFG, _P, _P, _P]),
    "rk_step": (C.c_int32, [_CFG, _P, _P, _P, C.c_double, C.c_int32, C.c_int32, _P, _P,
                            C.c_size_t, C.POINTER(C.c_int32), _P]),
    "rk_substep": (C.c_int32, [_CFG, _P, _P, _P, C.c_int32, C.c_double, _P]),
    "tgv_workspace_bytes": (C.c_size_t, [_CFG]),
    "diagnostics_reduce": (C.c_int32, [_CFG, _P, _P, _P, C.c_size_t, _P]),
    "diagnostics_reduce_noalloc": (C.c_int32, [_CFG, _P, _P, _P]),
    "tgv_adjoint_workspace_bytes": (C.c_size_t, [_CFG]),
    "rhs_vjp": (C.c_int32, [_CFG, _P, _P, _P, _P, C.c_size_t, _P]),
    "rk_step_adjoint": (C.c_int32, [_CFG, _P, _P, C.c_double, _P, C.c_size_t, _P]),
    "tgv_grad_workspace_bytes": (C.c_size_t, [_CFG, C.c_int32, C.c_int32]),
    "tgv_grad_final_ke": (C.c_int32, [_CFG, _P, C.c_double, C.c_int32, C.c_int32, _P, _P, _P,
                                      C.c_size_t, _P]),
    "tgv_ensemble_create": (C.c_int32, [_CFG, C.c_int32, C.POINTER(C.c_void_p),
                                        C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                        C.POINTER(C.c_double), C.c_int32, _P,
                                        C.POINTER(C.c_void_p)]),
    "tgv_ensemble_run": (C.c_int32, [_P, C.c_int32, _P]),
    "tgv_ensemble_info": (C.c_int32, [_P] + [C.POINTER(C.c_int32)] * 5),
    "tgv_ensemble_destroy": (C.c_int32, [_P]),
    "tgv_slab_state_bytes": (C.c_size_t, [_CFG, _SLAB]),
    "tgv_slab_qt_bytes": (C.c_size_t, [_CFG, _SLAB]),
    "tgv_slab_init": (C.c_int32, [_CFG, _SLAB, _P, _P]),
    "tgv_slab_substep": (C.c_int32, [_CFG, _SLAB, _P, _P, _P, C.c_int32, C.c_double, _P, _P,
                                     C.c_size_t, _P]),
    "tgv_slab_exchange_local": (C.c_int32, [_CFG, C.c_int32, _SLAB, C.POINTER(C.c_void_p), _P]),
    "tgv_probe_fma": (C.c_int32, [C.c_int32, C.c_int32, C.c_int32, _P, C.c_size_t,
                                  C.POINTER(C.c_double), _P]),
    "tgv_run_host_workspace_bytes": (C.c_size_t, [_CFG, C.c_int32, C.c_int32]),
    "tgv_run_host": (C.c_int32, [_CFG, _P, _P, C.c_double, C.c_int32, C.c_int32, _P, _P,
                                 C.c_size_t, _P]),
    "tgv_run_host_stream_workspace_bytes": (C.c_size_t, [_CFG, C.c_int32, C.c_int32]),
    "tgv_run_host_stream": (C.c_int32, [_CFG, C.c_int32, C.POINTER(C.c_void_p),
                                        C.POINTER(C.c_void_p), C.c_double, C.c_int32, C.c_int32,
                                        _P, _P, C.c_size_t, _P, _P]),
}


def lib():
    """The loaded libtgv.so (raises if it is missing: build it first)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2505_20911_b300.build` "
                "(the CUDA path has no fallback)")
        handle = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        if handle.tgv_abi_version() != TGV_ABI_VERSION:
            raise ImportError("libtgv.so ABI version mismatch; rebuild it")
        _lib = handle
    return _lib


def strerror(status: int) -> str:
    return lib().tgv_strerror(status).decode()


def check(status: int, where: str) -> None:
    if status != TGV_OK:
        raise TGVError(status, where)
