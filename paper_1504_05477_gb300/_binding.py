"""ctypes binding of libbks.so (include/bks.h).  Argument marshalling only: every step
of the path runs in the library's CUDA kernels.  PyTorch supplies device memory and
streams; nothing here computes on the CPU or through torch operators."""
from __future__ import annotations

import ctypes
import os

from . import _build

# ------------------------------------------------------------------ C structures
BKS_OK, BKS_ERR_INVALID_ARG, BKS_ERR_CUDA, BKS_ERR_NOMEM = 0, 1, 2, 3
BKS_ERR_NONFINITE, BKS_ERR_BREAKDOWN, BKS_ERR_NOT_CONVERGED = 4, 5, 6
BKS_ERR_TIMEOUT, BKS_ERR_UNSUPPORTED, BKS_WARN_DEFLATED = 7, 8, 100
BKS_F64, BKS_F32, BKS_BF16 = 0, 1, 2
BKS_DENSE, BKS_CSR = 0, 1
PREC_AUTO, PREC_F64, PREC_F32, PREC_BF16 = 0, 1, 2, 3
REORTH = {"full": 0, "local": 1, "none": 2}


class BksMatrix(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("dtype", ctypes.c_int32),
        ("n", ctypes.c_int64), ("d", ctypes.c_int64), ("ld", ctypes.c_int64),
        ("vals", ctypes.c_void_p), ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
        ("nnz", ctypes.c_int64),
        ("t_row_ptr", ctypes.c_void_p), ("t_col_idx", ctypes.c_void_p), ("t_vals", ctypes.c_void_p),
        ("col_mean", ctypes.c_void_p),
    ]


class BksOpts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32), ("refine", ctypes.c_int32), ("basis_only", ctypes.c_int32),
        ("sign_fix", ctypes.c_int32), ("jacobi_max_sweeps", ctypes.c_int32),
        ("jacobi_tol", ctypes.c_double), ("profile", ctypes.c_int32),
        ("product_path", ctypes.c_int32), ("rr_mode", ctypes.c_int32), ("eig_mode", ctypes.c_int32),
        ("block_p", ctypes.c_int32), ("eig_f64", ctypes.c_int32), ("max_sms", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 1),
    ]


class BksStats(ctypes.Structure):
    _fields_ = [
        ("q_eff", ctypes.c_int32), ("width", ctypes.c_int32), ("jacobi_sweeps", ctypes.c_int32),
        ("chol_shifts", ctypes.c_int32), ("launches", ctypes.c_int32),
        ("product_launches", ctypes.c_int32),
        ("ms_product", ctypes.c_float), ("ms_orth", ctypes.c_float), ("ms_rr", ctypes.c_float),
        ("ms_total", ctypes.c_float),
        ("product_bytes", ctypes.c_double), ("product_flops", ctypes.c_double),
        ("ms_product_kernel", ctypes.c_float), ("product_kernel_launches", ctypes.c_int32),
        ("eig_path", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5),
    ]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_ if f[0] != "reserved"}


# (name, restype, argtypes) for every exported entry point of include/bks.h
_P, _I32, _I64, _U64, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
SIGNATURES = {
    "bks_create": (_I32, [ctypes.POINTER(_P), _I32]),
    "bks_destroy": (_I32, [_P]),
    "bks_set_stream": (_I32, [_P, _P]),
    "bks_set_workspace": (_I32, [_P, _P, _SZ]),
    "bks_workspace_size": (_I32, [ctypes.POINTER(BksMatrix), _I32, _I32, _I32,
                                  ctypes.POINTER(BksOpts), ctypes.POINTER(_SZ)]),
    "bks_opts_default": (None, [ctypes.POINTER(BksOpts)]),
    "bks_status_string": (ctypes.c_char_p, [_I32]),
    "bks_last_error": (ctypes.c_char_p, [_P]),
    "bks_version": (_I32, []),
    "bks_block_krylov": (_I32, [_P, ctypes.POINTER(BksMatrix), _I32, _I32, _U64, _P, _P, _P, _P,
                                ctypes.POINTER(BksOpts), ctypes.POINTER(BksStats)]),
    "bks_block_krylov_adaptive": (_I32, [_P, ctypes.POINTER(BksMatrix), _I32, _I32, ctypes.c_double, _U64, _P,
                                         _P, _P, _P, ctypes.POINTER(BksOpts), ctypes.POINTER(BksStats)]),
    "bks_simul_iter": (_I32, [_P, ctypes.POINTER(BksMatrix), _I32, _I32, _U64, _P, _P, _P, _P,
                              ctypes.POINTER(BksOpts), ctypes.POINTER(BksStats)]),
    "bks_block_lanczos": (_I32, [_P, ctypes.POINTER(BksMatrix), _I32, _I32, _I32, _U64, _P, _P, _P, _P,
                                 ctypes.POINTER(BksOpts), ctypes.POINTER(BksStats)]),
    "bks_gen_pi": (_I32, [_P, _U64, _I64, _I32, _I32, _P]),
    "bks_gen_pi_host": (_I32, [_U64, _I64, _I32, ctypes.POINTER(ctypes.c_float)]),
    "bks_csr_transpose": (_I32, [_P, ctypes.POINTER(BksMatrix), _P, _P, _P]),
    "bks_matmul": (_I32, [_P, ctypes.POINTER(BksMatrix), _I32, _I32, _P, _I64, _P, _I64, _I32]),
    "bks_orthonormalize": (_I32, [_P, _I32, _I64, _I32, _I32, _P, _I64, _P, _I64]),
    "bks_sym_eig": (_I32, [_P, _I32, _I32, _P, _I64, _P, _P, _I64]),
    "bks_sym_eig_noalloc": (_I32, [_P, _I32, _I32, _P, _I64, _P, _P, _I64]),
    "bks_selftest_wait": (_I32, [_P, _I32]),
    "bks_krylov_width": (_I32, [_I64, _I64, _I32, _I32, _I32]),
    "bks_block_krylov_batched": (_I32, [_P, _I32, ctypes.POINTER(BksMatrix), _I32, _I32, _P, _P, _P, _P, _P,
                                        ctypes.POINTER(BksOpts), ctypes.POINTER(BksStats), _P]),
    "bks_ritz_triplets": (_I32, [_P, ctypes.POINTER(BksMatrix), _I32, _I32, _U64, _P, _I32, _P, _P, _P,
                                 ctypes.POINTER(BksOpts), ctypes.POINTER(BksStats)]),
    "bks_backward": (_I32, [_P, _I32, _I64, _I64, _I32, _I32, _P, _P, _P, _P, _P, _P, ctypes.c_double]),
    "bks_batch_budget": (_I32, [_P, _I32, ctypes.POINTER(BksMatrix), _I32, _I32, _I32]),
    "bks_batched_autotune": (_I32, [_P, _I32, ctypes.POINTER(BksMatrix), _I32, _I32, _P, _P, _P, _P, _P,
                                    ctypes.POINTER(BksOpts), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    "bks_ritz_triplets_batched": (_I32, [_P, _I32, ctypes.POINTER(BksMatrix), _I32, _I32, _P, _P, _I32, _P, _P,
                                         _P, ctypes.POINTER(BksOpts), _P]),
    "bks_backward_batched": (_I32, [_P, _I32, _I32, _P, _P, _I32, _P, _P, _P, _P, _P, _P, _P, ctypes.c_double,
                                    _P]),
    "bks_low_rank": (_I32, [_P, _I32, _I64, _I64, _I32, _P, _I64, _P, _P, _I64, _P]),
}

_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libbks.so (building it first when it is missing or stale).  Raises if the
    library cannot be built or loaded: there is no fallback path."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libbks.so not found at {_build.LIB}; run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class BksError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def check(status: int, ctx=None, what="bks call", allow=(BKS_OK, BKS_WARN_DEFLATED)) -> int:
    if status in allow:
        return status
    lib = load()
    detail = lib.bks_last_error(ctx).decode() if ctx else ""
    text = lib.bks_status_string(status).decode()
    raise BksError(status, f"{what}: {text}" + (f": {detail}" if detail else ""))
