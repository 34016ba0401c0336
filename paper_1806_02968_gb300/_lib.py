"""ctypes declarations of the C ABI in include/lsq.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblsq.so")

LSQ_F64, LSQ_F32, LSQ_BF16, LSQ_F32X2 = 0, 1, 2, 3
STATUS = {0: "ok", 1: "invalid", 2: "cuda", 3: "nomem", 4: "not_converged", 5: "breakdown",
          6: "timeout", 7: "unsupported"}


class LsqMatrix(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("nnz", C.c_int64), ("dense", C.c_int32),
                ("ld", C.c_int64), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("vals", C.c_void_p), ("dtype", C.c_int32), ("vals_f64", C.c_void_p)]


class LsqOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int32), ("max_outer", C.c_int32),
                ("sweeps", C.c_int32), ("sample_factor", C.c_double), ("normalize", C.c_int32),
                ("precond_dtype", C.c_int32), ("seed", C.c_uint64), ("inner_tol", C.c_double),
                ("grid_ctas", C.c_int32), ("sampling", C.c_int32), ("device_loop", C.c_int32)]


class LsqInfo(C.Structure):
    _fields_ = [("k", C.c_int64), ("iters", C.c_void_p), ("outer", C.c_void_p),
                ("relres_rec", C.c_void_p), ("relres_true", C.c_void_p),
                ("relres_raw", C.c_void_p), ("converged", C.c_void_p), ("s", C.c_int64),
                ("nnz_M", C.c_int64), ("n_fixed_diag", C.c_int64), ("levels", C.c_int64),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double)]


class LsqBatchProblem(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("ld", C.c_int64), ("A", C.c_void_p),
                ("P", C.c_void_p), ("B", C.c_void_p), ("ldb", C.c_int64), ("X", C.c_void_p),
                ("ldx", C.c_int64)]


# name -> (restype, argtypes)
P, I64, D = C.c_void_p, C.c_int64, C.c_double
PROTOTYPES = {
    "lsq_default_opts": (None, [P]),
    "lsq_sample_size": (I64, [I64, D]),
    "lsq_sample_rows": (C.c_int, [P, P, I64, P, P, P, P, P]),
    "lsq_sample_rows_static": (C.c_int, [P, P, I64, P, P, P, P, P]),
    "lsq_build_precond": (C.c_int, [P, P, P, P, I64, P, P, P]),
    "lsq_precond_destroy": (None, [P]),
    "lsq_precond_get_M": (C.c_int, [P, P, P]),
    "lsq_precond_get_op": (C.c_int, [P, P, P]),
    "lsq_precond_get_M_csr": (C.c_int, [P, P, P, P, P, P]),
    "lsq_precond_apply": (C.c_int, [P, P, P, I64, P]),
    "lsq_pcg_solve": (C.c_int, [P, P, P, I64, I64, P, I64, P, P, P]),
    "lsq_pcg_adjoint": (C.c_int, [P, P, P, P, P, I64, I64, I64, P, P, P, P, P, P]),
    "lsq_split_f64": (C.c_int, [P, P, I64, P]),
    "lsq_batch_create": (C.c_int, [P, I64, I64, P, P, P]),
    "lsq_batch_solve": (C.c_int, [P, P]),
    "lsq_batch_autotune": (C.c_int, [P, P, P]),
    "lsq_batch_set_cluster": (C.c_int, [P, C.c_int32]),
    "lsq_batch_info": (C.c_int, [P, P, P]),
    "lsq_batch_destroy": (None, [P]),
    "lsq_status_string": (C.c_char_p, [C.c_int]),
    "lsq_last_error_string": (C.c_char_p, []),
    "lsq_kernel_launch_count": (I64, []),
    "lsq_set_wait_limit": (C.c_int, [I64]),
    "lsq_set_sweep_form": (C.c_int, [C.c_int32]),
    "lsq_measure_latency": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lsq_shard_colmax": (C.c_int, [P, P, P]),
    "lsq_shard_colsum": (C.c_int, [P, P, P, P]),
    "lsq_shard_weights": (C.c_int, [P, P, P, P, P, P, P, P]),
    "lsq_shard_offsets": (C.c_int, [P, C.c_int32, C.c_int32, P, P]),
    "lsq_shard_draw": (C.c_int, [P, I64, I64, P, P, P, I64, P, P, P]),
    "lsq_shard_draw_host": (C.c_int, [P, I64, I64, P, P, C.c_uint64, I64, I64, P]),
}

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load liblsq.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: run paper_1806_02968_gb300.build()")
            L = C.CDLL(path)
            for name, (res, args) in PROTOTYPES.items():
                f = getattr(L, name)
                f.restype, f.argtypes = res, args
            _lib = L
    return _lib


class LsqError(RuntimeError):
    def __init__(self, code: int, where: str):
        L = load()
        msg = L.lsq_last_error_string().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(code, code)} ({msg})")
        self.code = code
