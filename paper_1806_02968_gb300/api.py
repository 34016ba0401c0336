"""Python face of the C ABI: same call names, torch tensors as device buffers.

Every function here only builds the C argument structs from tensors and calls into
liblsq.so; all arithmetic of the method runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L

DTYPES = {torch.float64: L.LSQ_F64, torch.float32: L.LSQ_F32, torch.bfloat16: L.LSQ_BF16}


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _require(cond, msg):
    """Argument checks of the binding (kept under python -O, unlike assert)."""
    if not cond:
        raise ValueError(msg)


def _device_array(t, name, dtype=None):
    _require(isinstance(t, torch.Tensor) and t.is_cuda, f"{name} must be a CUDA tensor")
    _require(dtype is None or t.dtype == dtype, f"{name} must be {dtype}")
    _require(t.is_contiguous(), f"{name} must be contiguous")


def opts(**kw) -> L.LsqOpts:
    """lsq_default_opts() with keyword overrides."""
    o = L.LsqOpts()
    L.load().lsq_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Matrix:
    """A in R^{m x n} as device tensors (dense row-major (m, ld) or CSR)."""

    def __init__(self, dense=None, *, row_ptr=None, col_idx=None, vals=None, n=None,
                 vals_f64=None, f32x2=None):
        if dense is not None:
            _require(isinstance(dense, torch.Tensor) and dense.is_cuda, "A must be a CUDA tensor")
            _require(dense.dim() == 2 and dense.stride(1) == 1, "dense A must be 2-D with unit column stride")
            if f32x2:   # (m, 2 n) float32: element j of row i is the pair at columns 2j, 2j+1
                _require(dense.dtype == torch.float32 and dense.shape[1] % 2 == 0,
                         "double-float A must be float32 (m, 2 n) pairs")
                self.m, self.n = dense.shape[0], dense.shape[1] // 2
                self.ld = dense.stride(0) // 2
            else:
                self.m, self.n = dense.shape
                self.ld = dense.stride(0)
            self.vals = dense
            self.row_ptr = self.col_idx = None
            self.nnz = self.m * self.n
            self.dense = True
        else:
            _device_array(row_ptr, "row_ptr", torch.int64)
            _device_array(col_idx, "col_idx", torch.int32)
            _device_array(vals, "vals")
            _require(n is not None and int(n) > 0, "CSR A needs its column count n")
            self.m = row_ptr.numel() - 1
            self.n = int(n)
            self.ld = 0
            self.vals, self.row_ptr, self.col_idx = vals, row_ptr, col_idx
            self.nnz = vals.numel()
            self.dense = False
        _require(f32x2 or self.vals.dtype in DTYPES, "values must be float64, float32 or bfloat16")
        if vals_f64 is not None:
            _require(vals_f64.is_cuda and vals_f64.dtype == torch.float64, "vals_f64 must be a CUDA float64 tensor")
        self.dtype = L.LSQ_F32X2 if f32x2 else DTYPES[self.vals.dtype]
        self.vals_f64 = vals_f64
        self.c = L.LsqMatrix(self.m, self.n, self.nnz, 1 if self.dense else 0, self.ld,
                             _ptr(self.row_ptr), _ptr(self.col_idx), _ptr(self.vals), self.dtype,
                             _ptr(vals_f64))

    @property
    def ref(self):
        return C.byref(self.c)


def _check(code, where):
    if code != 0:
        raise L.LsqError(code, where)


def lsq_sample_size(n: int, C_factor: float = 4.0) -> int:
    return int(L.load().lsq_sample_size(int(n), float(C_factor)))


def lsq_sample_rows(A: Matrix, o=None, s: int = 0, stream=None):
    """Alg. 2 steps 1-2 / Alg. 1 -> (idx int32[s], p float64[s], colscale float64[n])."""
    o = o or opts()
    s_eff = s if s else lsq_sample_size(A.n, o.sample_factor)
    dev = A.vals.device
    idx = torch.empty(s_eff, dtype=torch.int32, device=dev)
    p = torch.empty(s_eff, dtype=torch.float64, device=dev)
    d = torch.empty(A.n, dtype=torch.float64, device=dev)
    s_out = C.c_int64(0)
    _check(L.load().lsq_sample_rows(A.ref, C.byref(o), s_eff, _ptr(idx), _ptr(p), _ptr(d),
                                    C.byref(s_out), _stream(stream)), "lsq_sample_rows")
    return idx, p, d


def lsq_sample_rows_static(A: Matrix, o=None, s: int = 0, stream=None):
    """lsq_sample_rows without any device allocation inside the library (its scratch is a
    fixed device array; at most 262144 rows and 4096 columns)."""
    o = o or opts()
    s_eff = s if s else lsq_sample_size(A.n, o.sample_factor)
    dev = A.vals.device
    idx = torch.empty(s_eff, dtype=torch.int32, device=dev)
    p = torch.empty(s_eff, dtype=torch.float64, device=dev)
    d = torch.empty(A.n, dtype=torch.float64, device=dev)
    s_out = C.c_int64(0)
    _check(L.load().lsq_sample_rows_static(A.ref, C.byref(o), s_eff, _ptr(idx), _ptr(p), _ptr(d),
                                           C.byref(s_out), _stream(stream)), "lsq_sample_rows_static")
    return idx, p, d


class Precond:
    """Owns an lsq_precond handle (Sec. 3.3 + Alg. 3)."""

    def __init__(self, handle, n):
        self.h = C.c_void_p(handle)
        self.n = n

    def __del__(self):
        if getattr(self, "h", None) and self.h.value:
            L.load().lsq_precond_destroy(self.h)
            self.h = C.c_void_p(None)

    def M(self, stream=None):
        out = torch.empty(self.n, self.n, dtype=torch.float64, device="cuda")
        _check(L.load().lsq_precond_get_M(self.h, _ptr(out), _stream(stream)), "lsq_precond_get_M")
        return out

    def M_csr(self, stream=None):
        """(row_ptr, col_idx, vals) of the sparse A_s^T A_s (sparse handles)."""
        nnz = C.c_int64(0)
        _check(L.load().lsq_precond_get_M_csr(self.h, C.byref(nnz), None, None, None, _stream(stream)),
               "lsq_precond_get_M_csr")
        rp = torch.empty(self.n + 1, dtype=torch.int64, device="cuda")
        ci = torch.empty(nnz.value, dtype=torch.int32, device="cuda")
        va = torch.empty(nnz.value, dtype=torch.float64, device="cuda")
        _check(L.load().lsq_precond_get_M_csr(self.h, C.byref(nnz), _ptr(rp), _ptr(ci), _ptr(va),
                                              _stream(stream)), "lsq_precond_get_M_csr")
        return rp, ci, va

    def op(self, stream=None):
        out = torch.empty(self.n, self.n, dtype=torch.float64, device="cuda")
        _check(L.load().lsq_precond_get_op(self.h, _ptr(out), _stream(stream)), "lsq_precond_get_op")
        return out

    def apply(self, r, stream=None):
        r = r.contiguous()
        k = 1 if r.dim() == 1 else r.shape[0]
        e = torch.empty_like(r)
        _check(L.load().lsq_precond_apply(self.h, _ptr(r), _ptr(e), k, _stream(stream)), "lsq_precond_apply")
        return e


def lsq_build_precond(A: Matrix, idx, p, colscale, o=None, stream=None) -> Precond:
    o = o or opts()
    h = C.c_void_p()
    _check(L.load().lsq_build_precond(A.ref, _ptr(idx), _ptr(p), _ptr(colscale), idx.numel(),
                                      C.byref(o), C.byref(h), _stream(stream)), "lsq_build_precond")
    return Precond(h.value, A.n)


@dataclass
class Info:
    iters: np.ndarray
    outer: np.ndarray
    relres_rec: np.ndarray
    relres_true: np.ndarray
    relres_raw: np.ndarray
    converged: np.ndarray
    status: int
    s: int = 0
    nnz_M: int = 0
    n_fixed_diag: int = 0
    levels: int = 0
    solve_ms: float = 0.0


def _info(k):
    arrs = dict(iters=np.zeros(k, np.int32), outer=np.zeros(k, np.int32),
                relres_rec=np.zeros(k), relres_true=np.zeros(k), relres_raw=np.zeros(k),
                converged=np.zeros(k, np.uint8))
    ci = L.LsqInfo(k, *(a.ctypes.data for a in arrs.values()))
    return ci, arrs


def _finish_info(ci, arrs, status):
    return Info(status=status, s=ci.s, nnz_M=ci.nnz_M, n_fixed_diag=ci.n_fixed_diag,
                levels=ci.levels, solve_ms=ci.solve_ms, **arrs)


ACCEPT = (0, 4)  # ok, not converged (reported in info)


def lsq_pcg_solve(A: Matrix, P: Precond, B, o=None, X=None, stream=None, raise_on=None):
    """Alg. 2 step 4 for k right-hand sides (B: (m,) or (k, m) float64) -> (X, Info)."""
    o = o or opts()
    B2 = B.reshape(1, -1) if B.dim() == 1 else B
    _require(B2.is_cuda and B2.dtype == torch.float64 and B2.stride(1) == 1,
             "B must be a CUDA float64 tensor (m,) or (k, m) with unit stride along m")
    k = B2.shape[0]
    if X is None:
        X = torch.empty(k, A.n, dtype=torch.float64, device=B.device)
    _require(X.is_cuda and X.dtype == torch.float64 and X.dim() == 2 and X.shape[0] == k
             and X.shape[1] >= A.n and X.stride(1) == 1, "X must be a CUDA float64 (k, n) tensor")
    ci, arrs = _info(k)
    code = L.load().lsq_pcg_solve(A.ref, P.h, _ptr(B2), k, B2.stride(0), _ptr(X), X.stride(0),
                                  C.byref(o), C.byref(ci), _stream(stream))
    if code not in ACCEPT or (raise_on and code in raise_on):
        raise L.LsqError(code, "lsq_pcg_solve")
    return (X.reshape(-1) if B.dim() == 1 else X), _finish_info(ci, arrs, code)


def lsq_pcg_adjoint(A: Matrix, P: Precond, X, B, G, o=None, want_grad_vals=True, stream=None):
    """Adjoint solve -> (grad_b (k, m), grad_vals (like A's values, FP64), Lambda (k, n), Info)."""
    o = o or opts()
    X2, B2, G2 = (t.reshape(1, -1) if t.dim() == 1 else t for t in (X, B, G))
    k = X2.shape[0]
    gb = torch.empty(k, A.m, dtype=torch.float64, device=X.device)
    lam = torch.empty(k, A.n, dtype=torch.float64, device=X.device)
    gv = None
    if want_grad_vals:
        gv = torch.zeros(A.m, A.ld, dtype=torch.float64, device=X.device) if A.dense else \
            torch.zeros(A.nnz, dtype=torch.float64, device=X.device)
    ci, arrs = _info(k)
    code = L.load().lsq_pcg_adjoint(A.ref, P.h, _ptr(X2), _ptr(B2), _ptr(G2), k, B2.stride(0),
                                    X2.stride(0), _ptr(gb), _ptr(gv), _ptr(lam), C.byref(o),
                                    C.byref(ci), _stream(stream))
    if code not in ACCEPT:
        raise L.LsqError(code, "lsq_pcg_adjoint")
    return gb, gv, lam, _finish_info(ci, arrs, code)


def lsq_split_f64(src, stream=None):
    """FP64 -> interleaved (hi, lo) float pairs (the LSQ_F32X2 storage); a (m, n) input
    gives a (m, 2 n) float32 tensor."""
    src = src.contiguous()
    shape = (*src.shape[:-1], 2 * src.shape[-1]) if src.dim() > 0 else (2,)
    dst = torch.empty(shape, dtype=torch.float32, device=src.device)
    _check(L.load().lsq_split_f64(_ptr(src), _ptr(dst), src.numel(), _stream(stream)), "lsq_split_f64")
    return dst


def launches() -> int:
    return int(L.load().lsq_kernel_launch_count())


# Row-sharded sampling (lsq_shard_* in lsq.h): one rank's phases; the caller does the
# collectives between them (MAX of colmax, SUM of limbs, all-gather of the totals, MAX merge
# of the draws).  colmax travels as int64 (bit patterns of non-negative doubles, below 2^63).
def shard_colmax(A: Matrix, stream=None):
    out = torch.empty(A.n, dtype=torch.int64, device=A.vals.device)
    _check(L.load().lsq_shard_colmax(A.ref, _ptr(out), _stream(stream)), "lsq_shard_colmax")
    return out


def shard_colsum(A: Matrix, colmax, stream=None):
    _device_array(colmax, "colmax", torch.int64)
    limbs = torch.empty(4 * A.n, dtype=torch.int64, device=A.vals.device)
    _check(L.load().lsq_shard_colsum(A.ref, _ptr(colmax), _ptr(limbs), _stream(stream)), "lsq_shard_colsum")
    return limbs


def shard_weights(A: Matrix, colmax, limbs, o=None, stream=None):
    """-> (colscale d, the rank's weight prefix as int64 (m + 1, 2), its total as 4 limbs)."""
    o = o or opts()
    _device_array(colmax, "colmax", torch.int64)
    _device_array(limbs, "limbs", torch.int64)
    d = torch.empty(A.n, dtype=torch.float64, device=A.vals.device)
    prefix = torch.empty(A.m + 1, 2, dtype=torch.int64, device=A.vals.device)
    W = np.zeros(4, np.int64)
    _check(L.load().lsq_shard_weights(A.ref, C.byref(o), _ptr(colmax), _ptr(limbs), _ptr(d), _ptr(prefix),
                                      W.ctypes.data, _stream(stream)), "lsq_shard_weights")
    return d, prefix, W


def shard_offsets(W_all, rank: int):
    """W_all: (world, 4) int64 limbs of every rank's total -> (offset, total) limbs."""
    W_all = np.ascontiguousarray(W_all, np.int64)
    off, tot = np.zeros(4, np.int64), np.zeros(4, np.int64)
    _check(L.load().lsq_shard_offsets(W_all.ctypes.data, W_all.shape[0], int(rank), off.ctypes.data,
                                      tot.ctypes.data), "lsq_shard_offsets")
    return off, tot


def shard_draw(prefix, row0: int, W_offset, W_total, s: int, o=None, stream=None):
    """-> (idx int32[s]: global row or -1, p float64[s]: its probability or 0)."""
    o = o or opts()
    _device_array(prefix, "prefix", torch.int64)
    off = np.ascontiguousarray(W_offset, np.int64)
    tot = np.ascontiguousarray(W_total, np.int64)
    idx = torch.empty(s, dtype=torch.int32, device=prefix.device)
    p = torch.empty(s, dtype=torch.float64, device=prefix.device)
    _check(L.load().lsq_shard_draw(_ptr(prefix), prefix.shape[0] - 1, int(row0), off.ctypes.data, tot.ctypes.data,
                                   C.byref(o), int(s), _ptr(idx), _ptr(p), _stream(stream)), "lsq_shard_draw")
    return idx, p


def shard_draw_host(prefix, row0: int, W_offset, W_total, seed: int, t0: int, s: int):
    """lsq_shard_draw on a host prefix (uint64 array of (m + 1) x 2 words) -> int32[s]."""
    prefix = np.ascontiguousarray(prefix, np.uint64)
    off = np.ascontiguousarray(W_offset, np.int64)
    tot = np.ascontiguousarray(W_total, np.int64)
    idx = np.empty(s, np.int32)
    _check(L.load().lsq_shard_draw_host(prefix.ctypes.data, prefix.size // 2 - 1, int(row0), off.ctypes.data,
                                        tot.ctypes.data, C.c_uint64(seed), int(t0), int(s), idx.ctypes.data),
           "lsq_shard_draw_host")
    return idx


def set_wait_limit(max_polls: int = 0):
    """Cap every device-side wait at max_polls polls (0: the library's defaults)."""
    _check(L.load().lsq_set_wait_limit(int(max_polls)), "lsq_set_wait_limit")


def set_sweep_form(form: int = 0):
    """Form of the sparse sweeps (lsq_set_sweep_form): 0 by shape, 1 grid, 2 one CTA, 3 one
    cluster; RHS blocks take only form 3, where their n x k vector fits."""
    _check(L.load().lsq_set_sweep_form(int(form)), "lsq_set_sweep_form")


def measure_latency(stream=None) -> dict:
    """The device's latency figures in ns (lsq_measure_latency): a dependent L2 load, a value's
    round trip between two SMs through global memory (without and with a fence before each
    store), an 8-CTA cluster barrier and a dependent load from another CTA's shared memory."""
    out = (C.c_double * 5)()
    _check(L.load().lsq_measure_latency(C.cast(out, C.c_void_p), _stream(stream)), "lsq_measure_latency")
    return {"l2_load_ns": out[0], "sm_round_trip_ns": out[1], "cluster_barrier_ns": out[2],
            "dsmem_load_ns": out[3], "sm_round_trip_fenced_ns": out[4]}


def solve(A: Matrix, b, o=None, stream=None):
    """Alg. 2 end to end: sample, build the preconditioner, PCG. Returns (x, Info, extras)."""
    o = o or opts()
    idx, p, d = lsq_sample_rows(A, o, stream=stream)
    P = lsq_build_precond(A, idx, p, d, o, stream=stream)
    x, info = lsq_pcg_solve(A, P, b, o, stream=stream)
    return x, info, dict(idx=idx, p=p, colscale=d, P=P)


class Batch:
    """A plan for many small dense problems solved in one launch (lsq_batch_* calls).

    problems: list of (A float32 (m, ld) row-major with ld % 4 == 0 (the first n columns are
    the matrix), n, Precond, B float64 (k, m)).  Solutions are written to X[p] (k, n)."""

    def __init__(self, problems, o=None, stream=None):
        self.o = o or opts()
        self.keep = []
        self.k = problems[0][3].shape[0] if problems[0][3].dim() == 2 else 1
        self.X = []
        arr = (L.LsqBatchProblem * len(problems))()
        for i, (A, n, P, B) in enumerate(problems):
            B2 = B.reshape(1, -1) if B.dim() == 1 else B
            _require(A.is_cuda and A.dtype == torch.float32 and A.stride(1) == 1,
                     "each batch A must be a CUDA float32 row-major tensor")
            _require(B2.is_cuda and B2.dtype == torch.float64 and B2.stride(1) == 1 and B2.shape[0] == self.k,
                     "each batch B must be a CUDA float64 (k, m) tensor with the batch's k")
            X = torch.zeros(self.k, n, dtype=torch.float64, device=A.device)
            self.keep += [A, B2, P]
            self.X.append(X)
            arr[i] = L.LsqBatchProblem(A.shape[0], n, A.stride(0), A.data_ptr(), P.h, B2.data_ptr(),
                                       B2.stride(0), X.data_ptr(), X.stride(0))
        self.count = len(problems)
        h = C.c_void_p()
        _check(L.load().lsq_batch_create(arr, self.count, self.k, C.byref(self.o), C.byref(h),
                                         _stream(stream)), "lsq_batch_create")
        self.h = h

    def solve(self, stream=None):
        """One launch; no host synchronisation (may be captured in a CUDA graph)."""
        _check(L.load().lsq_batch_solve(self.h, _stream(stream)), "lsq_batch_solve")

    def autotune(self, stream=None) -> int:
        c = C.c_int32()
        _check(L.load().lsq_batch_autotune(self.h, C.byref(c), _stream(stream)), "lsq_batch_autotune")
        return c.value

    def set_cluster(self, cluster: int):
        _check(L.load().lsq_batch_set_cluster(self.h, int(cluster)), "lsq_batch_set_cluster")

    def info(self, stream=None):
        """Per-problem Info of the last solve."""
        cis = (L.LsqInfo * self.count)()
        arrs = []
        for p in range(self.count):
            ci, a = _info(self.k)
            cis[p] = ci
            arrs.append(a)
        code = L.load().lsq_batch_info(self.h, cis, _stream(stream))
        if code not in ACCEPT:
            raise L.LsqError(code, "lsq_batch_info")
        return [_finish_info(cis[p], arrs[p], code) for p in range(self.count)]

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            L.load().lsq_batch_destroy(h)
            self.h = None


class LsqSolveFunction(torch.autograd.Function):
    """X = argmin_X ||A X - B|| (Alg. 2 step 4) as an autograd node.

    Backward reuses the sampled SGS preconditioner for the adjoint system A^T A lambda = dL/dX
    (lsq_pcg_adjoint), giving dL/dB = A lambda and dL/dA = r lambda^T - (A lambda) x^T (summed
    over the right-hand sides), restricted to A's pattern for a CSR matrix.  Inputs: A's value
    tensor (the one `A` was built from), B ((m,) or (k, m) float64), then the Matrix, the
    Precond and the options, which take no gradient."""

    @staticmethod
    def forward(ctx, vals, B, A, P, o):
        if A.dtype == L.LSQ_F32X2:
            raise ValueError("differentiation needs plain FP64/FP32/BF16 values")
        if vals.data_ptr() != A.vals.data_ptr():
            raise ValueError("vals must be the tensor the Matrix was built from")
        X, info = lsq_pcg_solve(A, P, B, o)
        ctx.A, ctx.P, ctx.o = A, P, o
        ctx.vals_shape, ctx.vals_dtype = vals.shape, vals.dtype
        ctx.info = info
        ctx.save_for_backward(X, B)
        return X

    @staticmethod
    def backward(ctx, gX):
        X, B = ctx.saved_tensors
        need_v, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        G = gX.to(torch.float64).contiguous()
        gb, gv, lam, info = lsq_pcg_adjoint(ctx.A, ctx.P, X, B, G, ctx.o, want_grad_vals=need_v)
        grad_vals = gv.reshape(ctx.vals_shape).to(ctx.vals_dtype) if need_v else None
        grad_b = gb.reshape(B.shape) if need_b else None
        return grad_vals, grad_b, None, None, None


def lsq_solve(A: Matrix, B, P: Precond, o=None):
    """Differentiable solve: gradients flow to A.vals and B (see LsqSolveFunction)."""
    return LsqSolveFunction.apply(A.vals, B, A, P, o or opts())
