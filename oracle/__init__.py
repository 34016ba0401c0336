"""Python face of the FP64 CPU oracle (``oracle/lsq_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by
the benchmark's CPU legs (the CPU baseline and the reference arm), never by the CUDA package.  It shares no code with
the CUDA path.  Matrices use the dict layout of :mod:`workloads`.

Each wrapper names the step of the paper it computes (Alg. 1-3, Eq. R2P, Sec. 3.3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lsq_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liblsq_oracle.so")
_lock = threading.Lock()
_lib = None


def compile_source(src: str, out: str) -> str:
    """gcc -O2 with FMA contraction off (every product rounded once) into a shared library."""
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared",
                           "-ffp-contract=off", "-fno-fast-math", "-o", out, src, "-lm"])
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/ (when the source is newer than the library)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        compile_source(_SRC, tmp)
        os.replace(tmp, _SO)
    return _SO


class _Mat(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("dense", C.c_int32), ("ld", C.c_int64),
                ("vals", C.c_void_p), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p)]


class _PcgInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("outer", C.c_int32), ("converged", C.c_int32),
                ("status", C.c_int32), ("relres_rec", C.c_double),
                ("relres_true", C.c_double), ("hnorm", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P, I64, I32, D, U64 = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_uint64
            L.orc_sample_size.argtypes, L.orc_sample_size.restype = [I64, D], I64
            L.orc_col_scales.argtypes = [P, I32, P, P, P, P]
            L.orc_col_scales.restype = C.c_int
            L.orc_row_weights.argtypes, L.orc_row_weights.restype = [P, P, P, P], C.c_int
            L.orc_prefix.argtypes, L.orc_prefix.restype = [I64, P, P, P, P], None
            L.orc_philox4x64_10.argtypes, L.orc_philox4x64_10.restype = [P, P, P], None
            L.orc_draw_rows.argtypes = [I64, P, P, U64, I64, I64, P]
            L.orc_draw_rows.restype = C.c_int
            L.orc_build_M.argtypes, L.orc_build_M.restype = [P, P, P, P, P, I64], P
            L.orc_M_nnz.argtypes, L.orc_M_nnz.restype = [P], I64
            L.orc_M_fixed_diag.argtypes, L.orc_M_fixed_diag.restype = [P], I64
            L.orc_M_copy.argtypes, L.orc_M_copy.restype = [P, P, P, P], None
            L.orc_M_free.argtypes, L.orc_M_free.restype = [P], None
            L.orc_M_view.argtypes, L.orc_M_view.restype = [P, I64, P, P, P], None
            L.orc_sgs_apply.argtypes, L.orc_sgs_apply.restype = [P, C.c_int, P, P], None
            L.orc_apply_A.argtypes, L.orc_apply_A.restype = [P, P, P, P], None
            L.orc_apply_AT.argtypes, L.orc_apply_AT.restype = [P, P, P, P], None
            L.orc_normal_matvec.argtypes, L.orc_normal_matvec.restype = [P, P, P, P], None
            L.orc_pcg.argtypes = [P, P, P, C.c_int, P, P, D, C.c_int, C.c_int, P, P]
            L.orc_pcg.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Mat:
    """Keeps the FP64 arrays alive and exposes the C view."""

    def __init__(self, mat: dict):
        if mat["kind"] == "dense":
            A = np.ascontiguousarray(mat["A"], dtype=np.float64)
            self.m, self.n = A.shape
            self.vals, self.row_ptr, self.col_idx = A, None, None
            self.c = _Mat(self.m, self.n, 1, self.n, A.ctypes.data, None, None)
        else:
            self.m, self.n = int(mat["m"]), int(mat["n"])
            self.vals = np.ascontiguousarray(mat["vals"], dtype=np.float64)
            self.row_ptr = np.ascontiguousarray(mat["row_ptr"], dtype=np.int64)
            self.col_idx = np.ascontiguousarray(mat["col_idx"], dtype=np.int32)
            self.c = _Mat(self.m, self.n, 0, 0, self.vals.ctypes.data,
                          self.row_ptr.ctypes.data, self.col_idx.ctypes.data)
        self.ref = C.byref(self.c)


def as_mat(mat) -> Mat:
    return mat if isinstance(mat, Mat) else Mat(mat)


def sample_size(n: int, C_factor: float = 4.0) -> int:
    """Alg. 2 step 2: s = ceil(C n ln n)."""
    return int(lib().orc_sample_size(int(n), float(C_factor)))


def col_scales(mat, normalize: bool = True):
    """Alg. 2 step 1 with exact fixed-point column sums -> (d2, d, inv_d2, E1)."""
    M = as_mat(mat)
    d2, d, inv = (np.empty(M.n) for _ in range(3))
    E1 = C.c_int32(0)
    st = lib().orc_col_scales(M.ref, int(bool(normalize)), _ptr(d2), _ptr(d), _ptr(inv), C.byref(E1))
    if st != 0:
        raise ValueError(f"orc_col_scales status {st}")
    return d2, d, inv, int(E1.value)


def row_weights(mat, inv_d2):
    """Eq. (R2P) as exact integers -> w as Python-int-ready (lo, hi) uint64 arrays."""
    M = as_mat(mat)
    lo, hi = np.empty(M.m, np.uint64), np.empty(M.m, np.uint64)
    lib().orc_row_weights(M.ref, _ptr(np.ascontiguousarray(inv_d2, np.float64)), _ptr(lo), _ptr(hi))
    return lo, hi


def prefix(w_lo, w_hi):
    m = w_lo.size
    P_lo, P_hi = np.empty(m + 1, np.uint64), np.empty(m + 1, np.uint64)
    lib().orc_prefix(m, _ptr(w_lo), _ptr(w_hi), _ptr(P_lo), _ptr(P_hi))
    return P_lo, P_hi


def philox4x64_10(ctr, key):
    c = np.array(ctr, dtype=np.uint64)
    k = np.array(key, dtype=np.uint64)
    out = np.empty(4, np.uint64)
    lib().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return [int(x) for x in out]


def draw_rows(P_lo, P_hi, seed: int, s: int, t0: int = 0):
    """Alg. 1 draws t0..t0+s-1 -> int32 row indices."""
    m = P_lo.size - 1
    idx = np.empty(s, np.int32)
    st = lib().orc_draw_rows(m, _ptr(P_lo), _ptr(P_hi), C.c_uint64(seed), int(t0), int(s), _ptr(idx))
    if st != 0:
        raise ValueError(f"orc_draw_rows status {st}")
    return idx


def u128(lo, hi):
    return [(int(h) << 64) | int(l) for l, h in zip(lo, hi)]


class Sample:
    """Everything Alg. 1 + Alg. 2 steps 1-2 produce for one matrix and seed.

    sampling="norm2" is the method's density, p_i proportional to the squared norm of the
    normalised row (Eq. R2P).  sampling="uniform" is the comparison of Sec. 3.1: every row
    has the same weight (w_i = 1, p_i = 1/m); the column scales of Alg. 2 step 1 are still
    computed, and the draws and the scaling 1/(s p_i) go through the same steps."""

    def __init__(self, mat, seed: int, s: int | None = None, normalize: bool = True,
                 C_factor: float = 4.0, sampling: str = "norm2"):
        self.mat = as_mat(mat)
        self.d2, self.d, self.inv_d2, self.E1 = col_scales(self.mat, normalize)
        if sampling == "uniform":
            self.w_lo = np.ones(self.mat.m, np.uint64)
            self.w_hi = np.zeros(self.mat.m, np.uint64)
        elif sampling == "norm2":
            self.w_lo, self.w_hi = row_weights(self.mat, self.inv_d2)
        else:
            raise ValueError(sampling)
        self.P_lo, self.P_hi = prefix(self.w_lo, self.w_hi)
        self.s = sample_size(self.mat.n, C_factor) if not s else int(s)
        self.seed = seed
        self.idx = draw_rows(self.P_lo, self.P_hi, seed, self.s)

    @property
    def W(self) -> int:
        return (int(self.P_hi[-1]) << 64) | int(self.P_lo[-1])


class SampledM:
    """A_s^T A_s (Sec. 3.3) in CSR, built by the oracle."""

    def __init__(self, smp: Sample, idx=None):
        L = lib()
        idx = smp.idx if idx is None else np.ascontiguousarray(idx, np.int32)
        h = L.orc_build_M(smp.mat.ref, _ptr(smp.d), _ptr(smp.w_lo), _ptr(smp.w_hi),
                          _ptr(idx), int(idx.size))
        if not h:
            raise MemoryError("orc_build_M failed")
        try:
            n = smp.mat.n
            nnz = L.orc_M_nnz(h)
            self.n_fixed_diag = int(L.orc_M_fixed_diag(h))
            self.row_ptr = np.empty(n + 1, np.int64)
            self.col = np.empty(nnz, np.int32)
            self.val = np.empty(nnz, np.float64)
            L.orc_M_copy(h, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val))
        finally:
            L.orc_M_free(h)
        self.n = smp.mat.n
        self._view()

    @classmethod
    def from_csr(cls, n, row_ptr, col, val):
        self = cls.__new__(cls)
        self.n = int(n)
        self.row_ptr = np.ascontiguousarray(row_ptr, np.int64)
        self.col = np.ascontiguousarray(col, np.int32)
        self.val = np.ascontiguousarray(val, np.float64)
        self.n_fixed_diag = 0
        self._view()
        return self

    def _view(self):
        # orc_M layout: n, nnz, n_fixed_diag (int64) then three pointers
        self._buf = (C.c_byte * 64)()
        lib().orc_M_view(C.byref(self._buf), self.n, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val))

    @property
    def handle(self):
        return C.byref(self._buf)

    def dense(self):
        D = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        D[rows, self.col] = self.val
        return D


def sgs_apply(Mo: SampledM, r, sweeps: int = 1):
    """Alg. 3 with e0 = 0 -> e."""
    r = np.ascontiguousarray(r, np.float64)
    e = np.empty_like(r)
    lib().orc_sgs_apply(Mo.handle, int(sweeps), _ptr(r), _ptr(e))
    return e


def apply_A(mat, d, p):
    M = as_mat(mat)
    q = np.empty(M.m)
    lib().orc_apply_A(M.ref, _ptr(np.ascontiguousarray(d, np.float64)),
                      _ptr(np.ascontiguousarray(p, np.float64)), _ptr(q))
    return q


def apply_AT(mat, d, q):
    M = as_mat(mat)
    w = np.empty(M.n)
    lib().orc_apply_AT(M.ref, _ptr(np.ascontiguousarray(d, np.float64)),
                       _ptr(np.ascontiguousarray(q, np.float64)), _ptr(w))
    return w


def normal_matvec(mat, d, p):
    """w = Â^T (Â p), Â = A D^{-1} (two passes)."""
    M = as_mat(mat)
    w = np.empty(M.n)
    lib().orc_normal_matvec(M.ref, _ptr(np.ascontiguousarray(d, np.float64)),
                            _ptr(np.ascontiguousarray(p, np.float64)), _ptr(w))
    return w


def pcg(mat, d, Mo: SampledM, b=None, h=None, tol=1e-10, maxit=10000, max_outer=5, sweeps=1):
    """Alg. 2 step 4.  Returns (y, info dict); x = y / d."""
    M = as_mat(mat)
    y = np.empty(M.n)
    info = _PcgInfo()
    bb = None if b is None else np.ascontiguousarray(b, np.float64)
    hh = None if h is None else np.ascontiguousarray(h, np.float64)
    lib().orc_pcg(M.ref, _ptr(np.ascontiguousarray(d, np.float64)), Mo.handle, int(sweeps),
                  _ptr(bb), _ptr(hh), float(tol), int(maxit), int(max_outer), _ptr(y),
                  C.byref(info))
    return y, {k: getattr(info, k) for k, _ in _PcgInfo._fields_}


def csr_matvec(mat: dict, x):
    if mat["kind"] == "dense":
        return mat["A"] @ x
    rows = np.repeat(np.arange(mat["m"]), np.diff(mat["row_ptr"]))
    return np.bincount(rows, weights=mat["vals"] * x[mat["col_idx"]], minlength=mat["m"])


def csr_rmatvec(mat: dict, r):
    if mat["kind"] == "dense":
        return mat["A"].T @ r
    rows = np.repeat(np.arange(mat["m"]), np.diff(mat["row_ptr"]))
    return np.bincount(mat["col_idx"], weights=mat["vals"] * r[rows], minlength=mat["n"])


class Solve:
    """Alg. 2 end to end: normalise, sample, build A_s^T A_s, PCG.  One right-hand side."""

    def __init__(self, mat: dict, b, seed: int, tol=1e-10, sweeps=1, maxit=10000,
                 max_outer=5, s=None, normalize=True, C_factor=4.0):
        self.raw = mat
        self.smp = Sample(mat, seed, s=s, normalize=normalize, C_factor=C_factor)
        self.M = SampledM(self.smp)
        self.sweeps = sweeps
        y, self.info = pcg(self.smp.mat, self.smp.d, self.M, b=b, tol=tol, maxit=maxit,
                           max_outer=max_outer, sweeps=sweeps)
        self.y = y
        self.x = y / self.smp.d
        r = np.asarray(b, np.float64) - csr_matvec(mat, self.x)
        Atb = csr_rmatvec(mat, np.asarray(b, np.float64))
        nb = np.linalg.norm(Atb)
        self.info["relres_raw"] = float(np.linalg.norm(csr_rmatvec(mat, r)) / nb) if nb > 0 else 0.0


def adjoint(mat: dict, smp: Sample, Mo: SampledM, x, b, G, tol=1e-10, sweeps=1, maxit=10000,
            max_outer=5):
    """Gradients of L(x(A, b)) for x = argmin ||A x - b||, given G = dL/dx (one column).

    A^T A lam = G is solved as Â^T Â mu = D^{-1} G with the same sampled preconditioner,
    lam = D^{-1} mu; then dL/db = A lam and dL/dA = r lam^T - (A lam) x^T, r = b - A x,
    restricted to A's stored entries.  Returns (grad_b, grad_vals, lam, info).
    """
    d = smp.d
    mu, info = pcg(smp.mat, d, Mo, h=np.asarray(G, np.float64) / d, tol=tol, maxit=maxit,
                   max_outer=max_outer, sweeps=sweeps)
    lam = mu / d
    Alam = csr_matvec(mat, lam)
    r = np.asarray(b, np.float64) - csr_matvec(mat, x)
    if mat["kind"] == "dense":
        gA = np.outer(r, lam) - np.outer(Alam, x)
        return Alam, gA, lam, info
    rows = np.repeat(np.arange(mat["m"]), np.diff(mat["row_ptr"]))
    cols = mat["col_idx"]
    gv = r[rows] * lam[cols] - Alam[rows] * x[cols]
    return Alam, gv, lam, info
