"""Host logic of the C ABI, without a GPU: documented defaults, status strings, and the
argument checks every entry point runs before it touches the device.  Each call here
fails one check, so no CUDA call is ever made (pointers are never dereferenced)."""
import ctypes as C
import re

import pytest

FAKE = 0x10000          # a non-NULL, 16-byte aligned address that is never dereferenced


def _mat(L, m=100, n=10, dense=1, ld=None, dtype=0, vals=FAKE, row_ptr=FAKE, col_idx=FAKE, nnz=0):
    A = L.LsqMatrix()
    A.m, A.n, A.nnz, A.dense, A.ld, A.dtype = m, n, nnz, dense, n if ld is None else ld, dtype
    A.vals, A.row_ptr, A.col_idx = vals, row_ptr, col_idx
    return A


def _opts(L, **kw):
    o = L.LsqOpts()
    L.load().lsq_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _err(lsq):
    return lsq.L.load().lsq_last_error_string().decode()


def test_default_opts_are_the_documented_ones(lsq):
    o = _opts(lsq.L)
    assert (o.tol, o.maxit, o.max_outer, o.sweeps, o.sample_factor, o.normalize, o.precond_dtype,
            o.seed, o.inner_tol, o.grid_ctas, o.sampling, o.device_loop) == (1e-10, 1000000, 20, 1, 4.0, 1, 0, 0, 0.0, 0, 0, 0)
    hdr = open(lsq.L.HERE + "/../include/lsq.h").read()
    for field, text in [("tol", "1e-10"), ("maxit", "1000000"), ("max_outer", "20"),
                        ("sample_factor", "4.0"), ("seed", "0")]:
        assert re.search(r"\b%s;.*;\s*%s\b" % (field, re.escape(text)), hdr), field


def test_status_strings_are_distinct(lsq):
    L = lsq.L.load()
    names = [L.lsq_status_string(c).decode() for c in range(8)]
    assert names[0] == "ok" and names[4] == "not converged" and len(set(names)) == 8
    assert L.lsq_status_string(99) == b"unknown status"


def test_sample_size_is_4_n_ln_n(lsq):
    L = lsq.L.load()
    assert [L.lsq_sample_size(n, 4.0) for n in (1, 2, 100, 200)] == [1, 6, 1843, 4239]


@pytest.mark.parametrize("case,msg", [
    ("null_A", "A is NULL"), ("zero_m", "positive"), ("ld_lt_n", "ld < n"), ("dtype", "dtype"),
    ("csr_null", "CSR arrays"), ("null_opts", "opts is NULL"), ("null_idx", "idx_out"),
    ("neg_s", "s < 0"), ("null_vals", "vals is NULL")])
def test_sample_rows_rejects(lsq, case, msg):
    L = lsq.L
    A = _mat(L)
    o = _opts(L)
    idx, s = FAKE, 0
    if case == "zero_m":
        A.m = 0
    elif case == "ld_lt_n":
        A.ld = 5
    elif case == "dtype":
        A.dtype = 9
    elif case == "csr_null":
        A = _mat(L, dense=0, row_ptr=None)
    elif case == "null_idx":
        idx = None
    elif case == "neg_s":
        s = -1
    elif case == "null_vals":
        A.vals = None
    pa = None if case == "null_A" else C.byref(A)
    po = None if case == "null_opts" else C.byref(o)
    st = L.load().lsq_sample_rows(pa, po, s, idx, None, None, None, None)
    assert st == 1 and msg in _err(lsq)


@pytest.mark.parametrize("case,msg", [
    ("sweeps_65", "sweeps must be in [0, 64]"), ("sweeps_neg", "sweeps must be in [0, 64]"),
    ("pdt", "precond_dtype"), ("dense_n", "n <= 2048"), ("csr_sweeps_33", "sweeps <= 32"),
    ("s_zero", "s must be positive"), ("null_idx", "NULL argument")])
def test_build_precond_rejects(lsq, case, msg):
    L = lsq.L
    A = _mat(L)
    o = _opts(L)
    s, idx = 50, FAKE
    if case == "sweeps_65":
        o.sweeps = 65
    elif case == "sweeps_neg":
        o.sweeps = -1
    elif case == "pdt":
        o.precond_dtype = 2
    elif case == "dense_n":
        A = _mat(L, m=5000, n=2049)
    elif case == "csr_sweeps_33":
        A = _mat(L, dense=0)
        o.sweeps = 33
    elif case == "s_zero":
        s = 0
    elif case == "null_idx":
        idx = None
    out = C.c_void_p(FAKE)
    st = L.load().lsq_build_precond(C.byref(A), idx, FAKE, FAKE, s, C.byref(o), C.byref(out), None)
    assert st == 1 and msg in _err(lsq)


@pytest.mark.parametrize("case,msg", [
    ("k0", "k must be >= 1"), ("ldb", "ldb >= m"), ("ldx", "ldx >= n"), ("tol", "tolerance"),
    ("outer", "tolerance or caps"), ("null_B", "NULL argument")])
def test_pcg_solve_rejects(lsq, case, msg):
    L = lsq.L
    A = _mat(L)
    o = _opts(L)
    k, ldb, ldx, B = 1, 100, 10, FAKE
    if case == "k0":
        k = 0
    elif case == "ldb":
        ldb = 99
    elif case == "ldx":
        ldx = 9
    elif case == "tol":
        o.tol = 0.0
    elif case == "outer":
        o.max_outer = 0
    elif case == "null_B":
        B = None
    st = L.load().lsq_pcg_solve(C.byref(A), FAKE, B, k, ldb, FAKE, ldx, C.byref(o), None, None)
    assert st == 1 and msg in _err(lsq)


@pytest.mark.parametrize("case,msg", [
    ("count0", "count must be"), ("k17", "k must be in [1, 16]"), ("n257", "1 <= n <= 256"),
    ("ld_odd", "multiple of 4"), ("misaligned", "16-byte aligned"), ("null_P", "dense handle"),
    ("opts", "bad options")])
def test_batch_create_rejects(lsq, case, msg):
    L = lsq.L
    q = L.LsqBatchProblem()
    q.m, q.n, q.ld, q.A, q.P, q.B, q.ldb, q.X, q.ldx = 100, 10, 12, FAKE, None, FAKE, 100, FAKE, 10
    o = _opts(L)
    count, k = 1, 2
    if case == "count0":
        count = 0
    elif case == "k17":
        k = 17
    elif case == "n257":
        q.n, q.ld = 257, 260
    elif case == "ld_odd":
        q.ld = 11
    elif case == "misaligned":
        q.A = FAKE + 4
    elif case == "opts":
        o.max_outer = 0
    out = C.c_void_p(FAKE)
    st = L.load().lsq_batch_create(C.byref(q), count, k, C.byref(o), C.byref(out), None)
    assert st == 1 and msg in _err(lsq)
    assert out.value is None       # the handle is cleared before any check can fail


def test_split_f64_checks_and_empty_input(lsq):
    L = lsq.L.load()
    assert L.lsq_split_f64(None, FAKE, 4, None) == 1
    assert L.lsq_split_f64(FAKE, FAKE, -1, None) == 1
    assert L.lsq_split_f64(FAKE, FAKE, 0, None) == 0     # nothing to convert: no launch


def test_binding_rejects_host_tensors_before_calling_the_library(lsq):
    """The Python layer checks where its tensors live before it hands pointers over (the C
    library cannot tell a host pointer from a device one)."""
    import types
    import torch
    with pytest.raises(ValueError, match="CUDA tensor"):
        lsq.Matrix(torch.zeros(8, 3, dtype=torch.float64))
    with pytest.raises(ValueError, match="row_ptr must be a CUDA tensor"):
        lsq.Matrix(row_ptr=torch.zeros(4, dtype=torch.int64), col_idx=torch.zeros(2, dtype=torch.int32),
                   vals=torch.zeros(2, dtype=torch.float64), n=2)
    with pytest.raises(ValueError, match="B must be a CUDA float64"):
        lsq.lsq_pcg_solve(types.SimpleNamespace(n=3), None, torch.zeros(8, dtype=torch.float64))
    with pytest.raises(KeyError):
        lsq.opts(no_such_option=1)


def test_wait_limit_argument_checks(lsq):
    """lsq_set_wait_limit takes 0 (the defaults) up to 2^31 polls; it touches no device."""
    for bad in (-1, (1 << 31) + 1):
        with pytest.raises(lsq.L.LsqError) as e:
            lsq.set_wait_limit(bad)
        assert e.value.code == 1
    lsq.set_wait_limit(1 << 31)
    lsq.set_wait_limit(0)


def test_sweep_form_argument_checks(lsq):
    """lsq_set_sweep_form takes 0 (by shape) to 3 (cluster); it only stores the setting."""
    for bad in (-1, 4, 100):
        with pytest.raises(lsq.L.LsqError) as e:
            lsq.set_sweep_form(bad)
        assert e.value.code == 1
        assert "form must be" in _err(lsq)
    for good in (1, 2, 3, 0):
        lsq.set_sweep_form(good)


def test_latency_probe_rejects_null_output(lsq):
    L = lsq.L.load()
    assert L.lsq_measure_latency(None, None) == 1
    assert "out_ns" in _err(lsq)
