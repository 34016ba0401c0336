"""lsq_sample_rows_static: the sampling entry point for callers that cannot allocate
device memory (its scratch is one fixed device array of the library).

It must give exactly what lsq_sample_rows gives, call after call, although every call
reuses the same array and so starts from the previous call's leftovers.  This file is
collected last so that a run stopping at the first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _both(lsq, Mx, o):
    a = lsq.lsq_sample_rows(Mx, o)
    b = lsq.lsq_sample_rows_static(Mx, o)
    torch.cuda.synchronize()
    return a, b


def test_static_scratch_matches_allocating_entry_point_twice(lsq):
    mats = [W.udv_dense(30000, 96, 1e4, 2)["A"], W.gaussian_dense(4096, 128, 1001)["A"]]
    for k, A in enumerate(mats):               # two calls in a row, different sizes
        Mx = lsq.Matrix(torch.from_numpy(A).cuda())
        o = lsq.opts(seed=1000 + k)
        (i1, p1, d1), (i2, p2, d2) = _both(lsq, Mx, o)
        assert torch.equal(i1, i2), "sampled rows differ"
        assert torch.equal(p1, p2), "sampling probabilities differ"
        assert torch.equal(d1, d2), "column scales differ"


def test_static_scratch_csr_and_repeat(lsq):
    mat = W.sparse_random(50000, 900, 8, 5)
    Mx = lsq.Matrix(row_ptr=torch.from_numpy(mat["row_ptr"]).cuda(),
                    col_idx=torch.from_numpy(mat["col_idx"]).cuda(),
                    vals=torch.from_numpy(mat["vals"]).cuda(), n=mat["n"])
    o = lsq.opts(seed=7)
    ref = lsq.lsq_sample_rows(Mx, o)
    for _ in range(2):
        got = lsq.lsq_sample_rows_static(Mx, o)
        for r, g in zip(ref, got):
            assert torch.equal(r, g)


def test_static_scratch_rejects_oversize(lsq):
    A = torch.zeros(262145, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(lsq.L.LsqError) as e:
        lsq.lsq_sample_rows_static(lsq.Matrix(A))
    assert e.value.code == 1 and "262144" in str(e.value)


def test_static_scratch_null_colscale_and_launch_count(lsq):
    """colscale_out = NULL keeps the column scales inside the fixed array; the indices and
    probabilities must not change.  Both entry points launch the same kernels, so the
    library's launch counter must rise by the same amount for each."""
    A = torch.from_numpy(W.gaussian_dense(5000, 64, 3)["A"]).cuda()
    Mx = lsq.Matrix(A)
    o = lsq.opts(seed=11)
    n0 = lsq.launches()
    ref_i, ref_p, _ = lsq.lsq_sample_rows(Mx, o)
    n1 = lsq.launches()
    s = ref_i.numel()
    for _ in range(2):
        idx = torch.empty(s, dtype=torch.int32, device="cuda")
        p = torch.empty(s, dtype=torch.float64, device="cuda")
        s_out = C.c_int64(0)
        code = lsq.L.load().lsq_sample_rows_static(Mx.ref, C.byref(o), s, C.c_void_p(idx.data_ptr()),
                                                   C.c_void_p(p.data_ptr()), None, C.byref(s_out),
                                                   lsq._stream(None))
        assert code == 0 and s_out.value == s
        torch.cuda.synchronize()
        assert torch.equal(idx, ref_i) and torch.equal(p, ref_p)
    n2 = lsq.launches()
    assert n1 - n0 == 9 and n2 - n1 == 2 * (n1 - n0)
