"""S1-S4 on the GPU vs the oracle: row indices and probabilities bit for bit."""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import to_device

pytestmark = pytest.mark.gpu


def _check(lsq, orc, mat, dtype="f64", seed=1, s=0, normalize=True, ld_pad=0, sampling="norm2"):
    Mx, keep, seen = to_device(lsq, mat, dtype, ld_pad=ld_pad)
    o = lsq.opts(seed=seed, normalize=int(normalize), sampling=1 if sampling == "uniform" else 0)
    idx, p, d = lsq.lsq_sample_rows(Mx, o, s=s)
    smp = orc.Sample(seen, seed=seed, s=s or None, normalize=normalize, sampling=sampling)
    gi = idx.cpu().numpy()
    assert gi.shape == smp.idx.shape
    assert np.array_equal(gi, smp.idx), f"first mismatch at {np.nonzero(gi != smp.idx)[0][:5]}"
    w = np.array(orc.u128(smp.w_lo, smp.w_hi), dtype=object)
    W_ = smp.W
    p_ref = np.array([float(w[i]) / float(W_) for i in smp.idx])
    assert np.array_equal(p.cpu().numpy(), p_ref)
    assert np.array_equal(d.cpu().numpy(), smp.d)
    return smp


@pytest.mark.parametrize("shape", [(4096, 128), (1000, 37), (3001, 129), (700, 1), (50, 200)])
def test_dense_f64_bitexact(lsq, orc, shape):
    m, n = shape
    _check(lsq, orc, W.gaussian_dense(m, n, 1001), seed=1001)


def test_dense_raw_weights_and_custom_s(lsq, orc):
    mat = W.gaussian_dense(2000, 50, 3)
    mat["A"] *= np.linspace(1e-3, 1e3, 2000)[:, None]
    _check(lsq, orc, mat, seed=9, s=100000, normalize=False)
    _check(lsq, orc, mat, seed=9, s=7)


def test_dense_column_scaling_extremes(lsq, orc):
    mat = W.gaussian_dense(1500, 20, 4)
    mat["A"] *= np.logspace(-100, 100, 20)[None, :]
    mat["A"][:, 5] = 0.0   # an all-zero column
    smp = _check(lsq, orc, mat, seed=2)
    assert smp.d[5] == 1.0


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_dense_low_precision_bitexact(lsq, orc, dtype):
    _check(lsq, orc, W.udv_dense(3000, 64, 1e3, 5), dtype=dtype, seed=77, ld_pad=8)


def test_csr_bitexact(lsq, orc):
    _check(lsq, orc, W.sparse_random(20000, 300, 8, 3), seed=1003)
    _check(lsq, orc, W.graph_incidence(3000, 12000, 4), seed=1004)


def test_coherent_matrix_draws_identity_rows(lsq, orc):
    smp = _check(lsq, orc, W.coherent_dense(5000, 16), seed=3, s=20000)
    assert smp.idx.max() < 16


def test_uniform_sampling_bitexact(lsq, orc):
    """The uniform density of the comparison in Sec. 3.1 (p_i = 1/m): dense, CSR, and the
    coherent matrix, where most draws land on zero rows."""
    _check(lsq, orc, W.gaussian_dense(3001, 40, 8), seed=12, sampling="uniform")
    _check(lsq, orc, W.sparse_random(20000, 300, 8, 3), seed=13, sampling="uniform")
    smp = _check(lsq, orc, W.coherent_dense(5000, 16), seed=3, s=20000, sampling="uniform")
    assert (smp.idx >= 16).mean() > 0.99


def test_udv_full_size_bitexact(lsq, orc):
    # the benchmark workload: 262144 x 512 UDV, kappa = 1e6 (large products on the device)
    mm = lambda X, Y: (torch.from_numpy(np.ascontiguousarray(X)).cuda()
                       @ torch.from_numpy(np.ascontiguousarray(Y)).cuda()).cpu().numpy()
    mat = W.udv_dense(262144, 512, 1e6, 2, matmul=mm)
    _check(lsq, orc, mat, seed=1002)


def test_sparse_full_size_bitexact(lsq, orc):
    # 4,000,000 x 40,000 CSR, 8 nonzeros per row plus one per column
    _check(lsq, orc, W.sparse_random(4_000_000, 40_000, 8, 3), dtype="f32", seed=1003)


def test_invalid_values_rejected(lsq):
    A = torch.randn(100, 4, dtype=torch.float64, device="cuda")
    A[3, 2] = float("nan")
    with pytest.raises(lsq.L.LsqError) as e:
        lsq.lsq_sample_rows(lsq.Matrix(A))
    assert e.value.code == 1
    with pytest.raises(lsq.L.LsqError):
        lsq.lsq_sample_rows(lsq.Matrix(torch.zeros(10, 3, dtype=torch.float64, device="cuda")))
