"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values printed in the
paper, closed forms, invariants, special cases that reduce to a textbook or library
routine (numpy / scipy LAPACK), brute force on tiny inputs, or an independent
implementation of a published definition (numpy's Philox).  None of them re-types the
oracle's own arithmetic.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl
from scipy import stats

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------
# Alg. 2 step 2: s = 4 n log n, pinned by the seven sample sizes the paper prints
# ---------------------------------------------------------------------------------------
def test_sample_size_matches_paper(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "sample_sizes.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 7
    for n, s in rows:
        assert orc.sample_size(int(n)) == int(s), (n, s)


# ---------------------------------------------------------------------------------------
# Philox4x64-10 (Salmon et al., SC'11) against numpy's independent implementation.
# numpy increments its 256-bit counter before producing a block, so block t comes from a
# generator started at counter t - 1.
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("key", [(0, 0x5A4D504C), (12345, 0x5A4D504C), (2**64 - 1, 7)])
@pytest.mark.parametrize("t", [0, 1, 2, 1000, 2**40 + 3])
def test_philox_matches_numpy(orc, key, t):
    ctr = (t - 1) % (1 << 256)
    words = [(ctr >> (64 * i)) & ((1 << 64) - 1) for i in range(4)]
    g = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(words, dtype=np.uint64))
    ref = [int(v) for v in g.random_raw(4)]
    assert orc.philox4x64_10((t, 0, 0, 0), key) == ref


# ---------------------------------------------------------------------------------------
# Eq. (R2P) and Alg. 2 step 1: the exact fixed-point weights against the plain formulas
# ---------------------------------------------------------------------------------------
def _dense_cases():
    return [W.gaussian_dense(300, 17, 1)["A"],
            W.udv_dense(500, 24, 1e4, 2)["A"],
            np.ldexp(W.gaussian_dense(64, 9, 3)["A"], 200),   # large scale
            np.ldexp(W.gaussian_dense(64, 9, 4)["A"], -300)]  # small scale


@pytest.mark.parametrize("case", range(4))
def test_column_scales_equal_column_norms(orc, case):
    A = _dense_cases()[case]
    d2, d, inv, E1 = orc.col_scales({"kind": "dense", "A": A})
    ref = (A * A).sum(axis=0)
    np.testing.assert_allclose(d2, ref, rtol=1e-12)
    np.testing.assert_allclose(d, np.linalg.norm(A, axis=0), rtol=1e-12)


@pytest.mark.parametrize("case", range(4))
def test_row_weights_equal_normalised_row_norms(orc, case):
    A = _dense_cases()[case]
    mat = {"kind": "dense", "A": A}
    d2, d, inv, E1 = orc.col_scales(mat)
    lo, hi = orc.row_weights(mat, inv)
    w = np.array([float((int(h) << 64) | int(l)) for l, h in zip(lo, hi)])
    p = w / w.sum()
    Ah = A / np.linalg.norm(A, axis=0)
    ref = (Ah * Ah).sum(axis=1) / A.shape[1]   # Eq. (R2P) on the normalised matrix: ||â_i||^2 / n
    np.testing.assert_allclose(p, ref, rtol=1e-9, atol=1e-15)
    # the normalised Frobenius norm is n (Sec. 4.1: ||A||_F^2 = n after normalisation)
    assert abs(w.sum() / 2.0**51 - A.shape[1]) < 1e-9 * A.shape[1]


def test_row_weights_raw_mode(orc):
    A = _dense_cases()[1]
    mat = {"kind": "dense", "A": A}
    d2, d, inv, E1 = orc.col_scales(mat, normalize=False)
    assert np.all(d == 1.0)
    lo, hi = orc.row_weights(mat, inv)
    w = np.array([float((int(h) << 64) | int(l)) for l, h in zip(lo, hi)])
    ref = (A * A).sum(axis=1)
    np.testing.assert_allclose(w / w.sum(), ref / ref.sum(), rtol=1e-9)


def test_prefix_is_cumulative_sum(orc):
    rng = np.random.default_rng(5)
    lo = rng.integers(0, 2**63, size=50, dtype=np.uint64)
    hi = rng.integers(0, 4, size=50, dtype=np.uint64)
    P_lo, P_hi = orc.prefix(lo, hi)
    vals = [(int(h) << 64) | int(l) for l, h in zip(lo, hi)]
    acc = 0
    for i in range(50):
        assert (int(P_hi[i]) << 64) | int(P_lo[i]) == acc
        acc += vals[i]
    assert (int(P_hi[50]) << 64) | int(P_lo[50]) == acc


# ---------------------------------------------------------------------------------------
# Alg. 1 draws: special cases and the law of the draws
# ---------------------------------------------------------------------------------------
def test_single_nonzero_row_is_always_drawn(orc):
    A = np.zeros((40, 5))
    A[17] = [1.0, -2.0, 3.0, 0.5, 1.0]
    smp = orc.Sample({"kind": "dense", "A": A}, seed=3, s=500)
    assert np.all(smp.idx == 17)


def test_coherent_Z_draws_only_identity_rows(orc):
    # Sec. 3.1, matrix Z = [I_n; 0]: norm-squared sampling puts all mass on the first n
    # rows, each with probability 1/n.
    m, n = 200, 8
    smp = orc.Sample(W.coherent_dense(m, n), seed=11, s=80000)
    assert smp.idx.max() < n
    counts = np.bincount(smp.idx, minlength=n)
    chi2 = stats.chisquare(counts).pvalue
    assert chi2 > 1e-4


def test_zero_weight_rows_never_drawn_and_chi_square(orc):
    rng = np.random.default_rng(7)
    m, n = 60, 4
    A = rng.standard_normal((m, n)) * rng.uniform(0.1, 3.0, size=(m, 1))
    A[::7] = 0.0                                  # zero rows
    smp = orc.Sample({"kind": "dense", "A": A}, seed=99, s=200000)
    assert not np.isin(smp.idx, np.arange(0, m, 7)).any()
    Ah = A / np.linalg.norm(A, axis=0)
    p = (Ah * Ah).sum(1) / n                      # Eq. (R2P)
    counts = np.bincount(smp.idx, minlength=m)
    keep = p > 0
    res = stats.chisquare(counts[keep], f_exp=p[keep] * smp.s)
    assert res.pvalue > 1e-4, res


def test_draws_reproduce_and_depend_on_seed(orc):
    mat = W.gaussian_dense(1000, 10, 1)
    a = orc.Sample(mat, seed=5).idx
    b = orc.Sample(mat, seed=5).idx
    c = orc.Sample(mat, seed=6).idx
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    # draw t does not depend on how many draws are taken (counter-based)
    smp = orc.Sample(mat, seed=5)
    assert smp.s == 93
    tail = orc.draw_rows(smp.P_lo, smp.P_hi, 5, 10, t0=50)
    assert np.array_equal(tail, smp.idx[50:60])


# ---------------------------------------------------------------------------------------
# Sec. 3.3: the sampled normal matrix
# ---------------------------------------------------------------------------------------
class _FullSample:
    """Every row once with equal weights: then (1/s) sum_t â^T â / p = Â^T Â exactly."""

    def __init__(self, orc, mat, normalize=True):
        self.mat = orc.as_mat(mat)
        self.d2, self.d, self.inv_d2, _ = orc.col_scales(self.mat, normalize)
        m = self.mat.m
        self.w_lo = np.ones(m, np.uint64)
        self.w_hi = np.zeros(m, np.uint64)
        self.idx = np.arange(m, dtype=np.int32)


def test_full_sampling_gives_normalised_normal_matrix(orc):
    A = W.gaussian_dense(50, 7, 8)["A"]
    A[:, 3] *= 100.0
    fs = _FullSample(orc, {"kind": "dense", "A": A})
    M = orc.SampledM(fs).dense()
    Ah = A / np.linalg.norm(A, axis=0)
    np.testing.assert_allclose(M, Ah.T @ Ah, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(np.diag(M), 1.0, rtol=1e-12)


def test_incidence_identity_laplacian(orc):
    # Sec. 5.5: B^T B = D - A for an oriented incidence matrix, whatever the orientation.
    rng = np.random.default_rng(3)
    N = 12
    edges = {(i, j) for i, j in rng.integers(0, N, size=(40, 2)) if i != j}
    edges = sorted({(min(i, j), max(i, j)) for i, j in edges})
    B = np.zeros((len(edges), N))
    for e, (i, j) in enumerate(edges):
        s = 1.0 if rng.random() < 0.5 else -1.0
        B[e, i], B[e, j] = s, -s
    fs = _FullSample(orc, W.csr_from_dense(B, keep_zeros=False), normalize=False)
    M = orc.SampledM(fs).dense()
    Adj = np.zeros((N, N))
    for i, j in edges:
        Adj[i, j] = Adj[j, i] = 1.0
    Lap = np.diag(Adj.sum(1)) - Adj
    deg0 = np.diag(Lap) == 0
    Lap[deg0, deg0] = 1.0   # an isolated node has a zero diagonal, replaced by 1
    np.testing.assert_allclose(M, Lap, atol=1e-12)


def test_sampled_normal_matrix_is_unbiased(orc):
    # Eq. (EATA): E[A_s^T A_s] = A^T A.  Monte Carlo over 400 seeds on a tiny matrix.
    A = W.gaussian_dense(30, 4, 2)["A"] * np.linspace(0.2, 3, 30)[:, None]
    mat = {"kind": "dense", "A": A}
    Ah = A / np.linalg.norm(A, axis=0)
    N = Ah.T @ Ah
    reps = [orc.SampledM(orc.Sample(mat, seed=sd, s=12)).dense() for sd in range(400)]
    mean = np.mean(reps, axis=0)
    se = np.std(reps, axis=0) / np.sqrt(len(reps))
    assert np.all(np.abs(mean - N) <= 5 * se + 1e-12)


def test_uniform_sampled_normal_matrix_is_unbiased(orc):
    """The same expectation under the uniform density of Sec. 3.1 (p_i = 1/m): each draw is
    weighted m/s, and the mean over 400 seeds must still be Â^T Â.  A uniform M that kept
    the norm-squared weights 1/(s p_i) for the drawn rows, or dropped the factor m, fails."""
    A = W.gaussian_dense(30, 4, 2)["A"] * np.linspace(0.2, 3, 30)[:, None]
    mat = {"kind": "dense", "A": A}
    Ah = A / np.linalg.norm(A, axis=0)
    N = Ah.T @ Ah
    reps = [orc.SampledM(orc.Sample(mat, seed=sd, s=12, sampling="uniform")).dense() for sd in range(400)]
    mean = np.mean(reps, axis=0)
    se = np.std(reps, axis=0) / np.sqrt(len(reps))
    assert np.all(np.abs(mean - N) <= 5 * se + 1e-12)


def test_spectral_error_within_the_paper_bound(orc):
    """Sec. 3.2, the approximation theorem: for ||Â||_F^2 = n, eps and delta in (0, 1),
    C = (2/3)(6 ||Â||^2 + 2 eps)(1 - log_n(delta / 2)) and s = C eps^-2 n log n give
    ||A_s^T A_s - Â^T Â||_2 <= eps with probability at least 1 - delta.  Twenty seeds must
    all meet it, and the error must shrink like s^(-1/2) (the matrix Bernstein rate)."""
    mat = W.gaussian_dense(2000, 20, 3)
    n = 20
    Ah = mat["A"] / np.linalg.norm(mat["A"], axis=0)
    N = Ah.T @ Ah
    eps, delta = 0.5, 0.01
    C = (2.0 / 3.0) * (6.0 * np.linalg.norm(Ah, 2) ** 2 + 2.0 * eps) * (1.0 - math.log(delta / 2) / math.log(n))
    s = math.ceil(C * n * math.log(n) / eps ** 2)

    def err(seed, draws):
        return np.linalg.norm(orc.SampledM(orc.Sample(mat, seed=seed, s=draws)).dense() - N, 2)
    errs = [err(sd, s) for sd in range(20)]
    assert max(errs) <= eps, (s, max(errs))
    errs16 = [err(sd, 16 * s) for sd in range(5)]
    ratio = np.mean(errs16) / np.mean(errs[:5])
    assert 0.15 <= ratio <= 0.4, ratio           # 1/sqrt(16) = 0.25


def test_unsampled_column_gets_unit_diagonal(orc):
    """A column no drawn row touches has M_jj = 0; it becomes 1, the diagonal of the
    normalised A^T A, and it is the only entry of its row and column.  Column 2 lives in
    row 9 only; column 3 is all zero, so no seed can reach it.  Which columns the draws
    miss is counted here by brute force from the drawn rows."""
    A = np.zeros((10, 4))
    A[:5, 0] = 1.0
    A[5:, 1] = 2.0
    A[9, 2] = 1e-30
    mat = {"kind": "dense", "A": A}
    seen_missed_2 = seen_hit_2 = False
    for seed in range(1, 60):
        smp = orc.Sample(mat, seed=seed, s=4)
        drawn = np.unique(smp.idx)
        missed = [j for j in range(4) if not np.any(A[drawn, j] != 0)]
        Mo = orc.SampledM(smp)
        Md = Mo.dense()
        assert Mo.n_fixed_diag == len(missed) and 3 in missed
        for j in range(4):
            if j in missed:
                assert Md[j, j] == 1.0
                assert np.count_nonzero(Md[j]) == 1 and np.count_nonzero(Md[:, j]) == 1
            else:
                assert Md[j, j] > 0.0
        seen_missed_2 |= 2 in missed
        seen_hit_2 |= 2 not in missed
    assert seen_missed_2 and seen_hit_2


def test_sparse_and_dense_M_agree(orc):
    mat = W.sparse_random(400, 30, 4, 9)
    dense = {"kind": "dense", "A": W.dense_from_csr(mat)}
    s1 = orc.Sample(mat, seed=4)
    s2 = orc.Sample(dense, seed=4)
    assert np.array_equal(s1.idx, s2.idx)   # zeros carry no weight: same law, same draws
    M1 = orc.SampledM(s1).dense()
    M2 = orc.SampledM(s2).dense()
    np.testing.assert_allclose(M1, M2, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------------------
# Alg. 3: the SGS preconditioner
# ---------------------------------------------------------------------------------------
def _spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    return (Q * np.logspace(0, -np.log10(cond), n)) @ Q.T


def _Mo(orc, Md):
    n = Md.shape[0]
    rows, cols = np.nonzero(np.ones_like(Md))
    return orc.SampledM.from_csr(n, np.arange(0, n * n + 1, n), cols.astype(np.int32), Md.reshape(-1))


def test_sgs_one_sweep_closed_form(orc):
    # t = 1 from e0 = 0: e = B^{-T} D B^{-1} r with B the lower triangle (incl. diagonal)
    Md = _spd(9, 1)
    Mo = _Mo(orc, Md)
    Bl = np.tril(Md)
    D = np.diag(np.diag(Md))
    P = sl.solve_triangular(Bl.T, D @ sl.solve_triangular(Bl, np.eye(9), lower=True), lower=False)
    rng = np.random.default_rng(2)
    for _ in range(3):
        r = rng.standard_normal(9)
        np.testing.assert_allclose(orc.sgs_apply(Mo, r, 1), P @ r, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("t", [1, 2, 5])
def test_sgs_symmetric_positive_definite(orc, t):
    Md = _spd(12, 3, cond=1e4)
    Mo = _Mo(orc, Md)
    P = np.column_stack([orc.sgs_apply(Mo, e, t) for e in np.eye(12)])
    np.testing.assert_allclose(P, P.T, rtol=1e-9, atol=1e-9 * np.abs(P).max())
    assert np.linalg.eigvalsh((P + P.T) / 2).min() > 0


def test_sgs_many_sweeps_converge_to_inverse(orc):
    # Gauss-Seidel converges for SPD matrices: t -> infinity gives M^{-1}
    Md = _spd(8, 4, cond=10.0)
    Mo = _Mo(orc, Md)
    r = np.random.default_rng(1).standard_normal(8)
    np.testing.assert_allclose(orc.sgs_apply(Mo, r, 200), np.linalg.solve(Md, r), rtol=1e-10)


def test_sgs_diagonal_matrix_is_exact_inverse(orc):
    d = np.array([2.0, 0.5, 4.0, 1.0])
    Mo = _Mo(orc, np.diag(d))
    r = np.array([1.0, -2.0, 3.0, 0.25])
    np.testing.assert_allclose(orc.sgs_apply(Mo, r, 1), r / d, rtol=1e-15)


# ---------------------------------------------------------------------------------------
# The two products and PCG (Alg. 2 step 4)
# ---------------------------------------------------------------------------------------
def test_normal_matvec_matches_numpy(orc):
    mat = W.sparse_random(300, 20, 5, 1)
    A = W.dense_from_csr(mat)
    d = np.linalg.norm(A, axis=0)
    p = np.random.default_rng(0).standard_normal(20)
    Ah = A / d
    np.testing.assert_allclose(orc.normal_matvec(mat, d, p), Ah.T @ (Ah @ p), rtol=1e-12)


@pytest.mark.parametrize("normal_form", [False, True])
def test_pcg_stop_test_is_relative(orc, normal_form):
    """Alg. 2 step 4 stops on a relative residual, so the method is homogeneous in b:
    scaling b (or h) by a power of two scales every iterate exactly and leaves the
    iteration count, the restarts and the reported ratios unchanged, bit for bit."""
    mat = W.udv_dense(400, 20, 1e3, 6)
    smp = orc.Sample(mat, seed=4)
    Mo = orc.SampledM(smp)
    xs, b = W.rhs_for(mat, 1, 1e-3, 8)
    v = orc.csr_rmatvec(mat, b[0]) / smp.d if normal_form else b[0]

    def run(vec):
        kw = {"h": vec} if normal_form else {"b": vec}
        return orc.pcg(smp.mat, smp.d, Mo, tol=1e-10, maxit=1000, max_outer=5, **kw)
    y0, i0 = run(v)
    assert i0["converged"] == 1 and i0["iters"] > 5
    for e in (-30, 30):
        y, i = run(np.ldexp(v, e))
        assert (i["iters"], i["outer"], i["converged"]) == (i0["iters"], i0["outer"], 1)
        assert i["relres_true"] == i0["relres_true"] and i["relres_rec"] == i0["relres_rec"]
        assert np.array_equal(y, np.ldexp(y0, e))


@pytest.mark.parametrize("gen", ["gauss", "udv", "sparse", "semi"])
def test_pcg_matches_lapack_least_squares(orc, gen):
    if gen == "gauss":
        mat = W.gaussian_dense(600, 20, 1)
    elif gen == "udv":
        mat = W.udv_dense(800, 16, 1e3, 2)
    elif gen == "semi":
        mat = W.semi_gaussian_dense(500, 16, 3)
    else:
        mat = W.sparse_random(900, 25, 6, 3)
    A = mat["A"] if mat["kind"] == "dense" else W.dense_from_csr(mat)
    xs, b = W.rhs_for(mat, 1, 1e-3, 4)
    S = orc.Solve(mat, b[0], seed=10, tol=1e-12)
    assert S.info["converged"] == 1
    x_ref = np.linalg.lstsq(A, b[0], rcond=None)[0]                   # QR / SVD (LAPACK)
    kappa2 = np.linalg.cond(A / np.linalg.norm(A, axis=0)) ** 2
    assert np.linalg.norm(S.x - x_ref) / np.linalg.norm(x_ref) <= 10 * kappa2 * 1e-12
    # also the Cholesky solve of the normal equation (Eq. NOR)
    c = sl.cho_factor(A.T @ A)
    x_ne = sl.cho_solve(c, A.T @ b[0])
    assert np.linalg.norm(S.x - x_ne) / np.linalg.norm(x_ne) <= 10 * kappa2 * 1e-12
    r = A.T @ (b[0] - A @ S.x)
    assert np.linalg.norm(r) / np.linalg.norm(A.T @ b[0]) <= 1e-11


def test_pcg_on_singular_graph_laplacian_gives_the_projection(orc):
    """Sec. 5.5: for the incidence matrix B of a graph, B^T B is singular (one constant null
    vector per connected component) but B^T B x = B^T b is consistent.  PCG then converges to
    a solution whose fitted values B x are the orthogonal projection of b onto range(B), which
    LAPACK's minimum-norm least-squares solution gives independently; the oracle's x may differ
    from that one only by a per-component constant."""
    mat = W.chung_lu_incidence(40, 3)
    B = W.dense_from_csr(mat)
    b = np.random.default_rng(2).standard_normal(mat["m"])
    for sweeps in (1, 5):
        S = orc.Solve(mat, b, seed=4, tol=1e-12, sweeps=sweeps)
        assert S.info["converged"] == 1
        x_mn, res, rank, sv = np.linalg.lstsq(B, b, rcond=None)
        assert rank < mat["n"]                                        # really singular
        kappa = sv[0] / sv[rank - 1]
        fit = B @ x_mn
        assert np.linalg.norm(B @ S.x - fit) / np.linalg.norm(fit) <= 10 * kappa ** 2 * 1e-12
        # the difference lies in the null space: B (x - x_mn) = 0 up to the same bar, and
        # x - x_mn is constant on each component
        dx = S.x - x_mn
        nul = sl.null_space(B)
        assert np.linalg.norm(dx - nul @ (nul.T @ dx)) <= 10 * kappa ** 2 * 1e-12 * np.linalg.norm(x_mn)


def test_pcg_energy_error_decreases_monotonically(orc):
    # CG minimises the A^T A-norm of the error over growing Krylov spaces.
    mat = W.udv_dense(400, 12, 1e2, 5)
    A = mat["A"]
    xs, b = W.rhs_for(mat, 1, 0.0, 6)
    smp = orc.Sample(mat, seed=3)
    Mo = orc.SampledM(smp)
    Ah = A / smp.d
    N = Ah.T @ Ah
    y_star = np.linalg.solve(N, Ah.T @ b[0])
    errs = []
    for k in range(1, 13):
        y, info = orc.pcg(smp.mat, smp.d, Mo, b=b[0], tol=1e-300, maxit=k, max_outer=1)
        e = y - y_star
        errs.append(e @ N @ e)
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) for i in range(len(errs) - 1))


def test_pcg_terminates_in_n_steps_when_well_conditioned(orc):
    # exact arithmetic terminates in at most n steps; FP64 on a well-conditioned problem
    # gets there up to rounding
    mat = W.udv_dense(400, 12, 3.0, 5)
    A = mat["A"]
    xs, b = W.rhs_for(mat, 1, 0.0, 6)
    smp = orc.Sample(mat, seed=3)
    Mo = orc.SampledM(smp)
    Ah = A / smp.d
    N = Ah.T @ Ah
    y_star = np.linalg.solve(N, Ah.T @ b[0])
    y0, _ = orc.pcg(smp.mat, smp.d, Mo, b=b[0], tol=1e-300, maxit=1, max_outer=1)
    y, _ = orc.pcg(smp.mat, smp.d, Mo, b=b[0], tol=1e-300, maxit=12, max_outer=1)
    e0, e = y0 - y_star, y - y_star
    assert e @ N @ e <= 1e-24 * (e0 @ N @ e0)


def _three_eigenvalue_matrix(m=300, pairs=5, ident=4, c=0.6, seed=8):
    """Unit-norm columns whose Gram matrix has exactly three distinct eigenvalues: an
    orthonormal Q (m x n) times a block-diagonal B with 2 x 2 blocks of unit columns at
    cosine c (eigenvalues 1 - c, 1 + c) and identity columns (eigenvalue 1)."""
    n = 2 * pairs + ident
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((m, n)))
    B = np.eye(n)
    for k in range(pairs):
        a = 2 * k
        B[a:a + 2, a:a + 2] = [[1.0, c], [0.0, math.sqrt(1 - c * c)]]
    return Q @ B


def test_cg_baseline_terminates_in_three_steps(orc):
    # t = 0: CG on the column-normalised matrix (the paper's comparison method).  With
    # three distinct eigenvalues of A^T A, CG reaches the solution in exactly three steps
    # in exact arithmetic (the Krylov space has dimension 3 for a generic right-hand side).
    A = _three_eigenvalue_matrix()
    mat = {"kind": "dense", "A": A}
    assert np.allclose(np.linalg.norm(A, axis=0), 1.0)
    ev = np.linalg.eigvalsh(A.T @ A)
    assert len(np.unique(np.round(ev, 12))) == 3
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    smp = orc.Sample(mat, seed=2)
    Mo = orc.SampledM(smp)
    y, info = orc.pcg(smp.mat, smp.d, Mo, b=b, tol=1e-10, maxit=50, max_outer=1, sweeps=0)
    assert info["converged"] == 1 and info["iters"] == 3
    x_ref = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(y / smp.d - x_ref) <= 1e-12 * np.linalg.norm(x_ref)
    # the sampled SGS preconditioner gives a different (preconditioned) iteration
    _, info1 = orc.pcg(smp.mat, smp.d, Mo, b=b, tol=1e-10, maxit=50, max_outer=1, sweeps=1)
    assert info1["converged"] == 1


def test_pcg_iteration_count_zero_for_zero_rhs(orc):
    mat = W.gaussian_dense(100, 5, 1)
    S = orc.Solve(mat, np.zeros(100), seed=1)
    assert S.info["iters"] == 0 and S.info["converged"] == 1 and np.all(S.x == 0)


# ---------------------------------------------------------------------------------------
# Adjoint: dL/db = A lam, dL/dA = r lam^T - (A lam) x^T with A^T A lam = dL/dx
# ---------------------------------------------------------------------------------------
def test_adjoint_matches_closed_form_and_finite_differences(orc):
    mat = W.gaussian_dense(80, 6, 2)
    A = mat["A"]
    xs, b = W.rhs_for(mat, 1, 1e-1, 3)
    b = b[0]
    target = np.random.default_rng(1).standard_normal(6)

    def loss(Am, bm):
        S = orc.Solve({"kind": "dense", "A": Am}, bm, seed=2, tol=1e-14)
        return np.sum((S.x - target) ** 2), S

    L0, S = loss(A, b)
    G = 2 * (S.x - target)
    gb, gA, lam, info = orc.adjoint(mat, S.smp, S.M, S.x, b, G, tol=1e-14)
    lam_ref = np.linalg.solve(A.T @ A, G)
    np.testing.assert_allclose(lam, lam_ref, rtol=1e-9)
    r = b - A @ S.x
    np.testing.assert_allclose(gA, np.outer(r, lam_ref) - np.outer(A @ lam_ref, S.x), rtol=1e-8, atol=1e-12)
    h = 1e-6
    for i in [0, 17, 79]:
        e = np.zeros_like(b)
        e[i] = h
        fd = (loss(A, b + e)[0] - loss(A, b - e)[0]) / (2 * h)
        assert abs(fd - gb[i]) <= 1e-6 * max(1.0, abs(gb[i]))
    for (i, j) in [(0, 0), (40, 3), (79, 5)]:
        E = np.zeros_like(A)
        E[i, j] = h
        fd = (loss(A + E, b)[0] - loss(A - E, b)[0]) / (2 * h)
        assert abs(fd - gA[i, j]) <= 1e-6 * max(1.0, abs(gA[i, j]))


def test_csr_adjoint_equals_the_dense_gradient_on_the_stored_entries(orc):
    """The CSR form of the adjoint returns dL/dA only at A's stored entries: those must be
    the entries of the dense closed form r lam^T - (A lam) x^T (pinned above) for the same
    matrix, and dL/db and lam must be the dense ones."""
    mat = W.sparse_random(400, 12, 4, 5)
    A = W.dense_from_csr(mat)
    xs, b = W.rhs_for(mat, 1, 1e-1, 3)
    b = b[0]
    S = orc.Solve(mat, b, seed=2, tol=1e-14)
    G = 2 * (S.x - np.random.default_rng(1).standard_normal(12))
    gb, gv, lam, info = orc.adjoint(mat, S.smp, S.M, S.x, b, G, tol=1e-14)
    lam_ref = np.linalg.solve(A.T @ A, G)
    np.testing.assert_allclose(lam, lam_ref, rtol=1e-9)
    np.testing.assert_allclose(gb, A @ lam_ref, rtol=1e-9, atol=1e-12)
    r = b - A @ S.x
    gA = np.outer(r, lam_ref) - np.outer(A @ lam_ref, S.x)
    rows = np.repeat(np.arange(400), np.diff(mat["row_ptr"]))
    np.testing.assert_allclose(gv, gA[rows, mat["col_idx"]], rtol=1e-8, atol=1e-12)
    # and central finite differences in three stored values
    target = S.x - G / 2

    def loss(vals):
        m2 = dict(mat)
        m2["vals"] = vals
        return np.sum((orc.Solve(m2, b, seed=2, tol=1e-14).x - target) ** 2)

    h = 1e-6
    for q in (0, 517, mat["vals"].size - 1):
        e = np.zeros_like(mat["vals"])
        e[q] = h
        fd = (loss(mat["vals"] + e) - loss(mat["vals"] - e)) / (2 * h)
        assert abs(fd - gv[q]) <= 1e-6 * max(1.0, abs(gv[q])), (q, fd, gv[q])


# ---------------------------------------------------------------------------------------
# Sec. 5.1-5.2: the iteration counts the paper prints for its well-conditioned examples.
# The paper does not state b; a standard normal b is used.  CG on the normalised A is a
# deterministic function of A, so its count must match the printed one up to the
# realisation of A (+-1); RS must fall inside the printed mean +- (3 std + 1).  The
# smaller rows keep the CPU suite short; all ten rows match (n up to 400).
# ---------------------------------------------------------------------------------------
def _paper_rows():
    rows = []
    for line in open(os.path.join(GOLDEN, "paper_iterations.txt")):
        if line.strip() and line[0] != "#":
            f = line.split()
            rows.append((f[0], int(f[1]), int(f[2]), int(f[3]), int(f[4]), float(f[5]), float(f[6])))
    return rows


@pytest.mark.parametrize("row", [r for r in _paper_rows() if r[1] <= 141],
                         ids=lambda r: f"{r[0]}{r[1]}x{r[2]}")
def test_iteration_counts_match_paper_tables(orc, row):
    family, n, m, it_cg, it_rs, rs_mean, rs_std = row
    mat = W.gaussian_dense(m, n, 1) if family == "gauss" else W.semi_gaussian_dense(m, n, 1)
    b = np.random.default_rng(5).standard_normal(m)
    counts = {}
    for sweeps, seeds in ((0, [1]), (5, [1, 2, 3, 4])):
        for sd in seeds:
            smp = orc.Sample(mat, seed=sd)
            assert smp.s == math.ceil(4 * n * math.log(n))
            y, info = orc.pcg(smp.mat, smp.d, orc.SampledM(smp), b=b, tol=1e-7, maxit=1000,
                              max_outer=5, sweeps=sweeps)
            assert info["converged"] == 1 and info["relres_true"] <= 1e-7
            counts.setdefault(sweeps, []).append(info["iters"])
    assert abs(counts[0][0] - it_cg) <= 1, (counts, it_cg)
    lo, hi = rs_mean - 3 * rs_std - 1, rs_mean + 3 * rs_std + 1
    assert all(lo <= c <= hi for c in counts[5]), (counts[5], rs_mean, rs_std)


# ---------------------------------------------------------------------------------------
# The uniform density of the comparison in Sec. 3.1 (p_i = 1/m) and why the method does not
# use it: on a coherent matrix uniform draws miss the rows that carry the columns.
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("m", [777, 4096])
def test_uniform_draws_are_floor_of_U_times_m(orc, m):
    """With every weight 1 the draw of Alg. 1 is i_t = floor(U_t m / 2^128), U_t the 128-bit
    word of Philox block t: computed here from numpy's independent Philox and Python ints."""
    mat = W.gaussian_dense(m, 5, 3)
    smp = orc.Sample(mat, seed=99, s=300, sampling="uniform")
    key = np.array([99, 0x5A4D504C], dtype=np.uint64)
    want = []
    for t in range(300):
        ctr = (t - 1) % (1 << 256)
        words = [(ctr >> (64 * i)) & ((1 << 64) - 1) for i in range(4)]
        raw = [int(v) for v in np.random.Philox(key=key, counter=np.array(words, dtype=np.uint64)).random_raw(2)]
        U = (raw[1] << 64) | raw[0]
        want.append((U * m) >> 128)
    assert smp.idx.tolist() == want


def test_uniform_draws_are_uniform(orc):
    m, s = 64, 64000
    smp = orc.Sample(W.gaussian_dense(m, 4, 5), seed=3, s=s, sampling="uniform")
    counts = np.bincount(smp.idx, minlength=m)
    chi2 = float(((counts - s / m) ** 2 / (s / m)).sum())
    assert chi2 < 120.0          # 63 degrees of freedom: the 0.9999 quantile is about 115


def test_uniform_sampling_misses_the_rows_of_a_coherent_matrix(orc):
    """Z = [I; 0] (Sec. 3.1): the norm-squared density draws only the n identity rows, so
    every column of A_s^T A_s is sampled; uniform draws almost always land on zero rows, so
    most diagonal entries of A_s^T A_s stay zero (replaced by 1) and A_s^T A_s is a poor
    approximation of A^T A = I."""
    m, n = 4000, 40
    mat = W.coherent_dense(m, n)
    s = orc.sample_size(n)
    nrm = orc.Sample(mat, seed=5)
    uni = orc.Sample(mat, seed=5, sampling="uniform")
    assert nrm.idx.max() < n and len(set(nrm.idx.tolist())) == n
    hits = int((uni.idx < n).sum())
    assert hits < 0.1 * s                     # about s n / m = 24 of 591 draws
    Mn, Mu = orc.SampledM(nrm), orc.SampledM(uni)
    assert Mn.n_fixed_diag == 0 and Mu.n_fixed_diag >= n // 2
    # with the method's density M is diag(counts) n / s, near the identity (Sec. 3.2); the
    # uniform draws that do hit an identity row weigh m / s each, far from it
    assert np.abs(Mn.dense() - np.eye(n)).max() < 1.0 < np.abs(Mu.dense() - np.eye(n)).max()


def test_uniform_sampling_on_the_semi_gaussian_identity_block(orc):
    """Sec. 5.2's [B 0; 0 I] under uniform draws (p_i = 1/m): an identity column j is touched
    only by its own row, so row j of A_s^T A_s is c_j m / s on the diagonal and zero elsewhere
    (c_j = times that row was drawn), and a column never drawn gets the replaced diagonal 1,
    which is exactly its entry of Â^T Â."""
    m, n = 3000, 40
    h = n // 2
    mat = W.semi_gaussian_dense(m, n, 21)
    smp = orc.Sample(mat, seed=7, sampling="uniform")
    M = orc.SampledM(smp).dense()
    first = m - (n - h)                        # the identity rows are the last n - h
    counts = np.bincount(smp.idx, minlength=m)[first:]
    assert (counts == 0).sum() >= 1 and (counts > 0).sum() >= 1
    for k in range(n - h):
        j = h + k
        want = 1.0 if counts[k] == 0 else counts[k] * m / smp.s
        assert M[j, j] == pytest.approx(want, rel=1e-14)
        assert np.count_nonzero(M[j]) == 1 and np.count_nonzero(M[:, j]) == 1
    assert orc.SampledM(smp).n_fixed_diag == int((counts == 0).sum())


def test_uniform_sampling_is_a_weaker_preconditioner_when_rows_differ(orc):
    """Sec. 3.1 on a matrix whose columns are carried by a few rows (400 Gaussian rows of
    20000; the rest scaled by 1e-3): PCG with the norm-squared density converges in a
    fraction of the iterations that uniform sampling needs (measured 18 against 96)."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((20000, 100))
    A[400:] *= 1e-3
    mat = {"kind": "dense", "A": A}
    xs, b = W.rhs_for(mat, 1, 1e-3, 6)
    its = {}
    for sampling in ("norm2", "uniform"):
        smp = orc.Sample(mat, seed=5, sampling=sampling)
        y, oi = orc.pcg(smp.mat, smp.d, orc.SampledM(smp), b=b[0], tol=1e-10, maxit=10000, max_outer=20)
        assert oi["converged"] == 1
        its[sampling] = oi["iters"]
    assert its["norm2"] <= 25 and its["uniform"] >= 3 * its["norm2"], its
