"""CSR path on the GPU vs the oracle: sampled normal matrix (SpGEMM), the Gauss-Seidel
sweeps of Alg. 3 on it, PCG and the adjoint."""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import assert_iterations, assert_solution, rel, rounding_variant_iters, to_device

pytestmark = pytest.mark.gpu


def _same_solution(seen, d, x_gpu, y_or, b, tol):
    """Both solutions meet the normal equation to tol, so Â^T Â (y_gpu - y_or) is the
    difference of their two residuals: its norm is at most (tol_gpu + tol_or) ||Â^T b||.
    This checks the GPU solution against the oracle's without forming or factoring Â."""
    import scipy.sparse as sps
    A = sps.csr_matrix((seen["vals"], seen["col_idx"], seen["row_ptr"]), shape=(seen["m"], seen["n"]))
    Ah = A @ sps.diags(1.0 / d)
    dy = x_gpu * d - y_or
    h = Ah.T @ b
    return np.linalg.norm(Ah.T @ (Ah @ dy)) <= 2.05 * tol * np.linalg.norm(h)


def _variants(orc, seen, smp, Mo, b, o):
    """The oracle's equally valid FP64 evaluations of this solve (computed on demand)."""
    return lambda: rounding_variant_iters(orc, seen, smp, Mo, b, o.tol, o.sweeps, o.maxit, o.max_outer)


def _setup(lsq, orc, mat, seed, sweeps=1, dtype="f64", pdt=0, with_f64=False):
    Mx, keep, seen = to_device(lsq, mat, dtype, with_f64=with_f64)
    o = lsq.opts(seed=seed, sweeps=sweeps, precond_dtype=pdt)
    idx, p, d = lsq.lsq_sample_rows(Mx, o)
    P = lsq.lsq_build_precond(Mx, idx, p, d, o)
    smp = orc.Sample(seen, seed=seed)
    Mo = orc.SampledM(smp)
    return Mx, keep, seen, o, P, smp, Mo


CASES = {
    "sprand": lambda: W.sparse_random(20000, 300, 8, 3),
    "graph": lambda: W.graph_incidence(2000, 9000, 4),
    "wide": lambda: W.sparse_random(60000, 2000, 8, 5),
    "mid": lambda: W.sparse_random(30000, 3000, 4, 7),
    # wide levels (~1000 rows each): the sweeps run on the whole grid, not in one CTA
    "graph_wide": lambda: W.graph_incidence(20000, 90000, 4),
}


@pytest.mark.parametrize("case", list(CASES))
def test_sparse_normal_matrix_pattern_and_values(lsq, orc, case):
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES[case](), 1003)
    rp, ci, va = (t.cpu().numpy() for t in P.M_csr())
    assert np.array_equal(rp, Mo.row_ptr), "row pointers of A_s^T A_s differ"
    assert np.array_equal(ci, Mo.col), "column pattern of A_s^T A_s differs"
    np.testing.assert_allclose(va, Mo.val, rtol=1e-12, atol=1e-14 * np.abs(Mo.val).max())


@pytest.mark.parametrize("sweeps", [1, 2])
@pytest.mark.parametrize("case", ["sprand", "graph", "wide", "graph_wide"])
def test_sparse_sweeps_match_alg3(lsq, orc, case, sweeps):
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES[case](), 1003, sweeps=sweeps)
    rng = np.random.default_rng(sweeps)
    R = rng.standard_normal((3, seen["n"]))
    E = P.apply(torch.from_numpy(R).cuda()).cpu().numpy()
    for c in range(3):
        assert rel(E[c], orc.sgs_apply(Mo, R[c], sweeps)) <= 1e-11


@pytest.mark.parametrize("case,noise", [("sprand", 1e-3), ("graph", 1e-4), ("graph_wide", 1e-4)])
def test_sparse_pcg_matches_oracle(lsq, orc, case, noise):
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES[case](), 1003)
    xs, b = W.rhs_for(seen, 2, noise, 17)
    X, info = lsq.lsq_pcg_solve(Mx, P, torch.from_numpy(b).cuda(), o)
    X = X.cpu().numpy()
    small = seen["n"] <= 5000
    if small:
        kappa = np.linalg.cond(W.dense_from_csr(seen) / smp.d)
    for c in range(2):
        y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[c], tol=o.tol, maxit=o.maxit, max_outer=o.max_outer)
        x_or = y / smp.d
        assert info.converged[c] == 1 and oi["converged"] == 1
        assert info.relres_true[c] <= o.tol
        if small:
            assert_solution(X[c], x_or, kappa, f"{case} column {c}")
        assert _same_solution(seen, smp.d, X[c], y, b[c], o.tol)
        assert_iterations(info.iters[c], oi["iters"], _variants(orc, seen, smp, Mo, b[c], o), f"{case} column {c}")
    assert info.nnz_M == Mo.val.size
    # forward level count of Alg. 3's dependency DAG, computed here from M's pattern
    lev = np.zeros(seen["n"], np.int64)
    for j in range(seen["n"]):
        cols = Mo.col[Mo.row_ptr[j]:Mo.row_ptr[j + 1]]
        dep = cols[cols < j]
        lev[j] = 1 + lev[dep].max() if dep.size else 0
    assert info.levels == lev.max() + 1


def test_sparse_f32_values_with_f64_refinement(lsq, orc):
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES["sprand"](), 7, dtype="f32", pdt=1, with_f64=True)
    o.max_outer = 30
    o.inner_tol = 1e-4
    xs, b = W.rhs_for(seen, 1, 1e-3, 9)
    X, info = lsq.lsq_pcg_solve(Mx, P, torch.from_numpy(b[0]).cuda(), o)
    assert info.converged[0] == 1 and info.relres_true[0] <= o.tol
    # against the oracle's FP64 solve of the same (FP32-rounded) matrix: both meet the
    # normal equation to tol, so their difference does in the Â^T Â norm
    y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[0], tol=o.tol, maxit=o.maxit, max_outer=20)
    assert oi["converged"] == 1
    assert _same_solution(seen, smp.d, X.cpu().numpy(), y, b[0], o.tol)


@pytest.mark.parametrize("device_loop", [0, 1])
def test_sparse_adjoint_matches_oracle(lsq, orc, device_loop):
    mat = W.sparse_random(5000, 60, 6, 2)
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, mat, 6)
    o.tol = 1e-12
    o.device_loop = device_loop
    xs, b = W.rhs_for(seen, 2, 1e-2, 8)
    B = torch.from_numpy(b).cuda()
    X, info = lsq.lsq_pcg_solve(Mx, P, B, o)
    G = 2 * (X - torch.from_numpy(xs).cuda())
    gb, gv, lam, ainfo = lsq.lsq_pcg_adjoint(Mx, P, X, B, G, o)
    Xh, Gh = X.cpu().numpy(), G.cpu().numpy()
    gsum = 0
    for c in range(2):
        gbr, gvr, lamr, _ = orc.adjoint(seen, smp, Mo, Xh[c], b[c], Gh[c], tol=1e-12)
        assert rel(lam[c].cpu().numpy(), lamr) <= 1e-8
        assert rel(gb[c].cpu().numpy(), gbr) <= 1e-8
        gsum = gsum + gvr
    assert rel(gv.cpu().numpy(), gsum) <= 1e-8


@pytest.mark.parametrize("case", ["sprand", "graph", "graph_wide"])
def test_sparse_pcg_single_column_matches_oracle(lsq, orc, case):
    """k = 1 runs the one-column path (lanes per row of A; scalar recurrences)."""
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES[case](), 2029)
    xs, b = W.rhs_for(seen, 1, 1e-3, 23)
    X, info = lsq.lsq_pcg_solve(Mx, P, torch.from_numpy(b[0]).cuda(), o)
    y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[0], tol=o.tol, maxit=o.maxit, max_outer=o.max_outer)
    assert info.converged[0] == 1 and oi["converged"] == 1
    x = X.cpu().numpy().reshape(-1)
    if seen["n"] <= 5000:
        kappa = np.linalg.cond(W.dense_from_csr(seen) / smp.d)
        assert_solution(x, y / smp.d, kappa, f"{case} one column")
    assert _same_solution(seen, smp.d, x, y, b[0], o.tol)
    assert_iterations(info.iters[0], oi["iters"], _variants(orc, seen, smp, Mo, b[0], o), f"{case} one column")


def test_sparse_block_ragged_mixed_columns(lsq, orc):
    """37 right-hand sides = a block of 32 and a ragged block of 5; one zero column, one
    consistent column (b in the range of A), the rest noisy.  Every column must match the
    same column solved alone (one-column path) and, for a few, the oracle."""
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES["sprand"](), 41)
    k = 37
    xs, b = W.rhs_for(seen, k, 1e-3, 5)
    b[3] = 0.0
    A = W.dense_from_csr(seen)
    b[6] = A @ xs[6]
    X, info = lsq.lsq_pcg_solve(Mx, P, torch.from_numpy(b).cuda(), o)
    X = X.cpu().numpy()
    kappa = np.linalg.cond(A / smp.d)
    assert np.all(X[3] == 0.0) and info.iters[3] == 0 and info.converged[3] == 1
    assert_solution(X[6], xs[6], kappa, "consistent column")
    for c in range(k):
        assert info.converged[c] == 1 and info.relres_true[c] <= o.tol, c
    for c in [0, 6, 31, 32, 36]:
        x1, i1 = lsq.lsq_pcg_solve(Mx, P, torch.from_numpy(b[c]).cuda(), o)
        assert_solution(X[c], x1.cpu().numpy().reshape(-1), kappa, f"block vs one column {c}")
        assert abs(int(info.iters[c]) - int(i1.iters[0])) <= 2, (c, info.iters[c], i1.iters[0])
    for c in [0, 36]:
        y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[c], tol=o.tol, maxit=o.maxit, max_outer=o.max_outer)
        assert_solution(X[c], y / smp.d, kappa, f"block column {c}")
        assert_iterations(info.iters[c], oi["iters"], _variants(orc, seen, smp, Mo, b[c], o), f"sprand block column {c}")


def test_sparse_block_maxit_and_two_sweeps(lsq, orc):
    """t = 2 sweeps per direction in the block path; a maxit cap freezes every column at
    exactly maxit iterations, reported as not converged."""
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES["graph"](), 77, sweeps=2)
    xs, b = W.rhs_for(seen, 3, 1e-4, 12)
    X, info = lsq.lsq_pcg_solve(Mx, P, torch.from_numpy(b).cuda(), o)
    X = X.cpu().numpy()
    A = W.dense_from_csr(seen)
    kappa = np.linalg.cond(A / smp.d)
    for c in range(3):
        y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[c], tol=o.tol, maxit=o.maxit, max_outer=o.max_outer, sweeps=2)
        assert info.converged[c] == 1 and oi["converged"] == 1
        assert_solution(X[c], y / smp.d, kappa, f"graph t=2 column {c}")
        assert_iterations(info.iters[c], oi["iters"], _variants(orc, seen, smp, Mo, b[c], o), f"graph t=2 column {c}")
    o.maxit = 3
    o.max_outer = 1
    X3, i3 = lsq.lsq_pcg_solve(Mx, P, torch.from_numpy(b).cuda(), o)
    assert list(i3.iters) == [3, 3, 3] and not any(i3.converged)
    for c in range(3):
        y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[c], tol=o.tol, maxit=3, max_outer=1, sweeps=2)
        assert oi["iters"] == 3
        assert rel(X3[c].cpu().numpy(), y / smp.d) <= 1e-10


@pytest.mark.parametrize("k", [1, 3])
def test_sparse_bf16_values_match_oracle(lsq, orc, k):
    """BF16 CSR values (k = 1: the one-column path; k = 3: the block path). Every value
    widens exactly to FP64, so the solve is the FP64 method on the BF16-rounded matrix,
    which is the matrix the oracle is given."""
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES["sprand"](), 3001, dtype="bf16")
    xs, b = W.rhs_for(seen, k, 1e-3, 29)
    X, info = lsq.lsq_pcg_solve(Mx, P, torch.from_numpy(b if k > 1 else b[0]).cuda(), o)
    X = X.cpu().numpy().reshape(k, -1)
    kappa = np.linalg.cond(W.dense_from_csr(seen) / smp.d)
    assert info.nnz_M == Mo.val.size
    for c in range(k):
        y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[c], tol=o.tol, maxit=o.maxit, max_outer=o.max_outer)
        assert info.converged[c] == 1 and oi["converged"] == 1 and info.relres_true[c] <= o.tol
        assert_solution(X[c], y / smp.d, kappa, f"bf16 k={k} column {c}")
        assert _same_solution(seen, smp.d, X[c], y, b[c], o.tol)
        assert_iterations(info.iters[c], oi["iters"], _variants(orc, seen, smp, Mo, b[c], o), f"bf16 k={k} column {c}")


def test_sparse_block_f32_refinement(lsq, orc):
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES["sprand"](), 8, dtype="f32", pdt=1, with_f64=True)
    o.max_outer = 30
    o.inner_tol = 1e-4
    xs, b = W.rhs_for(seen, 4, 1e-3, 19)
    X, info = lsq.lsq_pcg_solve(Mx, P, torch.from_numpy(b).cuda(), o)
    X = X.cpu().numpy()
    for c in range(4):
        assert info.converged[c] == 1 and info.relres_true[c] <= o.tol
        y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[c], tol=o.tol, maxit=o.maxit, max_outer=20)
        assert oi["converged"] == 1
        assert _same_solution(seen, smp.d, X[c], y, b[c], o.tol)


@pytest.mark.parametrize("case,k", [("mid", 4), ("sprand", 3), ("wide", 2)])
def test_sparse_block_long_rows_two_sweeps(lsq, orc, case, k):
    """Rows of M with ~60 dependency entries take the lane-per-entry block sweep, rows of
    hundreds take the CTA-per-row sweep; t = 2 also exercises their other-side terms (the
    previous sweep's values)."""
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES[case](), 313, sweeps=2)
    xs, b = W.rhs_for(seen, k, 1e-3, 31)
    X, info = lsq.lsq_pcg_solve(Mx, P, torch.from_numpy(b).cuda(), o)
    X = X.cpu().numpy()
    A = W.dense_from_csr(seen)
    kappa = np.linalg.cond(A / smp.d)
    for c in range(k):
        y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[c], tol=o.tol, maxit=o.maxit, max_outer=o.max_outer, sweeps=2)
        assert info.converged[c] == 1 and oi["converged"] == 1
        assert_solution(X[c], y / smp.d, kappa, f"{case} t=2 column {c}")
        assert_iterations(info.iters[c], oi["iters"], _variants(orc, seen, smp, Mo, b[c], o), f"{case} t=2 column {c}")


@pytest.mark.parametrize("k", [1, 3])
def test_sparse_cg_baseline_matches_oracle(lsq, orc, k):
    """sweeps = 0 (CG on the column-normalised A) through the one-column path (k = 1) and
    the block path (k = 3)."""
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES["sprand"](), 77, sweeps=0)
    xs, b = W.rhs_for(seen, k, 1e-3, 78)
    B = torch.from_numpy(b if k > 1 else b[0]).cuda()
    X, info = lsq.lsq_pcg_solve(Mx, P, B, o)
    X = X.cpu().numpy().reshape(k, -1)
    A = W.dense_from_csr(seen)
    kappa = np.linalg.cond(A / smp.d)
    for c in range(k):
        y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[c], tol=o.tol, maxit=o.maxit, max_outer=o.max_outer, sweeps=0)
        assert info.converged[c] == 1 and oi["converged"] == 1
        assert_solution(X[c], y / smp.d, kappa, f"CG sprand k={k} column {c}")
        assert_iterations(info.iters[c], oi["iters"], _variants(orc, seen, smp, Mo, b[c], o), f"CG sprand k={k} column {c}")
    r = torch.from_numpy(np.random.default_rng(0).standard_normal((2, seen["n"]))).cuda()
    assert torch.equal(P.apply(r), r)


def test_sparse_block_solve_captured_in_a_cuda_graph(lsq, orc):
    """A block of 32 right-hand sides (graph incidence, FP64) runs as one persistent launch
    plus its setup kernels, with no host synchronisation: lsq_pcg_solve is captured into a
    CUDA graph, and every replay writes the bits of the direct call."""
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES["graph"](), 1003)
    xs, b = W.rhs_for(seen, 32, 1e-4, 99)
    B = torch.from_numpy(b).cuda()
    X0, info = lsq.lsq_pcg_solve(Mx, P, B, o)
    assert all(info.converged == 1)
    X = torch.zeros_like(X0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    n0 = lsq.launches()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            lsq.lsq_pcg_solve(Mx, P, B, o, X=X, stream=s)
    assert 1 <= lsq.launches() - n0 <= 4       # the persistent kernel and its setup kernels
    for _ in range(2):
        X.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(X, X0)
    # one column against the oracle, for good measure
    y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[5], tol=o.tol, maxit=o.maxit, max_outer=o.max_outer)
    assert_solution(X[5].cpu().numpy(), y / smp.d, np.linalg.cond(W.dense_from_csr(seen) / smp.d), "captured")


@pytest.mark.parametrize("case,k,sweeps", [("sprand", 3, 1), ("graph", 4, 2), ("mid", 4, 2), ("sprand", 3, 0),
                                           ("wide", 2, 1), ("graph_wide", 32, 1)])
def test_sparse_block_persistent_matches_oracle(lsq, orc, case, k, sweeps):
    """The persistent form of the block solve (o.device_loop = 1: one cooperative launch for
    the whole solve, restarts included) against the oracle, for every sweep form (lane per
    column, lane per entry, CTA per row), t = 0, 1, 2, and blocks of 2 to 32 columns."""
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES[case](), 515, sweeps=sweeps)
    o.device_loop = 1
    xs, b = W.rhs_for(seen, k, 1e-3, 516)
    X, info = lsq.lsq_pcg_solve(Mx, P, torch.from_numpy(b).cuda(), o)
    X = X.cpu().numpy()
    small = seen["n"] <= 5000
    if small:
        kappa = np.linalg.cond(W.dense_from_csr(seen) / smp.d)
    for c in range(min(k, 4)):
        y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[c], tol=o.tol, maxit=o.maxit, max_outer=o.max_outer, sweeps=sweeps)
        assert info.converged[c] == 1 and oi["converged"] == 1 and info.relres_true[c] <= o.tol
        if small:
            assert_solution(X[c], y / smp.d, kappa, f"persistent {case} column {c}")
        assert _same_solution(seen, smp.d, X[c], y, b[c], o.tol)
        assert_iterations(info.iters[c], oi["iters"], _variants(orc, seen, smp, Mo, b[c], o),
                          f"persistent {case} t={sweeps} column {c}")
    assert all(info.converged[:k] == 1)


def _components(mat):
    """Connected-component label of every column of an incidence matrix (its null space of
    B^T B is spanned by the indicator vectors of these components)."""
    import scipy.sparse as sps
    from scipy.sparse.csgraph import connected_components
    B = sps.csr_matrix((mat["vals"], mat["col_idx"], mat["row_ptr"]), shape=(mat["m"], mat["n"]))
    return connected_components(abs(B.T @ B), directed=False)[1]


@pytest.mark.parametrize("n_param,sweeps,tol,k", [(96, 5, 1e-7, 1), (180, 5, 1e-7, 3), (96, 1, 1e-10, 3),
                                                  (180, 1, 1e-10, 1)])
def test_graph_laplacian_singular_matches_oracle(lsq, orc, n_param, sweeps, tol, k):
    """The random graph Laplacian family of Sec. 5.5 at the paper's sizes (n = 187 and 355
    vertices), with the paper's settings (t = 5, tolerance 1e-7) and the tight ones (t = 1,
    1e-10).  B^T B is singular (one constant vector per connected component), so the normal
    equations are consistent but x is unique only up to the null space: the fitted values,
    the range part of x, the iteration counts and the convergence flags are compared."""
    mat = W.chung_lu_incidence(n_param, 5)
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, mat, 31, sweeps=sweeps)
    o.tol = tol
    b = np.random.default_rng(n_param).standard_normal((k, seen["m"]))
    X, info = lsq.lsq_pcg_solve(Mx, P, torch.from_numpy(b if k > 1 else b[0]).cuda(), o)
    X = X.cpu().numpy().reshape(k, -1)
    B = W.dense_from_csr(seen)
    lab = _components(seen)
    ev = np.linalg.eigvalsh((B / smp.d).T @ (B / smp.d))
    kappa_eff = np.sqrt(ev[-1] / ev[ev > 1e-9 * ev[-1]][0])
    for c in range(k):
        y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[c], tol=tol, maxit=o.maxit, max_outer=o.max_outer, sweeps=sweeps)
        x_or = y / smp.d
        assert info.converged[c] == 1 and oi["converged"] == 1
        assert info.relres_true[c] <= tol
        assert _same_solution(seen, smp.d, X[c], y, b[c], tol)
        assert_iterations(info.iters[c], oi["iters"], _variants(orc, seen, smp, Mo, b[c], o),
                          f"graph Laplacian n={seen['n']} t={sweeps} column {c}")
        if tol <= 1e-10:
            # the range part: x minus its mean over each component (D-weighted projections
            # would do as well; the difference of two solutions is what is compared)
            def rng_part(v):
                return v - (np.bincount(lab, v) / np.bincount(lab))[lab]
            assert_solution(B @ X[c], B @ x_or, kappa_eff, f"fitted values column {c}")
            assert_solution(rng_part(X[c]), rng_part(x_or), kappa_eff, f"range part column {c}")


@pytest.fixture
def sweep_form(lsq):
    """Sets the process-wide form of the one-column sweeps for one test, then restores it."""
    def set_form(f):
        lsq.set_sweep_form(f)
    yield set_form
    lsq.set_sweep_form(0)


@pytest.mark.parametrize("sweeps", [1, 2])
@pytest.mark.parametrize("case", ["sprand", "graph", "wide", "mid", "graph_wide"])
def test_sweep_forms_are_bit_identical(lsq, orc, sweep_form, case, sweeps):
    """The grid, one-CTA and one-cluster forms of a sweep visit the same rows in the same level
    order with the same per-row arithmetic (a lane's entries in order, then the warp sum), so
    they give the same bits; each against the literal Alg. 3 at 1e-11."""
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES[case](), 1003, sweeps=sweeps)
    R = np.random.default_rng(5 + sweeps).standard_normal((3, seen["n"]))
    Rt = torch.from_numpy(R).cuda()
    outs = {}
    for form in (1, 2, 3):
        sweep_form(form)
        outs[form] = P.apply(Rt).cpu().numpy()
    for c in range(3):
        ref = orc.sgs_apply(Mo, R[c], sweeps)
        for form in (1, 2, 3):
            assert rel(outs[form][c], ref) <= 1e-11, (form, c)
    assert np.array_equal(outs[1], outs[2]), "grid and one-CTA sweeps differ"
    assert np.array_equal(outs[1], outs[3]), "grid and cluster sweeps differ"


@pytest.mark.parametrize("case", ["sprand", "mid", "graph"])
def test_cluster_sweep_solve_matches_oracle(lsq, orc, sweep_form, case):
    """A whole one-column solve with the cluster-form sweeps (the first carrying the
    convergence check) against the oracle, and bit for bit against the grid form."""
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES[case](), 2029)
    xs, b = W.rhs_for(seen, 1, 1e-3, 23)
    B = torch.from_numpy(b[0]).cuda()
    sweep_form(3)
    X3, i3 = lsq.lsq_pcg_solve(Mx, P, B, o)
    sweep_form(1)
    X1, i1 = lsq.lsq_pcg_solve(Mx, P, B, o)
    assert np.array_equal(X3.cpu().numpy(), X1.cpu().numpy()) and int(i3.iters[0]) == int(i1.iters[0])
    y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[0], tol=o.tol, maxit=o.maxit, max_outer=o.max_outer)
    assert i3.converged[0] == 1 and oi["converged"] == 1 and i3.relres_true[0] <= o.tol
    x = X3.cpu().numpy().reshape(-1)
    kappa = np.linalg.cond(W.dense_from_csr(seen) / smp.d)
    assert_solution(x, y / smp.d, kappa, f"{case} cluster sweeps")
    assert_iterations(i3.iters[0], oi["iters"], _variants(orc, seen, smp, Mo, b[0], o), f"{case} cluster sweeps")


@pytest.mark.parametrize("case,k,sweeps", [("sprand", 3, 1), ("sprand", 5, 2), ("graph", 4, 1), ("mid", 4, 2),
                                           ("wide", 2, 1), ("wide", 17, 1)])
def test_block_cluster_sweep_matches_oracle(lsq, orc, sweep_form, case, k, sweeps):
    """The block solve with its sweeps in one thread-block cluster (form 3) against the oracle;
    where the shape picks the CTA-per-row form anyway (more than 96 dependency entries per row),
    bit for bit against it, since both sum a row's entries in the same order."""
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES[case](), 717, sweeps=sweeps)
    xs, b = W.rhs_for(seen, k, 1e-3, 718)
    B = torch.from_numpy(b).cuda()
    sweep_form(3)
    X3, i3 = lsq.lsq_pcg_solve(Mx, P, B, o)
    sweep_form(1)
    X1, i1 = lsq.lsq_pcg_solve(Mx, P, B, o)
    X3 = X3.cpu().numpy()
    dep = (int(i3.nnz_M) - seen["n"]) / (2.0 * seen["n"])
    if dep > 96.0:
        assert np.array_equal(X3, X1.cpu().numpy()) and list(i3.iters) == list(i1.iters)
    kappa = np.linalg.cond(W.dense_from_csr(seen) / smp.d)
    for c in sorted({0, k // 2, k - 1}):
        y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[c], tol=o.tol, maxit=o.maxit, max_outer=o.max_outer, sweeps=sweeps)
        assert i3.converged[c] == 1 and oi["converged"] == 1 and i3.relres_true[c] <= o.tol
        assert_solution(X3[c], y / smp.d, kappa, f"cluster block {case} column {c}")
        assert_iterations(i3.iters[c], oi["iters"], _variants(orc, seen, smp, Mo, b[c], o),
                          f"cluster block {case} t={sweeps} column {c}")


def _sgs_reference(M, r, sweeps):
    """Alg. 3 in FP64 with scipy's triangular solves on the given sparse M: t forward sweeps
    e <- e + (D + L)^{-1} (r - M e), then t backward sweeps with (D + U), from e = 0."""
    import scipy.sparse as sps
    from scipy.sparse.linalg import spsolve_triangular
    lower = sps.tril(M, format="csr")
    upper = sps.triu(M, format="csr")
    e = np.zeros_like(r)
    for _ in range(sweeps):
        e = e + spsolve_triangular(lower, r - M @ e, lower=True)
    for _ in range(sweeps):
        e = e + spsolve_triangular(upper, r - M @ e, lower=False)
    return e


@pytest.mark.parametrize("sweeps", [1, 2])
@pytest.mark.parametrize("case", ["sprand", "graph", "wide", "mid", "graph_wide"])
def test_fp32_m_sweeps_in_float_pairs(lsq, orc, sweep_form, case, sweeps):
    """FP32 M (the precision form): the sweeps sum in double-float on the FP32 units.  Every
    form gives the same bits, and the result matches Alg. 3 in FP64 on the same matrix (the
    FP32-rounded off-diagonal entries, the FP64 diagonal; scipy triangular solves) to 1e-10:
    the double-float sums keep ~48 bits."""
    import scipy.sparse as sps
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES[case](), 1003, sweeps=sweeps, pdt=1)
    rp, ci, va = (t.cpu().numpy() for t in P.M_csr())
    n = seen["n"]
    # the sweeps use the FP32-rounded off-diagonal entries and the FP64 reciprocal diagonal
    rows = np.repeat(np.arange(n), np.diff(rp))
    v = np.where(rows == ci, va, va.astype(np.float32).astype(np.float64))
    M32 = sps.csr_matrix((v, ci, rp), shape=(n, n))
    R = np.random.default_rng(9 + sweeps).standard_normal((2, n))
    Rt = torch.from_numpy(R).cuda()
    outs = {}
    for form in (1, 2, 3):
        sweep_form(form)
        outs[form] = P.apply(Rt).cpu().numpy()
    assert np.array_equal(outs[1], outs[2]), "grid and one-CTA sweeps differ"
    assert np.array_equal(outs[1], outs[3]), "grid and cluster sweeps differ"
    for c in range(2):
        ref = _sgs_reference(M32, R[c], sweeps)
        assert rel(outs[1][c], ref) <= 1e-10, (case, c, rel(outs[1][c], ref))


@pytest.mark.parametrize("case,k,sweeps", [("sprand", 4, 1), ("sprand", 3, 2), ("wide", 16, 1), ("wide", 5, 2)])
def test_block_fp32_m_cta_sweeps_in_float_pairs(lsq, orc, case, k, sweeps):
    """FP32 M with the CTA-per-row block sweep (rows of more than 96 dependency entries): the
    sweeps sum in double-float on float-pair vectors.  Whole solves against the oracle (on the
    FP64 M: the FP32 operator only changes the preconditioner, and both solves meet the
    tolerance), and against the same block through the persistent kernel, whose sweeps keep
    FP64 sums."""
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, CASES[case](), 4242, sweeps=sweeps, pdt=1)
    xs, b = W.rhs_for(seen, k, 1e-3, 4243)
    B = torch.from_numpy(b).cuda()
    X, info = lsq.lsq_pcg_solve(Mx, P, B, o)
    X = X.cpu().numpy()
    assert (int(info.nnz_M) - seen["n"]) / (2.0 * seen["n"]) > 96.0   # the CTA-per-row form
    kappa = np.linalg.cond(W.dense_from_csr(seen) / smp.d)
    for c in sorted({0, k - 1}):
        y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[c], tol=o.tol, maxit=o.maxit, max_outer=o.max_outer, sweeps=sweeps)
        assert info.converged[c] == 1 and oi["converged"] == 1 and info.relres_true[c] <= o.tol
        assert_solution(X[c], y / smp.d, kappa, f"FP32 M block {case} column {c}")
    # the same block through the persistent kernel (the same FP32 M, FP64 sums): the same
    # solution within the bar and the same iteration counts within 2
    o.device_loop = 1
    Xp, ip = lsq.lsq_pcg_solve(Mx, P, B, o)
    for c in range(k):
        assert ip.converged[c] == 1
        assert_solution(X[c], Xp[c].cpu().numpy(), kappa, f"pairs vs persistent column {c}")
        assert abs(int(info.iters[c]) - int(ip.iters[c])) <= 2, (c, info.iters[c], ip.iters[c])
