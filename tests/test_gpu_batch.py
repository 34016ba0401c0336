"""Batches of uneven small dense problems in one launch (lsq_batch_*), against the oracle
on the same FP32 values and the same sampled preconditioner of each problem."""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import assert_solution, rel

pytestmark = pytest.mark.gpu


def _problem(lsq, mat, seed, k, noise, pad_nan=True, pdt=1):
    """FP32 A stored with a leading dimension padded to a multiple of 4 (NaN in the
    padding, which the batch must never use), its preconditioner and k right-hand sides."""
    A64 = np.asarray(mat["A"])
    m, n = A64.shape
    ld = (n + 3) // 4 * 4 + 4
    T = torch.full((m, ld), float("nan") if pad_nan else 0.0, dtype=torch.float32, device="cuda")
    T[:, :n] = torch.from_numpy(A64).float().cuda()
    Mx = lsq.Matrix(T[:, :n])
    o = lsq.opts(seed=seed, precond_dtype=pdt)
    idx, p, d = lsq.lsq_sample_rows(Mx, o)
    P = lsq.lsq_build_precond(Mx, idx, p, d, o)
    seen = {"kind": "dense", "A": T[:, :n].double().cpu().numpy()}
    xs, b = W.rhs_for(seen, k, noise, seed + 1)
    return dict(T=T, n=n, P=P, B=torch.from_numpy(b).cuda(), b=b, seen=seen, seed=seed, Mx=Mx)


def _opts(lsq):
    return lsq.opts(tol=1e-10, max_outer=30, inner_tol=1e-4, maxit=20000)


def _check_against_oracle(orc, pr, X, info, tol, cols):
    A = pr["seen"]["A"]
    smp = orc.Sample(pr["seen"], seed=pr["seed"])
    Mo = orc.SampledM(smp)
    kappa = np.linalg.cond(A / smp.d)
    for c in cols:
        y, oi = orc.pcg(smp.mat, smp.d, Mo, b=pr["b"][c], tol=tol, maxit=100000, max_outer=20)
        assert oi["converged"] == 1
        assert info.converged[c] == 1 and info.relres_true[c] <= tol, (c, info.relres_true[c])
        assert_solution(X[c], y / smp.d, kappa, f"batch column {c}")
        r = A.T @ (pr["b"][c] - A @ X[c])
        raw = np.linalg.norm(r) / np.linalg.norm(A.T @ pr["b"][c])
        # the batch computes its residuals in double-float (~48 bits): near roundoff the
        # reported ratio carries an absolute error of a few 1e-15
        assert abs(raw - info.relres_raw[c]) <= 1e-3 * raw + 1e-13


@pytest.mark.parametrize("pdt", [1, 0])
def test_batch_uneven_matches_oracle(lsq, orc, pdt):
    """pdt: the SGS operator stored in FP32 (1) or FP64 (0)."""
    mats = W.uneven_dense_batch(10, (300, 6000), (5, 200), 51)
    k = 3
    prs = [_problem(lsq, mt, 700 + i, k, 1e-3, pdt=pdt) for i, mt in enumerate(mats)]
    o = _opts(lsq)
    bt = lsq.Batch([(pr["T"], pr["n"], pr["P"], pr["B"]) for pr in prs], o)
    bt.solve()
    infos = bt.info()
    for pr, X, info in zip(prs, bt.X, infos):
        _check_against_oracle(orc, pr, X.cpu().numpy(), info, o.tol, range(k))


@pytest.mark.parametrize("cluster", [1, 2, 4, 8, 16])
def test_batch_every_cluster_size(lsq, orc, cluster):
    mats = W.uneven_dense_batch(6, (200, 3000), (16, 130), 52)
    k = 5    # rounded up to 8 columns inside; columns 5..7 are padding
    prs = [_problem(lsq, mt, 800 + i, k, 1e-2) for i, mt in enumerate(mats)]
    o = _opts(lsq)
    bt = lsq.Batch([(pr["T"], pr["n"], pr["P"], pr["B"]) for pr in prs], o)
    try:
        bt.set_cluster(cluster)
    except lsq.L.LsqError as e:
        if e.code == 7:
            pytest.skip("cluster size not available on this device")
        raise
    bt.solve()
    infos = bt.info()
    for pr, X, info in zip(prs, bt.X, infos):
        _check_against_oracle(orc, pr, X.cpu().numpy(), info, o.tol, [0, k - 1])


def test_batch_degenerate_problems(lsq, orc):
    """m smaller than the cluster (CTAs without rows), n = 1, a zero right-hand side, a
    consistent right-hand side, and a single right-hand side per problem."""
    rng = np.random.default_rng(3)
    mats = [{"kind": "dense", "A": rng.standard_normal((6, 3))},
            {"kind": "dense", "A": rng.standard_normal((50, 1))},
            {"kind": "dense", "A": rng.standard_normal((900, 37))}]
    prs = [_problem(lsq, mt, 900 + i, 2, 1e-3) for i, mt in enumerate(mats)]
    prs[2]["B"][0].zero_()
    prs[2]["b"][0] = 0.0
    A1 = prs[1]["seen"]["A"]
    xs1 = np.array([0.7])
    prs[1]["b"][1] = A1 @ xs1
    prs[1]["B"][1] = torch.from_numpy(prs[1]["b"][1]).cuda()
    o = _opts(lsq)
    bt = lsq.Batch([(pr["T"], pr["n"], pr["P"], pr["B"]) for pr in prs], o)
    bt.set_cluster(8)
    bt.solve()
    infos = bt.info()
    X = [x.cpu().numpy() for x in bt.X]
    assert np.all(X[2][0] == 0.0) and infos[2].iters[0] == 0 and infos[2].converged[0] == 1
    assert rel(X[1][1], xs1) <= 1e-9
    _check_against_oracle(orc, prs[0], X[0], infos[0], o.tol, [0, 1])
    _check_against_oracle(orc, prs[2], X[2], infos[2], o.tol, [1])
    single = _problem(lsq, mats[2], 990, 1, 1e-3)
    b1 = lsq.Batch([(single["T"], single["n"], single["P"], single["B"])], o)
    b1.solve()
    _check_against_oracle(orc, single, b1.X[0].cpu().numpy(), b1.info()[0], o.tol, [0])


def test_batch_maxit_reports_not_converged(lsq):
    mats = W.uneven_dense_batch(3, (500, 900), (20, 40), 53)
    prs = [_problem(lsq, mt, 950 + i, 2, 1e-3) for i, mt in enumerate(mats)]
    o = lsq.opts(tol=1e-14, maxit=4, max_outer=1)
    bt = lsq.Batch([(pr["T"], pr["n"], pr["P"], pr["B"]) for pr in prs], o)
    bt.solve()
    infos = bt.info()
    for info in infos:
        assert list(info.iters) == [4, 4] and not any(info.converged)
        assert info.status == 4


def test_batch_graph_capture_and_autotune(lsq, orc):
    """The solve is one capturable launch: a replayed CUDA graph gives the same bits as a
    direct solve; the autotuner picks a cluster size that still gives correct results."""
    mats = W.uneven_dense_batch(8, (500, 4000), (20, 160), 54)
    k = 4
    prs = [_problem(lsq, mt, 1000 + i, k, 1e-3) for i, mt in enumerate(mats)]
    o = _opts(lsq)
    bt = lsq.Batch([(pr["T"], pr["n"], pr["P"], pr["B"]) for pr in prs], o)
    C = bt.autotune()
    assert C in (1, 2, 4, 8, 16)
    bt.solve()
    torch.cuda.synchronize()
    ref = [x.clone() for x in bt.X]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            bt.solve(stream=s)
    torch.cuda.synchronize()
    for x in bt.X:
        x.zero_()
    g.replay()
    torch.cuda.synchronize()
    for x, r in zip(bt.X, ref):
        assert torch.equal(x, r)
    infos = bt.info()
    for pr, X, info in zip(prs, bt.X, infos):
        _check_against_oracle(orc, pr, X.cpu().numpy(), info, o.tol, [0, k - 1])
