"""Failure paths, made on purpose and safely (no fault, no trap, no endless wait).

* Timeouts: lsq_set_wait_limit caps every device-side wait at a handful of polls, so a
  wait runs out while its dependency is still being computed.  The kernel must record the
  timeout, let every other wait give up, return, and the call must report LSQ_ERR_TIMEOUT.
  The next call on the same handle, with the default bound, must give the normal result.
* Breakdown: a right-hand side with a NaN makes rho and p^T w non-finite; PCG must stop and
  report LSQ_ERR_BREAKDOWN, and the handle must still solve a normal right-hand side.
"""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import assert_solution, rel, to_device

pytestmark = pytest.mark.gpu

TIMEOUT, BREAKDOWN = 6, 5


def _setup(lsq, orc, mat, seed):
    Mx, keep, seen = to_device(lsq, mat)
    o = lsq.opts(seed=seed)
    idx, p, d = lsq.lsq_sample_rows(Mx, o)
    P = lsq.lsq_build_precond(Mx, idx, p, d, o)
    smp = orc.Sample(seen, seed=seed)
    return Mx, keep, seen, o, P, smp, orc.SampledM(smp)


def test_sparse_sweep_wait_timeout_then_recovers(lsq, orc):
    """The sweeps of a graph incidence matrix with wide levels run on the whole grid, each
    row waiting for the values it depends on: with 2 polls per wait those waits run out."""
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, W.graph_incidence(20000, 90000, 4), 1003)
    r = torch.from_numpy(np.random.default_rng(1).standard_normal((2, seen["n"]))).cuda()
    xs, b = W.rhs_for(seen, 1, 1e-4, 17)
    B = torch.from_numpy(b[0]).cuda()
    lsq.set_wait_limit(2)
    try:
        with pytest.raises(lsq.L.LsqError) as e:
            P.apply(r)
        assert e.value.code == TIMEOUT
        with pytest.raises(lsq.L.LsqError) as e:
            lsq.lsq_pcg_solve(Mx, P, B, o)
        assert e.value.code == TIMEOUT
    finally:
        lsq.set_wait_limit(0)
    E = P.apply(r).cpu().numpy()
    for c in range(2):
        assert rel(E[c], orc.sgs_apply(Mo, r[c].cpu().numpy(), 1)) <= 1e-11
    X, info = lsq.lsq_pcg_solve(Mx, P, B, o)
    y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[0], tol=o.tol, maxit=o.maxit, max_outer=o.max_outer)
    assert info.status == 0 and info.converged[0] == 1
    assert abs(int(info.iters[0]) - oi["iters"]) <= 2


@pytest.mark.parametrize("device_loop", [0, 1])
def test_sparse_block_sweep_wait_timeout(lsq, orc, device_loop):
    """The same for a block of right-hand sides (the block sweep forms; stream-ordered and the
    persistent launch, whose grid barriers are capped too)."""
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, W.graph_incidence(20000, 90000, 4), 1003)
    o.device_loop = device_loop
    xs, b = W.rhs_for(seen, 4, 1e-4, 17)
    B = torch.from_numpy(b).cuda()
    lsq.set_wait_limit(2)
    try:
        with pytest.raises(lsq.L.LsqError) as e:
            lsq.lsq_pcg_solve(Mx, P, B, o)
        assert e.value.code == TIMEOUT
    finally:
        lsq.set_wait_limit(0)
    X, info = lsq.lsq_pcg_solve(Mx, P, B, o)
    assert info.status == 0 and all(info.converged == 1)


def test_level_builder_wait_timeout(lsq, orc):
    """Building the sparse handle computes the level schedules with dependency waits too."""
    Mx, keep, seen = to_device(lsq, W.graph_incidence(20000, 90000, 4))
    o = lsq.opts(seed=1003)
    idx, p, d = lsq.lsq_sample_rows(Mx, o)
    lsq.set_wait_limit(2)
    try:
        with pytest.raises(lsq.L.LsqError) as e:
            lsq.lsq_build_precond(Mx, idx, p, d, o)
        assert e.value.code == TIMEOUT
    finally:
        lsq.set_wait_limit(0)
    P = lsq.lsq_build_precond(Mx, idx, p, d, o)
    smp = orc.Sample(seen, seed=1003)
    Mo = orc.SampledM(smp)
    rp, ci, va = (t.cpu().numpy() for t in P.M_csr())
    assert np.array_equal(rp, Mo.row_ptr) and np.array_equal(ci, Mo.col)


def test_dense_grid_barrier_timeout_then_recovers(lsq, orc):
    """The persistent dense PCG kernel meets at grid barriers; with 2 polls per barrier the
    early CTAs give up, drain their copies in flight and leave."""
    mat = W.gaussian_dense(20000, 256, 11)
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, mat, 11)
    xs, b = W.rhs_for(seen, 1, 1e-2, 18)
    B = torch.from_numpy(b[0]).cuda()
    lsq.set_wait_limit(2)
    try:
        with pytest.raises(lsq.L.LsqError) as e:
            lsq.lsq_pcg_solve(Mx, P, B, o)
        assert e.value.code == TIMEOUT
    finally:
        lsq.set_wait_limit(0)
    X, info = lsq.lsq_pcg_solve(Mx, P, B, o)
    y, oi = orc.pcg(smp.mat, smp.d, Mo, b=b[0], tol=o.tol, maxit=o.maxit, max_outer=o.max_outer)
    assert info.status == 0 and info.converged[0] == 1 and info.iters[0] == oi["iters"]
    assert_solution(X.cpu().numpy(), y / smp.d, np.linalg.cond(mat["A"] / smp.d), "after timeout")


@pytest.mark.parametrize("kind", ["dense", "csr1", "csr3", "csr3_persistent"])
def test_breakdown_on_nan_rhs_then_recovers(lsq, orc, kind):
    mat = W.gaussian_dense(4096, 128, 1001) if kind == "dense" else W.sparse_random(20000, 300, 8, 3)
    Mx, keep, seen, o, P, smp, Mo = _setup(lsq, orc, mat, 1001)
    o.device_loop = 1 if kind == "csr3_persistent" else 0
    k = 3 if kind.startswith("csr3") else 1
    xs, b = W.rhs_for(seen, k, 1e-3, 5)
    bad = b.copy()
    bad[0, 17] = np.nan
    with pytest.raises(lsq.L.LsqError) as e:
        lsq.lsq_pcg_solve(Mx, P, torch.from_numpy(bad if k > 1 else bad[0]).cuda(), o)
    assert e.value.code == BREAKDOWN
    X, info = lsq.lsq_pcg_solve(Mx, P, torch.from_numpy(b if k > 1 else b[0]).cuda(), o)
    assert info.status == 0 and all(info.converged[:k] == 1)
