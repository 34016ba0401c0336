"""Differentiation through the solver: the autograd Function's gradients w.r.t. b and A's
values against the dense closed form (torch autograd through lstsq, CPU FP64) and central
finite differences."""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import rel

pytestmark = pytest.mark.gpu


def _loss_ref(A, b, xs):
    """Plain PyTorch CPU FP64 reference: x = lstsq(A, b), loss = sum ||x - x*||^2."""
    X = torch.linalg.lstsq(A, b.T, driver="gelsd").solution.T
    return ((X - xs) ** 2).sum()


def test_autograd_dense_matches_lstsq_gradient(lsq):
    mat = W.gaussian_dense(600, 24, 11)
    xs, b = W.rhs_for(mat, 3, 1e-2, 5)
    At = torch.from_numpy(mat["A"]).cuda().requires_grad_(True)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    Mx = lsq.Matrix(At.detach())
    Mx.vals = At   # the autograd input is the same storage
    o = lsq.opts(seed=5, tol=1e-13)
    idx, p, d = lsq.lsq_sample_rows(Mx, o)
    P = lsq.lsq_build_precond(Mx, idx, p, d, o)
    X = lsq.lsq_solve(Mx, bt, P, o)
    loss = ((X - torch.from_numpy(xs).cuda()) ** 2).sum()
    loss.backward()
    Ar = torch.from_numpy(mat["A"]).requires_grad_(True)
    br = torch.from_numpy(b).requires_grad_(True)
    lr = _loss_ref(Ar, br, torch.from_numpy(xs))
    lr.backward()
    assert abs(loss.item() - lr.item()) <= 1e-9 * abs(lr.item())
    assert rel(bt.grad.cpu().numpy(), br.grad.numpy()) <= 1e-8
    assert rel(At.grad.cpu().numpy(), Ar.grad.numpy()) <= 1e-8


def test_autograd_csr_finite_differences(lsq):
    mat = W.sparse_random(3000, 40, 6, 13)
    rp = torch.from_numpy(mat["row_ptr"]).cuda()
    ci = torch.from_numpy(mat["col_idx"]).cuda()
    v = torch.from_numpy(mat["vals"]).cuda().requires_grad_(True)
    Mx = lsq.Matrix(row_ptr=rp, col_idx=ci, vals=v.detach(), n=mat["n"])
    Mx.vals = v
    xs, b = W.rhs_for(mat, 2, 1e-2, 3)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    o = lsq.opts(seed=9, tol=1e-14, max_outer=8)
    idx, p, d = lsq.lsq_sample_rows(Mx, o)
    P = lsq.lsq_build_precond(Mx, idx, p, d, o)
    xst = torch.from_numpy(xs).cuda()

    def loss_of(vals, bb):
        M2 = lsq.Matrix(row_ptr=rp, col_idx=ci, vals=vals, n=mat["n"])
        X, _ = lsq.lsq_pcg_solve(M2, P, bb, o)
        return ((X - xst) ** 2).sum().item()

    X = lsq.lsq_solve(Mx, bt, P, o)
    ((X - xst) ** 2).sum().backward()
    gv, gb = v.grad.cpu().numpy(), bt.grad.cpu().numpy()
    rng = np.random.default_rng(0)
    h = 1e-4
    base_v = v.detach().clone()
    for e in rng.choice(mat["vals"].size, 6, replace=False):
        vp, vm = base_v.clone(), base_v.clone()
        vp[e] += h
        vm[e] -= h
        fd = (loss_of(vp, bt.detach()) - loss_of(vm, bt.detach())) / (2 * h)
        assert abs(fd - gv[e]) <= 1e-5 * max(1.0, abs(gv[e])), (e, fd, gv[e])
    for (c, i) in [(0, 5), (1, 2999), (1, 1234)]:
        bp, bm = bt.detach().clone(), bt.detach().clone()
        bp[c, i] += h
        bm[c, i] -= h
        fd = (loss_of(base_v, bp) - loss_of(base_v, bm)) / (2 * h)
        assert abs(fd - gb[c, i]) <= 1e-5 * max(1.0, abs(gb[c, i])), (c, i, fd, gb[c, i])


def test_autograd_csr_f32_values_closed_form(lsq):
    """FP32 values (FP64 scalars and residuals): gradients against the dense closed form on
    the same FP32-rounded values, lambda = (A^T A)^{-1} g, grad_b = A lambda,
    grad_A = r lambda^T - (A lambda) x^T on the pattern."""
    mat = W.sparse_random(4000, 50, 6, 21)
    rp = torch.from_numpy(mat["row_ptr"]).cuda()
    ci = torch.from_numpy(mat["col_idx"]).cuda()
    v32 = torch.from_numpy(mat["vals"]).cuda().float().requires_grad_(True)
    v64 = v32.detach().double()
    Mx = lsq.Matrix(row_ptr=rp, col_idx=ci, vals=v32.detach(), n=mat["n"], vals_f64=v64)
    Mx.vals = v32
    seen = dict(mat)
    seen["vals"] = v64.cpu().numpy()
    A = W.dense_from_csr(seen)
    xs, b = W.rhs_for(seen, 1, 1e-2, 4)
    bt = torch.from_numpy(b[0]).cuda().requires_grad_(True)
    o = lsq.opts(seed=2, tol=1e-12, max_outer=30, inner_tol=1e-4, precond_dtype=1)
    idx, p, d = lsq.lsq_sample_rows(Mx, o)
    P = lsq.lsq_build_precond(Mx, idx, p, d, o)
    x = lsq.lsq_solve(Mx, bt, P, o)
    ((x - torch.from_numpy(xs[0]).cuda()) ** 2).sum().backward()
    assert v32.grad.dtype == torch.float32
    xr = np.linalg.lstsq(A, b[0], rcond=None)[0]
    g = 2 * (xr - xs[0])
    lam = np.linalg.solve(A.T @ A, g)
    r = b[0] - A @ xr
    Al = A @ lam
    rows = np.repeat(np.arange(A.shape[0]), np.diff(mat["row_ptr"]))
    gA = r[rows] * lam[mat["col_idx"]] - Al[rows] * xr[mat["col_idx"]]
    assert rel(bt.grad.cpu().numpy(), Al) <= 1e-7
    assert rel(v32.grad.double().cpu().numpy(), gA) <= 1e-6
