"""Shared test helpers: move seeded workloads to the device and compare with the oracle."""
import numpy as np


def to_device(lsq, mat, dtype="f64", with_f64=False, ld_pad=0):
    """workloads dict -> (api.Matrix, keepalive list, the FP64 values the oracle must see)."""
    import torch
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    keep = []
    if mat["kind"] == "dense":
        A = np.asarray(mat["A"], dtype=np.float64)
        m, n = A.shape
        ld = n + ld_pad
        T = torch.zeros(m, ld, dtype=tdt, device="cuda")
        T[:, :n] = torch.from_numpy(A).to("cuda").to(tdt)
        view = T[:, :n] if ld_pad else T
        f64 = None
        if with_f64:
            f64 = torch.zeros(m, ld, dtype=torch.float64, device="cuda")
            f64[:, :n] = T[:, :n].double()
            keep.append(f64)
        keep.append(T)
        Mx = lsq.Matrix(view if not ld_pad else T[:, :n], vals_f64=f64)
        seen = T[:, :n].double().cpu().numpy()
        return Mx, keep, {"kind": "dense", "A": seen}
    rp = torch.from_numpy(np.asarray(mat["row_ptr"], np.int64)).cuda()
    ci = torch.from_numpy(np.asarray(mat["col_idx"], np.int32)).cuda()
    v = torch.from_numpy(np.asarray(mat["vals"], np.float64)).cuda().to(tdt)
    f64 = v.double() if with_f64 else None
    keep += [rp, ci, v] + ([f64] if f64 is not None else [])
    Mx = lsq.Matrix(row_ptr=rp, col_idx=ci, vals=v, n=mat["n"], vals_f64=f64)
    seen = dict(mat)
    seen["vals"] = v.double().cpu().numpy()
    return Mx, keep, seen


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def solution_bar(kappa):
    """The solution bar of the parity tests: ||x - x_oracle|| / ||x_oracle|| <= 1e-8 kappa(Â)."""
    return 1e-8 * float(kappa)


def assert_solution(x, x_or, kappa, what=""):
    """x against the oracle's x: relative 2-norm within 1e-8 kappa, and every component
    within that bar scaled by its own size plus the largest component (so a few wrong small
    entries cannot hide inside a good norm)."""
    x, x_or = np.asarray(x, np.float64).reshape(-1), np.asarray(x_or, np.float64).reshape(-1)
    bar = solution_bar(kappa)
    r = rel(x, x_or)
    assert r <= bar, f"{what}: ||x - x_oracle||/||x_oracle|| = {r:.3e} > 1e-8 kappa = {bar:.3e}"
    np.testing.assert_allclose(x, x_or, rtol=bar, atol=bar * float(np.abs(x_or).max()), err_msg=what)


def _permuted_rows(mat, perm):
    """The same matrix with its rows in the order perm (dense or CSR)."""
    if mat["kind"] == "dense":
        return {"kind": "dense", "A": np.ascontiguousarray(np.asarray(mat["A"])[perm])}
    rp, ci, v = (np.asarray(mat[k]) for k in ("row_ptr", "col_idx", "vals"))
    lens = np.diff(rp)[perm]
    nrp = np.zeros(int(mat["m"]) + 1, np.int64)
    np.cumsum(lens, out=nrp[1:])
    take = np.repeat(rp[:-1][perm], lens) + (np.arange(nrp[-1]) - np.repeat(nrp[:-1], lens))
    return {"kind": "csr", "m": int(mat["m"]), "n": int(mat["n"]), "row_ptr": nrp,
            "col_idx": ci[take].astype(np.int32), "vals": v[take].astype(np.float64)}


def _numpy_pcg_iters(orc, mat, d, Mo, b, tol, sweeps, maxit, max_outer, blocks=0):
    """The same PCG (restarts from the true residual included) with every product in
    numpy's BLAS summation order and p^T w taken as ||Â p||^2, which equals it in exact
    arithmetic.  With blocks > 0 the sums over the rows of Â^T q are taken as partial sums
    over `blocks` contiguous row blocks, combined pairwise (the shape of the GPU's
    reduction: a partial per thread block, then a tree).  Returns the number of products
    Â^T Â p."""
    import scipy.sparse as sps
    if mat["kind"] == "dense":
        Ah = np.asarray(mat["A"], np.float64) / d
    else:
        A = sps.csr_matrix((mat["vals"], mat["col_idx"], mat["row_ptr"]), shape=(mat["m"], mat["n"]))
        Ah = (A @ sps.diags(1.0 / d)).tocsr()
    m = Ah.shape[0]

    def ATq(q):
        if blocks <= 0:
            return Ah.T @ q
        B = -(-m // blocks)
        parts = [Ah[i:i + B].T @ q[i:i + B] for i in range(0, m, B)]
        while len(parts) > 1:
            parts = [parts[i] + parts[i + 1] if i + 1 < len(parts) else parts[i] for i in range(0, len(parts), 2)]
        return parts[0]

    P = (lambda v: orc.sgs_apply(Mo, v, sweeps)) if sweeps > 0 else (lambda v: v.copy())
    h = ATq(b)
    hn = np.linalg.norm(h)
    y = np.zeros(h.shape[0])
    it = 0
    for outer in range(max_outer):
        g = ATq(b - Ah @ y)
        if np.linalg.norm(g) <= tol * hn or it >= maxit:
            break
        z = P(g)
        p, rho = z.copy(), g @ z
        while it < maxit:
            q = Ah @ p
            w = ATq(q)
            alpha = rho / (q @ q)
            y += alpha * p
            g -= alpha * w
            it += 1
            if np.linalg.norm(g) <= tol * hn:
                break
            z = P(g)
            rho_new = g @ z
            p = z + (rho_new / rho) * p
            rho = rho_new
    return it


def rounding_variant_iters(orc, mat, smp, Mo, b, tol, sweeps=1, maxit=1000000, max_outer=20, nperm=2):
    """Iteration counts of equally valid FP64 evaluations of the same PCG on the same
    problem (same D, same sampled A_s^T A_s): the oracle on row-permuted copies of A and b
    (only the summation order of the products changes), a numpy evaluation in BLAS order
    with p^T w = ||Â p||^2 (the form the fused pass computes), and the same with the sums
    over rows taken as 152 block partials combined pairwise (the reduction shape of the GPU
    path, more accurate than one sequential sum over m rows).  Their spread around the
    oracle's own count is the rounding sensitivity of CG on this problem."""
    b = np.asarray(b, np.float64)
    m = int(smp.mat.m)
    rng = np.random.default_rng(12345)
    out = []
    for _ in range(nperm):
        perm = rng.permutation(m)
        pm = _permuted_rows(mat, perm)
        _, oi = orc.pcg(orc.as_mat(pm), smp.d, Mo, b=b[perm], tol=tol, maxit=maxit,
                        max_outer=max_outer, sweeps=sweeps)
        out.append(int(oi["iters"]))
    out.append(_numpy_pcg_iters(orc, mat, smp.d, Mo, b, tol, sweeps, maxit, max_outer))
    out.append(_numpy_pcg_iters(orc, mat, smp.d, Mo, b, tol, sweeps, maxit, max_outer, blocks=152))
    return out


def assert_iterations(gpu_iters, or_iters, variants, what=""):
    """Iteration parity: within +-2 of the oracle, or, where rounding alone moves the count
    further (ill-conditioned problems), within twice the largest distance of the oracle's
    equally valid FP64 evaluations (``variants``: a list, or a callable giving one, called
    only when the +-2 bar is missed)."""
    gap = abs(int(gpu_iters) - int(or_iters))
    if gap <= 2:
        record_parity(what, gpu_iters=int(gpu_iters), oracle_iters=int(or_iters))
        return
    vs = variants() if callable(variants) else variants
    spread = max(abs(int(v) - int(or_iters)) for v in vs)
    assert gap <= max(2, 2 * spread), (
        f"{what}: GPU {gpu_iters} vs oracle {or_iters} iterations; FP64 rounding variants {vs} "
        f"(spread {spread}) allow {max(2, 2 * spread)}")
    record_parity(what, gpu_iters=int(gpu_iters), oracle_iters=int(or_iters), variants=list(vs))


def record_parity(what, **kw):
    """Append one measured parity line to $LSQ_PARITY_LOG (JSON lines), if set."""
    import json
    import os
    path = os.environ.get("LSQ_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"case": what, **kw}) + "\n")
