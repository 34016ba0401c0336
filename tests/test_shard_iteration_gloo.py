"""The row-sharded PCG iteration with world-size-2 and -3 gloo ranks on CPU (the exchange
step of the multi-GPU design; no GPU).

A rank holds a contiguous block of rows A_r and b_r.  Because Â^T Â p = Σ_r Â_r^T (Â_r p),
one iteration needs exactly one all-reduce of an n-vector: every rank forms its partial
normal product and the all-reduced sum is the same on every rank.  Everything else of the
iteration (the SGS apply on the replicated M, the dots, alpha, beta, the updates of y, g, p)
works on replicated n-vectors and needs no communication.  The right-hand side Â^T b and
each outer step's true residual Â^T (b - Â y) are one all-reduce each in the same way.

Each rank computes its partial products with the oracle's Â p and Â^T q on its own rows,
and M comes from the merged draws (which the sharded-sampling test shows equal to one
process's).  The iteration below follows the same textbook steps as the oracle's PCG
(Alg. 2 step 4, with the stop test of Sec. 5 on the normalised residual) so that the two
can be compared: the sharded solve must give the single-process iteration count within
the ±2 bar, a solution within rounding of the single-process one, and bit-identical
replicated state on every rank.

The preconditioner's matrix shards the same way (Sec. 3.3): A_s^T A_s = Σ_t â_{i_t}^T
â_{i_t} / (s p_{i_t}) splits by the rank that owns row i_t, so each rank sums the draws
that landed in its rows, with the global s and p_i = w_i / W, and one all-reduce of the
n×n partials (before the zero-diagonal fix, which belongs to the sum) gives the matrix one
process builds."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    # name: (world, matrix builder, tol, sweeps)
    "dense_gauss_3001x40": (2, lambda W: W.gaussian_dense(3001, 40, 7), 1e-10, 1),
    "csr_5000x300": (3, lambda W: W.sparse_random(5000, 300, 8, 3), 1e-10, 1),
    "dense_udv_2000x48_k1e3": (2, lambda W: W.udv_dense(2000, 48, 1e3, 5), 1e-10, 2),
}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _row_block(mat, r0, r1):
    if mat["kind"] == "dense":
        return {"kind": "dense", "A": np.ascontiguousarray(mat["A"][r0:r1])}
    rp = mat["row_ptr"]
    return {"kind": "csr", "m": r1 - r0, "n": mat["n"], "row_ptr": rp[r0:r1 + 1] - rp[r0],
            "col_idx": mat["col_idx"][rp[r0]:rp[r1]], "vals": mat["vals"][rp[r0]:rp[r1]]}


def _rank(rank, world, port, case, out_dir):
    import datetime
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    _, build, tol, sweeps = CASES[case]
    mat = build(W)
    _, B = W.rhs_for(mat, 1, 1e-3, 11)
    b = B[0]
    smp = oracle.Sample(mat, seed=17)
    Mo = oracle.SampledM(smp)
    d = smp.d
    m, n = smp.mat.m, smp.mat.n
    bounds = [m * r // world for r in range(world + 1)]
    r0, r1 = bounds[rank], bounds[rank + 1]
    local = _row_block(mat, r0, r1)
    b_r = np.ascontiguousarray(b[r0:r1])
    exchanged = [0]

    def allreduce(v):
        t = torch.from_numpy(np.ascontiguousarray(v, np.float64).copy())
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        exchanged[0] += 1
        return t.numpy()

    def normal(p):                        # Σ_r Â_r^T (Â_r p): the one exchange of an iteration
        return allreduce(oracle.normal_matvec(local, d, p))

    # a single product first: the all-reduced partials against the whole matrix's product
    p_test = np.random.default_rng(3).standard_normal(n)   # the same p on every rank
    w_sum = normal(p_test)
    w_one = oracle.normal_matvec(mat, d, p_test)
    prod_err = float(np.linalg.norm(w_sum - w_one) / np.linalg.norm(w_one))

    exchanged[0] = 0
    h = allreduce(oracle.apply_AT(local, d, b_r))
    hnorm = float(np.sqrt(h @ h))
    y = np.zeros(n)
    iters, outer, converged = 0, 0, False
    per_iter = []
    for _outer in range(5):
        res = b_r - oracle.apply_A(local, d, y)
        g = allreduce(oracle.apply_AT(local, d, res))
        if np.sqrt(g @ g) <= tol * hnorm:
            converged = True
            break
        outer += 1
        z = oracle.sgs_apply(Mo, g, sweeps)
        p = z.copy()
        rho = float(g @ z)
        while iters < 10000:
            before = exchanged[0]
            w = normal(p)
            per_iter.append(exchanged[0] - before)
            alpha = rho / float(p @ w)
            y += alpha * p
            g -= alpha * w
            iters += 1
            if np.sqrt(g @ g) <= tol * hnorm:
                break
            z = oracle.sgs_apply(Mo, g, sweeps)
            rho_new = float(g @ z)
            p = z + (rho_new / rho) * p
            rho = rho_new
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"y{rank}.npy"), y)
    with open(os.path.join(out_dir, f"info{rank}.txt"), "w") as f:
        f.write(f"{iters} {outer} {int(converged)} {prod_err!r} {max(per_iter)} {min(per_iter)} "
                f"{exchanged[0]}\n")
    if rank == 0:
        y1, info = oracle.pcg(mat, d, Mo, b=b, tol=tol, sweeps=sweeps)
        np.save(os.path.join(out_dir, "y_single.npy"), y1)
        with open(os.path.join(out_dir, "single.txt"), "w") as f:
            f.write(f"{info['iters']} {info['outer']} {info['converged']}\n")


@pytest.mark.parametrize("case", list(CASES))
def test_sharded_iteration_matches_one_process(tmp_path, case):
    import torch.multiprocessing as mp
    world = CASES[case][0]
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, case, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    infos = [open(tmp_path / f"info{r}.txt").read().split() for r in range(world)]
    ys = [np.load(tmp_path / f"y{r}.npy") for r in range(world)]
    # replicated state: every rank ends with the same bits
    for r in range(1, world):
        assert np.array_equal(ys[r], ys[0])
        assert infos[r][:3] == infos[0][:3]
    iters, outer, conv = (int(v) for v in infos[0][:3])
    prod_err = float(infos[0][3])
    most, least, total = (int(v) for v in infos[0][4:7])
    assert prod_err < 1e-13                       # partial products sum to the whole product
    assert most == least == 1                     # one n-vector all-reduce per iteration
    assert total == iters + outer + 2             # plus Â^T b once and a true residual before each outer step and at the end
    assert conv == 1
    s_iters, s_outer, s_conv = (int(v) for v in open(tmp_path / "single.txt").read().split())
    assert s_conv == 1
    assert abs(iters - s_iters) <= 2
    y1 = np.load(tmp_path / "y_single.npy")
    # the solution bar of the GPU parity tests, 1e-8·kappa(Â), with kappa(Â) from the SVD of
    # the normalised matrix (measured: 1e-15 on the well-conditioned cases, 8e-9 at 1e3)
    sys.path.insert(0, ROOT)
    import oracle
    import workloads as W
    mat = CASES[case][1](W)
    A = mat["A"] if mat["kind"] == "dense" else W.dense_from_csr(mat)
    sv = np.linalg.svd(A / oracle.Sample(mat, seed=17).d, compute_uv=False)
    kappa = sv[0] / sv[-1]
    assert np.linalg.norm(ys[0] - y1) / np.linalg.norm(y1) <= 1e-8 * kappa


def _rank_M(rank, world, port, case, s_draws, out_dir):
    import datetime
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    mat = CASES[case][1](W)
    smp = oracle.Sample(mat, seed=17, s=s_draws)
    m, n = smp.mat.m, smp.mat.n
    bounds = [m * r // world for r in range(world + 1)]
    r0, r1 = bounds[rank], bounds[rank + 1]
    A = mat["A"] if mat["kind"] == "dense" else W.dense_from_csr(mat)
    # the draws this rank owns, as rows with their counts
    rows, counts = np.unique(smp.idx[(smp.idx >= r0) & (smp.idx < r1)], return_counts=True)
    Wd = float(smp.W)
    p = np.array([float(int(smp.w_hi[i]) << 64 | int(smp.w_lo[i])) for i in rows]) / Wd
    Ahat = A[rows] / smp.d
    M_r = (Ahat * (counts / (smp.s * p))[:, None]).T @ Ahat
    t = torch.from_numpy(np.ascontiguousarray(M_r))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    M = t.numpy().copy()
    fixed = np.flatnonzero(np.diag(M) == 0.0)
    M[fixed, fixed] = 1.0
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"M{rank}.npy"), M)
    with open(os.path.join(out_dir, f"own{rank}.txt"), "w") as f:
        f.write(f"{int(counts.sum())} {fixed.size}\n")
    if rank == 0:
        Mo = oracle.SampledM(smp)
        np.save(os.path.join(out_dir, "M_single.npy"), Mo.dense())
        with open(os.path.join(out_dir, "single.txt"), "w") as f:
            f.write(f"{smp.s} {Mo.n_fixed_diag}\n")


@pytest.mark.parametrize("case,s_draws", [("dense_gauss_3001x40", None), ("csr_5000x300", None),
                                          ("csr_5000x300", 150)])
def test_sharded_normal_matrix_matches_one_process(tmp_path, case, s_draws):
    """With 150 draws most columns of the CSR matrix are never sampled: their diagonal is
    fixed to 1 once, after the sum, and a column that only another rank sampled keeps
    that rank's value."""
    import torch.multiprocessing as mp
    world = CASES[case][0]
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_M, args=(r, world, port, case, s_draws, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    Ms = [np.load(tmp_path / f"M{r}.npy") for r in range(world)]
    for r in range(1, world):
        assert np.array_equal(Ms[r], Ms[0])          # the all-reduced M is the same on every rank
    owns = [open(tmp_path / f"own{r}.txt").read().split() for r in range(world)]
    s, n_fixed = (int(v) for v in open(tmp_path / "single.txt").read().split())
    assert sum(int(o[0]) for o in owns) == s          # every draw is summed by exactly one rank
    assert all(int(o[1]) == n_fixed for o in owns)
    assert (n_fixed > 0) == (s_draws is not None)
    M1 = np.load(tmp_path / "M_single.npy")
    assert np.array_equal(Ms[0] != 0.0, M1 != 0.0)   # the same pattern
    assert np.max(np.abs(Ms[0] - M1)) <= 1e-13 * np.max(np.abs(M1))
