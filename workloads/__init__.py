"""Seeded synthetic inputs for the row-sampling SGS-preconditioned PCG least-squares solver.

This module only draws random matrices and right-hand sides; it holds none of the
method's arithmetic (no norms, no sampling, no preconditioner, no solve).  Both the
CPU oracle's tests and the CUDA path's tests and benchmark take their inputs from
here, so that the two sides see the same bits.

Every generator is a pure function of its arguments (numpy ``default_rng(seed)``),
returns host numpy arrays, and describes its matrix as either

* dense:  ``{"kind": "dense", "A": (m, n) float64 C-contiguous}``
* CSR:    ``{"kind": "csr", "m", "n", "row_ptr": int64[m+1], "col_idx": int32[nnz],
            "vals": float64[nnz]}`` with strictly increasing columns inside a row.

The workload families follow the paper's experiment classes (Section 5): Gaussian
(5.1), UDV (5.4), sparse random (5.3) and graph incidence (5.5), at the sizes of the
solver's benchmark configurations.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "gaussian_dense", "udv_dense", "semi_gaussian_dense", "coherent_dense",
    "sparse_random", "graph_incidence", "chung_lu_incidence", "rhs_for", "uneven_dense_batch",
    "csr_from_dense", "dense_from_csr", "orthonormal_q",
]


def _rng(seed):
    return np.random.default_rng(seed)


def gaussian_dense(m: int, n: int, seed: int) -> dict:
    """A = randn(m, n): i.i.d. N(0,1) entries (Section 5.1, Gaussian matrix)."""
    A = _rng(seed).standard_normal((m, n))
    return {"kind": "dense", "A": np.ascontiguousarray(A)}


def orthonormal_q(G: np.ndarray, matmul=None) -> np.ndarray:
    """The Q factor with positive-diagonal R of a tall full-rank G (it is unique), by
    Cholesky QR applied twice: R = chol(G^T G), Q = G R^{-1}, repeated once on Q.

    ``matmul(X, Y) -> X @ Y`` may run the two large products elsewhere (for example on a
    device); the n x n Cholesky factors and inverses are computed here in FP64.
    """
    mm = matmul or (lambda X, Y: X @ Y)
    Q = np.asarray(G, dtype=np.float64)
    R_total = np.eye(Q.shape[1])
    for _ in range(2):
        Gram = np.asarray(mm(Q.T, Q))
        R = np.linalg.cholesky((Gram + Gram.T) / 2).T
        Rinv = np.linalg.inv(R)
        Q = np.asarray(mm(Q, Rinv))
        R_total = R @ R_total
    return Q


def udv_dense(m: int, n: int, kappa: float, seed: int, matmul=None, spacing: str = "log") -> dict:
    """A = U diag(sigma) V^T (Section 5.4, UDV matrix).

    U is the orthonormal Q factor of a seeded Gaussian m x n, V the Q factor of a
    seeded Gaussian n x n (both with positive-diagonal R).  sigma is log-spaced from 1
    down to 1/kappa ("log"), or evenly spaced from 1 up to kappa ("linear", the paper's
    D = diag[1, 1 + (c - 1)/n, ..., c] with c = kappa); either way kappa(A) = kappa.
    ``matmul`` may run the large products on another device (see orthonormal_q).
    """
    rng = _rng(seed)
    G = rng.standard_normal((m, n))
    H = rng.standard_normal((n, n))
    U = orthonormal_q(G, matmul)
    V = orthonormal_q(H)
    if spacing == "linear":
        sigma = np.linspace(1.0, kappa, n)
    else:
        sigma = np.logspace(0.0, -math.log10(kappa), n)
    mm = matmul or (lambda X, Y: X @ Y)
    A = np.asarray(mm(U * sigma[None, :], V.T))
    return {"kind": "dense", "A": np.ascontiguousarray(A), "sigma": sigma}


def semi_gaussian_dense(m: int, n: int, seed: int) -> dict:
    """[B 0; 0 I_{n/2}] with B Gaussian (m - n/2) x n/2 (Section 5.2, coherent)."""
    h = n // 2
    A = np.zeros((m, n))
    A[: m - (n - h), :h] = _rng(seed).standard_normal((m - (n - h), h))
    A[m - (n - h):, h:] = np.eye(n - h)
    return {"kind": "dense", "A": A}


def coherent_dense(m: int, n: int) -> dict:
    """Z = [I_n; 0] (Section 3.1, the fully coherent example)."""
    A = np.zeros((m, n))
    A[:n, :n] = np.eye(n)
    return {"kind": "dense", "A": A}


def _csr_from_coo(m, n, rows, cols, vals):
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return {"kind": "csr", "m": int(m), "n": int(n), "row_ptr": row_ptr,
            "col_idx": cols.astype(np.int32), "vals": vals.astype(np.float64)}


def sparse_random(m: int, n: int, nnz_per_row: int, seed: int,
                  log10_scale: float = 2.0) -> dict:
    """Sparse random CSR in the spirit of the paper's ``sprand`` tests (Section 5.3).

    Each row has ``nnz_per_row`` distinct uniform random columns; every column j gets
    one extra entry at a uniform random row (skipped if already present), so that no
    column is empty.  Values are N(0,1) times a per-row scale 10^U(-s, s) with
    s = ``log10_scale`` (rows of very different norms, which the norm-squared
    sampling density is designed for).
    """
    rng = _rng(seed)
    k = nnz_per_row
    cols = rng.integers(0, n, size=(m, k), dtype=np.int64)
    # redraw duplicates inside a row until every row has k distinct columns
    while True:
        s = np.sort(cols, axis=1)
        dup_rows = np.nonzero((s[:, 1:] == s[:, :-1]).any(axis=1))[0]
        if dup_rows.size == 0:
            break
        cols[dup_rows] = rng.integers(0, n, size=(dup_rows.size, k), dtype=np.int64)
    extra_rows = rng.integers(0, m, size=n, dtype=np.int64)
    extra_cols = np.arange(n, dtype=np.int64)
    present = (cols[extra_rows] == extra_cols[:, None]).any(axis=1)
    er, ec = extra_rows[~present], extra_cols[~present]
    scale = 10.0 ** rng.uniform(-log10_scale, log10_scale, size=m)
    nb = m * k
    z = rng.standard_normal(nb + er.size)   # the k entries of every row in turn, then the extras
    vb = z[:nb].reshape(m, k) * scale[:, None]
    ve = z[nb:] * scale[er]
    # CSR with sorted columns: sort each row's k entries, then merge the extra entries (at
    # most one per column, so at most n of them) into their rows
    order = np.argsort(cols, axis=1, kind="stable")
    cs = np.take_along_axis(cols, order, axis=1)
    vs = np.take_along_axis(vb, order, axis=1)
    eo = np.lexsort((ec, er))
    er, ec, ve = er[eo], ec[eo], ve[eo]
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(k + np.bincount(er, minlength=m), out=row_ptr[1:])
    # slot of an extra entry: its row's start + the row's smaller base columns + the row's
    # earlier extra entries
    pos_e = row_ptr[er] + (cs[er] < ec[:, None]).sum(axis=1) + (np.arange(er.size) - np.searchsorted(er, er))
    nnz = int(row_ptr[-1])
    col_idx = np.empty(nnz, dtype=np.int64)
    vals = np.empty(nnz, dtype=np.float64)
    base = np.ones(nnz, dtype=bool)
    base[pos_e] = False
    col_idx[pos_e], vals[pos_e] = ec, ve
    col_idx[base], vals[base] = cs.reshape(-1), vs.reshape(-1)
    return {"kind": "csr", "m": int(m), "n": int(n), "row_ptr": row_ptr,
            "col_idx": col_idx.astype(np.int32), "vals": vals}


def graph_incidence(n_nodes: int, n_edges: int, seed: int,
                    log10_w: float = 3.0) -> dict:
    """Weighted incidence matrix of a random connected graph (Section 5.5).

    ``n_edges`` edges with uniform random endpoints (self-loops redrawn, duplicate
    edges allowed) plus a spanning path over a seeded random permutation of the
    nodes, so the graph is connected.  Edge e with weight w_e = 10^U(-3,3) gives a
    row with +sqrt(w_e) at its source and -sqrt(w_e) at its target.  Node 0 is
    grounded (its column removed), so the matrix has full column rank n_nodes - 1.
    """
    rng = _rng(seed)
    src = rng.integers(0, n_nodes, size=n_edges, dtype=np.int64)
    dst = rng.integers(0, n_nodes, size=n_edges, dtype=np.int64)
    while True:
        loops = np.nonzero(src == dst)[0]
        if loops.size == 0:
            break
        dst[loops] = rng.integers(0, n_nodes, size=loops.size, dtype=np.int64)
    perm = rng.permutation(n_nodes).astype(np.int64)
    src = np.concatenate([src, perm[:-1]])
    dst = np.concatenate([dst, perm[1:]])
    m = src.size
    w = 10.0 ** rng.uniform(-log10_w, log10_w, size=m)
    sw = np.sqrt(w)
    rows = np.concatenate([np.arange(m), np.arange(m)])
    cols = np.concatenate([src, dst])
    vals = np.concatenate([sw, -sw])
    keep = cols != 0
    return _csr_from_coo(m, n_nodes - 1, rows[keep], cols[keep] - 1, vals[keep])


def _chung_lu_edges(rng, n, beta, d, i0):
    """Edges (i < j) of a Chung-Lu random graph with power-law expected degrees
    w_i = c (i0 + i)^(-1/(beta-1)), c = (beta-2)/(beta-1) d n^(1/(beta-1)) (so that the mean
    degree is about d); edge (i, j) present with probability min(1, w_i w_j / sum w)."""
    c = (beta - 2.0) / (beta - 1.0) * d * n ** (1.0 / (beta - 1.0))
    w = c * (i0 + np.arange(n, dtype=np.float64)) ** (-1.0 / (beta - 1.0))
    P = np.minimum(1.0, np.outer(w, w) / w.sum())
    upper = np.triu(rng.random((n, n)) < P, k=1)
    return np.nonzero(upper)


def chung_lu_incidence(n: int, seed: int, beta1: float = 5.0, d1: float = 30.0,
                       beta2: float = 8.0, d2_per_node: float = 5.0, i0: int = 11,
                       overlap: int = 5, ground: bool = False) -> dict:
    """The random graph Laplacian family of Section 5.5: the incidence matrix B of a graph.

    Two Chung-Lu power-law graphs on n vertices each: a sparse ill-conditioned one
    (beta = 5, mean degree 30) and a dense well-conditioned one (beta = 8, mean degree 5 n,
    capped by the edge probability 1), glued so that the last `overlap` vertices of the first
    are the first of the second (2n - overlap vertices).  Every edge (i < j) is a row with +1
    at i and -1 at j, so B^T B = D - A, the graph Laplacian.  Vertices without edges are
    dropped.  B^T B is then singular (the constant vector of each connected component), as
    in the paper, whose condition numbers for this family are the effective ones; the normal
    equations stay consistent and the fitted values B x are unique.  With ground=True the
    first vertex of every component is grounded (its column removed) instead, which gives
    full column rank.
    """
    rng = _rng(seed)
    s1, t1 = _chung_lu_edges(rng, n, beta1, d1, i0)
    s2, t2 = _chung_lu_edges(rng, n, beta2, d2_per_node * n, i0)
    off = n - overlap
    src = np.concatenate([s1, s2 + off]).astype(np.int64)
    dst = np.concatenate([t1, t2 + off]).astype(np.int64)
    nv = 2 * n - overlap
    used = np.zeros(nv, bool)
    used[src] = True
    used[dst] = True
    # connected components (union-find over the edges): one grounded vertex each on request
    parent = np.arange(nv)
    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    for a, b in zip(src.tolist(), dst.tolist()):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(v) for v in range(nv)])
    grounded = used & (roots == np.arange(nv)) if ground else np.zeros(nv, bool)
    keep = used & ~grounded
    col_of = -np.ones(nv, np.int64)
    col_of[keep] = np.arange(int(keep.sum()))
    m = src.size
    rows = np.concatenate([np.arange(m), np.arange(m)])
    cols = np.concatenate([col_of[src], col_of[dst]])
    vals = np.concatenate([np.ones(m), -np.ones(m)])
    ok = cols >= 0
    return _csr_from_coo(m, int(keep.sum()), rows[ok], cols[ok], vals[ok])


def rhs_for(mat: dict, k: int, noise: float, seed: int):
    """x* ~ N(0,1) (n x k) and b = A x* + noise * N(0,1) (m x k), column-major blocks.

    Returns (xstar, b) as float64 arrays of shape (k, n) and (k, m): row c of each is
    right-hand side / solution number c, contiguous.
    """
    rng = _rng(seed)
    if mat["kind"] == "dense":
        m, n = mat["A"].shape
    else:
        m, n = mat["m"], mat["n"]
    xstar = rng.standard_normal((k, n))
    if mat["kind"] == "dense":
        Ax = (mat["A"] @ xstar.T).T
    else:
        Ax = np.empty((k, m))
        rp, ci, v = mat["row_ptr"], mat["col_idx"], mat["vals"]
        rows = np.repeat(np.arange(m), np.diff(rp))
        for c in range(k):
            Ax[c] = np.bincount(rows, weights=v * xstar[c][ci], minlength=m)
    b = Ax + noise * rng.standard_normal((k, m))
    return np.ascontiguousarray(xstar), np.ascontiguousarray(b)


def uneven_dense_batch(count: int, m_range, n_range, seed: int):
    """``count`` dense Gaussian problems with m, n drawn log-uniform in the ranges."""
    rng = _rng(seed)
    out = []
    for _ in range(count):
        m = int(round(math.exp(rng.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        n = min(n, m)
        out.append({"kind": "dense", "A": rng.standard_normal((m, n))})
    return out


def csr_from_dense(A: np.ndarray, keep_zeros: bool = True) -> dict:
    """CSR view of a dense matrix (all entries stored when ``keep_zeros``)."""
    m, n = A.shape
    if keep_zeros:
        rows = np.repeat(np.arange(m, dtype=np.int64), n)
        cols = np.tile(np.arange(n, dtype=np.int64), m)
        vals = A.reshape(-1)
    else:
        rows, cols = np.nonzero(A)
        vals = A[rows, cols]
    return _csr_from_coo(m, n, rows.astype(np.int64), cols.astype(np.int64), vals)


def dense_from_csr(mat: dict) -> np.ndarray:
    A = np.zeros((mat["m"], mat["n"]))
    rows = np.repeat(np.arange(mat["m"]), np.diff(mat["row_ptr"]))
    np.add.at(A, (rows, mat["col_idx"]), mat["vals"])
    return A
