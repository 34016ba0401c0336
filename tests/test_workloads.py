"""The seeded input generators have the structure the paper's examples describe.

These check the inputs, not the method: the generators hold none of the method's
arithmetic and serve both the oracle and the GPU path.
"""
import math

import numpy as np

import workloads as W


def test_gaussian_condition_number_is_the_bai_yin_limit():
    """Sec. 5.1: for A = randn(m, n), kappa(A^T A) tends to ((sqrt m + sqrt n)/(sqrt m - sqrt n))^2
    (the paper prints the ratio without the square; the square is the Bai-Yin limit of the
    extreme eigenvalues, (1 +- sqrt(n/m))^2 m)."""
    m, n = 4096, 128
    A = W.gaussian_dense(m, n, 1)["A"]
    kappa = np.linalg.cond(A.T @ A)
    limit = ((math.sqrt(m) + math.sqrt(n)) / (math.sqrt(m) - math.sqrt(n))) ** 2
    assert abs(kappa / limit - 1.0) < 0.1, (kappa, limit)


def test_udv_has_the_prescribed_singular_values():
    """Sec. 5.4: A = U D V with orthonormal U, V, so the singular values are exactly D's."""
    for spacing in ("log", "linear"):
        mat = W.udv_dense(2000, 40, 1e3, 2, spacing=spacing)
        sv = np.linalg.svd(mat["A"], compute_uv=False)
        want = np.sort(mat["sigma"])[::-1]
        np.testing.assert_allclose(sv, want, rtol=1e-10)
        assert abs(sv[0] / sv[-1] - 1e3) < 1e-6 * 1e3
    lin = W.udv_dense(500, 10, 50.0, 3, spacing="linear")["sigma"]
    np.testing.assert_allclose(np.diff(lin), np.full(9, 49.0 / 9.0))


def test_semi_gaussian_block_structure():
    """Sec. 5.2: A = [B 0; 0 I_{n/2}], so A^T A = diag(B^T B, I) and the last n/2 rows are
    the identity (the coherent rows)."""
    m, n = 500, 16
    A = W.semi_gaussian_dense(m, n, 4)["A"]
    h = n // 2
    G = A.T @ A
    np.testing.assert_array_equal(G[:h, h:], 0.0)
    np.testing.assert_array_equal(G[h:, h:], np.eye(h))
    np.testing.assert_array_equal(A[m - h:, h:], np.eye(h))
    assert np.count_nonzero(A[: m - h, :h]) == (m - h) * h


def test_graph_incidence_rows_and_laplacian():
    """Sec. 5.5: each row of a weighted incidence matrix holds +sqrt(w) and -sqrt(w), so with
    the grounded node put back, B^T B is a weighted Laplacian (zero row sums)."""
    n_nodes = 300
    mat = W.graph_incidence(n_nodes, 1200, 5)
    m = mat["m"]
    rows = np.repeat(np.arange(m), np.diff(mat["row_ptr"]))
    B = np.zeros((m, n_nodes))
    full = W.dense_from_csr(mat)
    B[:, 1:] = full
    # the grounded node's entry is whatever makes the row sum to zero
    B[:, 0] = -full.sum(axis=1)
    per_row = np.diff(mat["row_ptr"])
    assert set(np.unique(per_row)) <= {1, 2}
    L = B.T @ B
    np.testing.assert_allclose(L.sum(axis=1), 0.0, atol=1e-9 * np.abs(L).max())
    w = np.abs(mat["vals"]) ** 2
    assert 1e-3 * (1 - 1e-12) <= w.min() and w.max() <= 1e3 * (1 + 1e-12)
    # connected (the spanning path): the grounded Laplacian is nonsingular
    assert np.linalg.matrix_rank(full) == n_nodes - 1
    assert rows.size == mat["vals"].size


def test_chung_lu_laplacian_family_sizes_and_structure():
    """Sec. 5.5: B is the incidence matrix of two glued Chung-Lu graphs.  Each row holds +1 and
    -1, B^T B = D - A (degrees on the diagonal, -1 per edge), isolated vertices are dropped and
    the null space of B is the constant vector on each connected component.  The vertex count
    for 2 n - 5 glued vertices and nnz(B^T B) = n + 2 m are the paper's printed sizes (its
    table: n = 187, 355, 536, 709, 856; the number of edges is random, within 15 % of the
    printed m = 5078 ... 101829)."""
    paper = {96: (187, 5078), 180: (355, 19475), 270: (536, 41032), 357: (709, 68969),
             430: (856, 101829)}
    for n_param, (n_paper, m_paper) in paper.items():
        mat = W.chung_lu_incidence(n_param, 5)
        assert abs(mat["n"] - n_paper) <= 1, (mat["n"], n_paper)
        assert abs(mat["m"] / m_paper - 1.0) < 0.16, (mat["m"], m_paper)
    mat = W.chung_lu_incidence(96, 5)
    B = W.dense_from_csr(mat)
    m, n = B.shape
    assert np.array_equal(np.sort(B, axis=1)[:, [0, -1]], np.tile([-1.0, 1.0], (m, 1)))
    assert np.count_nonzero(B) == 2 * m
    L = B.T @ B
    deg = np.count_nonzero(B, axis=0)
    assert deg.min() >= 1
    np.testing.assert_array_equal(np.diag(L), deg)
    off = L - np.diag(np.diag(L))
    assert set(np.unique(off)) <= {-1.0, 0.0, -2.0}   # -2 only for an edge present in both graphs
    np.testing.assert_array_equal(L.sum(axis=1), 0.0)
    assert np.count_nonzero(L) == n + 2 * len({tuple(r) for r in np.argwhere(off != 0) if r[0] < r[1]})
    # one null vector per component: rank n - (#components)
    comps = int(np.sum(np.linalg.eigvalsh(L) < 1e-9 * n))
    assert comps >= 1 and np.linalg.matrix_rank(B) == n - comps
    g = W.chung_lu_incidence(96, 5, ground=True)
    assert g["m"] == m and g["n"] == n - comps
    assert np.linalg.matrix_rank(W.dense_from_csr(g)) == g["n"]
