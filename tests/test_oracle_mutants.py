"""Planted mistakes: the oracle pins must catch a plausible error anywhere in the oracle.

Each case copies the oracle's C source, plants one mistake of the kind a careful reader
could still make (a dropped term, a wrong sign, index or operand, a swapped ratio), builds
the copy with the oracle's own compile step and runs the pin suite against it.  The pins
pass on the unmodified oracle and must fail on every copy: otherwise they would not pin
the step the mistake sits in.  Mistakes are planted on the CPU only.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lsq_oracle.c")
PY = os.path.join(ROOT, "oracle", "__init__.py")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (id, step of the paper, text in the oracle, planted replacement)
MUTANTS = [
    ("sample_size_log2", "Alg. 2 step 2: s = 4 n log n with the natural log",
     "log((double)n)", "log2((double)n)"),
    ("col_scale_no_sqrt", "Alg. 2 step 1: D_jj is the column norm, not its square",
     "d[j] = sqrt(d2[j]);", "d[j] = d2[j];"),
    ("weights_unnormalised", "Eq. (R2P) on the normalised matrix: a^2 / d^2",
     "double u = t * inv_d2[row_col(A, i, k)];", "double u = t;"),
    ("philox_key_word", "Philox4x64-10 (Salmon et al.): key word k0 enters n0",
     "uint64_t n0 = hi1 ^ c1 ^ k0,", "uint64_t n0 = hi1 ^ c1 ^ k1,"),
    ("philox_nine_rounds", "Philox4x64-10 (Salmon et al.): ten rounds",
     "for (int r = 0; r < 10; ++r) {", "for (int r = 0; r < 9; ++r) {"),
    ("philox_weyl_constant", "Philox4x64-10: Weyl constant of the first key word",
     "W0 = 0x9E3779B97F4A7C15ull", "W0 = 0x9E3779B97F4A7C17ull"),
    ("prefix_inclusive", "Alg. 1: the search runs over the exclusive prefix",
     "        P_lo[i] = (uint64_t)acc;\n        P_hi[i] = (uint64_t)(acc >> 64);\n"
     "        acc += ((u128)w_hi[i] << 64) | w_lo[i];\n",
     "        acc += ((u128)w_hi[i] << 64) | w_lo[i];\n        P_lo[i] = (uint64_t)acc;\n"
     "        P_hi[i] = (uint64_t)(acc >> 64);\n"),
    ("draw_words_swapped", "Alg. 1: the 128-bit uniform is word1 * 2^64 + word0",
     "u128 U = ((u128)r[1] << 64) | r[0];", "u128 U = ((u128)r[0] << 64) | r[1];"),
    ("M_scale_wrong_column", "Sec. 3.3: entry (j, c) of a draw's outer product is a_ij a_ic / (d_j d_c)",
     "acc[c] += coef * (v[k] / d[c]);", "acc[c] += coef * (v[k] / d[j]);"),
    ("M_scale_drops_s", "Sec. 3.3: each draw is scaled by 1 / (s p_i)",
     "gam[t] = 1.0 / ((double)s * p);", "gam[t] = 1.0 / p;"),
    ("M_unnormalised_column", "Sec. 3.3: M is built from the normalised rows a_i D^{-1}",
     "acc[c] += coef * (v[k] / d[c]);", "acc[c] += coef * v[k];"),
    ("M_zero_diagonal_kept", "a zero diagonal of M is replaced by 1",
     "if (c == j && val == 0.0) { val = 1.0;", "if (c == j && val == 0.0) { val = 0.5;"),
    ("sgs_forward_takes_diagonal", "Alg. 3: B is the lower triangle; the diagonal divides",
     "if (M->col[q] < j) acc -= M->val[q] * del[M->col[q]];",
     "if (M->col[q] <= j) acc -= M->val[q] * del[M->col[q]];"),
    ("sgs_backward_lower_triangle", "Alg. 3: the backward sweep uses B^T, the upper triangle",
     "if (M->col[q] > j) acc -= M->val[q] * del[M->col[q]];",
     "if (M->col[q] < j) acc -= M->val[q] * del[M->col[q]];"),
    ("sgs_backward_runs_forward", "Alg. 3: the backward correction is a back substitution, row n-1 first",
     "for (int64_t j = n - 1; j >= 0; --j) {", "for (int64_t j = 0; j < n; ++j) {"),
    ("sgs_correction_replaces_e", "Alg. 3: each correction is added to e",
     "for (int64_t j = 0; j < n; ++j) e[j] += del[j];", "for (int64_t j = 0; j < n; ++j) e[j] = del[j];"),
    ("sgs_residual_sign", "Alg. 3: the correction solves for r - M e",
     "res[j] = r[j] - acc;", "res[j] = r[j] + acc;"),
    ("apply_A_unnormalised", "Sec. 4.2: q = A D^{-1} p",
     "acc += (v[k] / d[j]) * p[j];", "acc += v[k] * p[j];"),
    ("apply_A_times_d", "Sec. 4.2: q = A D^{-1} p divides by the column scale",
     "acc += (v[k] / d[j]) * p[j];", "acc += (v[k] * d[j]) * p[j];"),
    ("apply_AT_wrong_operand", "Sec. 4.2: w = D^{-1} A^T q, entry (i, j) times q_i",
     "w[j] += (v[k] / d[j]) * q[i];", "w[j] += (v[k] / d[j]) * q[i] * (i % 2 ? 1.0 : -1.0);"),
    ("pcg_residual_sign", "Alg. 2 step 4: g <- g - alpha A^T A p",
     "g[j] -= alpha * w[j];", "g[j] += alpha * w[j];"),
    ("pcg_beta_inverted", "Alg. 2 step 4: beta = rho_new / rho",
     "double beta = rho_new / rho;", "double beta = rho / rho_new;"),
    ("pcg_direction_drops_z", "Alg. 2 step 4: p = z + beta p",
     "p[j] = z[j] + beta * p[j];", "p[j] = g[j] + beta * p[j];"),
    ("col_sum_global_exponent", "Alg. 2 step 1: each column is summed at its own exponent",
     "c[j] += (u128)floor_scaled(t, E1j[j]);", "c[j] += (u128)floor_scaled(t, E1);"),
    ("weights_abs_not_square", "Eq. (R2P): squared row norms",
     "double t = v[k] * v[k];\n            double u", "double t = fabs(v[k]);\n            double u"),
    ("sgs_no_backward_sweep", "Alg. 3: t forward then t backward corrections",
     "for (int dir = 0; dir < 2; ++dir) {", "for (int dir = 0; dir < 1; ++dir) {"),
    ("apply_AT_times_d", "Sec. 4.2: w = D^{-1} A^T q",
     "w[j] += (v[k] / d[j]) * q[i];", "w[j] += (v[k] * d[j]) * q[i];"),
    ("pcg_rho_unpreconditioned", "Alg. 2 step 4: rho = g^T z with z = P g",
     "double rho = dot(n, g, z);", "double rho = dot(n, g, g);"),
    ("pcg_alpha_half", "Alg. 2 step 4: alpha = rho / p^T A^T A p",
     "double alpha = rho / pw;", "double alpha = 0.5 * rho / pw;"),
    ("pcg_stop_absolute", "Alg. 2 step 4: the stop test is relative to ||A^T b||",
     "if (gn <= tol * hnorm) break;", "if (gn <= tol) break;"),
    ("pcg_true_residual_sign", "Alg. 2 step 4: the true residual is A^T (b - A y)",
     "for (int64_t i = 0; i < m; ++i) r[i] = b[i] - r[i];\n            orc_apply_AT(A, d, r, g);\n"
     "        } else {\n            orc_normal_matvec(A, d, y, w);\n"
     "            for (int64_t j = 0; j < n; ++j) g[j] = h[j] - w[j];\n        }\n"
     "        double gn",
     "for (int64_t i = 0; i < m; ++i) r[i] = b[i] + r[i];\n            orc_apply_AT(A, d, r, g);\n"
     "        } else {\n            orc_normal_matvec(A, d, y, w);\n"
     "            for (int64_t j = 0; j < n; ++j) g[j] = h[j] - w[j];\n        }\n"
     "        double gn"),
]


def _run_pins(lib):
    env = dict(os.environ, LSQ_ORACLE_MUTANT=lib, PYTHONDONTWRITEBYTECODE="1")
    return subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider",
                           "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


def _build(tmp_path, src_text):
    import oracle
    src = tmp_path / "lsq_oracle.c"
    src.write_text(src_text)
    return oracle.compile_source(str(src), str(tmp_path / "liblsq_oracle.so"))


def test_pins_pass_on_the_oracle_built_as_a_copy(tmp_path):
    """The harness itself: an unmodified copy, built the same way, passes every pin."""
    out = _run_pins(_build(tmp_path, open(SRC).read()))
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-2000:]


@pytest.mark.parametrize("mid,step,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, mid, step, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, f"{mid}: the planted text must occur once in the oracle"
    out = _run_pins(_build(tmp_path, text.replace(old, new)))
    # 1: a pin failed.  A crash of the copy (negative: killed by a signal) also counts as
    # caught; 2-5 (interrupted, internal or usage error, nothing collected) do not.
    assert out.returncode == 1 or out.returncode < 0, (mid, step, out.returncode, out.stdout[-1500:])


# Mistakes in the oracle's Python layer (oracle/__init__.py): the steps it computes itself
# rather than in C.  (id, step of the paper, text, planted replacement)
PY_MUTANTS = [
    ("solve_x_times_d", "Alg. 2: x = D^{-1} y", "self.x = y / self.smp.d", "self.x = y * self.smp.d"),
    ("adjoint_rhs_times_d", "adjoint: A^T A lam = G is solved as Â^T Â mu = D^{-1} G",
     "h=np.asarray(G, np.float64) / d", "h=np.asarray(G, np.float64) * d"),
    ("adjoint_lam_times_d", "adjoint: lam = D^{-1} mu", "lam = mu / d", "lam = mu * d"),
    ("adjoint_dense_sign", "adjoint: dL/dA = r lam^T - (A lam) x^T",
     "gA = np.outer(r, lam) - np.outer(Alam, x)", "gA = np.outer(r, lam) + np.outer(Alam, x)"),
    ("adjoint_csr_operand", "adjoint: dL/dA_ij = r_i lam_j - (A lam)_i x_j",
     "gv = r[rows] * lam[cols] - Alam[rows] * x[cols]", "gv = r[rows] * lam[cols] - Alam[rows] * x[rows % x.size]"),
    ("uniform_keeps_norm2", "Sec. 3.1: uniform sampling gives every row the same weight",
     "self.w_lo = np.ones(self.mat.m, np.uint64)", "self.w_lo, _ = row_weights(self.mat, self.inv_d2)"),
]


def _run_pins_py(pkg_dir):
    env = dict(os.environ, LSQ_ORACLE_PKG=str(pkg_dir), PYTHONDONTWRITEBYTECODE="1")
    env.pop("LSQ_ORACLE_MUTANT", None)
    return subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider",
                           "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


def _copy_package(tmp_path, py_text):
    d = tmp_path / "oracle"
    d.mkdir()
    (d / "lsq_oracle.c").write_text(open(SRC).read())
    (d / "__init__.py").write_text(py_text)
    return tmp_path


def test_pins_pass_on_the_oracle_package_copied(tmp_path):
    """The Python harness itself: an unmodified copy of the package passes every pin."""
    out = _run_pins_py(_copy_package(tmp_path, open(PY).read()))
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-2000:]


@pytest.mark.parametrize("mid,step,old,new", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_pins_catch_planted_mistake_in_the_python_layer(tmp_path, mid, step, old, new):
    text = open(PY).read()
    assert text.count(old) == 1, f"{mid}: the planted text must occur once in the oracle"
    out = _run_pins_py(_copy_package(tmp_path, text.replace(old, new)))
    assert out.returncode == 1 or out.returncode < 0, (mid, step, out.returncode, out.stdout[-1500:])
