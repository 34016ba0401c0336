/*
 * FP64 CPU oracle for PCG on the normal equation with a row-sampling SGS preconditioner
 * (Chen & Wu, "A Preconditioner based on Non-uniform Row Sampling for Linear Least
 * Squares Problems", arXiv:1806.02968).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct statement
 * of what the CUDA path computes.  Only the test suite, the smoke check and the
 * benchmark's CPU legs (the CPU baseline and the reference arm) may load it.  It shares no code, header or constant
 * table with the CUDA library, and the CUDA library never calls it.
 *
 * Every function follows one step of the paper, in the paper's order and notation:
 *   Alg. 2 step 1  normalisation A <- A D^{-1}, D_jj = ||a^j||       orc_col_scales
 *   Eq. (R2P)      sampling density p_k = ||a_k||^2 / ||A||_F^2       orc_row_weights
 *   Alg. 1         i.i.d. draws i_t ~ p, S_{t,i_t} = 1/sqrt(s p_i)    orc_prefix, orc_draw_rows
 *   Alg. 2 step 2  s = 4 n log n                                      orc_sample_size
 *   Sec. 3.3       A_s^T A_s = (1/s) sum_t a_{i_t}^T a_{i_t} / p_{i_t} orc_build_M
 *   Alg. 3         t forward then t backward Gauss-Seidel corrections orc_sgs_apply
 *   Alg. 2 step 4  PCG on A^T A x = A^T b                             orc_pcg
 *
 * Where the paper is silent the following readings are used (each is listed with its
 * reason in the design notes of the repository):
 *   - The sampling law is made exactly reproducible: squared entries are rounded once
 *     in FP64 (no fused multiply-add), column sums are exact 128-bit fixed-point sums,
 *     row weights are exact 128-bit sums of entries quantised at 2^-51, and the draws
 *     use the counter-based Philox4x64-10 generator (Salmon et al., SC'11) with
 *     key (seed, 0x5A4D504C) and counter (t, 0, 0, 0).  The quantised weights w_i/W
 *     ARE the sampling probabilities p_i used in the scaling 1/(s p_i).
 *   - "log" in s = 4 n log n is the natural logarithm, rounded up.
 *   - B in Alg. 3 is the lower triangle of A_s^T A_s including the diagonal; e0 = 0.
 *   - A zero diagonal entry of A_s^T A_s (a column never sampled) is replaced by 1,
 *     the diagonal of the normalised A^T A.
 *   - "relative residual" in Alg. 2 step 4 is ||g_k|| / ||g_0|| for the normalised
 *     normal-equation residual g = D^{-1} A^T (b - A x); a run succeeds when the
 *     recomputed (true) residual also meets the tolerance, otherwise PCG restarts
 *     from the current iterate (an outer step).
 *
 * Build: gcc -std=c11 -O2 -fPIC -shared -ffp-contract=off (FMA contraction must stay
 * off so that every product is rounded exactly once).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------------------
 * Matrix view: dense row-major (leading dimension ld) or CSR with sorted columns.
 * ------------------------------------------------------------------------------------ */
typedef struct {
    int64_t m, n;
    int32_t dense;          /* 1: dense row-major, 0: CSR */
    int64_t ld;             /* dense only */
    const double* vals;     /* dense: m*ld entries; CSR: nnz entries */
    const int64_t* row_ptr; /* CSR only, m+1 entries */
    const int32_t* col_idx; /* CSR only */
} orc_mat;

/* Entries of row i: count, and either a column list (CSR) or NULL (dense 0..n-1). */
static int64_t row_len(const orc_mat* A, int64_t i) {
    return A->dense ? A->n : A->row_ptr[i + 1] - A->row_ptr[i];
}
static const double* row_vals(const orc_mat* A, int64_t i) {
    return A->dense ? A->vals + i * A->ld : A->vals + A->row_ptr[i];
}
static int64_t row_col(const orc_mat* A, int64_t i, int64_t k) {
    return A->dense ? k : (int64_t)A->col_idx[A->row_ptr[i] + k];
}

enum { ORC_OK = 0, ORC_ERR_INVALID = 1, ORC_ERR_NOMEM = 3, ORC_ERR_NOT_CONVERGED = 4,
       ORC_ERR_BREAKDOWN = 5 };

/* ------------------------------------------------------------------------------------
 * Alg. 2 step 2: s = 4 n log n  (natural log, rounded up; C is the leading factor).
 * ------------------------------------------------------------------------------------ */
int64_t orc_sample_size(int64_t n, double C) {
    if (n < 2) return 1;
    return (int64_t)ceil(C * (double)n * log((double)n));
}

/* floor(x * 2^e) for x >= 0 as an unsigned integer (x * 2^e < 2^64 assumed). */
static uint64_t floor_scaled(double x, int e) {
    double y = ldexp(x, e);
    if (y < 1.0) return 0;
    return (uint64_t)y; /* truncation == floor for y >= 0 */
}

/* ------------------------------------------------------------------------------------
 * Alg. 2 step 1 (normalisation), with the column norms taken as exact fixed-point sums.
 *
 *   t_ij = fl(a_ij * a_ij),  T_j = max_i t_ij,  E1_j = 52 - floor(log2 T_j)
 *   c_j  = sum_i floor(t_ij * 2^E1_j)          (exact, 128-bit)
 *   d2_j = RNE(c_j) * 2^-E1_j,   d_j = sqrt(d2_j),   inv_d2_j = fl(1 / d2_j)
 * Each column is quantised relative to its own largest entry, so d_j carries a relative
 * error of at most m 2^-52 whatever the column scaling.  An all-zero column keeps d_j = 1
 * and inv_d2_j = 0 (it carries no sampling weight).  Without normalisation d_j = 1 and
 * inv_d2_j = 2^(E1-52) for every j, with E1 = min_j E1_j (the global largest entry), so
 * the weights below reduce to the raw squared row norms (Eq. R2P on A itself).
 * Returns E1 through *E1_out.  Every non-zero T_j must lie in [2^-900, 2^900].
 * ------------------------------------------------------------------------------------ */
int orc_col_scales(const orc_mat* A, int normalize, double* d2, double* d, double* inv_d2,
                   int32_t* E1_out) {
    int64_t m = A->m, n = A->n;
    double* amax = (double*)calloc((size_t)n, sizeof(double));
    int* E1j = (int*)calloc((size_t)n, sizeof(int));
    u128* c = (u128*)calloc((size_t)n, sizeof(u128));
    if (!amax || !E1j || !c) { free(amax); free(E1j); free(c); return ORC_ERR_NOMEM; }
    for (int64_t i = 0; i < m; ++i) {
        const double* v = row_vals(A, i);
        for (int64_t k = 0; k < row_len(A, i); ++k) {
            double a = fabs(v[k]);
            if (!(a == a) || isinf(a)) { free(amax); free(E1j); free(c); return ORC_ERR_INVALID; }
            int64_t j = row_col(A, i, k);
            if (a > amax[j]) amax[j] = a;
        }
    }
    int E1 = 0, any = 0;
    for (int64_t j = 0; j < n; ++j) {
        if (amax[j] == 0.0) continue;
        double T = amax[j] * amax[j]; /* fl(x^2) is monotone in |x|: this is max_i t_ij */
        if (!(T >= ldexp(1.0, -900) && T <= ldexp(1.0, 900))) { free(amax); free(E1j); free(c); return ORC_ERR_INVALID; }
        E1j[j] = 52 - ilogb(T);
        if (!any || E1j[j] < E1) E1 = E1j[j];
        any = 1;
    }
    if (!any) { free(amax); free(E1j); free(c); return ORC_ERR_INVALID; }
    for (int64_t i = 0; i < m; ++i) {
        const double* v = row_vals(A, i);
        for (int64_t k = 0; k < row_len(A, i); ++k) {
            int64_t j = row_col(A, i, k);
            double t = v[k] * v[k];
            c[j] += (u128)floor_scaled(t, E1j[j]);
        }
    }
    for (int64_t j = 0; j < n; ++j) {
        d2[j] = ldexp((double)c[j], -E1j[j]); /* (double) of a 128-bit integer rounds to nearest even */
        if (!normalize) {
            d[j] = 1.0;
            inv_d2[j] = ldexp(1.0, E1 - 52);
        } else if (c[j] == 0) {
            d[j] = 1.0;
            inv_d2[j] = 0.0;
        } else {
            d[j] = sqrt(d2[j]);
            inv_d2[j] = 1.0 / d2[j];
        }
    }
    free(amax); free(E1j); free(c);
    *E1_out = E1;
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * Eq. (R2P): p_i = ||a_i D^{-1}||^2 / ||A D^{-1}||_F^2, carried as exact integers.
 *
 *   u_ij = fl(t_ij * inv_d2_j)   (= a_ij^2 / d_j^2, one rounding),   u_ij < 2
 *   w_i  = sum_j floor(u_ij * 2^51)   (exact, 128-bit);   p_i = w_i / W,  W = sum_i w_i
 * ------------------------------------------------------------------------------------ */
int orc_row_weights(const orc_mat* A, const double* inv_d2, uint64_t* w_lo, uint64_t* w_hi) {
    for (int64_t i = 0; i < A->m; ++i) {
        const double* v = row_vals(A, i);
        u128 w = 0;
        for (int64_t k = 0; k < row_len(A, i); ++k) {
            double t = v[k] * v[k];
            double u = t * inv_d2[row_col(A, i, k)];
            w += (u128)floor_scaled(u, 51);
        }
        w_lo[i] = (uint64_t)w;
        w_hi[i] = (uint64_t)(w >> 64);
    }
    return ORC_OK;
}

/* Alg. 1 support: exclusive prefix P_0 = 0, P_{i+1} = P_i + w_i, so P_m = W. */
void orc_prefix(int64_t m, const uint64_t* w_lo, const uint64_t* w_hi, uint64_t* P_lo,
                uint64_t* P_hi) {
    u128 acc = 0;
    for (int64_t i = 0; i < m; ++i) {
        P_lo[i] = (uint64_t)acc;
        P_hi[i] = (uint64_t)(acc >> 64);
        acc += ((u128)w_hi[i] << 64) | w_lo[i];
    }
    P_lo[m] = (uint64_t)acc;
    P_hi[m] = (uint64_t)(acc >> 64);
}

/* ------------------------------------------------------------------------------------
 * Philox4x64-10, as published by Salmon, Moraes, Dror and Shaw (SC'11): ten rounds of
 * two 64x64->128 multiplications with the key bumped by the Weyl constants between
 * rounds.
 * ------------------------------------------------------------------------------------ */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        u128 p0 = (u128)M0 * c0;
        u128 p1 = (u128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (r < 9) { k0 += W0; k1 += W1; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* High 128 bits of the 256-bit product a * b. */
static u128 mul_hi128(u128 a, u128 b) {
    uint64_t a0 = (uint64_t)a, a1 = (uint64_t)(a >> 64);
    uint64_t b0 = (uint64_t)b, b1 = (uint64_t)(b >> 64);
    u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1, p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
    u128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10; /* < 3 * 2^64 */
    return p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);
}

/* ------------------------------------------------------------------------------------
 * Alg. 1: draws t = t0 .. t0+count-1 of the i.i.d. sequence.
 *   (r0, r1, r2, r3) = Philox4x64-10(key = (seed, 0x5A4D504C), ctr = (t, 0, 0, 0))
 *   U_t = r1 * 2^64 + r0,   r_t = floor(U_t * W / 2^128) in [0, W)
 *   i_t = max { i : P_i <= r_t }   (a row of zero weight is never chosen)
 * ------------------------------------------------------------------------------------ */
int orc_draw_rows(int64_t m, const uint64_t* P_lo, const uint64_t* P_hi, uint64_t seed,
                  int64_t t0, int64_t count, int32_t* idx) {
    u128 W = ((u128)P_hi[m] << 64) | P_lo[m];
    if (W == 0) return ORC_ERR_INVALID;
    const uint64_t key[2] = {seed, 0x5A4D504Cull};
    for (int64_t k = 0; k < count; ++k) {
        uint64_t ctr[4] = {(uint64_t)(t0 + k), 0, 0, 0}, r[4];
        orc_philox4x64_10(ctr, key, r);
        u128 U = ((u128)r[1] << 64) | r[0];
        u128 target = mul_hi128(U, W);
        int64_t lo = 0, hi = m; /* invariant: P_lo_index <= target < P_hi_index */
        while (hi - lo > 1) {
            int64_t mid = lo + (hi - lo) / 2;
            u128 Pm = ((u128)P_hi[mid] << 64) | P_lo[mid];
            if (Pm <= target) lo = mid; else hi = mid;
        }
        idx[k] = (int32_t)lo;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * Sampled normal matrix (Sec. 3.3):  M = A_s^T A_s = (1/s) sum_{t=1}^{s} (1/p_{i_t})
 * â_{i_t}^T â_{i_t}, â_i = a_i D^{-1}, p_i = w_i / W.  Stored as CSR with sorted columns
 * and an explicit diagonal; a zero or missing diagonal entry is set to 1.
 *
 * Row j is accumulated Gustavson-style: for every draw t (in draw order) whose row has
 * an entry in column j, add (1/(s p_{i_t})) â_{i_t j} â_{i_t k} to M_jk for each entry
 * k of that row.
 * ------------------------------------------------------------------------------------ */
typedef struct {
    int64_t n, nnz, n_fixed_diag;
    int64_t* row_ptr;
    int32_t* col;
    double* val;
} orc_M;

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

void orc_M_free(orc_M* M) {
    if (!M) return;
    free(M->row_ptr); free(M->col); free(M->val); free(M);
}

orc_M* orc_build_M(const orc_mat* A, const double* d, const uint64_t* w_lo,
                   const uint64_t* w_hi, const int32_t* idx, int64_t s) {
    int64_t n = A->n;
    u128 W = 0;
    for (int64_t i = 0; i < A->m; ++i) W += ((u128)w_hi[i] << 64) | w_lo[i];
    double Wd = (double)W;
    /* scale of draw t: 1 / (s p_{i_t}) */
    double* gam = (double*)malloc((size_t)(s > 0 ? s : 1) * sizeof(double));
    /* column lists of the sampled matrix: (draw t, entry position) per column j */
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!gam || !cnt) { free(gam); free(cnt); return NULL; }
    for (int64_t t = 0; t < s; ++t) {
        int64_t i = idx[t];
        double p = (double)(((u128)w_hi[i] << 64) | w_lo[i]) / Wd;
        gam[t] = 1.0 / ((double)s * p);
        for (int64_t k = 0; k < row_len(A, i); ++k) cnt[row_col(A, i, k) + 1]++;
    }
    for (int64_t j = 0; j < n; ++j) cnt[j + 1] += cnt[j];
    int64_t tot = cnt[n];
    int64_t* lst_t = (int64_t*)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int64_t));
    double* lst_v = (double*)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(double));
    int64_t* fill = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    double* acc = (double*)calloc((size_t)n, sizeof(double));
    int32_t* mark = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    int32_t* touched = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    orc_M* M = (orc_M*)calloc(1, sizeof(orc_M));
    if (!lst_t || !lst_v || !fill || !acc || !mark || !touched || !M) goto fail;
    memcpy(fill, cnt, (size_t)n * sizeof(int64_t));
    for (int64_t j = 0; j < n; ++j) mark[j] = -1;
    for (int64_t t = 0; t < s; ++t) {
        int64_t i = idx[t];
        const double* v = row_vals(A, i);
        for (int64_t k = 0; k < row_len(A, i); ++k) {
            int64_t j = row_col(A, i, k);
            lst_t[fill[j]] = t;
            lst_v[fill[j]] = v[k] / d[j];
            fill[j]++;
        }
    }
    /* first pass: row lengths; second pass: values (recomputed, to keep it simple) */
    M->n = n;
    M->row_ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!M->row_ptr) goto fail;
    for (int pass = 0; pass < 2; ++pass) {
        for (int64_t j = 0; j < n; ++j) {
            int64_t nt = 0;
            for (int64_t q = cnt[j]; q < cnt[j + 1]; ++q) {
                int64_t t = lst_t[q];
                int64_t i = idx[t];
                double coef = gam[t] * lst_v[q];
                const double* v = row_vals(A, i);
                for (int64_t k = 0; k < row_len(A, i); ++k) {
                    int64_t c = row_col(A, i, k);
                    if (mark[c] != (int32_t)j) { mark[c] = (int32_t)j; touched[nt++] = (int32_t)c; acc[c] = 0.0; }
                    acc[c] += coef * (v[k] / d[c]);
                }
            }
            if (mark[j] != (int32_t)j) { mark[j] = (int32_t)j; touched[nt++] = (int32_t)j; acc[j] = 0.0; }
            if (pass == 0) {
                M->row_ptr[j + 1] = nt;
            } else {
                qsort(touched, (size_t)nt, sizeof(int32_t), cmp_i32);
                int64_t base = M->row_ptr[j];
                for (int64_t q = 0; q < nt; ++q) {
                    int32_t c = touched[q];
                    double val = acc[c];
                    if (c == j && val == 0.0) { val = 1.0; M->n_fixed_diag++; }
                    M->col[base + q] = c;
                    M->val[base + q] = val;
                }
            }
        }
        for (int64_t j = 0; j < n; ++j) mark[j] = -1;
        if (pass == 0) {
            for (int64_t j = 0; j < n; ++j) M->row_ptr[j + 1] += M->row_ptr[j];
            M->nnz = M->row_ptr[n];
            M->col = (int32_t*)malloc((size_t)(M->nnz > 0 ? M->nnz : 1) * sizeof(int32_t));
            M->val = (double*)malloc((size_t)(M->nnz > 0 ? M->nnz : 1) * sizeof(double));
            if (!M->col || !M->val) goto fail;
        }
    }
    free(gam); free(cnt); free(lst_t); free(lst_v); free(fill); free(acc); free(mark); free(touched);
    return M;
fail:
    free(gam); free(cnt); free(lst_t); free(lst_v); free(fill); free(acc); free(mark); free(touched);
    orc_M_free(M);
    return NULL;
}

int64_t orc_M_nnz(const orc_M* M) { return M->nnz; }
int64_t orc_M_fixed_diag(const orc_M* M) { return M->n_fixed_diag; }
void orc_M_copy(const orc_M* M, int64_t* row_ptr, int32_t* col, double* val) {
    memcpy(row_ptr, M->row_ptr, (size_t)(M->n + 1) * sizeof(int64_t));
    memcpy(col, M->col, (size_t)M->nnz * sizeof(int32_t));
    memcpy(val, M->val, (size_t)M->nnz * sizeof(double));
}

/* Wrap caller-owned CSR arrays as an orc_M (no copy; do not free with orc_M_free). */
void orc_M_view(orc_M* M, int64_t n, int64_t* row_ptr, int32_t* col, double* val) {
    M->n = n; M->row_ptr = row_ptr; M->col = col; M->val = val;
    M->nnz = row_ptr[n]; M->n_fixed_diag = 0;
}

/* ------------------------------------------------------------------------------------
 * Alg. 3: e = 0; t times e <- e + B^{-1}(r - M e), B the lower triangle of M (with the
 * diagonal); then t times e <- e + B^{-T}(r - M e), B^T the upper triangle.
 * ------------------------------------------------------------------------------------ */
static double diag_of(const orc_M* M, int64_t j) {
    for (int64_t q = M->row_ptr[j]; q < M->row_ptr[j + 1]; ++q)
        if (M->col[q] == j) return M->val[q];
    return 1.0;
}

void orc_sgs_apply(const orc_M* M, int t, const double* r, double* e) {
    int64_t n = M->n;
    double* res = (double*)malloc((size_t)n * sizeof(double));
    double* del = (double*)malloc((size_t)n * sizeof(double));
    for (int64_t j = 0; j < n; ++j) e[j] = 0.0;
    for (int dir = 0; dir < 2; ++dir) {
        for (int it = 0; it < t; ++it) {
            for (int64_t j = 0; j < n; ++j) { /* res = r - M e */
                double acc = 0.0;
                for (int64_t q = M->row_ptr[j]; q < M->row_ptr[j + 1]; ++q) acc += M->val[q] * e[M->col[q]];
                res[j] = r[j] - acc;
            }
            if (dir == 0) { /* forward substitution with B (lower triangle) */
                for (int64_t j = 0; j < n; ++j) {
                    double acc = res[j];
                    for (int64_t q = M->row_ptr[j]; q < M->row_ptr[j + 1]; ++q)
                        if (M->col[q] < j) acc -= M->val[q] * del[M->col[q]];
                    del[j] = acc / diag_of(M, j);
                }
            } else {        /* back substitution with B^T (upper triangle) */
                for (int64_t j = n - 1; j >= 0; --j) {
                    double acc = res[j];
                    for (int64_t q = M->row_ptr[j]; q < M->row_ptr[j + 1]; ++q)
                        if (M->col[q] > j) acc -= M->val[q] * del[M->col[q]];
                    del[j] = acc / diag_of(M, j);
                }
            }
            for (int64_t j = 0; j < n; ++j) e[j] += del[j];
        }
    }
    free(res); free(del);
}

/* ------------------------------------------------------------------------------------
 * The two products PCG needs (Sec. 4.2: only A u and A^T v, never A^T A):
 *   q = Â p  (Â = A D^{-1}),  w = Â^T q.
 * ------------------------------------------------------------------------------------ */
void orc_apply_A(const orc_mat* A, const double* d, const double* p, double* q) {
    for (int64_t i = 0; i < A->m; ++i) {
        const double* v = row_vals(A, i);
        double acc = 0.0;
        for (int64_t k = 0; k < row_len(A, i); ++k) {
            int64_t j = row_col(A, i, k);
            acc += (v[k] / d[j]) * p[j];
        }
        q[i] = acc;
    }
}

void orc_apply_AT(const orc_mat* A, const double* d, const double* q, double* w) {
    for (int64_t j = 0; j < A->n; ++j) w[j] = 0.0;
    for (int64_t i = 0; i < A->m; ++i) {
        const double* v = row_vals(A, i);
        for (int64_t k = 0; k < row_len(A, i); ++k) {
            int64_t j = row_col(A, i, k);
            w[j] += (v[k] / d[j]) * q[i];
        }
    }
}

void orc_normal_matvec(const orc_mat* A, const double* d, const double* p, double* w) {
    double* q = (double*)malloc((size_t)A->m * sizeof(double));
    orc_apply_A(A, d, p, q);
    orc_apply_AT(A, d, q, w);
    free(q);
}

static double dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += a[j] * b[j];
    return s;
}

/* z = P g: the SGS operator of Alg. 3 with t sweeps, or, for t = 0, the identity.  t = 0
 * is the paper's comparison method of Sec. 5, CG on the column-normalised matrix
 * (diagonally preconditioned CG); Alg. 3 itself would give the zero operator there. */
static void precond_apply(const orc_M* M, int t, const double* g, double* z) {
    if (t == 0) memcpy(z, g, (size_t)M->n * sizeof(double));
    else orc_sgs_apply(M, t, g, z);
}

/* ------------------------------------------------------------------------------------
 * Alg. 2 step 4: PCG on Â^T Â y = h, with z = P g from orc_sgs_apply (t sweeps; t = 0:
 * P = I, the comparison method of Sec. 5).
 *
 * Least-squares form (b != NULL): h = Â^T b and the true residual is Â^T (b - Â y).
 * Normal-equation form (b == NULL, h given): the true residual is h - Â^T (Â y).
 * Textbook PCG (y0 = 0 or the current iterate on restarts):
 *   g = true residual, z = P g, p = z, rho = g^T z
 *   repeat: w = Â^T Â p, alpha = rho / p^T w, y += alpha p, g -= alpha w
 *           stop if ||g|| <= tol ||h||;  z = P g, rho' = g^T z, p = z + (rho'/rho) p
 * On stop the true residual is recomputed; if it misses the tolerance PCG restarts
 * from y (outer step), up to max_outer steps.  iters counts products Â^T Â p.
 * ------------------------------------------------------------------------------------ */
typedef struct {
    int32_t iters, outer, converged, status;
    double relres_rec, relres_true, hnorm;
} orc_pcg_info;

int orc_pcg(const orc_mat* A, const double* d, const orc_M* M, int sweeps, const double* b,
            const double* h_in, double tol, int maxit, int max_outer, double* y,
            orc_pcg_info* info) {
    int64_t m = A->m, n = A->n;
    double* h = (double*)malloc((size_t)n * sizeof(double));
    double* g = (double*)malloc((size_t)n * sizeof(double));
    double* z = (double*)malloc((size_t)n * sizeof(double));
    double* p = (double*)malloc((size_t)n * sizeof(double));
    double* w = (double*)malloc((size_t)n * sizeof(double));
    double* r = (double*)malloc((size_t)m * sizeof(double));
    memset(info, 0, sizeof(*info));
    if (b) orc_apply_AT(A, d, b, h);
    else memcpy(h, h_in, (size_t)n * sizeof(double));
    double hnorm = sqrt(dot(n, h, h));
    info->hnorm = hnorm;
    for (int64_t j = 0; j < n; ++j) y[j] = 0.0;
    int status = ORC_ERR_NOT_CONVERGED;
    if (hnorm == 0.0) { info->converged = 1; status = ORC_OK; goto done; }
    for (int outer = 0; outer < max_outer; ++outer) {
        /* true residual */
        if (b) {
            orc_apply_A(A, d, y, r);
            for (int64_t i = 0; i < m; ++i) r[i] = b[i] - r[i];
            orc_apply_AT(A, d, r, g);
        } else {
            orc_normal_matvec(A, d, y, w);
            for (int64_t j = 0; j < n; ++j) g[j] = h[j] - w[j];
        }
        double gn = sqrt(dot(n, g, g));
        info->relres_true = gn / hnorm;
        if (outer == 0) info->relres_rec = gn / hnorm;
        if (gn <= tol * hnorm) { info->converged = 1; status = ORC_OK; break; }
        if (info->iters >= maxit) break;
        info->outer = outer + 1; /* PCG (re)starts that ran */
        precond_apply(M, sweeps, g, z);
        for (int64_t j = 0; j < n; ++j) p[j] = z[j];
        double rho = dot(n, g, z);
        while (info->iters < maxit) {
            orc_normal_matvec(A, d, p, w);
            double pw = dot(n, p, w);
            if (!(pw > 0.0) || !(rho > 0.0)) { status = ORC_ERR_BREAKDOWN; goto done; }
            double alpha = rho / pw;
            for (int64_t j = 0; j < n; ++j) { y[j] += alpha * p[j]; g[j] -= alpha * w[j]; }
            info->iters++;
            gn = sqrt(dot(n, g, g));
            info->relres_rec = gn / hnorm;
            if (gn <= tol * hnorm) break;
            precond_apply(M, sweeps, g, z);
            double rho_new = dot(n, g, z);
            double beta = rho_new / rho;
            rho = rho_new;
            for (int64_t j = 0; j < n; ++j) p[j] = z[j] + beta * p[j];
        }
    }
    if (status != ORC_OK && info->converged == 0) {
        /* final true residual after the last outer step */
        if (b) {
            orc_apply_A(A, d, y, r);
            for (int64_t i = 0; i < m; ++i) r[i] = b[i] - r[i];
            orc_apply_AT(A, d, r, g);
        } else {
            orc_normal_matvec(A, d, y, w);
            for (int64_t j = 0; j < n; ++j) g[j] = h[j] - w[j];
        }
        info->relres_true = sqrt(dot(n, g, g)) / hnorm;
        if (info->relres_true <= tol) { info->converged = 1; status = ORC_OK; }
    }
done:
    info->status = status;
    free(h); free(g); free(z); free(p); free(w); free(r);
    return status;
}
