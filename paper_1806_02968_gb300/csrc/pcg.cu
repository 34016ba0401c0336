// C ABI of Alg. 2 step 4 (lsq_pcg_solve), the adjoint solve (lsq_pcg_adjoint) and small
// utilities.  The iteration itself runs in the persistent kernel of pcg_kernel.cuh.
#include "pcg_launch.cuh"
#include "values.cuh"
#include "sparse.cuh"

#include <vector>

namespace lsq {

const char* last_error();

static int64_t pick_nmax(int dt, int dtr, int64_t n) {
    const int64_t lo = 128;
    const int64_t hi = (dt == LSQ_F32 && dtr == LSQ_F32) ? 2048 : 1024;
    for (int64_t c = lo; c <= hi; c *= 2)
        if (n <= c) return c;
    return 0;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

struct SolveWork {
    Scratch sc;
    double *y, *g, *z, *part_w, *part_s, *out_d;
    unsigned *bar, *err;
    int32_t* out_i;
    size_t ctl_bytes;
    lsq_status alloc(int64_t n, cudaStream_t st) {
        const int Gmax = pcg_max_grid();
        size_t off = 0;
        auto take = [&](size_t b) { size_t at = off; off += (b + 255) & ~size_t(255); return at; };
        size_t o_ctl = take(256), o_y = take(8 * n), o_g = take(8 * n), o_z = take(8 * n),
               o_ps = take(8 * (size_t)Gmax * PART_S), o_pw = take(8 * (size_t)Gmax * n);
        LSQ_CUDA(sc.alloc(off, st));
        char* b = sc.as<char>();
        bar = (unsigned*)b; err = bar + 2; out_i = (int32_t*)(b + 16); out_d = (double*)(b + 64);
        ctl_bytes = 256;
        y = (double*)(b + o_y); g = (double*)(b + o_g); z = (double*)(b + o_z);
        part_s = (double*)(b + o_ps); part_w = (double*)(b + o_pw);
        return LSQ_OK;
    }
};

// Validates A/P for the dense PCG kernel and fills the type selection.
static lsq_status check_dense_solve(const lsq_matrix* A, const lsq_precond* P, int* dt, int* dtr,
                                    int64_t* nmax) {
    lsq_status s0 = check_matrix(A);
    if (s0 != LSQ_OK) return s0;
    LSQ_CHECK_ARG(P != nullptr, "preconditioner handle is NULL");
    LSQ_CHECK_ARG(P->n == A->n, "preconditioner was built for a different n");
    if (!A->dense || !P->dense) {
        set_error("sparse PCG is not available in this build");
        return LSQ_ERR_UNSUPPORTED;
    }
    const size_t es = elem_size(A->dtype);
    LSQ_CHECK_ARG(aligned16(A->vals), "A->vals must be 16-byte aligned");
    LSQ_CHECK_ARG(((size_t)A->ld * es) % 16 == 0, "A->ld * element size must be a multiple of 16 bytes");
    LSQ_CHECK_ARG((size_t)A->ld * es * 3 <= (size_t)ring_bytes(2048),
                  "dense PCG needs 3 * ld * element size <= the staging ring");
    if (A->vals_f64 && A->dtype != LSQ_F64) {
        LSQ_CHECK_ARG(aligned16(A->vals_f64), "A->vals_f64 must be 16-byte aligned");
        LSQ_CHECK_ARG((size_t)A->ld * 8 * 3 <= (size_t)ring_bytes(2048),
                      "dense PCG needs 3 * ld * 8 <= the staging ring for the FP64 residual copy");
    }
    *dt = A->dtype;
    *dtr = (A->dtype == LSQ_F64 || A->vals_f64) ? LSQ_F64 : A->dtype;
    *nmax = pick_nmax(*dt, *dtr, A->n);
    if (*nmax == 0) {
        set_error("dense PCG supports n <= 2048 with FP32 values and residuals, n <= 1024 otherwise");
        return LSQ_ERR_UNSUPPORTED;
    }
    return LSQ_OK;
}

// One persistent-kernel solve per column.  h_cols (n-space right-hand sides) selects the
// normal form used by the adjoint.
static lsq_status solve_columns(const lsq_matrix* A, const lsq_precond* P, const double* B,
                                const double* Hcols, int64_t k, int64_t ldb, double* X, int64_t ldx,
                                const lsq_opts* o, lsq_info* info, cudaStream_t st) {
    int dt, dtr;
    int64_t nmax;
    lsq_status s0 = check_dense_solve(A, P, &dt, &dtr, &nmax);
    if (s0 != LSQ_OK) return s0;
    const int64_t m = A->m, n = A->n;
    SolveWork wk;
    s0 = wk.alloc(n, st);
    if (s0 != LSQ_OK) return s0;
    cudaEvent_t e0, e1;
    LSQ_CUDA(cudaEventCreate(&e0));
    LSQ_CUDA(cudaEventCreate(&e1));
    LSQ_CUDA(cudaEventRecord(e0, st));
    lsq_status worst = LSQ_OK;
    for (int64_t c = 0; c < k; ++c) {
        LSQ_CUDA(cudaMemsetAsync(wk.bar, 0, wk.ctl_bytes, st));
        PcgArgs a{};
        a.m = m; a.n = n; a.ld = A->ld;
        a.vals = A->vals;
        a.vals_res = (dtr == LSQ_F64 && A->dtype != LSQ_F64) ? (const void*)A->vals_f64 : A->vals;
        a.inv_d = P->inv_d;
        a.op = P->op;
        a.b = B ? B + c * ldb : nullptr;
        a.h_in = Hcols ? Hcols + c * ldb : nullptr;
        a.x = X + c * ldx;
        a.y = wk.y; a.g = wk.g; a.z = wk.z;
        a.part_w = wk.part_w; a.part_s = wk.part_s;
        a.bar = reinterpret_cast<unsigned long long*>(wk.bar); a.err = wk.err;
        a.tol = o->tol;
        a.inner_tol = o->inner_tol > 0 ? o->inner_tol : 0.0;
        a.maxit = o->maxit; a.max_outer = o->max_outer;
        a.out_i = wk.out_i; a.out_d = wk.out_d;
        a.max_polls = barrier_wait_polls();
        int G = 0;
        lsq_status ls = dt == LSQ_F64 ? launch_pcg_f64(nmax, P->op_dtype, a, o->grid_ctas, st, &G)
                      : dt == LSQ_F32 ? launch_pcg_f32(nmax, dtr, P->op_dtype, a, o->grid_ctas, st, &G)
                      : dt == LSQ_BF16 ? launch_pcg_bf16(nmax, dtr, P->op_dtype, a, o->grid_ctas, st, &G)
                                      : launch_pcg_f32x2(nmax, dtr, P->op_dtype, a, o->grid_ctas, st, &G);
        if (ls != LSQ_OK) return ls;
        LSQ_CUDA(cudaGetLastError());
        int32_t oi[4];
        double od[3];
        unsigned bits = 0;
        LSQ_CUDA(cudaMemcpyAsync(oi, wk.out_i, sizeof(oi), cudaMemcpyDeviceToHost, st));
        LSQ_CUDA(cudaMemcpyAsync(od, wk.out_d, sizeof(od), cudaMemcpyDeviceToHost, st));
        lsq_status es = read_dev_error(wk.err, st, &bits);
        if (es != LSQ_OK) return es;
        if (info && c < info->k) {
            if (info->iters) info->iters[c] = oi[0];
            if (info->outer) info->outer[c] = oi[1];
            if (info->converged) info->converged[c] = (uint8_t)oi[2];
            if (info->relres_rec) info->relres_rec[c] = od[0];
            if (info->relres_true) info->relres_true[c] = od[1];
            if (info->relres_raw) info->relres_raw[c] = od[2];
        }
        lsq_status cs = (lsq_status)oi[3];
        if (cs == LSQ_ERR_BREAKDOWN) worst = LSQ_ERR_BREAKDOWN;
        else if (cs != LSQ_OK && worst == LSQ_OK) worst = LSQ_ERR_NOT_CONVERGED;
    }
    LSQ_CUDA(cudaEventRecord(e1, st));
    LSQ_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) {
        info->s = P->s; info->nnz_M = P->nnz_M; info->n_fixed_diag = P->n_fixed_diag;
        info->levels = P->levels; info->solve_ms = ms;
    }
    if (worst == LSQ_ERR_NOT_CONVERGED) set_error("PCG did not reach the tolerance");
    if (worst == LSQ_ERR_BREAKDOWN) set_error("PCG breakdown (non-positive or non-finite curvature)");
    return worst;
}

// out[c][i] = alpha_b * b[c][i] + alpha_a * (a_i . v[c]) for dense A (FP64 view of values)
template <int DT>
__global__ void k_rowdot(lsq_matrix A, const double* v, int64_t ldv, const double* b, int64_t ldb,
                         double alpha_b, double alpha_a, int64_t kcols, double* out, int64_t ldo) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t rc = warp; rc < A.m * kcols; rc += nw) {
        int64_t c = rc / A.m, i = rc % A.m;
        double acc = 0.0;
        for (int64_t j = lane; j < A.n; j += 32) acc = fma(Val<DT>::load(A.vals, i * A.ld + j), v[c * ldv + j], acc);
        acc = warp_sum(acc);
        if (lane == 0) out[c * ldo + i] = (b ? alpha_b * b[c * ldb + i] : 0.0) + alpha_a * acc;
    }
}

// grad[i][j] = sum_c (r[c][i] lam[c][j] - al[c][i] x[c][j]) on every dense entry
__global__ void k_sddmm_dense(int64_t m, int64_t n, int64_t ld, int64_t kcols, const double* r,
                              const double* al, int64_t ldm, const double* lam, const double* x,
                              int64_t ldn, double* grad) {
    int64_t total = m * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / n, j = e % n;
        double acc = 0.0;
        for (int64_t c = 0; c < kcols; ++c)
            acc += r[c * ldm + i] * lam[c * ldn + j] - al[c * ldm + i] * x[c * ldn + j];
        grad[i * ld + j] = acc;
    }
}

__global__ void k_scale_cols(int64_t n, int64_t kcols, const double* src, int64_t lds,
                             const double* s, double* dst, int64_t ldd) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * kcols;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = e / n, j = e % n;
        dst[c * ldd + j] = src[c * lds + j] * s[j];
    }
}

__global__ void k_split_f64(const double* src, float* dst, int64_t count) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x) {
        double v = src[e];
        float hi = __double2float_rn(v);
        float lo = __double2float_rn(v - (double)hi);
        dst[2 * e] = hi;
        dst[2 * e + 1] = lo;
    }
}

template <int DT>
static lsq_status adjoint_dense(const lsq_matrix* A, const lsq_precond* P, const double* X,
                                const double* B, const double* Gr, int64_t k, int64_t ldb,
                                int64_t ldx, double* grad_b, double* grad_vals, double* Lambda,
                                const lsq_opts* o, lsq_info* info, cudaStream_t st) {
    const int64_t m = A->m, n = A->n;
    Scratch sc;
    // h = D^{-1} G (n x k), lambda (n x k), r, A lambda (m x k)
    size_t bytes = 8 * (size_t)(2 * n * k + 2 * m * k) + 256;
    LSQ_CUDA(sc.alloc(bytes, st));
    double* h = sc.as<double>();
    double* lam = h + n * k;
    double* r = lam + n * k;
    double* al = r + m * k;
    unsigned g1 = (unsigned)std::min<int64_t>((n * k + 255) / 256, 4096);
    k_scale_cols<<<g1, 256, 0, st>>>(n, k, Gr, ldx, P->inv_d, h, n);
    count_launch();
    // A^T A lambda = G  <=>  Â^T Â mu = D^{-1} G with lambda = D^{-1} mu; the kernel's output
    // x = D^{-1} y is therefore lambda itself
    lsq_status s = solve_columns(A, P, nullptr, h, k, n, lam, n, o, info, st);
    if (s != LSQ_OK && s != LSQ_ERR_NOT_CONVERGED) return s;
    unsigned g2 = (unsigned)std::min<int64_t>((m * k * 32 + 255) / 256, 152 * 16);
    k_rowdot<DT><<<g2, 256, 0, st>>>(*A, lam, n, nullptr, 0, 0.0, 1.0, k, al, m);
    k_rowdot<DT><<<g2, 256, 0, st>>>(*A, X, ldx, B, ldb, 1.0, -1.0, k, r, m);
    count_launch(2);
    if (grad_b) {
        for (int64_t c = 0; c < k; ++c)
            LSQ_CUDA(cudaMemcpyAsync(grad_b + c * ldb, al + c * m, 8 * m, cudaMemcpyDeviceToDevice, st));
    }
    if (grad_vals) {
        unsigned g3 = (unsigned)std::min<int64_t>((m * n + 255) / 256, 152 * 32);
        k_sddmm_dense<<<g3, 256, 0, st>>>(m, n, A->ld, k, r, al, m, lam, X, ldx, grad_vals);
        count_launch();
    }
    if (Lambda) {
        for (int64_t c = 0; c < k; ++c)
            LSQ_CUDA(cudaMemcpyAsync(Lambda + c * ldx, lam + c * n, 8 * n, cudaMemcpyDeviceToDevice, st));
    }
    LSQ_CUDA(cudaGetLastError());
    LSQ_CUDA(cudaStreamSynchronize(st));
    return s;
}

}  // namespace lsq

using namespace lsq;

extern "C" lsq_status lsq_pcg_solve(const lsq_matrix* A, const lsq_precond* P, const double* B,
                                    int64_t k, int64_t ldb, double* X, int64_t ldx,
                                    const lsq_opts* o, lsq_info* info, void* stream) {
    LSQ_CHECK_ARG(A && P && B && X && o, "NULL argument");
    LSQ_CHECK_ARG(k >= 1, "k must be >= 1");
    LSQ_CHECK_ARG(ldb >= A->m && ldx >= A->n, "ldb >= m and ldx >= n required");
    LSQ_CHECK_ARG(o->tol > 0 && o->maxit >= 0 && o->max_outer >= 1, "bad tolerance or caps");
    LSQ_CHECK_ARG(o->device_loop == 0 || o->device_loop == 1, "device_loop must be 0 or 1");
    if (!A->dense) {
        lsq_status s0 = check_matrix(A);
        if (s0 != LSQ_OK) return s0;
        return sparse_solve(A, P, B, nullptr, k, ldb, X, ldx, o, info, (cudaStream_t)stream);
    }
    return solve_columns(A, P, B, nullptr, k, ldb, X, ldx, o, info, (cudaStream_t)stream);
}

extern "C" lsq_status lsq_pcg_adjoint(const lsq_matrix* A, const lsq_precond* P, const double* X,
                                      const double* B, const double* G, int64_t k, int64_t ldb,
                                      int64_t ldx, double* grad_b, double* grad_vals,
                                      double* Lambda, const lsq_opts* o, lsq_info* info,
                                      void* stream) {
    LSQ_CHECK_ARG(A && P && X && B && G && o, "NULL argument");
    LSQ_CHECK_ARG(k >= 1, "k must be >= 1");
    LSQ_CHECK_ARG(ldb >= A->m && ldx >= A->n, "ldb >= m and ldx >= n required");
    if (!A->dense) {
        lsq_status s1 = check_matrix(A);
        if (s1 != LSQ_OK) return s1;
        return sparse_adjoint(A, P, X, B, G, k, ldb, ldx, grad_b, grad_vals, Lambda, o, info, (cudaStream_t)stream);
    }
    int dt, dtr;
    int64_t nmax;
    lsq_status s0 = check_dense_solve(A, P, &dt, &dtr, &nmax);
    if (s0 != LSQ_OK) return s0;
    cudaStream_t st = (cudaStream_t)stream;
    if (A->dtype == LSQ_F64)
        return adjoint_dense<LSQ_F64>(A, P, X, B, G, k, ldb, ldx, grad_b, grad_vals, Lambda, o, info, st);
    if (A->dtype == LSQ_F32X2)
        return adjoint_dense<LSQ_F32X2>(A, P, X, B, G, k, ldb, ldx, grad_b, grad_vals, Lambda, o, info, st);
    if (A->dtype == LSQ_BF16)
        return adjoint_dense<LSQ_BF16>(A, P, X, B, G, k, ldb, ldx, grad_b, grad_vals, Lambda, o, info, st);
    return adjoint_dense<LSQ_F32>(A, P, X, B, G, k, ldb, ldx, grad_b, grad_vals, Lambda, o, info, st);
}

extern "C" lsq_status lsq_split_f64(const double* src, float* dst_pairs, int64_t count, void* stream) {
    LSQ_CHECK_ARG(src && dst_pairs && count >= 0, "bad argument");
    if (count == 0) return LSQ_OK;
    cudaStream_t st = (cudaStream_t)stream;
    k_split_f64<<<(unsigned)std::min<int64_t>((count + 255) / 256, 152 * 32), 256, 0, st>>>(src, dst_pairs, count);
    count_launch();
    LSQ_CUDA(cudaGetLastError());
    LSQ_CUDA(cudaStreamSynchronize(st));
    return LSQ_OK;
}

extern "C" const char* lsq_status_string(lsq_status s) {
    switch (s) {
        case LSQ_OK: return "ok";
        case LSQ_ERR_INVALID: return "invalid argument";
        case LSQ_ERR_CUDA: return "CUDA error";
        case LSQ_ERR_NOMEM: return "out of device memory";
        case LSQ_ERR_NOT_CONVERGED: return "not converged";
        case LSQ_ERR_BREAKDOWN: return "PCG breakdown";
        case LSQ_ERR_TIMEOUT: return "device wait timed out";
        case LSQ_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

extern "C" const char* lsq_last_error_string(void) { return last_error(); }

extern "C" int64_t lsq_kernel_launch_count(void) { return g_launches.load(); }
