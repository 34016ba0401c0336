// Sec. 3.3 (sampled normal matrix) and Alg. 3 (symmetric Gauss-Seidel preconditioner).
//
// Dense path: M = A_s^T A_s is assembled by a split-K tiled product over the draws
// (deterministic: partial tiles are summed in a fixed order), made exactly symmetric, and
// its zero diagonal entries are replaced by 1.  The SGS operator of Alg. 3 is then
// materialised: column j of the operator is the result of running the t forward and t
// backward Gauss-Seidel sweeps, in the natural row order, on the unit vector e_j from a
// zero start.  Inside PCG the preconditioner is one parallel matrix-vector product with
// that operator instead of a 2n-step dependency chain per application.
#include "common.cuh"
#include "values.cuh"
#include "sparse.cuh"

namespace lsq {

constexpr int MT = 64;   // M tile edge
constexpr int MK = 16;   // draws per smem stage

__global__ void k_gamma(const double* p, int64_t s, double* gam) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < s;
         t += (int64_t)gridDim.x * blockDim.x)
        gam[t] = __drcp_rn(__dmul_rn((double)s, p[t]));  // 1 / (s p_{i_t})
}

// part[z][j][k] = sum over draws t in split z of gam_t â_{i_t j} â_{i_t k}, for the tile
// pair (blockIdx.x = j tile, blockIdx.y = k tile), k tile >= j tile.
template <int DT>
__global__ void __launch_bounds__(256) k_build_M_dense(lsq_matrix A, const int32_t* idx,
                                                      const double* gam, const double* inv_d,
                                                      int64_t s, int64_t per_split, double* part) {
    if (blockIdx.y < blockIdx.x) return;
    const int64_t n = A.n;
    const int64_t j0 = (int64_t)blockIdx.x * MT, k0 = (int64_t)blockIdx.y * MT;
    const int64_t t_begin = (int64_t)blockIdx.z * per_split;
    const int64_t t_end = min(s, t_begin + per_split);
    __shared__ double Xj[MK][MT], Xk[MK][MT];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int64_t t0 = t_begin; t0 < t_end; t0 += MK) {
        for (int e = threadIdx.x; e < MK * MT; e += 256) {
            int tt = e / MT, c = e % MT;
            int64_t t = t0 + tt;
            double vj = 0.0, vk = 0.0;
            if (t < t_end) {
                int64_t row = (int64_t)idx[t] * A.ld;
                if (j0 + c < n) vj = __dmul_rn(__dmul_rn(Val<DT>::load(A.vals, row + j0 + c), inv_d[j0 + c]), gam[t]);
                if (k0 + c < n) vk = __dmul_rn(Val<DT>::load(A.vals, row + k0 + c), inv_d[k0 + c]);
            }
            Xj[tt][c] = vj;
            Xk[tt][c] = vk;
        }
        __syncthreads();
#pragma unroll
        for (int tt = 0; tt < MK; ++tt) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) { a[r] = Xj[tt][ty * 4 + r]; b[r] = Xk[tt][tx * 4 + r]; }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = fma(a[r], b[q], acc[r][q]);
        }
        __syncthreads();
    }
    double* out = part + (int64_t)blockIdx.z * n * n;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int64_t j = j0 + ty * 4 + r;
        if (j >= n) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int64_t k = k0 + tx * 4 + q;
            if (k < n) out[j * n + k] = acc[r][q];
        }
    }
}

// M[j][k] = M[k][j] = sum_z part[z][j][k] for j <= k (fixed order); zero diagonal -> 1.
__global__ void k_reduce_M(int64_t n, int splits, const double* part, double* M,
                           unsigned long long* n_fixed) {
    int64_t total = n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = e / n, k = e % n;
        if (k < j) continue;
        double v = 0.0;
        for (int z = 0; z < splits; ++z) v += part[(int64_t)z * total + e];
        if (j == k && v == 0.0) { v = 1.0; atomicAdd(n_fixed, 1ull); }
        M[j * n + k] = v;
        M[k * n + j] = v;
    }
}

// The identity operator (t = 0: CG on the column-normalised system, the paper's comparison
// method in Sec. 5)
template <typename OT>
__global__ void k_identity_op(int64_t n, OT* op) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += (int64_t)gridDim.x * blockDim.x)
        op[t] = (t / n == t % n) ? OT(1) : OT(0);
}

// Column j of the SGS operator: Alg. 3 on r = e_j from e = 0, t forward sweeps (rows
// 0..n-1) then t backward sweeps (rows n-1..0), each the in-place Gauss-Seidel update
// e_k <- (r_k - sum_{l != k} M_kl e_l) / M_kk (equal to e <- e + B^{-1}(r - M e) forward
// and e <- e + B^{-T}(r - M e) backward).  One warp per column; e lives in shared memory.
template <typename OT>
__global__ void k_sgs_materialize(int64_t n, int sweeps, const double* M, OT* op) {
    extern __shared__ double s_e[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
    if (j >= n) return;
    double* e = s_e + (int64_t)wid * n;
    for (int64_t l = lane; l < n; l += 32) e[l] = 0.0;
    __syncwarp();
    for (int sw = 0; sw < 2 * sweeps; ++sw) {
        const bool fwd = sw < sweeps;
        for (int64_t kk = 0; kk < n; ++kk) {
            const int64_t k = fwd ? kk : n - 1 - kk;
            int64_t lo = 0, hi = n;
            if (sw == 0) {  // first forward sweep from zero: only rows >= j move, and only
                if (k < j) continue;  // already-updated entries l in [j, k) contribute
                lo = j; hi = k;
            }
            const double* Mk = M + k * n;
            double part = 0.0;
            for (int64_t l = lo + lane; l < hi; l += 32)
                if (l != k) part = fma(Mk[l], e[l], part);
            double ssum = warp_sum(part);
            if (lane == 0) e[k] = ((k == j ? 1.0 : 0.0) - ssum) / Mk[k];
            __syncwarp();
        }
    }
    for (int64_t k = lane; k < n; k += 32) op[k * n + j] = (OT)e[k];
}

template <typename OT>
__global__ void k_op_apply(int64_t n, int64_t kcols, const OT* op, const double* r, double* z) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t rowc = warp; rowc < n * kcols; rowc += nw) {
        int64_t c = rowc / n, row = rowc % n;
        const OT* P = op + row * n;
        const double* rc = r + c * n;
        double acc = 0.0;
        for (int64_t l = lane; l < n; l += 32) acc = fma((double)P[l], rc[l], acc);
        acc = warp_sum(acc);
        if (lane == 0) z[c * n + row] = acc;
    }
}

__global__ void k_inv(int64_t n, const double* d, double* dst_d, double* inv_d) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        double v = d[j];
        dst_d[j] = v;
        inv_d[j] = 1.0 / v;
    }
}

__global__ void k_op_to_f64(int64_t count, const float* src, double* dst) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = (double)src[e];
}

template <int DT>
static lsq_status build_dense(const lsq_matrix* A, const int32_t* idx, const double* p,
                              int64_t s, lsq_precond* H, cudaStream_t st) {
    const int64_t n = A->n;
    const int64_t ntj = (n + MT - 1) / MT;
    const int64_t active = ntj * (ntj + 1) / 2;
    int64_t splits = (4 * 152 + active - 1) / active;
    int64_t max_splits = (s + 63) / 64;
    if (splits > max_splits) splits = max_splits;
    if (splits < 1) splits = 1;
    if (splits > 64) splits = 64;
    int64_t per_split = (s + splits - 1) / splits;
    per_split = (per_split + MK - 1) / MK * MK;
    splits = (s + per_split - 1) / per_split;

    Scratch sc;
    size_t bytes = 256 + 8 * (size_t)s + 8 * (size_t)splits * n * n;
    LSQ_CUDA(sc.alloc(bytes, st));
    unsigned long long* n_fixed = sc.as<unsigned long long>();
    double* gam = (double*)(sc.as<char>() + 256);
    double* part = gam + s;
    LSQ_CUDA(cudaMemsetAsync(n_fixed, 0, 16, st));

    k_gamma<<<(unsigned)std::min<int64_t>((s + 255) / 256, 4096), 256, 0, st>>>(p, s, gam);
    dim3 grid((unsigned)ntj, (unsigned)ntj, (unsigned)splits);
    k_build_M_dense<DT><<<grid, 256, 0, st>>>(*A, idx, gam, H->inv_d, s, per_split, part);
    k_reduce_M<<<(unsigned)std::min<int64_t>((n * n + 255) / 256, 152 * 16), 256, 0, st>>>(
        n, (int)splits, part, H->M, n_fixed);
    count_launch(3);
    const int wpb = 4;
    size_t smem = (size_t)wpb * n * sizeof(double);
    unsigned g = (unsigned)((n + wpb - 1) / wpb);
    if (H->sweeps == 0) {   // the comparison method: P = I on the normalised system
        const unsigned gi = (unsigned)std::min<int64_t>((n * n + 255) / 256, 152 * 16);
        if (H->op_dtype == LSQ_F32) k_identity_op<float><<<gi, 256, 0, st>>>(n, (float*)H->op);
        else k_identity_op<double><<<gi, 256, 0, st>>>(n, (double*)H->op);
    } else if (H->op_dtype == LSQ_F32) {
        if (smem > 48 * 1024)
            LSQ_CUDA(cudaFuncSetAttribute(k_sgs_materialize<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_sgs_materialize<float><<<g, 32 * wpb, smem, st>>>(n, H->sweeps, H->M, (float*)H->op);
    } else {
        if (smem > 48 * 1024)
            LSQ_CUDA(cudaFuncSetAttribute(k_sgs_materialize<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_sgs_materialize<double><<<g, 32 * wpb, smem, st>>>(n, H->sweeps, H->M, (double*)H->op);
    }
    count_launch();
    LSQ_CUDA(cudaGetLastError());
    unsigned long long nf = 0;
    LSQ_CUDA(cudaMemcpyAsync(&nf, n_fixed, 8, cudaMemcpyDeviceToHost, st));
    LSQ_CUDA(cudaStreamSynchronize(st));
    H->n_fixed_diag = (int64_t)nf;
    H->nnz_M = n * n;
    H->levels = n;
    return LSQ_OK;
}

static void free_handle(lsq_precond* H) {
    if (!H) return;
    if (H->M) cudaFree(H->M);
    if (H->op) cudaFree(H->op);
    if (H->colscale) cudaFree(H->colscale);
    if (H->inv_d) cudaFree(H->inv_d);
    if (H->sp) free_sparse(H->sp);
    delete H;
}

}  // namespace lsq

using namespace lsq;

extern "C" lsq_status lsq_build_precond(const lsq_matrix* A, const int32_t* idx, const double* p,
                                        const double* colscale, int64_t s, const lsq_opts* o,
                                        lsq_precond** P_out, void* stream) {
    lsq_status st0 = check_matrix(A);
    if (st0 != LSQ_OK) return st0;
    LSQ_CHECK_ARG(o && P_out && idx && p && colscale, "NULL argument");
    LSQ_CHECK_ARG(s > 0, "s must be positive");
    LSQ_CHECK_ARG(o->sweeps >= 0 && o->sweeps <= 64, "sweeps must be in [0, 64]");
    LSQ_CHECK_ARG(o->precond_dtype == LSQ_F64 || o->precond_dtype == LSQ_F32, "precond_dtype must be F64 or F32");
    *P_out = nullptr;
    if (A->dense) LSQ_CHECK_ARG(A->n <= 2048, "dense path supports n <= 2048");
    else LSQ_CHECK_ARG(o->sweeps <= 32, "sparse preconditioners support sweeps <= 32");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = A->n;
    lsq_precond* H = new lsq_precond();
    H->n = n; H->s = s; H->dense = A->dense ? 1 : 0; H->sweeps = o->sweeps; H->op_dtype = o->precond_dtype;
    H->stream = st;
    auto fail = [&](lsq_status code) { free_handle(H); return code; };
    cudaError_t e;
    if ((e = cudaMalloc(&H->colscale, sizeof(double) * n)) != cudaSuccess ||
        (e = cudaMalloc(&H->inv_d, sizeof(double) * n)) != cudaSuccess) {
        set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return fail(LSQ_ERR_NOMEM);
    }
    k_inv<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, colscale, H->colscale, H->inv_d);
    count_launch();
    if (!A->dense) {
        lsq_status rs = build_sparse(A, idx, p, s, H, st);
        if (rs != LSQ_OK) return fail(rs);
        *P_out = H;
        return LSQ_OK;
    }
    if ((e = cudaMalloc(&H->M, sizeof(double) * n * n)) != cudaSuccess ||
        (e = cudaMalloc(&H->op, elem_size(o->precond_dtype) * n * n)) != cudaSuccess) {
        set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return fail(LSQ_ERR_NOMEM);
    }
    lsq_status r;
    switch (A->dtype) {
        case LSQ_F64: r = build_dense<LSQ_F64>(A, idx, p, s, H, st); break;
        case LSQ_F32: r = build_dense<LSQ_F32>(A, idx, p, s, H, st); break;
        case LSQ_BF16: r = build_dense<LSQ_BF16>(A, idx, p, s, H, st); break;
        default: r = build_dense<LSQ_F32X2>(A, idx, p, s, H, st); break;
    }
    if (r != LSQ_OK) return fail(r);
    *P_out = H;
    return LSQ_OK;
}

extern "C" void lsq_precond_destroy(lsq_precond* P) { free_handle(P); }

extern "C" lsq_status lsq_precond_get_M(const lsq_precond* P, double* M_out, void* stream) {
    LSQ_CHECK_ARG(P && M_out, "NULL argument");
    LSQ_CHECK_ARG(P->dense, "only dense handles hold a dense M");
    LSQ_CUDA(cudaMemcpyAsync(M_out, P->M, sizeof(double) * P->n * P->n, cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
    LSQ_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return LSQ_OK;
}

extern "C" lsq_status lsq_precond_get_op(const lsq_precond* P, double* op_out, void* stream) {
    LSQ_CHECK_ARG(P && op_out, "NULL argument");
    LSQ_CHECK_ARG(P->dense, "only dense handles hold a materialised operator");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t cnt = P->n * P->n;
    if (P->op_dtype == LSQ_F64) {
        LSQ_CUDA(cudaMemcpyAsync(op_out, P->op, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, st));
    } else {
        k_op_to_f64<<<(unsigned)std::min<int64_t>((cnt + 255) / 256, 4096), 256, 0, st>>>(cnt, (const float*)P->op, op_out);
        count_launch();
    }
    LSQ_CUDA(cudaGetLastError());
    LSQ_CUDA(cudaStreamSynchronize(st));
    return LSQ_OK;
}

extern "C" lsq_status lsq_precond_get_M_csr(const lsq_precond* P, int64_t* nnz_out, int64_t* row_ptr,
                                            int32_t* col_idx, double* vals, void* stream) {
    LSQ_CHECK_ARG(P && nnz_out, "NULL argument");
    LSQ_CHECK_ARG(!P->dense && P->sp, "only sparse handles hold a CSR M");
    *nnz_out = P->sp->nnz_M;
    cudaStream_t st = (cudaStream_t)stream;
    if (row_ptr) LSQ_CUDA(cudaMemcpyAsync(row_ptr, P->sp->mptr, 8 * (size_t)(P->n + 1), cudaMemcpyDeviceToDevice, st));
    if (col_idx) LSQ_CUDA(cudaMemcpyAsync(col_idx, P->sp->mcol, 4 * (size_t)P->sp->nnz_M, cudaMemcpyDeviceToDevice, st));
    if (vals) LSQ_CUDA(cudaMemcpyAsync(vals, P->sp->mval, 8 * (size_t)P->sp->nnz_M, cudaMemcpyDeviceToDevice, st));
    LSQ_CUDA(cudaStreamSynchronize(st));
    return LSQ_OK;
}

extern "C" lsq_status lsq_precond_apply(const lsq_precond* P, const double* r, double* e,
                                        int64_t k, void* stream) {
    LSQ_CHECK_ARG(P && r && e && k >= 1, "bad argument");
    if (!P->dense) return sparse_apply(P, r, e, k, (cudaStream_t)stream);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned g = (unsigned)std::min<int64_t>((P->n * k * 32 + 255) / 256, 152 * 8);
    if (P->op_dtype == LSQ_F64) k_op_apply<double><<<g, 256, 0, st>>>(P->n, k, (const double*)P->op, r, e);
    else k_op_apply<float><<<g, 256, 0, st>>>(P->n, k, (const float*)P->op, r, e);
    count_launch();
    LSQ_CUDA(cudaGetLastError());
    LSQ_CUDA(cudaStreamSynchronize(st));
    return LSQ_OK;
}
