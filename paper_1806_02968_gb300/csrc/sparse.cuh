// Sparse (CSR) preconditioner data shared by sparse_build.cu and pcg_sparse.cu.
#pragma once
#include "common.cuh"

namespace lsq {

struct SparseHandle {
    int64_t m = 0, nnz_A = 0, nnz_M = 0, n_unique = 0;
    // M = A_s^T A_s in CSR (sorted columns, diagonal always stored)
    int64_t* mptr = nullptr;
    int32_t* mcol = nullptr;
    double* mval = nullptr;
    float* mval32 = nullptr;    // FP32 copy when the operator dtype is F32
    double* dinv = nullptr;     // 1 / M_jj
    int64_t* mdiag = nullptr;   // position of M_jj in row j (rows are sorted, the diagonal is stored)
    // rows listed by forward / backward level (Gauss-Seidel dependency order)
    int32_t* sched_f = nullptr;
    int32_t* sched_b = nullptr;
    int64_t nlev_f = 0, nlev_b = 0;
    int64_t* loff_f = nullptr;    // first schedule slot of every level (nlev + 1 entries)
    int64_t* loff_b = nullptr;
    // transposed pattern of A: column pointers, row indices, source entry of each
    int64_t* atptr = nullptr;
    int32_t* atrow = nullptr;
    int64_t* atperm = nullptr;
};

lsq_status scan_i64(const int64_t* in, int64_t n, int64_t* out, int64_t* scratch, cudaStream_t st);
lsq_status transpose_pattern(const int64_t* rptr, const int32_t* col, int64_t nr, int64_t nc, int64_t nnz,
                             int64_t* cptr, int32_t* trow, int64_t* tperm, cudaStream_t st);
lsq_status build_sparse(const lsq_matrix* A, const int32_t* idx, const double* p, int64_t s,
                        lsq_precond* H, cudaStream_t st);
void free_sparse(SparseHandle* S);
// The sweep form set by lsq_set_sweep_form (0 by shape, 1 grid, 2 one CTA, 3 one cluster).
int sweep_form_setting();
// Blocks of a grid-form sweep: enough that every row of an average level has its own warp
// (units_per_block rows per block at a time) twice over, at least one block per SM (152) and
// at most the resident maximum.  Waiting warps poll their dependencies; fewer of them leave
// L2 to the writes that end the waits (4e6 x 40,000, 1583 levels of ~25 rows: 5.18 ms per
// sweep on 152 blocks against 5.81 ms on all 456 resident ones; 76 or 38 blocks: no better).
inline int sweep_grid(int resident, int64_t n, int64_t nlev, int units_per_block) {
    const double per_level = nlev > 0 ? (double)n / (double)nlev : (double)n;
    int64_t want = (int64_t)(2.0 * per_level / (double)units_per_block) + 1;
    if (want < 152) want = 152;
    return want < resident ? (int)want : resident;
}
lsq_status sparse_solve(const lsq_matrix* A, const lsq_precond* P, const double* B, const double* Hcols,
                        int64_t k, int64_t ldb, double* X, int64_t ldx, const lsq_opts* o, lsq_info* info,
                        cudaStream_t st);
// k >= 2 right-hand sides: blocks of up to 32 columns advanced together (pcg_sparse_block.cu)
lsq_status sparse_block_solve(const lsq_matrix* A, const lsq_precond* P, const double* B, const double* Hcols,
                              int64_t k, int64_t ldb, double* X, int64_t ldx, const lsq_opts* o, lsq_info* info,
                              cudaStream_t st);
lsq_status sparse_apply(const lsq_precond* P, const double* r, double* e, int64_t k, cudaStream_t st);
lsq_status sparse_adjoint(const lsq_matrix* A, const lsq_precond* P, const double* X, const double* B,
                          const double* G, int64_t k, int64_t ldb, int64_t ldx, double* grad_b,
                          double* grad_vals, double* Lambda, const lsq_opts* o, lsq_info* info, cudaStream_t st);

}  // namespace lsq
