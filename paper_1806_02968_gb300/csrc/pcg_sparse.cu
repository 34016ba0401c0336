// Alg. 2 step 4 for CSR matrices: PCG on Â^T Â y = Â^T b with the Gauss-Seidel sweeps of
// Alg. 3 on the sparse A_s^T A_s.
//
// Per iteration (one stream, no host synchronisation inside a batch of iterations):
//   k_sp_rows   q = Â p over the rows of A (CSR), partials of ||q||^2 = p^T w
//   k_sp_cols   w = Â^T q over the columns (the cached transposed pattern; no atomics)
//   k_sp_update alpha = rho / p^T w, y += alpha p, g -= alpha w, partials of ||g||^2
//   k_sp_sweep  forward then backward Gauss-Seidel sweep (the first checks convergence)
//   k_sp_pnext  rho' = g^T z, beta, p = z + beta p
// The sweeps keep the natural row order of Alg. 3: each row waits for the rows it depends
// on (its lower, resp. upper, entries).  Warps take rows in level order from a ticket
// counter, so a row's dependencies are always held by running or finished warps; the
// waits on the per-row completion flags are bounded.  A device flag ends the remaining
// kernels of a batch once PCG has converged.
#include "sparse.cuh"
#include "values.cuh"

#include <algorithm>

namespace lsq {

struct SpState {
    double rho, hn, gstart, rec;
    int32_t iters, done, status, napply;   // napply: preconditioner applications so far
    unsigned err, pad, r0, r1;
    unsigned ticket[64];                   // one row counter per sweep of an application
};

struct SpArgs {
    int64_t m, n;
    const int64_t* row_ptr;   // A (CSR)
    const int32_t* col_idx;
    const void* vals;         // values of the iteration (dtype DT)
    const void* vals_res;     // values of h and the true residuals (DTR)
    const int64_t* atptr;     // A^T pattern
    const int32_t* atrow;
    const void* valsT;        // A^T values (DT), gathered
    const void* valsT_res;    // A^T values (DTR), gathered
    const double* inv_d;
    const double* b;
    const double* h_in;       // normal form right-hand side, or NULL
    // M
    const int64_t* mptr;
    const int32_t* mcol;
    const void* mval;         // double or float (op dtype)
    const double* dinv;
    const int32_t* sched_f;
    const int32_t* sched_b;
    int sweeps;
    // vectors
    double *y, *g, *z, *p, *pt, *w, *q, *e0, *e1, *h;
    unsigned *flag_f, *flag_b;
    double* part;             // per-block partials
    int nblk;                 // blocks of the reduction kernels
    SpState* S;
    double tol, inner_tol;
    int32_t maxit;
};

__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < nw; ++w) t += sh[w];
        sh[32] = t;
    }
    __syncthreads();
    t = sh[32];
    __syncthreads();
    return t;
}
// sum of part[0..cnt) in a fixed order, every caller gets the same bits
__device__ __forceinline__ double sum_parts(const double* part, int cnt, double* sh) {
    double t = 0.0;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) t += part[i];
    return block_sum(t, sh);
}

constexpr int SP_T = 256;
enum { SPM_MATVEC = 0, SPM_RHS = 1, SPM_RESID = 2 };

// q_i = sum_e a_e x_{col e} (x = D^{-1} p or D^{-1} y), or b_i, or b_i - that; 8 lanes per row
template <int DT>
__global__ void __launch_bounds__(SP_T) k_sp_rows(SpArgs a, int mode, int use_res, const double* x) {
    __shared__ double sh[40];
    if (a.S->done) return;
    const void* vals = use_res ? a.vals_res : a.vals;
    const int sub = threadIdx.x & 7;
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) >> 3;
    double qq = 0.0;
    for (int64_t i0 = 0; i0 < a.m; i0 += ngrp) {
        const int64_t i = i0 + grp;
        double dot = 0.0;
        if (i < a.m && mode != SPM_RHS) {
            for (int64_t e = a.row_ptr[i] + sub; e < a.row_ptr[i + 1]; e += 8) {
                const double v = Val<DT>::load(vals, e);
                dot = fma(v, x[a.col_idx[e]], dot);
            }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if (i < a.m && sub == 0) {
            const double q = mode == SPM_MATVEC ? dot : (mode == SPM_RHS ? a.b[i] : a.b[i] - dot);
            a.q[i] = q;
            qq = fma(q, q, qq);
        }
    }
    const double t = block_sum(qq, sh);
    if (threadIdx.x == 0) a.part[blockIdx.x] = t;
}

// w_j = (1/d_j) sum_{i in column j} a_ij q_i, one warp per column (fixed order)
template <int DT>
__global__ void __launch_bounds__(SP_T) k_sp_cols(SpArgs a, int use_res, double* out) {
    if (a.S->done) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const void* vals = use_res ? a.valsT_res : a.valsT;
    for (int64_t j = warp; j < a.n; j += nw) {
        double t = 0.0;
        for (int64_t e = a.atptr[j] + lane; e < a.atptr[j + 1]; e += 32) {
            const double v = Val<DT>::load(vals, e);
            t = fma(v, a.q[a.atrow[e]], t);
        }
        t = warp_sum(t);
        if (lane == 0) out[j] = t * a.inv_d[j];
    }
}

// alpha = rho / p^T w, y += alpha p, g -= alpha w; partial ||g||^2; resets the sweep tickets
__global__ void __launch_bounds__(SP_T) k_sp_update(SpArgs a, int nparts) {
    __shared__ double sh[40];
    if (a.S->done) return;
    const double pw = sum_parts(a.part, nparts, sh);
    const double rho = a.S->rho;
    if (!(pw > 0.0) || !(rho > 0.0) || !isfinite(pw) || !isfinite(rho)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) { a.S->status = LSQ_ERR_BREAKDOWN; a.S->done = 1; }
        return;
    }
    const double alpha = rho / pw;
    double gg = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += (int64_t)gridDim.x * blockDim.x) {
        a.y[j] = fma(alpha, a.p[j], a.y[j]);
        const double gj = fma(-alpha, a.w[j], a.g[j]);
        a.g[j] = gj;
        gg = fma(gj, gj, gg);
    }
    const double t = block_sum(gg, sh);
    if (threadIdx.x == 0) a.part[a.nblk + blockIdx.x] = t;
}

__device__ __forceinline__ unsigned ld_acquire_flag(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_flag(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One Gauss-Seidel sweep of Alg. 3 on M (FWD: rows in natural order, lower entries are
// the dependencies; otherwise reverse order, upper entries):
//   e_new_j = (r_j - sum_{other side} M_jk e_old_k - sum_{dependency side} M_jk e_new_k) / M_jj
// With `identity` (the backward sweep right after a single forward sweep from zero,
// t = 1): r - L e_old = D e_old, so e_new_j = e_old_j - (sum_{k>j} M_jk e_new_k) / M_jj.
// `check` (first sweep of an iteration): reduce ||g||^2 first and stop when converged.
template <typename MT, bool FWD>
__global__ void __launch_bounds__(SP_T) k_sp_sweep(SpArgs a, const double* r, const double* e_old,
                                                   double* e_new, int identity, int check, int nparts,
                                                   int sweep_idx) {
    __shared__ double sh[40];
    __shared__ int s_stop;
    if (a.S->done) return;
    if (check) {
        const double gg = sum_parts(a.part + a.nblk, nparts, sh);
        if (threadIdx.x == 0) {
            const double gn = sqrt(gg);
            int stop = 0;
            if (gn <= a.tol * a.S->hn || gn <= a.inner_tol * a.S->gstart) stop = 1;
            if (a.S->iters >= a.maxit) stop = 1;
            s_stop = stop;
            if (blockIdx.x == 0) a.S->rec = gn / a.S->hn;
        }
        __syncthreads();
        if (s_stop) {
            if (blockIdx.x == 0 && threadIdx.x == 0) a.S->done = 1;
            return;
        }
    }
    // completion flags hold the sweep's number: distinct for every sweep of a solve
    const unsigned epoch = (unsigned)(a.S->napply * 2 * a.sweeps + sweep_idx + 1);
    unsigned* flags = FWD ? a.flag_f : a.flag_b;
    unsigned* ticket = &a.S->ticket[sweep_idx];
    const int32_t* sched = FWD ? a.sched_f : a.sched_b;
    const MT* mv = reinterpret_cast<const MT*>(a.mval);
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned slot = 0;
        if (lane == 0) slot = atomicAdd(ticket, 1u);
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if ((int64_t)slot >= a.n) break;
        const int64_t j = sched[slot];
        const int64_t e0 = a.mptr[j], e1 = a.mptr[j + 1];
        double acc = 0.0;
        bool ok = true;
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int64_t k = a.mcol[e];
            if (k == j) continue;
            const double mjk = (double)mv[e];
            const bool dep = FWD ? (k < j) : (k > j);
            if (dep) {
                unsigned polls = 0;
                while (ld_acquire_flag(&flags[k]) != epoch) {
                    if (++polls > (1u << 24)) { ok = false; break; }
                    if (polls > 32) __nanosleep(64);
                }
                acc = fma(mjk, e_new[k], acc);
            } else if (!identity && e_old) {
                acc = fma(mjk, e_old[k], acc);
            }
        }
        acc = warp_sum(acc);
        const unsigned any_bad = __ballot_sync(0xffffffffu, !ok);
        if (lane == 0) {
            if (any_bad) atomicOr(&a.S->err, DEV_ERR_TIMEOUT);
            const double dj = a.dinv[j];
            const double v = identity ? e_old[j] - acc * dj : (r[j] - acc) * dj;
            e_new[j] = v;
            st_release_flag(&flags[j], epoch);
        }
        __syncwarp();
    }
}

// rho' = g^T z; first: p = z, else beta = rho'/rho, p = z + beta p; pt = D^{-1} p; epoch++
__global__ void __launch_bounds__(SP_T) k_sp_gz(SpArgs a) {
    __shared__ double sh[40];
    if (a.S->done) return;
    double t = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += (int64_t)gridDim.x * blockDim.x)
        t = fma(a.g[j], a.z[j], t);
    t = block_sum(t, sh);
    if (threadIdx.x == 0) a.part[2 * a.nblk + blockIdx.x] = t;
}
__global__ void __launch_bounds__(SP_T) k_sp_pnext(SpArgs a, int first, int nparts) {
    __shared__ double sh[40];
    if (a.S->done) return;
    const double rho_new = sum_parts(a.part + 2 * a.nblk, nparts, sh);
    const double beta = first ? 0.0 : rho_new / a.S->rho;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += (int64_t)gridDim.x * blockDim.x) {
        const double pj = first ? a.z[j] : fma(beta, a.p[j], a.z[j]);
        a.p[j] = pj;
        a.pt[j] = pj * a.inv_d[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // every block has read rho above; the last block to finish moves the state on
        __threadfence();
        const unsigned done_blocks = atomicAdd(&a.S->pad, 1u);
        if (done_blocks == gridDim.x - 1) {
            a.S->rho = rho_new;
            a.S->pad = 0;
            a.S->napply += 1;
            for (int t = 0; t < 2 * a.sweeps; ++t) a.S->ticket[t] = 0;
        }
    }
}
// sums of ||x||^2 and ||D x||^2 into S (single block)
__global__ void k_sp_norms(SpArgs a, const double* x, double* out2) {
    __shared__ double sh[40];
    double t = 0.0, r = 0.0;
    for (int64_t j = threadIdx.x; j < a.n; j += blockDim.x) {
        const double v = x[j], vr = v / a.inv_d[j];
        t = fma(v, v, t);
        r = fma(vr, vr, r);
    }
    t = block_sum(t, sh);
    r = block_sum(r, sh);
    if (threadIdx.x == 0) { out2[0] = t; out2[1] = r; }
}
__global__ void k_sp_iter_inc(SpState* S) {
    if (!S->done) S->iters += 1;
}
__global__ void k_sp_scale(const double* src, const double* s, double* dst, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        dst[j] = src[j] * s[j];
}
__global__ void k_sp_diff(const double* h, const double* w, double* g, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        g[j] = h[j] - w[j];
}
template <typename T>
__global__ void k_gather_vals(const void* src, const int64_t* perm, int64_t nnz, void* dst) {
    const T* s = reinterpret_cast<const T*>(src);
    T* d = reinterpret_cast<T*>(dst);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        d[e] = s[perm[e]];
}
__global__ void k_gather_pairs(const float* src, const int64_t* perm, int64_t nnz, float* dst) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        dst[2 * e] = src[2 * perm[e]];
        dst[2 * e + 1] = src[2 * perm[e] + 1];
    }
}

static unsigned gridn(int64_t work, int64_t cap = 152 * 8) {
    int64_t g = (work + SP_T - 1) / SP_T;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

template <int DT>
static lsq_status sp_solve_impl(const lsq_matrix* A, const lsq_precond* P, const double* B,
                                const double* Hcols, int64_t k, int64_t ldb, double* X, int64_t ldx,
                                const lsq_opts* o, lsq_info* info, cudaStream_t st) {
    const SparseHandle* SH = P->sp;
    const int64_t m = A->m, n = A->n, nnz = A->nnz;
    const bool res64 = A->vals_f64 != nullptr || DT == LSQ_F64;
    const size_t es = elem_size(A->dtype);
    const int nblk = 152 * 4;
    // workspace
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off += (bytes + 255) & ~size_t(255); return at; };
    size_t o_S = take(sizeof(SpState)), o_vT = take(es * nnz), o_vT64 = take(res64 && DT != LSQ_F64 ? 8 * nnz : 16),
           o_vec = take(8 * (size_t)n * 10), o_q = take(8 * (size_t)m), o_ff = take(4 * (size_t)n),
           o_fb = take(4 * (size_t)n), o_part = take(8 * (size_t)nblk * 3), o_n2 = take(64);
    Scratch sc;
    LSQ_CUDA(sc.alloc(off, st));
    char* base = sc.as<char>();
    SpState* S = (SpState*)(base + o_S);
    double* vec = (double*)(base + o_vec);
    SpArgs a{};
    a.m = m; a.n = n; a.row_ptr = A->row_ptr; a.col_idx = A->col_idx;
    a.vals = A->vals;
    a.vals_res = res64 ? (DT == LSQ_F64 ? A->vals : (const void*)A->vals_f64) : A->vals;
    a.atptr = SH->atptr; a.atrow = SH->atrow;
    a.valsT = base + o_vT;
    a.valsT_res = res64 ? (DT == LSQ_F64 ? a.valsT : (const void*)(base + o_vT64)) : a.valsT;
    a.inv_d = P->inv_d;
    a.mptr = SH->mptr; a.mcol = SH->mcol;
    a.mval = P->op_dtype == LSQ_F32 ? (const void*)SH->mval32 : (const void*)SH->mval;
    a.dinv = SH->dinv; a.sched_f = SH->sched_f; a.sched_b = SH->sched_b;
    a.sweeps = P->sweeps;
    a.y = vec; a.g = vec + n; a.z = vec + 2 * n; a.p = vec + 3 * n; a.pt = vec + 4 * n;
    a.w = vec + 5 * n; a.e0 = vec + 6 * n; a.e1 = vec + 7 * n; a.h = vec + 8 * n;
    double* tmpv = vec + 9 * n;
    a.q = (double*)(base + o_q);
    a.flag_f = (unsigned*)(base + o_ff); a.flag_b = (unsigned*)(base + o_fb);
    a.part = (double*)(base + o_part); a.nblk = nblk;
    a.S = S;
    a.tol = o->tol; a.inner_tol = o->inner_tol > 0 ? o->inner_tol : 0.0; a.maxit = o->maxit;
    double* n2 = (double*)(base + o_n2);
    // A^T values in column order
    if (DT == LSQ_F32X2) k_gather_pairs<<<gridn(nnz), SP_T, 0, st>>>((const float*)A->vals, SH->atperm, nnz, (float*)(base + o_vT));
    else if (es == 8) k_gather_vals<double><<<gridn(nnz), SP_T, 0, st>>>(A->vals, SH->atperm, nnz, base + o_vT);
    else if (es == 4) k_gather_vals<float><<<gridn(nnz), SP_T, 0, st>>>(A->vals, SH->atperm, nnz, base + o_vT);
    else k_gather_vals<__nv_bfloat16><<<gridn(nnz), SP_T, 0, st>>>(A->vals, SH->atperm, nnz, base + o_vT);
    if (res64 && DT != LSQ_F64) k_gather_vals<double><<<gridn(nnz), SP_T, 0, st>>>(A->vals_f64, SH->atperm, nnz, base + o_vT64);
    count_launch(2);
    const unsigned grows = gridn((m * 8 + 7) / 8 * 8, nblk), gcols = gridn(n * 32), gvec = gridn(n, nblk);
    const unsigned gsweep = (unsigned)std::min<int64_t>((n * 32 + SP_T - 1) / SP_T, 152 * 8);
    // residual passes read FP64 values when there are FP64 values (the matrix's own or the
    // supplied copy), otherwise the matrix's own dtype
    auto rows = [&](int mode, int use_res, const double* x) {
        if (use_res && res64) k_sp_rows<LSQ_F64><<<grows, SP_T, 0, st>>>(a, mode, 1, x);
        else k_sp_rows<DT><<<grows, SP_T, 0, st>>>(a, mode, 0, x);
    };
    auto cols = [&](int use_res, double* out) {
        if (use_res && res64) k_sp_cols<LSQ_F64><<<gcols, SP_T, 0, st>>>(a, 1, out);
        else k_sp_cols<DT><<<gcols, SP_T, 0, st>>>(a, 0, out);
    };
    // z = P g with t forward and t backward sweeps; epoch advanced per sweep
    auto sweep = [&](bool fwd, const double* r, const double* eold, double* enew, int identity, int check, int idx) {
        if (P->op_dtype == LSQ_F32) {
            if (fwd) k_sp_sweep<float, true><<<gsweep, SP_T, 0, st>>>(a, r, eold, enew, identity, check, gvec, idx);
            else k_sp_sweep<float, false><<<gsweep, SP_T, 0, st>>>(a, r, eold, enew, identity, check, gvec, idx);
        } else {
            if (fwd) k_sp_sweep<double, true><<<gsweep, SP_T, 0, st>>>(a, r, eold, enew, identity, check, gvec, idx);
            else k_sp_sweep<double, false><<<gsweep, SP_T, 0, st>>>(a, r, eold, enew, identity, check, gvec, idx);
        }
    };
    // z = P g: t forward then t backward sweeps (the first may carry the convergence check)
    auto precond = [&](int check) {
        const double* eold = nullptr;
        double* bufs[2] = {a.e0, a.e1};
        int cur = 0, idx = 0;
        for (int t = 0; t < P->sweeps; ++t, ++idx) {
            sweep(true, a.g, eold, bufs[cur], 0, (t == 0) ? check : 0, idx);
            eold = bufs[cur];
            cur ^= 1;
        }
        for (int t = 0; t < P->sweeps; ++t, ++idx) {
            double* dst = (t == P->sweeps - 1) ? a.z : bufs[cur];
            sweep(false, a.g, eold, dst, (P->sweeps == 1) ? 1 : 0, 0, idx);
            eold = dst;
            cur ^= 1;
        }
    };
    const int batch = 8;
    lsq_status worst = LSQ_OK;
    cudaEvent_t ev0, ev1;
    LSQ_CUDA(cudaEventCreate(&ev0));
    LSQ_CUDA(cudaEventCreate(&ev1));
    LSQ_CUDA(cudaEventRecord(ev0, st));
    for (int64_t c = 0; c < k; ++c) {
        LSQ_CUDA(cudaMemsetAsync(S, 0, sizeof(SpState), st));
        LSQ_CUDA(cudaMemsetAsync(a.flag_f, 0, 4 * (size_t)n, st));
        LSQ_CUDA(cudaMemsetAsync(a.flag_b, 0, 4 * (size_t)n, st));
        LSQ_CUDA(cudaMemsetAsync(a.y, 0, 8 * (size_t)n, st));
        a.b = B ? B + c * ldb : nullptr;
        a.h_in = Hcols ? Hcols + c * ldb : nullptr;
        if (a.h_in) {
            LSQ_CUDA(cudaMemcpyAsync(a.h, a.h_in, 8 * (size_t)n, cudaMemcpyDeviceToDevice, st));
        } else {
            rows(SPM_RHS, 1, a.pt);
            cols(1, a.h);
        }
        k_sp_norms<<<1, 1024, 0, st>>>(a, a.h, n2);
        LSQ_CUDA(cudaMemcpyAsync(a.g, a.h, 8 * (size_t)n, cudaMemcpyDeviceToDevice, st));
        double hn2[2];
        LSQ_CUDA(cudaMemcpyAsync(hn2, n2, 16, cudaMemcpyDeviceToHost, st));
        LSQ_CUDA(cudaStreamSynchronize(st));
        const double hn = std::sqrt(hn2[0]), hn_raw = std::sqrt(hn2[1]);
        int iters = 0, outer_used = 0, converged = 0, status = LSQ_ERR_NOT_CONVERGED, napply = 0;
        double rec = 1.0, tru = 1.0, raw = 1.0, gg = hn2[0], ggraw = hn2[1];
        bool dirty = false;
        auto true_residual = [&]() -> lsq_status {
            // the iteration kernels stopped on S->done; the residual kernels must run
            LSQ_CUDA(cudaMemsetAsync(&S->done, 0, sizeof(int32_t), st));
            k_sp_scale<<<gvec, SP_T, 0, st>>>(a.y, a.inv_d, tmpv, n);
            if (a.h_in) {
                rows(SPM_MATVEC, 1, tmpv);
                cols(1, a.w);
                k_sp_diff<<<gvec, SP_T, 0, st>>>(a.h, a.w, a.g, n);
            } else {
                rows(SPM_RESID, 1, tmpv);
                cols(1, a.g);
            }
            k_sp_norms<<<1, 1024, 0, st>>>(a, a.g, n2);
            double r2[2];
            LSQ_CUDA(cudaMemcpyAsync(r2, n2, 16, cudaMemcpyDeviceToHost, st));
            LSQ_CUDA(cudaStreamSynchronize(st));
            gg = r2[0]; ggraw = r2[1];
            dirty = false;
            return LSQ_OK;
        };
        if (hn == 0.0) {
            converged = 1; status = LSQ_OK; rec = tru = raw = 0.0;
        } else {
            for (int outer = 0; outer < o->max_outer; ++outer) {
                if (outer > 0) {
                    lsq_status rs = true_residual();
                    if (rs != LSQ_OK) return rs;
                }
                tru = std::sqrt(gg) / hn;
                raw = std::sqrt(ggraw) / hn_raw;
                if (outer == 0) rec = tru;
                if (tru <= o->tol) { converged = 1; status = LSQ_OK; break; }
                if (iters >= o->maxit) break;
                outer_used = outer + 1;
                SpState init{};
                init.hn = hn; init.gstart = std::sqrt(gg); init.iters = iters; init.napply = napply;
                init.rec = tru;
                LSQ_CUDA(cudaMemcpyAsync(S, &init, sizeof(SpState), cudaMemcpyHostToDevice, st));
                // z = P g, rho = g^T z, p = z
                precond(0);
                k_sp_gz<<<gvec, SP_T, 0, st>>>(a);
                k_sp_pnext<<<gvec, SP_T, 0, st>>>(a, 1, gvec);
                count_launch(2 * P->sweeps + 2);
                SpState hs{};
                while (true) {
                    for (int b = 0; b < batch; ++b) {
                        rows(SPM_MATVEC, 0, a.pt);
                        cols(0, a.w);
                        k_sp_update<<<gvec, SP_T, 0, st>>>(a, grows);
                        k_sp_iter_inc<<<1, 1, 0, st>>>(S);
                        precond(1);
                        k_sp_gz<<<gvec, SP_T, 0, st>>>(a);
                        k_sp_pnext<<<gvec, SP_T, 0, st>>>(a, 0, gvec);
                        count_launch(2 * P->sweeps + 6);
                    }
                    LSQ_CUDA(cudaGetLastError());
                    LSQ_CUDA(cudaMemcpyAsync(&hs, S, sizeof(SpState), cudaMemcpyDeviceToHost, st));
                    LSQ_CUDA(cudaStreamSynchronize(st));
                    if (hs.err) { set_error("sparse Gauss-Seidel sweep: a dependency wait timed out"); return LSQ_ERR_TIMEOUT; }
                    if (hs.done || hs.iters >= o->maxit) break;
                }
                dirty = dirty || hs.iters > iters;
                iters = hs.iters;
                napply = hs.napply;
                rec = hs.rec;
                if (hs.status == LSQ_ERR_BREAKDOWN) { status = LSQ_ERR_BREAKDOWN; break; }
            }
            if (!converged && status != LSQ_ERR_BREAKDOWN && dirty) {
                lsq_status rs = true_residual();
                if (rs != LSQ_OK) return rs;
                tru = std::sqrt(gg) / hn;
                raw = std::sqrt(ggraw) / hn_raw;
                if (tru <= o->tol) { converged = 1; status = LSQ_OK; }
            }
        }
        k_sp_scale<<<gvec, SP_T, 0, st>>>(a.y, a.inv_d, X + c * ldx, n);
        count_launch();
        if (info && c < info->k) {
            if (info->iters) info->iters[c] = iters;
            if (info->outer) info->outer[c] = outer_used;
            if (info->converged) info->converged[c] = (uint8_t)converged;
            if (info->relres_rec) info->relres_rec[c] = rec;
            if (info->relres_true) info->relres_true[c] = tru;
            if (info->relres_raw) info->relres_raw[c] = raw;
        }
        if (status == LSQ_ERR_BREAKDOWN) worst = LSQ_ERR_BREAKDOWN;
        else if (status != LSQ_OK && worst == LSQ_OK) worst = LSQ_ERR_NOT_CONVERGED;
    }
    LSQ_CUDA(cudaEventRecord(ev1, st));
    LSQ_CUDA(cudaEventSynchronize(ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (info) {
        info->s = P->s; info->nnz_M = P->nnz_M; info->n_fixed_diag = P->n_fixed_diag;
        info->levels = P->levels; info->solve_ms = ms;
    }
    LSQ_CUDA(cudaGetLastError());
    if (worst == LSQ_ERR_NOT_CONVERGED) set_error("PCG did not reach the tolerance");
    if (worst == LSQ_ERR_BREAKDOWN) set_error("PCG breakdown (non-positive or non-finite curvature)");
    return worst;
}

// e = P r for k vectors (column c at r + c n): the sweeps of Alg. 3 alone
lsq_status sparse_apply(const lsq_precond* P, const double* r, double* e, int64_t k, cudaStream_t st) {
    const SparseHandle* SH = P->sp;
    const int64_t n = P->n;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off += (bytes + 255) & ~size_t(255); return at; };
    size_t o_S = take(sizeof(SpState)), o_e = take(16 * (size_t)n), o_f = take(8 * (size_t)n);
    Scratch sc;
    LSQ_CUDA(sc.alloc(off, st));
    char* base = sc.as<char>();
    SpArgs a{};
    a.n = n;
    a.mptr = SH->mptr; a.mcol = SH->mcol;
    a.mval = P->op_dtype == LSQ_F32 ? (const void*)SH->mval32 : (const void*)SH->mval;
    a.dinv = SH->dinv; a.sched_f = SH->sched_f; a.sched_b = SH->sched_b; a.sweeps = P->sweeps;
    a.e0 = (double*)(base + o_e); a.e1 = a.e0 + n;
    a.flag_f = (unsigned*)(base + o_f); a.flag_b = a.flag_f + n;
    a.S = (SpState*)(base + o_S);
    const unsigned gsweep = (unsigned)std::min<int64_t>((n * 32 + SP_T - 1) / SP_T, 152 * 8);
    for (int64_t c = 0; c < k; ++c) {
        LSQ_CUDA(cudaMemsetAsync(a.S, 0, sizeof(SpState), st));
        LSQ_CUDA(cudaMemsetAsync(a.flag_f, 0, 8 * (size_t)n, st));
        const double* rc = r + c * n;
        double* out = e + c * n;
        const double* eold = nullptr;
        double* bufs[2] = {a.e0, a.e1};
        int cur = 0, idx = 0;
        for (int t = 0; t < P->sweeps; ++t, ++idx) {
            if (P->op_dtype == LSQ_F32) k_sp_sweep<float, true><<<gsweep, SP_T, 0, st>>>(a, rc, eold, bufs[cur], 0, 0, 0, idx);
            else k_sp_sweep<double, true><<<gsweep, SP_T, 0, st>>>(a, rc, eold, bufs[cur], 0, 0, 0, idx);
            eold = bufs[cur];
            cur ^= 1;
        }
        for (int t = 0; t < P->sweeps; ++t, ++idx) {
            double* dst = (t == P->sweeps - 1) ? out : bufs[cur];
            const int ident = P->sweeps == 1 ? 1 : 0;
            if (P->op_dtype == LSQ_F32) k_sp_sweep<float, false><<<gsweep, SP_T, 0, st>>>(a, rc, eold, dst, ident, 0, 0, idx);
            else k_sp_sweep<double, false><<<gsweep, SP_T, 0, st>>>(a, rc, eold, dst, ident, 0, 0, idx);
            eold = dst;
            cur ^= 1;
        }
        count_launch(2 * P->sweeps);
    }
    LSQ_CUDA(cudaGetLastError());
    SpState hs{};
    LSQ_CUDA(cudaMemcpyAsync(&hs, a.S, sizeof(SpState), cudaMemcpyDeviceToHost, st));
    LSQ_CUDA(cudaStreamSynchronize(st));
    if (hs.err) { set_error("sparse Gauss-Seidel sweep: a dependency wait timed out"); return LSQ_ERR_TIMEOUT; }
    return LSQ_OK;
}

// grad_b = A lambda, r = b - A x and grad_vals[e] = sum_c r_i lambda_j - (A lambda)_i x_j
template <int DT>
__global__ void k_csr_rowdot(int64_t m, const int64_t* rp, const int32_t* ci, const void* vals,
                             const double* v, const double* b, double sb, double sa, double* out) {
    const int sub = threadIdx.x & 7;
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) >> 3;
    for (int64_t i0 = 0; i0 < m; i0 += ngrp) {
        const int64_t i = i0 + grp;
        double t = 0.0;
        if (i < m)
            for (int64_t e = rp[i] + sub; e < rp[i + 1]; e += 8) t = fma(Val<DT>::load(vals, e), v[ci[e]], t);
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (i < m && sub == 0) out[i] = (b ? sb * b[i] : 0.0) + sa * t;
    }
}
__global__ void k_sddmm_csr(int64_t m, const int64_t* rp, const int32_t* ci, int64_t kcols,
                            const double* r, const double* al, int64_t ldm, const double* lam,
                            const double* x, int64_t ldn, double* grad) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < m; i += nw) {
        for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) {
            const int64_t j = ci[e];
            double acc = 0.0;
            for (int64_t c = 0; c < kcols; ++c)
                acc += r[c * ldm + i] * lam[c * ldn + j] - al[c * ldm + i] * x[c * ldn + j];
            grad[e] = acc;
        }
    }
}
__global__ void k_scale_into(const double* src, int64_t lds, const double* s, double* dst, int64_t n, int64_t kcols) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * kcols; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t / n, j = t % n;
        dst[c * n + j] = src[c * lds + j] * s[j];
    }
}

template <int DT>
static lsq_status sp_adjoint_impl(const lsq_matrix* A, const lsq_precond* P, const double* X, const double* B,
                                  const double* G, int64_t k, int64_t ldb, int64_t ldx, double* grad_b,
                                  double* grad_vals, double* Lambda, const lsq_opts* o, lsq_info* info,
                                  cudaStream_t st) {
    const int64_t m = A->m, n = A->n;
    Scratch sc;
    LSQ_CUDA(sc.alloc(8 * (size_t)(2 * n * k + 2 * m * k) + 256, st));
    double* h = sc.as<double>();
    double* lam = h + n * k;
    double* r = lam + n * k;
    double* al = r + m * k;
    k_scale_into<<<gridn(n * k), SP_T, 0, st>>>(G, ldx, P->inv_d, h, n, k);
    count_launch();
    // A^T A lambda = G  <=>  Â^T Â mu = D^{-1} G, lambda = D^{-1} mu (the solver's output)
    lsq_status s = sparse_solve(A, P, nullptr, h, k, n, lam, n, o, info, st);
    if (s != LSQ_OK && s != LSQ_ERR_NOT_CONVERGED) return s;
    const void* vals = A->vals;
    for (int64_t c = 0; c < k; ++c) {
        k_csr_rowdot<DT><<<gridn(m * 8), SP_T, 0, st>>>(m, A->row_ptr, A->col_idx, vals, lam + c * n, nullptr, 0.0, 1.0, al + c * m);
        k_csr_rowdot<DT><<<gridn(m * 8), SP_T, 0, st>>>(m, A->row_ptr, A->col_idx, vals, X + c * ldx, B + c * ldb, 1.0, -1.0, r + c * m);
        count_launch(2);
        if (grad_b) LSQ_CUDA(cudaMemcpyAsync(grad_b + c * ldb, al + c * m, 8 * (size_t)m, cudaMemcpyDeviceToDevice, st));
        if (Lambda) LSQ_CUDA(cudaMemcpyAsync(Lambda + c * ldx, lam + c * n, 8 * (size_t)n, cudaMemcpyDeviceToDevice, st));
    }
    if (grad_vals) {
        k_sddmm_csr<<<gridn(m * 32), SP_T, 0, st>>>(m, A->row_ptr, A->col_idx, k, r, al, m, lam, X, ldx, grad_vals);
        count_launch();
    }
    LSQ_CUDA(cudaGetLastError());
    LSQ_CUDA(cudaStreamSynchronize(st));
    return s;
}

lsq_status sparse_adjoint(const lsq_matrix* A, const lsq_precond* P, const double* X, const double* B,
                          const double* G, int64_t k, int64_t ldb, int64_t ldx, double* grad_b,
                          double* grad_vals, double* Lambda, const lsq_opts* o, lsq_info* info, cudaStream_t st) {
    LSQ_CHECK_ARG(P->sp != nullptr, "preconditioner was built for a dense matrix");
    switch (A->dtype) {
        case LSQ_F64: return sp_adjoint_impl<LSQ_F64>(A, P, X, B, G, k, ldb, ldx, grad_b, grad_vals, Lambda, o, info, st);
        case LSQ_F32: return sp_adjoint_impl<LSQ_F32>(A, P, X, B, G, k, ldb, ldx, grad_b, grad_vals, Lambda, o, info, st);
        case LSQ_BF16: return sp_adjoint_impl<LSQ_BF16>(A, P, X, B, G, k, ldb, ldx, grad_b, grad_vals, Lambda, o, info, st);
        default: return sp_adjoint_impl<LSQ_F32X2>(A, P, X, B, G, k, ldb, ldx, grad_b, grad_vals, Lambda, o, info, st);
    }
}

lsq_status sparse_solve(const lsq_matrix* A, const lsq_precond* P, const double* B, const double* Hcols,
                        int64_t k, int64_t ldb, double* X, int64_t ldx, const lsq_opts* o, lsq_info* info,
                        cudaStream_t st) {
    LSQ_CHECK_ARG(P->sp != nullptr, "preconditioner was built for a dense matrix");
    LSQ_CHECK_ARG(P->sp->nnz_A == A->nnz && P->sp->m == A->m, "preconditioner was built for another pattern");
    LSQ_CHECK_ARG(P->sweeps <= 32, "sparse sweeps must be <= 32");
    switch (A->dtype) {
        case LSQ_F64: return sp_solve_impl<LSQ_F64>(A, P, B, Hcols, k, ldb, X, ldx, o, info, st);
        case LSQ_F32: return sp_solve_impl<LSQ_F32>(A, P, B, Hcols, k, ldb, X, ldx, o, info, st);
        case LSQ_BF16: return sp_solve_impl<LSQ_BF16>(A, P, B, Hcols, k, ldb, X, ldx, o, info, st);
        default: return sp_solve_impl<LSQ_F32X2>(A, P, B, Hcols, k, ldb, X, ldx, o, info, st);
    }
}

}  // namespace lsq
