// Alg. 2 step 4 for a block of K <= 32 right-hand sides of a CSR matrix: K independent PCG
// recurrences advanced together, so that every pass over A and every Gauss-Seidel sweep
// over A_s^T A_s serves all K columns.
//
// Vectors are stored row-major n x K (element (j, c) at j*K + c); a group of GK lanes
// (GK = K rounded up to a power of two) handles one row and lane c its column c.  Every
// column keeps its own alpha, beta, rho and convergence state: a column whose recursive
// residual meets the tolerance (or that reaches maxit, or breaks down) is frozen (alpha = 0
// from then on, p and rho no longer updated), so each column follows the iteration it would
// follow alone; the batch stops when every column is frozen.
//
// Per iteration:
//   k_bk_rows   q = Â p for all columns; the last block sums the partials of p^T w = ||q||^2
//   k_bk_cols   w = Â^T q
//   k_bk_update alpha, y += alpha p, g -= alpha w; the last block sums ||g||^2 and freezes
//               converged columns
//   k_bk_sweep  t forward and t backward level-ordered Gauss-Seidel sweeps (one level wait
//               per row for all K columns)
//   k_bk_gz     rho' = g^T z; the last block forms beta and moves rho on
//   k_bk_pnext  p = z + beta p, pt = D^{-1} p
// Reductions are fixed-order (per-block partials, then one block sums them in block order),
// so results do not depend on timing.
#include "bk_device.cuh"
#include "sparse_persist.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <unordered_map>

namespace lsq {

template <int DT>
__global__ void __launch_bounds__(BK_T) k_bk_rows(BkArgs a, int mode, int use_res, const double* x) {
    if (a.S->done) return;
    bk_rows_body<DT>(a, mode, use_res, x);
}

template <int DT>
__global__ void __launch_bounds__(BK_T) k_bk_cols(BkArgs a, int use_res, double* out) {
    if (a.S->done) return;
    bk_cols_body<DT>(a, use_res, out);
}

__global__ void __launch_bounds__(BK_T) k_bk_update(BkArgs a) {
    if (a.S->done) return;
    bk_update_body(a);
}

__global__ void k_bk_fill_empty(double* e, int64_t cnt) {
    bk_fill_empty_body(e, cnt);
}

// every block sweep kernel takes the same arguments (one launch path); out64 is used by the
// pair form of the CTA-per-row sweep only
template <typename MT, bool FWD>
__global__ void __launch_bounds__(BK_T) k_bk_sweep(BkArgs a, const double* r, const double* e_old,
                                                   double* e_new, int identity, int sweep_idx, double* out64) {
    if (a.S->done) return;
    bk_sweep_body<MT, FWD>(a, r, e_old, e_new, identity, sweep_idx);
    (void)out64;
}

template <typename MT, bool FWD, int KT>
__global__ void __launch_bounds__(BK_T) k_bk_sweep_ep(BkArgs a, const double* r, const double* e_old,
                                                      double* e_new, int identity, int sweep_idx, double* out64) {
    if (a.S->done) return;
    bk_sweep_ep_body<MT, FWD, KT>(a, r, e_old, e_new, identity, sweep_idx);
    (void)out64;
}

template <typename MT, bool FWD, int KT, bool PAIRS>
__global__ void __launch_bounds__(BK_T) k_bk_sweep_cta(BkArgs a, const double* r, const double* e_old,
                                                       double* e_new, int identity, int sweep_idx, double* out64) {
    if (a.S->done) return;
    bk_sweep_cta_body<MT, FWD, KT, PAIRS>(a, r, e_old, e_new, identity, sweep_idx, out64);
}

// The CTA-per-row sweep in ONE thread-block cluster of C = 2^lg CTAs, for deep level
// structures whose block vector (n x K) fits in the cluster's shared memory.  Row j's K values
// live in CTA (j mod C) at slots (j / C) K ... (j / C) K + K - 1.  CTA r takes rows r, r + C,
// ... of each level, and its threads take a row's dependency entries as in the CTA form
// (thread t: entries t, t + BK_T, ..., the same order, so the same sums); the gathers read the
// owners' shared memory (DSMEM) and the levels meet at cluster barriers, so nothing is
// polled.  The CTA's first row of the next level (its indices and values) is loaded before
// the barrier.  Every value is also stored to e_new in global memory.
template <typename MT, bool FWD, int KT>
__global__ void __launch_bounds__(BK_T, 1) k_bk_sweep_cl(BkArgs a, const double* r, const double* e_old,
                                                         double* e_new, int identity, const int64_t* loff,
                                                         int64_t nlev, int lg) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) double xs[];   // this CTA's rows of e_new, K values each
    __shared__ double s_part[BK_T / 32][KT];
    // the same exit in every CTA: done only changes in the update step, not during a sweep
    if (a.S->done) return;
    cg::cluster_group cl = cg::this_cluster();
    const unsigned C = 1u << lg, me = cl.block_rank(), cmask = C - 1u;
    const int32_t* sched = FWD ? a.sched_f : a.sched_b;
    const MT* mv = reinterpret_cast<const MT*>(a.mval);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int K = a.K;
    const bool other = !identity && e_old != nullptr;
    constexpr int SH = (KT >= 32) ? 0 : (KT >= 16 ? 1 : (KT >= 8 ? 2 : (KT >= 4 ? 3 : (KT >= 2 ? 4 : 5))));
    constexpr int PF = 2;   // dependency entries per thread loaded ahead (rows up to 2 BK_T entries)
    struct Row {
        int64_t j, d0, d1;
        int32_t kk[PF];
        MT mm[PF];
    };
    auto load_row = [&](int64_t j, Row& R) {
        R.j = j;
        const int64_t e0 = a.mptr[j], e1 = a.mptr[j + 1], ed = a.mdiag[j];
        R.d0 = FWD ? e0 : ed + 1;
        R.d1 = FWD ? ed : e1;
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const int64_t e = R.d0 + tid + (int64_t)BK_T * u;
            R.kk[u] = -1;
            R.mm[u] = MT(0);
            if (e < R.d1) { R.kk[u] = a.mcol[e]; R.mm[u] = mv[e]; }
        }
    };
    auto entry = [&](int32_t k, double mk, double (&acc)[KT]) {
        const double* src = cl.map_shared_rank(xs, (unsigned)k & cmask) + (int64_t)((unsigned)k >> lg) * K;
        double v[KT];
#pragma unroll
        for (int c = 0; c < KT; ++c) v[c] = c < K ? src[c] : 0.0;
#pragma unroll
        for (int c = 0; c < KT; ++c)
            if (c < K) acc[c] = fma(mk, v[c], acc[c]);
    };
    auto finish_row = [&](const Row& R) {
        const int64_t j = R.j;
        double acc[KT];
#pragma unroll
        for (int c = 0; c < KT; ++c) acc[c] = 0.0;
        if (other) {
            const int64_t e0 = a.mptr[j], e1 = a.mptr[j + 1], ed = a.mdiag[j];
            const int64_t o0 = FWD ? ed + 1 : e0, o1 = FWD ? e1 : ed;
            for (int64_t e = o0 + tid; e < o1; e += BK_T) {
                const int64_t k = a.mcol[e];
                const double mk = (double)mv[e];
#pragma unroll
                for (int c = 0; c < KT; ++c)
                    if (c < K) acc[c] = fma(mk, e_old[k * K + c], acc[c]);
            }
        }
#pragma unroll
        for (int u = 0; u < PF; ++u)
            if (R.kk[u] >= 0) entry(R.kk[u], (double)R.mm[u], acc);
        for (int64_t e = R.d0 + tid + (int64_t)BK_T * PF; e < R.d1; e += BK_T)
            entry(a.mcol[e], (double)mv[e], acc);
        const double tot = bk_reduce_scatter<KT>(acc, lane);
        if ((lane & ((1 << SH) - 1)) == 0) s_part[wid][lane >> SH] = tot;
        __syncthreads();
        if (wid == 0 && lane < K) {
            double sum = 0.0;
#pragma unroll
            for (int w = 0; w < BK_T / 32; ++w) sum += s_part[w][lane];
            const double dj = a.dinv[j];
            const int64_t at = j * K + lane;
            const double val = identity ? e_old[at] - sum * dj : (r[at] - sum) * dj;
            double* dst = cl.map_shared_rank(xs, (unsigned)j & cmask) + (int64_t)((unsigned)j >> lg) * K;
            dst[lane] = val;
            e_new[at] = val;
        }
        __syncthreads();   // s_part is reused by the next row
    };
    Row cur;
    int64_t lo = loff[0], hi = loff[1];
    if ((int64_t)me < hi - lo) load_row(sched[lo + me], cur);
    cl.sync();   // every CTA of the cluster runs before any shared memory is read remotely
    for (int64_t L = 0; L < nlev; ++L) {
        const int64_t cnt = hi - lo;
        for (int64_t q = me; q < cnt; q += C) {
            if (q != (int64_t)me) load_row(sched[lo + q], cur);
            finish_row(cur);
        }
        if (L + 1 < nlev) {
            lo = hi;
            hi = loff[L + 2];
            if ((int64_t)me < hi - lo) load_row(sched[lo + me], cur);
        }
        cl.sync();   // this level's values are visible in every CTA; after the last, no CTA reads another's memory
    }
}

__global__ void __launch_bounds__(BK_T) k_bk_gz(BkArgs a, int first) {
    if (a.S->done) return;
    bk_gz_body(a, first);
}

__global__ void __launch_bounds__(BK_T) k_bk_pnext(BkArgs a) {
    if (a.S->done) return;
    bk_pnext_body(a);
}

__global__ void __launch_bounds__(BK_T) k_bk_norms(BkArgs a, const double* x, double* out2) {
    bk_norms_body(a, x, out2);
}

// column-major (leading dimension ld) -> row-major n x K
__global__ void k_bk_to_rows(const double* src, int64_t ld, int64_t n, int K, double* dst) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * K; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / K, c = t % K;
        dst[t] = src[c * ld + j];
    }
}
// row-major n x K scaled by s_j -> column-major (leading dimension ld)
__global__ void k_bk_from_rows(const double* src, int64_t n, int K, const double* s, double* dst, int64_t ld) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * K; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t / n, j = t % n;
        dst[c * ld + j] = src[j * K + c] * s[j];
    }
}
__global__ void k_bk_diff(const double* h, const double* w, double* g, int64_t cnt) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        g[t] = h[t] - w[t];
}
__global__ void k_bk_scale(const double* src, int64_t n, int K, const double* s, double* dst) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * K; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = src[t] * s[t / K];
}
template <typename T>
__global__ void k_bk_gather(const void* src, const int64_t* perm, int64_t nnz, void* dst) {
    const T* s = reinterpret_cast<const T*>(src);
    T* d = reinterpret_cast<T*>(dst);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        d[e] = s[perm[e]];
}
__global__ void k_bk_gather_pairs(const float* src, const int64_t* perm, int64_t nnz, float* dst) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        dst[2 * e] = src[2 * perm[e]];
        dst[2 * e + 1] = src[2 * perm[e] + 1];
    }
}

static unsigned bk_grid(int64_t work, int64_t cap) {
    int64_t g = (work + BK_T - 1) / BK_T;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

// Cooperative launch: every warp of the sweep must be resident for the level waits to end.
// The grid (SMs x resident blocks) is computed once per kernel.
static lsq_status bk_launch_sweep(const void* kern, const BkArgs& a, const double* r, const double* eold,
                                  double* enew, double* out64, int identity, int idx, int64_t nlev,
                                  int units_per_block, cudaStream_t st) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> grids;
    int grid = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = grids.find(kern);
        if (it != grids.end()) {
            grid = it->second;
        } else {
            int dev = 0, sms = 0, per = 0;
            LSQ_CUDA(cudaGetDevice(&dev));
            LSQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            LSQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, BK_T, 0));
            if (per < 1) { set_error("block sweep kernel does not fit on an SM"); return LSQ_ERR_CUDA; }
            grid = sms * per;
            grids[kern] = grid;
        }
    }
    const int64_t cnt = a.n * a.K;   // every value of e_new starts as the empty marker
    k_bk_fill_empty<<<(unsigned)std::min<int64_t>((cnt + BK_T - 1) / BK_T, 152 * 8), BK_T, 0, st>>>(enew, cnt);
    count_launch();
    BkArgs av = a;
    void* params[] = {&av, (void*)&r, (void*)&eold, (void*)&enew, &identity, &idx, (void*)&out64};
    const int g_sweep = sweep_grid(grid, a.n, nlev, units_per_block);
    LSQ_CUDA(cudaLaunchCooperativeKernel(kern, dim3(g_sweep), dim3(BK_T), params, 0, st));
    count_launch();
    return LSQ_OK;
}

// lane-per-column sweep for short rows, entry-parallel sweep (KT >= K accumulators) for long
// mode 0: lane per column (short rows); 1: warp per row, lane per entry; 2: CTA per row (with
// float-pair sums when PAIRS)
template <typename MT, bool FWD, bool PAIRS = false>
static const void* bk_sweep_kernel(int mode, int K) {
    if (mode == 0) return (const void*)k_bk_sweep<MT, FWD>;
    if (mode == 1) {
        if (K <= 2) return (const void*)k_bk_sweep_ep<MT, FWD, 2>;
        if (K <= 4) return (const void*)k_bk_sweep_ep<MT, FWD, 4>;
        if (K <= 8) return (const void*)k_bk_sweep_ep<MT, FWD, 8>;
        if (K <= 16) return (const void*)k_bk_sweep_ep<MT, FWD, 16>;
        return (const void*)k_bk_sweep_ep<MT, FWD, 32>;
    }
    if (K <= 2) return (const void*)k_bk_sweep_cta<MT, FWD, 2, PAIRS>;
    if (K <= 4) return (const void*)k_bk_sweep_cta<MT, FWD, 4, PAIRS>;
    if (K <= 8) return (const void*)k_bk_sweep_cta<MT, FWD, 8, PAIRS>;
    if (K <= 16) return (const void*)k_bk_sweep_cta<MT, FWD, 16, PAIRS>;
    return (const void*)k_bk_sweep_cta<MT, FWD, 32, PAIRS>;
}

template <typename MT, bool FWD>
static const void* bk_sweep_cl_kernel(int K) {
    if (K <= 2) return (const void*)k_bk_sweep_cl<MT, FWD, 2>;
    if (K <= 4) return (const void*)k_bk_sweep_cl<MT, FWD, 4>;
    if (K <= 8) return (const void*)k_bk_sweep_cl<MT, FWD, 8>;
    if (K <= 16) return (const void*)k_bk_sweep_cl<MT, FWD, 16>;
    return (const void*)k_bk_sweep_cl<MT, FWD, 32>;
}

// The cluster form's size (8 CTAs, the portable maximum) and shared-memory budget per CTA.
constexpr int BC_LG = 3;
constexpr int64_t BC_SMEM = 200 * 1024;
static int64_t bk_cl_smem(int64_t n, int K) { return 8 * K * ((n + (1 << BC_LG) - 1) >> BC_LG); }

// True when the cluster form of this kernel can run on this device (once per kernel).
static bool bk_cluster_fits(const void* kern) {
    static std::mutex mu;
    static std::unordered_map<const void*, bool> ok;
    std::lock_guard<std::mutex> lk(mu);
    auto it = ok.find(kern);
    if (it != ok.end()) return it->second;
    bool f = false;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BC_SMEM) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 1 << BC_LG;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(1 << BC_LG);
        cfg.blockDim = dim3(BK_T);
        cfg.dynamicSmemBytes = BC_SMEM;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int clusters = 0;
        f = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess && clusters > 0;
    }
    cudaGetLastError();   // a refused query leaves the grid forms in use, not an error
    ok[kern] = f;
    return f;
}

static lsq_status bk_launch_sweep_cl(const void* kern, const BkArgs& a, const double* r, const double* eold,
                                     double* enew, int identity, const int64_t* loff, int64_t nlev,
                                     cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1 << BC_LG;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(1 << BC_LG);
    cfg.blockDim = dim3(BK_T);
    cfg.dynamicSmemBytes = (size_t)bk_cl_smem(a.n, a.K);
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    BkArgs av = a;
    int lg = BC_LG;
    void* params[] = {&av, (void*)&r, (void*)&eold, (void*)&enew, &identity, (void*)&loff, &nlev, &lg};
    LSQ_CUDA(cudaLaunchKernelExC(&cfg, kern, params));
    count_launch();
    return LSQ_OK;
}

struct BkOut {
    int32_t iters[BK_MAX], outer[BK_MAX];
    uint8_t conv[BK_MAX];
    double rec[BK_MAX], tru[BK_MAX], raw[BK_MAX];
    lsq_status status[BK_MAX];
};

// One block of K columns: B (m x K) or Hcols (n x K) column-major with leading dimension ldb,
// X column-major with leading dimension ldx.
template <int DT>
static lsq_status bk_solve_impl(const lsq_matrix* A, const lsq_precond* P, const double* B, const double* Hcols,
                                int K, int64_t ldb, double* X, int64_t ldx, const lsq_opts* o, BkOut* out,
                                bool capturing, cudaStream_t st) {
    const SparseHandle* SH = P->sp;
    const int64_t m = A->m, n = A->n, nnz = A->nnz;
    const bool res64 = A->vals_f64 != nullptr || DT == LSQ_F64;
    const size_t es = elem_size(A->dtype);
    const int64_t grid_cap = 152 * 16;
    int GK = 1;
    while (GK < K) GK <<= 1;
    const int64_t nK = n * K;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off += (bytes + 255) & ~size_t(255); return at; };
    const size_t o_S = take(sizeof(BkState)), o_vT = take(es * nnz),
                 o_vT64 = take(res64 && DT != LSQ_F64 ? 8 * nnz : 16), o_vec = take(8 * (size_t)nK * 10),
                 o_q = take(8 * (size_t)m * K), o_b = take(B ? 8 * (size_t)m * K : 16),
                 o_part = take(8 * (size_t)2 * grid_cap * K), o_n2 = take(8 * 2 * BK_MAX),
                 o_flag = take(4 * (size_t)2 * n), o_pbar = take(8), o_pout = take(sizeof(BkPersistOut));
    Scratch sc;
    LSQ_CUDA(sc.alloc(off, st));
    char* base = sc.as<char>();
    BkState* S = (BkState*)(base + o_S);
    double* vec = (double*)(base + o_vec);
    BkArgs a{};
    a.max_polls = dep_wait_polls();
    a.m = m; a.n = n; a.K = K; a.GK = GK;
    a.row_ptr = A->row_ptr; a.col_idx = A->col_idx; a.vals = A->vals;
    a.vals_res = res64 ? (DT == LSQ_F64 ? A->vals : (const void*)A->vals_f64) : A->vals;
    a.atptr = SH->atptr; a.atrow = SH->atrow;
    a.valsT = base + o_vT;
    a.valsT_res = res64 ? (DT == LSQ_F64 ? a.valsT : (const void*)(base + o_vT64)) : a.valsT;
    a.inv_d = P->inv_d;
    a.b = B ? (const double*)(base + o_b) : nullptr;
    a.mptr = SH->mptr; a.mcol = SH->mcol; a.mdiag = SH->mdiag;
    a.mval = P->op_dtype == LSQ_F32 ? (const void*)SH->mval32 : (const void*)SH->mval;
    a.dinv = SH->dinv; a.sched_f = SH->sched_f; a.sched_b = SH->sched_b;
    a.sweeps = P->sweeps;
    a.rflag_f = (unsigned*)(base + o_flag); a.rflag_b = a.rflag_f + n;
    a.y = vec; a.g = vec + nK; a.z = vec + 2 * nK; a.p = vec + 3 * nK; a.pt = vec + 4 * nK;
    a.w = vec + 5 * nK; a.e0 = vec + 6 * nK; a.e1 = vec + 7 * nK; a.h = vec + 8 * nK;
    double* tmpv = vec + 9 * nK;
    a.q = (double*)(base + o_q);
    a.part = (double*)(base + o_part);
    a.S = S;
    a.tol = o->tol; a.inner_tol = o->inner_tol > 0 ? o->inner_tol : 0.0; a.maxit = o->maxit;
    double* n2 = (double*)(base + o_n2);
    // A^T values in column order; the right-hand sides row-major
    if (DT == LSQ_F32X2) k_bk_gather_pairs<<<bk_grid(nnz, 4096), BK_T, 0, st>>>((const float*)A->vals, SH->atperm, nnz, (float*)(base + o_vT));
    else if (es == 8) k_bk_gather<double><<<bk_grid(nnz, 4096), BK_T, 0, st>>>(A->vals, SH->atperm, nnz, base + o_vT);
    else if (es == 4) k_bk_gather<float><<<bk_grid(nnz, 4096), BK_T, 0, st>>>(A->vals, SH->atperm, nnz, base + o_vT);
    else k_bk_gather<__nv_bfloat16><<<bk_grid(nnz, 4096), BK_T, 0, st>>>(A->vals, SH->atperm, nnz, base + o_vT);
    count_launch();
    if (res64 && DT != LSQ_F64) {
        k_bk_gather<double><<<bk_grid(nnz, 4096), BK_T, 0, st>>>(A->vals_f64, SH->atperm, nnz, base + o_vT64);
        count_launch();
    }
    if (B) {
        k_bk_to_rows<<<bk_grid(m * K, 4096), BK_T, 0, st>>>(B, ldb, m, K, (double*)(base + o_b));
        count_launch();
    }
    const unsigned grows = bk_grid(m * GK, grid_cap), gcols = bk_grid(n * GK, grid_cap), gvec = bk_grid(n * GK, 152 * 4);
    auto rows = [&](int mode, int use_res, const double* x) {
        if (use_res && res64) k_bk_rows<LSQ_F64><<<grows, BK_T, 0, st>>>(a, mode, 1, x);
        else k_bk_rows<DT><<<grows, BK_T, 0, st>>>(a, mode, 0, x);
        count_launch();
    };
    auto cols = [&](int use_res, double* dst) {
        if (use_res && res64) k_bk_cols<LSQ_F64><<<gcols, BK_T, 0, st>>>(a, 1, dst);
        else k_bk_cols<DT><<<gcols, BK_T, 0, st>>>(a, 0, dst);
        count_launch();
    };
    // the sweep form follows the mean length of a row's dependency side: lane per column up to
    // 24 entries, lane per entry up to 96, a CTA per row beyond
    const double dep = (double)(SH->nnz_M - n) / (2.0 * (double)n);
    const int smode = dep > 96.0 ? 2 : (dep > 24.0 ? 1 : 0);
    const bool m32 = P->op_dtype == LSQ_F32;
    // one cluster on request (lsq_set_sweep_form 3) where the block vector fits in the
    // cluster's shared memory; the stream-ordered solve only (the persistent kernel keeps the
    // grid forms).  Never chosen by shape: on the 1e6 x 1e4 workload with 16 columns (1227
    // levels of ~8 rows with ~350 dependency entries) the solve took 686 ms against 395 ms with
    // the CTA-per-row grid form.
    const int form = sweep_form_setting();
    const void* cf = m32 ? bk_sweep_cl_kernel<float, true>(K) : bk_sweep_cl_kernel<double, true>(K);
    const void* cb = m32 ? bk_sweep_cl_kernel<float, false>(K) : bk_sweep_cl_kernel<double, false>(K);
    auto want_cl = [&](int64_t nlev) {
        (void)nlev;
        return form == 3 && bk_cl_smem(n, K) <= BC_SMEM;
    };
    const bool cl_f = want_cl(SH->nlev_f) && bk_cluster_fits(cf);
    const bool cl_b = want_cl(SH->nlev_b) && bk_cluster_fits(cb);
    // FP32 M with the CTA-per-row form: double-float sums on float-pair sweep vectors, the
    // last sweep also writing z in FP64 (a dependent FP64 step costs ~64 cycles on GB300);
    // the cluster and persistent forms keep FP64 sums
    const bool pairs = m32 && smode == 2 && !cl_f && !cl_b;
    const void* kf = pairs ? bk_sweep_kernel<float, true, true>(smode, K)
                           : (m32 ? bk_sweep_kernel<float, true>(smode, K) : bk_sweep_kernel<double, true>(smode, K));
    const void* kb = pairs ? bk_sweep_kernel<float, false, true>(smode, K)
                           : (m32 ? bk_sweep_kernel<float, false>(smode, K) : bk_sweep_kernel<double, false>(smode, K));
    lsq_status sweep_status = LSQ_OK;
    auto sweep = [&](bool fwd, const double* r, const double* eold, double* enew, double* out64, int identity,
                     int idx) {
        lsq_status q;
        if (fwd && cl_f) q = bk_launch_sweep_cl(cf, a, r, eold, enew, identity, SH->loff_f, SH->nlev_f, st);
        else if (!fwd && cl_b) q = bk_launch_sweep_cl(cb, a, r, eold, enew, identity, SH->loff_b, SH->nlev_b, st);
        else q = bk_launch_sweep(fwd ? kf : kb, a, r, eold, enew, out64, identity, idx,
                                 fwd ? SH->nlev_f : SH->nlev_b, smode == 2 ? 1 : BK_T / 32, st);
        if (q != LSQ_OK) sweep_status = q;
    };
    // z = P g: t forward then t backward sweeps
    auto precond = [&]() {
        if (P->sweeps == 0) {   // the comparison method: P = I
            const cudaError_t ce = cudaMemcpyAsync(a.z, a.g, 8 * (size_t)nK, cudaMemcpyDeviceToDevice, st);
            if (ce != cudaSuccess) {
                set_error(std::string("cudaMemcpyAsync: ") + cudaGetErrorString(ce));
                sweep_status = LSQ_ERR_CUDA;
            }
            return;
        }
        const double* eold = nullptr;
        double* bufs[2] = {a.e0, a.e1};
        int cur = 0, idx = 0;
        for (int t = 0; t < P->sweeps; ++t, ++idx) {
            sweep(true, a.g, eold, bufs[cur], nullptr, 0, idx);
            eold = bufs[cur];
            cur ^= 1;
        }
        for (int t = 0; t < P->sweeps; ++t, ++idx) {
            const bool last = t == P->sweeps - 1;
            double* dst = (last && !pairs) ? a.z : bufs[cur];
            sweep(false, a.g, eold, dst, (last && pairs) ? a.z : nullptr, (P->sweeps == 1) ? 1 : 0, idx);
            eold = dst;
            cur ^= 1;
        }
    };
    double gn[BK_MAX], gn_raw[BK_MAX];
    auto norms = [&](const double* x) -> lsq_status {
        k_bk_norms<<<gvec, BK_T, 0, st>>>(a, x, n2);
        count_launch();
        double hb[2 * BK_MAX];
        LSQ_CUDA(cudaMemcpyAsync(hb, n2, sizeof(hb), cudaMemcpyDeviceToHost, st));
        LSQ_CUDA(cudaStreamSynchronize(st));
        for (int c = 0; c < K; ++c) { gn[c] = std::sqrt(hb[c]); gn_raw[c] = std::sqrt(hb[BK_MAX + c]); }
        return LSQ_OK;
    };
    LSQ_CUDA(cudaMemsetAsync(S, 0, sizeof(BkState), st));
    LSQ_CUDA(cudaMemsetAsync(a.rflag_f, 0, 4 * (size_t)2 * n, st));
    LSQ_CUDA(cudaMemsetAsync(a.y, 0, 8 * (size_t)nK, st));
    if ((DT == LSQ_F64 || DT == LSQ_F32) && (capturing || o->device_loop == 1)) {
        // the whole solve in one persistent kernel: no host decision, no synchronisation
        // until the results are read (none at all under stream capture)
        unsigned long long* pbar = (unsigned long long*)(base + o_pbar);
        BkPersistOut* pout = (BkPersistOut*)(base + o_pout);
        LSQ_CUDA(cudaMemsetAsync(pbar, 0, 8, st));
        if (Hcols) {
            k_bk_to_rows<<<bk_grid(nK, 4096), BK_T, 0, st>>>(Hcols, ldb, n, K, a.h);
            count_launch();
        }
        lsq_status lr = bk_persist_launch(DT, m32 ? 1 : 0, a, pbar, n2, tmpv, X, ldx, pout, Hcols ? 1 : 0,
                                          res64 ? 1 : 0, smode, o->max_outer, st);
        if (lr != LSQ_OK) return lr;
        LSQ_CUDA(cudaGetLastError());
        if (capturing) {
            for (int c = 0; c < K; ++c) out->status[c] = LSQ_OK;
            return LSQ_OK;
        }
        BkPersistOut ho;
        unsigned herr = 0;
        LSQ_CUDA(cudaMemcpyAsync(&ho, pout, sizeof(ho), cudaMemcpyDeviceToHost, st));
        LSQ_CUDA(cudaMemcpyAsync(&herr, &S->err, sizeof(herr), cudaMemcpyDeviceToHost, st));
        LSQ_CUDA(cudaStreamSynchronize(st));
        if (herr) { set_error("block PCG: a device wait timed out"); return LSQ_ERR_TIMEOUT; }
        for (int c = 0; c < K; ++c) {
            out->iters[c] = ho.iters[c]; out->outer[c] = ho.outer[c]; out->conv[c] = (uint8_t)ho.conv[c];
            out->rec[c] = ho.rec[c]; out->tru[c] = ho.tru[c]; out->raw[c] = ho.raw[c];
            out->status[c] = (lsq_status)ho.status[c];
        }
        return LSQ_OK;
    }
    if (Hcols) {
        k_bk_to_rows<<<bk_grid(nK, 4096), BK_T, 0, st>>>(Hcols, ldb, n, K, a.h);
        count_launch();
    } else {
        rows(1, 1, a.pt);
        cols(1, a.h);
    }
    LSQ_CUDA(cudaMemcpyAsync(a.g, a.h, 8 * (size_t)nK, cudaMemcpyDeviceToDevice, st));
    lsq_status r0 = norms(a.h);
    if (r0 != LSQ_OK) return r0;
    double hn[BK_MAX], hn_raw[BK_MAX];
    for (int c = 0; c < K; ++c) { hn[c] = gn[c]; hn_raw[c] = gn_raw[c]; }
    int iters[BK_MAX] = {}, outer_used[BK_MAX] = {}, conv[BK_MAX] = {}, broke[BK_MAX] = {};
    bool dirty[BK_MAX] = {};
    double rec[BK_MAX], tru[BK_MAX], raw[BK_MAX];
    int napply = 0;
    auto true_residual = [&]() -> lsq_status {
        LSQ_CUDA(cudaMemsetAsync(&S->done, 0, sizeof(int32_t), st));
        k_bk_scale<<<bk_grid(nK, 4096), BK_T, 0, st>>>(a.y, n, K, a.inv_d, tmpv);
        count_launch();
        if (Hcols) {
            rows(0, 1, tmpv);
            cols(1, a.w);
            k_bk_diff<<<bk_grid(nK, 4096), BK_T, 0, st>>>(a.h, a.w, a.g, nK);
            count_launch();
        } else {
            rows(2, 1, tmpv);
            cols(1, a.g);
        }
        for (int c = 0; c < K; ++c) dirty[c] = false;
        return norms(a.g);
    };
    for (int c = 0; c < K; ++c) {
        rec[c] = tru[c] = raw[c] = 1.0;
        if (hn[c] == 0.0) { conv[c] = 1; rec[c] = tru[c] = raw[c] = 0.0; }
    }
    for (int outer = 0; outer < o->max_outer; ++outer) {
        if (outer > 0) {
            lsq_status rs = true_residual();
            if (rs != LSQ_OK) return rs;
        }
        BkState init{};
        int nact = 0;
        for (int c = 0; c < K; ++c) {
            init.hn[c] = hn[c] > 0.0 ? hn[c] : 1.0;
            if (hn[c] == 0.0 || broke[c]) continue;
            tru[c] = gn[c] / hn[c];
            raw[c] = hn_raw[c] > 0.0 ? gn_raw[c] / hn_raw[c] : 0.0;
            if (outer == 0) rec[c] = tru[c];
            if (tru[c] <= o->tol) { conv[c] = 1; continue; }
            if (iters[c] >= o->maxit) continue;
            init.active[c] = 1;
            init.gstart[c] = gn[c];
            outer_used[c] = outer + 1;
            ++nact;
        }
        if (nact == 0) break;
        for (int c = 0; c < K; ++c) { init.iters[c] = iters[c]; init.rec[c] = rec[c]; }
        init.napply = napply;
        LSQ_CUDA(cudaMemcpyAsync(S, &init, sizeof(BkState), cudaMemcpyHostToDevice, st));
        // z = P g, rho = g^T z, p = z
        precond();
        k_bk_gz<<<gvec, BK_T, 0, st>>>(a, 1);
        k_bk_pnext<<<gvec, BK_T, 0, st>>>(a);
        count_launch(2);
        BkState hs{};
        while (true) {
            for (int b = 0; b < 8; ++b) {
                rows(0, 0, a.pt);
                cols(0, a.w);
                k_bk_update<<<gvec, BK_T, 0, st>>>(a);
                precond();
                k_bk_gz<<<gvec, BK_T, 0, st>>>(a, 0);
                k_bk_pnext<<<gvec, BK_T, 0, st>>>(a);
                count_launch(3);
            }
            if (sweep_status != LSQ_OK) return sweep_status;
            LSQ_CUDA(cudaGetLastError());
            LSQ_CUDA(cudaMemcpyAsync(&hs, S, sizeof(BkState), cudaMemcpyDeviceToHost, st));
            LSQ_CUDA(cudaStreamSynchronize(st));
            if (hs.err) { set_error("block Gauss-Seidel sweep: a level wait timed out"); return LSQ_ERR_TIMEOUT; }
            if (hs.done) break;
        }
        for (int c = 0; c < K; ++c) {
            if (!init.active[c]) continue;
            if (hs.iters[c] > iters[c]) dirty[c] = true;
            iters[c] = hs.iters[c];
            rec[c] = hs.rec[c];
            if (hs.broke[c]) broke[c] = 1;
        }
        napply = hs.napply;
    }
    bool was[BK_MAX];
    bool any_dirty = false;
    for (int c = 0; c < K; ++c) {
        was[c] = dirty[c] && !broke[c] && !conv[c];
        any_dirty = any_dirty || was[c];
    }
    if (any_dirty) {
        lsq_status rs = true_residual();
        if (rs != LSQ_OK) return rs;
        for (int c = 0; c < K; ++c) {
            if (!was[c]) continue;
            tru[c] = gn[c] / hn[c];
            raw[c] = hn_raw[c] > 0.0 ? gn_raw[c] / hn_raw[c] : 0.0;
            if (tru[c] <= o->tol) conv[c] = 1;
        }
    }
    k_bk_from_rows<<<bk_grid(nK, 4096), BK_T, 0, st>>>(a.y, n, K, a.inv_d, X, ldx);
    count_launch();
    LSQ_CUDA(cudaGetLastError());
    LSQ_CUDA(cudaStreamSynchronize(st));
    for (int c = 0; c < K; ++c) {
        out->iters[c] = iters[c]; out->outer[c] = outer_used[c]; out->conv[c] = (uint8_t)conv[c];
        out->rec[c] = rec[c]; out->tru[c] = tru[c]; out->raw[c] = raw[c];
        out->status[c] = conv[c] ? LSQ_OK : (broke[c] ? LSQ_ERR_BREAKDOWN : LSQ_ERR_NOT_CONVERGED);
    }
    return LSQ_OK;
}

lsq_status sparse_block_solve(const lsq_matrix* A, const lsq_precond* P, const double* B, const double* Hcols,
                              int64_t k, int64_t ldb, double* X, int64_t ldx, const lsq_opts* o, lsq_info* info,
                              cudaStream_t st) {
    LSQ_CHECK_ARG(P->sp != nullptr, "preconditioner was built for a dense matrix");
    LSQ_CHECK_ARG(P->sp->nnz_A == A->nnz && P->sp->m == A->m, "preconditioner was built for another pattern");
    LSQ_CHECK_ARG(P->sweeps <= 32, "sparse sweeps must be <= 32");
    // under stream capture nothing may wait for the device: no timing events, no results
    // read back (the graph writes X; per-column results are not reported)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    LSQ_CUDA(cudaStreamIsCapturing(st, &cap));
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    if (capturing && !(A->dtype == LSQ_F64 || A->dtype == LSQ_F32)) {
        set_error("stream capture of a CSR block solve needs FP64 or FP32 values");
        return LSQ_ERR_UNSUPPORTED;
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (!capturing) {
        LSQ_CUDA(cudaEventCreate(&ev0));
        LSQ_CUDA(cudaEventCreate(&ev1));
        LSQ_CUDA(cudaEventRecord(ev0, st));
    }
    lsq_status worst = LSQ_OK;
    for (int64_t c0 = 0; c0 < k; c0 += BK_MAX) {
        const int K = (int)std::min<int64_t>(BK_MAX, k - c0);
        BkOut bo{};
        const double* Bc = B ? B + c0 * ldb : nullptr;
        const double* Hc = Hcols ? Hcols + c0 * ldb : nullptr;
        double* Xc = X + c0 * ldx;
        lsq_status r;
        switch (A->dtype) {
            case LSQ_F64: r = bk_solve_impl<LSQ_F64>(A, P, Bc, Hc, K, ldb, Xc, ldx, o, &bo, capturing, st); break;
            case LSQ_F32: r = bk_solve_impl<LSQ_F32>(A, P, Bc, Hc, K, ldb, Xc, ldx, o, &bo, capturing, st); break;
            case LSQ_BF16: r = bk_solve_impl<LSQ_BF16>(A, P, Bc, Hc, K, ldb, Xc, ldx, o, &bo, capturing, st); break;
            default: r = bk_solve_impl<LSQ_F32X2>(A, P, Bc, Hc, K, ldb, Xc, ldx, o, &bo, capturing, st); break;
        }
        if (r != LSQ_OK) return r;
        if (capturing) continue;
        for (int c = 0; c < K; ++c) {
            const int64_t at = c0 + c;
            if (info && at < info->k) {
                if (info->iters) info->iters[at] = bo.iters[c];
                if (info->outer) info->outer[at] = bo.outer[c];
                if (info->converged) info->converged[at] = bo.conv[c];
                if (info->relres_rec) info->relres_rec[at] = bo.rec[c];
                if (info->relres_true) info->relres_true[at] = bo.tru[c];
                if (info->relres_raw) info->relres_raw[at] = bo.raw[c];
            }
            if (bo.status[c] == LSQ_ERR_BREAKDOWN) worst = LSQ_ERR_BREAKDOWN;
            else if (bo.status[c] != LSQ_OK && worst == LSQ_OK) worst = bo.status[c];
        }
    }
    if (capturing) return LSQ_OK;
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
    if (worst == LSQ_ERR_NOT_CONVERGED) set_error("PCG did not reach the tolerance");
    if (worst == LSQ_ERR_BREAKDOWN) set_error("PCG breakdown (non-positive or non-finite curvature)");
    return worst;
}

}  // namespace lsq
