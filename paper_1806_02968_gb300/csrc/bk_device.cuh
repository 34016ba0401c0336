// Device code of the CSR block PCG (K <= 32 right-hand sides advanced together): argument
// and state structs, fixed-order reductions, and the body of every step of an iteration as a
// device function.  The stream-ordered kernels of pcg_sparse_block.cu wrap one body each;
// the persistent kernel of pcg_sparse_persist.cu calls them in turn between grid barriers.
#pragma once
#include "sparse.cuh"
#include "values.cuh"
#include "dfloat.cuh"

#include <type_traits>

namespace lsq {

constexpr int BK_T = 256;
constexpr int BK_MAX = 32;
constexpr int BK_PF = 8;       // dependency entries per lane loaded before a level wait

struct BkState {
    double rho[BK_MAX], hn[BK_MAX], gstart[BK_MAX], rec[BK_MAX];
    double pw[BK_MAX], beta[BK_MAX];
    int32_t iters[BK_MAX];
    int32_t active[BK_MAX];    // column still iterating in this inner solve
    int32_t broke[BK_MAX];     // breakdown (non-positive or non-finite curvature)
    int32_t done, napply;
    unsigned err;
    unsigned arrive[4];        // last-block counters: rows, update, gz, norms
};

struct BkArgs {
    int64_t m, n;
    int K, GK;
    const int64_t* row_ptr;
    const int32_t* col_idx;
    const void* vals;
    const void* vals_res;
    const int64_t* atptr;
    const int32_t* atrow;
    const void* valsT;
    const void* valsT_res;
    const double* inv_d;
    const double* b;          // m x K row-major (least-squares form) or NULL
    const int64_t* mptr;
    const int32_t* mcol;
    const void* mval;
    const int64_t* mdiag;
    const double* dinv;
    const int32_t* sched_f;
    const int32_t* sched_b;
    int sweeps;
    unsigned* rflag_f;        // CTA-per-row form: sweep epoch at which each row's values were written
    unsigned* rflag_b;
    double *y, *g, *z, *p, *pt, *w, *q, *e0, *e1, *h;
    double* part;             // per-block partials, [blocks][K] (x2 for the norms)
    BkState* S;
    double tol, inner_tol;
    int32_t maxit;
    unsigned max_polls = 1u << 22;   // bound of every dependency wait
};

// Thread t holds v for column t % GK; out[c] = that column's sum over the block (fixed order).
__device__ __forceinline__ void bk_block_partials(double v, int K, int GK, double* out, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    if ((int)threadIdx.x < K) {
        double t = 0.0;
        for (int i = threadIdx.x; i < (int)blockDim.x; i += GK) t += sh[i];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}
// After every block has written its partials: true in the one block that arrived last
// (the partials of all blocks are then visible to it).
__device__ __forceinline__ bool bk_last_block(unsigned* counter) {
    __shared__ unsigned s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        s_last = (t == gridDim.x - 1) ? 1u : 0u;
        if (s_last) *counter = 0;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}
// sh[c] = sum over blocks b of part[b*K + c], in a fixed order (a warp per column)
__device__ __forceinline__ void bk_total(const double* part, int nparts, int K, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c = wid; c < K; c += blockDim.x >> 5) {
        double t = 0.0;
        for (int b = lane; b < nparts; b += 32) t += __ldcg(part + (int64_t)b * K + c);
        t = warp_sum(t);
        if (lane == 0) sh[c] = t;
    }
    __syncthreads();
}

// q_i = A_i x, b_i, or b_i - A_i x (mode 0/1/2) for every column; the last block leaves the
// column sums of ||q||^2 in S->pw.  A lane group takes 4 consecutive rows and walks their
// entries flat, 4 at a time, so that several gathers are in flight; each row still sums its
// entries in order.
template <int DT>
__device__ __forceinline__ void bk_rows_body(BkArgs a, int mode, int use_res, const double* x) {
    __shared__ double sh[BK_T];
    const void* vals = use_res ? a.vals_res : a.vals;
    const int c = threadIdx.x & (a.GK - 1);
    const bool col_ok = c < a.K;
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / a.GK;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / a.GK;
    const int K = a.K;
    double qq = 0.0;
    if (col_ok)
        for (int64_t i0 = grp * 4; i0 < a.m; i0 += ngrp * 4) {
            const int nr = (int)min((int64_t)4, a.m - i0);
            int64_t rp[5];
#pragma unroll
            for (int r = 0; r < 5; ++r) rp[r] = a.row_ptr[min(i0 + r, a.m)];
            double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
            if (mode != 1) {
                const int64_t eend = rp[nr];
                for (int64_t e = rp[0]; e < eend; e += 4) {
                    int32_t col[4];
                    double v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        col[u] = 0;
                        v[u] = 0.0;
                        if (e + u < eend) { col[u] = a.col_idx[e + u]; v[u] = Val<DT>::load(vals, e + u); }
                    }
                    double xv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) xv[u] = (e + u < eend) ? x[(int64_t)col[u] * K + c] : 0.0;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int64_t ee = e + u;
                        if (ee < eend) {
                            const int r = (ee >= rp[1]) + (ee >= rp[2]) + (ee >= rp[3]);
                            if (r == 0) d0 = fma(v[u], xv[u], d0);
                            else if (r == 1) d1 = fma(v[u], xv[u], d1);
                            else if (r == 2) d2 = fma(v[u], xv[u], d2);
                            else d3 = fma(v[u], xv[u], d3);
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (r < nr) {
                    const int64_t i = i0 + r;
                    const double dot = r == 0 ? d0 : (r == 1 ? d1 : (r == 2 ? d2 : d3));
                    const double bi = mode == 0 ? 0.0 : a.b[i * K + c];
                    const double qv = mode == 0 ? dot : (mode == 1 ? bi : bi - dot);
                    a.q[i * K + c] = qv;
                    qq = fma(qv, qv, qq);
                }
            }
        }
    bk_block_partials(qq, a.K, a.GK, a.part + (int64_t)blockIdx.x * a.K, sh);
    if (!bk_last_block(&a.S->arrive[0])) return;
    bk_total(a.part, gridDim.x, a.K, sh);
    if ((int)threadIdx.x < a.K) a.S->pw[threadIdx.x] = sh[threadIdx.x];
}

// out_j = (1/d_j) A^T_j q for every column (the transposed pattern; no atomics); entries are
// loaded 4 at a time before their gathers
template <int DT>
__device__ __forceinline__ void bk_cols_body(BkArgs a, int use_res, double* out) {
    const void* vals = use_res ? a.valsT_res : a.valsT;
    const int c = threadIdx.x & (a.GK - 1);
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / a.GK;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / a.GK;
    const int K = a.K;
    if (c >= K) return;
    for (int64_t j = grp; j < a.n; j += ngrp) {
        double t = 0.0;
        const int64_t eend = a.atptr[j + 1];
        for (int64_t e = a.atptr[j]; e < eend; e += 4) {
            int32_t row[4];
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                row[u] = 0;
                v[u] = 0.0;
                if (e + u < eend) { row[u] = a.atrow[e + u]; v[u] = Val<DT>::load(vals, e + u); }
            }
            double qv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) qv[u] = (e + u < eend) ? a.q[(int64_t)row[u] * K + c] : 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (e + u < eend) t = fma(v[u], qv[u], t);
        }
        out[j * K + c] = t * a.inv_d[j];
    }
}

// alpha_c = rho_c / p_c^T w_c (0 for frozen columns), y += alpha p, g -= alpha w.  The last
// block sums ||g||^2, counts the iteration of every active column and freezes the columns
// that met the tolerance or maxit; S->done once none is left.
__device__ __forceinline__ void bk_update_body(BkArgs a) {
    __shared__ double sh[BK_T];
    __shared__ double s_alpha[BK_MAX];
    __shared__ int s_any;
    if ((int)threadIdx.x < a.K) {
        const int c = threadIdx.x;
        const double pw = a.S->pw[c], rho = a.S->rho[c];
        const bool ok = pw > 0.0 && rho > 0.0 && isfinite(pw) && isfinite(rho);
        s_alpha[c] = (a.S->active[c] && ok) ? rho / pw : 0.0;
    }
    __syncthreads();
    const int c = threadIdx.x & (a.GK - 1);
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / a.GK;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / a.GK;
    double gg = 0.0;
    if (c < a.K) {
        const double al = s_alpha[c];
        for (int64_t j = grp; j < a.n; j += ngrp) {
            const int64_t at = j * a.K + c;
            a.y[at] = fma(al, a.p[at], a.y[at]);
            const double gj = fma(-al, a.w[at], a.g[at]);
            a.g[at] = gj;
            gg = fma(gj, gj, gg);
        }
    }
    bk_block_partials(gg, a.K, a.GK, a.part + (int64_t)blockIdx.x * a.K, sh);
    if (!bk_last_block(&a.S->arrive[1])) return;
    bk_total(a.part, gridDim.x, a.K, sh);
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    if ((int)threadIdx.x < a.K) {
        const int cc = threadIdx.x;
        if (a.S->active[cc]) {
            const double pw = a.S->pw[cc], rho = a.S->rho[cc];
            if (!(pw > 0.0 && rho > 0.0 && isfinite(pw) && isfinite(rho))) {
                a.S->broke[cc] = 1;
                a.S->active[cc] = 0;
            } else {
                a.S->iters[cc] += 1;
                const double gn = sqrt(sh[cc]);
                a.S->rec[cc] = gn / a.S->hn[cc];
                if (gn <= a.tol * a.S->hn[cc] || gn <= a.inner_tol * a.S->gstart[cc] || a.S->iters[cc] >= a.maxit)
                    a.S->active[cc] = 0;
            }
        }
        if (a.S->active[cc]) atomicOr(&s_any, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0 && !s_any) a.S->done = 1;
}

// Gauss-Seidel sweeps of Alg. 3 for all K columns, with the values themselves as completion
// flags: before a sweep every entry of e_new holds BK_EMPTY, a signalling NaN that no
// arithmetic produces; a row polls the values it depends on (volatile loads, issued in
// batches, bounded) until none is BK_EMPTY, then stores its own.  Rows run in level order over
// a cooperative grid, so every wait ends; a row waits for its real dependencies only.  One
// failed wait sets the error word, which every wait checks, so a failure ends the launch within
// one wait bound.  Rows are sorted and hold their diagonal: the dependency side (lower entries
// forward, upper backward) and the other side are the two ranges around it.  `identity`: the
// backward sweep right after one forward sweep from zero (e_new = e_old - upper terms / M_jj).
constexpr unsigned long long BK_EMPTY = 0xFFF7DEADBEEFCAFEull;
__device__ __forceinline__ void bk_fill_empty_body(double* e, int64_t cnt) {
    unsigned long long* u = reinterpret_cast<unsigned long long*>(e);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x)
        u[t] = BK_EMPTY;
}
__device__ __forceinline__ unsigned bk_ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void bk_st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long bk_ldv(const double* p) {
    unsigned long long v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void bk_stv(double* p, double v) {
    asm volatile("st.volatile.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
// Loads N values (use[i] false: skipped), polling the missing ones until all are written;
// called by all 32 lanes of a warp together.
template <int N>
__device__ __forceinline__ bool bk_gather_ready(const double* const* ptr, const bool* use, double* out,
                                                unsigned* err, unsigned max_polls) {
    unsigned long long u[N];
#pragma unroll
    for (int i = 0; i < N; ++i) u[i] = use[i] ? bk_ldv(ptr[i]) : 0ull;
    // warp-collective: every lane of the warp calls this together and the warp leaves the wait
    // as one (__any_sync), converged for the shuffles that follow
    unsigned polls = 0, ns = 32;
    bool ok = true;
    while (true) {
        bool missing = false;
#pragma unroll
        for (int i = 0; i < N; ++i) missing = missing || (use[i] && u[i] == BK_EMPTY);
        if (!__any_sync(0xffffffffu, missing)) break;
        ++polls;
        const bool give_up = polls > max_polls || ((polls & 255u) == 0 && *(volatile unsigned*)err != 0u);
        if (__any_sync(0xffffffffu, give_up)) {
            if ((threadIdx.x & 31) == 0) atomicOr(err, DEV_ERR_TIMEOUT);
            ok = false;
#pragma unroll
            for (int i = 0; i < N; ++i) if (u[i] == BK_EMPTY) u[i] = 0ull;
            break;
        }
        if (polls > 4) { __nanosleep(ns); ns = ns < 256 ? 2 * ns : 256; }
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (use[i] && u[i] == BK_EMPTY) u[i] = bk_ldv(ptr[i]);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = use[i] ? __longlong_as_double((long long)u[i]) : 0.0;
    return ok;
}

// Short rows: a warp takes a row; its entries are loaded 32 at a time and broadcast by
// shuffles, 8 gathers in flight per lane; lane c accumulates column c.
template <typename MT, bool FWD>
__device__ __forceinline__ void bk_sweep_body(BkArgs a, const double* r, const double* e_old,
                                                   double* e_new, int identity, int sweep_idx) {
    const int32_t* sched = FWD ? a.sched_f : a.sched_b;
    const MT* mv = reinterpret_cast<const MT*>(a.mval);
    const int lane = threadIdx.x & 31;
    const int K = a.K;
    const bool col_ok = lane < K;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool other = !identity && e_old != nullptr;
    (void)sweep_idx;
    for (int64_t slot = gw; slot < a.n; slot += W) {
        const int64_t j = sched[slot];
        const int64_t e0 = a.mptr[j], e1 = a.mptr[j + 1], ed = a.mdiag[j];
        const int64_t d0 = FWD ? e0 : ed + 1, d1 = FWD ? ed : e1;
        const int64_t o0 = FWD ? ed + 1 : e0, o1 = FWD ? e1 : ed;
        double acc = 0.0;
        if (other) {   // previous sweep's values on the other side: complete already
            for (int64_t base = o0; base < o1; base += 32) {
                const int64_t e = base + lane;
                int32_t kk = 0;
                double mm = 0.0;
                if (e < o1) { kk = a.mcol[e]; mm = (double)mv[e]; }
                const int cnt = (int)min((int64_t)32, o1 - base);
                for (int t = 0; t < cnt; ++t) {
                    const int32_t k = __shfl_sync(0xffffffffu, kk, t);
                    const double mk = __shfl_sync(0xffffffffu, mm, t);
                    if (col_ok) acc = fma(mk, e_old[(int64_t)k * K + lane], acc);
                }
            }
        }
        for (int64_t base = d0; base < d1; base += 32) {
            const int64_t e = base + lane;
            int32_t kk = 0;
            double mm = 0.0;
            if (e < d1) { kk = a.mcol[e]; mm = (double)mv[e]; }
            const int cnt = (int)min((int64_t)32, d1 - base);
            for (int t0 = 0; t0 < cnt; t0 += 8) {
                const double* ptr[8];
                bool use[8];
                double mk[8], val[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int t = (t0 + i) & 31;
                    const int32_t k = __shfl_sync(0xffffffffu, kk, t);
                    mk[i] = __shfl_sync(0xffffffffu, mm, t);
                    use[i] = col_ok && t0 + i < cnt;
                    ptr[i] = e_new + (int64_t)k * K + lane;
                }
                bk_gather_ready<8>(ptr, use, val, &a.S->err, a.max_polls);
#pragma unroll
                for (int i = 0; i < 8; ++i) acc = fma(mk[i], val[i], acc);
            }
        }
        if (col_ok) {
            const double dj = a.dinv[j];
            const int64_t at = j * K + lane;
            bk_stv(e_new + at, identity ? e_old[at] - acc * dj : (r[at] - acc) * dj);
        }
        __syncwarp();
    }
}

// acc[0..KT) per lane -> lane l holds the warp total of column l >> (5 - log2 KT)
// (a butterfly reduce-scatter: each step halves the columns a lane keeps)
template <int KT>
__device__ __forceinline__ double bk_reduce_scatter(double (&v)[KT], int lane) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int o = 16 >> s;
        const int half = KT >> (s + 1);
        if (half >= 1) {
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < half; ++i) {
                const double send = upper ? v[i] : v[i + half];
                const double keep = upper ? v[i + half] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
    }
    return v[0];
}

// One dependency entry for KT column accumulators: its K contiguous values, polled until
// all are written.
template <typename MT, int KT>
__device__ __forceinline__ void bk_entry(const BkArgs& a, const double* e_new, int64_t e, double (&acc)[KT]) {
    const int K = a.K;
    const MT* mv = reinterpret_cast<const MT*>(a.mval);
    const double* row = e_new + (int64_t)a.mcol[e] * K;
    const double mk = (double)mv[e];
    unsigned long long u[KT];
#pragma unroll
    for (int c = 0; c < KT; ++c) u[c] = c < K ? bk_ldv(row + c) : 0ull;
    unsigned polls = 0, ns = 32;
    while (true) {
        bool missing = false;
#pragma unroll
        for (int c = 0; c < KT; ++c) missing = missing || (c < K && u[c] == BK_EMPTY);
        if (!missing) break;
        ++polls;
        if (polls > a.max_polls || ((polls & 255u) == 0 && *(volatile unsigned*)&a.S->err != 0u)) {
            atomicOr(&a.S->err, DEV_ERR_TIMEOUT);
#pragma unroll
            for (int c = 0; c < KT; ++c) if (u[c] == BK_EMPTY) u[c] = 0ull;
            break;
        }
        if (polls > 4) { __nanosleep(ns); ns = ns < 256 ? 2 * ns : 256; }
#pragma unroll
        for (int c = 0; c < KT; ++c)
            if (c < K && u[c] == BK_EMPTY) u[c] = bk_ldv(row + c);
    }
#pragma unroll
    for (int c = 0; c < KT; ++c)
        if (c < K) acc[c] = fma(mk, __longlong_as_double((long long)u[c]), acc[c]);
}

// Long rows: lanes take the row's entries (lane l: entries l, l + 32, ...) and keep KT column
// accumulators; one reduce-scatter per row combines them.
template <typename MT, bool FWD, int KT>
__device__ __forceinline__ void bk_sweep_ep_body(BkArgs a, const double* r, const double* e_old,
                                                      double* e_new, int identity, int sweep_idx) {
    const int32_t* sched = FWD ? a.sched_f : a.sched_b;
    const MT* mv = reinterpret_cast<const MT*>(a.mval);
    const int lane = threadIdx.x & 31;
    const int K = a.K;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool other = !identity && e_old != nullptr;
    constexpr int SH = (KT >= 32) ? 0 : (KT >= 16 ? 1 : (KT >= 8 ? 2 : (KT >= 4 ? 3 : (KT >= 2 ? 4 : 5))));
    const int my_col = lane >> SH;
    const bool writer = (lane & ((1 << SH) - 1)) == 0 && my_col < K;
    (void)sweep_idx;
    for (int64_t slot = gw; slot < a.n; slot += W) {
        const int64_t j = sched[slot];
        const int64_t e0 = a.mptr[j], e1 = a.mptr[j + 1], ed = a.mdiag[j];
        const int64_t d0 = FWD ? e0 : ed + 1, d1 = FWD ? ed : e1;
        const int64_t o0 = FWD ? ed + 1 : e0, o1 = FWD ? e1 : ed;
        double acc[KT];
#pragma unroll
        for (int c = 0; c < KT; ++c) acc[c] = 0.0;
        if (other)
            for (int64_t e = o0 + lane; e < o1; e += 32) {
                const int64_t k = a.mcol[e];
                const double mk = (double)mv[e];
#pragma unroll
                for (int c = 0; c < KT; ++c)
                    if (c < K) acc[c] = fma(mk, e_old[k * K + c], acc[c]);
            }
        for (int64_t e = d0 + lane; e < d1; e += 32) bk_entry<MT, KT>(a, e_new, e, acc);
        const double tot = bk_reduce_scatter<KT>(acc, lane);
        if (writer) {
            const double dj = a.dinv[j];
            const int64_t at = j * K + my_col;
            bk_stv(e_new + at, identity ? e_old[at] - tot * dj : (r[at] - tot) * dj);
        }
        __syncwarp();
    }
}

// Very long rows: a whole CTA takes a row (CTA b: schedule slots b, b + G, ...); thread t takes
// entries t, t + 256, ... with KT column accumulators; the warps' reduce-scattered partials are
// added in warp order.  Here a row's K values are published by one flag per row (the sweep's
// epoch, release) after they are written, so a reader polls one flag per dependency (acquire,
// batched, bounded) and then loads the values; the flags are cumulative over the solve, so
// nothing is reset between sweeps.  PAIRS (FP32 M, stream-ordered solves): the sums run in
// double-float on the FP32 units and the sweep vectors hold (hi, lo) float pairs, with the
// last sweep also writing FP64 values to out64; otherwise FP64 sums on FP64 vectors.
constexpr int BK_PFC = 4;
__device__ __forceinline__ f2 bk_pair(unsigned long long u) {
    return f2{__uint_as_float((unsigned)u), __uint_as_float((unsigned)(u >> 32))};
}
__device__ __forceinline__ unsigned long long bk_bits(f2 v) {
    return (unsigned long long)__float_as_uint(v.hi) | ((unsigned long long)__float_as_uint(v.lo) << 32);
}
// acc += m v (float m, pair v) in the cascaded double-float form
__device__ __forceinline__ void bk_mad_pair(f2& acc, float m, f2 v) {
    float p, pe;
    two_prod(m, v.hi, p, pe);
    pe = fmaf(m, v.lo, pe);
    float s, e;
    two_sum(acc.hi, p, s, e);
    acc.hi = s;
    acc.lo += e + pe;
}
__device__ __forceinline__ f2 bk_mul_pair(f2 a, f2 b) {
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float hi = p + e;
    return f2{hi, e - (hi - p)};
}
// the pair form of bk_reduce_scatter: lane l ends with the warp total of column l >> (5 - log2 KT)
template <int KT>
__device__ __forceinline__ f2 bk_reduce_scatter_pair(f2 (&v)[KT], int lane) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int o = 16 >> s;
        const int half = KT >> (s + 1);
        if (half >= 1) {
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < half; ++i) {
                const f2 send = upper ? v[i] : v[i + half];
                f2 keep = upper ? v[i + half] : v[i];
                df_add(keep, df_shfl_xor(send, o));
                v[i] = keep;
            }
        } else {
            df_add(v[0], df_shfl_xor(v[0], o));
        }
    }
    return v[0];
}
template <typename MT, bool FWD, int KT, bool PAIRS = false>
__device__ __forceinline__ void bk_sweep_cta_body(BkArgs a, const double* r, const double* e_old,
                                                       double* e_new, int identity, int sweep_idx,
                                                       double* out64 = nullptr) {
    static_assert(!PAIRS || sizeof(MT) == 4, "float pairs need FP32 M");
    __shared__ double s_part[BK_T / 32][KT];
    const int tdir = FWD ? sweep_idx : sweep_idx - a.sweeps;
    const unsigned epoch = (unsigned)((unsigned long long)a.S->napply * a.sweeps + tdir + 1);
    unsigned* flag = FWD ? a.rflag_f : a.rflag_b;
    const int32_t* sched = FWD ? a.sched_f : a.sched_b;
    const MT* mv = reinterpret_cast<const MT*>(a.mval);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int K = a.K;
    const bool other = !identity && e_old != nullptr;
    constexpr int SH = (KT >= 32) ? 0 : (KT >= 16 ? 1 : (KT >= 8 ? 2 : (KT >= 4 ? 3 : (KT >= 2 ? 4 : 5))));
    typedef typename std::conditional<PAIRS, f2, double>::type Acc;
    const unsigned long long* eold_u = reinterpret_cast<const unsigned long long*>(e_old);
    const unsigned long long* enew_u = reinterpret_cast<const unsigned long long*>(e_new);
    for (int64_t slot = blockIdx.x; slot < a.n; slot += gridDim.x) {
        const int64_t j = sched[slot];
        const int64_t e0 = a.mptr[j], e1 = a.mptr[j + 1], ed = a.mdiag[j];
        const int64_t d0 = FWD ? e0 : ed + 1, d1 = FWD ? ed : e1;
        const int64_t o0 = FWD ? ed + 1 : e0, o1 = FWD ? e1 : ed;
        Acc acc[KT];
#pragma unroll
        for (int c = 0; c < KT; ++c) {
            if constexpr (PAIRS) acc[c] = f2{0.f, 0.f};
            else acc[c] = 0.0;
        }
        if (other)
            for (int64_t e = o0 + tid; e < o1; e += BK_T) {
                const int64_t k = a.mcol[e];
#pragma unroll
                for (int c = 0; c < KT; ++c)
                    if (c < K) {
                        if constexpr (PAIRS) bk_mad_pair(acc[c], (float)mv[e], bk_pair(eold_u[k * K + c]));
                        else acc[c] = fma((double)mv[e], e_old[k * K + c], acc[c]);
                    }
            }
        // batches from a CTA-uniform base, polled as a warp (__any_sync), so every warp leaves
        // the wait converged for its reduce-scatter; thread t still takes entries t, t + BK_T, ...
        for (int64_t bb = d0; bb < d1; bb += BK_T * BK_PFC) {
            int32_t kk[BK_PFC];
            MT mm[BK_PFC];
            unsigned f[BK_PFC];
#pragma unroll
            for (int u = 0; u < BK_PFC; ++u) {
                const int64_t e = bb + tid + (int64_t)BK_T * u;
                kk[u] = -1;
                mm[u] = MT(0);
                if (e < d1) { kk[u] = a.mcol[e]; mm[u] = mv[e]; }
            }
#pragma unroll
            for (int u = 0; u < BK_PFC; ++u) f[u] = kk[u] >= 0 ? bk_ld_acquire_u32(flag + kk[u]) : epoch;
            unsigned polls = 0, ns = 32;
            while (true) {
                bool missing = false;
#pragma unroll
                for (int u = 0; u < BK_PFC; ++u) missing = missing || f[u] < epoch;
                if (!__any_sync(0xffffffffu, missing)) break;
                ++polls;
                const bool give_up = polls > a.max_polls ||
                                     ((polls & 255u) == 0 && *(volatile unsigned*)&a.S->err != 0u);
                if (__any_sync(0xffffffffu, give_up)) {
                    if (lane == 0) atomicOr(&a.S->err, DEV_ERR_TIMEOUT);
                    break;
                }
                if (polls > 4) { __nanosleep(ns); ns = ns < 256 ? 2 * ns : 256; }
#pragma unroll
                for (int u = 0; u < BK_PFC; ++u)
                    if (f[u] < epoch) f[u] = bk_ld_acquire_u32(flag + kk[u]);
            }
#pragma unroll
            for (int u = 0; u < BK_PFC; ++u) {
                if (kk[u] >= 0) {
                    if constexpr (PAIRS) {
                        const unsigned long long* row = enew_u + (int64_t)kk[u] * K;
#pragma unroll
                        for (int c = 0; c < KT; ++c)
                            if (c < K) bk_mad_pair(acc[c], (float)mm[u], bk_pair(__ldcg(row + c)));
                    } else {
                        const double* row = e_new + (int64_t)kk[u] * K;
#pragma unroll
                        for (int c = 0; c < KT; ++c)
                            if (c < K) acc[c] = fma((double)mm[u], __ldcg(row + c), acc[c]);
                    }
                }
            }
        }
        if constexpr (PAIRS) {
#pragma unroll
            for (int c = 0; c < KT; ++c) acc[c] = df_norm(acc[c]);
            const f2 tot = bk_reduce_scatter_pair<KT>(acc, lane);
            if ((lane & ((1 << SH) - 1)) == 0)
                reinterpret_cast<unsigned long long*>(&s_part[wid][0])[lane >> SH] = bk_bits(tot);
        } else {
            const double tot = bk_reduce_scatter<KT>(acc, lane);
            if ((lane & ((1 << SH) - 1)) == 0) s_part[wid][lane >> SH] = tot;
        }
        __syncthreads();
        if (wid == 0) {
            if (lane < K) {
                const double dj = a.dinv[j];
                const int64_t at = j * K + lane;
                if constexpr (PAIRS) {
                    f2 sum{0.f, 0.f};
#pragma unroll
                    for (int w = 0; w < BK_T / 32; ++w)
                        df_add(sum, bk_pair(reinterpret_cast<const unsigned long long*>(&s_part[w][0])[lane]));
                    const f2 djp = df_from_double(dj);
                    f2 v;
                    if (identity) {
                        v = bk_pair(eold_u[at]);
                        const f2 t = bk_mul_pair(sum, djp);
                        df_add(v, f2{-t.hi, -t.lo});
                    } else {
                        f2 b = df_from_double(r[at]);
                        df_add(b, f2{-sum.hi, -sum.lo});
                        v = bk_mul_pair(b, djp);
                    }
                    reinterpret_cast<unsigned long long*>(e_new)[at] = bk_bits(v);
                    if (out64) out64[at] = df_to_double(v);
                } else {
                    double sum = 0.0;
#pragma unroll
                    for (int w = 0; w < BK_T / 32; ++w) sum += s_part[w][lane];
                    e_new[at] = identity ? e_old[at] - sum * dj : (r[at] - sum) * dj;
                }
            }
            __syncwarp();
            if (lane == 0) bk_st_release_u32(flag + j, epoch);
        }
        __syncthreads();   // s_part is reused by the next row
    }
}

// rho'_c = g_c^T z_c; the last block sets beta_c = rho'_c / rho_c (0 on the first call) and
// rho_c = rho'_c for the active columns, and counts the preconditioner application
__device__ __forceinline__ void bk_gz_body(BkArgs a, int first) {
    __shared__ double sh[BK_T];
    const int c = threadIdx.x & (a.GK - 1);
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / a.GK;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / a.GK;
    double t = 0.0;
    if (c < a.K)
        for (int64_t j = grp; j < a.n; j += ngrp) t = fma(a.g[j * a.K + c], a.z[j * a.K + c], t);
    bk_block_partials(t, a.K, a.GK, a.part + (int64_t)blockIdx.x * a.K, sh);
    if (!bk_last_block(&a.S->arrive[2])) return;
    bk_total(a.part, gridDim.x, a.K, sh);
    if ((int)threadIdx.x < a.K) {
        const int cc = threadIdx.x;
        if (a.S->active[cc]) {
            a.S->beta[cc] = first ? 0.0 : sh[cc] / a.S->rho[cc];
            a.S->rho[cc] = sh[cc];
        }
    }
    if (threadIdx.x == 0) a.S->napply += 1;
}
// p = z + beta p (p = z first), pt = D^{-1} p, for the active columns
__device__ __forceinline__ void bk_pnext_body(BkArgs a) {
    const int c = threadIdx.x & (a.GK - 1);
    if (c >= a.K || !a.S->active[c]) return;
    const double be = a.S->beta[c];
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / a.GK;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / a.GK;
    for (int64_t j = grp; j < a.n; j += ngrp) {
        const int64_t at = j * a.K + c;
        const double pj = fma(be, a.p[at], a.z[at]);
        a.p[at] = pj;
        a.pt[at] = pj * a.inv_d[j];
    }
}
// out2[c] = ||x_c||^2, out2[BK_MAX + c] = ||D x_c||^2 (runs whatever S->done says)
__device__ __forceinline__ void bk_norms_body(BkArgs a, const double* x, double* out2) {
    __shared__ double sh[BK_T];
    const int c = threadIdx.x & (a.GK - 1);
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / a.GK;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / a.GK;
    double t = 0.0, r = 0.0;
    if (c < a.K)
        for (int64_t j = grp; j < a.n; j += ngrp) {
            const double v = x[j * a.K + c], vr = v / a.inv_d[j];
            t = fma(v, v, t);
            r = fma(vr, vr, r);
        }
    double* part2 = a.part + (int64_t)gridDim.x * a.K;
    bk_block_partials(t, a.K, a.GK, a.part + (int64_t)blockIdx.x * a.K, sh);
    bk_block_partials(r, a.K, a.GK, part2 + (int64_t)blockIdx.x * a.K, sh);
    if (!bk_last_block(&a.S->arrive[3])) return;
    bk_total(a.part, gridDim.x, a.K, sh);
    if ((int)threadIdx.x < a.K) out2[threadIdx.x] = sh[threadIdx.x];
    __syncthreads();
    bk_total(part2, gridDim.x, a.K, sh);
    if ((int)threadIdx.x < a.K) out2[BK_MAX + threadIdx.x] = sh[threadIdx.x];
}

}  // namespace lsq
