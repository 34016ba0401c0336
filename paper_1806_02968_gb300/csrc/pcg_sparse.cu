// Alg. 2 step 4 for CSR matrices: PCG on Â^T Â y = Â^T b with the Gauss-Seidel sweeps of
// Alg. 3 on the sparse A_s^T A_s.
//
// Per iteration (one stream, no host synchronisation inside a batch of iterations):
//   k_sp_rows   q = Â p over the rows of A (CSR), partials of ||q||^2 = p^T w
//   k_sp_cols   w = Â^T q over the columns (the cached transposed pattern; no atomics)
//   k_sp_update alpha = rho / p^T w, y += alpha p, g -= alpha w, partials of ||g||^2
//   sweeps      forward then backward Gauss-Seidel sweeps (the first checks convergence):
//               k_sp_sweep_vf on the grid, or k_sp_sweep_1cta in one CTA for narrow levels
//   k_sp_pnext  rho' = g^T z, beta, p = z + beta p
// The sweeps keep the natural row order of Alg. 3: a row depends on the rows of its lower
// (forward) or upper (backward) entries.  Rows run in level order; on the grid each row
// waits (bounded) for the values of its own dependencies, in one CTA the levels meet at
// block barriers.  A device flag ends the remaining kernels of a batch once PCG has
// converged.
#include "sparse.cuh"
#include "values.cuh"
#include "dfloat.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace lsq {

struct SpState {
    double rho, hn, gstart, rec;
    int32_t iters, done, status, napply;   // napply: preconditioner applications so far
    unsigned err, pad, r0, r1;
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
    const int64_t* mdiag;     // position of the diagonal in each row
    const double* dinv;
    const int32_t* sched_f;
    const int32_t* sched_b;
    const int64_t* loff_f;      // first slot of each level
    const int64_t* loff_b;
    int64_t one_f, one_b;       // level count when that direction runs in one CTA, else 0
    int64_t cl_f, cl_b;         // level count when that direction runs in one cluster, else 0
    int64_t nlev_f, nlev_b;     // level counts of the two schedules
    int cl_lg;                  // log2 of that cluster's size
    int lpr, lpc;               // lanes per row of A, lanes per column of A (powers of two <= 32)
    int sweeps;
    // vectors
    double *y, *g, *z, *p, *pt, *w, *q, *e0, *e1, *h;
    double* pt2;              // pt as (hi, lo) float pairs for FP32/BF16 row passes, or NULL
    double* part;             // per-block partials: [row pass: rblk][update: nblk][g^T z: nblk]
    int nblk;                 // blocks of the vector kernels
    int rblk;                 // capacity for the row pass's blocks
    SpState* S;
    double tol, inner_tol;
    int32_t maxit;
    unsigned max_polls = 1u << 22;   // bound of every dependency wait
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

// q_i = sum_e a_e x_{col e} (x = D^{-1} p or D^{-1} y), or b_i, or b_i - that.  A group of
// LPR lanes (a power of two, about the mean row length) takes 4 consecutive rows per step and
// walks their entries flat, so that the loads of 4 rows are in flight together; each row sums
// its entries in a fixed order.
template <int DT>
__global__ void __launch_bounds__(SP_T) k_sp_rows(SpArgs a, int mode, int use_res, const double* x) {
    __shared__ double sh[40];
    if (a.S->done) return;
    const void* vals = use_res ? a.vals_res : a.vals;
    const bool pairs = mode == SPM_MATVEC && !use_res && a.pt2 != nullptr && x == a.pt;
    const int L = a.lpr;
    const int sub = threadIdx.x & (L - 1);
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / L;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / L;
    double qq = 0.0;
    // the trip count is the same for every lane of a warp (the shuffles below need all 32)
    for (int64_t base = 0; base < a.m; base += ngrp * 4) {
        const int64_t i0 = base + grp * 4;
        int64_t rp[5];
#pragma unroll
        for (int r = 0; r < 5; ++r) rp[r] = a.row_ptr[min(i0 + r, a.m)];
        double dot[4] = {0.0, 0.0, 0.0, 0.0};
        // FP32 or BF16 values times the float-pair copy of x: double-float sums on the FP32
        // units (the FP64 unit would take ~64 cycles per dependent step); one conversion to
        // FP64 per row
        constexpr bool PAIR_OK = DT == LSQ_F32 || DT == LSQ_BF16;
        if (PAIR_OK && pairs) {
            f2 ds[4] = {f2{0.f, 0.f}, f2{0.f, 0.f}, f2{0.f, 0.f}, f2{0.f, 0.f}};
            const unsigned long long* x2 = reinterpret_cast<const unsigned long long*>(a.pt2);
            for (int64_t e0 = rp[0] + sub; e0 < rp[4]; e0 += 4 * L) {
                float av[4];
                int32_t cv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t e = e0 + (int64_t)u * L;
                    const bool in = e < rp[4];
                    av[u] = in ? (float)Val<DT>::load(vals, e) : 0.f;
                    cv[u] = in ? a.col_idx[e] : -1;
                }
                unsigned long long xb[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) xb[u] = cv[u] >= 0 ? x2[cv[u]] : 0ull;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t e = e0 + (int64_t)u * L;
                    if (cv[u] >= 0) {
                        const int r = (e >= rp[1]) + (e >= rp[2]) + (e >= rp[3]);
                        const f2 xv = f2{__uint_as_float((unsigned)xb[u]), __uint_as_float((unsigned)(xb[u] >> 32))};
                        float pp, pe;
                        two_prod(av[u], xv.hi, pp, pe);
                        pe = fmaf(av[u], xv.lo, pe);
                        auto add = [&](f2& d) {
                            float s1, e1;
                            two_sum(d.hi, pp, s1, e1);
                            d.hi = s1;
                            d.lo += e1 + pe;
                        };
                        if (r == 0) add(ds[0]);
                        else if (r == 1) add(ds[1]);
                        else if (r == 2) add(ds[2]);
                        else add(ds[3]);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                f2 v = df_norm(ds[r]);
                for (int o = L >> 1; o > 0; o >>= 1) df_add(v, df_shfl_xor(v, o));
                dot[r] = sub == 0 ? df_to_double(v) : 0.0;
            }
        } else {
            if (mode != SPM_RHS) {
                // the 4 rows' entries are contiguous: walk them flat, 4 per lane at a time, all
                // loads (and then all gathers) of a step in flight together; each entry goes to
                // its row's sum, every row still summing its entries in order per lane
                for (int64_t e0 = rp[0] + sub; e0 < rp[4]; e0 += 4 * L) {
                    double av[4];
                    int32_t cv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int64_t e = e0 + (int64_t)u * L;
                        const bool in = e < rp[4];
                        av[u] = in ? (double)Val<DT>::load(vals, e) : 0.0;
                        cv[u] = in ? a.col_idx[e] : -1;
                    }
                    double xv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) xv[u] = cv[u] >= 0 ? x[cv[u]] : 0.0;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int64_t e = e0 + (int64_t)u * L;
                        if (cv[u] >= 0) {
                            const int r = (e >= rp[1]) + (e >= rp[2]) + (e >= rp[3]);
                            if (r == 0) dot[0] = fma(av[u], xv[u], dot[0]);
                            else if (r == 1) dot[1] = fma(av[u], xv[u], dot[1]);
                            else if (r == 2) dot[2] = fma(av[u], xv[u], dot[2]);
                            else dot[3] = fma(av[u], xv[u], dot[3]);
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
                for (int o = L >> 1; o > 0; o >>= 1) dot[r] += __shfl_xor_sync(0xffffffffu, dot[r], o);
        }
        if (sub == 0) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int64_t i = i0 + r;
                if (i < a.m) {
                    const double q = mode == SPM_MATVEC ? dot[r] : (mode == SPM_RHS ? a.b[i] : a.b[i] - dot[r]);
                    a.q[i] = q;
                    qq = fma(q, q, qq);
                }
            }
        }
    }
    const double t = block_sum(qq, sh);
    if (threadIdx.x == 0) a.part[blockIdx.x] = t;
}

// w_j = (1/d_j) sum_{i in column j} a_ij q_i; a group of LPC lanes per column (fixed order)
template <int DT>
__global__ void __launch_bounds__(SP_T) k_sp_cols(SpArgs a, int use_res, double* out) {
    if (a.S->done) return;
    const int L = a.lpc;
    const int sub = threadIdx.x & (L - 1);
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / L;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / L;
    const void* vals = use_res ? a.valsT_res : a.valsT;
    for (int64_t j0 = 0; j0 < a.n; j0 += ngrp) {
        const int64_t j = j0 + grp;
        double t = 0.0;
        if (j < a.n)
            for (int64_t e = a.atptr[j] + sub; e < a.atptr[j + 1]; e += L) t = fma(Val<DT>::load(vals, e), a.q[a.atrow[e]], t);
        for (int o = L >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (j < a.n && sub == 0) out[j] = t * a.inv_d[j];
    }
}

// alpha = rho / p^T w, y += alpha p, g -= alpha w; partial ||g||^2
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
    if (threadIdx.x == 0) a.part[a.rblk + blockIdx.x] = t;
}

// One Gauss-Seidel sweep of Alg. 3 on M (FWD: rows in natural order, lower entries are
// the dependencies; otherwise reverse order, upper entries):
//   e_new_j = (r_j - sum_{other side} M_jk e_old_k - sum_{dependency side} M_jk e_new_k) / M_jj
// With `identity` (the backward sweep right after a single forward sweep from zero,
// t = 1): r - L e_old = D e_old, so e_new_j = e_old_j - (sum_{k>j} M_jk e_new_k) / M_jj.
constexpr int SW_PF = 16;           // dependency entries per lane held in registers

// The row arithmetic of a sweep.  A sweep is a chain of dependent row sums, one per level, so
// the latency of each operation counts, not its throughput.  With FP64 M the sums are FP64
// (SwArith<double>).  With FP32 M they are double-float on the FP32 units (SwArith<float>,
// about 48 significant bits): on GB300 a dependent FP64 operation takes ~64 cycles and an
// FP64 shuffle-and-add ~108, against 4.5 and 32 for FP32.  Sweep vectors hold one 8-byte slot
// per row: an FP64 value, or a (hi, lo) float pair; only the sweep's own buffers hold pairs,
// and `out64` receives FP64 values where a caller needs them.
template <typename MT> struct SwArith;
template <> struct SwArith<double> {
    typedef double Acc;
    typedef double Val;
    static __device__ __forceinline__ Acc zero() { return 0.0; }
    static __device__ __forceinline__ Val from_bits(unsigned long long u) { return __longlong_as_double((long long)u); }
    static __device__ __forceinline__ unsigned long long to_bits(Val v) { return (unsigned long long)__double_as_longlong(v); }
    static __device__ __forceinline__ Val load(const double* p, int64_t k) { return p[k]; }
    static __device__ __forceinline__ void mad(Acc& acc, double m, Val v) { acc = fma(m, v, acc); }
    static __device__ __forceinline__ Acc total(Acc a) { return warp_sum(a); }
    static __device__ __forceinline__ Val from_double(double x) { return x; }
    static __device__ __forceinline__ double to_double(Val v) { return v; }
    static __device__ __forceinline__ Val finish(Val base, Acc acc, Val dj, bool identity) {
        return identity ? base - acc * dj : (base - acc) * dj;
    }
};
template <> struct SwArith<float> {
    typedef f2 Acc;
    typedef f2 Val;
    static __device__ __forceinline__ Acc zero() { return f2{0.f, 0.f}; }
    static __device__ __forceinline__ Val from_bits(unsigned long long u) {
        return f2{__uint_as_float((unsigned)u), __uint_as_float((unsigned)(u >> 32))};
    }
    static __device__ __forceinline__ unsigned long long to_bits(Val v) {
        return (unsigned long long)__float_as_uint(v.hi) | ((unsigned long long)__float_as_uint(v.lo) << 32);
    }
    static __device__ __forceinline__ Val load(const double* p, int64_t k) {
        return from_bits(reinterpret_cast<const unsigned long long*>(p)[k]);
    }
    // acc += m v in the cascaded form (the high word takes the rounded sum, the errors of the
    // sum and of the product gather in the low word; total() renormalises)
    static __device__ __forceinline__ void mad(Acc& acc, float m, Val v) {
        float p, pe;
        two_prod(m, v.hi, p, pe);
        pe = fmaf(m, v.lo, pe);
        float s, e;
        two_sum(acc.hi, p, s, e);
        acc.hi = s;
        acc.lo += e + pe;
    }
    static __device__ __forceinline__ Acc total(Acc a) { return df_warp_sum(df_norm(a)); }
    static __device__ __forceinline__ Val from_double(double x) { return df_from_double(x); }
    static __device__ __forceinline__ double to_double(Val v) { return df_to_double(v); }
    static __device__ __forceinline__ f2 mul(f2 a, f2 b) {
        float p, e;
        two_prod(a.hi, b.hi, p, e);
        e = fmaf(a.hi, b.lo, e);
        e = fmaf(a.lo, b.hi, e);
        const float hi = p + e;
        return f2{hi, e - (hi - p)};
    }
    static __device__ __forceinline__ f2 sub(f2 a, f2 b) {
        f2 r = a;
        df_add(r, f2{-b.hi, -b.lo});
        return r;
    }
    static __device__ __forceinline__ Val finish(Val base, Acc acc, Val dj, bool identity) {
        return identity ? sub(base, mul(acc, dj)) : mul(sub(base, acc), dj);
    }
};

// The grid sweep with the values themselves as completion flags.  Before the sweep every slot
// of e_new holds SWEEP_EMPTY, a pattern no arithmetic produces (an FP64 signalling NaN, or a
// float pair whose low word is a NaN of a form no operation returns); a row polls the values
// it depends on (volatile loads, bounded) until none is SWEEP_EMPTY, then writes its own value.
// A row thus waits for its own dependencies only, and no counter has to be published and read
// back between levels.  Warp w takes schedule slots w, w + W, ... (rows sorted by level), all
// warps resident, so every wait ends.
constexpr unsigned long long SWEEP_EMPTY = 0xFFF7DEADBEEFCAFEull;
constexpr int SWG = 8;                 // dependency values a lane loads before it polls
constexpr unsigned SW_SPIN = 4;        // polls before the first back-off
constexpr unsigned SW_NS_CAP = 256;    // longest back-off between polls (ns)
constexpr int SW_T = 256;              // threads per block of the grid sweep
__global__ void k_fill_empty(double* e, int64_t n) {
    unsigned long long* u = reinterpret_cast<unsigned long long*>(e);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        u[j] = SWEEP_EMPTY;
}
__device__ __forceinline__ unsigned long long ld_volatile_u64(const double* p) {
    unsigned long long v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_volatile_u64(double* p, unsigned long long v) {
    asm volatile("st.volatile.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
template <typename MT, bool FWD>
__global__ void __launch_bounds__(SW_T) k_sp_sweep_vf(SpArgs a, const double* r, const double* e_old,
                                                      double* e_new, double* out64, int identity, int check,
                                                      int nparts) {
    typedef SwArith<MT> A;
    typedef typename A::Acc Acc;
    typedef typename A::Val Val;
    __shared__ double sh[40];
    __shared__ int s_stop;
    if (a.S->done) return;
    if (check) {
        const double gg = sum_parts(a.part + a.rblk, nparts, sh);
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
    const int32_t* sched = FWD ? a.sched_f : a.sched_b;
    const MT* mv = reinterpret_cast<const MT*>(a.mval);
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool other = !identity && e_old != nullptr;
    bool ok = true;
    // the values of up to SWG dependencies per lane: issue all loads, then poll the missing
    auto gather = [&](const int32_t (&kk)[SWG], const MT (&mm)[SWG], Acc& acc) {
        unsigned long long u[SWG];
#pragma unroll
        for (int c = 0; c < SWG; ++c) u[c] = kk[c] >= 0 ? ld_volatile_u64(e_new + kk[c]) : 0ull;
        // the warp polls as one: it leaves the loop when no lane misses a value, so it comes
        // out converged (a warp that left lane by lane ran its shuffle reduction ~7x slower)
        unsigned polls = 0, ns = 32;
        while (true) {
            bool missing = false;
#pragma unroll
            for (int c = 0; c < SWG; ++c) missing = missing || (kk[c] >= 0 && u[c] == SWEEP_EMPTY);
            if (!__any_sync(0xffffffffu, missing)) break;
            ++polls;
            const bool give_up = polls > a.max_polls ||
                                 ((polls & 255u) == 0 && *(volatile unsigned*)&a.S->err != 0u);
            if (__any_sync(0xffffffffu, give_up)) {
                ok = false;
                if (lane == 0) atomicOr(&a.S->err, DEV_ERR_TIMEOUT);
#pragma unroll
                for (int c = 0; c < SWG; ++c) if (u[c] == SWEEP_EMPTY) u[c] = 0ull;
                break;
            }
            if (polls > SW_SPIN) { __nanosleep(ns); ns = ns < SW_NS_CAP ? 2 * ns : SW_NS_CAP; }
#pragma unroll
            for (int c = 0; c < SWG; ++c)
                if (kk[c] >= 0 && u[c] == SWEEP_EMPTY) u[c] = ld_volatile_u64(e_new + kk[c]);
        }
#pragma unroll
        for (int c = 0; c < SWG; ++c)
            if (kk[c] >= 0) A::mad(acc, mm[c], A::from_bits(u[c]));
    };
    for (int64_t slot = gw; slot < a.n; slot += W) {
        const int64_t j = sched[slot];
        const int64_t e0 = a.mptr[j], e1 = a.mptr[j + 1], ed = a.mdiag[j];
        const int64_t d0 = FWD ? e0 : ed + 1, d1 = FWD ? ed : e1;
        const int64_t o0 = FWD ? ed + 1 : e0, o1 = FWD ? e1 : ed;
        Acc acc = A::zero();
        if (other)
            for (int64_t e = o0 + lane; e < o1; e += 32) A::mad(acc, mv[e], A::load(e_old, a.mcol[e]));
        const Val base = identity ? A::load(e_old, j) : A::from_double(r[j]);
        const Val dj = A::from_double(a.dinv[j]);
        // batches of 32 SWG entries from a warp-uniform base: every lane runs the same number
        // of batches (gather's polling is warp-collective); lane l takes entries l, l + 32, ...
        for (int64_t bb = d0; bb < d1; bb += 32 * SWG) {
            int32_t kk[SWG];
            MT mm[SWG];
#pragma unroll
            for (int c = 0; c < SWG; ++c) {
                const int64_t e = bb + lane + 32 * c;
                kk[c] = -1;
                mm[c] = MT(0);
                if (e < d1) { kk[c] = a.mcol[e]; mm[c] = mv[e]; }
            }
            gather(kk, mm, acc);
        }
        acc = A::total(acc);
        if (lane == 0) {
            const Val v = A::finish(base, acc, dj, identity != 0);
            st_volatile_u64(e_new + j, A::to_bits(v));
            if (out64) out64[j] = A::to_double(v);
        }
        __syncwarp();
    }
    (void)ok;
}

// The same sweep in ONE CTA, for deep and narrow level structures (few rows per level): the
// levels follow one another at block barriers instead of per-value waits.  Warp w takes
// rows w, w + NW, ... of each level; the indices and values of its first row of the next level
// (which do not depend on this sweep's values) are loaded before the barrier, so after it only
// the gathers of e_new stand between two levels.
constexpr int S1_T = 512;
template <typename MT, bool FWD>
__global__ void __launch_bounds__(S1_T, 1) k_sp_sweep_1cta(SpArgs a, const double* r, const double* e_old,
                                                           double* e_new, double* out64, int identity, int check,
                                                           int nparts, int64_t nlev) {
    typedef SwArith<MT> A;
    typedef typename A::Acc Acc;
    typedef typename A::Val Val;
    __shared__ double sh[40];
    __shared__ int s_stop;
    if (a.S->done) return;
    if (check) {
        const double gg = sum_parts(a.part + a.rblk, nparts, sh);
        if (threadIdx.x == 0) {
            const double gn = sqrt(gg);
            int stop = 0;
            if (gn <= a.tol * a.S->hn || gn <= a.inner_tol * a.S->gstart) stop = 1;
            if (a.S->iters >= a.maxit) stop = 1;
            s_stop = stop;
            a.S->rec = gn / a.S->hn;
            if (stop) a.S->done = 1;
        }
        __syncthreads();
        if (s_stop) return;
    }
    const int32_t* sched = FWD ? a.sched_f : a.sched_b;
    const int64_t* loff = FWD ? a.loff_f : a.loff_b;
    const MT* mv = reinterpret_cast<const MT*>(a.mval);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int NW = S1_T / 32;
    const bool other = !identity && e_old != nullptr;
    // one row's inputs that do not depend on this sweep
    struct Row {
        int64_t j, d0, d1;
        Val base;           // r_j (or e_old_j for the identity form)
        Val dj;             // 1 / M_jj
        Acc acc;            // this lane's other-side terms
        int32_t kk[SW_PF];
        MT mm[SW_PF];
    };
    auto load_row = [&](int64_t j, Row& R) {
        R.j = j;
        const int64_t e0 = a.mptr[j], e1 = a.mptr[j + 1], ed = a.mdiag[j];
        R.d0 = FWD ? e0 : ed + 1;
        R.d1 = FWD ? ed : e1;
        const int64_t o0 = FWD ? ed + 1 : e0, o1 = FWD ? e1 : ed;
        R.base = identity ? A::load(e_old, j) : A::from_double(r[j]);
        R.dj = A::from_double(a.dinv[j]);
        R.acc = A::zero();
        if (other)
            for (int64_t e = o0 + lane; e < o1; e += 32) A::mad(R.acc, mv[e], A::load(e_old, a.mcol[e]));
#pragma unroll
        for (int c = 0; c < SW_PF; ++c) {
            const int64_t e = R.d0 + lane + 32 * c;
            R.kk[c] = -1;
            R.mm[c] = MT(0);
            if (e < R.d1) { R.kk[c] = a.mcol[e]; R.mm[c] = mv[e]; }
        }
    };
    auto finish_row = [&](const Row& R) {
        Acc acc = R.acc;
#pragma unroll
        for (int c = 0; c < SW_PF; ++c)
            if (R.kk[c] >= 0) A::mad(acc, R.mm[c], A::load(e_new, R.kk[c]));
        for (int64_t base = R.d0 + 32 * SW_PF; base < R.d1; base += 32 * 8) {
            int32_t k2[8];
            MT m2[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t e = base + lane + 32 * u;
                k2[u] = -1;
                m2[u] = MT(0);
                if (e < R.d1) { k2[u] = a.mcol[e]; m2[u] = mv[e]; }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (k2[u] >= 0) A::mad(acc, m2[u], A::load(e_new, k2[u]));
        }
        acc = A::total(acc);
        if (lane == 0) {
            const Val v = A::finish(R.base, acc, R.dj, identity != 0);
            reinterpret_cast<unsigned long long*>(e_new)[R.j] = A::to_bits(v);
            if (out64) out64[R.j] = A::to_double(v);
        }
    };
    Row cur;
    int64_t lo = loff[0], hi = loff[1];
    if (w < hi - lo) load_row(sched[lo + w], cur);
    for (int64_t L = 0; L < nlev; ++L) {
        const int64_t cnt = hi - lo;
        for (int64_t q = w; q < cnt; q += NW) {
            if (q != w) load_row(sched[lo + q], cur);
            finish_row(cur);
        }
        if (L + 1 < nlev) {
            lo = hi;
            hi = loff[L + 2];
            if (w < hi - lo) load_row(sched[lo + w], cur);
        }
        __syncthreads();   // this level's values are visible to every warp
    }
}

// The same sweep in ONE thread-block cluster of C = 2^lg CTAs, for deep level structures
// whose levels are too wide for one SM but whose sweep vector fits in the cluster's shared
// memory.  e_new_j lives in the shared memory of CTA (j mod C) at slot j / C; a row's
// gathers read its owners' shared memory (DSMEM) and the levels meet at hardware cluster
// barriers, so no value makes a round trip through L2 and nothing is polled.  Warp w of CTA
// r takes rows w C + r, w C + r + C NW, ... of each level; its first row of the next level
// (indices, values, and the terms that do not depend on this sweep) is loaded before the
// barrier, as in the one-CTA form.  Every value is also stored to e_new in global memory
// for the kernels that follow.
constexpr int SC_T = 512;
template <typename MT, bool FWD>
__global__ void __launch_bounds__(SC_T, 1) k_sp_sweep_cl(SpArgs a, const double* r, const double* e_old,
                                                         double* e_new, double* out64, int identity, int check,
                                                         int nparts, int64_t nlev, int lg) {
    namespace cg = cooperative_groups;
    typedef SwArith<MT> A;
    typedef typename A::Acc Acc;
    typedef typename A::Val Val;
    extern __shared__ __align__(16) unsigned long long xs[];   // this CTA's slots of e_new
    __shared__ double sh[40];
    __shared__ int s_stop;
    // Every CTA takes the same exits before the first cluster barrier: done is only written
    // by this launch's check (rank 0), whose decision every CTA computes identically.
    if (a.S->done) return;
    cg::cluster_group cl = cg::this_cluster();
    const unsigned C = 1u << lg, me = cl.block_rank();
    if (check) {
        const double gg = sum_parts(a.part + a.rblk, nparts, sh);
        if (threadIdx.x == 0) {
            const double gn = sqrt(gg);
            int stop = 0;
            if (gn <= a.tol * a.S->hn || gn <= a.inner_tol * a.S->gstart) stop = 1;
            if (a.S->iters >= a.maxit) stop = 1;
            s_stop = stop;
            if (me == 0) {
                a.S->rec = gn / a.S->hn;
                if (stop) a.S->done = 1;
            }
        }
        __syncthreads();
        if (s_stop) return;
    }
    const int32_t* sched = FWD ? a.sched_f : a.sched_b;
    const int64_t* loff = FWD ? a.loff_f : a.loff_b;
    const MT* mv = reinterpret_cast<const MT*>(a.mval);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int NW = (int)(blockDim.x >> 5);
    const int64_t gw = (int64_t)w * C + me, GW = (int64_t)NW * C;
    const unsigned cmask = C - 1u;
    const bool other = !identity && e_old != nullptr;
    struct Row {
        int64_t j, d0, d1;
        Val base, dj;
        Acc acc;
        int32_t kk[SW_PF];
        MT mm[SW_PF];
    };
    auto load_row = [&](int64_t j, Row& R) {
        R.j = j;
        const int64_t e0 = a.mptr[j], e1 = a.mptr[j + 1], ed = a.mdiag[j];
        R.d0 = FWD ? e0 : ed + 1;
        R.d1 = FWD ? ed : e1;
        const int64_t o0 = FWD ? ed + 1 : e0, o1 = FWD ? e1 : ed;
        R.base = identity ? A::load(e_old, j) : A::from_double(r[j]);
        R.dj = A::from_double(a.dinv[j]);
        R.acc = A::zero();
        if (other)
            for (int64_t e = o0 + lane; e < o1; e += 32) A::mad(R.acc, mv[e], A::load(e_old, a.mcol[e]));
#pragma unroll
        for (int c = 0; c < SW_PF; ++c) {
            const int64_t e = R.d0 + lane + 32 * c;
            R.kk[c] = -1;
            R.mm[c] = MT(0);
            if (e < R.d1) { R.kk[c] = a.mcol[e]; R.mm[c] = mv[e]; }
        }
    };
    auto gather = [&](int32_t k) -> Val {
        const unsigned long long* src = cl.map_shared_rank(xs, (unsigned)k & cmask);
        return A::from_bits(src[(unsigned)k >> lg]);
    };
    auto finish_row = [&](const Row& R) {
        Val v[SW_PF];
#pragma unroll
        for (int c = 0; c < SW_PF; ++c) v[c] = R.kk[c] >= 0 ? gather(R.kk[c]) : A::from_bits(0ull);
        Acc acc = R.acc;
#pragma unroll
        for (int c = 0; c < SW_PF; ++c)
            if (R.kk[c] >= 0) A::mad(acc, R.mm[c], v[c]);
        for (int64_t b0 = R.d0 + 32 * SW_PF; b0 < R.d1; b0 += 32 * 8) {
            int32_t k2[8];
            MT m2[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t e = b0 + lane + 32 * u;
                k2[u] = -1;
                m2[u] = MT(0);
                if (e < R.d1) { k2[u] = a.mcol[e]; m2[u] = mv[e]; }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (k2[u] >= 0) A::mad(acc, m2[u], gather(k2[u]));
        }
        acc = A::total(acc);
        if (lane == 0) {
            const Val val = A::finish(R.base, acc, R.dj, identity != 0);
            const unsigned long long bits = A::to_bits(val);
            unsigned long long* dst = cl.map_shared_rank(xs, (unsigned)R.j & cmask);
            dst[(unsigned)R.j >> lg] = bits;
            reinterpret_cast<unsigned long long*>(e_new)[R.j] = bits;
            if (out64) out64[R.j] = A::to_double(val);
        }
    };
    Row cur;
    int64_t lo = loff[0], hi = loff[1];
    if (gw < hi - lo) load_row(sched[lo + gw], cur);
    cl.sync();   // every CTA of the cluster runs before any shared memory is read remotely
    for (int64_t L = 0; L < nlev; ++L) {
        const int64_t cnt = hi - lo;
        for (int64_t q = gw; q < cnt; q += GW) {
            if (q != gw) load_row(sched[lo + q], cur);
            finish_row(cur);
        }
        if (L + 1 < nlev) {
            lo = hi;
            hi = loff[L + 2];
            if (gw < hi - lo) load_row(sched[lo + gw], cur);
        }
        cl.sync();   // this level's values are visible in every CTA; after the last, no CTA reads another's memory
    }
}

// t = 0 (the comparison method, P = I): z = g, with the convergence check of the first sweep
__global__ void __launch_bounds__(SP_T) k_sp_identity(SpArgs a, const double* r, double* e, int check, int nparts) {
    __shared__ double sh[40];
    __shared__ int s_stop;
    if (a.S->done) return;
    if (check) {
        const double gg = sum_parts(a.part + a.rblk, nparts, sh);
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
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += (int64_t)gridDim.x * blockDim.x)
        e[j] = r[j];
}

// rho' = g^T z; first: p = z, else beta = rho'/rho, p = z + beta p; pt = D^{-1} p; epoch++
__global__ void __launch_bounds__(SP_T) k_sp_gz(SpArgs a) {
    __shared__ double sh[40];
    if (a.S->done) return;
    double t = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += (int64_t)gridDim.x * blockDim.x)
        t = fma(a.g[j], a.z[j], t);
    t = block_sum(t, sh);
    if (threadIdx.x == 0) a.part[a.rblk + a.nblk + blockIdx.x] = t;
}
__global__ void __launch_bounds__(SP_T) k_sp_pnext(SpArgs a, int first, int nparts) {
    __shared__ double sh[40];
    if (a.S->done) return;
    const double rho_new = sum_parts(a.part + a.rblk + a.nblk, nparts, sh);
    const double beta = first ? 0.0 : rho_new / a.S->rho;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += (int64_t)gridDim.x * blockDim.x) {
        const double pj = first ? a.z[j] : fma(beta, a.p[j], a.z[j]);
        a.p[j] = pj;
        const double ptj = pj * a.inv_d[j];
        a.pt[j] = ptj;
        if (a.pt2) {
            const f2 v = df_from_double(ptj);
            reinterpret_cast<unsigned long long*>(a.pt2)[j] =
                (unsigned long long)__float_as_uint(v.hi) | ((unsigned long long)__float_as_uint(v.lo) << 32);
        }
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

// The cluster form's size (8 CTAs, the portable maximum) and its shared-memory budget per CTA.
constexpr int SC_LG = 3;
constexpr int64_t SC_SMEM = 200 * 1024;
// Sweep form override (lsq_set_sweep_form): 0 chosen by shape, 1 grid, 2 one CTA, 3 one cluster.
static std::atomic<int> g_sweep_form{0};
int sweep_form_setting() { return g_sweep_form.load(std::memory_order_relaxed); }

// Launch of the cluster form; false (nothing launched) when the cluster does not fit.
template <typename MT, bool FWD>
static bool launch_sweep_cluster(const SpArgs& a, const double* r, const double* eold, double* enew,
                                 double* out64, int identity, int check, int nparts, int64_t nl,
                                 cudaStream_t st, lsq_status& status) {
    static std::atomic<int> fits{-1};   // per kernel instance: the cluster fits on this device
    auto kern = k_sp_sweep_cl<MT, FWD>;
    const int C = 1 << SC_LG;
    const size_t smem = (size_t)8 * (size_t)((a.n + C - 1) / C);
    if ((int64_t)smem > SC_SMEM) return false;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(SC_T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int f = fits.load(std::memory_order_relaxed);
    if (f < 0) {
        f = 0;
        if (cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SC_SMEM) ==
            cudaSuccess) {
            cudaLaunchConfig_t probe = cfg;
            probe.dynamicSmemBytes = SC_SMEM;
            int clusters = 0;
            if (cudaOccupancyMaxActiveClusters(&clusters, (const void*)kern, &probe) == cudaSuccess && clusters > 0)
                f = 1;
        }
        cudaGetLastError();   // a refused query leaves the grid form in use, not an error
        fits.store(f, std::memory_order_relaxed);
    }
    if (!f) return false;
    const int lg = SC_LG;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a, r, eold, enew, out64, identity, check, nparts, nl, lg);
    count_launch();
    status = e == cudaSuccess ? LSQ_OK : LSQ_ERR_CUDA;
    if (e != cudaSuccess) set_error(std::string("cluster sweep launch: ") + cudaGetErrorString(e));
    return true;
}

// Cooperative launch of a sweep with one co-resident grid (every warp must run at once for
// the level waits to end), or the one-CTA or one-cluster form when the schedule calls for it.
template <typename MT, bool FWD>
static lsq_status launch_sweep(const SpArgs& a, const double* r, const double* eold, double* enew,
                               double* out64, int identity, int check, int nparts, int idx, cudaStream_t st) {
    static std::atomic<int> grid_cache{0};   // one per kernel instance; callers may be threads
    auto kern = k_sp_sweep_vf<MT, FWD>;
    int grid = grid_cache.load(std::memory_order_relaxed);
    if (grid == 0) {
        int dev = 0, sms = 0, per = 0;
        LSQ_CUDA(cudaGetDevice(&dev));
        LSQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        LSQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, SW_T, 0));
        if (per < 1) { set_error("sweep kernel does not fit on an SM"); return LSQ_ERR_CUDA; }
        grid = sms * per;
        grid_cache.store(grid, std::memory_order_relaxed);
    }
    const int64_t nl = FWD ? a.one_f : a.one_b;
    if (nl > 0) {   // deep, narrow level structure: the whole sweep in one CTA
        k_sp_sweep_1cta<MT, FWD><<<1, S1_T, 0, st>>>(a, r, eold, enew, out64, identity, check, nparts, nl);
        count_launch();
        LSQ_CUDA(cudaGetLastError());
        return LSQ_OK;
    }
    const int64_t ncl = FWD ? a.cl_f : a.cl_b;
    if (ncl > 0) {   // deep levels of moderate width, the vector within a cluster's shared memory
        lsq_status q = LSQ_OK;
        if (launch_sweep_cluster<MT, FWD>(a, r, eold, enew, out64, identity, check, nparts, ncl, st, q)) return q;
    }
    // the grid form: fill e_new with the empty marker, then the value-flag sweep
    k_fill_empty<<<(unsigned)std::min<int64_t>((a.n + SP_T - 1) / SP_T, 152 * 8), SP_T, 0, st>>>(enew, a.n);
    count_launch();
    (void)idx;
    SpArgs av = a;
    void* params[] = {&av, (void*)&r, (void*)&eold, (void*)&enew, (void*)&out64, &identity, &check, &nparts};
    const int g_sweep = sweep_grid(grid, a.n, FWD ? a.nlev_f : a.nlev_b, SW_T / 32);
    LSQ_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(g_sweep), dim3(SW_T), params, 0, st));
    count_launch();
    return LSQ_OK;
}

// The sweep form of each direction.  By shape (form 0): one CTA when a level holds fewer than
// 2048 dependency entries on average: block barriers between levels are then cheaper than a
// grid of warps polling for the values they depend on, and one SM's loads still keep up with
// a level's gathers (at ~10,000 entries per level one SM is twice slower than the grid);
// otherwise the grid.  The cluster form is never chosen by shape: on the 4e6 x 4e4 workload
// (1583 levels of ~9,600 dependency entries) it took 8.0 ms per sweep against the grid's 5.8,
// because a cluster barrier's release waits for the next level's row loads still in flight
// and random gathers from other CTAs' shared memory are throughput-limited per SM.
static void choose_sweep_form(SpArgs& a, const SparseHandle* SH, int64_t n) {
    const double dep = 0.5 * (double)(SH->nnz_M - n);   // dependency entries per direction
    const int form = g_sweep_form.load(std::memory_order_relaxed);
    const bool fits = 8 * ((n + (1 << SC_LG) - 1) >> SC_LG) <= SC_SMEM;
    a.cl_lg = SC_LG;
    auto pick = [&](int64_t nlev, int64_t& one, int64_t& clv) {
        one = clv = 0;
        if (form == 2) one = nlev;
        else if (form == 3) clv = fits ? nlev : 0;
        else if (form == 0 && dep < 2048.0 * (double)nlev) one = nlev;
    };
    pick(SH->nlev_f, a.one_f, a.cl_f);
    pick(SH->nlev_b, a.one_b, a.cl_b);
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
    const int nblk = 152 * 4, rblk = 152 * 16;
    // workspace
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off += (bytes + 255) & ~size_t(255); return at; };
    size_t o_S = take(sizeof(SpState)), o_vT = take(es * nnz), o_vT64 = take(res64 && DT != LSQ_F64 ? 8 * nnz : 16),
           o_vec = take(8 * (size_t)n * 11), o_q = take(8 * (size_t)m),
           o_part = take(8 * (size_t)(rblk + 2 * nblk)),
           o_n2 = take(64);
    Scratch sc;
    LSQ_CUDA(sc.alloc(off, st));
    char* base = sc.as<char>();
    SpState* S = (SpState*)(base + o_S);
    double* vec = (double*)(base + o_vec);
    SpArgs a{};
    a.max_polls = dep_wait_polls();
    a.m = m; a.n = n; a.row_ptr = A->row_ptr; a.col_idx = A->col_idx;
    a.vals = A->vals;
    a.vals_res = res64 ? (DT == LSQ_F64 ? A->vals : (const void*)A->vals_f64) : A->vals;
    a.atptr = SH->atptr; a.atrow = SH->atrow;
    a.valsT = base + o_vT;
    a.valsT_res = res64 ? (DT == LSQ_F64 ? a.valsT : (const void*)(base + o_vT64)) : a.valsT;
    a.inv_d = P->inv_d;
    a.mptr = SH->mptr; a.mcol = SH->mcol; a.mdiag = SH->mdiag;
    a.mval = P->op_dtype == LSQ_F32 ? (const void*)SH->mval32 : (const void*)SH->mval;
    a.dinv = SH->dinv; a.sched_f = SH->sched_f; a.sched_b = SH->sched_b;
    a.sweeps = P->sweeps;
    a.y = vec; a.g = vec + n; a.z = vec + 2 * n; a.p = vec + 3 * n; a.pt = vec + 4 * n;
    a.w = vec + 5 * n; a.e0 = vec + 6 * n; a.e1 = vec + 7 * n; a.h = vec + 8 * n;
    double* tmpv = vec + 9 * n;
    a.pt2 = (DT == LSQ_F32 || DT == LSQ_BF16) ? vec + 10 * n : nullptr;
    a.q = (double*)(base + o_q);
    a.loff_f = SH->loff_f; a.loff_b = SH->loff_b; a.nlev_f = SH->nlev_f; a.nlev_b = SH->nlev_b;
    choose_sweep_form(a, SH, n);
    auto lanes_for = [](double mean) { int L = 1; while (L < 32 && L < mean) L <<= 1; return L; };
    a.lpr = lanes_for((double)nnz / (double)m);
    a.lpc = lanes_for((double)nnz / (double)n);
    a.part = (double*)(base + o_part); a.nblk = nblk; a.rblk = rblk;
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
    // enough lanes in flight for the gathers (the reductions read at most nblk partials)
    const unsigned grows = gridn(m * a.lpr, rblk), gcols = gridn(n * a.lpc, 152 * 16), gvec = gridn(n, nblk);
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
    lsq_status sweep_status = LSQ_OK;
    // FP32 M: the sweeps keep their vectors as float pairs in e0/e1 and the last one also writes
    // z in FP64; FP64 M: the last sweep writes z directly
    const bool pairs = P->op_dtype == LSQ_F32;
    auto sweep = [&](bool fwd, const double* r, const double* eold, double* enew, double* out64, int identity,
                     int check, int idx) {
        lsq_status q;
        if (pairs)
            q = fwd ? launch_sweep<float, true>(a, r, eold, enew, out64, identity, check, gvec, idx, st)
                    : launch_sweep<float, false>(a, r, eold, enew, out64, identity, check, gvec, idx, st);
        else
            q = fwd ? launch_sweep<double, true>(a, r, eold, enew, out64, identity, check, gvec, idx, st)
                    : launch_sweep<double, false>(a, r, eold, enew, out64, identity, check, gvec, idx, st);
        if (q != LSQ_OK) sweep_status = q;
    };
    // z = P g: t forward then t backward sweeps (the first may carry the convergence check)
    auto precond = [&](int check) {
        if (P->sweeps == 0) {
            k_sp_identity<<<gvec, SP_T, 0, st>>>(a, a.g, a.z, check, gvec);
            count_launch();
            return;
        }
        const double* eold = nullptr;
        double* bufs[2] = {a.e0, a.e1};
        int cur = 0, idx = 0;
        for (int t = 0; t < P->sweeps; ++t, ++idx) {
            sweep(true, a.g, eold, bufs[cur], nullptr, 0, (t == 0) ? check : 0, idx);
            eold = bufs[cur];
            cur ^= 1;
        }
        for (int t = 0; t < P->sweeps; ++t, ++idx) {
            const bool last = t == P->sweeps - 1;
            double* dst = (last && !pairs) ? a.z : bufs[cur];
            sweep(false, a.g, eold, dst, (last && pairs) ? a.z : nullptr, (P->sweeps == 1) ? 1 : 0, 0, idx);
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
                count_launch(2);
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
                        count_launch(6);
                    }
                    if (sweep_status != LSQ_OK) return sweep_status;
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
    size_t o_S = take(sizeof(SpState)), o_e = take(16 * (size_t)n);
    Scratch sc;
    LSQ_CUDA(sc.alloc(off, st));
    char* base = sc.as<char>();
    SpArgs a{};
    a.max_polls = dep_wait_polls();
    a.n = n;
    a.mptr = SH->mptr; a.mcol = SH->mcol; a.mdiag = SH->mdiag;
    a.mval = P->op_dtype == LSQ_F32 ? (const void*)SH->mval32 : (const void*)SH->mval;
    a.dinv = SH->dinv; a.sched_f = SH->sched_f; a.sched_b = SH->sched_b; a.sweeps = P->sweeps;
    a.e0 = (double*)(base + o_e); a.e1 = a.e0 + n;
    a.loff_f = SH->loff_f; a.loff_b = SH->loff_b; a.nlev_f = SH->nlev_f; a.nlev_b = SH->nlev_b;
    choose_sweep_form(a, SH, n);
    a.S = (SpState*)(base + o_S);
    if (P->sweeps == 0) {
        LSQ_CUDA(cudaMemcpyAsync(e, r, 8 * (size_t)n * k, cudaMemcpyDeviceToDevice, st));
        LSQ_CUDA(cudaStreamSynchronize(st));
        return LSQ_OK;
    }
    for (int64_t c = 0; c < k; ++c) {
        LSQ_CUDA(cudaMemsetAsync(a.S, 0, sizeof(SpState), st));
        const double* rc = r + c * n;
        double* out = e + c * n;
        const double* eold = nullptr;
        double* bufs[2] = {a.e0, a.e1};
        int cur = 0, idx = 0;
        // FP32 M: float pairs in e0/e1, the last sweep also writes out in FP64
        const bool pairs = P->op_dtype == LSQ_F32;
        for (int t = 0; t < P->sweeps; ++t, ++idx) {
            lsq_status q = pairs
                ? launch_sweep<float, true>(a, rc, eold, bufs[cur], nullptr, 0, 0, 0, idx, st)
                : launch_sweep<double, true>(a, rc, eold, bufs[cur], nullptr, 0, 0, 0, idx, st);
            if (q != LSQ_OK) return q;
            eold = bufs[cur];
            cur ^= 1;
        }
        for (int t = 0; t < P->sweeps; ++t, ++idx) {
            const bool last = t == P->sweeps - 1;
            double* dst = (last && !pairs) ? out : bufs[cur];
            double* out64 = (last && pairs) ? out : nullptr;
            const int ident = P->sweeps == 1 ? 1 : 0;
            lsq_status q = pairs
                ? launch_sweep<float, false>(a, rc, eold, dst, out64, ident, 0, 0, idx, st)
                : launch_sweep<double, false>(a, rc, eold, dst, out64, ident, 0, 0, idx, st);
            if (q != LSQ_OK) return q;
            eold = dst;
            cur ^= 1;
        }
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
    if (k >= 2) return sparse_block_solve(A, P, B, Hcols, k, ldb, X, ldx, o, info, st);
    switch (A->dtype) {
        case LSQ_F64: return sp_solve_impl<LSQ_F64>(A, P, B, Hcols, k, ldb, X, ldx, o, info, st);
        case LSQ_F32: return sp_solve_impl<LSQ_F32>(A, P, B, Hcols, k, ldb, X, ldx, o, info, st);
        case LSQ_BF16: return sp_solve_impl<LSQ_BF16>(A, P, B, Hcols, k, ldb, X, ldx, o, info, st);
        default: return sp_solve_impl<LSQ_F32X2>(A, P, B, Hcols, k, ldb, X, ldx, o, info, st);
    }
}

}  // namespace lsq

extern "C" lsq_status lsq_set_sweep_form(int32_t form) {
    if (form < 0 || form > 3) {
        lsq::set_error("lsq_set_sweep_form: form must be 0, 1, 2 or 3");
        return LSQ_ERR_INVALID;
    }
    lsq::g_sweep_form.store(form, std::memory_order_relaxed);
    return LSQ_OK;
}
