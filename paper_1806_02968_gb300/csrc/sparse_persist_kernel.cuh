// Alg. 2 step 4 for a block of K <= 32 right-hand sides of a CSR matrix in ONE persistent
// cooperative kernel: the row pass q = Â p, the column pass w = Â^T q fused with the update
// of y and g, the t forward and t backward level-ordered Gauss-Seidel sweeps of Alg. 3, the
// dot products and the direction update, the convergence masks of the K columns, and the
// restarts from the true residual, all between grid barriers, with no host synchronisation.
// The call makes no data-dependent host decision, so it can be captured in a CUDA graph.
//
// The steps are the device bodies of the stream-ordered block solver (bk_device.cuh), so
// both forms compute the same iteration.  Per inner iteration:
//   rows      q = Â p~ (and the sweep buffers are reset to their empty marker)   | barrier
//   cols      w = Â^T q                                                          | barrier
//   update    alpha, y, g, ||g||^2, the masks (one block, fixed order)           | barrier
//   sweeps    forward, then backward (each row waits for its own dependencies)   | barrier each
//   gz        rho' = g^T z, beta                                                  | barrier
//   pnext     p = z + beta p, p~ = D^{-1} p                                       | barrier
// The per-column control state (iterations, outer steps, recursive / true / raw residuals,
// convergence, breakdown) is kept in shared memory by every CTA; every CTA computes it from
// the same grid-wide sums in the same order, so all take the same decisions.  Block 0 alone
// writes the shared state words the bodies read, before the barrier that publishes them.
#pragma once
#include "bk_device.cuh"
#include "sparse_persist.cuh"

namespace lsq {

struct BkPersist {
    BkArgs a;
    unsigned long long* bar;  // grid barrier count (zeroed before the launch)
    double* n2;               // grid sums of the norms (2 * BK_MAX)
    double* tmpv;             // n x K scratch
    double* X;                // solutions, column-major with leading dimension ldx
    int64_t ldx;
    BkPersistOut* out;        // per-column results (device)
    int use_h;                // normal form: a.h holds the right-hand side on entry
    int res64;                // true residuals from FP64 values
    int max_outer;
    unsigned bar_polls;       // bound of every grid-barrier wait
};

__device__ __forceinline__ unsigned bk_ld_volatile_u32(const unsigned* p) {
    return *reinterpret_cast<const volatile unsigned*>(p);
}

// SMODE is the sweep form (0: lane per column, 1: lane per entry, 2: CTA per row); the
// lane-per-column form needs few registers, so that instantiation keeps 4 CTAs per SM.
template <int DT, typename MT, int SMODE, int KT>
__global__ void __launch_bounds__(BK_T, SMODE == 0 ? 3 : 2) k_bk_persist(BkPersist P) {
    BkArgs& a = P.a;
    const int K = a.K;
    const int tid = threadIdx.x;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nK = a.n * K;
    unsigned long long epoch = 0;
    __shared__ double s_hn[BK_MAX], s_hnraw[BK_MAX], s_gn[BK_MAX], s_gnraw[BK_MAX];
    __shared__ double s_rec[BK_MAX], s_tru[BK_MAX], s_raw[BK_MAX];
    __shared__ int s_iters[BK_MAX], s_outer[BK_MAX], s_conv[BK_MAX], s_broke[BK_MAX];
    __shared__ int s_dirty[BK_MAX], s_act0[BK_MAX];
    __shared__ int s_flag;

#define BK_BAR()                                                              \
    do {                                                                      \
        if (!grid_barrier(P.bar, gridDim.x, &a.S->err, epoch, P.bar_polls)) \
            return;                                                           \
    } while (0)

    auto rows = [&](int mode, int use_res, const double* x) {
        if (use_res && P.res64) bk_rows_body<LSQ_F64>(a, mode, 1, x);
        else bk_rows_body<DT>(a, mode, 0, x);
    };
    auto cols = [&](int use_res, double* dst) {
        if (use_res && P.res64) bk_cols_body<LSQ_F64>(a, 1, dst);
        else bk_cols_body<DT>(a, 0, dst);
    };
    auto fill_empty = [&](double* e) {
        unsigned long long* u = reinterpret_cast<unsigned long long*>(e);
        for (int64_t t = gtid; t < nK; t += gstride) u[t] = BK_EMPTY;
    };
    auto sweep = [&](bool fwd, const double* eold, double* enew, int identity, int idx) {
        if (fwd) {
            if constexpr (SMODE == 0) bk_sweep_body<MT, true>(a, a.g, eold, enew, identity, idx);
            else if constexpr (SMODE == 1) bk_sweep_ep_body<MT, true, KT>(a, a.g, eold, enew, identity, idx);
            else bk_sweep_cta_body<MT, true, KT>(a, a.g, eold, enew, identity, idx);
        } else {
            if constexpr (SMODE == 0) bk_sweep_body<MT, false>(a, a.g, eold, enew, identity, idx);
            else if constexpr (SMODE == 1) bk_sweep_ep_body<MT, false, KT>(a, a.g, eold, enew, identity, idx);
            else bk_sweep_cta_body<MT, false, KT>(a, a.g, eold, enew, identity, idx);
        }
    };
    // norms of x over the grid -> s_gn / s_gnraw (every CTA)
    auto norms = [&](const double* x) -> bool {
        bk_norms_body(a, x, P.n2);
        if (!grid_barrier(P.bar, gridDim.x, &a.S->err, epoch, P.bar_polls)) return false;
        if (tid < K) {
            s_gn[tid] = sqrt(__ldcg(P.n2 + tid));
            s_gnraw[tid] = sqrt(__ldcg(P.n2 + BK_MAX + tid));
        }
        __syncthreads();
        return true;
    };

    // h = Â^T b (least-squares form) or the given normal-form right-hand side; g = h
    if (!P.use_h) {
        rows(1, 1, a.pt);
        BK_BAR();
        cols(1, a.h);
        BK_BAR();
    }
    for (int64_t t = gtid; t < nK; t += gstride) a.g[t] = a.h[t];
    if (!norms(a.h)) return;
    if (tid < K) {
        s_hn[tid] = s_gn[tid];
        s_hnraw[tid] = s_gnraw[tid];
        s_rec[tid] = s_tru[tid] = s_raw[tid] = 1.0;
        s_iters[tid] = s_outer[tid] = s_conv[tid] = s_broke[tid] = s_dirty[tid] = 0;
        if (s_hn[tid] == 0.0) { s_conv[tid] = 1; s_rec[tid] = s_tru[tid] = s_raw[tid] = 0.0; }
    }
    __syncthreads();

    // g = Â^T (b - Â y) (or h - Â^T Â y) and its norms
    auto true_residual = [&]() -> bool {
        for (int64_t t = gtid; t < nK; t += gstride) P.tmpv[t] = a.y[t] * a.inv_d[t / K];
        if (!grid_barrier(P.bar, gridDim.x, &a.S->err, epoch, P.bar_polls)) return false;
        if (P.use_h) {
            rows(0, 1, P.tmpv);
            if (!grid_barrier(P.bar, gridDim.x, &a.S->err, epoch, P.bar_polls)) return false;
            cols(1, a.w);
            if (!grid_barrier(P.bar, gridDim.x, &a.S->err, epoch, P.bar_polls)) return false;
            for (int64_t t = gtid; t < nK; t += gstride) a.g[t] = a.h[t] - a.w[t];
        } else {
            rows(2, 1, P.tmpv);
            if (!grid_barrier(P.bar, gridDim.x, &a.S->err, epoch, P.bar_polls)) return false;
            cols(1, a.g);
        }
        if (!grid_barrier(P.bar, gridDim.x, &a.S->err, epoch, P.bar_polls)) return false;
        if (tid < K) s_dirty[tid] = 0;
        return norms(a.g);
    };

    // z = P g: t forward then t backward sweeps.  With prefilled, e0 and z already hold the
    // empty marker (t = 1 inside the iteration: reset during the row pass).
    auto precond = [&](bool prefilled) -> bool {
        if (a.sweeps == 0) {   // the comparison method: P = I
            for (int64_t t = gtid; t < nK; t += gstride) a.z[t] = a.g[t];
            // g^T z next reads z in another thread mapping
            return grid_barrier(P.bar, gridDim.x, &a.S->err, epoch, P.bar_polls);
        }
        const double* eold = nullptr;
        double* bufs[2] = {a.e0, a.e1};
        int cur = 0, idx = 0;
        const bool pre = prefilled && a.sweeps == 1;
        for (int t = 0; t < a.sweeps; ++t, ++idx) {
            if (!pre) {
                fill_empty(bufs[cur]);
                if (!grid_barrier(P.bar, gridDim.x, &a.S->err, epoch, P.bar_polls)) return false;
            }
            sweep(true, eold, bufs[cur], 0, idx);
            if (!grid_barrier(P.bar, gridDim.x, &a.S->err, epoch, P.bar_polls)) return false;
            if (bk_ld_volatile_u32(&a.S->err) != 0u) return false;
            eold = bufs[cur];
            cur ^= 1;
        }
        for (int t = 0; t < a.sweeps; ++t, ++idx) {
            double* dst = (t == a.sweeps - 1) ? a.z : bufs[cur];
            if (!pre) {
                fill_empty(dst);
                if (!grid_barrier(P.bar, gridDim.x, &a.S->err, epoch, P.bar_polls)) return false;
            }
            sweep(false, eold, dst, (a.sweeps == 1) ? 1 : 0, idx);
            if (!grid_barrier(P.bar, gridDim.x, &a.S->err, epoch, P.bar_polls)) return false;
            if (bk_ld_volatile_u32(&a.S->err) != 0u) return false;
            eold = dst;
            cur ^= 1;
        }
        return true;
    };
    auto fail = [&]() {
        if (tid == 0) atomicOr(P.bar, BAR_ERR);
    };

    int napply = 0;
    for (int outer = 0; outer < P.max_outer; ++outer) {
        if (outer > 0 && !true_residual()) { fail(); return; }
        // the columns that iterate in this inner solve (every CTA; block 0 writes the state)
        if (tid < K) {
            const int c = tid;
            int act = 0;
            const double hn = s_hn[c];
            if (!(hn == 0.0 || s_broke[c])) {
                s_tru[c] = s_gn[c] / hn;
                s_raw[c] = s_hnraw[c] > 0.0 ? s_gnraw[c] / s_hnraw[c] : 0.0;
                if (outer == 0) s_rec[c] = s_tru[c];
                if (s_tru[c] <= a.tol) s_conv[c] = 1;
                else if (s_iters[c] < a.maxit) {
                    act = 1;
                    s_outer[c] = outer + 1;
                }
            }
            s_act0[c] = act;
            if (blockIdx.x == 0) {
                a.S->hn[c] = hn > 0.0 ? hn : 1.0;
                a.S->active[c] = act;
                a.S->gstart[c] = s_gn[c];
                a.S->iters[c] = s_iters[c];
                a.S->rec[c] = s_rec[c];
                a.S->broke[c] = 0;
                a.S->rho[c] = 0.0;
                a.S->beta[c] = 0.0;
            }
        }
        if (blockIdx.x == 0 && tid == 0) { a.S->napply = napply; a.S->done = 0; }
        if (tid == 0) s_flag = 0;
        __syncthreads();
        if (tid < K && s_act0[tid]) atomicOr(&s_flag, 1);
        __syncthreads();
        if (!s_flag) break;
        // the sweep buffers start empty; the state above is visible after the barrier
        if (a.sweeps == 1) { fill_empty(a.e0); fill_empty(a.z); }
        BK_BAR();
        if (!precond(true)) { fail(); return; }
        bk_gz_body(a, 1);
        BK_BAR();
        bk_pnext_body(a);
        BK_BAR();
        while (true) {
            rows(0, 0, a.pt);
            if (a.sweeps == 1) { fill_empty(a.e0); fill_empty(a.z); }
            BK_BAR();
            cols(0, a.w);
            BK_BAR();
            bk_update_body(a);
            BK_BAR();
            if (__ldcg(&a.S->done)) break;
            if (!precond(true)) { fail(); return; }
            bk_gz_body(a, 0);
            BK_BAR();
            bk_pnext_body(a);
            BK_BAR();
        }
        if (tid < K && s_act0[tid]) {
            const int c = tid;
            const int it = __ldcg(&a.S->iters[c]);
            if (it > s_iters[c]) s_dirty[c] = 1;
            s_iters[c] = it;
            s_rec[c] = __ldcg(&a.S->rec[c]);
            if (__ldcg(&a.S->broke[c])) s_broke[c] = 1;
        }
        napply = __ldcg(&a.S->napply);
        __syncthreads();
        // block 0 resets the state words the next outer step writes, only after every CTA
        // has read them
        BK_BAR();
    }
    // a final true residual for the columns that iterated since the last one
    if (tid == 0) s_flag = 0;
    __syncthreads();
    if (tid < K && s_dirty[tid] && !s_broke[tid] && !s_conv[tid]) atomicOr(&s_flag, 1);
    __syncthreads();
    if (s_flag) {
        const bool was = tid < K && s_dirty[tid] && !s_broke[tid] && !s_conv[tid];
        if (!true_residual()) { fail(); return; }
        if (was) {
            const int c = tid;
            s_tru[c] = s_gn[c] / s_hn[c];
            s_raw[c] = s_hnraw[c] > 0.0 ? s_gnraw[c] / s_hnraw[c] : 0.0;
            if (s_tru[c] <= a.tol) s_conv[c] = 1;
        }
        __syncthreads();
    }
    // x = D^{-1} y, column-major
    for (int64_t t = gtid; t < nK; t += gstride) {
        const int64_t c = t / a.n, j = t % a.n;
        P.X[c * P.ldx + j] = a.y[j * K + c] * a.inv_d[j];
    }
    if (blockIdx.x == 0 && tid < K) {
        const int c = tid;
        P.out->iters[c] = s_iters[c];
        P.out->outer[c] = s_outer[c];
        P.out->conv[c] = s_conv[c];
        P.out->rec[c] = s_rec[c];
        P.out->tru[c] = s_tru[c];
        P.out->raw[c] = s_raw[c];
        P.out->status[c] = s_conv[c] ? LSQ_OK : (s_broke[c] ? LSQ_ERR_BREAKDOWN : LSQ_ERR_NOT_CONVERGED);
    }
#undef BK_BAR
}


// The kernel for a value type and an operator type, chosen by sweep form and K.
template <int DT, typename MT>
const void* persist_kernel(int smode, int K) {
    if (smode == 0) return (const void*)k_bk_persist<DT, MT, 0, 1>;
    if (smode == 1) {
        if (K <= 4) return (const void*)k_bk_persist<DT, MT, 1, 4>;
        if (K <= 16) return (const void*)k_bk_persist<DT, MT, 1, 16>;
        return (const void*)k_bk_persist<DT, MT, 1, 32>;
    }
    if (K <= 4) return (const void*)k_bk_persist<DT, MT, 2, 4>;
    if (K <= 16) return (const void*)k_bk_persist<DT, MT, 2, 16>;
    return (const void*)k_bk_persist<DT, MT, 2, 32>;
}

}  // namespace lsq
