// Alg. 2 step 4 for a batch of independent small dense problems (uneven m_p x n_p, n_p <= 256,
// FP32 values, k <= 16 right-hand sides each), all solved in ONE kernel launch.
//
// Each problem is solved by one thread-block cluster of C CTAs (C = 1..16, picked by the
// autotuner).  Clusters take problems from a queue, largest first, and never wait on one
// another; the C CTAs of a cluster split
// the problem's rows and meet at hardware cluster barriers, exchanging partial results through
// distributed shared memory.  Per iteration (K = k columns advanced together, each with its
// own alpha, beta, rho and convergence mask):
//   row pass   every CTA streams its rows of A through shared memory (cp.async, double
//              buffered) and computes Q = A P~ (P~ = D^{-1} P) then W += A^T Q on the tile,
//              with ||Q||^2 = p^T w per column on the side
//   cluster    CTA r sums its slice of W over the cluster (DSMEM, fixed order): alpha, y, g,
//              ||g||^2; the masks; z = (materialised SGS operator) g on the slice; rho', beta,
//              p, and the next P~ broadcast into every CTA's shared memory
// The inner iteration runs in FP32 (products and the W accumulation); all vectors, dots and
// scalars are FP64.  Restarts (outer steps) recompute g from the residual D^{-1} A^T (b - A x)
// in double-float on the FP32 units (about 48 bits; A's values are exact in FP32), which also
// refines x.
// Every decision (alpha, masks, loop exits) is computed identically by all CTAs of a cluster
// from the same sums in the same order, so their control flow cannot diverge.
#include "batch.cuh"
#include "dfloat.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

namespace cg = cooperative_groups;

namespace lsq {

constexpr int BT = 512;            // threads per CTA (16 warps; 128 registers each)
constexpr int BR = 32;             // rows per tile
constexpr int TPR = BT / BR;       // threads per tile row in the Q step (16)
constexpr int NPMAX = 256;         // largest padded n
constexpr int LDS = NPMAX + 8;     // shared-memory pitch of a tile row (floats; 8 keeps
                                   // the float4 reads of 4 rows on distinct banks)

// Shared-memory layout for KC columns (byte offsets; every part 16-byte aligned)
// P~ / x rows in shared memory are XP entries apart: 4 entries of padding (from 4 columns up)
// put the rows that the threads of one tile row read together on different banks
template <int KC> struct XPitch { static constexpr int v = KC >= 4 ? KC + 4 : KC; };
template <int KC>
struct BLayout {
    static constexpr size_t as = 0;                                   // two A tiles (float)
    static constexpr size_t xs = as + 2 * (size_t)BR * LDS * 4;       // P~ (float) or x (pairs)
    static constexpr size_t wp = xs + (size_t)NPMAX * XPitch<KC>::v * 8;   // this CTA's W
    static constexpr size_t qs = wp + (size_t)NPMAX * KC * 8;         // Q of the current tile
    static constexpr size_t red = qs + (size_t)BR * KC * 8;           // reduction scratch
    static constexpr size_t st = red + (size_t)BT * 4 * 8;            // per-column state
    static constexpr size_t bytes = st + 32 * 32 * 8;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool full) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = full ? 16 : 0;   // 0: fill the 16 bytes with zeros
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }


// Rows [r_lo, r_hi) of problem P, KC columns, arithmetic type T (float: inner iteration;
// double: FP64 residual):
//   Q = A X          (mode 0)   or   Q = b - A X   (mode 1, T = double)
//   Wp = A^T Q over these rows, qq_out[c] = sum of Q_ic^2 over these rows (c < k)
// X (npad x KC, rows j >= n zero) is in shared memory.  Tiles of BR rows are streamed with
// cp.async into two buffers; the next tile is in flight while the current one is used.
// Q step: TPR threads per tile row, each CQ columns over a JS-th of the row, combined by
// shuffles.  W step: a thread owns 4 consecutive j and CQ columns (RS threads split the rows
// when there are fewer such units than threads) and accumulates over all tiles in registers.
template <int KC, typename T>
__device__ void bt_row_pass(const BatchProb& P, int64_t r_lo, int64_t r_hi, int mode, int k,
                            float* As, const T* Xs, T* Qs, T* Wp, double* qq_out, double* red) {
    constexpr int CQ = KC < 4 ? KC : 4;
    constexpr int CG = KC / CQ;
    constexpr int JS = TPR / CG;
    const int tid = threadIdx.x;
    const int n = (int)P.n, npad = (int)P.npad, nch = npad / 4;
    const int64_t rows = r_hi > r_lo ? r_hi - r_lo : 0;
    const int ntile = (int)((rows + BR - 1) / BR);
    const int units = nch * CG;
    const int RS = units >= BT ? 1 : BT / units;
    const bool wact = tid < units * RS;
    const int unit = tid % units, rs = tid / units;
    const int jg = unit / CG, cgw = unit % CG;
    T acc[4][CQ];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < CQ; ++c) acc[u][c] = T(0);
    // ||Q||^2 in double-float on the FP32 units (the FP64 pipe runs at 1/64 of their rate)
    f2 qq[CQ];
#pragma unroll
    for (int c = 0; c < CQ; ++c) qq[c] = f2{0.f, 0.f};
    const int qr = tid / TPR, qsub = tid % TPR, qcg = qsub % CG, qjs = qsub / CG;

    auto load_tile = [&](int t, int buf) {
        float* dst = As + buf * BR * LDS;
        const int64_t row0 = r_lo + (int64_t)t * BR;
        for (int q = tid; q < BR * nch; q += BT) {
            const int r = q / nch, ch = q % nch;
            const int64_t i = row0 + r;
            const bool ok = i < r_hi;
            cp_async16(dst + r * LDS + 4 * ch, P.A + (ok ? i : r_lo) * P.ld + 4 * ch, ok);
        }
        cp_async_commit();
    };
    if (ntile > 0) load_tile(0, 0);
    for (int t = 0; t < ntile; ++t) {
        cp_async_wait_all();
        __syncthreads();   // tile t has landed; every thread is done with tile t-1
        if (t + 1 < ntile) load_tile(t + 1, (t + 1) & 1);
        float* At = As + (t & 1) * BR * LDS;
        if (n < npad) {    // A's padding columns n..npad-1 may hold anything
            const int pw = npad - n;
            for (int q = tid; q < BR * pw; q += BT) At[(q / pw) * LDS + n + q % pw] = 0.f;
            __syncthreads();
        }
        {   // Q step
            T sacc[CQ];
#pragma unroll
            for (int c = 0; c < CQ; ++c) sacc[c] = T(0);
            for (int ch = qjs; ch < nch; ch += JS) {
                const float4 a4 = *reinterpret_cast<const float4*>(At + qr * LDS + 4 * ch);
                const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const T* xr = Xs + (4 * ch + u) * XPitch<KC>::v + qcg * CQ;
                    T xv[CQ];
                    if constexpr (CQ == 4 && sizeof(T) == 4) {
                        const float4 x4 = *reinterpret_cast<const float4*>(xr);
                        xv[0] = x4.x; xv[1] = x4.y; xv[2] = x4.z; xv[3] = x4.w;
                    } else {
#pragma unroll
                        for (int c = 0; c < CQ; ++c) xv[c] = xr[c];
                    }
#pragma unroll
                    for (int c = 0; c < CQ; ++c) sacc[c] = fma((T)av[u], xv[c], sacc[c]);
                }
            }
#pragma unroll
            for (int o = CG; o < TPR; o <<= 1)
#pragma unroll
                for (int c = 0; c < CQ; ++c) sacc[c] += __shfl_xor_sync(0xffffffffu, sacc[c], o);
            if (qjs == 0) {
                const int64_t i = r_lo + (int64_t)t * BR + qr;
                const bool ok = i < r_hi;
#pragma unroll
                for (int cc = 0; cc < CQ; ++cc) {
                    const int c = qcg * CQ + cc;
                    T q = T(0);
                    if (ok && c < k) {
                        q = sacc[cc];
                        if (mode == 1) q = (T)(P.B[(int64_t)c * P.ldb + i] - (double)sacc[cc]);
                        df_add_sq(qq[cc], (float)q);
                    }
                    Qs[qr * KC + c] = q;
                }
            }
        }
        __syncthreads();
        if (wact) {   // W step
            for (int r = rs; r < BR; r += RS) {
                const float4 a4 = *reinterpret_cast<const float4*>(At + r * LDS + 4 * jg);
                const float av[4] = {a4.x, a4.y, a4.z, a4.w};
                T qv[CQ];
#pragma unroll
                for (int c = 0; c < CQ; ++c) qv[c] = Qs[r * KC + cgw * CQ + c];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int c = 0; c < CQ; ++c) acc[u][c] = fma((T)av[u], qv[c], acc[u][c]);
            }
        }
    }
    __syncthreads();
    // this CTA's W: the RS row groups added in a fixed order
    for (int gph = 0; gph < RS; ++gph) {
        if (wact && rs == gph) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int c = 0; c < CQ; ++c) {
                    const int at = (4 * jg + u) * KC + cgw * CQ + c;
                    Wp[at] = (gph == 0 ? T(0) : Wp[at]) + acc[u][c];
                }
        }
        __syncthreads();
    }
    // ||Q||^2 per column: the js == 0 threads of every tile row, in row order
#pragma unroll
    for (int c = 0; c < CQ; ++c) red[tid * CQ + c] = (qjs == 0) ? df_to_double(qq[c]) : 0.0;
    __syncthreads();
    if (tid < KC) {
        const int g = tid / CQ, cc = tid % CQ;
        double sum = 0.0;
        for (int r = 0; r < BR; ++r) sum += red[(r * TPR + g) * CQ + cc];
        qq_out[tid] = sum;
    }
    __syncthreads();
}

// The FP64-accurate residual pass in double-float on the FP32 units (A's values are exact
// in FP32; x and q are (hi, lo) float pairs; products and sums follow the cascaded Dot2 form
// of Ogita, Rump & Oishi):  Q = b - A X, Wp = A^T Q over rows [r_lo, r_hi) (pairs), qq_out
// unused.  Same tiling and thread roles as bt_row_pass.
__device__ __forceinline__ void bt_cascade(f2& acc, float a, f2 x) {
    float p, pe;
    two_prod(a, x.hi, p, pe);
    pe = fmaf(a, x.lo, pe);
    float s, e;
    two_sum(acc.hi, p, s, e);
    acc.hi = s;
    acc.lo += e + pe;
}
template <int KC>
__device__ void bt_residual_pass(const BatchProb& P, int64_t r_lo, int64_t r_hi, int k, float* As,
                                 const f2* Xs, f2* Qs, f2* Wp) {
    constexpr int CQ = KC < 4 ? KC : 4;
    constexpr int CG = KC / CQ;
    constexpr int JS = TPR / CG;
    const int tid = threadIdx.x;
    const int n = (int)P.n, npad = (int)P.npad, nch = npad / 4;
    const int64_t rows = r_hi > r_lo ? r_hi - r_lo : 0;
    const int ntile = (int)((rows + BR - 1) / BR);
    const int units = nch * CG;
    const int RS = units >= BT ? 1 : BT / units;
    const bool wact = tid < units * RS;
    const int unit = tid % units, rs = tid / units;
    const int jg = unit / CG, cgw = unit % CG;
    f2 acc[4][CQ];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < CQ; ++c) acc[u][c] = f2{0.f, 0.f};
    const int qr = tid / TPR, qsub = tid % TPR, qcg = qsub % CG, qjs = qsub / CG;
    auto load_tile = [&](int t, int buf) {
        float* dst = As + buf * BR * LDS;
        const int64_t row0 = r_lo + (int64_t)t * BR;
        for (int q = tid; q < BR * nch; q += BT) {
            const int r = q / nch, ch = q % nch;
            const int64_t i = row0 + r;
            const bool ok = i < r_hi;
            cp_async16(dst + r * LDS + 4 * ch, P.A + (ok ? i : r_lo) * P.ld + 4 * ch, ok);
        }
        cp_async_commit();
    };
    if (ntile > 0) load_tile(0, 0);
    for (int t = 0; t < ntile; ++t) {
        cp_async_wait_all();
        __syncthreads();
        if (t + 1 < ntile) load_tile(t + 1, (t + 1) & 1);
        float* At = As + (t & 1) * BR * LDS;
        if (n < npad) {
            const int pw = npad - n;
            for (int q = tid; q < BR * pw; q += BT) At[(q / pw) * LDS + n + q % pw] = 0.f;
            __syncthreads();
        }
        {   // Q = b - A x for this tile's rows
            f2 sacc[CQ];
#pragma unroll
            for (int c = 0; c < CQ; ++c) sacc[c] = f2{0.f, 0.f};
            for (int ch = qjs; ch < nch; ch += JS) {
                const float4 a4 = *reinterpret_cast<const float4*>(At + qr * LDS + 4 * ch);
                const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const f2* xr = Xs + (4 * ch + u) * XPitch<KC>::v + qcg * CQ;
#pragma unroll
                    for (int c = 0; c < CQ; ++c) bt_cascade(sacc[c], av[u], xr[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < CQ; ++c) sacc[c] = df_norm(sacc[c]);
#pragma unroll
            for (int o = CG; o < TPR; o <<= 1)
#pragma unroll
                for (int c = 0; c < CQ; ++c) df_add(sacc[c], df_shfl_xor(sacc[c], o));
            if (qjs == 0) {
                const int64_t i = r_lo + (int64_t)t * BR + qr;
                const bool ok = i < r_hi;
#pragma unroll
                for (int cc = 0; cc < CQ; ++cc) {
                    const int c = qcg * CQ + cc;
                    f2 q = f2{0.f, 0.f};
                    if (ok && c < k) q = df_from_double(P.B[(int64_t)c * P.ldb + i] - df_to_double(sacc[cc]));
                    Qs[qr * KC + c] = q;
                }
            }
        }
        __syncthreads();
        if (wact) {   // W += A^T Q
            for (int r = rs; r < BR; r += RS) {
                const float4 a4 = *reinterpret_cast<const float4*>(At + r * LDS + 4 * jg);
                const float av[4] = {a4.x, a4.y, a4.z, a4.w};
                f2 qv[CQ];
#pragma unroll
                for (int c = 0; c < CQ; ++c) qv[c] = Qs[r * KC + cgw * CQ + c];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int c = 0; c < CQ; ++c) bt_cascade(acc[u][c], av[u], qv[c]);
            }
        }
    }
    __syncthreads();
    for (int gph = 0; gph < RS; ++gph) {
        if (wact && rs == gph) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int c = 0; c < CQ; ++c) {
                    const int at = (4 * jg + u) * KC + cgw * CQ + c;
                    f2 v = df_norm(acc[u][c]);
                    if (gph > 0) df_add(v, Wp[at]);
                    Wp[at] = v;
                }
        }
        __syncthreads();
    }
}

// Per-column state of the problem being solved, identical in every CTA of the cluster
// (each CTA computes it from the same cluster sums in the same order)
struct BtState {
    double rho[16], hn[16], hnr[16], gst[16], gn[16], gnr[16], rec[16], tru[16], raw[16], alpha[16];
    double slot[2][2][16];   // two rotating pairs of per-CTA partial sums read by the cluster
    double t0[16], t1[16];   // cluster totals of the last reduction
    double qq[16];           // this CTA's ||Q||^2 per column
    int32_t active[16], iters[16], conv[16], broke[16], outer[16], dirty[16];
    int32_t any;
    int32_t next;            // rank 0: the queue position this cluster took
};
static_assert(sizeof(BtState) <= 32 * 32 * 8, "state does not fit its shared-memory slot");

// Per-column totals over the cluster of the two partial vectors in slot `sl`, read through
// distributed shared memory in rank order: t0[c], t1[c] (c < KC), then a block barrier.
template <int KC>
__device__ __forceinline__ void bt_cluster_sum(cg::cluster_group& cl, BtState* S, int sl, double* t0, double* t1) {
    const int tid = threadIdx.x;
    if (tid < 2 * KC) {
        const int which = tid / KC, c = tid % KC;
        double sum = 0.0;
        for (unsigned r = 0; r < cl.num_blocks(); ++r) {
            const BtState* R = cl.map_shared_rank(S, r);
            sum += R->slot[sl][which][c];
        }
        (which == 0 ? t0 : t1)[c] = sum;
    }
    __syncthreads();
}

// This CTA's per-column partial sums of a and b over its slice (thread t always holds
// column t % KC), written into slot `sl` in thread order.
template <int KC>
__device__ __forceinline__ void bt_slice_partials(double a, double b, BtState* S, int sl, double* red) {
    const int tid = threadIdx.x;
    red[tid] = a;
    red[BT + tid] = b;
    __syncthreads();
    if (tid < 2 * KC) {
        const int which = tid / KC, c = tid % KC;
        double sum = 0.0;
        for (int i = c; i < BT; i += KC) sum += red[which * BT + i];
        S->slot[sl][which][c] = sum;
    }
    __syncthreads();
}


// Solves one problem with the cluster: outer restarts from the FP64 residual around an FP32
// inner PCG, per-column masks.  Every CTA runs the same control flow.
template <int KC>
__device__ void bt_solve_problem(cg::cluster_group& cl, const BatchProb& P, int pid, int k, BatchOut* out,
                                 double tol, double inner_tol, int maxit, int max_outer, unsigned char* smem) {
    using Ly = BLayout<KC>;
    float* As = reinterpret_cast<float*>(smem + Ly::as);
    float* Xf = reinterpret_cast<float*>(smem + Ly::xs);
    f2* Xp = reinterpret_cast<f2*>(smem + Ly::xs);
    float* Wf = reinterpret_cast<float*>(smem + Ly::wp);
    f2* Wpp = reinterpret_cast<f2*>(smem + Ly::wp);
    float* Qf = reinterpret_cast<float*>(smem + Ly::qs);
    f2* Qp = reinterpret_cast<f2*>(smem + Ly::qs);
    double* red = reinterpret_cast<double*>(smem + Ly::red);
    BtState* S = reinterpret_cast<BtState*>(smem + Ly::st);
    const int tid = threadIdx.x;
    const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int n = (int)P.n, npad = (int)P.npad;
    const int64_t r_lo = P.m * rank / C, r_hi = P.m * (rank + 1) / C;
    const int e_lo = (int)((int64_t)npad * rank / C) * KC, e_hi = (int)((int64_t)npad * (rank + 1) / C) * KC;
    const int NK = npad * KC;
    constexpr int XP = XPitch<KC>::v;
    double* y = P.ws;
    double* g = y + NK;
    double* z = g + NK;
    double* p = z + NK;
    double* h = p + NK;
    int sl = 0;

    // g-like vector from the FP64 residual: dst = D^{-1} A^T (b - A x), x = D^{-1} y (or 0);
    // S->t0 = ||dst||^2, S->t1 = ||A^T (b - A x)||^2 per column
    auto residual = [&](bool from_zero, double* dst) {
        for (int e = tid; e < NK; e += BT) {
            const int j = e / KC, c = e % KC;
            Xp[j * XP + c] = df_from_double((!from_zero && j < n) ? __ldcg(y + e) * P.inv_d[j] : 0.0);
        }
        __syncthreads();
        bt_residual_pass<KC>(P, r_lo, r_hi, k, As, Xp, Qp, Wpp);
        cl.sync();
        double a = 0.0, b = 0.0;
        for (int e = e_lo + tid; e < e_hi; e += BT) {
            const int j = e / KC;
            double sum = 0.0;
            for (int r = 0; r < C; ++r) sum += df_to_double(cl.map_shared_rank(Wpp, r)[e]);
            const double v = j < n ? sum * P.inv_d[j] : 0.0;
            dst[e] = v;
            a = fma(v, v, a);
            b = fma(sum, sum, b);
        }
        bt_slice_partials<KC>(a, b, S, sl, red);
        __threadfence();
        cl.sync();
        bt_cluster_sum<KC>(cl, S, sl, S->t0, S->t1);
        sl ^= 1;
    };
    // z = (SGS operator) g on this CTA's slice, FP32 arithmetic; S->t0 = g^T z per column
    auto apply_op = [&]() {
        for (int e = tid; e < NK; e += BT) Xf[(e / KC) * XP + e % KC] = (float)__ldcg(g + e);
        __syncthreads();
        double a = 0.0;
        for (int e = e_lo + tid; e < e_hi; e += BT) {
            const int j = e / KC, c = e % KC;
            double zv = 0.0;
            if (j < n && c < k) {
                float sacc = 0.f;
                if (P.op_f32) {
                    const float* o = reinterpret_cast<const float*>(P.op) + (int64_t)j * n;
                    for (int l = 0; l < n; ++l) sacc = fmaf(o[l], Xf[l * XP + c], sacc);
                } else {
                    const double* o = reinterpret_cast<const double*>(P.op) + (int64_t)j * n;
                    for (int l = 0; l < n; ++l) sacc = fmaf((float)o[l], Xf[l * XP + c], sacc);
                }
                zv = sacc;
            }
            z[e] = zv;
            a = fma(g[e], zv, a);
        }
        bt_slice_partials<KC>(a, 0.0, S, sl, red);
        cl.sync();
        bt_cluster_sum<KC>(cl, S, sl, S->t0, S->t1);
        sl ^= 1;
    };
    // p = z (first) or z + beta p on the active columns (beta in S->alpha); P~ = D^{-1} p into
    // every CTA's Xf (zero for frozen columns and padding rows); then a cluster barrier
    auto next_p = [&](bool first) {
        for (int e = e_lo + tid; e < e_hi; e += BT) {
            const int j = e / KC, c = e % KC;
            float pt = 0.f;
            if (S->active[c]) {
                const double pv = first ? z[e] : fma(S->alpha[c], p[e], z[e]);
                p[e] = pv;
                if (j < n) pt = (float)(pv * P.inv_d[j]);
            }
            for (int r = 0; r < C; ++r) cl.map_shared_rank(Xf, r)[j * XP + c] = pt;
        }
        cl.sync();
    };

    // start: y = 0, h = D^{-1} A^T b, g = h
    for (int e = e_lo + tid; e < e_hi; e += BT) y[e] = 0.0;
    residual(true, h);
    for (int e = e_lo + tid; e < e_hi; e += BT) g[e] = h[e];
    if (tid < KC) {
        const int c = tid;
        S->hn[c] = sqrt(S->t0[c]);
        S->hnr[c] = sqrt(S->t1[c]);
        S->gn[c] = S->hn[c];
        S->gnr[c] = S->hnr[c];
        S->iters[c] = 0; S->outer[c] = 0; S->broke[c] = 0; S->dirty[c] = 0; S->active[c] = 0;
        S->conv[c] = (c >= k || S->hn[c] == 0.0) ? 1 : 0;
        const double one = S->hn[c] == 0.0 ? 0.0 : 1.0;
        S->rec[c] = one; S->tru[c] = one; S->raw[c] = one;
    }
    __threadfence();
    cl.sync();
    for (int outer = 0; outer < max_outer; ++outer) {
        if (outer > 0) {
            residual(false, g);
            if (tid < KC) {
                S->gn[tid] = sqrt(S->t0[tid]);
                S->gnr[tid] = sqrt(S->t1[tid]);
                S->dirty[tid] = 0;
            }
        }
        if (tid == 0) S->any = 0;
        __syncthreads();
        if (tid < KC) {
            const int c = tid;
            S->active[c] = 0;
            if (c < k && S->hn[c] != 0.0 && !S->broke[c]) {
                S->tru[c] = S->gn[c] / S->hn[c];
                S->raw[c] = S->hnr[c] > 0.0 ? S->gnr[c] / S->hnr[c] : 0.0;
                if (outer == 0) S->rec[c] = S->tru[c];
                if (S->tru[c] <= tol) {
                    S->conv[c] = 1;
                } else {
                    S->conv[c] = 0;
                    if (S->iters[c] < maxit) {
                        S->active[c] = 1;
                        S->gst[c] = S->gn[c];
                        S->outer[c] = outer + 1;
                        atomicOr(&S->any, 1);
                    }
                }
            }
        }
        __syncthreads();
        if (!S->any) break;
        // z = P g, rho = g^T z, p = z
        apply_op();
        if (tid < KC && S->active[tid]) S->rho[tid] = S->t0[tid];
        __syncthreads();
        next_p(true);
        while (true) {
            // q = Â p, w = Â^T q (this CTA's rows), p^T w = ||q||^2
            bt_row_pass<KC, float>(P, r_lo, r_hi, 0, k, As, Xf, Qf, Wf, S->qq, red);
            if (tid < KC) { S->slot[sl][0][tid] = S->qq[tid]; S->slot[sl][1][tid] = 0.0; }
            __syncthreads();
            cl.sync();
            bt_cluster_sum<KC>(cl, S, sl, S->t0, S->t1);
            sl ^= 1;
            if (tid < KC) {
                const int c = tid;
                double al = 0.0;
                if (S->active[c]) {
                    const double pw = S->t0[c], rho = S->rho[c];
                    if (!(pw > 0.0 && rho > 0.0 && isfinite(pw) && isfinite(rho))) {
                        S->broke[c] = 1;
                        S->active[c] = 0;
                    } else {
                        al = rho / pw;
                    }
                }
                S->alpha[c] = al;
            }
            __syncthreads();
            // y += alpha p, g -= alpha D^{-1} (sum of the cluster's W), ||g||^2
            double gg = 0.0;
            for (int e = e_lo + tid; e < e_hi; e += BT) {
                const int j = e / KC, c = e % KC;
                const double al = S->alpha[c];
                double w = 0.0;
                if (j < n) {
                    double sum = 0.0;
                    for (int r = 0; r < C; ++r) sum += (double)cl.map_shared_rank(Wf, r)[e];
                    w = sum * P.inv_d[j];
                }
                y[e] = fma(al, p[e], y[e]);
                const double gv = fma(-al, w, g[e]);
                g[e] = gv;
                gg = fma(gv, gv, gg);
            }
            bt_slice_partials<KC>(gg, 0.0, S, sl, red);
            __threadfence();
            cl.sync();
            bt_cluster_sum<KC>(cl, S, sl, S->t0, S->t1);
            sl ^= 1;
            if (tid == 0) S->any = 0;
            __syncthreads();
            if (tid < KC) {
                const int c = tid;
                if (S->active[c]) {
                    S->iters[c] += 1;
                    S->dirty[c] = 1;
                    const double gn = sqrt(S->t0[c]);
                    S->rec[c] = gn / S->hn[c];
                    if (gn <= tol * S->hn[c] || gn <= inner_tol * S->gst[c] || S->iters[c] >= maxit)
                        S->active[c] = 0;
                }
                if (S->active[c]) atomicOr(&S->any, 1);
            }
            __syncthreads();
            if (!S->any) break;
            apply_op();
            if (tid < KC && S->active[tid]) {
                S->alpha[tid] = S->t0[tid] / S->rho[tid];   // beta
                S->rho[tid] = S->t0[tid];
            }
            __syncthreads();
            next_p(false);
        }
    }
    // the true residual of columns that moved since their last check
    if (tid == 0) S->any = 0;
    __syncthreads();
    if (tid < KC && S->dirty[tid] && !S->conv[tid] && !S->broke[tid]) atomicOr(&S->any, 1);
    __syncthreads();
    if (S->any) {
        residual(false, g);
        if (tid < KC) {
            const int c = tid;
            if (S->dirty[c] && !S->conv[c] && !S->broke[c]) {
                S->tru[c] = sqrt(S->t0[c]) / S->hn[c];
                S->raw[c] = S->hnr[c] > 0.0 ? sqrt(S->t1[c]) / S->hnr[c] : 0.0;
                if (S->tru[c] <= tol) S->conv[c] = 1;
            }
        }
        __syncthreads();
    }
    // x = D^{-1} y
    for (int e = e_lo + tid; e < e_hi; e += BT) {
        const int j = e / KC, c = e % KC;
        if (j < n && c < k) P.X[(int64_t)c * P.ldx + j] = y[e] * P.inv_d[j];
    }
    if (rank == 0 && tid < k) {
        BatchOut o;
        o.iters = S->iters[tid]; o.outer = S->outer[tid]; o.conv = S->conv[tid]; o.broke = S->broke[tid];
        o.rec = S->rec[tid]; o.tru = S->tru[tid]; o.raw = S->raw[tid];
        out[(int64_t)pid * k + tid] = o;
    }
    __threadfence();
    cl.sync();   // the next problem reuses every shared-memory buffer
}

// One launch for the whole batch.  plist holds the problems largest first; each cluster takes
// the next one from a queue (rank 0 increments *queue, the cluster reads its value through
// distributed shared memory), so the clusters stay busy until the queue is empty.  The queue
// counter is zeroed before every launch.
template <int KC>
__global__ void __launch_bounds__(BT, 1) k_pcg_batch(const BatchProb* probs, const int32_t* plist, int count,
                                                     int* queue, int k, BatchOut* out, double tol,
                                                     double inner_tol, int maxit, int max_outer) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    BtState* S = reinterpret_cast<BtState*>(smem + BLayout<KC>::st);
    while (true) {
        if (cl.block_rank() == 0 && threadIdx.x == 0) S->next = atomicAdd(queue, 1);
        cl.sync();
        const int at = cl.map_shared_rank(S, 0)->next;   // the same value in every CTA
        if (at >= count) break;
        const int pid = plist[at];
        bt_solve_problem<KC>(cl, probs[pid], pid, k, out, tol, inner_tol, maxit, max_outer, smem);
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

}  // namespace lsq

// ---------------------------------------------------------------------------------------
// Host side: the plan, cluster assignment, launch, autotuner
// ---------------------------------------------------------------------------------------
struct lsq_batch {
    int64_t count = 0;
    int k = 1, kc = 1;
    lsq_opts o{};
    cudaStream_t stream = 0;
    std::vector<int64_t> cost;          // per problem: m x padded n (elements of A per pass)
    lsq::BatchProb* dprobs = nullptr;
    lsq::BatchOut* dout = nullptr;
    double* ws = nullptr;
    int32_t* dplist = nullptr;          // problems, largest first
    int* dqueue = nullptr;              // queue position, zeroed before each launch
    int max_clusters = 0;
    int cluster = 0, nclusters = 0;     // current plan
};

namespace lsq {

static const void* bt_kernel_for(int kc) {
    switch (kc) {
        case 1: return (const void*)k_pcg_batch<1>;
        case 2: return (const void*)k_pcg_batch<2>;
        case 4: return (const void*)k_pcg_batch<4>;
        case 8: return (const void*)k_pcg_batch<8>;
        default: return (const void*)k_pcg_batch<16>;
    }
}
static size_t bt_smem_for(int kc) {
    switch (kc) {
        case 1: return BLayout<1>::bytes;
        case 2: return BLayout<2>::bytes;
        case 4: return BLayout<4>::bytes;
        case 8: return BLayout<8>::bytes;
        default: return BLayout<16>::bytes;
    }
}

// Clusters of C CTAs that can be resident at once (0 if C is not available).
static lsq_status bt_max_clusters(int kc, int C, int* out) {
    const void* kern = bt_kernel_for(kc);
    const size_t smem = bt_smem_for(kc);
    LSQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    *out = 0;
    if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return LSQ_OK;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        nc = 0;
    }
    *out = nc;
    return LSQ_OK;
}

static lsq_status bt_set_cluster(lsq_batch* b, int C) {
    int nc = 0;
    lsq_status r = bt_max_clusters(b->kc, C, &nc);
    if (r != LSQ_OK) return r;
    if (nc < 1) {
        set_error("cluster size not available on this device");
        return LSQ_ERR_UNSUPPORTED;
    }
    nc = (int)std::min<int64_t>(nc, std::min<int64_t>(b->count, b->max_clusters));
    b->cluster = C;
    b->nclusters = nc;
    return LSQ_OK;
}

template <int KC>
static cudaError_t bt_launch(lsq_batch* b, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = b->cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(b->nclusters * b->cluster);
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = BLayout<KC>::bytes;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const double inner = b->o.inner_tol > 0 ? b->o.inner_tol : 0.0;
    return cudaLaunchKernelEx(&cfg, k_pcg_batch<KC>, (const BatchProb*)b->dprobs, (const int32_t*)b->dplist,
                              (int)b->count, b->dqueue, b->k, b->dout, b->o.tol, inner,
                              (int)b->o.maxit, (int)b->o.max_outer);
}

static lsq_status bt_solve(lsq_batch* b, cudaStream_t st) {
    LSQ_CUDA(cudaMemsetAsync(b->dqueue, 0, sizeof(int), st));
    cudaError_t e;
    switch (b->kc) {
        case 1: e = bt_launch<1>(b, st); break;
        case 2: e = bt_launch<2>(b, st); break;
        case 4: e = bt_launch<4>(b, st); break;
        case 8: e = bt_launch<8>(b, st); break;
        default: e = bt_launch<16>(b, st); break;
    }
    LSQ_CUDA(e);
    count_launch();
    return LSQ_OK;
}

}  // namespace lsq

using namespace lsq;

extern "C" lsq_status lsq_batch_create(const lsq_batch_problem* probs, int64_t count, int64_t k,
                                       const lsq_opts* o, lsq_batch** out, void* stream) {
    LSQ_CHECK_ARG(out != nullptr && probs != nullptr && o != nullptr, "null argument");
    *out = nullptr;
    LSQ_CHECK_ARG(count >= 1 && count < (1 << 30), "count must be in [1, 2^30)");
    LSQ_CHECK_ARG(k >= 1 && k <= 16, "k must be in [1, 16]");
    LSQ_CHECK_ARG(o->maxit >= 0 && o->max_outer >= 1 && o->tol >= 0.0, "bad options");
    cudaStream_t st = (cudaStream_t)stream;
    int kc = 1;
    while (kc < k) kc <<= 1;
    std::vector<BatchProb> hp(count);
    std::vector<int64_t> cost(count);
    size_t ws_total = 0;
    for (int64_t i = 0; i < count; ++i) {
        const lsq_batch_problem& q = probs[i];
        LSQ_CHECK_ARG(q.m >= 1 && q.n >= 1 && q.n <= NPMAX, "each problem needs m >= 1 and 1 <= n <= 256");
        LSQ_CHECK_ARG(q.ld >= q.n && q.ld % 4 == 0, "ld must be >= n and a multiple of 4");
        LSQ_CHECK_ARG(q.A != nullptr && ((uintptr_t)q.A & 15) == 0, "A must be 16-byte aligned");
        LSQ_CHECK_ARG(q.P != nullptr && q.P->sp == nullptr && q.P->op != nullptr && q.P->n == q.n,
                      "P must be a dense handle built for this problem");
        LSQ_CHECK_ARG(q.B != nullptr && q.ldb >= q.m && q.X != nullptr && q.ldx >= q.n, "bad B or X");
        BatchProb& b = hp[i];
        b.m = q.m; b.n = q.n; b.npad = (q.n + 3) / 4 * 4; b.ld = q.ld;
        b.A = q.A; b.op = q.P->op; b.op_f32 = q.P->op_dtype == LSQ_F32 ? 1 : 0; b.inv_d = q.P->inv_d;
        b.B = q.B; b.ldb = q.ldb; b.X = q.X; b.ldx = q.ldx;
        cost[i] = q.m * b.npad;
        ws_total += 5 * (size_t)b.npad * kc;
    }
    lsq_batch* B = new lsq_batch();
    B->count = count; B->k = (int)k; B->kc = kc; B->o = *o; B->stream = st; B->cost = cost;
    int dev = 0, sms = 0;
    auto fail = [&](lsq_status s) { lsq_batch_destroy(B); return s; };
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        set_error("no CUDA device");
        return fail(LSQ_ERR_CUDA);
    }
    B->max_clusters = sms;
    if (cudaMalloc(&B->dprobs, sizeof(BatchProb) * count) != cudaSuccess ||
        cudaMalloc(&B->dout, sizeof(BatchOut) * count * k) != cudaSuccess ||
        cudaMalloc(&B->ws, 8 * ws_total) != cudaSuccess ||
        cudaMalloc(&B->dplist, 4 * count) != cudaSuccess ||
        cudaMalloc(&B->dqueue, 256) != cudaSuccess) {
        cudaGetLastError();
        set_error("out of device memory for the batch plan");
        return fail(LSQ_ERR_NOMEM);
    }
    size_t off = 0;
    for (int64_t i = 0; i < count; ++i) {
        hp[i].ws = B->ws + off;
        off += 5 * (size_t)hp[i].npad * kc;
    }
    std::vector<int32_t> order(count);   // largest first (ties: lower index first)
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
    if (cudaMemcpyAsync(B->dprobs, hp.data(), sizeof(BatchProb) * count, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(B->dplist, order.data(), 4 * count, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess ||
        cudaMemsetAsync(B->dout, 0, sizeof(BatchOut) * count * k, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("copying the batch table failed");
        return fail(LSQ_ERR_CUDA);
    }
    // default cluster size: the largest available power of two up to 8
    lsq_status r = LSQ_ERR_UNSUPPORTED;
    for (int C = 8; C >= 1 && r != LSQ_OK; C >>= 1) r = bt_set_cluster(B, C);
    if (r != LSQ_OK) return fail(r);
    *out = B;
    return LSQ_OK;
}

extern "C" lsq_status lsq_batch_solve(lsq_batch* b, void* stream) {
    LSQ_CHECK_ARG(b != nullptr, "null plan");
    return bt_solve(b, (cudaStream_t)stream);
}

extern "C" lsq_status lsq_batch_set_cluster(lsq_batch* b, int32_t cluster) {
    LSQ_CHECK_ARG(b != nullptr, "null plan");
    LSQ_CHECK_ARG(cluster == 1 || cluster == 2 || cluster == 4 || cluster == 8 || cluster == 16,
                  "cluster must be 1, 2, 4, 8 or 16");
    return bt_set_cluster(b, cluster);
}

extern "C" lsq_status lsq_batch_autotune(lsq_batch* b, int32_t* cluster_out, void* stream) {
    LSQ_CHECK_ARG(b != nullptr, "null plan");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    LSQ_CUDA(cudaEventCreate(&e0));
    LSQ_CUDA(cudaEventCreate(&e1));
    int best = 0;
    float best_ms = 0.f;
    lsq_status r = LSQ_OK;
    for (int C : {1, 2, 4, 8, 16}) {
        int nc = 0;
        r = bt_max_clusters(b->kc, C, &nc);
        if (r != LSQ_OK) break;
        if (nc < 1) continue;
        if ((r = bt_set_cluster(b, C)) != LSQ_OK) break;
        if ((r = bt_solve(b, st)) != LSQ_OK) break;   // warm-up, the same work as the timed run
        if (cudaEventRecord(e0, st) != cudaSuccess) { r = LSQ_ERR_CUDA; break; }
        if ((r = bt_solve(b, st)) != LSQ_OK) break;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { r = LSQ_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best == 0 || ms < best_ms) { best = C; best_ms = ms; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != LSQ_OK) return r;
    if (best == 0) { set_error("no cluster size fits"); return LSQ_ERR_UNSUPPORTED; }
    if ((r = bt_set_cluster(b, best)) != LSQ_OK) return r;
    if ((r = bt_solve(b, st)) != LSQ_OK) return r;   // leave the solutions of the chosen size
    LSQ_CUDA(cudaStreamSynchronize(st));
    if (cluster_out) *cluster_out = best;
    return LSQ_OK;
}

extern "C" lsq_status lsq_batch_info(const lsq_batch* b, lsq_info* infos, void* stream) {
    LSQ_CHECK_ARG(b != nullptr && infos != nullptr, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<BatchOut> h(b->count * b->k);
    LSQ_CUDA(cudaMemcpyAsync(h.data(), b->dout, sizeof(BatchOut) * h.size(), cudaMemcpyDeviceToHost, st));
    LSQ_CUDA(cudaStreamSynchronize(st));
    bool all = true;
    for (int64_t p = 0; p < b->count; ++p) {
        lsq_info& I = infos[p];
        for (int c = 0; c < b->k && c < I.k; ++c) {
            const BatchOut& o = h[p * b->k + c];
            if (I.iters) I.iters[c] = o.iters;
            if (I.outer) I.outer[c] = o.outer;
            if (I.converged) I.converged[c] = (uint8_t)o.conv;
            if (I.relres_rec) I.relres_rec[c] = o.rec;
            if (I.relres_true) I.relres_true[c] = o.tru;
            if (I.relres_raw) I.relres_raw[c] = o.raw;
        }
        for (int c = 0; c < b->k; ++c) all = all && h[p * b->k + c].conv;
    }
    if (!all) {
        set_error("PCG did not reach the tolerance in some problem of the batch");
        return LSQ_ERR_NOT_CONVERGED;
    }
    return LSQ_OK;
}

extern "C" void lsq_batch_destroy(lsq_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    cudaFree(b->dprobs);
    cudaFree(b->dout);
    cudaFree(b->ws);
    cudaFree(b->dplist);
    cudaFree(b->dqueue);
    delete b;
}
