// Alg. 2 step 4: PCG on the normalised normal equation Â^T Â y = Â^T b, Â = A D^{-1},
// run to completion (including restarts from the true residual) inside ONE persistent
// cooperative kernel.
//
// Work split: CTA c owns the contiguous row block [c m/G, (c+1) m/G) of A for the fused
// pass w = Â^T (Â p) (each row is read from HBM once: its dot with p̃ = D^{-1} p gives q_i,
// and the same registers are then scaled by q_i into the CTA's n-vector partial), and the
// column slice [c n/G, (c+1) n/G) for the n-vector updates and for the rows of the
// materialised SGS operator.  p is replicated in every CTA's shared memory; y, g and z are
// global and written only by their owners.  Every reduction runs in a fixed order, so the
// result is deterministic for a given grid size.  Three grid barriers per iteration:
//   B1 after the fused pass (partials of w and of ||Â p||^2 = p^T w),
//   B2 after y += alpha p, g -= alpha w (partials of ||g||^2),
//   B3 after z = P g (partials of g^T z).
#pragma once
#include "common.cuh"

namespace lsq {

enum PassMode { PASS_MATVEC = 0, PASS_RHS = 1, PASS_RESID = 2 };
// part_s slots: 0 ||Â p||^2, 1 ||g||^2, 2 g^T z, 3 final ||g||^2, 4 ||D h||^2, 5 ||D g||^2
constexpr int PART_S = 8;

struct PcgArgs {
    int64_t m, n, ld;
    const void* vals;      // inner-iteration values (dtype DT)
    const void* vals_res;  // values for h and the true residual (dtype DTR)
    const double* inv_d;   // 1 / d_j
    const void* op;        // n x n row-major SGS operator (OPT)
    const double* b;       // m (least-squares form)
    const double* h_in;    // n: right-hand side of Â^T Â y = h (normal form), or NULL
    double* x;             // n (output)
    double* y;             // n workspace
    double* g;             // n workspace
    double* z;             // n workspace
    double* part_w;        // G x n
    double* part_s;        // G x PART_S
    unsigned* bar;         // 2 words
    unsigned* err;
    double tol, inner_tol;
    int32_t maxit, max_outer;
    int32_t* out_i;        // iters, outer, converged, status
    double* out_d;         // relres_rec, relres_true, relres_raw
};

// Storage/compute traits of a value dtype for the vectorised row pass.
template <int DT> struct RowT;
template <> struct RowT<LSQ_F64> {
    typedef double C;  // compute type
    static constexpr int VEC = 2;
    static __device__ __forceinline__ void load(const void* base, int64_t e, C (&a)[VEC]) {
        double2 v = __ldg(reinterpret_cast<const double2*>(reinterpret_cast<const double*>(base) + e));
        a[0] = v.x; a[1] = v.y;
    }
};
template <> struct RowT<LSQ_F32> {
    typedef float C;
    static constexpr int VEC = 4;
    static __device__ __forceinline__ void load(const void* base, int64_t e, C (&a)[VEC]) {
        float4 v = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(base) + e));
        a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
    }
};

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c) { return fma(a, b, c); }

// Fused row pass over rows [r0, r1):
//   MATVEC: q_i = â_i . p̃      RHS: q_i = b_i      RESID: q_i = b_i - â_i . ỹ
// with p̃ / ỹ = D^{-1} (vector) already in s_v (padded with zeros to NMAX).  Each warp
// accumulates sum_i q_i a_i in registers; the CTA partial (sum over warps in order) is
// written to part_w[cta][0..n) and sum_i q_i^2 to part_s[cta][0].
template <int DT, int NMAX>
__device__ __forceinline__ void row_pass(const PcgArgs& a, const void* vals, int mode,
                                         const double* s_v, double* s_red, double* s_scal,
                                         int64_t r0, int64_t r1) {
    typedef typename RowT<DT>::C C;
    constexpr int VEC = RowT<DT>::VEC;
    constexpr int NCH = NMAX / (32 * VEC);
    static_assert(NCH >= 1, "NMAX too small for this dtype");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t n = a.n;
    C acc[NCH][VEC];
#pragma unroll
    for (int c = 0; c < NCH; ++c)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[c][v] = C(0);
    double qq = 0.0;
    for (int64_t i = r0 + wid; i < r1; i += nwarps) {
        const int64_t rowoff = i * a.ld;
        C av[NCH][VEC];
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int col = c * 32 * VEC + lane * VEC;
            if (col < n) {
                RowT<DT>::load(vals, rowoff + col, av[c]);
#pragma unroll
                for (int v = 0; v < VEC; ++v)
                    if (col + v >= n) av[c][v] = C(0);
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) av[c][v] = C(0);
            }
        }
        double q;
        if (mode == PASS_RHS) {
            q = a.b[i];
        } else {
            C dot = C(0);
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int col = c * 32 * VEC + lane * VEC;
#pragma unroll
                for (int v = 0; v < VEC; ++v) dot = fma_t(av[c][v], (C)s_v[col + v], dot);
            }
            dot = warp_sum(dot);
            q = (mode == PASS_MATVEC) ? (double)dot : a.b[i] - (double)dot;
        }
        qq = fma(q, q, qq);
        const C qc = (C)q;
#pragma unroll
        for (int c = 0; c < NCH; ++c)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[c][v] = fma_t(qc, av[c][v], acc[c][v]);
    }
    // cross-warp reduction in a fixed order
    double* mine = s_red + (int64_t)wid * NMAX;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        const int col = c * 32 * VEC + lane * VEC;
#pragma unroll
        for (int v = 0; v < VEC; ++v) mine[col + v] = (double)acc[c][v];
    }
    if (lane == 0) s_scal[wid] = qq;  // qq is identical in all lanes; keep one copy
    __syncthreads();
    double* pw = a.part_w + (int64_t)blockIdx.x * n;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        double sacc = 0.0;
        for (int w = 0; w < nwarps; ++w) sacc += s_red[(int64_t)w * NMAX + j];
        pw[j] = sacc;
    }
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nwarps; ++w) t += s_scal[w];
        a.part_s[(int64_t)blockIdx.x * PART_S + 0] = t;
    }
    __syncthreads();
}

// sum_g part_s[g][slot] over all CTAs, same order in every CTA; result broadcast.
__device__ __forceinline__ double grid_scalar(const PcgArgs& a, int slot, double* s_scal) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        double t = 0.0;
        for (int g = lane; g < (int)gridDim.x; g += 32) t += a.part_s[(int64_t)g * PART_S + slot];
        t = warp_sum(t);
        if (lane == 0) s_scal[31] = t;
    }
    __syncthreads();
    double r = s_scal[31];
    __syncthreads();
    return r;
}

// w_j = inv_d_j sum_g part_w[g][j] for the owned columns, handed (on lane 0 of the warp
// that reduced it) to `fn(j, w_j)`, which returns this column's contributions to two CTA
// partials stored in part_s[cta][slot_a] and part_s[cta][slot_b].
template <typename F>
__device__ __forceinline__ void slice_reduce(const PcgArgs& a, int64_t c0, int64_t c1, int slot_a,
                                             int slot_b, double* s_scal, F fn) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    double pa = 0.0, pb = 0.0;
    for (int64_t j = c0 + wid; j < c1; j += nwarps) {
        double t = 0.0;
        for (int g = lane; g < (int)gridDim.x; g += 32) t += a.part_w[(int64_t)g * a.n + j];
        t = warp_sum(t);
        if (lane == 0) {
            double2 r = fn(j, t * a.inv_d[j]);
            pa += r.x;
            pb += r.y;
        }
    }
    if (lane == 0) { s_scal[wid] = pa; s_scal[16 + wid] = pb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < nwarps; ++w) { ta += s_scal[w]; tb += s_scal[16 + w]; }
        a.part_s[(int64_t)blockIdx.x * PART_S + slot_a] = ta;
        a.part_s[(int64_t)blockIdx.x * PART_S + slot_b] = tb;
    }
    __syncthreads();
}

// z_j = sum_k op_jk g_k for the owned rows (g staged in s_v); partial g^T z -> slot 2.
template <typename OPT>
__device__ __forceinline__ void op_rows(const PcgArgs& a, int64_t c0, int64_t c1,
                                        const double* s_v, double* s_scal) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const OPT* op = reinterpret_cast<const OPT*>(a.op);
    double part = 0.0;
    for (int64_t j = c0 + wid; j < c1; j += nwarps) {
        const OPT* row = op + j * a.n;
        OPT t = OPT(0);
        for (int64_t k = lane; k < a.n; k += 32) t = fma(row[k], (OPT)s_v[k], t);
        double zj = (double)warp_sum(t);
        if (lane == 0) a.z[j] = zj;
        part = fma(s_v[j], zj, part);
    }
    if (lane == 0) s_scal[wid] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nwarps; ++w) t += s_scal[w];
        a.part_s[(int64_t)blockIdx.x * PART_S + 2] = t;
    }
    __syncthreads();
}

template <int DT, int DTR, int NMAX, typename OPT>
__global__ void __launch_bounds__(256, 1) k_pcg_dense(PcgArgs a) {
    extern __shared__ double smem[];
    __shared__ double s_scal[32];
    const int64_t n = a.n;
    const int nwarps = blockDim.x >> 5;
    double* s_p = smem;              // NMAX: search direction p (replicated)
    double* s_v = s_p + NMAX;        // NMAX: D^{-1} x vector for the row pass, or g
    double* s_red = s_v + NMAX;      // nwarps x NMAX
    const unsigned G = gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * a.m / G, r1 = (int64_t)(blockIdx.x + 1) * a.m / G;
    const int64_t c0 = (int64_t)blockIdx.x * n / G, c1 = (int64_t)(blockIdx.x + 1) * n / G;
    for (int64_t j = threadIdx.x; j < NMAX; j += blockDim.x) { s_p[j] = 0.0; s_v[j] = 0.0; }
    __syncthreads();

    int iters = 0, outer_used = 0, converged = 0, status = LSQ_ERR_NOT_CONVERGED;
    double rec = 1.0, tru = 1.0, gg = 0.0;
    bool dirty = false;  // iterations since the last true residual

    // h = Â^T b (values of the residual dtype) or the given h; y = 0; g = h
    if (a.h_in) {
        double ha = 0.0, hb = 0.0;
        for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
            const double h = a.h_in[j], hr = h / a.inv_d[j];
            a.g[j] = h; a.y[j] = 0.0;
            ha = fma(h, h, ha); hb = fma(hr, hr, hb);
        }
        ha = warp_sum(ha); hb = warp_sum(hb);
        if ((threadIdx.x & 31) == 0) { s_scal[threadIdx.x >> 5] = ha; s_scal[16 + (threadIdx.x >> 5)] = hb; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double ta = 0.0, tb = 0.0;
            for (int w = 0; w < nwarps; ++w) { ta += s_scal[w]; tb += s_scal[16 + w]; }
            a.part_s[(int64_t)blockIdx.x * PART_S + 1] = ta;
            a.part_s[(int64_t)blockIdx.x * PART_S + 4] = tb;
        }
        __syncthreads();
    } else {
        row_pass<DTR, NMAX>(a, a.vals_res, PASS_RHS, s_v, s_red, s_scal, r0, r1);
        if (!grid_barrier(a.bar, G, a.err)) return;
        slice_reduce(a, c0, c1, 1, 4, s_scal, [&](int64_t j, double h) {
            a.g[j] = h; a.y[j] = 0.0;
            const double hr = h / a.inv_d[j];
            return make_double2(h * h, hr * hr); });
    }
    if (!grid_barrier(a.bar, G, a.err)) return;
    gg = grid_scalar(a, 1, s_scal);
    const double hn = sqrt(gg);
    const double hn_raw = sqrt(grid_scalar(a, 4, s_scal));
    double raw = 1.0;
    if (hn == 0.0) {
        converged = 1; status = LSQ_OK; rec = 0.0; tru = 0.0;
    } else {
        raw = 1.0;
        for (int outer = 0; outer < a.max_outer; ++outer) {
            if (outer > 0) {
                // true residual g = Â^T (b - Â y)
                for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s_v[j] = a.y[j] * a.inv_d[j];
                __syncthreads();
                row_pass<DTR, NMAX>(a, a.vals_res, a.h_in ? PASS_MATVEC : PASS_RESID, s_v, s_red, s_scal, r0, r1);
                if (!grid_barrier(a.bar, G, a.err)) return;
                slice_reduce(a, c0, c1, 1, 5, s_scal, [&](int64_t j, double t) {
                    if (a.h_in) t = a.h_in[j] - t;
                    a.g[j] = t;
                    const double tr = t / a.inv_d[j];
                    return make_double2(t * t, tr * tr); });
                if (!grid_barrier(a.bar, G, a.err)) return;
                gg = grid_scalar(a, 1, s_scal);
                raw = sqrt(grid_scalar(a, 5, s_scal)) / hn_raw;
                dirty = false;
            }
            tru = sqrt(gg) / hn;
            if (outer == 0) rec = tru;
            if (tru <= a.tol) { converged = 1; status = LSQ_OK; break; }
            if (iters >= a.maxit) break;
            outer_used = outer + 1;
            const double gstart = sqrt(gg);
            // z = P g, rho = g^T z, p = z
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s_v[j] = a.g[j];
            __syncthreads();
            op_rows<OPT>(a, c0, c1, s_v, s_scal);
            if (!grid_barrier(a.bar, G, a.err)) return;
            double rho = grid_scalar(a, 2, s_scal);
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s_p[j] = a.z[j];
            __syncthreads();
            bool broke = false;
            while (true) {
                // fused pass: w = Â^T (Â p)
                for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s_v[j] = s_p[j] * a.inv_d[j];
                __syncthreads();
                row_pass<DT, NMAX>(a, a.vals, PASS_MATVEC, s_v, s_red, s_scal, r0, r1);
                if (!grid_barrier(a.bar, G, a.err)) return;
                const double pw = grid_scalar(a, 0, s_scal);
                if (!(pw > 0.0) || !(rho > 0.0) || !isfinite(pw) || !isfinite(rho)) {
                    status = LSQ_ERR_BREAKDOWN; broke = true; break;
                }
                const double alpha = rho / pw;
                slice_reduce(a, c0, c1, 1, 6, s_scal, [&](int64_t j, double w) {
                    a.y[j] = fma(alpha, s_p[j], a.y[j]);
                    double gj = fma(-alpha, w, a.g[j]);
                    a.g[j] = gj;
                    return make_double2(gj * gj, 0.0); });
                if (!grid_barrier(a.bar, G, a.err)) return;
                ++iters;
                dirty = true;
                gg = grid_scalar(a, 1, s_scal);
                rec = sqrt(gg) / hn;
                if (rec <= a.tol || sqrt(gg) <= a.inner_tol * gstart) break;
                if (iters >= a.maxit) break;
                for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s_v[j] = a.g[j];
                __syncthreads();
                op_rows<OPT>(a, c0, c1, s_v, s_scal);
                if (!grid_barrier(a.bar, G, a.err)) return;
                const double rho_new = grid_scalar(a, 2, s_scal);
                const double beta = rho_new / rho;
                rho = rho_new;
                for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s_p[j] = fma(beta, s_p[j], a.z[j]);
                __syncthreads();
            }
            if (broke) break;
        }
        if (!converged && status != LSQ_ERR_BREAKDOWN && dirty) {
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s_v[j] = a.y[j] * a.inv_d[j];
            __syncthreads();
            row_pass<DTR, NMAX>(a, a.vals_res, a.h_in ? PASS_MATVEC : PASS_RESID, s_v, s_red, s_scal, r0, r1);
            if (!grid_barrier(a.bar, G, a.err)) return;
            slice_reduce(a, c0, c1, 3, 5, s_scal, [&](int64_t j, double t) {
                if (a.h_in) t = a.h_in[j] - t;
                a.g[j] = t;
                const double tr = t / a.inv_d[j];
                return make_double2(t * t, tr * tr); });
            if (!grid_barrier(a.bar, G, a.err)) return;
            tru = sqrt(grid_scalar(a, 3, s_scal)) / hn;
            raw = sqrt(grid_scalar(a, 5, s_scal)) / hn_raw;
            if (tru <= a.tol) { converged = 1; status = LSQ_OK; }
        }
    }
    for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) a.x[j] = a.y[j] * a.inv_d[j];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.out_i[0] = iters; a.out_i[1] = outer_used; a.out_i[2] = converged; a.out_i[3] = status;
        a.out_d[0] = rec; a.out_d[1] = tru; a.out_d[2] = (hn == 0.0) ? 0.0 : raw;
    }
}

// Host launcher (defined per dtype in pcg_f64.cu / pcg_f32.cu)
lsq_status launch_pcg_dense(int dt, int dtr, int opt_dtype, int64_t nmax, PcgArgs& args,
                            int grid_cap, cudaStream_t st, int* grid_used);

}  // namespace lsq
