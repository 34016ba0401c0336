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
#include "tma.cuh"
#include "dfloat.cuh"

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
    unsigned long long* bar;  // grid barrier count (zeroed before the launch)
    unsigned* err;
    double tol, inner_tol;
    int32_t maxit, max_outer;
    int32_t* out_i;        // iters, outer, converged, status
    double* out_d;         // relres_rec, relres_true, relres_raw
    unsigned max_polls = 1u << 26;   // bound of every grid-barrier wait
};

__device__ __forceinline__ int64_t imin64(int64_t x, int64_t y) { return x < y ? x : y; }

// Two-row warp reduction (pair_reduce2 below): lanes 0-15 end with sum(a), lanes 16-31
// with sum(b) (one exchange splits the rows, four butterfly steps finish each half), then
// both sums are broadcast.
__device__ __forceinline__ double shfl_d(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float shfl_f(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ f2 shfl_f2(f2 v, int o) { return df_shfl_xor(v, o); }
__device__ __forceinline__ double bcast_d(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ float bcast_f(float v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ f2 bcast_f2(f2 v, int l) {
    return f2{__shfl_sync(0xffffffffu, v.hi, l), __shfl_sync(0xffffffffu, v.lo, l)};
}
template <typename T, typename Add>
__device__ __forceinline__ void pair_reduce2(T& a, T& b, int lane, Add add, T (*xo)(T, int), T (*bc)(T, int)) {
    T send = (lane < 16) ? b : a;
    T mine = (lane < 16) ? a : b;
    add(mine, xo(send, 16));
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) add(mine, xo(mine, o));
    a = bc(mine, 0);
    b = bc(mine, 16);
}

// Per-dtype arithmetic of the fused row pass.  A lane owns VEC consecutive elements of
// each 32*VEC-wide chunk of a row (16-byte shared-memory reads); NCH chunks cover NMAX.
// A warp handles one row, or two rows at once (TWO) whose dot products share one warp
// reduction.  Elements beyond n (row padding) are masked to zero.
//   LSQ_F64   : FP64 products and sums.
//   LSQ_F32   : FP32 products, FP32 row dots and column accumulators; sum of q_i^2 in
//               double-float (no FP64 instruction per row).
//   LSQ_F32X2 : values stored as float pairs (hi, lo); products and sums in double-float
//               (about 48 bits) on the FP32 units.
template <int DT, int NMAX> struct RowOps;

template <int NMAX> struct RowOps<LSQ_F64, NMAX> {
    static constexpr int ES = 8, VEC = 2, NCH = NMAX / (32 * VEC);
    typedef double VT;   // staged vector element
    typedef double RT;   // cross-warp reduction element
    struct Acc { double v[NCH][VEC]; };
    struct Q { double s; };
    static __device__ __forceinline__ void zero(Acc& a, Q& q) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) { a.v[c][0] = 0.0; a.v[c][1] = 0.0; }
        q.s = 0.0;
    }
    static __device__ __forceinline__ VT stage(double x) { return x; }
    template <int MODE, bool TWO>
    static __device__ __forceinline__ void row(const char* rp0, const char* rp1, bool has1,
                                               const VT* sv, int lane, int64_t n, double b0,
                                               double b1, Acc& A, Q& Qa) {
        const double* r0 = reinterpret_cast<const double*>(rp0);
        const double* r1 = reinterpret_cast<const double*>(rp1);
        double q0, q1 = 0.0;
        if (MODE == PASS_RHS) {
            q0 = b0; q1 = b1;
        } else {
            double d0[4] = {0.0, 0.0, 0.0, 0.0}, d1[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int col = c * 32 * VEC + lane * VEC;
                if (col < n) {
                    const double2 sx = *reinterpret_cast<const double2*>(sv + col);
                    const bool in1 = col + 1 < n;
                    double2 v = *reinterpret_cast<const double2*>(r0 + col);
                    d0[(2 * c) & 3] = fma(v.x, sx.x, d0[(2 * c) & 3]);
                    d0[(2 * c + 1) & 3] = fma(in1 ? v.y : 0.0, sx.y, d0[(2 * c + 1) & 3]);
                    if (TWO) {
                        double2 w = *reinterpret_cast<const double2*>(r1 + col);
                        d1[(2 * c) & 3] = fma(w.x, sx.x, d1[(2 * c) & 3]);
                        d1[(2 * c + 1) & 3] = fma(in1 ? w.y : 0.0, sx.y, d1[(2 * c + 1) & 3]);
                    }
                }
            }
            double d0s = (d0[0] + d0[1]) + (d0[2] + d0[3]), d1s = (d1[0] + d1[1]) + (d1[2] + d1[3]);
            if (TWO) pair_reduce2<double>(d0s, d1s, lane, [](double& x, double y) { x += y; }, shfl_d, bcast_d);
            else d0s = warp_sum(d0s);
            q0 = (MODE == PASS_MATVEC) ? d0s : b0 - d0s;
            q1 = (MODE == PASS_MATVEC) ? d1s : b1 - d1s;
        }
        if (!has1) q1 = 0.0;
        if (lane == 0) { Qa.s = fma(q0, q0, Qa.s); if (TWO) Qa.s = fma(q1, q1, Qa.s); }
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int col = c * 32 * VEC + lane * VEC;
            if (col < n) {
                const bool in1 = col + 1 < n;
                double2 v = *reinterpret_cast<const double2*>(r0 + col);
                A.v[c][0] = fma(q0, v.x, A.v[c][0]);
                A.v[c][1] = fma(q0, in1 ? v.y : 0.0, A.v[c][1]);
                if (TWO) {
                    double2 w = *reinterpret_cast<const double2*>(r1 + col);
                    A.v[c][0] = fma(q1, w.x, A.v[c][0]);
                    A.v[c][1] = fma(q1, in1 ? w.y : 0.0, A.v[c][1]);
                }
            }
        }
    }
    static __device__ __forceinline__ void store(const Acc& A, RT* dst, int lane) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int col = c * 32 * VEC + lane * VEC;
            *reinterpret_cast<double2*>(dst + col) = make_double2(A.v[c][0], A.v[c][1]);
        }
    }
    static __device__ __forceinline__ void red_add(RT& acc, RT v) { acc += v; }
    static __device__ __forceinline__ RT red_zero() { return 0.0; }
    static __device__ __forceinline__ double red_out(RT v) { return v; }
    static __device__ __forceinline__ double q_out(const Q& q) { return q.s; }
};

template <int NMAX> struct RowOps<LSQ_F32, NMAX> {
    static constexpr int ES = 4, VEC = 4, NCH = NMAX / (32 * VEC);
    typedef float VT;
    typedef float RT;
    struct Acc { float v[NCH][VEC]; };
    struct Q { f2 s; };
    static __device__ __forceinline__ void zero(Acc& a, Q& q) {
#pragma unroll
        for (int c = 0; c < NCH; ++c)
#pragma unroll
            for (int v = 0; v < VEC; ++v) a.v[c][v] = 0.f;
        q.s = f2{0.f, 0.f};
    }
    static __device__ __forceinline__ VT stage(double x) { return (float)x; }
    static __device__ __forceinline__ float4 masked(float4 v, int col, int64_t n) {
        if (col + 4 <= n) return v;
        return make_float4(v.x, col + 1 < n ? v.y : 0.f, col + 2 < n ? v.z : 0.f, col + 3 < n ? v.w : 0.f);
    }
    template <int MODE, bool TWO>
    static __device__ __forceinline__ void row(const char* rp0, const char* rp1, bool has1,
                                               const VT* sv, int lane, int64_t n, double b0,
                                               double b1, Acc& A, Q& Qa) {
        const float* r0 = reinterpret_cast<const float*>(rp0);
        const float* r1 = reinterpret_cast<const float*>(rp1);
        float q0, q1 = 0.f;
        if (MODE == PASS_RHS) {
            q0 = (float)b0; q1 = (float)b1;
        } else {
            float4 d0 = make_float4(0.f, 0.f, 0.f, 0.f), d1 = d0;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int col = c * 32 * VEC + lane * VEC;
                if (col < n) {
                    const float4 sx = *reinterpret_cast<const float4*>(sv + col);
                    const float4 v = masked(*reinterpret_cast<const float4*>(r0 + col), col, n);
                    d0.x = fmaf(v.x, sx.x, d0.x); d0.y = fmaf(v.y, sx.y, d0.y);
                    d0.z = fmaf(v.z, sx.z, d0.z); d0.w = fmaf(v.w, sx.w, d0.w);
                    if (TWO) {
                        const float4 w = masked(*reinterpret_cast<const float4*>(r1 + col), col, n);
                        d1.x = fmaf(w.x, sx.x, d1.x); d1.y = fmaf(w.y, sx.y, d1.y);
                        d1.z = fmaf(w.z, sx.z, d1.z); d1.w = fmaf(w.w, sx.w, d1.w);
                    }
                }
            }
            float d0s = (d0.x + d0.y) + (d0.z + d0.w), d1s = (d1.x + d1.y) + (d1.z + d1.w);
            if (TWO) pair_reduce2<float>(d0s, d1s, lane, [](float& x, float y) { x += y; }, shfl_f, bcast_f);
            else d0s = warp_sum(d0s);
            if (MODE == PASS_MATVEC) { q0 = d0s; q1 = d1s; }
            else { q0 = (float)(b0 - (double)d0s); q1 = (float)(b1 - (double)d1s); }
        }
        if (!has1) q1 = 0.f;
        df_add_sq(Qa.s, q0);
        if (TWO) df_add_sq(Qa.s, q1);
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int col = c * 32 * VEC + lane * VEC;
            if (col < n) {
                const float4 v = masked(*reinterpret_cast<const float4*>(r0 + col), col, n);
                A.v[c][0] = fmaf(q0, v.x, A.v[c][0]); A.v[c][1] = fmaf(q0, v.y, A.v[c][1]);
                A.v[c][2] = fmaf(q0, v.z, A.v[c][2]); A.v[c][3] = fmaf(q0, v.w, A.v[c][3]);
                if (TWO) {
                    const float4 w = masked(*reinterpret_cast<const float4*>(r1 + col), col, n);
                    A.v[c][0] = fmaf(q1, w.x, A.v[c][0]); A.v[c][1] = fmaf(q1, w.y, A.v[c][1]);
                    A.v[c][2] = fmaf(q1, w.z, A.v[c][2]); A.v[c][3] = fmaf(q1, w.w, A.v[c][3]);
                }
            }
        }
    }
    static __device__ __forceinline__ void store(const Acc& A, RT* dst, int lane) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int col = c * 32 * VEC + lane * VEC;
            *reinterpret_cast<float4*>(dst + col) = make_float4(A.v[c][0], A.v[c][1], A.v[c][2], A.v[c][3]);
        }
    }
    static __device__ __forceinline__ void red_add(RT& acc, RT v) { acc += v; }
    static __device__ __forceinline__ RT red_zero() { return 0.f; }
    static __device__ __forceinline__ double red_out(RT v) { return (double)v; }
    static __device__ __forceinline__ double q_out(const Q& q) { return df_to_double(q.s); }
};

// BF16 values: a lane reads 8 values (16 bytes) per chunk and widens them exactly to FP32;
// products and sums as in the FP32 form (FP32 row dots and column accumulators, sum of
// q_i^2 in double-float).  The stored matrix is half the bytes of FP32.
__device__ __forceinline__ void bf16x8_to_f32(uint4 u, float (&f)[8]) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        f[2 * i] = __uint_as_float(w[i] << 16);            // element 2i (low half)
        f[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u); // element 2i + 1 (high half)
    }
}
template <int NMAX> struct RowOps<LSQ_BF16, NMAX> {
    static constexpr int ES = 2, VEC = 8, NCH = (NMAX + 32 * 8 - 1) / (32 * 8);
    typedef float VT;
    typedef float RT;
    struct Acc { float v[NCH][VEC]; };
    struct Q { f2 s; };
    static __device__ __forceinline__ void zero(Acc& a, Q& q) {
#pragma unroll
        for (int c = 0; c < NCH; ++c)
#pragma unroll
            for (int v = 0; v < VEC; ++v) a.v[c][v] = 0.f;
        q.s = f2{0.f, 0.f};
    }
    static __device__ __forceinline__ VT stage(double x) { return (float)x; }
    // the 8 values of chunk c of a row, zero beyond n (row padding)
    static __device__ __forceinline__ void load8(const char* rp, int col, int64_t n, float (&f)[8]) {
        bf16x8_to_f32(*reinterpret_cast<const uint4*>(rp + 2 * col), f);
        if (col + 8 > n) {
#pragma unroll
            for (int i = 0; i < 8; ++i) if (col + i >= n) f[i] = 0.f;
        }
    }
    template <int MODE, bool TWO>
    static __device__ __forceinline__ void row(const char* rp0, const char* rp1, bool has1,
                                               const VT* sv, int lane, int64_t n, double b0,
                                               double b1, Acc& A, Q& Qa) {
        float q0, q1 = 0.f;
        if (MODE == PASS_RHS) {
            q0 = (float)b0; q1 = (float)b1;
        } else {
            float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int col = c * 32 * VEC + lane * VEC;
                if (col < n) {
                    const float4 s0 = *reinterpret_cast<const float4*>(sv + col);
                    const float4 s1 = *reinterpret_cast<const float4*>(sv + col + 4);
                    const float sx[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
                    float v[8];
                    load8(rp0, col, n, v);
#pragma unroll
                    for (int i = 0; i < 8; ++i) d0[i & 3] = fmaf(v[i], sx[i], d0[i & 3]);
                    if (TWO) {
                        float w[8];
                        load8(rp1, col, n, w);
#pragma unroll
                        for (int i = 0; i < 8; ++i) d1[i & 3] = fmaf(w[i], sx[i], d1[i & 3]);
                    }
                }
            }
            float d0s = (d0[0] + d0[1]) + (d0[2] + d0[3]), d1s = (d1[0] + d1[1]) + (d1[2] + d1[3]);
            if (TWO) pair_reduce2<float>(d0s, d1s, lane, [](float& x, float y) { x += y; }, shfl_f, bcast_f);
            else d0s = warp_sum(d0s);
            if (MODE == PASS_MATVEC) { q0 = d0s; q1 = d1s; }
            else { q0 = (float)(b0 - (double)d0s); q1 = (float)(b1 - (double)d1s); }
        }
        if (!has1) q1 = 0.f;
        df_add_sq(Qa.s, q0);
        if (TWO) df_add_sq(Qa.s, q1);
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int col = c * 32 * VEC + lane * VEC;
            if (col < n) {
                float v[8];
                load8(rp0, col, n, v);
#pragma unroll
                for (int i = 0; i < 8; ++i) A.v[c][i] = fmaf(q0, v[i], A.v[c][i]);
                if (TWO) {
                    float w[8];
                    load8(rp1, col, n, w);
#pragma unroll
                    for (int i = 0; i < 8; ++i) A.v[c][i] = fmaf(q1, w[i], A.v[c][i]);
                }
            }
        }
    }
    static __device__ __forceinline__ void store(const Acc& A, RT* dst, int lane) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int col = c * 32 * VEC + lane * VEC;
            if (col < NMAX) {
                *reinterpret_cast<float4*>(dst + col) = make_float4(A.v[c][0], A.v[c][1], A.v[c][2], A.v[c][3]);
                *reinterpret_cast<float4*>(dst + col + 4) = make_float4(A.v[c][4], A.v[c][5], A.v[c][6], A.v[c][7]);
            }
        }
    }
    static __device__ __forceinline__ void red_add(RT& acc, RT v) { acc += v; }
    static __device__ __forceinline__ RT red_zero() { return 0.f; }
    static __device__ __forceinline__ double red_out(RT v) { return (double)v; }
    static __device__ __forceinline__ double q_out(const Q& q) { return df_to_double(q.s); }
};

template <int NMAX> struct RowOps<LSQ_F32X2, NMAX> {
    static constexpr int ES = 8, VEC = 2, NCH = NMAX / (32 * VEC);
    typedef f2 VT;
    typedef f2 RT;
    struct Acc { f2 v[NCH][VEC]; };
    struct Q { f2 s; };
    static __device__ __forceinline__ void zero(Acc& a, Q& q) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) { a.v[c][0] = f2{0.f, 0.f}; a.v[c][1] = f2{0.f, 0.f}; }
        q.s = f2{0.f, 0.f};
    }
    static __device__ __forceinline__ VT stage(double x) { return df_from_double(x); }
    template <int MODE, bool TWO>
    static __device__ __forceinline__ void row(const char* rp0, const char* rp1, bool has1,
                                               const VT* sv, int lane, int64_t n, double b0,
                                               double b1, Acc& A, Q& Qa) {
        const float* r0 = reinterpret_cast<const float*>(rp0);
        const float* r1 = reinterpret_cast<const float*>(rp1);
        f2 q0, q1{0.f, 0.f};
        if (MODE == PASS_RHS) {
            q0 = df_from_double(b0); q1 = df_from_double(b1);
        } else {
            f2 d0[4], d1[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) { d0[k] = f2{0.f, 0.f}; d1[k] = f2{0.f, 0.f}; }
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                const int col = c * 32 * VEC + lane * VEC;
                if (col < n) {
                    const float4 sx = *reinterpret_cast<const float4*>(sv + col);   // two pairs
                    const bool in1 = col + 1 < n;
                    const float4 v = *reinterpret_cast<const float4*>(r0 + 2 * col);  // hi0 lo0 hi1 lo1
                    df_fma_cascade(d0[(2 * c) & 3], f2{v.x, v.y}, f2{sx.x, sx.y});
                    if (in1) df_fma_cascade(d0[(2 * c + 1) & 3], f2{v.z, v.w}, f2{sx.z, sx.w});
                    if (TWO) {
                        const float4 w = *reinterpret_cast<const float4*>(r1 + 2 * col);
                        df_fma_cascade(d1[(2 * c) & 3], f2{w.x, w.y}, f2{sx.x, sx.y});
                        if (in1) df_fma_cascade(d1[(2 * c + 1) & 3], f2{w.z, w.w}, f2{sx.z, sx.w});
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) { d0[k] = df_norm(d0[k]); d1[k] = df_norm(d1[k]); }
            df_add(d0[0], d0[1]); df_add(d0[2], d0[3]); df_add(d0[0], d0[2]);
            df_add(d1[0], d1[1]); df_add(d1[2], d1[3]); df_add(d1[0], d1[2]);
            f2 d0a = d0[0], d1a = d1[0];
            if (TWO) pair_reduce2<f2>(d0a, d1a, lane, [](f2& x, f2 y) { df_add(x, y); }, shfl_f2, bcast_f2);
            else d0a = df_warp_sum(d0a);
            if (MODE == PASS_MATVEC) { q0 = d0a; q1 = d1a; }
            else { q0 = df_from_double(b0 - df_to_double(d0a)); q1 = df_from_double(b1 - df_to_double(d1a)); }
        }
        if (!has1) q1 = f2{0.f, 0.f};
        df_fma(Qa.s, q0, q0);
        if (TWO) df_fma(Qa.s, q1, q1);
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int col = c * 32 * VEC + lane * VEC;
            if (col < n) {
                const bool in1 = col + 1 < n;
                const float4 v = *reinterpret_cast<const float4*>(r0 + 2 * col);
                df_fma_cascade(A.v[c][0], q0, f2{v.x, v.y});
                if (in1) df_fma_cascade(A.v[c][1], q0, f2{v.z, v.w});
                if (TWO) {
                    const float4 w = *reinterpret_cast<const float4*>(r1 + 2 * col);
                    df_fma_cascade(A.v[c][0], q1, f2{w.x, w.y});
                    if (in1) df_fma_cascade(A.v[c][1], q1, f2{w.z, w.w});
                }
            }
        }
    }
    static __device__ __forceinline__ void store(const Acc& A, RT* dst, int lane) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const int col = c * 32 * VEC + lane * VEC;
            const f2 a0 = df_norm(A.v[c][0]), a1 = df_norm(A.v[c][1]);
            *reinterpret_cast<float4*>(dst + col) = make_float4(a0.hi, a0.lo, a1.hi, a1.lo);
        }
    }
    static __device__ __forceinline__ void red_add(RT& acc, RT v) { df_add(acc, v); }
    static __device__ __forceinline__ RT red_zero() { return f2{0.f, 0.f}; }
    static __device__ __forceinline__ double red_out(RT v) { return df_to_double(v); }
    static __device__ __forceinline__ double q_out(const Q& q) { return df_to_double(q.s); }
};

// Shared-memory staging ring for the rows of A; one mbarrier per slot.  The rest of the
// 208 KiB budget holds four n-vectors (p, the staged vector in FP64 and in the compute
// type, and 1/d).
constexpr int RING_SLOTS = 8;
constexpr int PCG_VEC_ARRAYS = 4;  // s_p, s_v, s_vc, s_invd (NMAX doubles each)
__host__ __device__ constexpr int ring_bytes(int nmax) {
    return ((208 * 1024 - PCG_VEC_ARRAYS * nmax * 8) / (16 * 1024)) * 16 * 1024;
}
// Dynamic shared memory of k_pcg_dense: the ring followed by the n-vectors.  The kernel's
// layout and the launcher both use this one definition.
__host__ __device__ constexpr size_t pcg_smem_bytes(int nmax) {
    return (size_t)ring_bytes(nmax) + (size_t)PCG_VEC_ARRAYS * nmax * sizeof(double);
}
struct Ring {
    char* buf;
    uint64_t* bars;
    uint32_t phase;       // bit s: parity of the next wait on slot s (same in every thread)
    int bytes;
    const char* pre_src;  // stages already in flight for a pass starting at pre_src
    uint32_t pre_stage;
    int pre_count;
    // split pass (row_pass_split): "q of this stage is ready" and "slot is free" barriers,
    // with their parity bits, and the per-stage q values (RING_SLOTS x 16 double-floats)
    uint64_t* qbars;
    uint64_t* ebars;
    uint32_t qphase, ephase;
    f2* s_q;
    uint64_t pol;         // L2 policy of the streamed rows (evict first)
};
// Stage geometry of a pass: rows per warp (2 when four stages of 2 rows per warp fit),
// rows per stage R, slots in the ring (>= 3 unless a row is very long).
struct Geo {
    int rpw, R, slots;
    uint32_t row_bytes, stage_bytes;
};
__device__ __forceinline__ Geo geometry(int64_t ld, int es, int nwarps, int rbytes) {
    Geo g;
    g.row_bytes = (uint32_t)(ld * es);
    if ((int64_t)4 * 2 * nwarps * g.row_bytes <= rbytes) {
        g.rpw = 2;
        g.R = 2 * nwarps;
    } else {
        g.rpw = 1;
        g.R = (int)(rbytes / (3 * (int64_t)g.row_bytes));
        if (g.R > nwarps) g.R = nwarps;
        if (g.R < 1) g.R = 1;
    }
    g.stage_bytes = (uint32_t)g.R * g.row_bytes;
    g.slots = rbytes / (int)g.stage_bytes;
    if (g.slots > RING_SLOTS) g.slots = RING_SLOTS;
    if (g.slots < 1) g.slots = 1;
    return g;
}
// thread 0: start the bulk copy of `bytes` at src into slot `slot`
__device__ __forceinline__ void ring_issue(Ring& ring, int slot, const Geo& g, const char* src, uint32_t bytes) {
    mbar_expect_tx(&ring.bars[slot], bytes);
    bulk_g2s_hint(ring.buf + slot * g.stage_bytes, src, bytes, &ring.bars[slot], ring.pol);
}
// all threads: wait for slot `slot`, flip its phase bit
__device__ __forceinline__ bool ring_wait(Ring& ring, int slot) {
    const bool ok = mbar_wait(&ring.bars[slot], (ring.phase >> slot) & 1u);
    ring.phase ^= (1u << slot);
    return ok;
}
// all threads: consume stages issued ahead that no pass will use, so the ring is idle
__device__ __forceinline__ void ring_drain(Ring& ring) {
    for (int i = 0; i < ring.pre_count; ++i) ring_wait(ring, i);
    ring.pre_count = 0;
    __syncthreads();
}
// all threads (uniform arguments): issue the first stages of a pass over `nrows` rows
// starting at src, ahead of time.  The ring must be idle.
__device__ __forceinline__ void ring_prefetch(Ring& ring, const char* src, const Geo& g, int64_t nrows) {
    const int nst = (int)((nrows + g.R - 1) / g.R);
    const int cnt = nst < g.slots ? nst : g.slots;
    if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        for (int i = 0; i < cnt; ++i)
            ring_issue(ring, i, g, src + (int64_t)i * g.stage_bytes,
                       (uint32_t)imin64(g.R, nrows - (int64_t)i * g.R) * g.row_bytes);
    }
    ring.pre_src = src;
    ring.pre_stage = g.stage_bytes;
    ring.pre_count = cnt;
}

// Fused row pass over the CTA's rows [r0, r1), streamed HBM -> shared memory with 1D bulk
// copies (the row block is one contiguous byte range):
//   MATVEC: q_i = â_i . p̃      RHS: q_i = b_i      RESID: q_i = b_i - â_i . ỹ
// with p̃ / ỹ = D^{-1} (vector) in s_v (zero beyond n).  Each warp accumulates
// sum_i q_i a_i in registers; the CTA partial (warps summed in order) goes to
// part_w[cta][0..n) and sum_i q_i^2 to part_s[cta][0].  Stages already in flight for this
// pass (ring_prefetch) are used; stages in flight for another pass are drained first.
// Returns false if a stage never arrived (bounded wait; the error word is set).
template <int DT, int NMAX, int MODE, int RPW>
__device__ __forceinline__ bool row_pass_rpw(const PcgArgs& a, const void* vals, const double* s_v,
                                             void* s_vc_raw, double* s_scal, int64_t r0, int64_t r1,
                                             Ring& ring, const Geo g) {
    typedef RowOps<DT, NMAX> Ops;
    typedef typename Ops::VT VT;
    typedef typename Ops::RT RT;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t n = a.n;
    VT* s_vc = reinterpret_cast<VT*>(s_vc_raw);
    for (int j = threadIdx.x; j < NMAX; j += blockDim.x) s_vc[j] = Ops::stage(s_v[j]);
    const int nrows = (int)(r1 - r0);
    const int nst = (nrows + g.R - 1) / g.R;
    const char* src = reinterpret_cast<const char*>(vals) + r0 * (int64_t)g.row_bytes;
    int have = 0;
    if (ring.pre_count > 0) {
        if (ring.pre_src == src && ring.pre_stage == g.stage_bytes) have = ring.pre_count;
        else ring_drain(ring);
    }
    ring.pre_count = 0;
    __syncthreads();   // s_vc ready; previous users of the ring are done
    if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        for (int i = have; i < nst && i < g.slots; ++i)
            ring_issue(ring, i, g, src + (int64_t)i * g.stage_bytes,
                       (uint32_t)min(g.R, nrows - i * g.R) * g.row_bytes);
    }
    typename Ops::Acc acc;
    typename Ops::Q qacc;
    Ops::zero(acc, qacc);
    bool ok = true;
    int slot = 0;
    for (int i = 0; i < nst; ++i) {
        if (!ring_wait(ring, slot)) ok = false;
        const int rows_here = min(g.R, nrows - i * g.R);
        const int lr = wid * RPW;    // first local row of this warp
        if (ok && lr < rows_here) {
            const char* base = ring.buf + slot * g.stage_bytes;
            const int64_t gi = r0 + (int64_t)i * g.R + lr;
            const bool has1 = (RPW == 2) && (lr + 1 < rows_here);
            const double b0 = (MODE == PASS_MATVEC) ? 0.0 : a.b[gi];
            const double b1 = (MODE == PASS_MATVEC || !has1) ? 0.0 : a.b[gi + 1];
            const char* rp0 = base + lr * g.row_bytes;
            const char* rp1 = has1 ? rp0 + g.row_bytes : rp0;
            Ops::template row<MODE, RPW == 2>(rp0, rp1, has1, s_vc, lane, n, b0, b1, acc, qacc);
        }
        __syncthreads();   // every warp is done with this slot
        if (threadIdx.x == 0 && i + g.slots < nst) {
            fence_proxy_async_smem();
            const int k = i + g.slots;
            ring_issue(ring, slot, g, src + (int64_t)k * g.stage_bytes,
                       (uint32_t)min(g.R, nrows - k * g.R) * g.row_bytes);
        }
        slot = (slot + 1 == g.slots) ? 0 : slot + 1;
    }
    if (!ok && threadIdx.x == 0) raise_grid_error(a.err, a.bar, DEV_ERR_TIMEOUT);
    // cross-warp reduction in a fixed order (the drained ring holds the per-warp vectors)
    RT* s_red = reinterpret_cast<RT*>(ring.buf);
    Ops::store(acc, s_red + (int64_t)wid * NMAX, lane);
    if (lane == 0) s_scal[wid] = Ops::q_out(qacc);
    __syncthreads();
    double* pw = a.part_w + (int64_t)blockIdx.x * n;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        RT sacc = Ops::red_zero();
        for (int w = 0; w < nwarps; ++w) Ops::red_add(sacc, s_red[(int64_t)w * NMAX + j]);
        pw[j] = Ops::red_out(sacc);
    }
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nwarps; ++w) t += s_scal[w];
        a.part_s[(int64_t)blockIdx.x * PART_S + 0] = t;
    }
    __syncthreads();
    return ok;
}

// The fused pass w = Â^T (Â p) for double-float values with the warps split by role, for
// stages of 16 rows (NMAX = 256 or 512, 16 warps):
//   warps 0-7  ("dot" warps) take two rows of each stage, compute q_i = â_i . p̃ for both in
//              double-float, reduce the two sums together, put q_i in s_q and arrive on the
//              stage's q barrier;
//   warps 8-15 ("axpy" warps) wait for q, and lane l of axpy warp v accumulates the columns
//              j = v NMAX/8 + l CPL + {0..CPL-1} of w over all 16 rows of the stage
//              (CPL = NMAX/256 columns per lane); they then arrive on the stage's empty
//              barrier, and lane 0 of warp 8 refills the slot with a later stage.
// No block-wide barrier inside the pass: each role waits only for the data it needs.  A
// column of w is owned by one lane for the whole pass, so its partial needs no cross-warp
// reduction; the sum of q_i^2 is reduced over the dot warps in a fixed order.  Every wait is
// bounded (a wait that gives up sets the error word; the roles still arrive so that the
// others' waits end).
template <int NMAX, bool FULL>
__device__ __forceinline__ bool row_pass_split(const PcgArgs& a, const void* vals, const double* s_v,
                                               void* s_vc_raw, double* s_scal, int64_t r0, int64_t r1,
                                               Ring& ring, const Geo g) {
    constexpr int CPL = NMAX / 256;           // columns per axpy lane
    constexpr int NCH = NMAX / 64;            // 64-column chunks of a row (two per lane)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t n = a.n;
    f2* s_vc = reinterpret_cast<f2*>(s_vc_raw);
    for (int j = threadIdx.x; j < NMAX; j += blockDim.x) s_vc[j] = df_from_double(s_v[j]);
    const int nrows = (int)(r1 - r0);
    const int nst = (nrows + 15) / 16;
    const char* src = reinterpret_cast<const char*>(vals) + r0 * (int64_t)g.row_bytes;
    int have = 0;
    if (ring.pre_count > 0) {
        if (ring.pre_src == src && ring.pre_stage == g.stage_bytes) have = ring.pre_count;
        else ring_drain(ring);
    }
    ring.pre_count = 0;
    __syncthreads();   // s_vc ready; previous users of the ring are done
    if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        for (int i = have; i < nst && i < g.slots; ++i)
            ring_issue(ring, i, g, src + (int64_t)i * g.stage_bytes,
                       (uint32_t)min(16, nrows - i * 16) * g.row_bytes);
    }
    bool ok = true;
    if (wid < 8) {
        // ---- dot warps: rows 2 wid and 2 wid + 1 of every stage
        f2 qs{0.f, 0.f};
        int slot = 0;
        for (int i = 0; i < nst; ++i) {
            if (ok && !mbar_wait(&ring.bars[slot], (ring.phase >> slot) & 1u)) ok = false;
            ok = __all_sync(0xffffffffu, ok);   // the shuffles below need the whole warp
            const int rows_here = min(16, nrows - i * 16);
            const int lr = 2 * wid;
            f2 q0{0.f, 0.f}, q1{0.f, 0.f};
            if (ok && lr < rows_here) {
                const bool has1 = lr + 1 < rows_here;
                const float* p0 = reinterpret_cast<const float*>(ring.buf + slot * g.stage_bytes + lr * g.row_bytes);
                const float* p1 = has1 ? p0 + g.row_bytes / 4 : p0;
                f2 d0[4], d1[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) { d0[k] = f2{0.f, 0.f}; d1[k] = f2{0.f, 0.f}; }
#pragma unroll
                for (int c = 0; c < NCH; ++c) {
                    const int col = c * 64 + lane * 2;
                    float4 sx = *reinterpret_cast<const float4*>(s_vc + col);   // p̃ (hi, lo) x 2
                    float4 v = *reinterpret_cast<const float4*>(p0 + 2 * col);   // row 0, 2 values
                    float4 w = *reinterpret_cast<const float4*>(p1 + 2 * col);   // row 1
                    if (!FULL) {
                        // columns beyond n (row padding) never enter the sums
                        if (col >= n) { v = make_float4(0.f, 0.f, 0.f, 0.f); w = v; }
                        else if (col + 1 >= n) { v.z = v.w = 0.f; w.z = w.w = 0.f; }
                    }
                    const int k0 = (c & 1) * 2;
                    df_fma_cascade(d0[k0], f2{v.x, v.y}, f2{sx.x, sx.y});
                    df_fma_cascade(d0[k0 + 1], f2{v.z, v.w}, f2{sx.z, sx.w});
                    df_fma_cascade(d1[k0], f2{w.x, w.y}, f2{sx.x, sx.y});
                    df_fma_cascade(d1[k0 + 1], f2{w.z, w.w}, f2{sx.z, sx.w});
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) { d0[k] = df_norm(d0[k]); d1[k] = df_norm(d1[k]); }
                df_add(d0[0], d0[1]); df_add(d0[2], d0[3]); df_add(d0[0], d0[2]);
                df_add(d1[0], d1[1]); df_add(d1[2], d1[3]); df_add(d1[0], d1[2]);
                q0 = d0[0]; q1 = d1[0];
                pair_reduce2<f2>(q0, q1, lane, [](f2& x, f2 y) { df_add(x, y); }, shfl_f2, bcast_f2);
                if (!has1) q1 = f2{0.f, 0.f};
            }
            if (lane == 0) {
                ring.s_q[slot * 16 + lr] = q0;
                ring.s_q[slot * 16 + lr + 1] = q1;
                df_fma(qs, q0, q0);
                df_fma(qs, q1, q1);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&ring.qbars[slot]);
            ring.phase ^= (1u << slot);
            ring.qphase ^= (1u << slot);
            ring.ephase ^= (1u << slot);
            slot = (slot + 1 == g.slots) ? 0 : slot + 1;
        }
        if (lane == 0) s_scal[wid] = df_to_double(qs);
    } else {
        // ---- axpy warps: CPL columns per lane, every row of every stage
        const int aw = wid - 8;
        const int col0 = aw * (NMAX / 8) + lane * CPL;
        const bool live = FULL || col0 < n;
        f2 acc[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc[c] = f2{0.f, 0.f};
        int slot = 0;
        for (int i = 0; i < nst; ++i) {
            if (ok && !mbar_wait(&ring.qbars[slot], (ring.qphase >> slot) & 1u)) ok = false;
            if (ok && !mbar_wait(&ring.bars[slot], (ring.phase >> slot) & 1u)) ok = false;
            const int rows_here = min(16, nrows - i * 16);
            if (ok && live) {
                const char* base = ring.buf + slot * g.stage_bytes + (size_t)col0 * 8;
                const f2* q = ring.s_q + slot * 16;
                for (int r = 0; r < rows_here; ++r) {
                    const f2 qr = q[r];
                    const float* rp = reinterpret_cast<const float*>(base + r * g.row_bytes);
                    if (CPL == 1) {
                        const float2 v = *reinterpret_cast<const float2*>(rp);
                        df_fma_cascade(acc[0], qr, f2{v.x, v.y});
                    } else {
#pragma unroll
                        for (int c = 0; c < CPL; c += 2) {
                            const float4 v = *reinterpret_cast<const float4*>(rp + 2 * c);
                            df_fma_cascade(acc[c], qr, f2{v.x, v.y});
                            df_fma_cascade(acc[c + 1], qr, f2{v.z, v.w});
                        }
                    }
                }
                // renormalise once per stage: the low word then collects the errors of at most
                // 16 products, so the cascade's second-order error grows with the number of
                // stages, not with the square of the number of rows a lane sums
#pragma unroll
                for (int c = 0; c < CPL; ++c) acc[c] = df_norm(acc[c]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&ring.ebars[slot]);
            // lane 0 of warp 8: refill this slot once all 8 axpy warps are done with it
            if (aw == 0 && lane == 0 && i + g.slots < nst) {
                if (ok && !mbar_wait(&ring.ebars[slot], (ring.ephase >> slot) & 1u)) ok = false;
                if (ok) {
                    fence_proxy_async_smem();
                    const int k = i + g.slots;
                    ring_issue(ring, slot, g, src + (int64_t)k * g.stage_bytes,
                               (uint32_t)min(16, nrows - k * 16) * g.row_bytes);
                }
            }
            ring.phase ^= (1u << slot);
            ring.qphase ^= (1u << slot);
            ring.ephase ^= (1u << slot);
            slot = (slot + 1 == g.slots) ? 0 : slot + 1;
        }
        double* pw = a.part_w + (int64_t)blockIdx.x * n;
#pragma unroll
        for (int c = 0; c < CPL; ++c)
            if (FULL || col0 + c < n) pw[col0 + c] = df_to_double(df_norm(acc[c]));
    }
    if (!ok) raise_grid_error(a.err, a.bar, DEV_ERR_TIMEOUT);
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += s_scal[w];
        a.part_s[(int64_t)blockIdx.x * PART_S + 0] = t;
    }
    __syncthreads();
    return ok;
}

template <int DT, int NMAX, int MODE>
__device__ __forceinline__ bool row_pass(const PcgArgs& a, const void* vals, const double* s_v,
                                         void* s_vc_raw, double* s_scal, int64_t r0, int64_t r1,
                                         Ring& ring) {
    const Geo g = geometry(a.ld, RowOps<DT, NMAX>::ES, blockDim.x >> 5, ring.bytes);
    if constexpr (DT == LSQ_F32X2 && MODE == PASS_MATVEC && (NMAX == 256 || NMAX == 512)) {
        if (g.rpw == 1 && g.R == 16 && g.slots >= 2 && blockDim.x == 512) {
            if (a.n == NMAX) return row_pass_split<NMAX, true>(a, vals, s_v, s_vc_raw, s_scal, r0, r1, ring, g);
            return row_pass_split<NMAX, false>(a, vals, s_v, s_vc_raw, s_scal, r0, r1, ring, g);
        }
    }
    if (g.rpw == 2) return row_pass_rpw<DT, NMAX, MODE, 2>(a, vals, s_v, s_vc_raw, s_scal, r0, r1, ring, g);
    return row_pass_rpw<DT, NMAX, MODE, 1>(a, vals, s_v, s_vc_raw, s_scal, r0, r1, ring, g);
}

// sum_g part_s[g][slot] over all CTAs, computed by the calling warp (every warp of every
// CTA sums in the same order, so all agree bit for bit); no block barrier.  Four loads per
// lane are in flight together.
__device__ __forceinline__ double warp_grid_scalar(const PcgArgs& a, int slot) {
    const int lane = threadIdx.x & 31, G = (int)gridDim.x;
    const double* ps = a.part_s + slot;
    double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
    int g = lane;
    for (; g + 96 < G; g += 128) {
        t0 += ps[(int64_t)g * PART_S];
        t1 += ps[(int64_t)(g + 32) * PART_S];
        t2 += ps[(int64_t)(g + 64) * PART_S];
        t3 += ps[(int64_t)(g + 96) * PART_S];
    }
    for (; g < G; g += 32) t0 += ps[(int64_t)g * PART_S];
    return warp_sum((t0 + t1) + (t2 + t3));
}

// Writes the CTA partials pa, pb (one per warp, in s_scal) to part_s[cta][slot_a/slot_b].
__device__ __forceinline__ void cta_partials(const PcgArgs& a, double pa, double pb, int slot_a,
                                             int slot_b, double* s_scal) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (lane == 0) { s_scal[wid] = pa; s_scal[32 + wid] = pb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < nwarps; ++w) { ta += s_scal[w]; tb += s_scal[32 + w]; }
        a.part_s[(int64_t)blockIdx.x * PART_S + slot_a] = ta;
        a.part_s[(int64_t)blockIdx.x * PART_S + slot_b] = tb;
    }
    __syncthreads();
}

// w_j = (1/d_j) sum_g part_w[g][j] for the owned columns (one warp per column), handed on
// lane 0 to `fn(j, w_j)`, which returns this column's contributions to two CTA partials.
template <typename F>
__device__ __forceinline__ void slice_reduce(const PcgArgs& a, int64_t c0, int64_t c1, int slot_a,
                                             int slot_b, double* s_scal, const double* s_invd, F fn) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    double pa = 0.0, pb = 0.0;
    for (int64_t j = c0 + wid; j < c1; j += nwarps) {
        double t = 0.0;
        for (int g = lane; g < (int)gridDim.x; g += 32) t += a.part_w[(int64_t)g * a.n + j];
        t = warp_sum(t);
        if (lane == 0) {
            double2 r = fn(j, t * s_invd[j]);
            pa += r.x;
            pb += r.y;
        }
    }
    cta_partials(a, pa, pb, slot_a, slot_b, s_scal);
}

// z_j = sum_k op_jk g_k for the owned rows (g staged in s_v); partial g^T z -> slot 2.
template <typename OPT>
__device__ __forceinline__ void op_rows(const PcgArgs& a, int64_t c0, int64_t c1,
                                        const double* s_v, double* s_scal) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const OPT* op = reinterpret_cast<const OPT*>(a.op);
    const int64_t n = a.n;
    double part = 0.0;
    for (int64_t j = c0 + wid; j < c1; j += nwarps) {
        const OPT* row = op + j * n;
        OPT t0 = OPT(0), t1 = OPT(0), t2 = OPT(0), t3 = OPT(0);
        int64_t k = lane;
#pragma unroll 4
        for (; k + 96 < n; k += 128) {
            t0 = fma(row[k], (OPT)s_v[k], t0);
            t1 = fma(row[k + 32], (OPT)s_v[k + 32], t1);
            t2 = fma(row[k + 64], (OPT)s_v[k + 64], t2);
            t3 = fma(row[k + 96], (OPT)s_v[k + 96], t3);
        }
        for (; k < n; k += 32) t0 = fma(row[k], (OPT)s_v[k], t0);
        const double zj = (double)warp_sum((t0 + t1) + (t2 + t3));
        if (lane == 0) {
            a.z[j] = zj;
            part = fma(s_v[j], zj, part);
        }
    }
    cta_partials(a, part, 0.0, 2, 7, s_scal);
}

// The phase after the fused pass: p^T w as the grid sum of the CTAs' ||Â p||^2 partials
// (computed by every warp), then for the owned columns w_j = (1/d_j) sum_g part_w[g][j],
// y_j += alpha p_j, g_j -= alpha w_j and the CTA's partial of ||g||^2 (slot 1).  The loads
// of p^T w's partials, of a warp's first column's partials and of its y_j and g_j are all
// issued before any of them is used.  Returns false on a PCG breakdown (non-positive or
// non-finite p^T w or rho), the same decision in every thread of the grid.
__device__ __forceinline__ bool step_update(const PcgArgs& a, int64_t c0, int64_t c1, double rho,
                                            const double* s_p, const double* s_invd, double* s_scal) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int G = (int)gridDim.x;
    const int64_t n = a.n;
    const int64_t j0 = c0 + wid;
    const bool own = j0 < c1;
    double yj = 0.0, gj = 0.0;
    if (own && lane == 0) { yj = a.y[j0]; gj = a.g[j0]; }
    const double* ps = a.part_s;
    const double* pw = a.part_w + (own ? j0 : 0);
    double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0, u0 = 0.0, u1 = 0.0, u2 = 0.0, u3 = 0.0;
    int g = lane;
    for (; g + 96 < G; g += 128) {
        t0 += ps[(int64_t)g * PART_S];
        t1 += ps[(int64_t)(g + 32) * PART_S];
        t2 += ps[(int64_t)(g + 64) * PART_S];
        t3 += ps[(int64_t)(g + 96) * PART_S];
        if (own) {
            u0 += pw[(int64_t)g * n];
            u1 += pw[(int64_t)(g + 32) * n];
            u2 += pw[(int64_t)(g + 64) * n];
            u3 += pw[(int64_t)(g + 96) * n];
        }
    }
    for (; g < G; g += 32) {
        t0 += ps[(int64_t)g * PART_S];
        if (own) u0 += pw[(int64_t)g * n];
    }
    const double pTw = warp_sum((t0 + t1) + (t2 + t3));
    const double wsum = warp_sum((u0 + u1) + (u2 + u3));
    if (!(pTw > 0.0) || !(rho > 0.0) || !isfinite(pTw) || !isfinite(rho)) return false;
    const double alpha = rho / pTw;
    double part = 0.0;
    if (own && lane == 0) {
        const double w = wsum * s_invd[j0];
        yj = fma(alpha, s_p[j0], yj);
        gj = fma(-alpha, w, gj);
        a.y[j0] = yj;
        a.g[j0] = gj;
        part = gj * gj;
    }
    for (int64_t j = j0 + nwarps; j < c1; j += nwarps) {   // more columns than warps
        double t = 0.0;
        for (int gg = lane; gg < G; gg += 32) t += a.part_w[(int64_t)gg * n + j];
        t = warp_sum(t);
        if (lane == 0) {
            const double w = t * s_invd[j];
            a.y[j] = fma(alpha, s_p[j], a.y[j]);
            const double gn = fma(-alpha, w, a.g[j]);
            a.g[j] = gn;
            part += gn * gn;
        }
    }
    cta_partials(a, part, 0.0, 1, 6, s_scal);
    return true;
}

// Copies the n-vector src (global) into s_dst and returns the grid sum of part_s[][slot];
// the vector's loads and the partials' loads are in flight together.
template <int NMAX>
__device__ __forceinline__ double stage_with_scalar(const PcgArgs& a, const double* src, double* s_dst, int slot) {
    constexpr int PER = (NMAX + 511) / 512;
    double v[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int64_t j = threadIdx.x + (int64_t)r * blockDim.x;
        v[r] = j < a.n ? src[j] : 0.0;
    }
    const double s = warp_grid_scalar(a, slot);
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int64_t j = threadIdx.x + (int64_t)r * blockDim.x;
        if (j < a.n) s_dst[j] = v[r];
    }
    return s;
}

template <int DT, int DTR, int NMAX, typename OPT>
__global__ void __launch_bounds__(512, 1) k_pcg_dense(PcgArgs a) {
    extern __shared__ __align__(128) char smem_raw[];
    __shared__ double s_scal[64];
    __shared__ __align__(8) uint64_t s_bars[RING_SLOTS];
    __shared__ __align__(8) uint64_t s_qbars[RING_SLOTS];
    __shared__ __align__(8) uint64_t s_ebars[RING_SLOTS];
    __shared__ __align__(16) f2 s_q[RING_SLOTS * 16];
    const int64_t n = a.n;
    const int nwarps = blockDim.x >> 5;
    const int lane = threadIdx.x & 31;
    const int RB = ring_bytes(NMAX);
    Ring ring{smem_raw, s_bars, 0u, RB, nullptr, 0u, 0, s_qbars, s_ebars, 0u, 0u, s_q, l2_evict_first_policy()};
    unsigned long long bar_epoch = 0;   // grid barriers passed (the same count in every CTA)
    double* s_p = reinterpret_cast<double*>(smem_raw + RB);  // NMAX: p (replicated)
    double* s_v = s_p + NMAX;        // NMAX: D^{-1} x vector for the row pass, or g
    double* s_vc = s_v + NMAX;       // NMAX: s_v in the compute type of the row pass
    double* s_invd = s_vc + NMAX;    // NMAX: 1 / d_j
    if (threadIdx.x == 0) {
        for (int i = 0; i < RING_SLOTS; ++i) {
            mbar_init(&s_bars[i], 1);
            mbar_init(&s_qbars[i], 8);   // the 8 dot warps of row_pass_split
            mbar_init(&s_ebars[i], 8);   // the 8 axpy warps
        }
        fence_mbar_init();
    }
    for (int64_t j = threadIdx.x; j < NMAX; j += blockDim.x) {
        s_p[j] = 0.0; s_v[j] = 0.0;
        s_invd[j] = j < n ? a.inv_d[j] : 0.0;
    }
    __syncthreads();
    const unsigned G = gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * a.m / G, r1 = (int64_t)(blockIdx.x + 1) * a.m / G;
    const int64_t c0 = (int64_t)blockIdx.x * n / G, c1 = (int64_t)(blockIdx.x + 1) * n / G;
    const Geo gmv = geometry(a.ld, RowOps<DT, NMAX>::ES, nwarps, RB);
    const char* mv_src = reinterpret_cast<const char*>(a.vals) + r0 * (int64_t)gmv.row_bytes;
#define LSQ_BARRIER()                                   \
    do {                                                \
        if (!grid_barrier(a.bar, G, a.err, bar_epoch, a.max_polls)) { \
            ring_drain(ring);                           \
            return;                                     \
        }                                               \
    } while (0)

    int iters = 0, outer_used = 0, converged = 0, status = LSQ_ERR_NOT_CONVERGED;
    double rec = 1.0, tru = 1.0, gg = 0.0;
    bool dirty = false;  // iterations since the last true residual

    // h = Â^T b (values of the residual dtype) or the given h; y = 0; g = h
    if (a.h_in) {
        double ha = 0.0, hb = 0.0;
        for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
            const double h = a.h_in[j], hr = h / s_invd[j];
            a.g[j] = h; a.y[j] = 0.0;
            ha = fma(h, h, ha); hb = fma(hr, hr, hb);
        }
        cta_partials(a, warp_sum(ha), warp_sum(hb), 1, 4, s_scal);
    } else {
        row_pass<DTR, NMAX, PASS_RHS>(a, a.vals_res, s_v, s_vc, s_scal, r0, r1, ring);
        ring_prefetch(ring, mv_src, gmv, r1 - r0);
        LSQ_BARRIER();
        slice_reduce(a, c0, c1, 1, 4, s_scal, s_invd, [&](int64_t j, double h) {
            a.g[j] = h; a.y[j] = 0.0;
            const double hr = h / s_invd[j];
            return make_double2(h * h, hr * hr); });
    }
    LSQ_BARRIER();
    gg = warp_grid_scalar(a, 1);
    const double hn = sqrt(gg);
    const double hn_raw = sqrt(warp_grid_scalar(a, 4));
    double raw = 1.0;
    if (hn == 0.0) {
        converged = 1; status = LSQ_OK; rec = 0.0; tru = 0.0;
    } else {
        for (int outer = 0; outer < a.max_outer; ++outer) {
            if (outer > 0) {
                // true residual g = Â^T (b - Â y)  (normal form: g = h - Â^T Â y)
                for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s_v[j] = a.y[j] * s_invd[j];
                __syncthreads();
                if (a.h_in) row_pass<DTR, NMAX, PASS_MATVEC>(a, a.vals_res, s_v, s_vc, s_scal, r0, r1, ring);
                else row_pass<DTR, NMAX, PASS_RESID>(a, a.vals_res, s_v, s_vc, s_scal, r0, r1, ring);
                ring_prefetch(ring, mv_src, gmv, r1 - r0);
                LSQ_BARRIER();
                slice_reduce(a, c0, c1, 1, 5, s_scal, s_invd, [&](int64_t j, double t) {
                    if (a.h_in) t = a.h_in[j] - t;
                    a.g[j] = t;
                    const double tr = t / s_invd[j];
                    return make_double2(t * t, tr * tr); });
                LSQ_BARRIER();
                gg = warp_grid_scalar(a, 1);
                raw = sqrt(warp_grid_scalar(a, 5)) / hn_raw;
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
            LSQ_BARRIER();
            double rho = warp_grid_scalar(a, 2);
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
                const double pj = a.z[j];
                s_p[j] = pj;
                s_v[j] = pj * s_invd[j];
            }
            __syncthreads();
            bool broke = false;
            while (true) {
                // fused pass: w = Â^T (Â p), ||Â p||^2 = p^T w
                row_pass<DT, NMAX, PASS_MATVEC>(a, a.vals, s_v, s_vc, s_scal, r0, r1, ring);
                ring_prefetch(ring, mv_src, gmv, r1 - r0);
                LSQ_BARRIER();
                if (!step_update(a, c0, c1, rho, s_p, s_invd, s_scal)) {
                    status = LSQ_ERR_BREAKDOWN; broke = true; break;
                }
                LSQ_BARRIER();
                ++iters;
                dirty = true;
                gg = stage_with_scalar<NMAX>(a, a.g, s_v, 1);
                rec = sqrt(gg) / hn;
                __syncthreads();
                if (rec <= a.tol || sqrt(gg) <= a.inner_tol * gstart) break;
                if (iters >= a.maxit) break;
                op_rows<OPT>(a, c0, c1, s_v, s_scal);
                LSQ_BARRIER();
                {
                    // rho' = g^T z over the grid and p = z + beta p; z's loads go out first
                    constexpr int PER = (NMAX + 511) / 512;
                    double zv[PER];
#pragma unroll
                    for (int r = 0; r < PER; ++r) {
                        const int64_t j = threadIdx.x + (int64_t)r * blockDim.x;
                        zv[r] = j < n ? a.z[j] : 0.0;
                    }
                    const double rho_new = warp_grid_scalar(a, 2);
                    const double beta = rho_new / rho;
                    rho = rho_new;
#pragma unroll
                    for (int r = 0; r < PER; ++r) {
                        const int64_t j = threadIdx.x + (int64_t)r * blockDim.x;
                        if (j < n) {
                            const double pj = fma(beta, s_p[j], zv[r]);
                            s_p[j] = pj;
                            s_v[j] = pj * s_invd[j];
                        }
                    }
                }
                __syncthreads();
            }
            if (broke) break;
        }
        if (!converged && status != LSQ_ERR_BREAKDOWN && dirty) {
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x) s_v[j] = a.y[j] * s_invd[j];
            __syncthreads();
            if (a.h_in) row_pass<DTR, NMAX, PASS_MATVEC>(a, a.vals_res, s_v, s_vc, s_scal, r0, r1, ring);
            else row_pass<DTR, NMAX, PASS_RESID>(a, a.vals_res, s_v, s_vc, s_scal, r0, r1, ring);
            LSQ_BARRIER();
            slice_reduce(a, c0, c1, 3, 5, s_scal, s_invd, [&](int64_t j, double t) {
                if (a.h_in) t = a.h_in[j] - t;
                a.g[j] = t;
                const double tr = t / s_invd[j];
                return make_double2(t * t, tr * tr); });
            LSQ_BARRIER();
            tru = sqrt(warp_grid_scalar(a, 3)) / hn;
            raw = sqrt(warp_grid_scalar(a, 5)) / hn_raw;
            if (tru <= a.tol) { converged = 1; status = LSQ_OK; }
        }
    }
#undef LSQ_BARRIER
    ring_drain(ring);
    for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) a.x[j] = a.y[j] * s_invd[j];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.out_i[0] = iters; a.out_i[1] = outer_used; a.out_i[2] = converged; a.out_i[3] = status;
        a.out_d[0] = rec; a.out_d[1] = tru; a.out_d[2] = (hn == 0.0) ? 0.0 : raw;
    }
    (void)lane;
}

// Host launcher (defined per dtype in pcg_f64.cu / pcg_f32.cu)
lsq_status launch_pcg_dense(int dt, int dtr, int opt_dtype, int64_t nmax, PcgArgs& args,
                            int grid_cap, cudaStream_t st, int* grid_used);

}  // namespace lsq
