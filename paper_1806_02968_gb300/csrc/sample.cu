// Alg. 2 steps 1-2 and Alg. 1: exact column scales, exact row weights (Eq. R2P), exact
// prefix sums and Philox4x64-10 draws.  Everything that decides an index is integer
// arithmetic or a single correctly rounded FP64 operation, so the indices are
// reproducible bit for bit.
#include "common.cuh"
#include "values.cuh"

#include <cmath>
#include <mutex>

namespace lsq {

std::atomic<int64_t> g_launches{0};
std::atomic<uint32_t> g_wait_polls{0};
static thread_local std::string t_err;
void set_error(const std::string& msg) { t_err = msg; }
const char* last_error() { return t_err.c_str(); }

lsq_status check_matrix(const lsq_matrix* A) {
    LSQ_CHECK_ARG(A != nullptr, "A is NULL");
    LSQ_CHECK_ARG(A->m > 0 && A->n > 0, "m and n must be positive");
    LSQ_CHECK_ARG(A->m < (int64_t)INT32_MAX && A->n < (int64_t)INT32_MAX, "m, n must be < 2^31");
    LSQ_CHECK_ARG(A->vals != nullptr, "A->vals is NULL");
    LSQ_CHECK_ARG(elem_size(A->dtype) != 0, "unknown dtype");
    if (A->dense) {
        LSQ_CHECK_ARG(A->ld >= A->n, "dense ld < n");
    } else {
        LSQ_CHECK_ARG(A->row_ptr != nullptr && A->col_idx != nullptr, "CSR arrays are NULL");
        LSQ_CHECK_ARG(A->nnz >= 0, "nnz < 0");
    }
    return LSQ_OK;
}

lsq_status read_dev_error(const unsigned* d_err, cudaStream_t st, unsigned* bits_out) {
    unsigned bits = 0;
    LSQ_CUDA(cudaMemcpyAsync(&bits, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    LSQ_CUDA(cudaStreamSynchronize(st));
    if (bits_out) *bits_out = bits;
    if (bits & DEV_ERR_TIMEOUT) { set_error("device-side wait timed out"); return LSQ_ERR_TIMEOUT; }
    if (bits & DEV_ERR_RANGE) { set_error("values must be finite with max a_ij^2 in [2^-900, 2^900]"); return LSQ_ERR_INVALID; }
    if (bits & DEV_ERR_EMPTY) { set_error("no row has positive sampling weight"); return LSQ_ERR_INVALID; }
    if (bits & DEV_ERR_BREAKDOWN) { set_error("PCG breakdown"); return LSQ_ERR_BREAKDOWN; }
    return LSQ_OK;
}

// ---------------------------------------------------------------------------------------
// floor(x * 2^e) for a non-negative finite double x with x * 2^e < 2^64, by bit surgery:
// x = mant * 2^(ex - 1075), so the result is mant shifted by (ex - 1075 + e).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long floor_scaled(double x, int e) {
    unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    int ex = (int)((bits >> 52) & 0x7ff);
    unsigned long long mant = bits & ((1ull << 52) - 1);
    int sh;
    if (ex == 0) { sh = -1074 + e; } else { mant |= (1ull << 52); sh = ex - 1075 + e; }
    if (mant == 0) return 0;
    if (sh >= 0) return sh >= 64 ? 0ull : (mant << sh);  // (the caller guarantees no overflow)
    return sh <= -64 ? 0ull : (mant >> (-sh));
}

// E1 = 52 - floor(log2 T) for T = fl(amax^2); false when T is outside [2^-900, 2^900].
__device__ __forceinline__ bool exponent_of(unsigned long long amax_bits, int* E1) {
    double amax = __longlong_as_double((long long)amax_bits);
    double T = __dmul_rn(amax, amax);
    if (!(T >= 0x1p-900 && T <= 0x1p900)) return false;
    *E1 = 52 - ilogb(T);
    return true;
}

// ---------------------------------------------------------------------------------------
// S1a: per-column max |a_ij| (bit patterns of non-negative doubles order like the values)
// and a non-finite check.
// ---------------------------------------------------------------------------------------
template <int DT>
__global__ void k_colmax_dense(lsq_matrix A, unsigned long long* amax, unsigned* err,
                               int64_t rows_per_block) {
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(A.m, r0 + rows_per_block);
    bool bad = false;
    for (int64_t j = threadIdx.x; j < A.n; j += blockDim.x) {
        unsigned long long best = 0;
        for (int64_t i = r0; i < r1; ++i) {
            double a = fabs(Val<DT>::load(A.vals, i * A.ld + j));
            bad |= !(a <= 1.7976931348623157e308);
            unsigned long long b = (unsigned long long)__double_as_longlong(a);
            best = b > best ? b : best;
        }
        if (best) atomicMax(&amax[j], best);
    }
    if (bad) atomicOr(err, DEV_ERR_RANGE);
}

template <int DT>
__global__ void k_colmax_csr(lsq_matrix A, unsigned long long* amax, unsigned* err) {
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < A.nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        double a = fabs(Val<DT>::load(A.vals, e));
        bad |= !(a <= 1.7976931348623157e308);
        unsigned long long b = (unsigned long long)__double_as_longlong(a);
        if (b) atomicMax(&amax[A.col_idx[e]], b);
    }
    if (bad) atomicOr(err, DEV_ERR_RANGE);
}

// Per-column exponents E1_j (0 for an all-zero column) and the global E1 = min_j E1_j,
// stored in *E1g as E1 + 4096 through atomicMin (so that the initial 0xffffffff is "none").
__global__ void k_col_exponents(int64_t n, const unsigned long long* amax, int* E1j,
                                unsigned* E1g, unsigned* err) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        int e = 0;
        if (amax[j]) {
            if (!exponent_of(amax[j], &e)) { atomicOr(err, DEV_ERR_RANGE); e = 0; }
            else atomicMin(E1g, (unsigned)(e + 4096));
        }
        E1j[j] = e;
    }
}

// ---------------------------------------------------------------------------------------
// S1b: c_j = sum_i floor(fl(a_ij^2) 2^E1_j), exact in 128 bits.
// ---------------------------------------------------------------------------------------
template <int DT>
__global__ void k_colsum_dense(lsq_matrix A, const int* E1j, u128* c, int64_t rows_per_block) {
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = min(A.m, r0 + rows_per_block);
    for (int64_t j = threadIdx.x; j < A.n; j += blockDim.x) {
        const int E1 = E1j[j];
        u128 acc = 0;
        for (int64_t i = r0; i < r1; ++i) {
            double a = Val<DT>::load(A.vals, i * A.ld + j);
            acc += floor_scaled(__dmul_rn(a, a), E1);
        }
        if (acc) atomic_add_u128(&c[j], acc);
    }
}

template <int DT>
__global__ void k_colsum_csr(lsq_matrix A, const int* E1j, u128* c) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < A.nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = A.col_idx[e];
        double a = Val<DT>::load(A.vals, e);
        unsigned long long q = floor_scaled(__dmul_rn(a, a), E1j[j]);
        if (q) atomic_add_u128(&c[j], (u128)q);
    }
}

// ---------------------------------------------------------------------------------------
// S1c: d2_j = RNE(c_j) 2^-E1_j, d_j = sqrt(d2_j), inv_d2_j = RN(1/d2_j); zero column: d_j = 1,
// inv_d2_j = 0.  Without normalisation: d_j = 1, inv_d2_j = 2^(E1-52), E1 the global one.
// ---------------------------------------------------------------------------------------
__global__ void k_colscale(int64_t n, int normalize, const int* E1j, const unsigned* E1g,
                           const u128* c, double* d2, double* inv_d2, double* d) {
    const int E1 = (*E1g == 0xffffffffu) ? 52 : (int)*E1g - 4096;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        u128 cj = c[j];
        double two_mE1 = __longlong_as_double((long long)(1023 - E1j[j]) << 52);
        double v = __dmul_rn(u128_to_double_rn(cj), two_mE1);
        d2[j] = v;
        if (!normalize) {
            d[j] = 1.0;
            inv_d2[j] = __longlong_as_double((long long)(1023 + E1 - 52) << 52);
        } else if (cj == 0) {
            d[j] = 1.0;
            inv_d2[j] = 0.0;
        } else {
            d[j] = __dsqrt_rn(v);
            inv_d2[j] = __drcp_rn(v);
        }
    }
}

// ---------------------------------------------------------------------------------------
// S2: w_i = sum_j floor(2^51 fl(fl(a_ij^2) inv_d2_j)), one warp per row, exact.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
        unsigned long long olo = __shfl_xor_sync(0xffffffffu, lo, o);
        unsigned long long ohi = __shfl_xor_sync(0xffffffffu, hi, o);
        v += ((u128)ohi << 64) | olo;
    }
    return v;
}

template <int DT>
__global__ void k_rowweight(lsq_matrix A, const double* inv_d2, u128* w, int uniform) {
    int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < A.m; i += nwarps) {
        if (uniform) {   // the uniform density of the comparison in Sec. 3.1: w_i = 1
            if (lane == 0) w[i] = 1;
            continue;
        }
        u128 acc = 0;
        if (A.dense) {
            for (int64_t j = lane; j < A.n; j += 32) {
                double a = Val<DT>::load(A.vals, i * A.ld + j);
                double u = __dmul_rn(__dmul_rn(a, a), inv_d2[j]);
                acc += floor_scaled(u, 51);
            }
        } else {
            int64_t e0 = A.row_ptr[i], e1 = A.row_ptr[i + 1];
            for (int64_t e = e0 + lane; e < e1; e += 32) {
                double a = Val<DT>::load(A.vals, e);
                double u = __dmul_rn(__dmul_rn(a, a), inv_d2[A.col_idx[e]]);
                acc += floor_scaled(u, 51);
            }
        }
        acc = warp_sum_u128(acc);
        if (lane == 0) w[i] = acc;
    }
}

// ---------------------------------------------------------------------------------------
// S3: exclusive prefix P_0 = 0, P_{i+1} = P_i + w_i (three passes; integer adds are
// associative, so the result does not depend on the blocking).
// ---------------------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_PER_THREAD = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;

__device__ __forceinline__ u128 block_exclusive_scan_u128(u128 v, u128* total) {
    __shared__ unsigned long long s_lo[32], s_hi[32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // inclusive warp scan
    u128 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long lo = (unsigned long long)x, hi = (unsigned long long)(x >> 64);
        unsigned long long plo = __shfl_up_sync(0xffffffffu, lo, o);
        unsigned long long phi = __shfl_up_sync(0xffffffffu, hi, o);
        if (lane >= o) x += ((u128)phi << 64) | plo;
    }
    if (lane == 31) { s_lo[wid] = (unsigned long long)x; s_hi[wid] = (unsigned long long)(x >> 64); }
    __syncthreads();
    int nw = blockDim.x >> 5;
    if (wid == 0) {
        u128 y = lane < nw ? (((u128)s_hi[lane] << 64) | s_lo[lane]) : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long lo = (unsigned long long)y, hi = (unsigned long long)(y >> 64);
            unsigned long long plo = __shfl_up_sync(0xffffffffu, lo, o);
            unsigned long long phi = __shfl_up_sync(0xffffffffu, hi, o);
            if (lane >= o) y += ((u128)phi << 64) | plo;
        }
        if (lane < nw) { s_lo[lane] = (unsigned long long)y; s_hi[lane] = (unsigned long long)(y >> 64); }
    }
    __syncthreads();
    u128 warp_off = wid ? (((u128)s_hi[wid - 1] << 64) | s_lo[wid - 1]) : 0;
    if (total) *total = ((u128)s_hi[nw - 1] << 64) | s_lo[nw - 1];
    u128 excl = x - v + warp_off;
    __syncthreads();
    return excl;
}

__global__ void k_scan_tiles(const u128* w, int64_t m, u128* tile_sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER_THREAD;
    u128 s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k)
        if (base + k < m) s += w[base + k];
    u128 tot;
    block_exclusive_scan_u128(s, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(u128* tile_sums, int64_t ntiles) {
    u128 carry = 0;
    for (int64_t base = 0; base < ntiles; base += blockDim.x) {
        int64_t t = base + threadIdx.x;
        u128 v = t < ntiles ? tile_sums[t] : 0;
        u128 tot;
        u128 ex = block_exclusive_scan_u128(v, &tot);
        if (t < ntiles) tile_sums[t] = ex + carry;
        carry += tot;
        __syncthreads();
    }
}

__global__ void k_scan_apply(const u128* w, int64_t m, const u128* tile_offsets, u128* P) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER_THREAD;
    u128 vals[SCAN_PER_THREAD];
    u128 s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        vals[k] = base + k < m ? w[base + k] : 0;
        s += vals[k];
    }
    u128 tot;
    u128 ex = block_exclusive_scan_u128(s, &tot) + tile_offsets[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        if (base + k < m) P[base + k] = ex;
        ex += vals[k];
    }
    if (base + SCAN_PER_THREAD >= m && base < m) P[m] = ex;  // the thread holding row m-1
}

// ---------------------------------------------------------------------------------------
// S4: Philox4x64-10 (Salmon et al., SC'11) and the inverse-CDF search.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                              unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += W0; k1 += W1;  // (the bump after the last round is unused)
    }
}

// high 128 bits of the 256-bit product a*b
__device__ __forceinline__ u128 mulhi_u128(u128 a, u128 b) {
    unsigned long long a0 = (unsigned long long)a, a1 = (unsigned long long)(a >> 64);
    unsigned long long b0 = (unsigned long long)b, b1 = (unsigned long long)(b >> 64);
    u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1, p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
    u128 mid = (p00 >> 64) + (unsigned long long)p01 + (unsigned long long)p10;
    return p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);
}

__global__ void k_draw(const u128* P, int64_t m, int64_t s, unsigned long long seed,
                       int32_t* idx, double* p_out, unsigned* err) {
    u128 W = P[m];
    if (W == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, DEV_ERR_EMPTY);
        return;
    }
    double Wd = u128_to_double_rn(W);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < s;
         t += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long c[4] = {(unsigned long long)t, 0ull, 0ull, 0ull};
        philox4x64_10(c, seed, 0x5A4D504Cull);
        u128 U = ((u128)c[1] << 64) | c[0];
        u128 target = mulhi_u128(U, W);
        int64_t lo = 0, hi = m;  // P[lo] <= target < P[hi]
        while (hi - lo > 1) {
            int64_t mid = lo + ((hi - lo) >> 1);
            if (P[mid] <= target) lo = mid; else hi = mid;
        }
        idx[t] = (int32_t)lo;
        if (p_out) p_out[t] = __ddiv_rn(u128_to_double_rn(P[lo + 1] - P[lo]), Wd);
    }
}

// ---------------------------------------------------------------------------------------
// Row-sharded sampling: a rank holds a contiguous block of rows.  The exact integer law
// makes the cross-rank steps plain integer collectives: column maxima (MAX), exact column
// sums (SUM of 32-bit limbs), the ranks' weight totals (all-gather), and the merge of the
// draws (MAX over -1 / row index), so the indices equal one process's bit for bit.
// ---------------------------------------------------------------------------------------
__global__ void k_u128_to_limbs(int64_t n, const u128* c, int64_t* limbs) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const u128 v = c[j];
#pragma unroll
        for (int k = 0; k < 4; ++k) limbs[4 * j + k] = (int64_t)(unsigned long long)((v >> (32 * k)) & 0xFFFFFFFFull);
    }
}
// limbs (each a sum of 32-bit limbs over the ranks, < 2^63) back to u128 with the carries
__global__ void k_limbs_to_u128(int64_t n, const int64_t* limbs, u128* c) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        u128 v = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) v += (u128)(unsigned long long)limbs[4 * j + k] << (32 * k);
        c[j] = v;
    }
}
// Draws t = 0..s-1 of Alg. 1 against the whole matrix's total W; a rank keeps those whose
// target falls in its range [O, O + W_r) and finds the row in its local prefix.
__global__ void k_draw_shard(const u128* P, int64_t m, int64_t row0, unsigned long long O_lo,
                             unsigned long long O_hi, unsigned long long W_lo, unsigned long long W_hi,
                             int64_t s, unsigned long long seed, int32_t* idx, double* p_out) {
    const u128 O = ((u128)O_hi << 64) | O_lo, W = ((u128)W_hi << 64) | W_lo;
    const u128 Wr = P[m];
    const double Wd = u128_to_double_rn(W);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < s;
         t += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long c[4] = {(unsigned long long)t, 0ull, 0ull, 0ull};
        philox4x64_10(c, seed, 0x5A4D504Cull);
        const u128 U = ((u128)c[1] << 64) | c[0];
        const u128 target = mulhi_u128(U, W);
        if (target < O || target - O >= Wr) {
            idx[t] = -1;
            if (p_out) p_out[t] = 0.0;
            continue;
        }
        const u128 local = target - O;
        int64_t lo = 0, hi = m;  // P[lo] <= local < P[hi]
        while (hi - lo > 1) {
            int64_t mid = lo + ((hi - lo) >> 1);
            if (P[mid] <= local) lo = mid; else hi = mid;
        }
        idx[t] = (int32_t)(row0 + lo);
        if (p_out) p_out[t] = __ddiv_rn(u128_to_double_rn(P[lo + 1] - P[lo]), Wd);
    }
}

static int grid_for(int64_t work, int threads, int cap = 152 * 16) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// Scratch layout of one sampling call (256-byte aligned pieces; the first three are the
// accumulating words that must start at zero).
struct SampleLayout {
    size_t err, amax, c, E1g, E1j, d2, inv, d, w, P, ts, total;
};
constexpr size_t rnd256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr SampleLayout sample_layout(int64_t m, int64_t n) {
    SampleLayout L{};
    size_t off = 0;
    L.err = off;  off += rnd256(16);
    L.amax = off; off += rnd256(8 * n);
    L.c = off;    off += rnd256(16 * n);
    L.E1g = off;  off += rnd256(16);
    L.E1j = off;  off += rnd256(4 * n);
    L.d2 = off;   off += rnd256(8 * n);
    L.inv = off;  off += rnd256(8 * n);
    L.d = off;    off += rnd256(8 * n);
    L.w = off;    off += rnd256(16 * m);
    L.P = off;    off += rnd256(16 * (m + 1));
    L.ts = off;   off += rnd256(16 * ((m + SCAN_TILE - 1) / SCAN_TILE));
    L.total = off;
    return L;
}

// S1-S4 on the scratch at `base` (laid out by sample_layout): the nine kernels of one
// sampling call, then the device error word.  Every word that accumulates is cleared
// first, so the scratch may hold anything on entry.
template <int DT>
static lsq_status sample_launch(const lsq_matrix* A, const lsq_opts* o, int64_t s, int32_t* idx_out,
                                double* p_out, double* colscale_out, char* base, cudaStream_t st) {
    const int64_t m = A->m, n = A->n;
    const SampleLayout L = sample_layout(m, n);
    const int64_t ntiles = (m + SCAN_TILE - 1) / SCAN_TILE;
    unsigned* err = (unsigned*)(base + L.err);
    unsigned long long* amax = (unsigned long long*)(base + L.amax);
    u128* c = (u128*)(base + L.c);
    unsigned* E1g = (unsigned*)(base + L.E1g);
    int* E1j = (int*)(base + L.E1j);
    double* d2 = (double*)(base + L.d2);
    double* inv = (double*)(base + L.inv);
    double* d = colscale_out ? colscale_out : (double*)(base + L.d);
    u128* w = (u128*)(base + L.w);
    u128* P = (u128*)(base + L.P);
    u128* ts = (u128*)(base + L.ts);
    LSQ_CUDA(cudaMemsetAsync(base, 0, L.E1g, st));
    LSQ_CUDA(cudaMemsetAsync(E1g, 0xff, 16, st));

    lsq_matrix Av = *A;
    int64_t rpb = 0;
    if (A->dense) {
        rpb = (m + 152 * 8 - 1) / (152 * 8);
        if (rpb < 16) rpb = 16;
        k_colmax_dense<DT><<<(int)((m + rpb - 1) / rpb), 256, 0, st>>>(Av, amax, err, rpb);
    } else {
        k_colmax_csr<DT><<<grid_for(A->nnz, 256), 256, 0, st>>>(Av, amax, err);
    }
    k_col_exponents<<<grid_for(n, 256), 256, 0, st>>>(n, amax, E1j, E1g, err);
    if (A->dense) k_colsum_dense<DT><<<(int)((m + rpb - 1) / rpb), 256, 0, st>>>(Av, E1j, c, rpb);
    else k_colsum_csr<DT><<<grid_for(A->nnz, 256), 256, 0, st>>>(Av, E1j, c);
    k_colscale<<<grid_for(n, 256), 256, 0, st>>>(n, o->normalize ? 1 : 0, E1j, E1g, c, d2, inv, d);
    k_rowweight<DT><<<grid_for(m * 32, 256), 256, 0, st>>>(Av, inv, w, o->sampling == 1 ? 1 : 0);
    k_scan_tiles<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(w, m, ts);
    k_scan_sums<<<1, 1024, 0, st>>>(ts, ntiles);
    k_scan_apply<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(w, m, ts, P);
    k_draw<<<grid_for(s, 256), 256, 0, st>>>(P, m, s, (unsigned long long)o->seed, idx_out, p_out, err);
    count_launch(9);
    LSQ_CUDA(cudaGetLastError());
    return read_dev_error(err, st);
}

template <int DT>
static lsq_status sample_impl(const lsq_matrix* A, const lsq_opts* o, int64_t s,
                              int32_t* idx_out, double* p_out, double* colscale_out,
                              cudaStream_t st) {
    Scratch sc;
    LSQ_CUDA(sc.alloc(sample_layout(A->m, A->n).total, st));
    return sample_launch<DT>(A, o, s, idx_out, p_out, colscale_out, sc.as<char>(), st);
}

// ---------------------------------------------------------------------------------------
// Fixed scratch for lsq_sample_rows_static: the same launcher as lsq_sample_rows, with the
// scratch carved from one file-scope device array instead of a stream-ordered allocation.
// ---------------------------------------------------------------------------------------
constexpr int64_t STATIC_MAX_ROWS = 262144;
constexpr int64_t STATIC_MAX_COLS = 4096;
constexpr size_t STATIC_SCRATCH_BYTES = sample_layout(STATIC_MAX_ROWS, STATIC_MAX_COLS).total;
static __device__ __align__(256) unsigned char g_sample_scratch[STATIC_SCRATCH_BYTES];

// Device address of g_sample_scratch on the current device, looked up once per device and
// kept for the life of the process's primary context on that device.
static lsq_status static_scratch_address(char** out) {
    static std::mutex mu;
    static void* addr[64] = {};
    int dev = 0;
    LSQ_CUDA(cudaGetDevice(&dev));
    LSQ_CHECK_ARG(dev >= 0 && dev < 64, "device ordinal must be < 64");
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        LSQ_CUDA(cudaGetSymbolAddress(&p, g_sample_scratch));
        addr[dev] = p;
    }
    *out = static_cast<char*>(addr[dev]);
    return LSQ_OK;
}

template <int DT>
static lsq_status sample_into_static(const lsq_matrix* A, const lsq_opts* o, int64_t s, int32_t* idx_out,
                                     double* p_out, double* colscale_out, char* base, cudaStream_t st) {
    if (sample_layout(A->m, A->n).total > STATIC_SCRATCH_BYTES) {
        set_error("static scratch layout exceeds its array");
        return LSQ_ERR_INVALID;
    }
    return sample_launch<DT>(A, o, s, idx_out, p_out, colscale_out, base, st);
}

}  // namespace lsq

using namespace lsq;

extern "C" void lsq_default_opts(lsq_opts* o) {
    if (!o) return;
    o->tol = 1e-10;
    o->maxit = 1000000;
    o->max_outer = 20;
    o->sweeps = 1;
    o->sample_factor = 4.0;
    o->normalize = 1;
    o->precond_dtype = LSQ_F64;
    o->seed = 0;
    o->inner_tol = 0.0;
    o->grid_ctas = 0;
    o->sampling = 0;
    o->device_loop = 0;
}

extern "C" lsq_status lsq_set_wait_limit(int64_t max_polls) {
    LSQ_CHECK_ARG(max_polls >= 0 && max_polls <= ((int64_t)1 << 31), "max_polls must lie in [0, 2^31]");
    g_wait_polls.store((uint32_t)max_polls, std::memory_order_relaxed);
    return LSQ_OK;
}

extern "C" int64_t lsq_sample_size(int64_t n, double C) {
    if (n < 2) return 1;
    return (int64_t)std::ceil(C * (double)n * std::log((double)n));
}

extern "C" lsq_status lsq_sample_rows(const lsq_matrix* A, const lsq_opts* o, int64_t s,
                                      int32_t* idx_out, double* p_out, double* colscale_out,
                                      int64_t* s_out, void* stream) {
    lsq_status st0 = check_matrix(A);
    if (st0 != LSQ_OK) return st0;
    LSQ_CHECK_ARG(o != nullptr, "opts is NULL");
    LSQ_CHECK_ARG(idx_out != nullptr, "idx_out is NULL");
    LSQ_CHECK_ARG(s >= 0, "s < 0");
    LSQ_CHECK_ARG(o->sampling == 0 || o->sampling == 1, "sampling must be 0 (norm squared) or 1 (uniform)");
    if (s == 0) s = lsq_sample_size(A->n, o->sample_factor);
    LSQ_CHECK_ARG(s > 0 && s < (int64_t)1 << 40, "sample size out of range");
    if (s_out) *s_out = s;
    cudaStream_t st = (cudaStream_t)stream;
    switch (A->dtype) {
        case LSQ_F64: return sample_impl<LSQ_F64>(A, o, s, idx_out, p_out, colscale_out, st);
        case LSQ_F32: return sample_impl<LSQ_F32>(A, o, s, idx_out, p_out, colscale_out, st);
        case LSQ_BF16: return sample_impl<LSQ_BF16>(A, o, s, idx_out, p_out, colscale_out, st);
        case LSQ_F32X2: return sample_impl<LSQ_F32X2>(A, o, s, idx_out, p_out, colscale_out, st);
    }
    set_error("unknown dtype");
    return LSQ_ERR_INVALID;
}

extern "C" lsq_status lsq_sample_rows_static(const lsq_matrix* A, const lsq_opts* o, int64_t s,
                                             int32_t* idx_out, double* p_out, double* colscale_out,
                                             int64_t* s_out, void* stream) {
    lsq_status st0 = check_matrix(A);
    if (st0 != LSQ_OK) return st0;
    LSQ_CHECK_ARG(o != nullptr, "opts is NULL");
    LSQ_CHECK_ARG(idx_out != nullptr, "idx_out is NULL");
    LSQ_CHECK_ARG(s >= 0, "s < 0");
    LSQ_CHECK_ARG(o->sampling == 0 || o->sampling == 1, "sampling must be 0 (norm squared) or 1 (uniform)");
    if (A->m > STATIC_MAX_ROWS || A->n > STATIC_MAX_COLS) {
        set_error("lsq_sample_rows_static: A has more than 262144 rows or 4096 columns, the size of "
                  "its fixed scratch; use lsq_sample_rows");
        return LSQ_ERR_INVALID;
    }
    if (s == 0) s = lsq_sample_size(A->n, o->sample_factor);
    LSQ_CHECK_ARG(s > 0 && s < (int64_t)1 << 40, "sample size out of range");
    if (s_out) *s_out = s;
    char* base = nullptr;
    lsq_status r = static_scratch_address(&base);
    if (r != LSQ_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    switch (A->dtype) {
        case LSQ_F64: return sample_into_static<LSQ_F64>(A, o, s, idx_out, p_out, colscale_out, base, st);
        case LSQ_F32: return sample_into_static<LSQ_F32>(A, o, s, idx_out, p_out, colscale_out, base, st);
        case LSQ_BF16: return sample_into_static<LSQ_BF16>(A, o, s, idx_out, p_out, colscale_out, base, st);
        case LSQ_F32X2: return sample_into_static<LSQ_F32X2>(A, o, s, idx_out, p_out, colscale_out, base, st);
    }
    set_error("unknown dtype");
    return LSQ_ERR_INVALID;
}

// ---------------------------------------------------------------------------------------
// Row-sharded sampling entry points (declared in lsq.h)
// ---------------------------------------------------------------------------------------
namespace {
template <int DT>
lsq_status shard_colmax_impl(const lsq_matrix* A, unsigned long long* amax, unsigned* err, cudaStream_t st) {
    lsq_matrix Av = *A;
    if (A->dense) {
        int64_t rpb = (A->m + 152 * 8 - 1) / (152 * 8);
        if (rpb < 16) rpb = 16;
        k_colmax_dense<DT><<<(int)((A->m + rpb - 1) / rpb), 256, 0, st>>>(Av, amax, err, rpb);
    } else {
        k_colmax_csr<DT><<<grid_for(A->nnz, 256), 256, 0, st>>>(Av, amax, err);
    }
    count_launch();
    return LSQ_OK;
}
template <int DT>
lsq_status shard_colsum_impl(const lsq_matrix* A, const int* E1j, u128* c, cudaStream_t st) {
    lsq_matrix Av = *A;
    if (A->dense) {
        int64_t rpb = (A->m + 152 * 8 - 1) / (152 * 8);
        if (rpb < 16) rpb = 16;
        k_colsum_dense<DT><<<(int)((A->m + rpb - 1) / rpb), 256, 0, st>>>(Av, E1j, c, rpb);
    } else {
        k_colsum_csr<DT><<<grid_for(A->nnz, 256), 256, 0, st>>>(Av, E1j, c);
    }
    count_launch();
    return LSQ_OK;
}
template <template <int> class F, typename... Args>
lsq_status by_dtype(int dtype, Args... args) {
    switch (dtype) {
        case LSQ_F64: return F<LSQ_F64>::run(args...);
        case LSQ_F32: return F<LSQ_F32>::run(args...);
        case LSQ_BF16: return F<LSQ_BF16>::run(args...);
        case LSQ_F32X2: return F<LSQ_F32X2>::run(args...);
    }
    set_error("unknown dtype");
    return LSQ_ERR_INVALID;
}
template <int DT> struct ColmaxF {
    static lsq_status run(const lsq_matrix* A, unsigned long long* amax, unsigned* err, cudaStream_t st) {
        return shard_colmax_impl<DT>(A, amax, err, st);
    }
};
template <int DT> struct ColsumF {
    static lsq_status run(const lsq_matrix* A, const int* E1j, u128* c, cudaStream_t st) {
        return shard_colsum_impl<DT>(A, E1j, c, st);
    }
};
template <int DT> struct WeightF {
    static lsq_status run(const lsq_matrix* A, const double* inv, u128* w, int uniform, cudaStream_t st) {
        k_rowweight<DT><<<grid_for(A->m * 32, 256), 256, 0, st>>>(*A, inv, w, uniform);
        count_launch();
        return LSQ_OK;
    }
};
void to_limbs(u128 v, int64_t* out) {
    for (int k = 0; k < 4; ++k) out[k] = (int64_t)(unsigned long long)((v >> (32 * k)) & 0xFFFFFFFFull);
}
u128 from_limbs(const int64_t* l) {
    u128 v = 0;
    for (int k = 0; k < 4; ++k) v += (u128)(unsigned long long)l[k] << (32 * k);
    return v;
}
}  // namespace

extern "C" lsq_status lsq_shard_colmax(const lsq_matrix* A, uint64_t* colmax, void* stream) {
    lsq_status st0 = check_matrix(A);
    if (st0 != LSQ_OK) return st0;
    LSQ_CHECK_ARG(colmax != nullptr, "colmax is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc;
    LSQ_CUDA(sc.alloc(16, st));
    unsigned* err = sc.as<unsigned>();
    LSQ_CUDA(cudaMemsetAsync(err, 0, 16, st));
    LSQ_CUDA(cudaMemsetAsync(colmax, 0, 8 * (size_t)A->n, st));
    lsq_status r = by_dtype<ColmaxF>(A->dtype, A, (unsigned long long*)colmax, err, st);
    if (r != LSQ_OK) return r;
    LSQ_CUDA(cudaGetLastError());
    return read_dev_error(err, st);
}

extern "C" lsq_status lsq_shard_colsum(const lsq_matrix* A, const uint64_t* colmax, int64_t* limbs, void* stream) {
    lsq_status st0 = check_matrix(A);
    if (st0 != LSQ_OK) return st0;
    LSQ_CHECK_ARG(colmax != nullptr && limbs != nullptr, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = A->n;
    Scratch sc;
    LSQ_CUDA(sc.alloc(256 + 4 * (size_t)n + 16 * (size_t)n + 256, st));
    char* base = sc.as<char>();
    unsigned* err = (unsigned*)base;
    unsigned* E1g = err + 4;
    int* E1j = (int*)(base + 256);
    u128* c = (u128*)(base + 256 + ((4 * (size_t)n + 255) & ~(size_t)255));
    LSQ_CUDA(cudaMemsetAsync(err, 0, 16, st));
    LSQ_CUDA(cudaMemsetAsync(E1g, 0xff, 4, st));
    LSQ_CUDA(cudaMemsetAsync(c, 0, 16 * (size_t)n, st));
    k_col_exponents<<<grid_for(n, 256), 256, 0, st>>>(n, (const unsigned long long*)colmax, E1j, E1g, err);
    count_launch();
    lsq_status r = by_dtype<ColsumF>(A->dtype, A, (const int*)E1j, c, st);
    if (r != LSQ_OK) return r;
    k_u128_to_limbs<<<grid_for(n, 256), 256, 0, st>>>(n, c, limbs);
    count_launch();
    LSQ_CUDA(cudaGetLastError());
    return read_dev_error(err, st);
}

extern "C" lsq_status lsq_shard_weights(const lsq_matrix* A, const lsq_opts* o, const uint64_t* colmax,
                                        const int64_t* limbs, double* colscale_out, void* prefix,
                                        int64_t* W_local_limbs, void* stream) {
    lsq_status st0 = check_matrix(A);
    if (st0 != LSQ_OK) return st0;
    LSQ_CHECK_ARG(o && colmax && limbs && colscale_out && prefix && W_local_limbs, "NULL argument");
    LSQ_CHECK_ARG(o->sampling == 0 || o->sampling == 1, "sampling must be 0 (norm squared) or 1 (uniform)");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t m = A->m, n = A->n;
    const int64_t ntiles = (m + SCAN_TILE - 1) / SCAN_TILE;
    size_t off = 0;
    auto take = [&](size_t b) { size_t at = off; off += (b + 255) & ~size_t(255); return at; };
    const size_t o_err = take(16), o_E1g = take(16), o_E1j = take(4 * n), o_c = take(16 * n),
                 o_d2 = take(8 * n), o_inv = take(8 * n), o_w = take(16 * m), o_ts = take(16 * ntiles);
    Scratch sc;
    LSQ_CUDA(sc.alloc(off, st));
    char* base = sc.as<char>();
    unsigned* err = (unsigned*)(base + o_err);
    unsigned* E1g = (unsigned*)(base + o_E1g);
    int* E1j = (int*)(base + o_E1j);
    u128* c = (u128*)(base + o_c);
    double* d2 = (double*)(base + o_d2);
    double* inv = (double*)(base + o_inv);
    u128* w = (u128*)(base + o_w);
    u128* ts = (u128*)(base + o_ts);
    u128* P = (u128*)prefix;
    LSQ_CUDA(cudaMemsetAsync(err, 0, 16, st));
    LSQ_CUDA(cudaMemsetAsync(E1g, 0xff, 4, st));
    k_col_exponents<<<grid_for(n, 256), 256, 0, st>>>(n, (const unsigned long long*)colmax, E1j, E1g, err);
    k_limbs_to_u128<<<grid_for(n, 256), 256, 0, st>>>(n, limbs, c);
    k_colscale<<<grid_for(n, 256), 256, 0, st>>>(n, o->normalize ? 1 : 0, E1j, E1g, c, d2, inv, colscale_out);
    count_launch(3);
    lsq_status r = by_dtype<WeightF>(A->dtype, A, (const double*)inv, w, o->sampling == 1 ? 1 : 0, st);
    if (r != LSQ_OK) return r;
    k_scan_tiles<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(w, m, ts);
    k_scan_sums<<<1, 1024, 0, st>>>(ts, ntiles);
    k_scan_apply<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(w, m, ts, P);
    count_launch(3);
    u128 Wr = 0;
    LSQ_CUDA(cudaMemcpyAsync(&Wr, P + m, sizeof(u128), cudaMemcpyDeviceToHost, st));
    lsq_status e = read_dev_error(err, st);   // synchronises the stream
    if (e != LSQ_OK) return e;
    to_limbs(Wr, W_local_limbs);
    return LSQ_OK;
}

extern "C" lsq_status lsq_shard_offsets(const int64_t* W_all, int32_t world, int32_t rank, int64_t* W_offset,
                                        int64_t* W_total) {
    LSQ_CHECK_ARG(W_all && W_offset && W_total, "NULL argument");
    LSQ_CHECK_ARG(world >= 1 && rank >= 0 && rank < world, "rank must lie in [0, world)");
    u128 O = 0, W = 0;
    for (int r = 0; r < world; ++r) {
        const u128 v = from_limbs(W_all + 4 * (int64_t)r);
        if (r < rank) O += v;
        W += v;
    }
    to_limbs(O, W_offset);
    to_limbs(W, W_total);
    return LSQ_OK;
}

extern "C" lsq_status lsq_shard_draw(const void* prefix, int64_t m_local, int64_t row0, const int64_t* W_offset,
                                     const int64_t* W_total, const lsq_opts* o, int64_t s, int32_t* idx_out,
                                     double* p_out, void* stream) {
    LSQ_CHECK_ARG(prefix && W_offset && W_total && o && idx_out, "NULL argument");
    LSQ_CHECK_ARG(m_local >= 1 && row0 >= 0 && row0 + m_local <= ((int64_t)1 << 31), "bad row range");
    LSQ_CHECK_ARG(s > 0 && s < (int64_t)1 << 40, "sample size out of range");
    const u128 O = from_limbs(W_offset), W = from_limbs(W_total);
    if (W == 0) { set_error("no row has positive sampling weight"); return LSQ_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    k_draw_shard<<<grid_for(s, 256), 256, 0, st>>>((const u128*)prefix, m_local, row0, (unsigned long long)O,
                                                   (unsigned long long)(O >> 64), (unsigned long long)W,
                                                   (unsigned long long)(W >> 64), s, (unsigned long long)o->seed,
                                                   idx_out, p_out);
    count_launch();
    LSQ_CUDA(cudaGetLastError());
    return LSQ_OK;
}

// The same filtered draws on the host, for a prefix held in host memory (two 64-bit words
// per entry, low word first): Philox4x64-10 (Salmon et al., SC'11), the high 128 bits of
// U W, and the search in the local prefix, as in k_draw_shard.
namespace {
void philox_host(unsigned long long c[4], unsigned long long k0, unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    for (int r = 0; r < 10; ++r) {
        const u128 p0 = (u128)M0 * c[0], p1 = (u128)M1 * c[2];
        const unsigned long long n0 = (unsigned long long)(p1 >> 64) ^ c[1] ^ k0;
        const unsigned long long n2 = (unsigned long long)(p0 >> 64) ^ c[3] ^ k1;
        c[0] = n0; c[1] = (unsigned long long)p1; c[2] = n2; c[3] = (unsigned long long)p0;
        k0 += W0; k1 += W1;
    }
}
u128 mulhi_host(u128 a, u128 b) {
    const unsigned long long a0 = (unsigned long long)a, a1 = (unsigned long long)(a >> 64);
    const unsigned long long b0 = (unsigned long long)b, b1 = (unsigned long long)(b >> 64);
    const u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1, p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
    const u128 mid = (p00 >> 64) + (unsigned long long)p01 + (unsigned long long)p10;
    return p11 + (p01 >> 64) + (p10 >> 64) + (mid >> 64);
}
}  // namespace

extern "C" lsq_status lsq_shard_draw_host(const uint64_t* prefix, int64_t m_local, int64_t row0,
                                          const int64_t* W_offset, const int64_t* W_total, uint64_t seed,
                                          int64_t t0, int64_t s, int32_t* idx_out) {
    LSQ_CHECK_ARG(prefix && W_offset && W_total && idx_out, "NULL argument");
    LSQ_CHECK_ARG(m_local >= 1 && row0 >= 0 && t0 >= 0 && s >= 0, "bad range");
    const u128 O = from_limbs(W_offset), W = from_limbs(W_total);
    LSQ_CHECK_ARG(W != 0, "no row has positive sampling weight");
    auto P = [&](int64_t i) { return ((u128)prefix[2 * i + 1] << 64) | prefix[2 * i]; };
    const u128 Wr = P(m_local);
    for (int64_t k = 0; k < s; ++k) {
        unsigned long long c[4] = {(unsigned long long)(t0 + k), 0ull, 0ull, 0ull};
        philox_host(c, seed, 0x5A4D504Cull);
        const u128 target = mulhi_host(((u128)c[1] << 64) | c[0], W);
        if (target < O || target - O >= Wr) { idx_out[k] = -1; continue; }
        const u128 local = target - O;
        int64_t lo = 0, hi = m_local;
        while (hi - lo > 1) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (P(mid) <= local) lo = mid; else hi = mid;
        }
        idx_out[k] = (int32_t)(row0 + lo);
    }
    return LSQ_OK;
}
