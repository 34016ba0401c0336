// Sec. 3.3 for CSR matrices: the sampled normal matrix M = A_s^T A_s as a CSR SpGEMM, its
// level schedule for the Gauss-Seidel sweeps of Alg. 3, and the transposed pattern of A
// used by the A^T q pass of PCG.
//
// Everything is deterministic: the draws are compacted with integer atomics; the
// transpose of the sampled rows is sorted inside each column; every output row of the
// SpGEMM sorts its candidate products on (column, sampled row) and sums them in that fixed
// order.
#include "sparse.cuh"
#include "values.cuh"

#include <algorithm>
#include <vector>

namespace lsq {

// ---------------------------------------------------------------------------------------
// int64 exclusive scan (three passes, any length)
// ---------------------------------------------------------------------------------------
constexpr int SC_T = 512;
__device__ __forceinline__ int64_t block_excl_scan_i64(int64_t v, int64_t* total) {
    __shared__ int64_t s_w[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t y = lane < nw ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        if (lane < nw) s_w[lane] = y;
    }
    __syncthreads();
    int64_t off = wid ? s_w[wid - 1] : 0;
    if (total) *total = s_w[nw - 1];
    int64_t r = x - v + off;
    __syncthreads();
    return r;
}
__global__ void k_scan64_tiles(const int64_t* in, int64_t n, int64_t* sums) {
    int64_t i = (int64_t)blockIdx.x * SC_T + threadIdx.x;
    int64_t tot;
    block_excl_scan_i64(i < n ? in[i] : 0, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}
__global__ void k_scan64_sums(int64_t* sums, int64_t nt) {
    int64_t carry = 0;
    for (int64_t b = 0; b < nt; b += blockDim.x) {
        int64_t i = b + threadIdx.x, tot;
        int64_t e = block_excl_scan_i64(i < nt ? sums[i] : 0, &tot);
        if (i < nt) sums[i] = e + carry;
        carry += tot;
    }
}
__global__ void k_scan64_apply(const int64_t* in, int64_t n, const int64_t* offs, int64_t* out) {
    int64_t i = (int64_t)blockIdx.x * SC_T + threadIdx.x;
    int64_t tot;
    int64_t e = block_excl_scan_i64(i < n ? in[i] : 0, &tot) + offs[blockIdx.x];
    if (i < n) out[i] = e;
    if (i == n - 1) out[n] = e + in[i];
}
// out[0..n] = exclusive prefix of in[0..n) with out[n] = total; scratch: ceil(n/512) int64
lsq_status scan_i64(const int64_t* in, int64_t n, int64_t* out, int64_t* scratch, cudaStream_t st) {
    if (n == 0) { LSQ_CUDA(cudaMemsetAsync(out, 0, 8, st)); return LSQ_OK; }
    int64_t nt = (n + SC_T - 1) / SC_T;
    k_scan64_tiles<<<(unsigned)nt, SC_T, 0, st>>>(in, n, scratch);
    k_scan64_sums<<<1, 1024, 0, st>>>(scratch, nt);
    k_scan64_apply<<<(unsigned)nt, SC_T, 0, st>>>(in, n, scratch, out);
    count_launch(3);
    LSQ_CUDA(cudaGetLastError());
    return LSQ_OK;
}

// Carves one scratch allocation into 256-byte aligned pieces; the size is computed with
// the same rounding as the carving.
struct Carve {
    size_t sizes[16];
    int n = 0;
    void add(size_t bytes) { sizes[n++] = (bytes + 255) & ~size_t(255); }
    size_t total() const { size_t t = 0; for (int i = 0; i < n; ++i) t += sizes[i]; return t; }
    char* at(char* base, int i) const { size_t o = 0; for (int k = 0; k < i; ++k) o += sizes[k]; return base + o; }
};

static unsigned grid1(int64_t work, int t = 256, int64_t cap = 152 * 32) {
    int64_t g = (work + t - 1) / t;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

// ---------------------------------------------------------------------------------------
// Draw compaction: count[i] = #draws of row i, prob[i] = p_i
// ---------------------------------------------------------------------------------------
__global__ void k_count_draws(const int32_t* idx, const double* p, int64_t s, int64_t* cnt, double* prob) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < s; t += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = idx[t];
        atomicAdd((unsigned long long*)&cnt[i], 1ull);
        prob[i] = p[t];  // every draw of row i carries the same p_i
    }
}
__global__ void k_flag(const int64_t* cnt, int64_t m, int64_t* flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = cnt[i] > 0 ? 1 : 0;
}
// unique rows in increasing order, their scale gamma_u = c_u / (s p_u) and row lengths
__global__ void k_compact(const int64_t* cnt, const double* prob, const int64_t* pos, int64_t m, int64_t s,
                          const int64_t* row_ptr, int32_t* urow, double* gam, int64_t* ulen) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        if (cnt[i] > 0) {
            int64_t u = pos[i];
            urow[u] = (int32_t)i;
            gam[u] = (double)cnt[i] / ((double)s * prob[i]);
            ulen[u] = row_ptr[i + 1] - row_ptr[i];
        }
    }
}
// A_s in CSR: row u holds (j, a_{i_u j} / d_j) for the stored entries of row i_u
template <int DT>
__global__ void k_fill_As(lsq_matrix A, const int32_t* urow, int64_t nu, const int64_t* sptr,
                          const double* inv_d, int32_t* scol, double* sval) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < nu; u += nw) {
        const int64_t i = urow[u];
        const int64_t e0 = A.row_ptr[i], len = A.row_ptr[i + 1] - e0, o = sptr[u];
        for (int64_t k = lane; k < len; k += 32) {
            const int32_t j = A.col_idx[e0 + k];
            scol[o + k] = j;
            sval[o + k] = Val<DT>::load(A.vals, e0 + k) * inv_d[j];
        }
    }
}

// ---------------------------------------------------------------------------------------
// Transpose of a CSR pattern (rows nr, columns nc): column counts, then fill, then each
// column's entries sorted by row so the order is deterministic.  perm[k] = source entry.
// ---------------------------------------------------------------------------------------
__global__ void k_col_count(const int32_t* col, int64_t nnz, int64_t* ccnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd((unsigned long long*)&ccnt[col[e]], 1ull);
}
__global__ void k_col_fill(const int64_t* rptr, const int32_t* col, int64_t nr, const int64_t* cptr,
                           int64_t* cfill, int32_t* trow, int64_t* tperm) {
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < nr; r += nw) {
        for (int64_t e = rptr[r] + lane; e < rptr[r + 1]; e += 32) {
            int32_t c = col[e];
            int64_t at = cptr[c] + (int64_t)atomicAdd((unsigned long long*)&cfill[c], 1ull);
            trow[at] = (int32_t)r;
            tperm[at] = e;
        }
    }
}
constexpr int SPG_CAP = 8192;   // candidates per output row (dynamic shared memory)
constexpr int SPG_T = 256;

// exclusive scan of one int per thread over the block; *total = block sum
__device__ __forceinline__ int block_excl_scan_int(int v, int* total) {
    __shared__ int s_w[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int y = lane < nw ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        if (lane < nw) s_w[lane] = y;
    }
    __syncthreads();
    const int off = wid ? s_w[wid - 1] : 0;
    *total = s_w[nw - 1];
    const int r = x - v + off;
    __syncthreads();
    return r;
}

// bitonic sort of s_key[0..P2) ascending, carrying one payload array (P2 a power of two)
template <typename V>
__device__ __forceinline__ void block_bitonic(unsigned long long* s_key, V* s_val, int P2) {
    for (int size = 2; size <= P2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P2; i += blockDim.x) {
                const int pj = i ^ stride;
                if (pj > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long a = s_key[i], b = s_key[pj];
                    if ((a > b) == up) {
                        s_key[i] = b; s_key[pj] = a;
                        const V t = s_val[i]; s_val[i] = s_val[pj]; s_val[pj] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// sort each column segment by row: one CTA per column; a bitonic sort in shared memory on
// (row, position) keys for segments up to 8192 entries, a serial insertion sort beyond
constexpr int CS_CAP = 8192;    // entries per column sorted in shared memory
__global__ void __launch_bounds__(256) k_col_sort(const int64_t* cptr, int64_t nc, int32_t* trow, int64_t* tperm) {
    extern __shared__ __align__(16) unsigned long long cs_smem[];
    unsigned long long* s_key = cs_smem;
    int64_t* s_perm = reinterpret_cast<int64_t*>(cs_smem + CS_CAP);
    for (int64_t c = blockIdx.x; c < nc; c += gridDim.x) {
        const int64_t a = cptr[c], b = cptr[c + 1];
        const int64_t len = b - a;
        if (len <= 1) continue;
        if (len <= CS_CAP) {
            int P2 = 1;
            while (P2 < len) P2 <<= 1;
            for (int i = threadIdx.x; i < P2; i += blockDim.x) {
                if (i < len) { s_key[i] = ((unsigned long long)(unsigned)trow[a + i] << 32) | (unsigned)i; s_perm[i] = tperm[a + i]; }
                else { s_key[i] = ~0ull; s_perm[i] = 0; }
            }
            __syncthreads();
            block_bitonic(s_key, s_perm, P2);
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                trow[a + i] = (int32_t)(s_key[i] >> 32);
                tperm[a + i] = s_perm[i];
            }
            __syncthreads();
        } else if (threadIdx.x == 0) {
            for (int64_t x = a + 1; x < b; ++x) {
                int32_t r = trow[x];
                int64_t pm = tperm[x];
                int64_t y = x - 1;
                while (y >= a && trow[y] > r) { trow[y + 1] = trow[y]; tperm[y + 1] = tperm[y]; --y; }
                trow[y + 1] = r;
                tperm[y + 1] = pm;
            }
        }
    }
}

lsq_status transpose_pattern(const int64_t* rptr, const int32_t* col, int64_t nr, int64_t nc, int64_t nnz,
                             int64_t* cptr, int32_t* trow, int64_t* tperm, cudaStream_t st) {
    Scratch sc;
    int64_t nt = (nc + SC_T - 1) / SC_T + 1;
    LSQ_CUDA(sc.alloc(8 * (size_t)(2 * nc + nt + 4), st));
    int64_t* ccnt = sc.as<int64_t>();
    int64_t* cfill = ccnt + nc;
    int64_t* ts = cfill + nc;
    LSQ_CUDA(cudaMemsetAsync(ccnt, 0, 16 * (size_t)nc, st));
    k_col_count<<<grid1(nnz), 256, 0, st>>>(col, nnz, ccnt);
    count_launch();
    lsq_status s = scan_i64(ccnt, nc, cptr, ts, st);
    if (s != LSQ_OK) return s;
    k_col_fill<<<grid1(nr * 32), 256, 0, st>>>(rptr, col, nr, cptr, cfill, trow, tperm);
    const int cs_smem = CS_CAP * 16;
    LSQ_CUDA(cudaFuncSetAttribute(k_col_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, cs_smem));
    k_col_sort<<<(unsigned)std::min<int64_t>(nc, 152 * 4), 256, cs_smem, st>>>(cptr, nc, trow, tperm);
    count_launch(2);
    LSQ_CUDA(cudaGetLastError());
    return LSQ_OK;
}

// ---------------------------------------------------------------------------------------
// SpGEMM M = A_s^T diag(gamma) A_s, one CTA per output row j:
//   candidates (k, u, gamma_u a_uj a_uk) for every sampled row u with an entry in column j
//   and every entry k of that row; bitonic sort on (k, u); segmented sums in that order.
// Pass 0 counts the distinct k (plus the diagonal if absent); pass 1 writes the row.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(SPG_T) k_spgemm_row(
    int pass, int64_t n, const int64_t* sptr, const int32_t* scol, const double* sval,
    const double* gam, const int64_t* tptr, const int32_t* trow, const int64_t* tperm,
    int64_t* mcnt, const int64_t* mptr, int32_t* mcol, double* mval,
    unsigned long long* n_fixed, unsigned* err) {
    extern __shared__ __align__(16) unsigned long long spg_smem[];
    unsigned long long* s_key = spg_smem;
    double* s_val = reinterpret_cast<double*>(spg_smem + SPG_CAP);
    __shared__ int s_cnt;
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        // gather candidates: thread t takes sampled rows q = tptr[j] + t, t + T, ...; the
        // offset of each row's products is an exclusive scan of the row lengths
        const int64_t q0 = tptr[j], q1 = tptr[j + 1];
        int carry = 0;
        for (int64_t qb = q0; qb < q1; qb += blockDim.x) {
            const int64_t q = qb + threadIdx.x;
            int len = 0, u = 0;
            double cuj = 0.0;
            int64_t e0 = 0;
            if (q < q1) {
                u = trow[q];
                cuj = gam[u] * sval[tperm[q]];
                e0 = sptr[u];
                len = (int)(sptr[u + 1] - e0);
            }
            int tot;
            const int off = block_excl_scan_int(len, &tot) + carry;
            for (int k = 0; k < len; ++k) {
                const int at = off + k;
                if (at < SPG_CAP) {
                    s_key[at] = ((unsigned long long)(unsigned)scol[e0 + k] << 32) | (unsigned)u;
                    s_val[at] = cuj * sval[e0 + k];
                }
            }
            carry += tot;
        }
        __syncthreads();
        int cnt = carry;
        if (cnt > SPG_CAP) {
            if (threadIdx.x == 0) atomicOr(err, 16u);
            cnt = SPG_CAP;
        }
        // bitonic sort of the candidates (padded to a power of two with +inf keys)
        int P2 = 1;
        while (P2 < cnt) P2 <<= 1;
        for (int i = cnt + threadIdx.x; i < P2; i += blockDim.x) { s_key[i] = ~0ull; s_val[i] = 0.0; }
        __syncthreads();
        block_bitonic(s_key, s_val, P2);
        // distinct columns: heads of runs of equal k
        if (pass == 0) {
            if (threadIdx.x == 0) s_cnt = 0;
            __syncthreads();
            int mine = 0, has_diag = 0;
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                const unsigned k = (unsigned)(s_key[i] >> 32);
                if (i == 0 || (unsigned)(s_key[i - 1] >> 32) != k) {
                    ++mine;
                    if ((int64_t)k == j) has_diag = 1;
                }
            }
            atomicAdd(&s_cnt, mine + 0);
            if (has_diag) atomicAdd(&s_cnt, 1 << 20);
            __syncthreads();
            if (threadIdx.x == 0) {
                const int c = s_cnt & ((1 << 20) - 1);
                const int d = s_cnt >> 20;
                mcnt[j] = c + (d ? 0 : 1);
            }
            __syncthreads();
        } else {
            // one thread walks the sorted list (fixed order), inserting the diagonal
            if (threadIdx.x == 0) {
                int64_t o = mptr[j];
                bool diag_done = false;
                int i = 0;
                while (i < cnt) {
                    const unsigned k = (unsigned)(s_key[i] >> 32);
                    if (!diag_done && (int64_t)k > j) {
                        mcol[o] = (int32_t)j; mval[o] = 1.0; ++o;
                        atomicAdd(n_fixed, 1ull);
                        diag_done = true;
                    }
                    double sum = 0.0;
                    while (i < cnt && (unsigned)(s_key[i] >> 32) == k) { sum += s_val[i]; ++i; }
                    if ((int64_t)k == j) {
                        diag_done = true;
                        if (sum == 0.0) { sum = 1.0; atomicAdd(n_fixed, 1ull); }
                    }
                    mcol[o] = (int32_t)k; mval[o] = sum; ++o;
                }
                if (!diag_done) { mcol[o] = (int32_t)j; mval[o] = 1.0; atomicAdd(n_fixed, 1ull); }
            }
            __syncthreads();
        }
    }
}

// diagonal inverse of M (the diagonal is always stored)
__global__ void k_diag_inv(const int64_t* mptr, const int32_t* mcol, const double* mval, int64_t n, double* dinv,
                           int64_t* mdiag) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double v = 1.0;
        int64_t at = mptr[j];
        for (int64_t e = mptr[j]; e < mptr[j + 1]; ++e)
            if (mcol[e] == j) { v = mval[e]; at = e; break; }
        dinv[j] = 1.0 / v;
        mdiag[j] = at;
    }
}
__global__ void k_to_f32(const double* src, float* dst, int64_t count) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        dst[e] = (float)src[e];
}

// Level schedules: lev_f(j) = 1 + max lev_f(k) over k < j with M_jk != 0 (rows in natural
// order), lev_b(j) = 1 + max lev_b(k) over k > j (reverse order), 0 for a row without such
// entries.  Each schedule lists the rows by level (any order inside a level: those rows are
// independent) with the level of every slot and the number of rows of every level.
//
// k_levels: cooperative launch; warp w takes rows w, w + W, ... in dependency order (natural
// order forward, reverse backward), so every row a row depends on is taken by a warp no later
// than the row itself and, every warp being resident, every wait ends.  lev1 holds level + 1
// (0 = not yet known).  Waits are bounded; one failed wait sets *err and ends them all.
__device__ __forceinline__ int ld_acquire_i32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_i32(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
template <bool FWD>
__global__ void __launch_bounds__(256) k_levels(int64_t n, const int64_t* mptr, const int32_t* mcol,
                                                const int64_t* mdiag, int* lev1, int* maxlev, unsigned* err,
                                                unsigned max_polls) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int mymax = 0;
    for (int64_t t = gw; t < n; t += W) {
        const int64_t j = FWD ? t : n - 1 - t;
        const int64_t d0 = FWD ? mptr[j] : mdiag[j] + 1, d1 = FWD ? mdiag[j] : mptr[j + 1];
        int mx = 0;
        // the dependencies in batches of 8 per lane: all loads of a batch are issued
        // together, then only the ones not known yet are polled again
        for (int64_t base = d0 + lane; base < d1; base += 32 * 8) {
            int32_t kk[8];
            int v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) kk[u] = base + 32 * u < d1 ? mcol[base + 32 * u] : -1;
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = kk[u] >= 0 ? ld_acquire_i32(lev1 + kk[u]) : 1;
            unsigned polls = 0, ns = 32;
            while (true) {
                bool missing = false;
#pragma unroll
                for (int u = 0; u < 8; ++u) missing = missing || v[u] == 0;
                if (!missing) break;
                ++polls;
                if (polls > max_polls || ((polls & 255u) == 0 && *(volatile unsigned*)err != 0u)) {
                    atomicOr(err, DEV_ERR_TIMEOUT);
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[u] = max(v[u], 1);
                    break;
                }
                if (polls > 4) { __nanosleep(ns); ns = ns < 256 ? 2 * ns : 256; }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (v[u] == 0) v[u] = ld_acquire_i32(lev1 + kk[u]);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) mx = max(mx, v[u]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) st_release_i32(lev1 + j, mx + 1);   // level(j) = mx, stored + 1
        mymax = max(mymax, mx);
    }
    if (lane == 0) atomicMax(maxlev, mymax);
}
// rows per level, from lev1 (level + 1)
__global__ void k_level_count(int64_t n, const int* lev1, unsigned long long* cnt) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + (lev1[j] - 1), 1ull);
}
// slot of every row: its level's offset plus a cursor (order inside a level is free)
__global__ void k_level_scatter(int64_t n, const int* lev1, const int64_t* off, unsigned long long* cur,
                                int32_t* sched) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int l = lev1[j] - 1;
        const int64_t at = off[l] + (int64_t)atomicAdd(cur + l, 1ull);
        sched[at] = (int32_t)j;
    }
}

// One direction's schedule on the device: sched (n rows, level by level), loff (levels + 1
// offsets into sched), nlev.
template <bool FWD>
static lsq_status device_levels(const SparseHandle* S, int64_t n, int32_t** sched, int64_t** loff, int64_t* nlev,
                                cudaStream_t st) {
    int dev = 0, sms = 0, per = 0;
    LSQ_CUDA(cudaGetDevice(&dev));
    LSQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LSQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_levels<FWD>, 256, 0));
    if (per < 1) { set_error("level kernel does not fit on an SM"); return LSQ_ERR_CUDA; }
    Scratch sc;
    LSQ_CUDA(sc.alloc(4 * (size_t)n + 256, st));
    int* lev1 = sc.as<int>();
    int* maxlev = lev1 + n;
    unsigned* err = reinterpret_cast<unsigned*>(maxlev + 1);
    LSQ_CUDA(cudaMemsetAsync(lev1, 0, 4 * (size_t)n + 256, st));
    int64_t nn = n;
    const int64_t* mptr = S->mptr;
    const int32_t* mcol = S->mcol;
    const int64_t* mdiag = S->mdiag;
    unsigned max_polls = dep_wait_polls();
    void* params[] = {&nn, (void*)&mptr, (void*)&mcol, (void*)&mdiag, &lev1, &maxlev, &err, &max_polls};
    LSQ_CUDA(cudaLaunchCooperativeKernel((const void*)k_levels<FWD>, dim3(sms * per), dim3(256), params, 0, st));
    count_launch();
    int hmax[2] = {0, 0};
    LSQ_CUDA(cudaMemcpyAsync(hmax, maxlev, 8, cudaMemcpyDeviceToHost, st));
    LSQ_CUDA(cudaStreamSynchronize(st));
    if (hmax[1] != 0) { set_error("level schedule: a dependency wait timed out"); return LSQ_ERR_TIMEOUT; }
    const int64_t L = (int64_t)hmax[0] + 1;
    LSQ_CUDA(cudaMalloc(sched, 4 * (size_t)n));
    Scratch sc2;
    const int64_t nt = (L + SC_T - 1) / SC_T;   // scan_i64: out[0..L], ceil(L / 512) scratch
    LSQ_CUDA(sc2.alloc(8 * (size_t)(L + (L + 1) + L + nt + 1), st));
    int64_t* lsize = sc2.as<int64_t>();         // rows per level
    int64_t* off = lsize + L;
    unsigned long long* cur = reinterpret_cast<unsigned long long*>(off + L + 1);
    int64_t* scan_scratch = off + (L + 1) + L;
    LSQ_CUDA(cudaMemsetAsync(lsize, 0, 8 * (size_t)L, st));
    LSQ_CUDA(cudaMemsetAsync(cur, 0, 8 * (size_t)L, st));
    k_level_count<<<grid1(n), 256, 0, st>>>(n, lev1, reinterpret_cast<unsigned long long*>(lsize));
    count_launch();
    lsq_status r = scan_i64(lsize, L, off, scan_scratch, st);
    if (r != LSQ_OK) return r;
    k_level_scatter<<<grid1(n), 256, 0, st>>>(n, lev1, off, cur, *sched);
    count_launch();
    LSQ_CUDA(cudaMalloc(loff, 8 * (size_t)(L + 1)));
    LSQ_CUDA(cudaMemcpyAsync(*loff, off, 8 * (size_t)(L + 1), cudaMemcpyDeviceToDevice, st));
    LSQ_CUDA(cudaGetLastError());
    LSQ_CUDA(cudaStreamSynchronize(st));
    *nlev = L;
    return LSQ_OK;
}

lsq_status build_sparse(const lsq_matrix* A, const int32_t* idx, const double* p, int64_t s,
                        lsq_precond* H, cudaStream_t st) {
    const int64_t m = A->m, n = A->n;
    SparseHandle* S = new SparseHandle();
    H->sp = S;
    // 1. compaction
    Scratch sc1;
    const int64_t ntm = (m + SC_T - 1) / SC_T + 1;
    Carve c1;
    c1.add(8 * (size_t)m); c1.add(8 * (size_t)m); c1.add(8 * (size_t)m); c1.add(8 * (size_t)(m + 1));
    c1.add(8 * (size_t)ntm);
    LSQ_CUDA(sc1.alloc(c1.total(), st));
    int64_t* cnt = (int64_t*)c1.at(sc1.as<char>(), 0);
    double* prob = (double*)c1.at(sc1.as<char>(), 1);
    int64_t* flag = (int64_t*)c1.at(sc1.as<char>(), 2);
    int64_t* pos = (int64_t*)c1.at(sc1.as<char>(), 3);   // m + 1
    int64_t* ts = (int64_t*)c1.at(sc1.as<char>(), 4);
    LSQ_CUDA(cudaMemsetAsync(cnt, 0, 8 * (size_t)m, st));
    k_count_draws<<<grid1(s), 256, 0, st>>>(idx, p, s, cnt, prob);
    k_flag<<<grid1(m), 256, 0, st>>>(cnt, m, flag);
    count_launch(2);
    lsq_status r = scan_i64(flag, m, pos, ts, st);
    if (r != LSQ_OK) return r;
    int64_t nu = 0;
    LSQ_CUDA(cudaMemcpyAsync(&nu, pos + m, 8, cudaMemcpyDeviceToHost, st));
    LSQ_CUDA(cudaStreamSynchronize(st));
    Scratch sc2;
    const int64_t ntu = (nu + SC_T - 1) / SC_T + 1;
    Carve c2;
    c2.add(4 * (size_t)nu); c2.add(8 * (size_t)nu); c2.add(8 * (size_t)nu); c2.add(8 * (size_t)(nu + 1));
    c2.add(8 * (size_t)ntu);
    LSQ_CUDA(sc2.alloc(c2.total(), st));
    int32_t* urow = (int32_t*)c2.at(sc2.as<char>(), 0);
    double* gam = (double*)c2.at(sc2.as<char>(), 1);
    int64_t* ulen = (int64_t*)c2.at(sc2.as<char>(), 2);
    int64_t* sptr = (int64_t*)c2.at(sc2.as<char>(), 3);   // nu + 1
    int64_t* ts2 = (int64_t*)c2.at(sc2.as<char>(), 4);
    k_compact<<<grid1(m), 256, 0, st>>>(cnt, prob, pos, m, s, A->row_ptr, urow, gam, ulen);
    count_launch();
    r = scan_i64(ulen, nu, sptr, ts2, st);
    if (r != LSQ_OK) return r;
    int64_t snnz = 0;
    LSQ_CUDA(cudaMemcpyAsync(&snnz, sptr + nu, 8, cudaMemcpyDeviceToHost, st));
    LSQ_CUDA(cudaStreamSynchronize(st));
    // 2. A_s and its transpose
    Scratch sc3;
    Carve c3;
    c3.add(4 * (size_t)snnz); c3.add(8 * (size_t)snnz); c3.add(8 * (size_t)(n + 1));
    c3.add(4 * (size_t)snnz); c3.add(8 * (size_t)snnz);
    LSQ_CUDA(sc3.alloc(c3.total(), st));
    int32_t* scol = (int32_t*)c3.at(sc3.as<char>(), 0);
    double* sval = (double*)c3.at(sc3.as<char>(), 1);
    int64_t* tptr = (int64_t*)c3.at(sc3.as<char>(), 2);
    int32_t* trow = (int32_t*)c3.at(sc3.as<char>(), 3);
    int64_t* tperm = (int64_t*)c3.at(sc3.as<char>(), 4);
    switch (A->dtype) {
        case LSQ_F64: k_fill_As<LSQ_F64><<<grid1(nu * 32), 256, 0, st>>>(*A, urow, nu, sptr, H->inv_d, scol, sval); break;
        case LSQ_F32: k_fill_As<LSQ_F32><<<grid1(nu * 32), 256, 0, st>>>(*A, urow, nu, sptr, H->inv_d, scol, sval); break;
        case LSQ_BF16: k_fill_As<LSQ_BF16><<<grid1(nu * 32), 256, 0, st>>>(*A, urow, nu, sptr, H->inv_d, scol, sval); break;
        default: k_fill_As<LSQ_F32X2><<<grid1(nu * 32), 256, 0, st>>>(*A, urow, nu, sptr, H->inv_d, scol, sval); break;
    }
    count_launch();
    r = transpose_pattern(sptr, scol, nu, n, snnz, tptr, trow, tperm, st);
    if (r != LSQ_OK) return r;
    // 3. SpGEMM: counts, row pointers, values
    Scratch sc4;
    int64_t ntn = (n + SC_T - 1) / SC_T + 1;
    LSQ_CUDA(sc4.alloc(8 * (size_t)(n + 16 + ntn), st));
    int64_t* mcnt = sc4.as<int64_t>();
    unsigned long long* nfix = reinterpret_cast<unsigned long long*>(mcnt + n);
    unsigned* err = reinterpret_cast<unsigned*>(nfix + 1);
    int64_t* ts4 = mcnt + n + 16;
    LSQ_CUDA(cudaMemsetAsync(nfix, 0, 16, st));
    LSQ_CUDA(cudaMalloc(&S->mptr, 8 * (size_t)(n + 1)));
    unsigned gs = (unsigned)std::min<int64_t>(n, 152 * 4);
    const int spg_smem = SPG_CAP * 16;
    LSQ_CUDA(cudaFuncSetAttribute(k_spgemm_row, cudaFuncAttributeMaxDynamicSharedMemorySize, spg_smem));
    k_spgemm_row<<<gs, SPG_T, spg_smem, st>>>(0, n, sptr, scol, sval, gam, tptr, trow, tperm, mcnt, nullptr,
                                       nullptr, nullptr, nfix, err);
    count_launch();
    r = scan_i64(mcnt, n, S->mptr, ts4, st);
    if (r != LSQ_OK) return r;
    int64_t mnnz = 0;
    unsigned errbits = 0;
    LSQ_CUDA(cudaMemcpyAsync(&mnnz, S->mptr + n, 8, cudaMemcpyDeviceToHost, st));
    LSQ_CUDA(cudaMemcpyAsync(&errbits, err, 4, cudaMemcpyDeviceToHost, st));
    LSQ_CUDA(cudaStreamSynchronize(st));
    if (errbits & 16u) {
        set_error("a row of A_s^T A_s has more than 8192 candidate products (unsupported in this build)");
        return LSQ_ERR_UNSUPPORTED;
    }
    LSQ_CUDA(cudaMalloc(&S->mcol, 4 * (size_t)mnnz));
    LSQ_CUDA(cudaMalloc(&S->mval, 8 * (size_t)mnnz));
    k_spgemm_row<<<gs, SPG_T, spg_smem, st>>>(1, n, sptr, scol, sval, gam, tptr, trow, tperm, nullptr, S->mptr,
                                       S->mcol, S->mval, nfix, err);
    count_launch();
    LSQ_CUDA(cudaMalloc(&S->dinv, 8 * (size_t)n));
    LSQ_CUDA(cudaMalloc(&S->mdiag, 8 * (size_t)n));
    k_diag_inv<<<grid1(n), 256, 0, st>>>(S->mptr, S->mcol, S->mval, n, S->dinv, S->mdiag);
    count_launch();
    if (H->op_dtype == LSQ_F32) {
        LSQ_CUDA(cudaMalloc(&S->mval32, 4 * (size_t)mnnz));
        k_to_f32<<<grid1(mnnz), 256, 0, st>>>(S->mval, S->mval32, mnnz);
        count_launch();
    }
    unsigned long long nf = 0;
    LSQ_CUDA(cudaMemcpyAsync(&nf, nfix, 8, cudaMemcpyDeviceToHost, st));
    LSQ_CUDA(cudaGetLastError());
    LSQ_CUDA(cudaStreamSynchronize(st));
    // 4. level schedules of the forward and backward sweeps (device)
    r = device_levels<true>(S, n, &S->sched_f, &S->loff_f, &S->nlev_f, st);
    if (r != LSQ_OK) return r;
    r = device_levels<false>(S, n, &S->sched_b, &S->loff_b, &S->nlev_b, st);
    if (r != LSQ_OK) return r;
    // 5. transposed pattern of A for the A^T q pass (values are gathered at solve time)
    LSQ_CUDA(cudaMalloc(&S->atptr, 8 * (size_t)(n + 1)));
    LSQ_CUDA(cudaMalloc(&S->atrow, 4 * (size_t)A->nnz));
    LSQ_CUDA(cudaMalloc(&S->atperm, 8 * (size_t)A->nnz));
    r = transpose_pattern(A->row_ptr, A->col_idx, m, n, A->nnz, S->atptr, S->atrow, S->atperm, st);
    if (r != LSQ_OK) return r;
    LSQ_CUDA(cudaStreamSynchronize(st));
    S->nnz_A = A->nnz;
    S->m = m;
    H->n_fixed_diag = (int64_t)nf;
    H->nnz_M = mnnz;
    H->levels = S->nlev_f;
    S->nnz_M = mnnz;
    S->n_unique = nu;
    return LSQ_OK;
}

void free_sparse(SparseHandle* S) {
    if (!S) return;
    cudaFree(S->mptr); cudaFree(S->mcol); cudaFree(S->mval); cudaFree(S->mval32); cudaFree(S->dinv); cudaFree(S->mdiag);
    cudaFree(S->sched_f); cudaFree(S->sched_b);
    cudaFree(S->atptr); cudaFree(S->atrow);
    cudaFree(S->atperm); cudaFree(S->loff_f); cudaFree(S->loff_b);
    delete S;
}

}  // namespace lsq
