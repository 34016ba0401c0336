// Internal helpers shared by the CUDA translation units of liblsq (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <atomic>

#include "../../include/lsq.h"


typedef unsigned __int128 u128;

namespace lsq {

// ---------------------------------------------------------------------------------------
// Host-side status plumbing
// ---------------------------------------------------------------------------------------
void set_error(const std::string& msg);
extern std::atomic<int64_t> g_launches;
inline void count_launch(int64_t k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }
// Cap on the polls of a device-side wait (lsq_set_wait_limit; 0 = the defaults below).
// Kernels receive it as an argument when they are launched.
extern std::atomic<uint32_t> g_wait_polls;
inline unsigned dep_wait_polls() {       // dependency waits of the sparse sweeps and levels
    const uint32_t v = g_wait_polls.load(std::memory_order_relaxed);
    return v ? v : (1u << 22);
}
inline unsigned barrier_wait_polls() {   // grid barriers of the persistent PCG kernel
    const uint32_t v = g_wait_polls.load(std::memory_order_relaxed);
    return v ? v : (1u << 26);
}

#define LSQ_CHECK_ARG(cond, msg)                                   \
    do {                                                           \
        if (!(cond)) {                                             \
            ::lsq::set_error(std::string("invalid argument: ") + (msg)); \
            return LSQ_ERR_INVALID;                                \
        }                                                          \
    } while (0)

#define LSQ_CUDA(call)                                                               \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            ::lsq::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));    \
            return e_ == cudaErrorMemoryAllocation ? LSQ_ERR_NOMEM : LSQ_ERR_CUDA;   \
        }                                                                            \
    } while (0)

// Device error word bits (written by kernels, read once by the host at the end of a call)
enum : unsigned {
    DEV_ERR_RANGE = 1u,      // max a_ij^2 outside [2^-900, 2^900] or non-finite input
    DEV_ERR_TIMEOUT = 2u,    // a grid barrier gave up
    DEV_ERR_BREAKDOWN = 4u,  // PCG breakdown
    DEV_ERR_EMPTY = 8u,      // W == 0: no row has sampling weight
};

inline size_t elem_size(int dtype) {
    switch (dtype) {
        case LSQ_F64: return 8;
        case LSQ_F32: return 4;
        case LSQ_BF16: return 2;
        case LSQ_F32X2: return 8;
        default: return 0;
    }
}

lsq_status check_matrix(const lsq_matrix* A);

// Stream-ordered scratch that is released on the same stream when it goes out of scope.
struct Scratch {
    void* ptr = nullptr;
    cudaStream_t st = 0;
    Scratch() = default;
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;
    cudaError_t alloc(size_t bytes, cudaStream_t s) {
        st = s;
        return cudaMallocAsync(&ptr, bytes ? bytes : 16, s);
    }
    ~Scratch() {
        if (ptr) cudaFreeAsync(ptr, st);
    }
    template <typename T> T* as() const { return reinterpret_cast<T*>(ptr); }
};

// Reads the device error word (after a stream sync) and maps it to a status.
lsq_status read_dev_error(const unsigned* d_err, cudaStream_t st, unsigned* bits_out = nullptr);

// ---------------------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void atomic_add_u128(u128* dst, u128 v) {
    unsigned long long* w = reinterpret_cast<unsigned long long*>(dst);
    unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    unsigned long long old = atomicAdd(&w[0], lo);
    unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    if (hi + carry) atomicAdd(&w[1], hi + carry);
}

// Round-to-nearest-even conversion of a 128-bit unsigned integer to double.
__device__ __forceinline__ double u128_to_double_rn(u128 x) {
    unsigned long long hi = (unsigned long long)(x >> 64), lo = (unsigned long long)x;
    if (hi == 0 && lo < (1ull << 53)) return __ull2double_rn(lo);
    int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    int sh = msb - 52;  // >= 1
    u128 mant = x >> sh;
    u128 rem = x & ((((u128)1) << sh) - 1);
    u128 half = ((u128)1) << (sh - 1);
    if (rem > half || (rem == half && (mant & 1))) mant += 1;  // may become 2^53: still exact
    double v = __ull2double_rn((unsigned long long)mant);
    // scale by 2^sh exactly (sh <= 75)
    double scale = __longlong_as_double((long long)(1023 + sh) << 52);
    return __dmul_rn(v, scale);
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned atom_add_release_u32(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long atom_add_acq_rel_u64(unsigned long long* p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of a cooperative launch on one monotonic 64-bit arrival count (zeroed
// before the launch).  Every CTA passes the same sequence of barriers and counts them in
// `epoch`; barrier number e is passed once the count reaches (e + 1) * nblocks, so the last
// CTA to arrive is released by its own arrival and the others by one load.  The top bit of
// the count is the grid's error flag (raise_grid_error): an arrival or a poll that sees it
// returns false, and callers leave the kernel.  Polls are bounded: after `max_polls` the
// barrier records DEV_ERR_TIMEOUT and returns false.
constexpr unsigned long long BAR_ERR = 1ull << 63;

__device__ __forceinline__ void raise_grid_error(unsigned* err, unsigned long long* bar, unsigned bits) {
    atomicOr(err, bits);
    atomicOr(bar, BAR_ERR);
}

__device__ __forceinline__ bool grid_barrier(unsigned long long* bar, unsigned nblocks, unsigned* err,
                                             unsigned long long& epoch, unsigned max_polls = (1u << 26)) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long target = (epoch + 1ull) * nblocks;
        unsigned long long seen = atom_add_acq_rel_u64(bar, 1ull) + 1ull;   // this CTA's writes
        unsigned polls = 0;
        int ok = 1;
        while (true) {
            if (seen & BAR_ERR) { ok = 0; break; }
            if (seen >= target) break;
            if (++polls > max_polls) {
                raise_grid_error(err, bar, DEV_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            if (polls > 64) __nanosleep(polls > 4096 ? 256 : 32);
            seen = ld_acquire_u64(bar);
        }
        s_ok = ok;
    }
    __syncthreads();
    ++epoch;
    return s_ok != 0;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace lsq

namespace lsq { struct SparseHandle; }

// Library-owned preconditioner handle (definition shared by the translation units).
struct lsq_precond {
    int64_t n = 0, s = 0;
    int32_t dense = 1;
    int32_t sweeps = 1;
    int32_t op_dtype = LSQ_F64;  // storage of the materialised operator
    int64_t nnz_M = 0, n_fixed_diag = 0, levels = 0;
    cudaStream_t stream = 0;
    double* M = nullptr;        // dense n x n FP64 (row-major)
    void* op = nullptr;         // dense n x n materialised SGS operator, op_dtype
    double* colscale = nullptr; // d_j (n)
    double* inv_d = nullptr;    // 1/d_j (n)
    lsq::SparseHandle* sp = nullptr;  // CSR matrices: sparse M, level schedules, A^T pattern
};
