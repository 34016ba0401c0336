// Scalar loads of matrix values as FP64 (exact for F64/F32/BF16; RN(hi + lo) for F32X2).
#pragma once
#include "common.cuh"

namespace lsq {

template <int DT> struct Val;
template <> struct Val<LSQ_F64> {
    typedef double T;
    static __device__ __forceinline__ double load(const void* p, int64_t e) {
        return reinterpret_cast<const double*>(p)[e];
    }
};
template <> struct Val<LSQ_F32> {
    typedef float T;
    static __device__ __forceinline__ double load(const void* p, int64_t e) {
        return (double)reinterpret_cast<const float*>(p)[e];
    }
};
template <> struct Val<LSQ_BF16> {
    typedef __nv_bfloat16 T;
    static __device__ __forceinline__ double load(const void* p, int64_t e) {
        return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[e]);
    }
};
template <> struct Val<LSQ_F32X2> {
    static __device__ __forceinline__ double load(const void* p, int64_t e) {
        const float* f = reinterpret_cast<const float*>(p);
        return __dadd_rn((double)f[2 * e], (double)f[2 * e + 1]);
    }
};

}  // namespace lsq
