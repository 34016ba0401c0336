// Double-float ("float-float") arithmetic from FP32 error-free transformations
// (Dekker 1971; Knuth's two-sum; two-product via fused multiply-add).  A value is the
// unevaluated sum hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits.  Used where
// GB300's FP32 units (64x the FP64 FMA rate) must deliver near-FP64 products and sums.
#pragma once
#include <cuda_runtime.h>

namespace lsq {

struct f2 { float hi, lo; };

// s + e = a + b exactly (Knuth two-sum, no magnitude precondition)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}
// p + e = a * b exactly (fused multiply-add residual)
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = a * b;
    e = fmaf(a, b, -p);
}
// acc += x (both double-float), renormalised
__device__ __forceinline__ void df_add(f2& acc, f2 x) {
    float s, e;
    two_sum(acc.hi, x.hi, s, e);
    e += acc.lo + x.lo;
    float hi = s + e;
    acc.lo = e - (hi - s);
    acc.hi = hi;
}
// acc += a * b for double-float a, b (the lo*lo term is below the working precision)
__device__ __forceinline__ void df_fma(f2& acc, f2 a, f2 b) {
    float p, pe;
    two_prod(a.hi, b.hi, p, pe);
    pe = fmaf(a.hi, b.lo, pe);
    pe = fmaf(a.lo, b.hi, pe);
    float s, e;
    two_sum(acc.hi, p, s, e);
    e += acc.lo + pe;
    float hi = s + e;
    acc.lo = e - (hi - s);
    acc.hi = hi;
}
// acc += a * b in the cascaded form of Ogita, Rump & Oishi's Dot2 (SIAM J. Sci. Comput.
// 26(6), 2005): the high word takes the rounded sum, the two-sum and product errors are
// summed into the low word without renormalising.  acc is then an unevaluated pair whose
// low word may exceed ulp(hi)/2; df_norm restores the normal form.  The result keeps the
// accuracy of twice the working precision.
__device__ __forceinline__ void df_fma_cascade(f2& acc, f2 a, f2 b) {
    float p, pe;
    two_prod(a.hi, b.hi, p, pe);
    pe = fmaf(a.hi, b.lo, pe);
    pe = fmaf(a.lo, b.hi, pe);
    float s, e;
    two_sum(acc.hi, p, s, e);
    acc.hi = s;
    acc.lo += e + pe;
}
// the normal form of a cascaded pair (|lo| small against |hi|: a fast two-sum suffices)
__device__ __forceinline__ f2 df_norm(f2 v) {
    const float hi = v.hi + v.lo;
    return f2{hi, v.lo - (hi - v.hi)};
}
// acc += a * a for a single float a (exact square folded into a double-float sum)
__device__ __forceinline__ void df_add_sq(f2& acc, float a) {
    float p, pe;
    two_prod(a, a, p, pe);
    float s, e;
    two_sum(acc.hi, p, s, e);
    e += acc.lo + pe;
    float hi = s + e;
    acc.lo = e - (hi - s);
    acc.hi = hi;
}
__device__ __forceinline__ f2 df_shfl_xor(f2 v, int o) {
    return f2{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ f2 df_warp_sum(f2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) df_add(v, df_shfl_xor(v, o));
    return v;
}
__device__ __forceinline__ double df_to_double(f2 v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ f2 df_from_double(double x) {
    float hi = __double2float_rn(x);
    return f2{hi, __double2float_rn(x - (double)hi)};
}

}  // namespace lsq
