// Device-side description of a batch of small dense problems (pcg_batch.cu).
#pragma once
#include "common.cuh"

namespace lsq {

struct BatchProb {
    int64_t m, n, npad, ld;
    const float* A;
    const void* op;        // materialised SGS operator, n x n row-major (float or double)
    int32_t op_f32;
    const double* inv_d;   // 1 / d_j
    const double* B;
    int64_t ldb;
    double* X;
    int64_t ldx;
    double* ws;            // y, g, z, p, h: 5 blocks of npad x KC doubles (row-major j*KC + c)
};

// Per problem and column, written by CTA 0 of the problem's cluster
struct BatchOut {
    int32_t iters, outer, conv, broke;
    double rec, tru, raw;
};

}  // namespace lsq
