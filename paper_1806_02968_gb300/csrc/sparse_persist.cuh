// The persistent form of the CSR block PCG (pcg_sparse_persist.cu): per-column results and
// the launcher the block solver calls.
#pragma once
#include "common.cuh"

namespace lsq {

struct BkArgs;

struct BkPersistOut {
    int32_t iters[32], outer[32], conv[32], status[32];
    double rec[32], tru[32], raw[32];
};

// One cooperative launch of the whole block solve (see pcg_sparse_persist.cu).  `a` is the
// block solver's argument set with its workspace; bar points at a zeroed 8-byte word.
lsq_status bk_persist_launch(int dt, int mt_f32, const BkArgs& a, unsigned long long* bar, double* n2,
                             double* tmpv, double* X, int64_t ldx, BkPersistOut* out, int use_h, int res64,
                             int smode, int max_outer, cudaStream_t st);

}  // namespace lsq
