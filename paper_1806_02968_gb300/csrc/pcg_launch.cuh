// Cooperative launch of one k_pcg_dense instantiation (included by pcg_f64.cu / pcg_f32.cu).
#pragma once
#include "pcg_kernel.cuh"

namespace lsq {

constexpr int PCG_THREADS = 512;

template <int DT, int DTR, int NMAX, typename OPT>
lsq_status launch_pcg_one(PcgArgs& a, int grid_cap, cudaStream_t st, int* grid_used) {
    auto kern = k_pcg_dense<DT, DTR, NMAX, OPT>;
    const size_t smem = pcg_smem_bytes(NMAX);
    LSQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    LSQ_CUDA(cudaGetDevice(&dev));
    LSQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    LSQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PCG_THREADS, smem));
    if (per_sm < 1) { set_error("PCG kernel does not fit on an SM"); return LSQ_ERR_CUDA; }
    int G = sms * per_sm;
    if (grid_cap > 0 && G > grid_cap) G = grid_cap;
    int64_t by_rows = a.m / 16;  // at least ~16 rows per CTA
    if (by_rows < 1) by_rows = 1;
    if (G > by_rows) G = (int)by_rows;
    *grid_used = G;
    void* params[] = {&a};
    LSQ_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(G), dim3(PCG_THREADS), params, smem, st));
    count_launch();
    return LSQ_OK;
}

// Upper bound on the grid any instantiation may use (workspace sizing).
inline int pcg_max_grid() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * 8;
}

lsq_status launch_pcg_f64(int64_t nmax, int opt_dtype, PcgArgs& a, int cap, cudaStream_t st, int* G);
lsq_status launch_pcg_f32(int64_t nmax, int dtr, int opt_dtype, PcgArgs& a, int cap, cudaStream_t st, int* G);
lsq_status launch_pcg_f32x2(int64_t nmax, int dtr, int opt_dtype, PcgArgs& a, int cap, cudaStream_t st, int* G);
lsq_status launch_pcg_bf16(int64_t nmax, int dtr, int opt_dtype, PcgArgs& a, int cap, cudaStream_t st, int* G);

}  // namespace lsq
