// Host launcher of the persistent CSR block PCG (the kernel is in sparse_persist_kernel.cuh,
// instantiated per value type in pcg_sparse_persist_f64.cu and pcg_sparse_persist_f32.cu).
#include "sparse_persist_kernel.cuh"

#include <mutex>
#include <unordered_map>

namespace lsq {

const void* persist_kernel_f64(int mt_f32, int smode, int K);
const void* persist_kernel_f32(int mt_f32, int smode, int K);

lsq_status bk_persist_launch(int dt, int mt_f32, const BkArgs& a, unsigned long long* bar, double* n2,
                             double* tmpv, double* X, int64_t ldx, BkPersistOut* out, int use_h, int res64,
                             int smode, int max_outer, cudaStream_t st) {
    const void* kern = nullptr;
    if (dt == LSQ_F64) kern = persist_kernel_f64(mt_f32, smode, a.K);
    else if (dt == LSQ_F32) kern = persist_kernel_f32(mt_f32, smode, a.K);
    else { set_error("persistent block PCG: value type"); return LSQ_ERR_UNSUPPORTED; }
    // the grid: every CTA resident (cooperative launch), computed once per kernel
    static std::mutex mu;
    static std::unordered_map<const void*, int> grids;
    int grid = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = grids.find(kern);
        if (it != grids.end()) {
            grid = it->second;
        } else {
            int dev = 0, sms = 0, per = 0;
            LSQ_CUDA(cudaGetDevice(&dev));
            LSQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            LSQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, BK_T, 0));
            if (per < 1) { set_error("persistent block PCG kernel does not fit on an SM"); return LSQ_ERR_CUDA; }
            grid = sms * per;
            grids[kern] = grid;
        }
    }
    if (grid > 152 * 16) grid = 152 * 16;   // the partial-sum buffers hold 152 * 16 blocks
    BkPersist P{};
    P.a = a;
    P.bar = bar; P.n2 = n2; P.tmpv = tmpv; P.X = X; P.ldx = ldx; P.out = out;
    P.use_h = use_h; P.res64 = res64; P.max_outer = max_outer;
    P.bar_polls = barrier_wait_polls();
    void* params[] = {&P};
    LSQ_CUDA(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(BK_T), params, 0, st));
    count_launch();
    return LSQ_OK;
}

}  // namespace lsq
