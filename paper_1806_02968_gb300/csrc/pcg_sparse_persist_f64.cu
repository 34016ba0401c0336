// Instantiations of the persistent CSR block PCG kernel for F64 values (both operator
// types, every sweep form and column-block width).
#include "sparse_persist_kernel.cuh"

namespace lsq {

const void* persist_kernel_f64(int mt_f32, int smode, int K) {
    return mt_f32 ? persist_kernel<LSQ_F64, float>(smode, K) : persist_kernel<LSQ_F64, double>(smode, K);
}

}  // namespace lsq
