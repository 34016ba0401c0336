// BF16-value instantiations of the persistent PCG kernel: values stored in BF16 and widened
// exactly to FP32, FP32 products and accumulation in the fused pass, FP64 vectors, dots and
// scalars; true residuals from FP64 values when an FP64 copy is supplied.
#include "pcg_launch.cuh"

namespace lsq {

template <int DTR, typename OPT>
static lsq_status bf16_by_n(int64_t nmax, PcgArgs& a, int cap, cudaStream_t st, int* G) {
    switch (nmax) {
        case 128: return launch_pcg_one<LSQ_BF16, DTR, 128, OPT>(a, cap, st, G);
        case 256: return launch_pcg_one<LSQ_BF16, DTR, 256, OPT>(a, cap, st, G);
        case 512: return launch_pcg_one<LSQ_BF16, DTR, 512, OPT>(a, cap, st, G);
        case 1024: return launch_pcg_one<LSQ_BF16, DTR, 1024, OPT>(a, cap, st, G);
    }
    set_error("BF16 dense PCG supports n <= 1024");
    return LSQ_ERR_UNSUPPORTED;
}

lsq_status launch_pcg_bf16(int64_t nmax, int dtr, int opt_dtype, PcgArgs& a, int cap, cudaStream_t st, int* G) {
    if (dtr == LSQ_F64)
        return opt_dtype == LSQ_F32 ? bf16_by_n<LSQ_F64, float>(nmax, a, cap, st, G)
                                    : bf16_by_n<LSQ_F64, double>(nmax, a, cap, st, G);
    return opt_dtype == LSQ_F32 ? bf16_by_n<LSQ_BF16, float>(nmax, a, cap, st, G)
                                : bf16_by_n<LSQ_BF16, double>(nmax, a, cap, st, G);
}

}  // namespace lsq
