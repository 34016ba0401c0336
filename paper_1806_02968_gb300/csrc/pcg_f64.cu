// FP64 instantiations of the persistent PCG kernel (values, residuals and dots in FP64).
#include "pcg_launch.cuh"

namespace lsq {

template <typename OPT>
static lsq_status f64_by_n(int64_t nmax, PcgArgs& a, int cap, cudaStream_t st, int* G) {
    switch (nmax) {
        case 128: return launch_pcg_one<LSQ_F64, LSQ_F64, 128, OPT>(a, cap, st, G);
        case 256: return launch_pcg_one<LSQ_F64, LSQ_F64, 256, OPT>(a, cap, st, G);
        case 512: return launch_pcg_one<LSQ_F64, LSQ_F64, 512, OPT>(a, cap, st, G);
        case 1024: return launch_pcg_one<LSQ_F64, LSQ_F64, 1024, OPT>(a, cap, st, G);
    }
    set_error("FP64 dense PCG supports n <= 1024");
    return LSQ_ERR_UNSUPPORTED;
}

lsq_status launch_pcg_f64(int64_t nmax, int opt_dtype, PcgArgs& a, int cap, cudaStream_t st, int* G) {
    return opt_dtype == LSQ_F32 ? f64_by_n<float>(nmax, a, cap, st, G) : f64_by_n<double>(nmax, a, cap, st, G);
}

}  // namespace lsq
