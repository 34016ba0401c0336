// Latency figures of the device, for the latency bound of the level-ordered Gauss-Seidel sweeps
// of Alg. 3 (a sweep is a chain of levels: each level hands values written on one SM to rows
// computed on another).  Four bounded probes, each a single launch:
//   k_lat_chase   one thread follows a pseudo-random cycle through a 64 MB buffer (L2): the
//                 time of one dependent load;
//   k_lat_flag    two CTAs (one cooperative launch, so both are resident) hand a counter back
//                 and forth through global memory: the round trip of a value between two SMs,
//                 without and with a fence before each store;
//   k_lat_clbar   8 CTAs of one cluster pass cluster barriers: the time of one barrier;
//   k_lat_dsmem   one thread of CTA 0 follows a cycle through CTA 1's shared memory: the time
//                 of one dependent load from another CTA of the cluster.
// Every loop has a fixed trip count and every wait a poll limit.
#include "common.cuh"

#include <cooperative_groups.h>

namespace lsq {

namespace {

constexpr unsigned LAT_LINES = 1u << 19;      // 128-byte lines: 64 MB
constexpr unsigned LAT_LINE_WORDS = 32;
constexpr int LAT_HOPS = 20000;
constexpr int LAT_ROUNDS = 20000;
constexpr unsigned LAT_SMEM_WORDS = 4096;

__device__ __forceinline__ unsigned long long lat_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// next[line] = a full-period LCG step over the lines (a = 5 mod 8 multiplier, odd increment),
// so the chase visits every line once per cycle in a scattered order
__global__ void k_lat_init(unsigned* buf) {
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < LAT_LINES; i += gridDim.x * blockDim.x)
        buf[(size_t)i * LAT_LINE_WORDS] = ((i * 1103515245u + 12345u) & (LAT_LINES - 1u)) * LAT_LINE_WORDS;
}

__global__ void k_lat_chase(const unsigned* buf, int hops, unsigned* sink, unsigned long long* ns) {
    unsigned i = 0;
    const unsigned long long t0 = lat_now();
    for (int h = 0; h < hops; ++h) i = __ldcg(buf + i);
    const unsigned long long t1 = lat_now();
    sink[0] = i;
    ns[0] = t1 - t0;
}

// CTA 0 waits for even values and writes the next odd one, CTA 1 the reverse.  fenced = 0:
// plain volatile loads and stores, the value being the flag, as in the sweeps' hand-offs;
// fenced = 1: a fence before each store, as a hand-off that publishes other data needs.
__global__ void k_lat_flag(unsigned* flag, int rounds, int fenced, unsigned* err, unsigned long long* ns) {
    if (threadIdx.x != 0) return;
    volatile unsigned* f = flag;
    const unsigned long long t0 = lat_now();
    for (int r = 0; r < rounds; ++r) {
        const unsigned want = 2u * (unsigned)r + blockIdx.x;
        unsigned polls = 0;
        while (*f != want) {
            if (++polls > (1u << 24)) { atomicOr(err, 1u); return; }
        }
        if (fenced) __threadfence();
        *f = want + 1u;
    }
    const unsigned long long t1 = lat_now();
    if (blockIdx.x == 0) ns[fenced ? 4 : 1] = t1 - t0;
}

__global__ void k_lat_clbar(int rounds, unsigned long long* ns) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    const unsigned long long t0 = lat_now();
    for (int r = 0; r < rounds; ++r) cl.sync();
    const unsigned long long t1 = lat_now();
    if (cl.block_rank() == 0 && threadIdx.x == 0) ns[2] = t1 - t0;
}

__global__ void k_lat_dsmem(int hops, unsigned* sink, unsigned long long* ns) {
    namespace cg = cooperative_groups;
    __shared__ unsigned nxt[LAT_SMEM_WORDS];
    cg::cluster_group cl = cg::this_cluster();
    for (unsigned i = threadIdx.x; i < LAT_SMEM_WORDS; i += blockDim.x)
        nxt[i] = (i * 1103515245u + 12345u) & (LAT_SMEM_WORDS - 1u);
    cl.sync();
    if (cl.block_rank() == 0 && threadIdx.x == 0) {
        const unsigned* remote = cl.map_shared_rank(nxt, 1);
        unsigned i = 0;
        const unsigned long long t0 = lat_now();
        for (int h = 0; h < hops; ++h) i = remote[i];
        const unsigned long long t1 = lat_now();
        sink[1] = i;
        ns[3] = t1 - t0;
    }
    cl.sync();   // CTA 1's shared memory stays alive until the chase is over
}

template <typename K, typename... Args>
cudaError_t lat_cluster_launch(K kern, int C, int threads, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(threads);
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace

}  // namespace lsq

using namespace lsq;

extern "C" lsq_status lsq_measure_latency(double* out_ns, void* stream) {
    LSQ_CHECK_ARG(out_ns != nullptr, "out_ns is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned* buf = nullptr;
    unsigned long long* dev = nullptr;
    LSQ_CUDA(cudaMalloc(&buf, (size_t)LAT_LINES * LAT_LINE_WORDS * sizeof(unsigned)));
    const size_t small = 5 * sizeof(unsigned long long) + 4 * sizeof(unsigned) + 64;
    if (cudaMalloc(&dev, small) != cudaSuccess) {
        cudaFree(buf);
        set_error("lsq_measure_latency: cudaMalloc failed");
        return LSQ_ERR_NOMEM;
    }
    unsigned long long* ns = dev;
    unsigned* flag = reinterpret_cast<unsigned*>(dev + 5);
    unsigned* err = flag + 1;
    unsigned* sink = flag + 2;
    lsq_status status = LSQ_OK;
    unsigned long long h_ns[5] = {0, 0, 0, 0, 0};
    unsigned h_err = 0;
    auto step = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && status == LSQ_OK) {
            set_error(std::string("lsq_measure_latency: ") + what + ": " + cudaGetErrorString(e));
            status = LSQ_ERR_CUDA;
        }
    };
    step(cudaMemsetAsync(dev, 0, small, st), "memset");
    k_lat_init<<<512, 256, 0, st>>>(buf);
    k_lat_chase<<<1, 1, 0, st>>>(buf, LAT_HOPS, sink, ns);   // brings the lines into L2
    k_lat_chase<<<1, 1, 0, st>>>(buf, LAT_HOPS, sink, ns);
    count_launch(3);
    step(cudaGetLastError(), "chase");
    for (int fenced = 0; fenced < 2; ++fenced) {
        int rounds = LAT_ROUNDS;
        step(cudaMemsetAsync(flag, 0, sizeof(unsigned), st), "memset");
        void* params[] = {&flag, &rounds, &fenced, &err, &ns};
        step(cudaLaunchCooperativeKernel((const void*)k_lat_flag, dim3(2), dim3(32), params, 0, st), "flag");
        count_launch();
    }
    step(lat_cluster_launch(k_lat_clbar, 8, 256, st, (int)LAT_ROUNDS, ns), "cluster barrier");
    step(lat_cluster_launch(k_lat_dsmem, 2, 256, st, (int)LAT_HOPS, sink, ns), "dsmem");
    count_launch(2);
    step(cudaMemcpyAsync(h_ns, ns, sizeof(h_ns), cudaMemcpyDeviceToHost, st), "copy");
    step(cudaMemcpyAsync(&h_err, err, sizeof(h_err), cudaMemcpyDeviceToHost, st), "copy");
    step(cudaStreamSynchronize(st), "synchronise");
    cudaFree(buf);
    cudaFree(dev);
    if (status != LSQ_OK) return status;
    if (h_err) {
        set_error("lsq_measure_latency: the flag hand-off ran out of polls");
        return LSQ_ERR_TIMEOUT;
    }
    out_ns[0] = (double)h_ns[0] / LAT_HOPS;
    out_ns[1] = (double)h_ns[1] / LAT_ROUNDS;
    out_ns[2] = (double)h_ns[2] / LAT_ROUNDS;
    out_ns[3] = (double)h_ns[3] / LAT_HOPS;
    out_ns[4] = (double)h_ns[4] / LAT_ROUNDS;
    return LSQ_OK;
}
