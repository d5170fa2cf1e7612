// probe.cu -- microbenchmark of shared-memory atomic throughput (the roofline
// of the vote's counting); declared in include/ht_probe.h.  Built as its own
// library (libht_probe.so), used by the benchmark only: not part of libht.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ht_probe.h"

namespace {

constexpr int kProbeThreads = 1024;

__global__ void __launch_bounds__(kProbeThreads)
k_probe_atoms(int iters, unsigned *__restrict__ sink)
{
    __shared__ unsigned cell[kProbeThreads];
    cell[threadIdx.x] = 0u;
    __syncthreads();
    unsigned *p = &cell[threadIdx.x];     // lane-distinct word, distinct banks
    for (int t = 0; t < iters; t += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) atomicAdd(p, 1u);
    }
    __syncthreads();
    if (cell[threadIdx.x] == 0xdeadbeefu) sink[blockIdx.x] = 1u;   // keep the work
}

}  // namespace

extern "C" ht_status ht_probe_shared_atomic_rate(int32_t iters, double *ops_per_s,
                                                 ht_stream stream)
{
    if (!ops_per_s || iters < 1 || iters > (1 << 20)) return HT_ERR_ARG;
    iters = (iters + 7) & ~7;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HT_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HT_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_atoms, kProbeThreads, 0) !=
        cudaSuccess)
        return HT_ERR_CUDA;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    unsigned *sink = nullptr;
    cudaEvent_t a, b;
    if (cudaMalloc(&sink, sizeof(unsigned) * blocks) != cudaSuccess) return HT_ERR_CUDA;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_probe_atoms<<<blocks, kProbeThreads, 0, st>>>(iters, sink);      // warm-up
    cudaEventRecord(a, st);
    k_probe_atoms<<<blocks, kProbeThreads, 0, st>>>(iters, sink);
    cudaEventRecord(b, st);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    if (e != cudaSuccess || ms <= 0.f) return HT_ERR_CUDA;
    *ops_per_s = (double)blocks * kProbeThreads * (double)iters / (ms * 1e-3);
    return HT_OK;
}
