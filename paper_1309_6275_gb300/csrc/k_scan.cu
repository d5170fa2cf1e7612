// k_scan.cu -- device-wide exclusive prefix sum of int32 counts, used to turn
// per-segment peak counts and per-candidate hit counts into output offsets.
//
// Three launches, all coalesced: per-block sums of 4096-element chunks
// (1024 threads x 4), one CTA scanning the block sums, per-block rescan with
// the block's offset.  The element count may live in device memory (graph
// capture: no host read).
#include <cuda_runtime.h>
#include <stdint.h>

#include "ht_internal.cuh"

namespace ht {
namespace {

constexpr int kScanT = 1024;
constexpr int kPer = 4;
constexpr int kChunk = kScanT * kPer;

__device__ __forceinline__ int scan_count(int n_cap, const int *d_n)
{
    return d_n ? max(0, min(*d_n, n_cap)) : n_cap;
}

// Block-wide exclusive scan of one int per thread (blockDim == kScanT);
// returns the block total.  All threads must call.
__device__ __forceinline__ int block_exclusive(int v, int &excl)
{
    __shared__ int wsum[kScanT / 32];
    __shared__ int s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int w = wsum[lane];
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        wsum[lane] = wi - w;
        if (lane == 31) s_total = wi;
    }
    __syncthreads();
    excl = wsum[warp] + incl - v;
    const int total = s_total;
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(kScanT)
k_scan_sums(const int *__restrict__ in, int n_cap, const int *__restrict__ d_n,
            int *__restrict__ sums)
{
    const int n = scan_count(n_cap, d_n);
    const int base = blockIdx.x * kChunk + threadIdx.x * kPer;
    int s = 0;
#pragma unroll
    for (int u = 0; u < kPer; ++u) s += (base + u < n) ? in[base + u] : 0;
    int excl;
    const int tot = block_exclusive(s, excl);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanT)
k_scan_top(int *__restrict__ sums, int nb)
{
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += kScanT) {
        const int b = b0 + threadIdx.x;
        const int v = b < nb ? sums[b] : 0;
        int excl;
        const int total = block_exclusive(v, excl);
        if (b < nb) sums[b] = carry + excl;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void __launch_bounds__(kScanT)
k_scan_apply(const int *__restrict__ in, int n_cap, const int *__restrict__ d_n,
             const int *__restrict__ sums, int nb, int *__restrict__ out,
             int *__restrict__ out2, int *__restrict__ total)
{
    const int n = scan_count(n_cap, d_n);
    const int base = blockIdx.x * kChunk + threadIdx.x * kPer;
    int v[kPer], s = 0;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        v[u] = (base + u < n) ? in[base + u] : 0;
        s += v[u];
    }
    int excl;
    block_exclusive(s, excl);
    int run = sums[blockIdx.x] + excl;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        if (base + u < n) {
            out[base + u] = run;
            if (out2) out2[base + u] = run;
        }
        run += v[u];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[n] = sums[nb];
        if (total) *total = sums[nb];
    }
}

}  // namespace

size_t scan_tmp_bytes(int n_cap) { return align256((size_t)((n_cap + kChunk - 1) / kChunk + 2) * 4); }

// out[0..n) = exclusive prefix of in[0..n), out[n] = sum (out needs n_cap + 1
// entries); n = min(*d_n, n_cap) when d_n is given.  out2 (optional) gets a
// copy of out[0..n); *total (optional) the sum.  tmp: scan_tmp_bytes(n_cap).
cudaError_t scan_exclusive(const int *in, int *out, int *out2, int n_cap, const int *d_n,
                           int *total, void *tmp, cudaStream_t st)
{
    const int nb = (n_cap + kChunk - 1) / kChunk;
    const int nbl = nb > 0 ? nb : 1;
    int *sums = reinterpret_cast<int *>(tmp);
    k_scan_sums<<<nbl, kScanT, 0, st>>>(in, n_cap, d_n, sums);
    k_scan_top<<<1, kScanT, 0, st>>>(sums, nbl);
    k_scan_apply<<<nbl, kScanT, 0, st>>>(in, n_cap, d_n, sums, nbl, out, out2, total);
    return cudaGetLastError();
}

}  // namespace ht
