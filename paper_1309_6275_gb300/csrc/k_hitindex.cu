// k_hitindex.cu -- per-event index of the hits by (layer, azimuth bin), for
// the candidate confirmation (k_confirm.cu).
//
// Cell (l, b) of event e holds the event's hits of layer l whose azimuth
// atan2(y, x) falls in bin b = floor((phi + pi) * kIdxAz / (2 pi)) (clamped
// to [0, kIdxAz)); the cells of an event are contiguous in layer-major order
// and the events follow one another, so event e's cells start at its first
// hit's batch position.  Each position holds the hit's x, y (float32), its
// event-local index and its layer; within a cell the order is that of the
// fill's atomics (the confirmation's results do not depend on it).  The
// per-(event, layer) radius range is kept for the confirmation's azimuth
// windows.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ht_internal.cuh"

namespace ht {
namespace {

__device__ __forceinline__ int event_of_hit(const int *off, int n_ev, int h)
{
    int lo = 0, hi = n_ev - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= h) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int az_bin(float xf, float yf)
{
    const float a = atan2f(yf, xf);
    const int b = (int)floorf((a + 3.14159265f) * (kIdxAz / 6.28318531f));
    return min(max(b, 0), kIdxAz - 1);
}

// pass 0: counts per cell and the radius range per (event, layer);
// pass 1: positions (cur holds each cell's next free position)
__global__ void k_hidx(const float *__restrict__ x, const float *__restrict__ y,
                       const uint8_t *__restrict__ layer, const int *__restrict__ off,
                       const int *__restrict__ d_nev, int *__restrict__ cnt,
                       unsigned *__restrict__ rmm, int *__restrict__ cur, HitIndex I)
{
    const int n_ev = *d_nev;
    const int n = off[n_ev];
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
        const int e = event_of_hit(off, n_ev, h);
        const float xf = x[h], yf = y[h];
        const int l = layer[h] & 15;
        const int cell = (e * 16 + l) * kIdxAz + az_bin(xf, yf);
        if (cur) {
            const int p = atomicAdd(&cur[cell], 1);
            I.x[p] = xf;
            I.y[p] = yf;
            I.h[p] = h - off[e];
            I.l[p] = (uint8_t)l;
        } else {
            atomicAdd(&cnt[cell], 1);
            const unsigned rb = __float_as_uint(sqrtf(fmaf(xf, xf, yf * yf)));
            atomicMin(&rmm[2 * (e * 16 + l)], rb);       // non-negative floats order as their bits
            atomicMax(&rmm[2 * (e * 16 + l) + 1], rb);
        }
    }
}

__global__ void k_hidx_init(unsigned *__restrict__ rmm, int n)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        rmm[2 * t] = 0x7f800000u;   // +inf: empty layer (min > max)
        rmm[2 * t + 1] = 0u;
    }
}

}  // namespace

size_t hit_index_bytes(int max_events, int max_hits)
{
    const size_t nc = (size_t)max_events * 16 * kIdxAz;
    const size_t mh = (size_t)(max_hits > 0 ? max_hits : 1);
    return 3 * align256((nc + 1) * 4) + align256((size_t)max_events * 16 * 8) +
           3 * align256(mh * 4) + align256(mh) + scan_tmp_bytes((int)nc);
}

HitIndex carve_hit_index(int max_events, int max_hits, void *ws)
{
    const size_t nc = (size_t)max_events * 16 * kIdxAz;
    const size_t mh = (size_t)(max_hits > 0 ? max_hits : 1);
    char *p = reinterpret_cast<char *>(ws);
    HitIndex I;
    I.cnt = reinterpret_cast<int *>(p);
    p += align256((nc + 1) * 4);
    I.offs = reinterpret_cast<int *>(p);
    p += align256((nc + 1) * 4);
    I.cur = reinterpret_cast<int *>(p);
    p += align256((nc + 1) * 4);
    I.rmm = reinterpret_cast<unsigned *>(p);
    p += align256((size_t)max_events * 16 * 8);
    I.x = reinterpret_cast<float *>(p);
    p += align256(mh * 4);
    I.y = reinterpret_cast<float *>(p);
    p += align256(mh * 4);
    I.h = reinterpret_cast<int *>(p);
    p += align256(mh * 4);
    I.l = reinterpret_cast<uint8_t *>(p);
    p += align256(mh);
    I.tmp = p;
    I.ncells = (int)nc;
    return I;
}

cudaError_t launch_hit_index(const float *x, const float *y, const uint8_t *layer,
                             const int *off, const int *d_nev, int max_events, int max_hits,
                             const HitIndex &I, int sms, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(I.cnt, 0, (size_t)I.ncells * 4, st);
    if (e != cudaSuccess) return e;
    k_hidx_init<<<32, 256, 0, st>>>(I.rmm, max_events * 16);
    const int grid = sms * 4;
    k_hidx<<<grid, 256, 0, st>>>(x, y, layer, off, d_nev, I.cnt, I.rmm, nullptr, I);
    e = scan_exclusive(I.cnt, I.offs, I.cur, I.ncells, nullptr, I.offs + I.ncells, I.tmp, st);
    if (e != cudaSuccess) return e;
    k_hidx<<<grid, 256, 0, st>>>(x, y, layer, off, d_nev, I.cnt, I.rmm, I.cur, I);
    (void)max_hits;
    return cudaGetLastError();
}

}  // namespace ht
