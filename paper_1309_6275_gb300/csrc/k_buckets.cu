// k_buckets.cu -- per-event lists of the hits that can vote in each group of
// kGroupCols phi0 columns, so that a tile's phase 1 scans only those hits
// instead of all of the event's (the batched tile kernels of tiles.cuh and
// k_tiles.cu).
//
// A hit can vote in column k only where c = r cos(phi0_k - psi) reaches the
// hit's angular window (hit_cos_window, ht_internal.cuh): |phi0_k - psi| <= w
// with cos w = cmin / r.  The lists keep every hit whose widened window
// (0.02 cm plus 4e-7 (|x| + |y|) on c, the bound of phase 1's float32
// error in c; 2e-3 rad on the angle, which also covers acos near 1 for an
// error below 2e-6 in its argument; one column on each side) meets a
// column of the group -- a superset of what phase 1 keeps, which still
// tests every column, so the votes are the same.  Hits within a list are in
// no particular order; nothing downstream depends on it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ht_internal.cuh"

namespace ht {
namespace {

__device__ __forceinline__ int event_of(const int *off, int n_ev, int h)
{
    int lo = 0, hi = n_ev;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= h) lo = mid; else hi = mid;
    }
    return lo;
}

// Column groups [g_lo, g_lo + ng) (mod the group count) whose columns a hit
// can reach; ng = the group count when the window covers the circle.
__device__ __forceinline__ void hit_groups(const DevGeom &G, float x, float y, int &g_lo,
                                           int &ng)
{
    const int NP = G.n_phi0, NG = NP / kGroupCols;
    const float r2 = fmaf(x, x, y * y);
    const float r = sqrtf(r2);
    const float cmin = hit_cos_window(G, r2);
    const float thr = (cmin - fmaf(4e-7f, fabsf(x) + fabsf(y), 0.02f)) / r;
    if (!(thr > -1.0f)) {            // window covers the circle (or r == 0)
        g_lo = 0;
        ng = NG;
        return;
    }
    const float w = acosf(fminf(thr, 1.0f)) + 2e-3f;
    const float dphi = 6.283185307179586f / (float)NP;
    const float kc = (atan2f(y, x) + 3.14159265358979f) / dphi - 0.5f;   // column coordinate
    const float kw = w / dphi;
    const int k_lo = (int)floorf(kc - kw) - 1, k_hi = (int)ceilf(kc + kw) + 1;
    if (k_hi - k_lo + 1 >= NP) {
        g_lo = 0;
        ng = NG;
        return;
    }
    const int a = (int)floorf((float)k_lo / (float)kGroupCols);
    const int b = (int)floorf((float)k_hi / (float)kGroupCols);
    ng = min(b - a + 1, NG);
    g_lo = ((a % NG) + NG) % NG;
}

// Hits are taken in chunks of kBkChunk consecutive batch positions (mostly
// one or two events).  A chunk's per-(event, group) counts gather in shared
// memory and go out with one global atomic per nonzero counter; hits of an
// event beyond the chunk's first kBkEv, or geometries with more than
// kBkMaxNG groups, use the global counters directly.
constexpr int kBkThreads = 256, kBkChunk = 2048, kBkEv = 4, kBkMaxNG = 256;

// Counts per (event, group); hg[h] = first group | group count << 16.
__global__ void __launch_bounds__(kBkThreads)
k_bucket_count(DevGeom G, const float *__restrict__ x, const float *__restrict__ y,
               const int *__restrict__ off, const int *__restrict__ d_nev, int *__restrict__ cnt,
               int *__restrict__ hg)
{
    __shared__ int s_cnt[kBkEv * kBkMaxNG];
    const int n_ev = *d_nev, n = off[n_ev], NG = G.n_phi0 / kGroupCols;
    const bool local = NG <= kBkMaxNG;
    for (int h0 = blockIdx.x * kBkChunk; h0 < n; h0 += gridDim.x * kBkChunk) {
        const int h1 = min(h0 + kBkChunk, n);
        const int e0 = event_of(off, n_ev, h0);
        for (int i = threadIdx.x; i < kBkEv * kBkMaxNG; i += kBkThreads) s_cnt[i] = 0;
        __syncthreads();
        for (int h = h0 + threadIdx.x; h < h1; h += kBkThreads) {
            const int e = event_of(off, n_ev, h);
            int g_lo, ng;
            hit_groups(G, x[h], y[h], g_lo, ng);
            hg[h] = g_lo | (ng << 16);
            const bool sh = local && e - e0 < kBkEv;
            for (int t = 0; t < ng; ++t) {
                const int gi = g_lo + t < NG ? g_lo + t : g_lo + t - NG;
                if (sh) atomicAdd(&s_cnt[(e - e0) * kBkMaxNG + gi], 1);
                else atomicAdd(&cnt[e * NG + gi], 1);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kBkEv * kBkMaxNG; i += kBkThreads) {
            const int v = s_cnt[i];
            if (v) atomicAdd(&cnt[(e0 + i / kBkMaxNG) * NG + i % kBkMaxNG], v);
        }
        __syncthreads();
    }
}

// Entries: a chunk reserves one range per nonzero (event, group) counter
// and places its hits there through shared cursors.
__global__ void __launch_bounds__(kBkThreads)
k_bucket_fill(DevGeom G, const int *__restrict__ off, const int *__restrict__ d_nev,
              const int *__restrict__ hg, int *__restrict__ cursor, int *__restrict__ ent)
{
    __shared__ int s_cnt[kBkEv * kBkMaxNG];
    const int n_ev = *d_nev, n = off[n_ev], NG = G.n_phi0 / kGroupCols;
    const bool local = NG <= kBkMaxNG;
    for (int h0 = blockIdx.x * kBkChunk; h0 < n; h0 += gridDim.x * kBkChunk) {
        const int h1 = min(h0 + kBkChunk, n);
        const int e0 = event_of(off, n_ev, h0);
        for (int i = threadIdx.x; i < kBkEv * kBkMaxNG; i += kBkThreads) s_cnt[i] = 0;
        __syncthreads();
        for (int h = h0 + threadIdx.x; h < h1; h += kBkThreads) {
            const int e = event_of(off, n_ev, h);
            if (!(local && e - e0 < kBkEv)) continue;
            const int g = hg[h], g_lo = g & 0xffff, ng = g >> 16;
            for (int t = 0; t < ng; ++t) {
                const int gi = g_lo + t < NG ? g_lo + t : g_lo + t - NG;
                atomicAdd(&s_cnt[(e - e0) * kBkMaxNG + gi], 1);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kBkEv * kBkMaxNG; i += kBkThreads) {
            const int v = s_cnt[i];
            if (v) s_cnt[i] = atomicAdd(&cursor[(e0 + i / kBkMaxNG) * NG + i % kBkMaxNG], v);
        }
        __syncthreads();
        for (int h = h0 + threadIdx.x; h < h1; h += kBkThreads) {
            const int e = event_of(off, n_ev, h);
            const bool sh = local && e - e0 < kBkEv;
            const int g = hg[h], g_lo = g & 0xffff, ng = g >> 16;
            for (int t = 0; t < ng; ++t) {
                const int gi = g_lo + t < NG ? g_lo + t : g_lo + t - NG;
                const int pos = sh ? atomicAdd(&s_cnt[(e - e0) * kBkMaxNG + gi], 1)
                                   : atomicAdd(&cursor[e * NG + gi], 1);
                ent[pos] = h - off[e];
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t hit_bucket_bytes(const DevGeom &G, int max_events, int max_hits)
{
    const size_t nc = (size_t)max_events * (G.n_phi0 / kGroupCols);
    return 3 * align256((nc + 1) * 4) + scan_tmp_bytes((int)nc) +
           align256((size_t)max_hits * (G.n_phi0 / kGroupCols) * 4) +
           align256((size_t)(max_hits > 0 ? max_hits : 1) * 4);
}

HitBuckets carve_hit_buckets(const DevGeom &G, int max_events, int max_hits, void *ws)
{
    const size_t nc = (size_t)max_events * (G.n_phi0 / kGroupCols);
    char *p = reinterpret_cast<char *>(ws);
    HitBuckets b;
    b.cnt = reinterpret_cast<int *>(p);
    b.start = reinterpret_cast<int *>(p + align256((nc + 1) * 4));
    b.cursor = reinterpret_cast<int *>(p + 2 * align256((nc + 1) * 4));
    b.tmp = p + 3 * align256((nc + 1) * 4);
    b.ent = reinterpret_cast<int *>(p + 3 * align256((nc + 1) * 4) + scan_tmp_bytes((int)nc));
    b.hg = b.ent + align256((size_t)max_hits * (G.n_phi0 / kGroupCols) * 4) / 4;
    b.ngroups = G.n_phi0 / kGroupCols;
    b.ncells = (int)nc;
    return b;
}

cudaError_t launch_hit_buckets(const DevGeom &G, const float *x, const float *y, const int *off,
                               const int *d_nev, int max_hits, const HitBuckets &b, int sms,
                               cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(b.cnt, 0, (size_t)b.ncells * 4, st);
    if (e != cudaSuccess || max_hits <= 0) return e;
    const int blocks = min((max_hits + kBkChunk - 1) / kBkChunk, 4 * sms);
    k_bucket_count<<<blocks, kBkThreads, 0, st>>>(G, x, y, off, d_nev, b.cnt, b.hg);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = scan_exclusive(b.cnt, b.start, b.cursor, b.ncells, nullptr, nullptr, b.tmp, st);
    if (e != cudaSuccess) return e;
    k_bucket_fill<<<blocks, kBkThreads, 0, st>>>(G, off, d_nev, b.hg, b.cursor, b.ent);
    return cudaGetLastError();
}

}  // namespace ht
