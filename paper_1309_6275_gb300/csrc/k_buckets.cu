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

__global__ void k_bucket_count(DevGeom G, const float *__restrict__ x,
                               const float *__restrict__ y, const int *__restrict__ off,
                               const int *__restrict__ d_nev, int *__restrict__ cnt)
{
    const int n_ev = *d_nev, n = off[n_ev], NG = G.n_phi0 / kGroupCols;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
        const int e = event_of(off, n_ev, h);
        int g_lo, ng;
        hit_groups(G, x[h], y[h], g_lo, ng);
        for (int t = 0; t < ng; ++t) {
            const int gi = g_lo + t < NG ? g_lo + t : g_lo + t - NG;
            atomicAdd(&cnt[e * NG + gi], 1);
        }
    }
}

__global__ void k_bucket_fill(DevGeom G, const float *__restrict__ x,
                              const float *__restrict__ y, const int *__restrict__ off,
                              const int *__restrict__ d_nev, int *__restrict__ cursor,
                              int *__restrict__ ent)
{
    const int n_ev = *d_nev, n = off[n_ev], NG = G.n_phi0 / kGroupCols;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
        const int e = event_of(off, n_ev, h);
        int g_lo, ng;
        hit_groups(G, x[h], y[h], g_lo, ng);
        for (int t = 0; t < ng; ++t) {
            const int gi = g_lo + t < NG ? g_lo + t : g_lo + t - NG;
            ent[atomicAdd(&cursor[e * NG + gi], 1)] = h - off[e];
        }
    }
}

}  // namespace

size_t hit_bucket_bytes(const DevGeom &G, int max_events, int max_hits)
{
    const size_t nc = (size_t)max_events * (G.n_phi0 / kGroupCols);
    return 3 * align256((nc + 1) * 4) + scan_tmp_bytes((int)nc) +
           align256((size_t)max_hits * (G.n_phi0 / kGroupCols) * 4);
}

HitBuckets carve_hit_buckets(const DevGeom &G, int max_events, void *ws)
{
    const size_t nc = (size_t)max_events * (G.n_phi0 / kGroupCols);
    char *p = reinterpret_cast<char *>(ws);
    HitBuckets b;
    b.cnt = reinterpret_cast<int *>(p);
    b.start = reinterpret_cast<int *>(p + align256((nc + 1) * 4));
    b.cursor = reinterpret_cast<int *>(p + 2 * align256((nc + 1) * 4));
    b.tmp = p + 3 * align256((nc + 1) * 4);
    b.ent = reinterpret_cast<int *>(p + 3 * align256((nc + 1) * 4) + scan_tmp_bytes((int)nc));
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
    const int blocks = min((max_hits + 255) / 256, 8 * sms);
    k_bucket_count<<<blocks, 256, 0, st>>>(G, x, y, off, d_nev, b.cnt);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = scan_exclusive(b.cnt, b.start, b.cursor, b.ncells, nullptr, nullptr, b.tmp, st);
    if (e != cudaSuccess) return e;
    k_bucket_fill<<<blocks, 256, 0, st>>>(G, x, y, off, d_nev, b.cursor, b.ent);
    return cudaGetLastError();
}

}  // namespace ht
