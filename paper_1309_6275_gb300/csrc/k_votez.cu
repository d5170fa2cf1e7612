// k_votez.cu -- per-candidate (z0, cot theta) vote.
//
// The paper works in the transverse plane only (Section 5's detector model);
// this second vote completes each candidate along z.  Reading: at the
// candidate's cell centres the arc length to a hit is L = theta / rho with
// theta = atan2(rho c, 1 + rho (s + d0)); each hit votes z0 = z - L t_q for
// every cot-theta centre t_q; the result is the histogram's maximum cell,
// ties to the smallest n n_cot + q.
//
// Design (GB300):
//  * Hits are grouped by candidate in device memory (count, one-CTA scan,
//    scatter), so every candidate reads only its own hits.
//  * Candidates with at most 32 hits (nearly all): one warp per candidate,
//    lane = hit.  For each cot column q every lane bins its hit; the count of
//    each lane's bin is __match_any_sync's popcount (warp-aggregated, no
//    histogram in memory) and one redux.sync max over (count, -n) gives the
//    column's best cell.
//  * Larger candidates: one CTA per candidate with an n_z0 x n_cot uint32
//    histogram in shared memory and a block argmax.
//  * Arithmetic: float32 with a proven error bound per (hit, q); any bin
//    coordinate within its bound of an edge is redone in float64 in the
//    definition's order with the basic-operation atan2, so every vote
//    matches the float64 definition bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ht_internal.cuh"

namespace ht {
namespace {

constexpr int kBigThreads = 256;

struct ZCand {
    float rho, invrho, sn, cs, d0c;
    double rho64, sn64, cs64, d0c64;
    bool rho0;
};

__device__ __forceinline__ ZCand z_cand(const DevGeom &G, const ht_peak &p)
{
    ZCand c;
    c.rho = G.rho32[p.i_rho];
    c.invrho = G.invrho32[p.i_rho];
    c.sn = G.sn32[p.k_phi0];
    c.cs = G.cs32[p.k_phi0];
    c.rho64 = G.rho64[p.i_rho];
    c.sn64 = G.sn64[p.k_phi0];
    c.cs64 = G.cs64[p.k_phi0];
    c.d0c64 = __dmul_rn(__dsub_rn((double)p.j_d0, __dmul_rn(0.5, (double)G.n_d0)), G.delta);
    c.d0c = (float)c.d0c64;
    c.rho0 = c.rho64 == 0.0;
    return c;
}

// Arc length in float32 and a bound on its error (turning angle from atan2f,
// taken as <= 4 ulp, plus the propagated rounding of its arguments).
__device__ __forceinline__ void arc32(const ZCand &C, float x, float y, float &L, float &eL)
{
    const float s = fmaf(x, C.sn, -(y * C.cs));
    const float c = fmaf(x, C.cs, y * C.sn);
    const float R1 = fabsf(x) + fabsf(y);
    const float Es = 3.0f * kEps * R1;
    if (C.rho0) {
        L = c;
        eL = kSafe * Es;
        return;
    }
    const float a = C.rho * c;
    const float w = s + C.d0c;
    const float bb = fmaf(C.rho, w, 1.0f);
    const float th = atan2f(a, bb);
    L = th * C.invrho;
    const float ar = fabsf(C.rho);
    const float da = fmaf(ar, Es, 2.0f * kEps * fabsf(a));
    const float dbb = fmaf(ar, Es + kEps * (fabsf(w) + fabsf(C.d0c)), kEps * (fabsf(C.rho * w) + fabsf(bb)));
    const float den = fmaf(a, a, bb * bb);
    const float dth = 8.0f * kEps * fabsf(th) + __fdividef(fmaf(fabsf(bb), da, fabsf(a) * dbb), den);
    eL = kSafe * fmaf(fabsf(C.invrho), dth, 2.0f * kEps * fabsf(L));
    if (!(den > 1e-6f)) eL = 3.4e38f;   // hit at the circle's centre: exact path
}

// Arc length in float64, in the definition's operation order.
__device__ __forceinline__ double arc64(const ZCand &C, float xf, float yf)
{
    const double x = xf, y = yf;
    const double s = __dsub_rn(__dmul_rn(x, C.sn64), __dmul_rn(y, C.cs64));
    const double c = __dadd_rn(__dmul_rn(x, C.cs64), __dmul_rn(y, C.sn64));
    if (C.rho64 == 0.0) return c;
    const double th = atan2_basic64(__dmul_rn(C.rho64, c),
                                    __dadd_rn(1.0, __dmul_rn(C.rho64, __dadd_rn(s, C.d0c64))));
    return __ddiv_rn(th, C.rho64);
}

// z0 bin of one (hit, q): float32 if provably decided, else float64 (L64 is
// computed on first need and cached by the caller through `have64`).
__device__ __forceinline__ int z_bin(const DevGeom &G, const ZCand &C, float xf, float yf,
                                     float z, float L, float eL, int q, bool &have64,
                                     double &L64)
{
    const float t = G.cstep_f * (float)(2 * q + 1 - G.n_cot);
    const float zz = z + G.z0_max_f;
    const float v = fmaf(-L, t, zz);
    const float u = v * G.inv_dz_f;
    const float err = fmaf(fmaf(fabsf(t), eL, kSafe * kEps * (2.0f * fabsf(L * t) + fabsf(zz) + fabsf(v))),
                           G.inv_dz_f, kSafe * kEps * fabsf(u));
    const float nz = (float)G.n_z0;
    if (u + err < 0.0f || u - err >= nz) return -1;
    const float f = floorf(u);
    const float fr = u - f;
    // u + 1 (u in (-1, 0)) is rounded: only f >= 0 is decided here
    if (f >= 0.0f && fminf(fr, 1.0f - fr) > err) return (int)f;
    if (!have64) {
        L64 = arc64(C, xf, yf);
        have64 = true;
    }
    const double t64 = __dmul_rn((double)(2 * q + 1 - G.n_cot), G.cstep);
    const double z0 = __dsub_rn((double)z, __dmul_rn(L64, t64));
    const double u64 = __ddiv_rn(__dadd_rn(z0, G.z0_max), G.dz);
    if (u64 >= 0.0 && u64 < (double)G.n_z0) return (int)floor(u64);
    return -1;
}

__global__ void k_z_count(const int *__restrict__ assign, int n, const int *__restrict__ d_count,
                          int cap, int *__restrict__ cnt)
{
    const int ncand = min(*d_count, cap);
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
        const int a = assign[h];
        if (a >= 0 && a < ncand) atomicAdd(&cnt[a], 1);
    }
}

__global__ void k_z_scatter(const int *__restrict__ assign, int n, const int *__restrict__ d_count,
                            int cap, int *__restrict__ cur, int *__restrict__ list)
{
    const int ncand = min(*d_count, cap);
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
        const int a = assign[h];
        if (a >= 0 && a < ncand) list[atomicAdd(&cur[a], 1)] = h;
    }
}

// (z0, cot theta) result of one candidate with 1..32 hits list[o .. o + nh),
// one warp, lane = hit.  Every lane returns the result.
__device__ __forceinline__ ht_zres z_small_cand(const DevGeom &G, const float *__restrict__ x,
                                                const float *__restrict__ y,
                                                const float *__restrict__ z, const ht_peak &pk,
                                                const int *__restrict__ list, int o, int nh,
                                                int lane)
{
    const ZCand C = z_cand(G, pk);
    const bool act = lane < nh;
    float xf = 0.f, yf = 0.f, zf = 0.f, L = 0.f, eL = 0.f;
    if (act) {
        const int h = list[o + lane];
        xf = x[h];
        yf = y[h];
        zf = z[h];
        arc32(C, xf, yf, L, eL);
    }
    bool have64 = false;
    double L64 = 0.0;
    unsigned best_c = 0u;
    int best_idx = 0x7fffffff;
    for (int q = 0; q < G.n_cot; ++q) {
        const int nb = act ? z_bin(G, C, xf, yf, zf, L, eL, q, have64, L64) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, nb);
        const unsigned key = nb >= 0 ? ((unsigned)__popc(peers) << 16) | (0xffffu - (unsigned)nb) : 0u;
        const unsigned top = __reduce_max_sync(0xffffffffu, key);
        if (top) {
            const unsigned cq = top >> 16;
            const int idx = (int)(0xffffu - (top & 0xffffu)) * G.n_cot + q;
            if (cq > best_c || (cq == best_c && idx < best_idx)) {
                best_c = cq;
                best_idx = idx;
            }
        }
    }
    return best_c ? ht_zres{best_idx / G.n_cot, best_idx % G.n_cot, (int)best_c}
                  : ht_zres{-1, -1, 0};
}

// One warp per candidate with <= 32 hits; larger ones go to the big list.
__global__ void k_z_small(DevGeom G, const float *__restrict__ x, const float *__restrict__ y,
                          const float *__restrict__ z, const ht_peak *__restrict__ peaks,
                          const int *__restrict__ d_count, int cap, const int *__restrict__ off,
                          const int *__restrict__ list, ht_zres *__restrict__ out,
                          int *__restrict__ big, int *__restrict__ nbig)
{
    const int ncand = min(*d_count, cap);
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int m = gw; m < ncand; m += nw) {
        const int o = off[m], nh = off[m + 1] - o;
        if (nh == 0) {
            if (lane == 0) out[m] = ht_zres{-1, -1, 0};
            continue;
        }
        if (nh > 32) {
            if (lane == 0) big[atomicAdd(nbig, 1)] = m;
            continue;
        }
        const ht_zres r = z_small_cand(G, x, y, z, peaks[m], list, o, nh, lane);
        if (lane == 0) out[m] = r;
    }
}

// (z0, cot theta) result of one candidate with any number of hits, one CTA:
// n_z0 x n_cot uint32 histogram in shared memory and a block argmax.
// Thread 0 returns the result.  All threads must call.
__device__ __forceinline__ ht_zres z_big_cand(const DevGeom &G, const float *__restrict__ x,
                                              const float *__restrict__ y,
                                              const float *__restrict__ z, const ht_peak &pk,
                                              const int *__restrict__ list, int o, int nh)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned *hist = reinterpret_cast<unsigned *>(smem);
    __shared__ float sL[kBigThreads], seL[kBigThreads], sx[kBigThreads], sy[kBigThreads],
        sz[kBigThreads];
    __shared__ unsigned long long red[kBigThreads / 32];
    const int NC = G.n_cot, NZ = G.n_z0, ncell = NZ * NC;
    const ZCand C = z_cand(G, pk);
    for (int t = threadIdx.x; t < ncell; t += kBigThreads) hist[t] = 0u;
    for (int c0 = 0; c0 < nh; c0 += kBigThreads) {
        __syncthreads();
        const int hc = min(kBigThreads, nh - c0);
        if (threadIdx.x < hc) {
            const int h = list[o + c0 + threadIdx.x];
            sx[threadIdx.x] = x[h];
            sy[threadIdx.x] = y[h];
            sz[threadIdx.x] = z[h];
            arc32(C, sx[threadIdx.x], sy[threadIdx.x], sL[threadIdx.x], seL[threadIdx.x]);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < hc * NC; t += kBigThreads) {
            const int hl = t / NC, q = t - hl * NC;
            bool have64 = false;
            double L64 = 0.0;
            const int nbin = z_bin(G, C, sx[hl], sy[hl], sz[hl], sL[hl], seL[hl], q, have64, L64);
            if (nbin >= 0) atomicAdd(&hist[nbin * NC + q], 1u);
        }
    }
    __syncthreads();
    // argmax: key = count << 32 | ~index (largest count, then smallest index)
    unsigned long long bk = 0ull;
    for (int t = threadIdx.x; t < ncell; t += kBigThreads) {
        const unsigned c = hist[t];
        const unsigned long long k = ((unsigned long long)c << 32) | (0xffffffffull - (unsigned)t);
        if (c && k > bk) bk = k;
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) bk = max(bk, __shfl_xor_sync(0xffffffffu, bk, s));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = bk;
    __syncthreads();
    ht_zres r{-1, -1, 0};
    if (threadIdx.x == 0) {
        unsigned long long b = 0ull;
        for (int w = 0; w < kBigThreads / 32; ++w) b = max(b, red[w]);
        if (b) {
            const int idx = (int)(0xffffffffu - (unsigned)(b & 0xffffffffull));
            r = ht_zres{idx / NC, idx % NC, (int)(b >> 32)};
        }
    }
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kBigThreads)
k_z_big(DevGeom G, const float *__restrict__ x, const float *__restrict__ y,
        const float *__restrict__ z, const ht_peak *__restrict__ peaks,
        const int *__restrict__ off, const int *__restrict__ list,
        const int *__restrict__ big, const int *__restrict__ nbig, ht_zres *__restrict__ out)
{
    const int nb = *nbig;
    for (int bi = blockIdx.x; bi < nb; bi += gridDim.x) {
        const int m = big[bi];
        const ht_zres r = z_big_cand(G, x, y, z, peaks[m], list, off[m], off[m + 1] - off[m]);
        if (threadIdx.x == 0) out[m] = r;
    }
}

// ---------------------------------------------------------------- batches
// Global candidate id g = e * cap + m (event slot e, candidate m); hits carry
// batch-wide indices; off[0..n_ev] are the events' hit offsets.
__device__ __forceinline__ int event_of(const int *__restrict__ off, int n_ev, int h)
{
    int lo = 0, hi = n_ev;          // off[lo] <= h < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= h) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_zb_group(const int *__restrict__ assign, const int *__restrict__ off,
                           const int *__restrict__ d_nev, const int *__restrict__ counts,
                           int cap, int *__restrict__ cnt, int *__restrict__ cur,
                           int *__restrict__ list)
{
    const int n_ev = *d_nev, n = off[n_ev];
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
        const int a = assign[h];
        if (a < 0) continue;
        const int e = event_of(off, n_ev, h);
        if (a >= min(counts[e], cap)) continue;
        const size_t g = (size_t)e * cap + a;
        if (list) list[atomicAdd(&cur[g], 1)] = h;
        else atomicAdd(&cnt[g], 1);
    }
}

__global__ void k_zb_small(DevGeom G, const float *__restrict__ x, const float *__restrict__ y,
                           const float *__restrict__ z, const ht_peak *__restrict__ peaks,
                           const int *__restrict__ counts, const int *__restrict__ d_nev,
                           int cap, const int *__restrict__ off, const int *__restrict__ list,
                           ht_zres *__restrict__ out, int *__restrict__ big,
                           int *__restrict__ nbig)
{
    const int e = blockIdx.y;
    if (e >= *d_nev) return;
    const int ncand = min(counts[e], cap);
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int m = gw; m < ncand; m += nw) {
        const size_t g = (size_t)e * cap + m;
        const int o = off[g], nh = off[g + 1] - o;
        if (nh == 0) {
            if (lane == 0) out[g] = ht_zres{-1, -1, 0};
            continue;
        }
        if (nh > 32) {
            if (lane == 0) big[atomicAdd(nbig, 1)] = (int)g;
            continue;
        }
        const ht_zres r = z_small_cand(G, x, y, z, peaks[g], list, o, nh, lane);
        if (lane == 0) out[g] = r;
    }
}

__global__ void __launch_bounds__(kBigThreads)
k_zb_big(DevGeom G, const float *__restrict__ x, const float *__restrict__ y,
         const float *__restrict__ z, const ht_peak *__restrict__ peaks,
         const int *__restrict__ off, const int *__restrict__ list,
         const int *__restrict__ big, const int *__restrict__ nbig, ht_zres *__restrict__ out)
{
    const int nb = *nbig;
    for (int bi = blockIdx.x; bi < nb; bi += gridDim.x) {
        const int g = big[bi];
        const ht_zres r = z_big_cand(G, x, y, z, peaks[g], list, off[g], off[g + 1] - off[g]);
        if (threadIdx.x == 0) out[g] = r;
    }
}

struct ZWs {
    int *cnt, *off, *cur, *list, *big, *nbig;
    void *tmp;
};

ZWs carve(void *ws, int n, int cap)
{
    char *p = reinterpret_cast<char *>(ws);
    ZWs w;
    w.cnt = reinterpret_cast<int *>(p); p += align256((size_t)(cap + 1) * 4);
    w.off = reinterpret_cast<int *>(p); p += align256((size_t)(cap + 1) * 4);
    w.cur = reinterpret_cast<int *>(p); p += align256((size_t)(cap + 1) * 4);
    w.big = reinterpret_cast<int *>(p); p += align256((size_t)(cap + 1) * 4);
    w.nbig = reinterpret_cast<int *>(p); p += 256;
    w.tmp = p; p += scan_tmp_bytes(cap);
    w.list = reinterpret_cast<int *>(p);
    return w;
}

}  // namespace

size_t vote_z_workspace_bytes(const DevGeom &, int n, int cap)
{
    return 4 * align256((size_t)(cap + 1) * 4) + 256 + scan_tmp_bytes(cap) +
           align256((size_t)(n > 0 ? n : 1) * 4);
}

size_t z_big_smem(const DevGeom &G) { return (size_t)G.n_z0 * G.n_cot * 4; }

cudaError_t prepare_z_kernels(int max_smem)
{
    const void *fns[] = {(const void *)k_z_big, (const void *)k_zb_big};
    for (const void *f : fns) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_smem - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Batch z vote: candidates of all n_ev event slots at once (global id
// e * cap + m), hits grouped per candidate with batch-wide indices.
size_t vote_z_batch_workspace_bytes(int n_ev, int cap, int max_hits)
{
    const size_t ng = (size_t)n_ev * cap;
    return 4 * align256((ng + 1) * 4) + 256 + scan_tmp_bytes((int)ng) +
           align256((size_t)(max_hits > 0 ? max_hits : 1) * 4);
}

cudaError_t launch_vote_z_batch(const DevGeom &G, const float *x, const float *y, const float *z,
                                const int *assign, const int *off, const int *d_nev,
                                const ht_peak *peaks, const int *counts, int cap, int n_ev,
                                ht_zres *out, void *ws, int max_hits, cudaStream_t st)
{
    const size_t ng = (size_t)n_ev * cap;
    char *p = reinterpret_cast<char *>(ws);
    int *cnt = reinterpret_cast<int *>(p); p += align256((ng + 1) * 4);
    int *zoff = reinterpret_cast<int *>(p); p += align256((ng + 1) * 4);
    int *cur = reinterpret_cast<int *>(p); p += align256((ng + 1) * 4);
    int *big = reinterpret_cast<int *>(p); p += align256((ng + 1) * 4);
    int *nbig = reinterpret_cast<int *>(p); p += 256;
    void *tmp = p; p += scan_tmp_bytes((int)ng);
    int *list = reinterpret_cast<int *>(p);
    cudaError_t e = cudaMemsetAsync(cnt, 0, (ng + 1) * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(nbig, 0, 4, st);
    if (e != cudaSuccess) return e;
    const int nb = min(4096, max_hits / 256 + 1);
    k_zb_group<<<nb, 256, 0, st>>>(assign, off, d_nev, counts, cap, cnt, nullptr, nullptr);
    e = scan_exclusive(cnt, zoff, cur, (int)ng, nullptr, nullptr, tmp, st);
    if (e != cudaSuccess) return e;
    k_zb_group<<<nb, 256, 0, st>>>(assign, off, d_nev, counts, cap, nullptr, cur, list);
    dim3 gs(max(1, min(device_sms() * 8 / max(n_ev, 1), 1024)), n_ev);
    k_zb_small<<<gs, 256, 0, st>>>(G, x, y, z, peaks, counts, d_nev, cap, zoff, list, out, big,
                                   nbig);
    k_zb_big<<<device_sms() * 2, kBigThreads, z_big_smem(G), st>>>(G, x, y, z, peaks, zoff, list, big,
                                                           nbig, out);
    return cudaGetLastError();
}

cudaError_t launch_vote_z(const DevGeom &G, const float *x, const float *y, const float *z,
                          int n, const int *assign, const ht_peak *peaks, const int *d_count,
                          int cap, ht_zres *out, void *ws, cudaStream_t st)
{
    if (cap == 0) return cudaSuccess;
    ZWs w = carve(ws, n, cap);
    cudaError_t e = cudaMemsetAsync(w.cnt, 0, (size_t)(cap + 1) * 4, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(w.nbig, 0, 4, st);
    if (e != cudaSuccess) return e;
    const int nb = n > 0 ? min(4096, (n + 255) / 256) : 1;
    if (n > 0) k_z_count<<<nb, 256, 0, st>>>(assign, n, d_count, cap, w.cnt);
    e = scan_exclusive(w.cnt, w.off, w.cur, cap, d_count, nullptr, w.tmp, st);
    if (e != cudaSuccess) return e;
    if (n > 0) k_z_scatter<<<nb, 256, 0, st>>>(assign, n, d_count, cap, w.cur, w.list);
    const int warps_needed = cap;
    const int blocks = min(device_sms() * 16, (warps_needed + 7) / 8);
    k_z_small<<<blocks, 256, 0, st>>>(G, x, y, z, peaks, d_count, cap, w.off, w.list, out, w.big,
                                      w.nbig);
    k_z_big<<<device_sms() * 2, kBigThreads, z_big_smem(G), st>>>(G, x, y, z, peaks, w.off, w.list, w.big,
                                                          w.nbig, out);
    return cudaGetLastError();
}

}  // namespace ht
