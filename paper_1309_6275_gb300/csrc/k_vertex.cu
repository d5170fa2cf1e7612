// k_vertex.cu -- the second Hough transform (ht_vertex_* in include/ht.h):
// candidate tracks vote for displaced vertices (Section 6, Fig. 6: tracks
// from one vertex lie on a sinusoid in track-parameter space), the peak
// finder of Sections 5-7 runs on the vertex space, and peaks inside the beam
// pipe are dropped (Section 7).
//
// Readings: a candidate is the straight line of its cell centre (perigee
// d0 n, n = (-sin phi0, cos phi0)); a vertex r (cos theta, sin theta) lies
// on it iff d0 = r sin(theta - phi0).  For every theta column the candidate
// votes at r = d0 / (sin theta cos phi0 - cos theta sin phi0) if
// 0 <= r / dr < n_r.
//
// Design (GB300): one CTA per (event, 32 theta columns), lane = theta
// column, warps stride over the event's candidates.  Counters [r][32] live
// in shared memory (a warp's 32 atomics fall in 32 banks whatever the radius
// bins).  Arithmetic: float32 with a first-order error bound; a column it
// cannot prove (rare) is redone in float64 in the definition's order, so the
// votes equal the float64 definition.  Integer counting, no tensor cores.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "ht_internal.cuh"

struct ht_vertex {
    ht_vertex_desc desc;
    const ht_geometry *g;
    ht::DevGeom P;     // the 1 x n_r x n_theta peak search
    float *d_t32;      // sin, cos theta [2][n_theta], then d0 of each bin [n_d0] (float32)
    double *d_t64;     // the same in float64
    double dr, d0_off;
    float inv_dr_f;
    int j_keep;        // first radius bin whose centre is >= r_keep
};

namespace ht {
namespace {

struct VtxArgs {
    const float *st32, *ct32;
    const double *st64, *ct64;
    const float *d0t32;           // d0 of candidate bin j: (j - n_d0/2) delta
    const double *d0t64;
    const float *sp32, *cp32;     // track geometry sin/cos phi0
    const double *sp64, *cp64;
    double delta, half_nd, dr;
    float inv_dr_f;
    int n_r, n_theta, min_count;
};

constexpr int kVtxThreads = 256;

__global__ void __launch_bounds__(kVtxThreads)
k_vertex_vote(VtxArgs A, const ht_peak *__restrict__ peaks, const int *__restrict__ counts,
              int cap, int *__restrict__ acc, unsigned long long *__restrict__ stats)
{
    extern __shared__ unsigned cnt[];   // [n_r][32]
    __shared__ unsigned long long s_st[2];
    const int e = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = blockIdx.x * 32 + lane;
    const float st = A.st32[q], ct = A.ct32[q];
    for (int t = threadIdx.x; t < A.n_r * 32; t += kVtxThreads) cnt[t] = 0u;
    if (threadIdx.x < 2) s_st[threadIdx.x] = 0ull;
    __syncthreads();
    const int nc = min(counts[e], cap);
    const ht_peak *pk = peaks + (size_t)e * cap;
    unsigned long long votes = 0, redo = 0;
    const float nr = (float)A.n_r;
    // candidate records are loaded one step ahead of their use
    constexpr int kStep = kVtxThreads / 32;
    ht_peak nxt = warp < nc ? pk[warp] : ht_peak{0, 0, 0, 0};
    for (int m = warp; m < nc; m += kStep) {
        const ht_peak p = nxt;
        if (m + kStep < nc) nxt = pk[m + kStep];
        if (p.count < A.min_count) continue;           // uniform over the warp
        const double d0 = A.d0t64[p.j_d0];             // (j - n_d0/2) delta, as defined
        const float d0f = A.d0t32[p.j_d0];
        const float sp = A.sp32[p.k_phi0], cp = A.cp32[p.k_phi0];
        const float den = fmaf(st, cp, -(ct * sp));
        const float aden = fabsf(den);
        int bin;
        if (d0 == 0.0) {
            // r = +-0: bin 0 whenever the float64 denominator is not zero
            bin = aden > 8.0f * kEps ? 0 : -2;
        } else {
            const float u = __fdividef(d0f, den) * A.inv_dr_f;
            // |den error| <= 4u (|s c| + |c s| <= 1); d0, the division, 1/dr
            // and the product add 5u relative; x kSafe
            const float eb = fabsf(u) * (kSafe * kEps) * (4.0f / aden + 6.0f);
            bin = decide(u, eb, nr);
        }
        if (bin == -2) {
            ++redo;
            const double den64 = __dsub_rn(__dmul_rn(A.st64[q], A.cp64[p.k_phi0]),
                                           __dmul_rn(A.ct64[q], A.sp64[p.k_phi0]));
            const double u64 = __ddiv_rn(__ddiv_rn(d0, den64), A.dr);
            bin = (u64 >= 0.0 && u64 < (double)A.n_r) ? (int)floor(u64) : -1;
        }
        if (bin >= 0) {
            atomicAdd(&cnt[bin * 32 + lane], 1u);
            ++votes;
        }
    }
    __syncthreads();
    int *out = acc + (size_t)e * A.n_r * A.n_theta + blockIdx.x * 32;
    for (int t = threadIdx.x; t < A.n_r * 32; t += kVtxThreads)
        out[(size_t)(t >> 5) * A.n_theta + (t & 31)] = (int)cnt[t];
    if (stats) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            votes += __shfl_xor_sync(0xffffffffu, votes, o);
            redo += __shfl_xor_sync(0xffffffffu, redo, o);
        }
        if (lane == 0) {
            atomicAdd(&s_st[0], votes);
            atomicAdd(&s_st[1], redo);
        }
        __syncthreads();
        if (threadIdx.x < 2) atomicAdd(&stats[2 * e + threadIdx.x], s_st[threadIdx.x]);
    }
}

// first[e] = index of the first peak of event e outside the beam-pipe radius
// (peaks are in radius-bin-major order, so the ones inside are a prefix).
__global__ void k_vertex_first(const ht_peak *__restrict__ peaks, const int *__restrict__ counts,
                               int cap, int n_ev, int j_keep, int *__restrict__ first)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_ev) return;
    const ht_peak *pk = peaks + (size_t)e * cap;
    int lo = 0, hi = min(counts[e], cap);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pk[mid].j_d0 < j_keep) lo = mid + 1;
        else hi = mid;
    }
    first[e] = lo;
}

ht_status vfail(ht_status s, const char *msg) { return set_error(s, msg); }

}  // namespace
}  // namespace ht

extern "C" {

ht_status ht_vertex_create(const ht_geometry *g, const ht_vertex_desc *d, ht_vertex **out)
{
    if (!g || !d || !out) return ht::vfail(HT_ERR_ARG, "ht_vertex_create: null argument");
    *out = nullptr;
    if (d->n_r < 1 || d->n_r > 4096 || d->n_theta < 32 || d->n_theta % 32 != 0 ||
        d->n_theta > 65536 || d->threshold < 1 || !(d->r_max > 0.0) || !(d->r_keep >= 0.0) ||
        (double)d->n_r * d->n_theta > 2147483647.0)
        return ht::vfail(HT_ERR_ARG, "ht_vertex_create: descriptor out of range");
    ht_vertex *v = new (std::nothrow) ht_vertex();
    if (!v) return ht::vfail(HT_ERR_ARG, "ht_vertex_create: out of host memory");
    v->desc = *d;
    v->g = g;
    const int NT = d->n_theta;
    v->dr = d->r_max / (double)d->n_r;
    v->inv_dr_f = (float)(1.0 / v->dr);
    v->d0_off = 0.5 * (double)g->desc.n_d0;
    int jk = 0;
    while (jk < d->n_r && ((double)jk + 0.5) * v->dr < d->r_keep) ++jk;
    v->j_keep = jk;
    const int ND = g->desc.n_d0;
    std::vector<double> t64(2 * NT + ND);
    std::vector<float> t32(2 * NT + ND);
    for (int q = 0; q < NT; ++q) {
        const double th = (double)(2 * q + 1 - NT) * (ht::kPi / (double)NT);
        t64[q] = sin(th);
        t64[NT + q] = cos(th);
        t32[q] = (float)t64[q];
        t32[NT + q] = (float)t64[NT + q];
    }
    for (int j = 0; j < ND; ++j) {   // the same two float64 operations as the definition
        t64[2 * NT + j] = ((double)j - v->d0_off) * g->G.delta;
        t32[2 * NT + j] = (float)t64[2 * NT + j];
    }
    const size_t nt = (size_t)2 * NT + ND;
    cudaError_t e = cudaMalloc((void **)&v->d_t64, sizeof(double) * nt);
    if (e == cudaSuccess) e = cudaMalloc((void **)&v->d_t32, sizeof(float) * nt);
    if (e == cudaSuccess)
        e = cudaMemcpy(v->d_t64, t64.data(), sizeof(double) * nt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(v->d_t32, t32.data(), sizeof(float) * nt, cudaMemcpyHostToDevice);
    int dev = 0, max_smem = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess && (size_t)d->n_r * 32 * 4 + 1024 > (size_t)max_smem) {
        cudaFree(v->d_t64);
        cudaFree(v->d_t32);
        delete v;
        return ht::vfail(HT_ERR_ARG, "ht_vertex_create: n_r too large for shared memory");
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ht::k_vertex_vote, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_smem - 1024);
    if (e != cudaSuccess) {
        cudaFree(v->d_t64);
        cudaFree(v->d_t32);
        delete v;
        return ht::vfail(HT_ERR_CUDA, "ht_vertex_create: device set-up failed");
    }
    memset(&v->P, 0, sizeof v->P);
    v->P.n_rho = 1;
    v->P.n_d0 = d->n_r;
    v->P.n_phi0 = NT;
    v->P.threshold = d->threshold;
    v->P.count_bits = 32;
    *out = v;
    return HT_OK;
}

ht_status ht_vertex_destroy(ht_vertex *v)
{
    if (!v) return HT_OK;
    cudaFree(v->d_t64);
    cudaFree(v->d_t32);
    delete v;
    return HT_OK;
}

size_t ht_vertex_accumulator_bytes(const ht_vertex *v)
{
    return v ? (size_t)v->desc.n_r * v->desc.n_theta * sizeof(int32_t) : 0;
}

size_t ht_vertex_workspace_size(const ht_vertex *v)
{
    return v ? ht::peaks_workspace_bytes(v->P) : 0;
}

ht_status ht_vertex_vote(const ht_vertex *v, const ht_peak *cands, const int32_t *d_count,
                         int32_t cap, int32_t n_events, int32_t *acc, uint64_t *stats,
                         ht_stream stream)
{
    if (!v || !d_count || !acc || n_events < 1 || cap < 0 || (cap > 0 && !cands))
        return ht::vfail(HT_ERR_ARG, "ht_vertex_vote: bad argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const ht::DevGeom &G = v->g->G;
    ht::VtxArgs A;
    A.st32 = v->d_t32;
    A.ct32 = v->d_t32 + v->desc.n_theta;
    A.st64 = v->d_t64;
    A.ct64 = v->d_t64 + v->desc.n_theta;
    A.d0t32 = v->d_t32 + 2 * v->desc.n_theta;
    A.d0t64 = v->d_t64 + 2 * v->desc.n_theta;
    A.sp32 = G.sn32;
    A.cp32 = G.cs32;
    A.sp64 = G.sn64;
    A.cp64 = G.cs64;
    A.delta = G.delta;
    A.half_nd = v->d0_off;
    A.dr = v->dr;
    A.inv_dr_f = v->inv_dr_f;
    A.n_r = v->desc.n_r;
    A.n_theta = v->desc.n_theta;
    A.min_count = v->desc.min_count;
    cudaError_t e = cudaSuccess;
    if (stats) e = cudaMemsetAsync(stats, 0, (size_t)n_events * 16, st);
    if (e == cudaSuccess) {
        dim3 grid(v->desc.n_theta / 32, n_events);
        ht::k_vertex_vote<<<grid, ht::kVtxThreads, (size_t)v->desc.n_r * 32 * 4, st>>>(
            A, cands, d_count, cap, acc, reinterpret_cast<unsigned long long *>(stats));
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? HT_OK : ht::vfail(HT_ERR_CUDA, cudaGetErrorString(e));
}

ht_status ht_vertex_find(const ht_vertex *v, const int32_t *acc, int32_t n_events, ht_peak *out,
                         int32_t cap, int32_t *d_count, int32_t *d_first, void *workspace,
                         size_t workspace_bytes, ht_stream stream)
{
    if (!v || !acc || !d_count || !d_first || !workspace || n_events < 1 || cap < 0 ||
        (cap > 0 && !out))
        return ht::vfail(HT_ERR_ARG, "ht_vertex_find: bad argument");
    if (workspace_bytes < ht::peaks_workspace_bytes(v->P) ||
        reinterpret_cast<uintptr_t>(workspace) % 256 != 0 ||
        reinterpret_cast<uintptr_t>(acc) % 16 != 0)
        return ht::vfail(HT_ERR_ARG, "ht_vertex_find: workspace size or alignment");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t cells = (size_t)v->desc.n_r * v->desc.n_theta;
    cudaError_t e = cudaSuccess;
    for (int ev = 0; ev < n_events && e == cudaSuccess; ++ev)
        e = ht::launch_peaks(v->P, acc + ev * cells, out + (size_t)ev * cap, cap, d_count + ev,
                             workspace, st);
    if (e == cudaSuccess) {
        ht::k_vertex_first<<<(n_events + 127) / 128, 128, 0, st>>>(out, d_count, cap, n_events,
                                                                    v->j_keep, d_first);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? HT_OK : ht::vfail(HT_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
