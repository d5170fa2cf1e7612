// k_peaks.cu -- 3x3x3 local-maximum peak finding over the accumulator with
// order-preserving compaction (Sections 5-7 of arXiv:1309.6275: candidates
// are the local maxima of the vote space; the threshold reflects the peak
// finder's tuning for tracks of 7 or more hits).
//
// Design (GB300, HBM-bound stencil):
//  * A CTA of 256 threads owns one segment row (i, j-block, k-block): thread
//    = phi0 column k, and the CTA walks d0 bins j over its block keeping a
//    rolling 3 (rho) x 3 (d0) x 3 (phi0) window in registers, so each step
//    loads one new d0 slice (9 coalesced loads per thread, neighbours in
//    phi0 served from L1).  Rows beyond rho/d0 edges read as absent; phi0
//    wraps.
//  * Compaction keeps increasing logical index l = (i n_d0 + j) n_phi0 + k:
//    pass 1 counts the peaks of every (i, j, k-block) segment, a
//    device-wide scan turns counts into offsets (and the total), pass 2
//    recomputes and writes each peak at its segment offset plus its rank in
//    the CTA (warp ballots + a per-warp prefix).  Segments are ordered by l,
//    so the output is too.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ht_internal.cuh"

namespace ht {

constexpr int kPkThreads = 256;   // phi0 columns per CTA

namespace {

constexpr int kJB = 16;           // d0 bins walked per CTA

// MASKED: only cells inside *mask (a learned proposal's regions) can be
// peaks; a CTA whose bins are all outside reads nothing.  An inside cell's
// 26 neighbours lie in the mask's halo, which the masked vote fills exactly.
template <typename T, bool WRITE, bool MASKED>
__global__ void __launch_bounds__(kPkThreads)
k_peaks(DevGeom G, const T *__restrict__ acc, int *__restrict__ segcnt,
        const int *__restrict__ segoff, ht_peak *__restrict__ out, int cap,
        const unsigned long long *__restrict__ mask)
{
    const int NP = G.n_phi0, ND = G.n_d0, NR = G.n_rho;
    const int nkb = (NP + kPkThreads - 1) / kPkThreads;
    const int kb = blockIdx.x, i = blockIdx.z;
    const int k = kb * kPkThreads + threadIdx.x;
    const bool kok = k < NP;
    const int km = (k == 0) ? NP - 1 : k - 1;
    const int kp = (k >= NP - 1) ? 0 : k + 1;
    const int j0 = blockIdx.y * kJB, j1 = min(j0 + kJB, ND);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ int wcnt[kPkThreads / 32];
    unsigned inside = 0xffu;   // d0 blocks inside the mask in row i's rho block
    if (MASKED) {
        inside = (unsigned)(*mask >> (8 * region_block(i, NR))) & 0xffu;
        const int b0 = region_block(j0, ND), b1 = region_block(j1 - 1, ND);
        if (!(inside & ((2u << b1) - 1u) & ~((1u << b0) - 1u))) {
            if (!WRITE)
                for (int j = j0 + threadIdx.x; j < j1; j += kPkThreads)
                    segcnt[(i * ND + j) * nkb + kb] = 0;
            return;   // uniform over the CTA
        }
    }

    int w[3][3][3];  // [rho -1..+1][d0 -1..+1][phi0 -1..+1]; -1 = absent
    auto load = [&](int slot, int jj) {
#pragma unroll
        for (int di = 0; di < 3; ++di) {
            const int ii = i + di - 1;
            const bool ok = kok && ii >= 0 && ii < NR && jj >= 0 && jj < ND;
            const size_t rowb = ok ? ((size_t)ii * ND + jj) * NP : 0;
            w[di][slot][0] = ok ? (int)acc[rowb + km] : -1;
            w[di][slot][1] = ok ? (int)acc[rowb + k] : -1;
            w[di][slot][2] = ok ? (int)acc[rowb + kp] : -1;
        }
    };
    load(0, j0 - 1);
    load(1, j0);
    for (int j = j0; j < j1; ++j) {
        load(2, j + 1);
        const int v = w[1][1][1];
        bool pk = kok && v >= G.threshold &&
                  (!MASKED || ((inside >> region_block(j, ND)) & 1u));
        // rows i-1 and d0 bin j-1 (at row i) precede l: strictly greater;
        // rows i+1 and d0 bin j+1 follow l: greater or equal.
#pragma unroll
        for (int dj = 0; dj < 3; ++dj)
#pragma unroll
            for (int dk = 0; dk < 3; ++dk) {
                pk = pk && (v > w[0][dj][dk]) && (v >= w[2][dj][dk]);
            }
#pragma unroll
        for (int dk = 0; dk < 3; ++dk) pk = pk && (v > w[1][0][dk]) && (v >= w[1][2][dk]);
        // same (i, j): phi0 neighbours; their order flips across the wrap
        pk = pk && ((k != 0) ? (v > w[1][1][0]) : (v >= w[1][1][0]));
        pk = pk && ((k != NP - 1) ? (v >= w[1][1][2]) : (v > w[1][1][2]));

        const int seg = (i * ND + j) * nkb + kb;
        if (!WRITE) {
            const int c = __syncthreads_count(pk);
            if (threadIdx.x == 0) segcnt[seg] = c;
        } else {
            const unsigned bal = __ballot_sync(0xffffffffu, pk);
            if (lane == 0) wcnt[warp] = __popc(bal);
            __syncthreads();
            int pos = segoff[seg] + __popc(bal & ((1u << lane) - 1u));
            for (int w2 = 0; w2 < warp; ++w2) pos += wcnt[w2];
            if (pk && pos < cap) out[pos] = ht_peak{i, j, k, v};
            __syncthreads();
        }
#pragma unroll
        for (int di = 0; di < 3; ++di)
#pragma unroll
            for (int dk = 0; dk < 3; ++dk) {
                w[di][0][dk] = w[di][1][dk];
                w[di][1][dk] = w[di][2][dk];
            }
    }
}

template <typename T, bool MASKED>
cudaError_t run_peaks(const DevGeom &G, const T *acc, ht_peak *peaks, int cap, int *d_count,
                      int *segcnt, int *segoff, void *tmp, const unsigned long long *mask,
                      cudaStream_t st)
{
    const int nkb = (G.n_phi0 + kPkThreads - 1) / kPkThreads;
    dim3 grid(nkb, (G.n_d0 + kJB - 1) / kJB, G.n_rho);
    const int nseg = G.n_rho * G.n_d0 * nkb;
    k_peaks<T, false, MASKED><<<grid, kPkThreads, 0, st>>>(G, acc, segcnt, nullptr, nullptr, 0,
                                                           mask);
    cudaError_t e = scan_exclusive(segcnt, segoff, nullptr, nseg, nullptr, d_count, tmp, st);
    if (e != cudaSuccess) return e;
    k_peaks<T, true, MASKED><<<grid, kPkThreads, 0, st>>>(G, acc, nullptr, segoff, peaks, cap,
                                                          mask);
    return cudaGetLastError();
}

}  // namespace

size_t peaks_workspace_bytes(const DevGeom &G)
{
    const size_t nkb = (G.n_phi0 + kPkThreads - 1) / kPkThreads;
    const size_t nseg = (size_t)G.n_rho * G.n_d0 * nkb;
    return 2 * align256((nseg + 1) * 4) + scan_tmp_bytes((int)nseg);
}

cudaError_t launch_peaks(const DevGeom &G, const void *acc, ht_peak *peaks, int cap,
                         int *d_count, void *ws, cudaStream_t st, const unsigned long long *mask)
{
    const size_t nkb = (G.n_phi0 + kPkThreads - 1) / kPkThreads;
    const size_t nseg = (size_t)G.n_rho * G.n_d0 * nkb;
    char *p = reinterpret_cast<char *>(ws);
    int *segcnt = reinterpret_cast<int *>(p);
    int *segoff = reinterpret_cast<int *>(p + align256((nseg + 1) * 4));
    void *tmp = p + 2 * align256((nseg + 1) * 4);
    const uint16_t *a16 = reinterpret_cast<const uint16_t *>(acc);
    const int32_t *a32 = reinterpret_cast<const int32_t *>(acc);
    if (mask) {
        if (G.count_bits == 16)
            return run_peaks<uint16_t, true>(G, a16, peaks, cap, d_count, segcnt, segoff, tmp,
                                             mask, st);
        return run_peaks<int32_t, true>(G, a32, peaks, cap, d_count, segcnt, segoff, tmp, mask,
                                        st);
    }
    if (G.count_bits == 16)
        return run_peaks<uint16_t, false>(G, a16, peaks, cap, d_count, segcnt, segoff, tmp,
                                          nullptr, st);
    return run_peaks<int32_t, false>(G, a32, peaks, cap, d_count, segcnt, segoff, tmp, nullptr,
                                     st);
}

}  // namespace ht

// ---------------------------------------------------------------------------
// Peak finding without any allocation (ht_find_peaks_noalloc in ht.h).
//
// The scratch that ht_find_peaks takes from the caller's workspace -- one
// count and one offset per (rho row, d0 bin, phi0 block of 256) segment plus
// the scan's block sums -- lives here in a file-scope device array, sized
// for at most kNoallocMaxSegments segments.  Every GPU that loads the library
// holds it until the process exits.  The array's name is only a host-side
// stand-in in host code, so its device address is looked up once per device
// with cudaGetSymbolAddress (on the first call made with that device
// current) and passed to the kernels.  Nothing in it needs clearing between
// calls: each word a call reads was written earlier in the same call.
#include <mutex>

namespace {

constexpr int kNoallocMaxSegments = 1 << 19;
constexpr size_t kNoallocSegBytes = ht::align256(((size_t)kNoallocMaxSegments + 1) * 4);
constexpr size_t kNoallocScratchBytes =
    2 * kNoallocSegBytes + ht::align256(((size_t)kNoallocMaxSegments / 4096 + 2) * 4);
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::once_flag g_noalloc_once[kNoallocMaxDevices];
void *g_noalloc_ptr[kNoallocMaxDevices];
cudaError_t g_noalloc_status[kNoallocMaxDevices];

}  // namespace

extern "C" ht_status ht_find_peaks_noalloc(const ht_geometry *g, const void *acc, ht_peak *peaks,
                                           int32_t cap, int32_t *d_count, ht_stream stream)
{
    if (!g || !acc || !d_count || (cap > 0 && !peaks))
        return ht::set_error(HT_ERR_ARG, "ht_find_peaks_noalloc: null argument");
    if (cap < 0) return ht::set_error(HT_ERR_ARG, "ht_find_peaks_noalloc: cap < 0");
    const size_t nkb = (g->G.n_phi0 + ht::kPkThreads - 1) / ht::kPkThreads;
    const size_t nseg = (size_t)g->G.n_rho * g->G.n_d0 * nkb;
    if (nseg > (size_t)kNoallocMaxSegments)
        return ht::set_error(HT_ERR_CAPACITY,
                             "ht_find_peaks_noalloc: geometry has more than 524288 segments "
                             "(n_rho * n_d0 * ceil(n_phi0 / 256)); use ht_find_peaks");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ht::set_error(HT_ERR_CUDA, "ht_find_peaks_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kNoallocMaxDevices)
        return ht::set_error(HT_ERR_ARG, "ht_find_peaks_noalloc: device index above 63");
    std::call_once(g_noalloc_once[dev], [dev] {
        g_noalloc_status[dev] = cudaGetSymbolAddress(&g_noalloc_ptr[dev], g_noalloc_scratch);
    });
    if (g_noalloc_status[dev] != cudaSuccess)
        return ht::set_error(HT_ERR_CUDA,
                             "ht_find_peaks_noalloc: cudaGetSymbolAddress of the scratch failed");
    e = ht::launch_peaks(g->G, acc, peaks, cap, d_count, g_noalloc_ptr[dev],
                         reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return ht::set_error(HT_ERR_CUDA, cudaGetErrorString(e));
    return HT_OK;
}
