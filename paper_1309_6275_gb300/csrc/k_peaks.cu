// k_peaks.cu -- 3x3x3 local-maximum peak finding over the accumulator with
// order-preserving compaction (Sections 5-7 of arXiv:1309.6275: candidates
// are the local maxima of the vote space; the threshold reflects the peak
// finder's tuning for tracks of at least seven hits).
//
// Design (GB300, HBM-bound stencil):
//  * A CTA of 256 threads owns one segment row (i, j-block of 16 d0 bins,
//    block of 256 phi0 columns).  It first stages rows i-1..i+1 x bins
//    j0-1..j0+16 x its columns plus one wrapped column on each side into
//    shared memory with 16-byte loads, all issued before any is used, so a
//    CTA waits for memory once instead of once per d0 bin; absent rows and
//    bins read as -1.  Then thread = phi0 column walks the bins keeping, per
//    row and bin of the rolling 3 x 3 x 3 window, the largest of its three
//    columns (9 shared loads and 3 three-input maxima per cell); the 26
//    comparisons become two against the maxima of the preceding and of the
//    following neighbours.
//  * Compaction keeps increasing logical index l = (i n_d0 + j) n_phi0 + k:
//    pass 1 counts the peaks of every (i, j, k-block) segment, a
//    device-wide scan turns counts into offsets (and the total), pass 2
//    recomputes and writes each peak at its segment offset plus its rank in
//    the CTA (warp ballots kept per bin, one barrier per pass).  Segments
//    are ordered by l, so the output is too.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ht_internal.cuh"

namespace ht {

constexpr int kPkThreads = 256;   // phi0 columns per CTA

namespace {

constexpr int kJB = 16;                         // d0 bins per CTA
constexpr int kSlices = 3 * (kJB + 2);          // staged (row, bin) slices

// A staged slice holds the CTA's columns at [kOff, kOff + 256) -- 16-byte
// aligned, so a 16-byte global load lands in one 16-byte shared store --
// with the wrapped neighbour columns at kOff - 1 and kOff + ncol.
template <typename T>
struct Stage {
    static constexpr int kOff = 16 / (int)sizeof(T);
    static constexpr int kSW = kPkThreads + 2 * kOff;   // elements per slice
    static constexpr size_t kBytes = (size_t)kSlices * kSW * sizeof(T);
};
constexpr size_t kPkSmemMax = Stage<int32_t>::kBytes;

// Spilled peaks (single stencil pass): the count pass also writes the
// peaks of every tile that has at most q of them into the tile's q slots, in
// the tile's l order, with each peak's rank within its segment; tiletot
// holds every tile's peak count.  The write pass then copies a spilled tile's
// peaks to their segment offsets and runs the stencil again only for tiles
// with more than q peaks.  q == 0: no spill (every tile's stencil runs
// twice).
struct PeakSpill {
    ht_peak *pk;
    int *rk;
    int *tiletot;
    int q;
};

// One tile: (rho row i, 16 d0 bins from j0 = jb * kJB, 256 phi0 columns
// from k0 = kb * kPkThreads), tile index t.  Count pass (!WRITE): the
// segment counts, the tile's total and, when sp.q allows, the spilled peaks.
// Write pass: every peak at its segment offset.
//
// MASKED: only cells inside *mask (a learned proposal's regions) can be
// peaks; a tile whose bins are all outside reads nothing.  An inside cell's
// 26 neighbours lie in the mask's halo, which the masked vote fills exactly.
template <typename T, bool WRITE, bool MASKED>
__device__ __forceinline__ void peaks_tile(const DevGeom &G, const T *__restrict__ acc, int kb,
                                           int jb, int i, int t, int thr,
                                           int *__restrict__ segcnt,
                                           const int *__restrict__ segoff,
                                           ht_peak *__restrict__ out, int cap,
                                           const unsigned long long *__restrict__ mask,
                                           const PeakSpill &sp, T *sw,
                                           unsigned (*bal_s)[kPkThreads / 32], int *s_jpre)
{
    constexpr int kOff = Stage<T>::kOff, kSW = Stage<T>::kSW;
    const int NP = G.n_phi0, ND = G.n_d0, NR = G.n_rho;
    const int nkb = (NP + kPkThreads - 1) / kPkThreads;
    const int k0 = kb * kPkThreads, ncol = min(kPkThreads, NP - k0);
    const int j0 = jb * kJB, j1 = min(j0 + kJB, ND);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned inside = 0xffu;   // d0 blocks inside the mask in row i's rho block
    if (MASKED) {
        inside = (unsigned)(*mask >> (8 * region_block(i, NR))) & 0xffu;
        const int b0 = region_block(j0, ND), b1 = region_block(j1 - 1, ND);
        if (!(inside & ((2u << b1) - 1u) & ~((1u << b0) - 1u))) {
            if (!WRITE) {
                for (int j = j0 + threadIdx.x; j < j1; j += kPkThreads)
                    segcnt[(i * ND + j) * nkb + kb] = 0;
                if (sp.q > 0 && threadIdx.x == 0) sp.tiletot[t] = 0;
            }
            return;   // uniform over the CTA
        }
    }

    // ---- stage the window: interior columns with 16-byte loads and stores.
    // Absent rows and bins read as 0: a peak has v >= threshold >= 1, so a 0
    // neighbour never decides a comparison (as no neighbour at all).
    constexpr int VEC = 16 / (int)sizeof(T);
    const int nvec = ncol / VEC;                         // ncol is a multiple of 8
    for (int v = threadIdx.x; v < kSlices * nvec; v += kPkThreads) {
        const int sl = v / nvec, q = v - sl * nvec;
        const int ii = i - 1 + sl / (kJB + 2), jj = j0 - 1 + sl % (kJB + 2);
        uint4 u = make_uint4(0, 0, 0, 0);
        if (ii >= 0 && ii < NR && jj >= 0 && jj < ND)
            u = *reinterpret_cast<const uint4 *>(acc + ((size_t)ii * ND + jj) * NP + k0 + q * VEC);
        *reinterpret_cast<uint4 *>(sw + sl * kSW + kOff + q * VEC) = u;
    }
    // the two wrapped neighbour columns of every slice
    for (int v = threadIdx.x; v < 2 * kSlices; v += kPkThreads) {
        const int sl = v >> 1, side = v & 1;
        const int ii = i - 1 + sl / (kJB + 2), jj = j0 - 1 + sl % (kJB + 2);
        const int kk = side ? (k0 + ncol) % NP : (k0 + NP - 1) % NP;
        const bool ok = ii >= 0 && ii < NR && jj >= 0 && jj < ND;
        sw[sl * kSW + (side ? kOff + ncol : kOff - 1)] =
            ok ? acc[((size_t)ii * ND + jj) * NP + kk] : (T)0;
    }
    __syncthreads();

    // ---- walk the bins.  cm[r][s]: largest of columns k-1, k, k+1 in row
    // i-1+r at bin j-1+s; c1/n1: the three columns of row i at bins j and
    // j+1.  A cell is a peak when v >= T, v exceeds every neighbour that
    // precedes it in l (row i-1, bin j-1 of row i, column k-1 of its own
    // bin) and is at least every neighbour that follows it (row i+1, bin j+1,
    // column k+1) -- the two maxima below; across the phi0 wrap the order of
    // the column neighbours flips.
    const int c = threadIdx.x;
    const bool cok = c < ncol;
    const int k = k0 + c;
    const int cc = cok ? c : 0;                           // stays inside the staged row
    // q[-1], q[0], q[1]: columns k - 1, k, k + 1 of slice (r, jj)
    auto S = [&](int r, int jj) -> const T * {
        return sw + (r * (kJB + 2) + jj) * kSW + kOff + cc;
    };
    int cm[3][3], c1[3], n1[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
            const T *q = S(r, sl);
            const int a = (int)q[-1], b = (int)q[0], d = (int)q[1];
            cm[r][sl] = __vimax3_s32(a, b, d);
            if (r == 1 && sl == 1) { c1[0] = a; c1[1] = b; c1[2] = d; }
        }
    const bool wrap_lo = k == 0, wrap_hi = k == NP - 1;
    unsigned mine = 0u;
    const int nj = j1 - j0;
#pragma unroll
    for (int jl = 0; jl < kJB; ++jl) {
        if (jl < nj) {   // uniform over the CTA
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const T *q = S(r, jl + 2);
                const int a = (int)q[-1], b = (int)q[0], d = (int)q[1];
                cm[r][2] = __vimax3_s32(a, b, d);
                if (r == 1) { n1[0] = a; n1[1] = b; n1[2] = d; }
            }
            const int v = c1[1];
            const int before = max(__vimax3_s32(cm[0][0], cm[0][1], cm[0][2]),
                                   __vimax3_s32(cm[1][0], wrap_lo ? 0 : c1[0],
                                                wrap_hi ? c1[2] : 0));
            const int after = max(__vimax3_s32(cm[2][0], cm[2][1], cm[2][2]),
                                  __vimax3_s32(cm[1][2], wrap_lo ? c1[0] : 0,
                                               wrap_hi ? 0 : c1[2]));
            const bool pk = cok && v >= thr && v > before && v >= after &&
                            (!MASKED || ((inside >> region_block(j0 + jl, ND)) & 1u));
            const unsigned bal = __ballot_sync(0xffffffffu, pk);
            if (lane == 0) bal_s[jl][warp] = bal;
            mine |= (unsigned)pk << jl;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                cm[r][0] = cm[r][1];
                cm[r][1] = cm[r][2];
            }
            c1[0] = n1[0]; c1[1] = n1[1]; c1[2] = n1[2];
        }
    }
    __syncthreads();
    // rank of the lane's peak in bin jl within its segment (CTA order = l order)
    auto seg_rank = [&](int jl) {
        int r = __popc(bal_s[jl][warp] & ((1u << lane) - 1u));
        for (int w2 = 0; w2 < warp; ++w2) r += __popc(bal_s[jl][w2]);
        return r;
    };
    if constexpr (!WRITE) {
        for (int jl = threadIdx.x; jl < nj; jl += kPkThreads) {
            int cnt = 0;
#pragma unroll
            for (int w2 = 0; w2 < kPkThreads / 32; ++w2) cnt += __popc(bal_s[jl][w2]);
            segcnt[(i * ND + j0 + jl) * nkb + kb] = cnt;
            if (sp.q > 0) s_jpre[jl + 1] = cnt;
        }
        if (sp.q > 0) {
            __syncthreads();
            if (threadIdx.x == 0) {
                s_jpre[0] = 0;
                for (int jl = 0; jl < nj; ++jl) s_jpre[jl + 1] += s_jpre[jl];
                sp.tiletot[t] = s_jpre[nj];
            }
            __syncthreads();
            if (s_jpre[nj] <= sp.q) {   // uniform
                while (mine) {
                    const int jl = __ffs(mine) - 1;
                    mine &= mine - 1u;
                    const int r = seg_rank(jl);
                    const size_t slot = (size_t)t * sp.q + s_jpre[jl] + r;
                    sp.pk[slot] = ht_peak{i, j0 + jl, k, (int)S(1, jl + 1)[0]};
                    sp.rk[slot] = r;
                }
            }
        }
    } else {
        while (mine) {
            const int jl = __ffs(mine) - 1;
            mine &= mine - 1u;
            const int pos = segoff[(i * ND + j0 + jl) * nkb + kb] + seg_rank(jl);
            if (pos < cap) out[pos] = ht_peak{i, j0 + jl, k, (int)S(1, jl + 1)[0]};
        }
    }
}

// d_thr (null: the geometry's threshold): a device threshold for this event.
// Count pass: one CTA per tile.
template <typename T, bool MASKED>
__global__ void __launch_bounds__(kPkThreads)
k_peaks_count(DevGeom G, const T *__restrict__ acc, int *__restrict__ segcnt,
              const unsigned long long *__restrict__ mask, const int *__restrict__ d_thr,
              PeakSpill sp)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ unsigned bal_s[kJB][kPkThreads / 32];
    __shared__ int s_jpre[kJB + 1];
    const int thr = d_thr ? *d_thr : G.threshold;
    const int t = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    peaks_tile<T, false, MASKED>(G, acc, blockIdx.x, blockIdx.y, blockIdx.z, t, thr, segcnt,
                                 nullptr, nullptr, 0, mask, sp, reinterpret_cast<T *>(smraw),
                                 bal_s, s_jpre);
}

// Write pass, persistent over the tiles: a spilled tile is copied, the
// others run the stencil again.
template <typename T, bool MASKED>
__global__ void __launch_bounds__(kPkThreads)
k_peaks_write(DevGeom G, const T *__restrict__ acc, const int *__restrict__ segoff,
              ht_peak *__restrict__ out, int cap, const unsigned long long *__restrict__ mask,
              const int *__restrict__ d_thr, PeakSpill sp, int nkb, int njb)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ unsigned bal_s[kJB][kPkThreads / 32];
    const int thr = d_thr ? *d_thr : G.threshold;
    const int ND = G.n_d0;
    const int ntiles = nkb * njb * G.n_rho;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int kb = t % nkb, jb = (t / nkb) % njb, i = t / (nkb * njb);
        if (sp.q > 0) {
            const int tot = sp.tiletot[t];
            if (tot <= sp.q) {   // uniform
                for (int r = threadIdx.x; r < tot; r += kPkThreads) {
                    const size_t slot = (size_t)t * sp.q + r;
                    const ht_peak pk = sp.pk[slot];
                    const int pos = segoff[(pk.i_rho * ND + pk.j_d0) * nkb + kb] + sp.rk[slot];
                    if (pos < cap) out[pos] = pk;
                }
                continue;
            }
        }
        peaks_tile<T, true, MASKED>(G, acc, kb, jb, i, t, thr, nullptr, segoff, out, cap, mask,
                                    sp, reinterpret_cast<T *>(smraw), bal_s, nullptr);
        __syncthreads();   // the staged window is refilled by the next tile
    }
}

template <typename T, bool MASKED>
cudaError_t run_peaks(const DevGeom &G, const T *acc, ht_peak *peaks, int cap, int *d_count,
                      int *segcnt, int *segoff, void *tmp, const unsigned long long *mask,
                      cudaStream_t st, const int *d_thr, const PeakSpill &sp)
{
    const int nkb = (G.n_phi0 + kPkThreads - 1) / kPkThreads;
    const int njb = (G.n_d0 + kJB - 1) / kJB;
    dim3 grid(nkb, njb, G.n_rho);
    const int nseg = G.n_rho * G.n_d0 * nkb;
    k_peaks_count<T, MASKED><<<grid, kPkThreads, Stage<T>::kBytes, st>>>(G, acc, segcnt, mask,
                                                                         d_thr, sp);
    cudaError_t e = scan_exclusive(segcnt, segoff, nullptr, nseg, nullptr, d_count, tmp, st);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_peaks_write<T, MASKED>,
                                                          kPkThreads, Stage<T>::kBytes);
    if (e != cudaSuccess) return e;
    const int ntiles = nkb * njb * G.n_rho;
    const int pgrid = min(ntiles, sms * (occ > 0 ? occ : 1));
    k_peaks_write<T, MASKED><<<pgrid, kPkThreads, Stage<T>::kBytes, st>>>(
        G, acc, segoff, peaks, cap, mask, d_thr, sp, nkb, njb);
    return cudaGetLastError();
}

}  // namespace

// The staged window needs more than the default 48 KB of dynamic shared
// memory.  Called once per device.
cudaError_t prepare_peaks_kernels()
{
    const void *fns[] = {
        (const void *)k_peaks_count<uint16_t, false>, (const void *)k_peaks_write<uint16_t, false>,
        (const void *)k_peaks_count<uint16_t, true>,  (const void *)k_peaks_write<uint16_t, true>,
        (const void *)k_peaks_count<int32_t, false>,  (const void *)k_peaks_write<int32_t, false>,
        (const void *)k_peaks_count<int32_t, true>,   (const void *)k_peaks_write<int32_t, true>};
    for (const void *f : fns) {
        const cudaError_t e =
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPkSmemMax);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t peaks_workspace_bytes(const DevGeom &G)
{
    const size_t nkb = (G.n_phi0 + kPkThreads - 1) / kPkThreads;
    const size_t nseg = (size_t)G.n_rho * G.n_d0 * nkb;
    return 2 * align256((nseg + 1) * 4) + scan_tmp_bytes((int)nseg);
}

// Spill slots per tile: a tile (one row, 16 bins, 256 columns) has at most
// 1024 peaks (no two peaks are neighbours), usually a few; tiles above this
// run the stencil twice.
constexpr int kSpillQ = 64;

size_t peak_spill_bytes(const DevGeom &G)
{
    const size_t nkb = (G.n_phi0 + kPkThreads - 1) / kPkThreads;
    const size_t nt = nkb * ((G.n_d0 + kJB - 1) / kJB) * G.n_rho;
    return align256(nt * 4) + align256(nt * kSpillQ * sizeof(ht_peak)) +
           align256(nt * kSpillQ * 4);
}

cudaError_t launch_peaks(const DevGeom &G, const void *acc, ht_peak *peaks, int cap,
                         int *d_count, void *ws, cudaStream_t st, const unsigned long long *mask,
                         const int *d_thr, void *spill)
{
    const size_t nkb = (G.n_phi0 + kPkThreads - 1) / kPkThreads;
    const size_t nseg = (size_t)G.n_rho * G.n_d0 * nkb;
    char *p = reinterpret_cast<char *>(ws);
    int *segcnt = reinterpret_cast<int *>(p);
    int *segoff = reinterpret_cast<int *>(p + align256((nseg + 1) * 4));
    void *tmp = p + 2 * align256((nseg + 1) * 4);
    PeakSpill sp{nullptr, nullptr, nullptr, 0};
    if (spill) {
        const size_t nt = nkb * ((G.n_d0 + kJB - 1) / kJB) * G.n_rho;
        char *q = reinterpret_cast<char *>(spill);
        sp.tiletot = reinterpret_cast<int *>(q);
        q += align256(nt * 4);
        sp.pk = reinterpret_cast<ht_peak *>(q);
        q += align256(nt * kSpillQ * sizeof(ht_peak));
        sp.rk = reinterpret_cast<int *>(q);
        sp.q = kSpillQ;
    }
    const uint16_t *a16 = reinterpret_cast<const uint16_t *>(acc);
    const int32_t *a32 = reinterpret_cast<const int32_t *>(acc);
    if (mask) {
        if (G.count_bits == 16)
            return run_peaks<uint16_t, true>(G, a16, peaks, cap, d_count, segcnt, segoff, tmp,
                                             mask, st, d_thr, sp);
        return run_peaks<int32_t, true>(G, a32, peaks, cap, d_count, segcnt, segoff, tmp, mask,
                                        st, d_thr, sp);
    }
    if (G.count_bits == 16)
        return run_peaks<uint16_t, false>(G, a16, peaks, cap, d_count, segcnt, segoff, tmp,
                                          nullptr, st, d_thr, sp);
    return run_peaks<int32_t, false>(G, a32, peaks, cap, d_count, segcnt, segoff, tmp, nullptr,
                                     st, d_thr, sp);
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
// stand-in in host code, so its device address is looked up per device with
// cudaGetSymbolAddress (on the first successful call made with that device
// current; a failed lookup is not cached, so the next call tries again) and
// passed to the kernels.  Nothing in it needs clearing between calls: each
// word a call reads was written earlier in the same call.
#include <mutex>

namespace {

constexpr int kNoallocMaxSegments = 1 << 19;
constexpr size_t kNoallocSegBytes = ht::align256(((size_t)kNoallocMaxSegments + 1) * 4);
constexpr size_t kNoallocScratchBytes =
    2 * kNoallocSegBytes + ht::align256(((size_t)kNoallocMaxSegments / 4096 + 2) * 4);
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kNoallocMaxDevices];   // null until a lookup on that device succeeds

}  // namespace

extern "C" ht_status ht_find_peaks_noalloc(const ht_geometry *g, const void *acc, ht_peak *peaks,
                                           int32_t cap, int32_t *d_count, ht_stream stream)
{
    if (!g || !acc || !d_count || (cap > 0 && !peaks))
        return ht::set_error(HT_ERR_ARG, "ht_find_peaks_noalloc: null argument");
    if (cap < 0) return ht::set_error(HT_ERR_ARG, "ht_find_peaks_noalloc: cap < 0");
    if (reinterpret_cast<uintptr_t>(acc) % 16 != 0)
        return ht::set_error(HT_ERR_ARG, "ht_find_peaks_noalloc: accumulator not 16-byte aligned");
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
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();   // clear it: the next call looks the address up again
                return ht::set_error(HT_ERR_CUDA, "ht_find_peaks_noalloc: cudaGetSymbolAddress "
                                                  "of the scratch failed (retried next call)");
            }
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    e = ht::launch_peaks(g->G, acc, peaks, cap, d_count, scratch,
                         reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return ht::set_error(HT_ERR_CUDA, cudaGetErrorString(e));
    return HT_OK;
}
