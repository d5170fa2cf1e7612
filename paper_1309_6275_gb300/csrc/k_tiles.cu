// k_tiles.cu -- the two passes over an event's hits that follow the tile
// scheme: the Hough vote (Section 5 of arXiv:1309.6275) and the hit
// association that confirms candidates (Section 5, last step).
//
// Design (GB300):
//  * One CTA owns a parameter-space tile of 32 rho rows x KT phi0 columns x
//    all n_d0 bins, held in shared memory row-fastest ([column][d0][row]):
//    uint32 vote counters for the vote, candidate keys for the association.
//    Lane = row, so a warp's 32 shared accesses always fall in 32 distinct
//    banks whatever d0 bins the rows hit.
//  * The CTA streams the hits in chunks of blockDim.  Phase 1 (one thread per
//    hit): an angular window and a curvature-range test select the (hit,
//    column) pairs that can vote in the tile, and compute each pair's error
//    bound constants once; survivors are appended to a shared work list with
//    one atomic per warp (warp-aggregated append).  Phase 2 (one warp per
//    item): lane = rho row evaluates its root(s) with eval32.
//  * Arithmetic: guarded float32 (eval32); every column it cannot prove is
//    redone in float64 in the definition's order (cell_bins64), so the votes
//    are bit-identical to the float64 definition.  The work is integer
//    counting: no tensor cores.
//  * Vote write-back stores every cell once, saturated, so the accumulator
//    needs no clearing and crosses HBM once.
//  * Association: each tile first scatters the candidates whose 3x3x3 box
//    meets it into the tile (atomicMax of key = count << 32 | ~m), then
//    replays the vote and takes, per hit, the maximum key over the cells it
//    votes in: max over compatible candidates of (count, -m).
#include <cuda_runtime.h>
#include <stdint.h>

#include "tiles.cuh"

namespace ht {
namespace {

// ----------------------------------------------------------- association
__device__ __forceinline__ int lower_bound_l(const ht_peak *__restrict__ pk, int n,
                                             long long l, int ND, int NP)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const ht_peak p = pk[mid];
        const long long lm = ((long long)p.i_rho * ND + p.j_d0) * NP + p.k_phi0;
        if (lm < l) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <int KT>
__global__ void __launch_bounds__(kThreads, 2)
k_assoc(DevGeom G, const float *__restrict__ x, const float *__restrict__ y, int n,
        const ht_peak *__restrict__ peaks, const int *__restrict__ d_count, int cap,
        unsigned long long *__restrict__ gbest)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int ND = G.n_d0, NP = G.n_phi0;
    constexpr int QCAP = kThreads * KT;
    unsigned long long *map = reinterpret_cast<unsigned long long *>(smem);   // [KT][ND][32]
    unsigned long long *bestk = map + KT * ND * 32;
    unsigned char *p = reinterpret_cast<unsigned char *>(bestk + kThreads);
    const WorkList W = carve_worklist(p, QCAP);
    const RedoQueue R = carve_redo(p + (size_t)QCAP * kItemBytes);
    __shared__ int qn[2][2], rn;   // [parity][plain, others]
    __shared__ int band[2];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nwarps = kThreads / 32;
    TileCtx<KT> T;
    T.init(G, lane, blockIdx.x, blockIdx.y);
    {
        uint4 *m4 = reinterpret_cast<uint4 *>(map);
        for (int t = threadIdx.x; t < KT * ND * 16; t += kThreads) m4[t] = make_uint4(0, 0, 0, 0);
    }
    bestk[threadIdx.x] = 0ull;
    if (threadIdx.x < 4) qn[threadIdx.x >> 1][threadIdx.x & 1] = 0;
    if (threadIdx.x == 0) rn = 0;
    const int ncand = min(*d_count, cap);
    if (threadIdx.x == 0) {
        const int ib0 = max(T.i0 - 1, 0), ib1 = min(T.i0 + 32, G.n_rho - 1);
        band[0] = lower_bound_l(peaks, ncand, (long long)ib0 * ND * NP, ND, NP);
        band[1] = lower_bound_l(peaks, ncand, (long long)(ib1 + 1) * ND * NP, ND, NP);
    }
    __syncthreads();

    // scatter each candidate's 3x3x3 box into the tile
    for (int m = band[0] + threadIdx.x; m < band[1]; m += kThreads) {
        const ht_peak pk = peaks[m];
        int kls[3];
        bool any = false;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int kk = pk.k_phi0 - 1 + d;
            kk += (kk < 0) ? NP : 0;
            kk -= (kk >= NP) ? NP : 0;
            kls[d] = kk - T.k0;
            any |= (kls[d] >= 0 && kls[d] < KT);
        }
        if (!any) continue;
        const unsigned long long key =
            ((unsigned long long)(unsigned)pk.count << 32) | (0xffffffffull - (unsigned)m);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int kl = kls[d];
            if (kl < 0 || kl >= KT) continue;
            for (int di = -1; di <= 1; ++di) {
                const int ii = pk.i_rho + di, il = ii - T.i0;
                if (il < 0 || il >= 32 || ii >= G.n_rho) continue;
                for (int dj = -1; dj <= 1; ++dj) {
                    const int jj = pk.j_d0 + dj;
                    if (jj < 0 || jj >= ND) continue;
                    atomicMax(&map[(kl * ND + jj) * 32 + il], key);
                }
            }
        }
    }
    __syncthreads();

    int parity = 0;
    const HitSeq S{nullptr, n};
    HitPrefetch pf;
    pf.start(x, y, S);
    for (int base = 0; base < n; base += kThreads, parity ^= 1) {
        int ha;
        float xh, yh;
        pf.next(x, y, S, base, ha, xh, yh);
        collect<KT>(G, T, xh, yh, n, base + threadIdx.x, ha, lane, qn[parity], W);
        __syncthreads();
        const int nf = qn[parity][0], nq = nf + qn[parity][1];
        if (threadIdx.x == 0) {
            qn[parity ^ 1][0] = 0;
            qn[parity ^ 1][1] = 0;
        }
        for (int tt = warp; tt < nq; tt += nwarps) {
            const int t = item_slot<KT>(tt, nf);
            const int m = W.meta[t];
            unsigned long long key = 0ull;
            if (T.row_ok) {
                const unsigned long long *col = map + (m & kMetaCol) * ND * 32 + lane;
                int jj[2];
                int nv = item_bins32<KT>(G, T, W, t, m, jj);
                if (nv < 0 && !push_redo(R, &rn, m >> 6, lane, m & kMetaCol))
                    nv = redo_bins(G, x[m >> 6], y[m >> 6], T.irow, T.k0 + (m & kMetaCol), jj);
                if (nv > 0) key = col[jj[0] * 32];
                if (nv > 1) key = max(key, col[jj[1] * 32]);
            }
            // warp max of (count, -m): high word first, then low word among ties
            const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(key >> 32));
            if (hi) {
                const unsigned lo = __reduce_max_sync(
                    0xffffffffu, (unsigned)(key >> 32) == hi ? (unsigned)key : 0u);
                if (lane == 0)
                    atomicMax(&bestk[(m >> 6) - base], ((unsigned long long)hi << 32) | lo);
            }
        }
        __syncthreads();
        // flush this chunk's per-hit best keys (slot t belongs to thread t)
        const unsigned long long b = bestk[threadIdx.x];
        if (b) {
            atomicMax(&gbest[base + threadIdx.x], b);
            bestk[threadIdx.x] = 0ull;
        }
        // drain the deferred redos when the queue is half full or at the end;
        // their keys go straight to the global per-hit maximum
        const int nr = min(rn, kRedoCap);
        if (nr >= kRedoCap / 2 || base + kThreads >= n) {
            for (int t = threadIdx.x; t < nr; t += kThreads) {
                const int h = R.hit[t], rc = R.rc[t];
                const int il = rc >> 4, kl = rc & 15;
                int jj[2];
                const int nv = redo_bins(G, x[h], y[h], T.i0 + il, T.k0 + kl, jj);
                const unsigned long long *col = map + kl * ND * 32 + il;
                unsigned long long key = 0ull;
                for (int v = 0; v < nv; ++v) key = max(key, col[jj[v] * 32]);
                if (key) atomicMax(&gbest[h], key);
            }
            __syncthreads();
            if (threadIdx.x == 0) rn = 0;
        }
    }
}

__global__ void k_assoc_final(const unsigned long long *__restrict__ gbest, int n,
                              int *__restrict__ assign)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= n) return;
    const unsigned long long b = gbest[h];
    assign[h] = b ? (int)(0xffffffffu - (unsigned)(b & 0xffffffffull)) : -1;
}

// ------------------------------------- association with 32-bit keys
// For uint16 accumulators (counts <= 65535).  A pre-pass lists, for every
// tile, the candidates whose 3x3x3 box touches it; the tile sorts its list by
// candidate index, so a 16-bit rank is monotone in m, and scatters
// key = count << 16 | (65535 - rank) with native 32-bit shared atomicMax.
// Peaks form an independent set of the 26-neighbour grid (of two adjacent
// cells at most one can be a peak), so a tile's list holds at most one
// candidate per 2x2x2 block of its 34 x (KT + 2) x n_d0 halo region.
// Tiles a candidate's box touches: up to 2 row tiles x 3 column tiles (3
// column tiles only when a tile is one column wide).
constexpr int kMaxTilesPerCand = 6;

__device__ __forceinline__ int tiles_of(const ht_peak &p, int NR, int NP, int KT, int nct,
                                        int out[kMaxTilesPerCand])
{
    const int rt0 = max(p.i_rho - 1, 0) >> 5, rt1 = min(p.i_rho + 1, NR - 1) >> 5;
    int ct[3], nc = 0;
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
        int kk = p.k_phi0 + d;
        kk += (kk < 0) ? NP : 0;
        kk -= (kk >= NP) ? NP : 0;
        const int c = kk / KT;
        bool dup = false;
        for (int u = 0; u < nc; ++u) dup |= (ct[u] == c);
        if (!dup) ct[nc++] = c;
    }
    int no = 0;
    for (int rt = rt0; rt <= rt1; ++rt)
        for (int u = 0; u < nc; ++u) out[no++] = rt * nct + ct[u];
    return no;
}

__global__ void k_cand_tiles(const ht_peak *__restrict__ peaks, const int *__restrict__ d_count,
                             int cap, int NR, int NP, int KT, int nct, int *__restrict__ tcnt,
                             int *__restrict__ tcur, int *__restrict__ list)
{
    const int ncand = min(*d_count, cap);
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < ncand; m += gridDim.x * blockDim.x) {
        int t[kMaxTilesPerCand];
        const int nt = tiles_of(peaks[m], NR, NP, KT, nct, t);
        for (int u = 0; u < nt; ++u) {
            if (list) list[atomicAdd(&tcur[t[u]], 1)] = m;
            else atomicAdd(&tcnt[t[u]], 1);
        }
    }
}

// The same lists built with one shared-memory histogram per CTA: each CTA
// takes a contiguous chunk of the candidates, counts its (candidate, tile)
// pairs in shared memory and touches each global tile counter once; the fill
// pass reserves the CTA's slots per tile with one global atomic and places
// candidates with shared atomics.  Order inside a tile's list is arbitrary
// (the association sorts each list).
__global__ void __launch_bounds__(256)
k_cand_hist(const ht_peak *__restrict__ peaks, const int *__restrict__ d_count, int cap, int NR,
            int NP, int KT, int nct, int ntiles, int *__restrict__ tcnt, int *__restrict__ tcur,
            int *__restrict__ list)
{
    extern __shared__ int hist[];   // [ntiles]
    const int ncand = min(*d_count, cap);
    const int per = (ncand + gridDim.x - 1) / gridDim.x;
    const int a = blockIdx.x * per, b = min(ncand, a + per);
    if (a >= b) return;   // uniform over the CTA
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    for (int m = a + threadIdx.x; m < b; m += blockDim.x) {
        int t[kMaxTilesPerCand];
        const int nt = tiles_of(peaks[m], NR, NP, KT, nct, t);
        for (int u = 0; u < nt; ++u) atomicAdd(&hist[t[u]], 1);
    }
    __syncthreads();
    if (!list) {
        for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
            if (hist[t]) atomicAdd(&tcnt[t], hist[t]);
        return;
    }
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
        if (hist[t]) hist[t] = atomicAdd(&tcur[t], hist[t]);
    __syncthreads();
    for (int m = a + threadIdx.x; m < b; m += blockDim.x) {
        int t[kMaxTilesPerCand];
        const int nt = tiles_of(peaks[m], NR, NP, KT, nct, t);
        for (int u = 0; u < nt; ++u) list[atomicAdd(&hist[t[u]], 1)] = m;
    }
}

constexpr int kCandHistMaxTiles = 24 * 1024;   // 96 KB of shared counters

// One pass of the candidate tile lists: counts (list null) or fill.
inline void cand_tiles_pass(const ht_peak *peaks, const int *d_count, int cap, int NR, int NP,
                            int KT, int nct, int ntiles, int *tcnt, int *tcur, int *list,
                            cudaStream_t st)
{
    if (ntiles <= kCandHistMaxTiles) {
        const int sms = device_sms();
        k_cand_hist<<<sms, 256, (size_t)ntiles * 4, st>>>(peaks, d_count, cap, NR, NP, KT, nct,
                                                          ntiles, tcnt, tcur, list);
        return;
    }
    const int nb = min(4096, (cap + 255) / 256 > 0 ? (cap + 255) / 256 : 1);
    k_cand_tiles<<<nb, 256, 0, st>>>(peaks, d_count, cap, NR, NP, KT, nct, list ? nullptr : tcnt,
                                     list ? tcur : nullptr, list);
}

// hl (optional): scan only the nl hits hl[0 .. nl) of the event (a superset
// of those that can vote in the tile's columns); otherwise all n.
template <int KT>
__device__ __forceinline__ void assoc32_tile(const DevGeom &G, const float *__restrict__ x,
                                             const float *__restrict__ y, int n,
                                             const ht_peak *__restrict__ peaks,
                                             const int *__restrict__ toff,
                                             const int *__restrict__ tlist, int lcap,
                                             unsigned long long *__restrict__ gbest, int tx,
                                             int ty, const int *__restrict__ hl = nullptr,
                                             int nl = 0)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int ND = G.n_d0;
    constexpr int QCAP = kThreads * KT;
    uint32_t *map = reinterpret_cast<uint32_t *>(smem);          // [KT][ND][32]
    int *local = reinterpret_cast<int *>(map + KT * ND * 32);    // sorted candidate indices
    uint32_t *bestk = reinterpret_cast<uint32_t *>(local + lcap);
    unsigned char *p = reinterpret_cast<unsigned char *>(bestk + kThreads);
    const WorkList W = carve_worklist(p, QCAP);
    const RedoQueue R = carve_redo(p + (size_t)QCAP * kItemBytes);
    __shared__ int qn[2][2], rn;   // [parity][plain, others]

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nwarps = kThreads / 32;
    TileCtx<KT> T;
    T.init(G, lane, tx, ty);
    const int tile = ty * (G.n_phi0 / KT) + tx;
    const int l0 = toff[tile];
    const int L = min(toff[tile + 1] - l0, lcap);
    if (L == 0) return;   // no candidate box meets the tile (uniform over the CTA)
    __shared__ int s_ext[4];   // rows and d0 bins spanned by the candidates
    __shared__ int s_mrange[3];   // smallest and largest candidate index, largest count
    if (threadIdx.x == 0) {
        s_ext[0] = s_ext[2] = 0x7fffffff;
        s_ext[1] = s_ext[3] = -1;
        s_mrange[0] = 0x7fffffff;
        s_mrange[1] = s_mrange[2] = -1;
    }
    __syncthreads();
    // 32-bit cell keys must order (count, -m).  When the tile's candidates
    // span fewer than 2^20 indices and no count passes 4095 (the usual case)
    // the key is count << 20 | (2^20 - 1 - (m - m_min)); otherwise the
    // candidates are sorted and the key is count << 16 | (65535 - rank).
    {
        int mlo = 0x7fffffff, mhi = -1, chi = -1;
        for (int r = threadIdx.x; r < L; r += kThreads) {
            const int m = tlist[l0 + r];
            mlo = min(mlo, m);
            mhi = max(mhi, m);
            chi = max(chi, peaks[m].count);
        }
        mlo = __reduce_min_sync(0xffffffffu, mlo);
        mhi = __reduce_max_sync(0xffffffffu, mhi);
        chi = __reduce_max_sync(0xffffffffu, chi);
        if (lane == 0) {
            atomicMin(&s_mrange[0], mlo);
            atomicMax(&s_mrange[1], mhi);
            atomicMax(&s_mrange[2], chi);
        }
    }
    __syncthreads();
    const int m_min = s_mrange[0];
    const bool offs = s_mrange[1] - m_min < (1 << 20) && s_mrange[2] < 4096;   // uniform
    if (offs) {
        for (int t = threadIdx.x; t < L; t += kThreads) local[t] = tlist[l0 + t];
    } else {
        // sort the tile's candidates by index: bitonic sort in the map's space
        int P = 1;
        while (P < L) P <<= 1;
        int *sb = reinterpret_cast<int *>(map);
        for (int t = threadIdx.x; t < P; t += kThreads) sb[t] = t < L ? tlist[l0 + t] : 0x7fffffff;
        __syncthreads();
        for (int k2 = 2; k2 <= P; k2 <<= 1)
            for (int j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
                for (int t = threadIdx.x; t < P; t += kThreads) {
                    const int o = t ^ j2;
                    if (o > t) {
                        const int a = sb[t], b = sb[o];
                        const bool up = (t & k2) == 0;
                        if ((a > b) == up) { sb[t] = b; sb[o] = a; }
                    }
                }
                __syncthreads();
            }
        for (int t = threadIdx.x; t < L; t += kThreads) local[t] = sb[t];
    }
    __syncthreads();
    {
        uint4 *m4 = reinterpret_cast<uint4 *>(map);
        for (int t = threadIdx.x; t < KT * ND * 8; t += kThreads) m4[t] = make_uint4(0, 0, 0, 0);
    }
    bestk[threadIdx.x] = 0u;
    if (threadIdx.x < 4) qn[threadIdx.x >> 1][threadIdx.x & 1] = 0;
    if (threadIdx.x == 0) rn = 0;
    __syncthreads();

    // scatter each candidate's box with its key
    int emin_i = 0x7fffffff, emax_i = -1, emin_j = 0x7fffffff, emax_j = -1;
    for (int r = threadIdx.x; r < L; r += kThreads) {
        const ht_peak pk = peaks[local[r]];
        emin_i = min(emin_i, pk.i_rho); emax_i = max(emax_i, pk.i_rho);
        emin_j = min(emin_j, pk.j_d0); emax_j = max(emax_j, pk.j_d0);
        const uint32_t key =
            offs ? ((uint32_t)pk.count << 20) | (uint32_t)(0xfffff - (local[r] - m_min))
                 : ((uint32_t)pk.count << 16) | (uint32_t)(0xffff - r);
#pragma unroll
        for (int d = -1; d <= 1; ++d) {
            int kk = pk.k_phi0 + d;
            kk += (kk < 0) ? G.n_phi0 : 0;
            kk -= (kk >= G.n_phi0) ? G.n_phi0 : 0;
            const int kl = kk - T.k0;
            if (kl < 0 || kl >= KT) continue;
            for (int di = -1; di <= 1; ++di) {
                const int ii = pk.i_rho + di, il = ii - T.i0;
                if (il < 0 || il >= 32 || ii >= G.n_rho) continue;
                for (int dj = -1; dj <= 1; ++dj) {
                    const int jj = pk.j_d0 + dj;
                    if (jj < 0 || jj >= ND) continue;
                    atomicMax(&map[(kl * ND + jj) * 32 + il], key);
                }
            }
        }
    }
    emin_i = __reduce_min_sync(0xffffffffu, emin_i);
    emax_i = __reduce_max_sync(0xffffffffu, emax_i);
    emin_j = __reduce_min_sync(0xffffffffu, emin_j);
    emax_j = __reduce_max_sync(0xffffffffu, emax_j);
    if (lane == 0) {
        atomicMin(&s_ext[0], emin_i); atomicMax(&s_ext[1], emax_i);
        atomicMin(&s_ext[2], emin_j); atomicMax(&s_ext[3], emax_j);
    }
    __syncthreads();
    // Only votes inside the candidates' boxes matter: phase 1 keeps the
    // (hit, column) pairs whose circle can reach the boxes' d0 bins within
    // their rows (the masked vote's filter, with one window).
    MaskCtx M;
    {
        const int jlo = max(s_ext[2] - 1, 0), jhi = min(s_ext[3] + 1, ND - 1);
        const int ilast = min(T.i0 + 31, G.n_rho - 1);
        const int ilo = min(max(s_ext[0] - 1, T.i0), ilast);
        const int ihi = max(min(s_ext[1] + 1, ilast), ilo);
        M.bm = M.tile_bm = 0u;
        M.nrun = 1;
        M.wlo[0] = (float)(((double)jlo - G.off) * G.delta) - 0.01f;
        M.whi[0] = (float)(((double)jhi + 1.0 - G.off) * G.delta) + 0.01f;
#pragma unroll
        for (int r = 1; r < 4; ++r) M.wlo[r] = M.whi[r] = 0.0f;
        M.rho_lo = G.rho32[ilo] - G.drho_f;
        M.rho_hi = G.rho32[ihi] + G.drho_f;
    }

    auto to64 = [&](uint32_t k32) -> unsigned long long {
        const int m = offs ? m_min + (0xfffff - (int)(k32 & 0xfffffu))
                           : local[0xffff - (int)(k32 & 0xffffu)];
        const unsigned cnt = offs ? k32 >> 20 : k32 >> 16;
        return ((unsigned long long)cnt << 32) | (0xffffffffull - (unsigned)m);
    };

    int parity = 0;
    const HitSeq S{hl, hl ? nl : n};
    HitPrefetch pf;
    pf.start(x, y, S);
    for (int base = 0; base < S.n; base += kThreads, parity ^= 1) {
        int ha;
        float xh, yh;
        pf.next(x, y, S, base, ha, xh, yh);
        collect<KT, kModeEvent>(G, T, xh, yh, S.n, base + threadIdx.x, ha, lane, qn[parity], W,
                                &M);
        __syncthreads();
        const int nf = qn[parity][0], ns = qn[parity][1];
        if (threadIdx.x == 0) {
            qn[parity ^ 1][0] = 0;
            qn[parity ^ 1][1] = 0;
        }
        // plain items: one root, no flags to test
#pragma unroll 2
        for (int t = warp; t < nf; t += nwarps) {
            const int m = W.meta[t];
            uint32_t key = 0u;
            if (T.row_ok) {
                const uint32_t *col = map + (m & kMetaCol) * ND * 32 + lane;
                int j;
                const int r = fast_bin32<KT>(G, T, W, t, j);
                if (r == kFastVote) {
                    key = col[j * 32];
                } else if (r == kFastRedo) {
                    const int hh = S.hit(m >> 6);
                    if (!push_redo(R, &rn, hh, lane, m & kMetaCol)) {
                        int jj[2];
                        const int nv =
                            redo_bins(G, x[hh], y[hh], T.irow, T.k0 + (m & kMetaCol), jj);
                        for (int v = 0; v < nv; ++v) key = max(key, col[jj[v] * 32]);
                    }
                }
            }
            const uint32_t top = __reduce_max_sync(0xffffffffu, key);
            if (top && lane == 0) atomicMax(&bestk[(m >> 6) - base], top);
        }
        // unsure items and items whose second root can reach the axis
        for (int t = QCAP - ns + warp; t < QCAP; t += nwarps) {
            const int m = W.meta[t];
            uint32_t key = 0u;
            if (T.row_ok) {
                const uint32_t *col = map + (m & kMetaCol) * ND * 32 + lane;
                int jj[2];
                int nv = item_bins32<KT>(G, T, W, t, m, jj);
                if (nv < 0) {
                    const int hh = S.hit(m >> 6);
                    if (!push_redo(R, &rn, hh, lane, m & kMetaCol))
                        nv = redo_bins(G, x[hh], y[hh], T.irow, T.k0 + (m & kMetaCol), jj);
                }
                if (nv > 0) key = col[jj[0] * 32];
                if (nv > 1) key = max(key, col[jj[1] * 32]);
            }
            const uint32_t top = __reduce_max_sync(0xffffffffu, key);
            if (top && lane == 0) atomicMax(&bestk[(m >> 6) - base], top);
        }
        __syncthreads();
        // flush this round's per-position best keys (slot t belongs to thread t)
        const uint32_t b = bestk[threadIdx.x];
        if (b) {
            atomicMax(&gbest[ha], to64(b));
            bestk[threadIdx.x] = 0u;
        }
        const int nr = min(rn, kRedoCap);
        if (nr >= kRedoCap / 2 || base + kThreads >= S.n) {
            for (int t = threadIdx.x; t < nr; t += kThreads) {
                const int h = R.hit[t], rc = R.rc[t];
                const int il = rc >> 4, kl = rc & 15;
                int jj[2];
                const int nv = redo_bins(G, x[h], y[h], T.i0 + il, T.k0 + kl, jj);
                const uint32_t *col = map + kl * ND * 32 + il;
                uint32_t key = 0u;
                for (int v = 0; v < nv; ++v) key = max(key, col[jj[v] * 32]);
                if (key) atomicMax(&gbest[h], to64(key));
            }
            __syncthreads();
            if (threadIdx.x == 0) rn = 0;
        }
    }
}

template <int KT>
__global__ void __launch_bounds__(kThreads, 3)
k_assoc32(DevGeom G, const float *__restrict__ x, const float *__restrict__ y, int n,
          const ht_peak *__restrict__ peaks, const int *__restrict__ toff,
          const int *__restrict__ tlist, int lcap, unsigned long long *__restrict__ gbest)
{
    assoc32_tile<KT>(G, x, y, n, peaks, toff, tlist, lcap, gbest, blockIdx.x, blockIdx.y);
}

// Persistent association over a batch, items as in k_vote_batch.  Event e
// uses peaks + e * cap, its tile lists at toff + e * (ntiles + 1) and
// tlist + e * lstride, and its hits' keys at gbest + off[e].
template <int KT>
__global__ void __launch_bounds__(kThreads, 3)
k_assoc32_batch(DevGeom G, const float *__restrict__ x, const float *__restrict__ y,
                const int *__restrict__ off, const int *__restrict__ order,
                const int *__restrict__ d_nev,
                const ht_peak *__restrict__ peaks, int cap, const int *__restrict__ toff,
                size_t tstride, const int *__restrict__ tlist, size_t lstride, int lcap,
                unsigned long long *__restrict__ gbest, int *__restrict__ head, BucketView bk)
{
    __shared__ int s_item;
    const int ntx = G.n_phi0 / KT, nty = (G.n_rho + 31) / 32, ntiles = ntx * nty;
    const int total = *d_nev * ntiles;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(head, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        const int e = order[item / ntiles], t = item % ntiles;
        const int a = off[e], n = off[e + 1] - a;
        const int *hl = nullptr;
        int nl = 0;
        if (bk.ent) bk.list(e, (t % ntx) * KT, hl, nl);
        if (n > 0)
            assoc32_tile<KT>(G, x + a, y + a, n, peaks + (size_t)e * cap,
                             toff + (size_t)e * tstride, tlist + (size_t)e * lstride, lcap,
                             gbest + a, t % ntx, t / ntx, hl, nl);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- launch
template <int KT>
size_t assoc_smem(const DevGeom &G)
{
    return (size_t)KT * 32 * G.n_d0 * 8 + (size_t)kThreads * 8 + (size_t)kThreads * KT * kItemBytes +
           kRedoBytes;
}

template <int KT>
int assoc32_lcap(const DevGeom &G)
{
    return 17 * ((KT + 3) / 2) * ((G.n_d0 + 1) / 2) + 32;
}

template <int KT>
size_t assoc32_smem(const DevGeom &G)
{
    const size_t map = (size_t)KT * 32 * G.n_d0 * 4;
    size_t sortbuf = 1;
    while (sortbuf < (size_t)assoc32_lcap<KT>(G)) sortbuf <<= 1;
    return (map > sortbuf * 4 ? map : sortbuf * 4) + (size_t)assoc32_lcap<KT>(G) * 4 +
           (size_t)kThreads * 4 + (size_t)kThreads * KT * kItemBytes + kRedoBytes;
}


template <int KT>
cudaError_t launch_assoc32_kt(const DevGeom &G, const float *x, const float *y, int n,
                              const ht_peak *peaks, const int *d_count, int cap,
                              unsigned long long *gbest, char *ws, cudaStream_t st)
{
    const int nct = G.n_phi0 / KT, nrt = (G.n_rho + 31) / 32, ntiles = nct * nrt;
    int *tcnt = reinterpret_cast<int *>(ws);
    int *toff = reinterpret_cast<int *>(ws + align256((size_t)(ntiles + 1) * 4));
    int *tcur = reinterpret_cast<int *>(ws + 2 * align256((size_t)(ntiles + 1) * 4));
    void *tmp = ws + 3 * align256((size_t)(ntiles + 1) * 4);
    int *tlist = reinterpret_cast<int *>(ws + 3 * align256((size_t)(ntiles + 1) * 4) +
                                         scan_tmp_bytes(ntiles));
    cudaError_t e = cudaMemsetAsync(tcnt, 0, (size_t)ntiles * 4, st);
    if (e != cudaSuccess) return e;
    cand_tiles_pass(peaks, d_count, cap, G.n_rho, G.n_phi0, KT, nct, ntiles, tcnt, nullptr,
                    nullptr, st);
    e = scan_exclusive(tcnt, toff, tcur, ntiles, nullptr, nullptr, tmp, st);
    if (e != cudaSuccess) return e;
    cand_tiles_pass(peaks, d_count, cap, G.n_rho, G.n_phi0, KT, nct, ntiles, nullptr, tcur, tlist,
                    st);
    dim3 grid(nct, nrt);
    k_assoc32<KT><<<grid, kThreads, assoc32_smem<KT>(G), st>>>(G, x, y, n, peaks, toff, tlist,
                                                               assoc32_lcap<KT>(G), gbest);
    return cudaGetLastError();
}

template <int KT>
cudaError_t launch_assoc_kt(const DevGeom &G, const float *x, const float *y, int n,
                            const ht_peak *peaks, const int *d_count, int cap,
                            unsigned long long *gbest, cudaStream_t st)
{
    dim3 grid(G.n_phi0 / KT, (G.n_rho + 31) / 32);
    k_assoc<KT><<<grid, kThreads, assoc_smem<KT>(G), st>>>(G, x, y, n, peaks, d_count, cap,
                                                           gbest);
    return cudaGetLastError();
}

}  // namespace

// Allow every tile kernel the device's opt-in shared memory (the launch
// still passes only what the chosen tile needs).  Called once per device.
cudaError_t prepare_tile_kernels(int max_smem)
{
    const void *fns[] = {(const void *)k_assoc<4>,   (const void *)k_assoc<2>,
                         (const void *)k_assoc<1>,   (const void *)k_assoc32<4>,
                         (const void *)k_assoc32<2>, (const void *)k_assoc32<1>,
                         (const void *)k_cand_hist};
    const cudaError_t e = allow_smem(fns, (int)(sizeof fns / sizeof fns[0]), max_smem);
    return e == cudaSuccess ? prepare_vote_kernels_t<kModePlain>(max_smem) : e;
}

// Largest tile shared memory any geometry with n_d0 bins needs.
size_t tile_smem_need(const DevGeom &G)
{
    const size_t v = vote_smem<1>(G, false), a = assoc_smem<1>(G), a32 = assoc32_smem<1>(G);
    return v > a ? (v > a32 ? v : a32) : (a > a32 ? a : a32);
}

cudaError_t launch_vote(const DevGeom &G, const float *x, const float *y, int n, void *acc,
                        unsigned long long *stats, cudaStream_t st)
{
    return launch_vote_t<kModePlain>(G, x, y, n, acc, stats, nullptr, st);
}

// Association workspace: per-hit best keys, then (uint16 geometries) the
// per-tile candidate lists: counts, offsets, cursors, scan scratch and up to
// kMaxTilesPerCand tile entries per candidate.
size_t associate_workspace_bytes(const DevGeom &G, int n, int cap)
{
    size_t b = align256((size_t)(n > 0 ? n : 1) * 8);
    const int KT = 4;   // the narrowest tiling used below has the most tiles
    const int ntiles = (G.n_phi0 / 1) * ((G.n_rho + 31) / 32);
    (void)KT;
    b += 3 * align256((size_t)(ntiles + 1) * 4) + scan_tmp_bytes(ntiles) +
         align256((size_t)(cap > 0 ? cap : 1) * kMaxTilesPerCand * 4);
    return b;
}

cudaError_t launch_associate(const DevGeom &G, const float *x, const float *y, int n,
                             const ht_peak *peaks, const int *d_count, int cap, int *assign,
                             void *ws, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    unsigned long long *gbest = reinterpret_cast<unsigned long long *>(ws);
    char *rest = reinterpret_cast<char *>(ws) + align256((size_t)n * 8);
    cudaError_t e = cudaMemsetAsync(gbest, 0, (size_t)n * 8, st);
    if (e != cudaSuccess) return e;
    if (G.count_bits == 16 && cap > 0) {
        if (assoc32_smem<4>(G) <= kSmemBudget3)
            e = launch_assoc32_kt<4>(G, x, y, n, peaks, d_count, cap, gbest, rest, st);
        else if (assoc32_smem<2>(G) <= kSmemBudget3)
            e = launch_assoc32_kt<2>(G, x, y, n, peaks, d_count, cap, gbest, rest, st);
        else
            e = launch_assoc32_kt<1>(G, x, y, n, peaks, d_count, cap, gbest, rest, st);
    } else if (assoc_smem<4>(G) <= kSmemBudget2) {
        e = launch_assoc_kt<4>(G, x, y, n, peaks, d_count, cap, gbest, st);
    } else if (assoc_smem<2>(G) <= kSmemBudget2) {
        e = launch_assoc_kt<2>(G, x, y, n, peaks, d_count, cap, gbest, st);
    } else {
        e = launch_assoc_kt<1>(G, x, y, n, peaks, d_count, cap, gbest, st);
    }
    if (e != cudaSuccess) return e;
    k_assoc_final<<<(n + 255) / 256, 256, 0, st>>>(gbest, n, assign);
    return cudaGetLastError();
}

// ------------------------------------------------------------- batches
cudaError_t launch_vote_batch(const DevGeom &G, const float *x, const float *y, const int *off,
                              const int *order, const int *d_nev, uint16_t *acc,
                              size_t acc_stride, unsigned long long *stats, int *head, bool pack,
                              int kt, int sms, cudaStream_t st, const HitBuckets *hb)
{
    return launch_vote_batch_t<kModePlain>(G, x, y, off, order, d_nev, acc, acc_stride, stats,
                                           head, pack, kt, sms, nullptr, st, bucket_view(hb));
}

// Association tile width for uint16 geometries (largest fitting three CTAs
// per SM) and the matching per-event tile-list sizes.
int assoc32_kt(const DevGeom &G)
{
    return assoc32_smem<4>(G) <= kSmemBudget3 ? 4 : assoc32_smem<2>(G) <= kSmemBudget3 ? 2 : 1;
}

int assoc32_ntiles(const DevGeom &G, int kt) { return (G.n_phi0 / kt) * ((G.n_rho + 31) / 32); }

// Per-event candidate tile lists (count, scan, scatter) into caller-carved
// buffers: tcnt/toff/tcur (ntiles + 1), tmp (scan), tlist (6 cap).
cudaError_t launch_cand_lists(const DevGeom &G, int kt, const ht_peak *peaks, const int *d_count,
                              int cap, int *tcnt, int *toff, int *tcur, void *tmp, int *tlist,
                              cudaStream_t st)
{
    const int nct = G.n_phi0 / kt, ntiles = assoc32_ntiles(G, kt);
    cudaError_t e = cudaMemsetAsync(tcnt, 0, (size_t)ntiles * 4, st);
    if (e != cudaSuccess) return e;
    cand_tiles_pass(peaks, d_count, cap, G.n_rho, G.n_phi0, kt, nct, ntiles, tcnt, nullptr,
                    nullptr, st);
    e = scan_exclusive(tcnt, toff, tcur, ntiles, nullptr, nullptr, tmp, st);
    if (e != cudaSuccess) return e;
    cand_tiles_pass(peaks, d_count, cap, G.n_rho, G.n_phi0, kt, nct, ntiles, nullptr, tcur, tlist,
                    st);
    return cudaGetLastError();
}

cudaError_t launch_assoc_batch(const DevGeom &G, int kt, const float *x, const float *y,
                               const int *off, const int *order, const int *d_nev,
                               const ht_peak *peaks, int cap, const int *toff, size_t tstride,
                               const int *tlist, size_t lstride, unsigned long long *gbest,
                               int *head, int sms, cudaStream_t st, const HitBuckets *hb)
{
    const BucketView bk = bucket_view(hb);
#define HT_AB(KTV)                                                                            \
    do {                                                                                      \
        int occ = 0;                                                                          \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_assoc32_batch<KTV>, kThreads,   \
                                                      assoc32_smem<KTV>(G));                  \
        k_assoc32_batch<KTV><<<sms * (occ > 0 ? occ : 1), kThreads, assoc32_smem<KTV>(G),    \
                               st>>>(G, x, y, off, order, d_nev, peaks, cap, toff, tstride,   \
                                     tlist, lstride, assoc32_lcap<KTV>(G), gbest, head, bk);  \
        return cudaGetLastError();                                                            \
    } while (0)
    if (kt == 4) HT_AB(4);
    if (kt == 2) HT_AB(2);
    HT_AB(1);
#undef HT_AB
}

__global__ void k_assoc_final_batch(const unsigned long long *__restrict__ gbest,
                                    const int *__restrict__ off, const int *__restrict__ d_nev,
                                    int *__restrict__ assign)
{
    const int n = off[*d_nev];
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
        const unsigned long long b = gbest[h];
        assign[h] = b ? (int)(0xffffffffu - (unsigned)(b & 0xffffffffull)) : -1;
    }
}

cudaError_t launch_assoc_final_batch(const unsigned long long *gbest, const int *off,
                                     const int *d_nev, int *assign, int max_hits, cudaStream_t st)
{
    k_assoc_final_batch<<<min(4096, (max_hits + 255) / 256 + 1), 256, 0, st>>>(gbest, off,
                                                                               d_nev, assign);
    return cudaGetLastError();
}

cudaError_t prepare_batch_kernels(int max_smem)
{
    const void *fns[] = {(const void *)k_assoc32_batch<4>, (const void *)k_assoc32_batch<2>,
                         (const void *)k_assoc32_batch<1>};
    return allow_smem(fns, (int)(sizeof fns / sizeof fns[0]), max_smem);
}

}  // namespace ht
