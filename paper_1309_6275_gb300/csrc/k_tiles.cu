// k_tiles.cu -- the two passes over an event's hits that follow the tile
// scheme: the Hough vote (Section 5 of arXiv:1309.6275) and the hit
// association that confirms candidates (Section 5, last step).
//
// Design (GB300):
//  * One CTA owns a parameter-space tile of 32 rho rows x KT phi0 columns x
//    all n_d0 bins, held in shared memory: uint32 vote counters for the
//    vote, the best candidate key per cell for the association.  Rows are
//    padded to n_d0 + 1 words, so 32 rows at the same d0 bin fall in 32
//    different banks.
//  * The CTA streams the hits in chunks of blockDim.  Phase 1 (one thread per
//    hit): an angular window and a curvature-range test select the (hit,
//    column) pairs that can vote in the tile; survivors are appended to a
//    shared work list with one atomic per warp (warp-aggregated append).
//    Phase 2 (one warp per item): lane = rho row, so the 32 atomics a warp
//    issues hit 32 distinct cells in 32 distinct banks.
//  * Arithmetic: guarded float32 (cell_bins32); every column it cannot prove
//    is redone in float64 in the definition's order (cell_bins64), so the
//    votes are bit-identical to the float64 definition.  The work is integer
//    counting: no tensor cores.
//  * Vote write-back stores every cell once, saturated, with vector stores:
//    the accumulator needs no clearing and crosses HBM once.
//  * Association: each tile first scatters the candidates whose 3x3x3 box
//    meets it into the tile (atomicMax of key = count << 32 | ~m), then
//    replays the vote and takes, per hit, the maximum key over the cells it
//    votes in: max over compatible candidates of (count, -m).
#include <cuda_runtime.h>
#include <stdint.h>

#include "ht_internal.cuh"

namespace ht {
namespace {

constexpr int kThreads = 256;

template <typename T, int KT>
struct VecOf;  // KT counts of type T as one aligned store
template <> struct VecOf<uint16_t, 2> { using type = uint32_t; };
template <> struct VecOf<uint16_t, 4> { using type = uint2; };
template <> struct VecOf<uint16_t, 8> { using type = uint4; };
template <> struct VecOf<int32_t, 2> { using type = uint2; };
template <> struct VecOf<int32_t, 4> { using type = uint4; };

template <typename OutT>
__device__ __forceinline__ OutT saturate(uint32_t v)
{
    if (sizeof(OutT) == 2) return (OutT)(v > 65535u ? 65535u : v);
    return (OutT)(v > 2147483647u ? 2147483647u : v);
}

// Shared work list of (hit, column) items, structure of arrays.
struct WorkList {
    float *s, *c, *r2, *R1;
    int *meta;          // hit << 6 | unsure << 5 | column-in-tile
};

__device__ __forceinline__ WorkList carve_worklist(unsigned char *p, int cap)
{
    WorkList w;
    w.s = reinterpret_cast<float *>(p);
    w.c = w.s + cap;
    w.r2 = w.c + cap;
    w.R1 = w.r2 + cap;
    w.meta = reinterpret_cast<int *>(w.R1 + cap);
    return w;
}

// Per-tile constants of the lane's row and of the tile's columns.
template <int KT>
struct TileCtx {
    int i0, k0, irow;
    bool row_ok, has_b;
    float rho, invrho, arho, ainvrho, rho_lo, rho_hi;
    float sk[KT], ck[KT], pk[KT];

    __device__ __forceinline__ void init(const DevGeom &G, int lane)
    {
        k0 = blockIdx.x * KT;
        i0 = blockIdx.y * 32;
        irow = i0 + lane;
        row_ok = irow < G.n_rho;
        rho = row_ok ? G.rho32[irow] : 0.0f;
        invrho = row_ok ? G.invrho32[irow] : 0.0f;
        has_b = row_ok && (G.rho64[irow] != 0.0);
        arho = fabsf(rho);
        ainvrho = fabsf(invrho);
        const int ilast = min(i0 + 31, G.n_rho - 1);
        rho_lo = G.rho32[i0] - G.drho_f;
        rho_hi = G.rho32[ilast] + G.drho_f;
#pragma unroll
        for (int kl = 0; kl < KT; ++kl) {
            sk[kl] = G.sn32[k0 + kl];
            ck[kl] = G.cs32[k0 + kl];
            pk[kl] = G.phi32[k0 + kl];
        }
    }
};

// Phase 1 for hit h (h >= n: no items).  Appends this warp's items to the
// list with a single atomicAdd on *qn (all 32 lanes must call).
template <int KT>
__device__ __forceinline__ void collect(const DevGeom &G, const TileCtx<KT> &T,
                                        const float *__restrict__ x,
                                        const float *__restrict__ y, int n, int h,
                                        int lane, int *qn, const WorkList &W)
{
    float is_[KT], ic_[KT];
    unsigned sel = 0u, unsure = 0u;
    float r2 = 0.0f, R1 = 0.0f;
    if (h < n) {
        const float xh = x[h], yh = y[h];
        r2 = fmaf(xh, xh, yh * yh);
        R1 = fabsf(xh) + fabsf(yh);
        const float win = hit_window(G, sqrtf(r2));
        const float phh = atan2f(yh, xh);
        const float Ec = (kSafe * 3.0f * kEps) * R1;
#pragma unroll
        for (int kl = 0; kl < KT; ++kl) {
            if (fabsf(wrap_pi(T.pk[kl] - phh)) > win) continue;
            const float s = fmaf(xh, T.sk[kl], -(yh * T.ck[kl]));
            const float c = fmaf(xh, T.ck[kl], yh * T.sk[kl]);
            if (c < -Ec) continue;
            if (c <= Ec) {
                unsure |= 1u << kl;
            } else if (c > 1.0f) {
                float gmin, gmax;
                rho_range(G, s, c, gmin, gmax);
                if (gmax < T.rho_lo || gmin > T.rho_hi) continue;
            }
            sel |= 1u << kl;
            is_[kl] = s;
            ic_[kl] = c;
        }
    }
    const int mine = __popc(sel);
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    int wbase = 0;
    if (lane == 31 && incl > 0) wbase = atomicAdd(qn, incl);
    wbase = __shfl_sync(0xffffffffu, wbase, 31);
    int pos = wbase + incl - mine;
#pragma unroll
    for (int kl = 0; kl < KT; ++kl) {
        if (sel & (1u << kl)) {
            W.s[pos] = is_[kl];
            W.c[pos] = ic_[kl];
            W.r2[pos] = r2;
            W.R1[pos] = R1;
            W.meta[pos] = (h << 6) | (int)(((unsure >> kl) & 1u) << 5) | kl;
            ++pos;
        }
    }
}

// Bins of item `it` for the lane's row: guarded float32, else float64.
template <int KT>
__device__ __forceinline__ int item_bins(const DevGeom &G, const TileCtx<KT> &T,
                                         const float *__restrict__ x,
                                         const float *__restrict__ y, const WorkList &W,
                                         int it, int jj[2], int &n_edge, int &n_fb)
{
    const int m = W.meta[it];
    if (!(m & 32)) {
        int jA, jB;
        if (cell_bins32(G, T.rho, T.arho, T.invrho, T.ainvrho, T.has_b, W.s[it], W.c[it],
                        W.r2[it], W.R1[it], jA, jB, n_edge)) {
            int nv = 0;
            if (jA >= 0) jj[nv++] = jA;
            if (jB >= 0) jj[nv++] = jB;
            return nv;
        }
    }
    ++n_fb;
    const int hh = m >> 6;
    return cell_bins64(G, x[hh], y[hh], T.irow, T.k0 + (m & 31), jj, &n_edge);
}

// ------------------------------------------------------------------ vote
template <int KT, typename OutT>
__global__ void __launch_bounds__(kThreads, 2)
k_vote(DevGeom G, const float *__restrict__ x, const float *__restrict__ y, int n,
       OutT *__restrict__ acc, unsigned long long *__restrict__ stats)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int ND = G.n_d0, NDP = ND + 1;
    constexpr int QCAP = kThreads * KT;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);
    const WorkList W = carve_worklist(reinterpret_cast<unsigned char *>(cnt + KT * 32 * NDP), QCAP);
    __shared__ int qn[2];
    __shared__ unsigned long long s_stats[3];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nwarps = kThreads / 32;
    TileCtx<KT> T;
    T.init(G, lane);
    for (int t = threadIdx.x; t < KT * 32 * NDP; t += kThreads) cnt[t] = 0u;
    if (threadIdx.x < 2) qn[threadIdx.x] = 0;
    if (threadIdx.x < 3) s_stats[threadIdx.x] = 0ull;
    __syncthreads();

    int my_votes = 0, my_fb = 0, my_edge = 0;
    int parity = 0;
    for (int base = 0; base < n; base += kThreads, parity ^= 1) {
        collect<KT>(G, T, x, y, n, base + threadIdx.x, lane, &qn[parity], W);
        __syncthreads();
        const int nq = qn[parity];
        if (threadIdx.x == 0) qn[parity ^ 1] = 0;   // last read before the previous barrier
        if (T.row_ok) {
            for (int it = warp; it < nq; it += nwarps) {
                uint32_t *col = cnt + ((W.meta[it] & 31) * 32 + lane) * NDP;
                int jj[2];
                const int nv = item_bins<KT>(G, T, x, y, W, it, jj, my_edge, my_fb);
                for (int t = 0; t < nv; ++t) atomicAdd(col + jj[t], 1u);
                my_votes += nv;
            }
        }
        __syncthreads();
    }

    using Vec = typename VecOf<OutT, KT>::type;
    for (int t = threadIdx.x; t < 32 * ND; t += kThreads) {
        const int il = t / ND, j = t - il * ND;
        const int i = T.i0 + il;
        if (i >= G.n_rho) break;
        union { Vec v; OutT e[KT]; } u;
#pragma unroll
        for (int kl = 0; kl < KT; ++kl) u.e[kl] = saturate<OutT>(cnt[(kl * 32 + il) * NDP + j]);
        *reinterpret_cast<Vec *>(acc + ((size_t)i * ND + j) * G.n_phi0 + T.k0) = u.v;
    }

    if (stats) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            my_votes += __shfl_xor_sync(0xffffffffu, my_votes, o);
            my_fb += __shfl_xor_sync(0xffffffffu, my_fb, o);
            my_edge += __shfl_xor_sync(0xffffffffu, my_edge, o);
        }
        if (lane == 0) {
            atomicAdd(&s_stats[0], (unsigned long long)my_votes);
            atomicAdd(&s_stats[1], (unsigned long long)my_fb);
            atomicAdd(&s_stats[2], (unsigned long long)my_edge);
        }
        __syncthreads();
        if (threadIdx.x < 3) atomicAdd(&stats[threadIdx.x], s_stats[threadIdx.x]);
    }
}

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
    const int ND = G.n_d0, NDP = ND + 1, NP = G.n_phi0;
    constexpr int QCAP = kThreads * KT;
    unsigned long long *map = reinterpret_cast<unsigned long long *>(smem);
    unsigned long long *bestk = map + KT * 32 * NDP;
    const WorkList W = carve_worklist(reinterpret_cast<unsigned char *>(bestk + kThreads), QCAP);
    __shared__ int qn[2];
    __shared__ int band[2];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nwarps = kThreads / 32;
    TileCtx<KT> T;
    T.init(G, lane);
    for (int t = threadIdx.x; t < KT * 32 * NDP; t += kThreads) map[t] = 0ull;
    bestk[threadIdx.x] = 0ull;
    if (threadIdx.x < 2) qn[threadIdx.x] = 0;
    const int ncand = min(*d_count, cap);
    if (threadIdx.x == 0) {
        const int ib0 = max(T.i0 - 1, 0), ib1 = min(T.i0 + 32, G.n_rho - 1);
        band[0] = lower_bound_l(peaks, ncand, (long long)ib0 * ND * NP, ND, NP);
        band[1] = lower_bound_l(peaks, ncand, (long long)(ib1 + 1) * ND * NP, ND, NP);
    }
    __syncthreads();

    // scatter each candidate's 3x3x3 box into the tile
    for (int m = band[0] + threadIdx.x; m < band[1]; m += kThreads) {
        const ht_peak p = peaks[m];
        const unsigned long long key =
            ((unsigned long long)(unsigned)p.count << 32) | (0xffffffffull - (unsigned)m);
#pragma unroll
        for (int dk = -1; dk <= 1; ++dk) {
            int kk = p.k_phi0 + dk;
            kk += (kk < 0) ? NP : 0;
            kk -= (kk >= NP) ? NP : 0;
            const int kl = kk - T.k0;
            if (kl < 0 || kl >= KT) continue;
            for (int di = -1; di <= 1; ++di) {
                const int ii = p.i_rho + di, il = ii - T.i0;
                if (il < 0 || il >= 32 || ii >= G.n_rho) continue;
                for (int dj = -1; dj <= 1; ++dj) {
                    const int jj = p.j_d0 + dj;
                    if (jj < 0 || jj >= ND) continue;
                    atomicMax(&map[(kl * 32 + il) * NDP + jj], key);
                }
            }
        }
    }
    __syncthreads();

    int my_edge = 0, my_fb = 0;
    int parity = 0;
    for (int base = 0; base < n; base += kThreads, parity ^= 1) {
        collect<KT>(G, T, x, y, n, base + threadIdx.x, lane, &qn[parity], W);
        __syncthreads();
        const int nq = qn[parity];
        if (threadIdx.x == 0) qn[parity ^ 1] = 0;
        for (int it = warp; it < nq; it += nwarps) {
            unsigned long long key = 0ull;
            if (T.row_ok) {
                const unsigned long long *col = map + ((W.meta[it] & 31) * 32 + lane) * NDP;
                int jj[2];
                const int nv = item_bins<KT>(G, T, x, y, W, it, jj, my_edge, my_fb);
                for (int t = 0; t < nv; ++t) key = max(key, col[jj[t]]);
            }
            if (__any_sync(0xffffffffu, key != 0ull)) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    key = max(key, __shfl_xor_sync(0xffffffffu, key, o));
                if (lane == 0 && key) atomicMax(&bestk[(W.meta[it] >> 6) - base], key);
            }
        }
        __syncthreads();
        // flush this chunk's per-hit best keys (slot t belongs to thread t)
        const unsigned long long b = bestk[threadIdx.x];
        if (b) {
            atomicMax(&gbest[base + threadIdx.x], b);
            bestk[threadIdx.x] = 0ull;
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

// ---------------------------------------------------------------- launch
template <int KT, typename OutT>
size_t vote_smem(const DevGeom &G)
{
    return (size_t)KT * 32 * (G.n_d0 + 1) * 4 + (size_t)kThreads * KT * 20;
}

template <int KT>
size_t assoc_smem(const DevGeom &G)
{
    return (size_t)KT * 32 * (G.n_d0 + 1) * 8 + (size_t)kThreads * 8 + (size_t)kThreads * KT * 20;
}

constexpr size_t kSmemBudget = 100 * 1024;   // two CTAs per SM

template <int KT, typename OutT>
cudaError_t launch_vote_kt(const DevGeom &G, const float *x, const float *y, int n, void *acc,
                           unsigned long long *stats, cudaStream_t st)
{
    const size_t smem = vote_smem<KT, OutT>(G);
    dim3 grid(G.n_phi0 / KT, (G.n_rho + 31) / 32);
    k_vote<KT, OutT><<<grid, kThreads, smem, st>>>(G, x, y, n, reinterpret_cast<OutT *>(acc),
                                                  stats);
    return cudaGetLastError();
}

template <int KT>
cudaError_t launch_assoc_kt(const DevGeom &G, const float *x, const float *y, int n,
                            const ht_peak *peaks, const int *d_count, int cap,
                            unsigned long long *gbest, cudaStream_t st)
{
    const size_t smem = assoc_smem<KT>(G);
    dim3 grid(G.n_phi0 / KT, (G.n_rho + 31) / 32);
    k_assoc<KT><<<grid, kThreads, smem, st>>>(G, x, y, n, peaks, d_count, cap, gbest);
    return cudaGetLastError();
}

}  // namespace

// Allow every tile kernel the device's opt-in shared memory (the launch
// still passes only what the chosen tile needs).  Called once per device.
cudaError_t prepare_tile_kernels(int max_smem)
{
    const void *fns[] = {(const void *)k_vote<8, uint16_t>, (const void *)k_vote<4, uint16_t>,
                         (const void *)k_vote<2, uint16_t>, (const void *)k_vote<4, int32_t>,
                         (const void *)k_vote<2, int32_t>,  (const void *)k_assoc<4>,
                         (const void *)k_assoc<2>,          (const void *)k_assoc<1>};
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

// Largest tile shared memory any geometry with n_d0 bins needs.
size_t tile_smem_need(const DevGeom &G)
{
    size_t v = G.count_bits == 16 ? vote_smem<2, uint16_t>(G) : vote_smem<2, int32_t>(G);
    size_t a = assoc_smem<1>(G);
    return v > a ? v : a;
}

// Tile width: the widest KT whose tile and work list leave room for two CTAs
// per SM.
cudaError_t launch_vote(const DevGeom &G, const float *x, const float *y, int n, void *acc,
                        unsigned long long *stats, cudaStream_t st)
{
    if (G.count_bits == 16) {
        if (vote_smem<8, uint16_t>(G) <= kSmemBudget)
            return launch_vote_kt<8, uint16_t>(G, x, y, n, acc, stats, st);
        if (vote_smem<4, uint16_t>(G) <= kSmemBudget)
            return launch_vote_kt<4, uint16_t>(G, x, y, n, acc, stats, st);
        return launch_vote_kt<2, uint16_t>(G, x, y, n, acc, stats, st);
    }
    if (vote_smem<4, int32_t>(G) <= kSmemBudget)
        return launch_vote_kt<4, int32_t>(G, x, y, n, acc, stats, st);
    return launch_vote_kt<2, int32_t>(G, x, y, n, acc, stats, st);
}

size_t associate_workspace_bytes(const DevGeom &, int n)
{
    return align256((size_t)(n > 0 ? n : 1) * 8);
}

cudaError_t launch_associate(const DevGeom &G, const float *x, const float *y, int n,
                             const ht_peak *peaks, const int *d_count, int cap, int *assign,
                             void *ws, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    unsigned long long *gbest = reinterpret_cast<unsigned long long *>(ws);
    cudaError_t e = cudaMemsetAsync(gbest, 0, (size_t)n * 8, st);
    if (e != cudaSuccess) return e;
    if (assoc_smem<4>(G) <= kSmemBudget)
        e = launch_assoc_kt<4>(G, x, y, n, peaks, d_count, cap, gbest, st);
    else if (assoc_smem<2>(G) <= kSmemBudget)
        e = launch_assoc_kt<2>(G, x, y, n, peaks, d_count, cap, gbest, st);
    else
        e = launch_assoc_kt<1>(G, x, y, n, peaks, d_count, cap, gbest, st);
    if (e != cudaSuccess) return e;
    k_assoc_final<<<(n + 255) / 256, 256, 0, st>>>(gbest, n, assign);
    return cudaGetLastError();
}

}  // namespace ht
