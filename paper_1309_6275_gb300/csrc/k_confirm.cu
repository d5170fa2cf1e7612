// k_confirm.cu -- confirmation of Hough candidates and the final hit
// assignment (ht_confirm, and the confirmation stage of ht_batch_run_tracks).
//
// Section 5 of arXiv:1309.6275: local maxima of the vote space are
// candidates, which costlier computations then confirm; Fig. 5 refines the
// candidates by a fit.  Reading, for candidate m = (i, j, k) and every hit h
// of its event, with b the bins of h's roots in column (rho_i, phi0_k)
// exactly as the vote casts them:
//   own(h)   some b == j,   pool(h)   some |b - j| <= pool;
//   seed layers: the layers with exactly one own hit (at least three); the
//   first, the last, and the one between them nearest their middle index;
//   seed circle: through those three own hits;
//   inliers: per layer, the pool hit closest to the circle (smaller hit
//   index on a tie) if its distance is below tol;
//   confirmed iff the inlier layers number at least min_layers.
// Then each hit goes to the confirmed candidate that lists it with the most
// inlier layers, ties to the smallest candidate index.
//
// One warp per candidate, persistent over every candidate of a batch.  The
// bins are decided by the vote's guarded float32 evaluation, redone in
// float64 in the definition's operation order where float32 cannot prove
// them, so own and pool membership are exactly the vote's; the circle and
// the distances are float64 with one correctly rounded operation at a time
// (no contraction), in the order of the plain definition.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tiles.cuh"

namespace ht {


namespace {

// The bins of hit (xf, yf) in column (rho_i, phi0_k), exactly as the vote
// casts them; returns their number (0 to 2) and writes them to j[].
__device__ __forceinline__ int column_bins(const DevGeom &G, float xf, float yf, int i, int k,
                                           int j[2])
{
    const float sk = G.sn32[k], ck = G.cs32[k];
    const float c = fmaf(xf, ck, yf * sk);
    const float R1 = fabsf(xf) + fabsf(yf);
    const float Ec = (kSafe * 3.0f * kEps) * R1;
    if (c < -Ec) return 0;   // c <= 0 proven: the hit is not on a first half turn here
    int edge = 0;
    if (c <= Ec) return cell_bins64(G, xf, yf, i, k, j, &edge);
    const float s = fmaf(xf, sk, -(yf * ck));
    const float r2 = fmaf(xf, xf, yf * yf);
    const float rho = G.rho32[i], invrho = G.invrho32[i];
    const Item it = make_item(G, s, c, r2, R1, fabsf(rho) * 1.0001f);
    int jA, jB, r;
    if (G.rho64[i] != 0.0)
        r = eval32<true>(G, rho, fabsf(invrho) * G.err_scale, invrho, it, jA, jB);
    else
        r = eval32<false>(G, rho, 0.0f, invrho, it, jA, jB);
    if (r == kRedo) return cell_bins64(G, xf, yf, i, k, j, &edge);
    int nv = 0;
    if (jA >= 0) j[nv++] = jA;
    if (jB >= 0) j[nv++] = jB;
    return nv;
}

// Circle through three points: centre = P1 + ((b_y |a|^2 - a_y |b|^2) / d,
// (a_x |b|^2 - b_x |a|^2) / d) with a = P2 - P1, b = P3 - P1,
// d = 2 (a_x b_y - a_y b_x); false when d == 0 (collinear).
__device__ __forceinline__ bool circle3(double x1, double y1, double x2, double y2, double x3,
                                        double y3, double &xc, double &yc, double &R)
{
    const double ax = __dsub_rn(x2, x1), ay = __dsub_rn(y2, y1);
    const double bx = __dsub_rn(x3, x1), by = __dsub_rn(y3, y1);
    const double d = __dmul_rn(2.0, __dsub_rn(__dmul_rn(ax, by), __dmul_rn(ay, bx)));
    if (d == 0.0) return false;
    const double a2 = __dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay));
    const double b2 = __dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by));
    const double ux = __ddiv_rn(__dsub_rn(__dmul_rn(by, a2), __dmul_rn(ay, b2)), d);
    const double uy = __ddiv_rn(__dsub_rn(__dmul_rn(ax, b2), __dmul_rn(bx, a2)), d);
    xc = __dadd_rn(x1, ux);
    yc = __dadd_rn(y1, uy);
    R = __dsqrt_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)));
    return true;
}

// |sqrt((x - xc)^2 + (y - yc)^2) - R|
__device__ __forceinline__ double circle_dist(float xf, float yf, double xc, double yc, double R)
{
    const double dx = __dsub_rn((double)xf, xc), dy = __dsub_rn((double)yf, yc);
    return fabs(__dsub_rn(__dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy))), R));
}

// (d, h) < (bd, bh) lexicographically; h < 0 is "none" (larger than all).
__device__ __forceinline__ bool closer(double d, int h, double bd, int bh)
{
    if (h < 0) return false;
    if (bh < 0) return true;
    return d < bd || (d == bd && h < bh);
}


constexpr int kCfThreads = 256, kCfWarps = kCfThreads / 32;
constexpr int kCfCap = 256;   // pool hits held per pass (more: further passes)

struct CfWarp {
    int n_own[16], own_hit[16];
    int best_h[16];
    double best_d[16];
    int pool_h[kCfCap];
    double pool_d[kCfCap];
    unsigned char pool_l[kCfCap];
};

// Event of flattened candidate f: the last e with cpre[e] <= f (cpre is the
// exclusive prefix of the per-event kept-candidate counts, n_ev + 1 entries).
__device__ __forceinline__ int event_of(const int *cpre, int n_ev, int f)
{
    int lo = 0, hi = n_ev - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cpre[mid] <= f) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One pass over the hit sequence of a candidate: collects the pool hits of
// rank [r0, r0 + kCfCap) into the warp's list (in hit order) and, when
// count_own, the own hits per layer.  Returns the total number of pool hits.
__device__ __forceinline__ int scan_pool(const DevGeom &G, const float *__restrict__ x,
                                         const float *__restrict__ y,
                                         const uint8_t *__restrict__ layer, const int *hl,
                                         int nl, int i, int j, int k, int pool, int r0,
                                         bool count_own, CfWarp &W, int lane)
{
    int rank = 0;
    for (int base = 0; base < nl; base += 32) {
        const int p = base + lane;
        int h = -1, l = 0;
        bool own = false, inp = false;
        if (p < nl) {
            h = hl ? __ldg(hl + p) : p;
            int jj[2];
            const int nv = column_bins(G, __ldg(x + h), __ldg(y + h), i, k, jj);
            for (int v = 0; v < nv; ++v) {
                own |= jj[v] == j;
                inp |= abs(jj[v] - j) <= pool;
            }
            if (inp) l = __ldg(layer + h) & 15;   // layers are 0 .. 15 (bounds the per-layer arrays)
        }
        if (count_own && own) {
            atomicAdd(&W.n_own[l], 1);
            W.own_hit[l] = h;   // read only where the layer holds exactly one own hit
        }
        const unsigned bal = __ballot_sync(0xffffffffu, inp);
        const int r = rank + __popc(bal & ((1u << lane) - 1u));
        if (inp && r >= r0 && r < r0 + kCfCap) {
            W.pool_h[r - r0] = h;
            W.pool_l[r - r0] = (unsigned char)l;
        }
        rank += __popc(bal);
    }
    __syncwarp();
    return rank;
}

// Confirmation of every kept candidate of a batch (see the file comment).
// Event e's hits are x[off[e] ..), its candidates peaks[e cap ..
// e cap + min(counts[e], cap)); cpre: exclusive prefix of those kept counts
// (cpre[n_ev] = total).  Outputs per candidate slot e cap + m: score (0 =
// not confirmed) and inl[16 (e cap + m) + l] (event-local inlier hit of
// layer l, -1 none).  bk (ent null for none): per-event hit lists by column
// group -- a superset of the hits with a root in any column of the group.
__global__ void __launch_bounds__(kCfThreads)
k_confirm(DevGeom G, ConfirmDev P, const float *__restrict__ x, const float *__restrict__ y,
          const uint8_t *__restrict__ layer, const int *__restrict__ off,
          const int *__restrict__ d_nev, const ht_peak *__restrict__ peaks, int cap,
          const int *__restrict__ cpre, int *__restrict__ score, int *__restrict__ inl,
          int *__restrict__ head, BucketView bk)
{
    __shared__ CfWarp sw[kCfWarps];
    const int lane = threadIdx.x & 31;
    CfWarp &W = sw[threadIdx.x >> 5];
    const int n_ev = *d_nev;
    const int total = cpre[n_ev];
    for (;;) {
        int f = 0;
        if (lane == 0) f = atomicAdd(head, 1);
        f = __shfl_sync(0xffffffffu, f, 0);
        if (f >= total) break;
        const int e = event_of(cpre, n_ev, f);
        const int m = f - cpre[e];
        const size_t slot = (size_t)e * cap + m;
        const ht_peak pk = peaks[slot];
        const int a = off[e], n = off[e + 1] - a;
        const int *hl = nullptr;
        int nl = n;
        if (bk.ent) bk.list(e, pk.k_phi0, hl, nl);
        if (lane < 16) {
            W.n_own[lane] = 0;
            W.best_h[lane] = -1;
            W.best_d[lane] = 0.0;
        }
        __syncwarp();
        const float *xe = x + a, *ye = y + a;
        const uint8_t *le = layer + a;
        const int npool = scan_pool(G, xe, ye, le, hl, nl, pk.i_rho, pk.j_d0, pk.k_phi0, P.pool,
                                    0, true, W, lane);
        // seed layers (every lane computes the same)
        int la = -1, lc = -1, ns = 0;
        for (int l = 0; l < P.n_layers; ++l)
            if (W.n_own[l] == 1) {
                if (la < 0) la = l;
                lc = l;
                ++ns;
            }
        int lb = -1, gap = 1 << 30;
        for (int l = la + 1; ns >= 3 && l < lc; ++l)
            if (W.n_own[l] == 1 && abs(2 * l - (la + lc)) < gap) {
                gap = abs(2 * l - (la + lc));
                lb = l;
            }
        double xc = 0.0, yc = 0.0, R = 0.0;
        bool ok = ns >= 3;
        if (ok) {
            const int ha = W.own_hit[la], hb = W.own_hit[lb], hc = W.own_hit[lc];
            ok = circle3((double)xe[ha], (double)ye[ha], (double)xe[hb], (double)ye[hb],
                         (double)xe[hc], (double)ye[hc], xc, yc, R);
        }
        int sc = 0;
        if (ok) {
            for (int r0 = 0; r0 < npool; r0 += kCfCap) {
                if (r0 > 0)
                    scan_pool(G, xe, ye, le, hl, nl, pk.i_rho, pk.j_d0, pk.k_phi0, P.pool, r0,
                              false, W, lane);
                const int nq = min(npool - r0, kCfCap);
                for (int q = lane; q < nq; q += 32) {
                    const int h = W.pool_h[q];
                    W.pool_d[q] = circle_dist(xe[h], ye[h], xc, yc, R);
                }
                __syncwarp();
                for (int l = 0; l < P.n_layers; ++l) {
                    double bd = 0.0;
                    int bh = -1;
                    for (int q = lane; q < nq; q += 32)
                        if (W.pool_l[q] == l && closer(W.pool_d[q], W.pool_h[q], bd, bh)) {
                            bd = W.pool_d[q];
                            bh = W.pool_h[q];
                        }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const double od = __shfl_xor_sync(0xffffffffu, bd, o);
                        const int oh = __shfl_xor_sync(0xffffffffu, bh, o);
                        if (closer(od, oh, bd, bh)) {
                            bd = od;
                            bh = oh;
                        }
                    }
                    if (lane == 0 && closer(bd, bh, W.best_d[l], W.best_h[l])) {
                        W.best_d[l] = bd;
                        W.best_h[l] = bh;
                    }
                }
                __syncwarp();
            }
            for (int l = 0; l < P.n_layers; ++l)
                sc += (W.best_h[l] >= 0 && W.best_d[l] < P.tol) ? 1 : 0;
        }
        const bool conf = ok && sc >= P.min_layers;
        if (lane < 16) {
            const bool in = conf && lane < P.n_layers && W.best_h[lane] >= 0 &&
                            W.best_d[lane] < P.tol;
            inl[slot * 16 + lane] = in ? W.best_h[lane] : -1;
        }
        if (lane == 0) score[slot] = conf ? sc : 0;
        __syncwarp();
    }
}


// cpre[e] = sum over events before e of min(counts[e], cap); cpre[n_ev] is
// the total.  One block; n_ev <= 4096.
__global__ void __launch_bounds__(1024)
k_cand_prefix(const int *__restrict__ counts, const int *__restrict__ d_nev, int cap,
              int *__restrict__ cpre)
{
    __shared__ int part[1024];
    const int n_ev = *d_nev;
    const int per = (n_ev + 1023) / 1024;
    const int e0 = threadIdx.x * per;
    int sum = 0;
    for (int e = e0; e < min(e0 + per, n_ev); ++e) sum += min(counts[e], cap);
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {   // inclusive scan (Hillis-Steele)
        const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int e = e0; e < min(e0 + per, n_ev); ++e) {
        cpre[e] = run;
        run += min(counts[e], cap);
    }
    if (threadIdx.x == 1023) cpre[n_ev] = part[1023];
}

// Final assignment: every inlier of a confirmed candidate offers the key
// score << 32 | (2^32 - 1 - m) to its hit; the largest wins (most inlier
// layers, then the smallest candidate index).  gbest (batch hit index) must
// be zero; k_assoc_final_batch decodes it.
__global__ void k_confirm_offer(const int *__restrict__ off, const int *__restrict__ d_nev,
                                const int *__restrict__ cpre, int cap,
                                const int *__restrict__ score, const int *__restrict__ inl,
                                unsigned long long *__restrict__ gbest)
{
    const int n_ev = *d_nev;
    const long long total = (long long)cpre[n_ev] * 16;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(t >> 4), l = (int)(t & 15);
        const int e = event_of(cpre, n_ev, f);
        const int m = f - cpre[e];
        const size_t slot = (size_t)e * cap + m;
        const int sc = score[slot];
        if (sc <= 0) continue;
        const int h = inl[slot * 16 + l];
        if (h < 0) continue;
        atomicMax(&gbest[off[e] + h],
                  ((unsigned long long)sc << 32) | (0xffffffffull - (unsigned)m));
    }
}

__global__ void k_single_offsets(int *__restrict__ off, int *__restrict__ nev, int n)
{
    off[0] = 0;
    off[1] = n;
    nev[0] = 1;
}

}  // namespace

cudaError_t launch_assoc_final_batch(const unsigned long long *gbest, const int *off,
                                     const int *d_nev, int *assign, int max_hits, cudaStream_t st);

// Confirmation and final assignment of a batch (device offsets and event
// count).  ws: confirm_workspace_bytes(max_events, max_hits).
size_t confirm_workspace_bytes(int max_events, int max_hits)
{
    return align256((size_t)(max_events + 1) * 4) + align256(64) +
           align256((size_t)(max_hits > 0 ? max_hits : 1) * 8);
}

cudaError_t launch_confirm_batch(const DevGeom &G, const ConfirmDev &P, const float *x,
                                 const float *y, const uint8_t *layer, const int *off,
                                 const int *d_nev, int max_events, int max_hits,
                                 const ht_peak *peaks, const int *counts, int cap, int *score,
                                 int *inl, int *assign, void *ws, int sms, cudaStream_t st,
                                 const HitBuckets *hb)
{
    char *w = reinterpret_cast<char *>(ws);
    int *cpre = reinterpret_cast<int *>(w);
    w += align256((size_t)(max_events + 1) * 4);
    int *head = reinterpret_cast<int *>(w);
    w += align256(64);
    unsigned long long *gbest = reinterpret_cast<unsigned long long *>(w);
    cudaError_t e = cudaMemsetAsync(head, 0, 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(gbest, 0, (size_t)max_hits * 8, st);
    if (e != cudaSuccess) return e;
    k_cand_prefix<<<1, 1024, 0, st>>>(counts, d_nev, cap, cpre);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_confirm, kCfThreads, 0);
    k_confirm<<<sms * (occ > 0 ? occ : 1), kCfThreads, 0, st>>>(
        G, P, x, y, layer, off, d_nev, peaks, cap, cpre, score, inl, head, bucket_view(hb));
    k_confirm_offer<<<sms * 8, 256, 0, st>>>(off, d_nev, cpre, cap, score, inl, gbest);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_assoc_final_batch(gbest, off, d_nev, assign, max_hits, st);
}

// One event (host hit count n, device candidate count d_count).
size_t confirm_workspace_bytes_single(int n)
{
    return align256(16) + confirm_workspace_bytes(1, n);
}

cudaError_t launch_confirm(const DevGeom &G, const ConfirmDev &P, const float *x, const float *y,
                           const uint8_t *layer, int n, const ht_peak *peaks, const int *d_count,
                           int cap, int *score, int *inl, int *assign, void *ws, cudaStream_t st)
{
    int *meta = reinterpret_cast<int *>(ws);   // off[2], n_ev
    k_single_offsets<<<1, 1, 0, st>>>(meta, meta + 2, n);
    return launch_confirm_batch(G, P, x, y, layer, meta, meta + 2, 1, n, peaks, d_count, cap,
                                score, inl, assign, reinterpret_cast<char *>(ws) + align256(16),
                                device_sms(), st, nullptr);
}

}  // namespace ht
