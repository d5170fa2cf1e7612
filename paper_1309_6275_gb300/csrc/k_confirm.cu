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
// One warp per candidate, persistent over the candidates of a batch grouped
// by (event, column group).  A candidate scans only the hits of each layer
// whose azimuth can give a root near its bin (a per-event index by layer and
// azimuth, k_hitindex.cu; a superset of the pool).  Each of those hits
// gets the vote's exact bin decision (guarded float32, then double-float,
// then float64 in the definition's operation order), so own and pool
// membership are exactly the vote's.  The seed circle is float64 in the definition's order;
// distances are estimated in float32 with an error bound, and the float64
// distance of the definition is computed for every hit the bound cannot
// settle, so every decision is the definition's.  The results are
// bit-identical to the float64 plain definition.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tiles.cuh"

namespace ht {


namespace {

// Per-candidate constants of its column (rho_i, phi0_k) for column_bins.
struct ColumnCtx {
    int i, k;
    float sk, ck, rho, invrho, invrho_es, rt;
    bool has_b;

    __device__ __forceinline__ void init(const DevGeom &G, int i_, int k_)
    {
        i = i_;
        k = k_;
        sk = G.sn32[k];
        ck = G.cs32[k];
        rho = G.rho32[i];
        invrho = G.invrho32[i];
        invrho_es = fabsf(invrho) * G.err_scale;
        rt = fabsf(rho) * 1.0001f;
        has_b = G.rho64[i] != 0.0;
    }
};

// The bins of hit (xf, yf) in the candidate's column, exactly as the vote
// casts them (guarded float32, then the vote's double-float and float64
// tiers for what float32 cannot prove); returns their number (0 to 2) and
// writes them to j[].
__device__ __forceinline__ int column_bins(const DevGeom &G, const ColumnCtx &C, float xf,
                                           float yf, int j[2])
{
    const float c = fmaf(xf, C.ck, yf * C.sk);
    const float R1 = fabsf(xf) + fabsf(yf);
    const float Ec = (kSafe * 3.0f * kEps) * R1;
    if (c < -Ec) return 0;   // c <= 0 proven: the hit is not on a first half turn here
    if (c <= Ec) return redo_bins(G, xf, yf, C.i, C.k, j);
    const float s = fmaf(xf, C.sk, -(yf * C.ck));
    const float r2 = fmaf(xf, xf, yf * yf);
    const Item it = make_item(G, s, c, r2, R1, C.rt);
    int jA, jB, r;
    if (C.has_b)
        r = eval32<true>(G, C.rho, C.invrho_es, C.invrho, it, jA, jB);
    else
        r = eval32<false>(G, C.rho, 0.0f, C.invrho, it, jA, jB);
    if (r == kRedo) return redo_bins(G, xf, yf, C.i, C.k, j);
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

// Float32 frame of the seed circle at its first point P1, for the distance
// estimate t(w) = (k |w|^2 - 2 w.n) / (|k w - n| + 1), w = P - P1 (exact for
// a unit n towards the centre and k = 1 / R), and the coefficients of a
// bound e(w) = B2 |w|^2 + B1 (|w_x| + |w_y|) + B0 on |t(w)| minus the
// float64 distance of the definition (circle3, then circle_dist).  With
// a = P2 - P1, b = P3 - P1 (exact in float64), c = a_x b_y - a_y b_x and
// v = (b_y |a|^2 - a_y |b|^2, a_x |b|^2 - b_x |a|^2), the centre is
// P1 + v / (2 c) and |v| = |a| |b| |b - a|, so n = sign(c) v / |v| and
// k = 2 |c| / |v|: v and c take float64 products and sums only (no division
// or square root), the rest is float32.  The terms of the bound, u = 2^-24,
// r = (|a| + |b|) / |b - a|, S = |a| |b| / |c| (one over the sine of the
// angle at P1):
//  - turning n by an angle moves t by at most |w| times it (a rotation
//    about P1), a norm 1 + eta by at most 3 |eta| |w|: 13 u |w| for float32,
//    2^-53 (6 sqrt2 r + 1) |w| for the float64 error of v;
//  - |dt/dk| <= 2 |w|^2 (a circle through P1 is within |w| of P), times
//    k's relative error 5.5 u + 2^-53 (S + 8.5 r + 2);
//  - the float64 definition is within 2^-53 R (17 r + 2 S + 13) (+1e-12 cm)
//    of the exact circle through the three points (R = 1 / k);
//  - the float32 evaluation of t: 6e-7 (k |w|^2 + 2 (|w_x| + |w_y|)) + 1e-6
//    cm;
// each first-order and taken with a margin.  Returns false exactly when
// circle3 does (c == 0 in its operation order).  A degenerate frame (an
// underflow, r or S huge) gets B0 = +inf, which sends every distance to the
// float64 definition.
struct SeedFrame {
    float x1, y1, nx, ny, kap, B0, B1, B2;
};

__device__ __forceinline__ bool seed_frame(float x1, float y1, float x2, float y2, float x3,
                                           float y3, SeedFrame &F)
{
    const double ax = __dsub_rn((double)x2, (double)x1), ay = __dsub_rn((double)y2, (double)y1);
    const double bx = __dsub_rn((double)x3, (double)x1), by = __dsub_rn((double)y3, (double)y1);
    const double c = __dsub_rn(__dmul_rn(ax, by), __dmul_rn(ay, bx));
    if (c == 0.0) return false;
    const double a2 = __fma_rn(ax, ax, __dmul_rn(ay, ay));
    const double b2 = __fma_rn(bx, bx, __dmul_rn(by, by));
    const float vx = (float)__fma_rn(by, a2, -__dmul_rn(ay, b2));
    const float vy = (float)__fma_rn(ax, b2, -__dmul_rn(bx, a2));
    const float cf = fabsf((float)c);
    const float vn = sqrtf(fmaf(vx, vx, vy * vy));
    const float ex = (float)__dsub_rn((double)x3, (double)x2);
    const float ey = (float)__dsub_rn((double)y3, (double)y2);
    const float la = sqrtf((float)a2), lb = sqrtf((float)b2);
    const float r = 1.001f * (la + lb) / sqrtf(fmaf(ex, ex, ey * ey));
    const float S = 1.001f * (la * lb) / cf;
    F.x1 = x1;
    F.y1 = y1;
    if (!(vn > 0.0f && vn < 3.0e38f && cf > 0.0f && r < 1.0e6f && S < 1.0e9f)) {
        F.nx = 1.0f;
        F.ny = 0.0f;
        F.kap = 0.0f;
        F.B2 = F.B1 = 0.0f;
        F.B0 = __int_as_float(0x7f800000);
        return true;
    }
    const float sg = c > 0.0 ? 1.0f : -1.0f;
    F.nx = sg * (vx / vn);
    F.ny = sg * (vy / vn);
    F.kap = 2.0f * cf / vn;
    const float R = vn / (2.0f * cf);
    F.B2 = F.kap * (1.3e-6f + 2.5e-16f * S + 2.2e-15f * r + 5e-16f);
    F.B1 = 2.0e-6f + 1.2e-15f * r;
    F.B0 = 1.0e-6f + 1.0e-12f + 1.22e-16f * R * (17.0f * r + 2.0f * S + 13.0f);
    return true;
}

constexpr int kCfThreads = 128, kCfWarps = kCfThreads / 32;
constexpr int kCfCap = 384;        // pool hits held per pass (more: further passes)
constexpr int kCfBlk = 256;        // 32-hit blocks of a scan whose pool counts are kept

struct CfWarp {
    int n_own[16], own_pos[16];
    int best_h[16];
    double best_d[16];
    // per layer, over the pool hits of the pass: least lower and upper bound
    // of a distance (float bits), contenders (count, one of them) and the
    // pass's positions [qs, qe) (the pool is in layer order)
    unsigned lbmin[16], ubmin[16];
    int ncont[16], cq[16], qs[16], qe[16];
    int rs[32], rp[33];     // runs of index positions scanned: start, exclusive prefix of lengths
    unsigned short blk[kCfBlk];   // pool hits of each 32-hit block of the first pass
    int pool_p[kCfCap], pool_h[kCfCap];   // index position and event-local hit index
    float pool_lo[kCfCap], pool_hi[kCfCap];   // bounds on the hit's float64 distance
    unsigned char pool_l[kCfCap];
    SeedFrame F;            // the candidate's float32 seed frame
    double xc, yc, R;       // and its float64 seed circle, once computed
    int seed_pos[3];        // index positions of the three seed hits
};

// The warps' state of k_confirm (at namespace scope, so that the functions
// that take a warp's index address it as shared memory).
__shared__ CfWarp g_cfw[kCfWarps];

// The hits a candidate scans: the t-th of the runs W.rs / W.rp of the
// event's hit index (k_hitindex.cu).
struct HitView {
    const float *x, *y;
    const int *h;
    const uint8_t *l;
    int wid;   // the warp's state in g_cfw
    int n;     // total positions

    __device__ __forceinline__ int pos(int t) const
    {
        int lo = 0, hi = 31;   // the last run r with rp[r] <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (g_cfw[wid].rp[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        return g_cfw[wid].rs[lo] + (t - g_cfw[wid].rp[lo]);
    }
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

// Azimuth window of the hits of one layer that can have a root within
// d0 in [lo, hi] (cm) in column (rho, phi0_k); returns its runs of index
// cells as bins [b0, b1] (b1 - b0 + 1 >= kIdxAz or full: the whole layer;
// empty: no hit can).  A root d0 of the circle equation gives
//   s = -(2 d0 + rho (d0^2 + r^2)) / (2 u),   u = 1 + rho d0,
// with ds/dd0 = -(u^2 + 1 - rho^2 r^2) / (2 u^2) and ds/d(r^2) = -rho / (2 u):
// for u > 0, s is monotone in r^2 (sign -rho), and in d0 (decreasing) while
// u^2 + 1 > rho^2 r^2; otherwise |ds/dd0| <= (1 + (1 + rho^2 r^2) / u^2) / 2
// bounds it around the middle of [lo, hi].  So over the window and the
// layer's radius range [rmin, rmax] s lies in an interval given by two
// corners (or the middle and that bound); with c > 0 the hit's azimuth is
// phi0_k - asin(s / r).  A layer beyond the circles' reach (the farthest
// point of a circle with perigee d0 is |d0 + 1/rho| + 1/|rho| from the
// origin) is empty.  Margins (1e-3 cm plus 1e-5 relative on s and on the
// reach, 2e-3 rad on the azimuth) cover float32 rounding; where u > 0 is not
// proven the whole layer is scanned.
__device__ __forceinline__ void layer_window(float rho, float phik, float lo, float hi,
                                             float rmin, float rmax, bool &full, bool &empty,
                                             int &b0, int &b1)
{
    full = false;
    empty = !(rmin <= rmax);
    b0 = b1 = 0;
    if (empty) return;
    const float tl = fmaf(rho, lo, 1.0f), th = fmaf(rho, hi, 1.0f);
    const float tmin = fminf(tl, th);
    if (!(tmin >= 0.05f) || !(rmin >= 1e-3f)) {
        full = true;
        return;
    }
    const float ir = 1.0f / rho;   // +-inf for rho = 0: no reach limit
    const float reach = fmaxf(fabsf(lo + ir), fabsf(hi + ir)) + fabsf(ir);
    if (rmin > fmaf(reach, 1.0f + 1e-5f, 1e-3f)) {
        empty = true;
        return;
    }
    const float rA = rho > 0.0f ? rmin : rmax, rB = rho > 0.0f ? rmax : rmin;
    float s_hi, s_lo;
    if (fmaf(rho * rho * 1.001f, rmax * rmax, 1e-3f) < fmaf(tmin, tmin, 1.0f)) {
        s_hi = -fmaf(rho, fmaf(lo, lo, rA * rA), 2.0f * lo) / (2.0f * tl);
        s_lo = -fmaf(rho, fmaf(hi, hi, rB * rB), 2.0f * hi) / (2.0f * th);
    } else {
        const float mid = 0.5f * (lo + hi), tm = fmaf(rho, mid, 1.0f);
        const float L = 0.5f * (1.0f + fmaf(rho * rho, rmax * rmax, 1.0f) / (tmin * tmin));
        const float ds = 1.001f * L * 0.5f * (hi - lo);
        s_hi = -fmaf(rho, fmaf(mid, mid, rA * rA), 2.0f * mid) / (2.0f * tm) + ds;
        s_lo = -fmaf(rho, fmaf(mid, mid, rB * rB), 2.0f * mid) / (2.0f * tm) - ds;
    }
    const float ms = fmaf(1e-5f, fabsf(s_hi) + fabsf(s_lo), 1e-3f);
    s_hi += ms;
    s_lo -= ms;
    const float a_hi = s_hi / (s_hi > 0.0f ? rmin : rmax);
    const float a_lo = s_lo / (s_lo < 0.0f ? rmin : rmax);
    if (a_lo > 1.0f || a_hi < -1.0f) {
        empty = true;
        return;
    }
    const float dmax = asinf(fminf(a_hi, 1.0f)), dmin = asinf(fmaxf(a_lo, -1.0f));
    const float k = kIdxAz / 6.28318531f;
    b0 = (int)floorf((phik - dmax - 2e-3f + 3.14159265f) * k);
    b1 = (int)floorf((phik - dmin + 2e-3f + 3.14159265f) * k);
    if (b1 - b0 + 1 >= kIdxAz) full = true;
}

// One pass over a candidate's hit sequence: collects the pool hits of rank
// [r0, r0 + kCfCap) into the warp's list (in sequence order) and, when
// count_own (the first pass, r0 = 0), the own hits per layer.  Returns the
// total number of pool hits (first pass).  Every scanned hit gets the
// vote's exact bin decision in the candidate's column, one hit per lane
// (the index windows already hold few hits far from the pool, so no cheaper
// screen pays for itself).  The first pass keeps each 32-hit block's pool
// count, so a later pass evaluates only the blocks whose pool hits can fall
// in its rank range.
__device__ __noinline__ int scan_pool(const DevGeom &G, const HitView V, int i, int j, int k,
                                      int pool, int r0, bool count_own, int lane)
{
    CfWarp &W = g_cfw[V.wid];
    ColumnCtx C;
    C.init(G, i, k);
    const unsigned lt = (1u << lane) - 1u;
    int rank = 0;
    for (int base = 0; base < V.n; base += 32) {
        const int b = base >> 5;
        if (!count_own && b < kCfBlk) {   // uniform
            const int cnt = W.blk[b];
            if (rank + cnt <= r0) {
                rank += cnt;
                continue;
            }
            if (rank >= r0 + kCfCap) break;
        }
        const int t = base + lane;
        int p = -1, l = 0;
        bool own = false, inp = false;
        if (t < V.n) {
            p = V.pos(t);
            int jj[2];
            const int nv = column_bins(G, C, V.x[p], V.y[p], jj);
            for (int v = 0; v < nv; ++v) {
                own |= jj[v] == j;
                inp |= abs(jj[v] - j) <= pool;
            }
            if (inp) l = V.l[p];
        }
        if (count_own && own) {
            atomicAdd(&W.n_own[l], 1);
            W.own_pos[l] = p;   // read only where the layer holds exactly one own hit
        }
        const unsigned bal = __ballot_sync(0xffffffffu, inp);
        const int r = rank + __popc(bal & lt);
        if (inp && r >= r0 && r < r0 + kCfCap) {
            W.pool_p[r - r0] = p;
            W.pool_h[r - r0] = V.h[p];
            W.pool_l[r - r0] = (unsigned char)l;
        }
        if (count_own && lane == 0 && b < kCfBlk) W.blk[b] = (unsigned short)__popc(bal);
        rank += __popc(bal);
    }
    __syncwarp();
    return rank;
}

// The runs of index positions a candidate of event e in column (rho_i,
// phi0_k) with bin j scans: per layer its azimuth window (layer_window) for
// d0 within two bins beyond the pool, as one or two runs of cells (the
// window may wrap); lane r takes run r = 2 l + part.
__device__ __forceinline__ void candidate_runs(const DevGeom &G, const ConfirmDev &P,
                                               const HitIndex &I, int e, int i, int j, int k,
                                               CfWarp &W, HitView &V, int lane)
{
    const int l = lane >> 1, part = lane & 1;
    int start = 0, len = 0;
    if (l < P.n_layers) {
        const float lo = ((float)(j - P.pool - 2) - G.off_f) * G.delta_f;
        const float hi = ((float)(j + P.pool + 3) - G.off_f) * G.delta_f;
        const float rmin = __uint_as_float(I.rmm[2 * (e * 16 + l)]);
        const float rmax = __uint_as_float(I.rmm[2 * (e * 16 + l) + 1]);
        bool full, empty;
        int b0, b1;
        layer_window(G.rho32[i], G.phi32[k], lo, hi, rmin, rmax, full, empty, b0, b1);
        const int base = (e * 16 + l) * kIdxAz;
        if (full) {
            if (part == 0) {
                start = I.offs[base];
                len = I.offs[base + kIdxAz] - start;
            }
        } else if (!empty) {
            const int b0m = ((b0 % kIdxAz) + kIdxAz) % kIdxAz, nb = b1 - b0 + 1;
            if (b0m + nb <= kIdxAz) {
                if (part == 0) {
                    start = I.offs[base + b0m];
                    len = I.offs[base + b0m + nb] - start;
                }
            } else if (part == 0) {
                start = I.offs[base + b0m];
                len = I.offs[base + kIdxAz] - start;
            } else {
                start = I.offs[base];
                len = I.offs[base + b0m + nb - kIdxAz] - start;
            }
        }
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    W.rs[lane] = start;
    W.rp[lane + 1] = incl;
    if (lane == 0) W.rp[0] = 0;
    __syncwarp();
    V.n = W.rp[32];
}

// Confirmation of one candidate by one warp (see the file comment).  Writes
// score[slot] (0 = not confirmed) and inl[16 slot + l].
//
// Distances: the float32 estimate of seed_frame and its bound give every
// pool hit an interval [lo, hi] holding its float64 distance.  Per layer
// the contenders are the hits with lo at most the layer's least hi and
// below tol; the layer's nearest hit is one of them.  A layer without a
// contender has no inlier, a single contender certainly below tol is the
// inlier, and otherwise the float64 distances of the contenders decide
// (the definition's seed circle is computed then, once per candidate).
// When fewer than min_layers layers can hold an inlier the candidate is not
// confirmed, without any float64 distance.  Pools larger than kCfCap go in
// passes of kCfCap hits, every contender by its float64 distance.
__device__ __forceinline__ void confirm_one(const DevGeom &G, const ConfirmDev &P,
                                            const HitIndex &I, int e, const ht_peak pk,
                                            size_t slot, float tol_lo, float tol_hi,
                                            int *__restrict__ score, int *__restrict__ inl,
                                            int wid, int lane)
{
    CfWarp &W = g_cfw[wid];
    constexpr unsigned kAll = 0xffffffffu;
    const float kInf = __int_as_float(0x7f800000);
    HitView V{I.x, I.y, I.h, I.l, wid, 0};
    candidate_runs(G, P, I, e, pk.i_rho, pk.j_d0, pk.k_phi0, W, V, lane);
    if (lane < 16) {
        W.n_own[lane] = 0;
        W.best_h[lane] = -1;
        W.best_d[lane] = 0.0;
    }
    __syncwarp();
    const long long tol_bits = __double_as_longlong(P.tol);
    const SeedFrame &F = W.F;
    bool ok = false, exact = false, rejected = false;
    const int npool = scan_pool(G, V, pk.i_rho, pk.j_d0, pk.k_phi0, P.pool, 0, true, lane);
    {
        // seed layers (every lane computes the same)
        int la = -1, lb = -1, lc = -1, ns = 0;
        for (int l = 0; l < P.n_layers; ++l)
            if (W.n_own[l] == 1) {
                if (la < 0) la = l;
                lc = l;
                ++ns;
            }
        int gap = 1 << 30;
        for (int l = la + 1; ns >= 3 && l < lc; ++l)
            if (W.n_own[l] == 1 && abs(2 * l - (la + lc)) < gap) {
                gap = abs(2 * l - (la + lc));
                lb = l;
            }
        if (ns >= 3) {
            if (lane == 0) {
                const int pa = W.own_pos[la], pb = W.own_pos[lb], pc = W.own_pos[lc];
                const bool f = seed_frame(V.x[pa], V.y[pa], V.x[pb], V.y[pb], V.x[pc], V.y[pc], W.F);
                W.seed_pos[0] = f ? pa : -1;
                W.seed_pos[1] = pb;
                W.seed_pos[2] = pc;
            }
            __syncwarp();
            ok = W.seed_pos[0] >= 0;
        }
    }
    for (int r0 = 0; ok && r0 < npool; r0 += kCfCap) {
        if (r0 > 0) scan_pool(G, V, pk.i_rho, pk.j_d0, pk.k_phi0, P.pool, r0, false, lane);
        const bool single = npool <= kCfCap;
        const int nq = min(npool - r0, kCfCap);
        if (lane < 16) {
            W.lbmin[lane] = W.ubmin[lane] = 0x7f800000u;   // +inf
            W.ncont[lane] = 0;
            W.qs[lane] = kCfCap;
            W.qe[lane] = 0;
        }
        __syncwarp();
        // the bounds of every pool hit, and their least values per layer
        // (the pool is in layer order: each layer is one run of lanes)
        for (int q0 = 0; q0 < nq; q0 += 32) {
            const int q = q0 + lane;
            int l = 16;
            float lo = kInf, hi = kInf;
            if (q < nq) {
                const int p = W.pool_p[q];
                l = W.pool_l[q];
                const float wx = V.x[p] - F.x1, wy = V.y[p] - F.y1;
                const float w2 = fmaf(wx, wx, wy * wy);
                const float wn = fmaf(wx, F.nx, wy * F.ny);
                const float num = fmaf(F.kap, w2, -2.0f * wn);
                const float qx = fmaf(F.kap, wx, -F.nx), qy = fmaf(F.kap, wy, -F.ny);
                const float d = fabsf(num / (sqrtf(fmaf(qx, qx, qy * qy)) + 1.0f));
                const float er = fmaf(F.B2, w2, fmaf(F.B1, fabsf(wx) + fabsf(wy), F.B0));
                const float dl = __fsub_rd(d, er);
                lo = dl > 0.0f ? dl : 0.0f;   // +0 (the bits order as the values)
                hi = __fadd_ru(d, er);
                W.pool_lo[q] = lo;
                W.pool_hi[q] = hi;
            }
            float slo = lo, shi = hi;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float olo = __shfl_down_sync(kAll, slo, o);
                const float ohi = __shfl_down_sync(kAll, shi, o);
                const int ol = __shfl_down_sync(kAll, l, o);
                if (lane + o < 32 && ol == l) {
                    slo = fminf(slo, olo);
                    shi = fminf(shi, ohi);
                }
            }
            const int lp = __shfl_up_sync(kAll, l, 1), ln = __shfl_down_sync(kAll, l, 1);
            if (q < nq && (lane == 0 || lp != l)) {
                atomicMin(&W.lbmin[l], __float_as_uint(slo));
                atomicMin(&W.ubmin[l], __float_as_uint(shi));
                atomicMin(&W.qs[l], q);
            }
            if (q < nq && (lane == 31 || ln != l)) atomicMax(&W.qe[l], q + 1);
        }
        __syncwarp();
        if (single) {
            // layers that can hold an inlier at all: too few, not confirmed
            const bool can = lane < P.n_layers && __uint_as_float(W.lbmin[lane]) < tol_hi;
            if (__popc(__ballot_sync(kAll, can)) < P.min_layers) {
                rejected = true;
                break;
            }
        }
        for (int q = lane; q < nq; q += 32) {
            const int l = W.pool_l[q];
            const float lo = W.pool_lo[q];
            if (lo <= __uint_as_float(W.ubmin[l]) && lo < tol_hi) {
                atomicAdd(&W.ncont[l], 1);
                W.cq[l] = q;   // read only where the layer has one contender
            }
        }
        __syncwarp();
        bool need = false;
        if (lane < P.n_layers) {
            const int nc = W.ncont[lane];
            if (single && nc == 1 && W.pool_hi[W.cq[lane]] < tol_lo) {
                W.best_h[lane] = W.pool_h[W.cq[lane]];   // certainly the inlier
                W.best_d[lane] = 0.0;                     // (below tol)
            } else {
                need = nc > 0;
            }
        }
        const unsigned need_m = __ballot_sync(kAll, need);
        if (need_m != 0u && !exact) {
            if (lane == 0) {
                const int pa = W.seed_pos[0], pb = W.seed_pos[1], pc = W.seed_pos[2];
                circle3((double)V.x[pa], (double)V.y[pa], (double)V.x[pb], (double)V.y[pb],
                        (double)V.x[pc], (double)V.y[pc], W.xc, W.yc, W.R);
            }
            __syncwarp();
            exact = true;
        }
        for (unsigned m = need_m; m != 0u; m &= m - 1u) {
            const int l = __ffs(m) - 1;
            const float ub = __uint_as_float(W.ubmin[l]);
            long long bk = 0x7fffffffffffffffll;   // none: above every distance's bits
            int bh = -1;
            for (int q = W.qs[l] + lane; q < W.qe[l]; q += 32) {
                const float lo = W.pool_lo[q];
                if (!(lo <= ub && lo < tol_hi)) continue;
                const int p = W.pool_p[q], h = W.pool_h[q];
                const long long key = __double_as_longlong(circle_dist(V.x[p], V.y[p], W.xc, W.yc, W.R));
                if (key < bk || (key == bk && h < bh)) {
                    bk = key;
                    bh = h;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long ok2 = __shfl_xor_sync(kAll, bk, o);
                const int oh = __shfl_xor_sync(kAll, bh, o);
                if (ok2 < bk || (ok2 == bk && oh < bh)) {
                    bk = ok2;
                    bh = oh;
                }
            }
            if (lane == 0 && bh >= 0) {
                const long long cur = __double_as_longlong(W.best_d[l]);
                if (W.best_h[l] < 0 || bk < cur || (bk == cur && bh < W.best_h[l])) {
                    W.best_d[l] = __longlong_as_double(bk);
                    W.best_h[l] = bh;
                }
            }
        }
        __syncwarp();
    }
    const bool in_l = ok && !rejected && lane < P.n_layers && W.best_h[lane] >= 0 &&
                      __double_as_longlong(W.best_d[lane]) < tol_bits;
    const int sc = __popc(__ballot_sync(kAll, in_l));
    const bool conf = ok && !rejected && sc >= P.min_layers;
    if (lane < 16) inl[slot * 16 + lane] = conf && in_l ? W.best_h[lane] : -1;
    if (lane == 0) score[slot] = conf ? sc : 0;
    __syncwarp();
}

// Confirmation of every kept candidate of a batch.  The candidates are
// ordered by (event, column group of kGroupCols columns) in order[] (flattened
// indices; cpre is the exclusive prefix of the kept counts), so that the
// consecutive candidates are nearby columns of one event; each warp takes
// chunks of kCfChunk consecutive entries from a device counter (*head, zero
// at launch) and confirms them one after another.  I: the batch's hit index
// (k_hitindex.cu).
constexpr int kCfChunk = 8;

__global__ void __launch_bounds__(kCfThreads, 6)
k_confirm(DevGeom G, ConfirmDev P, HitIndex I, const int *__restrict__ d_nev,
          const ht_peak *__restrict__ peaks, int cap, const int *__restrict__ cpre,
          const int *__restrict__ order, int *__restrict__ score, int *__restrict__ inl,
          int *__restrict__ head)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_ev = *d_nev;
    const int total = cpre[n_ev];
    float tol_hi = (float)P.tol;   // tol rounded up to float32
    if ((double)tol_hi < P.tol) tol_hi = nextafterf(tol_hi, 3.0e38f);
    float tol_lo = (float)P.tol;   // and down
    if ((double)tol_lo > P.tol) tol_lo = nextafterf(tol_lo, 0.0f);
    // each warp claims its own chunks (its state in g_cfw is private and it
    // synchronises only itself), so a warp never waits for its CTA's others
    for (;;) {
        int c = 0;
        if (lane == 0) c = atomicAdd(head, 1);
        const int t0 = __shfl_sync(0xffffffffu, c, 0) * kCfChunk;
        if (t0 >= total) break;
        const int t1 = min(t0 + kCfChunk, total);
        for (int t = t0; t < t1; ++t) {
            const int f = __ldg(order + t);
            const int e = event_of(cpre, n_ev, f);
            const size_t slot = (size_t)e * cap + (f - cpre[e]);
            confirm_one(G, P, I, e, peaks[slot], slot, tol_lo, tol_hi, score, inl, warp, lane);
        }
    }
}

// Candidates of each (event, column group) item: counts, then positions.
__global__ void k_cf_group(const int *__restrict__ d_nev, const int *__restrict__ cpre,
                           const ht_peak *__restrict__ peaks, int cap, int ngroups,
                           int *__restrict__ gcnt, int *__restrict__ gcur, int *__restrict__ order)
{
    const int n_ev = *d_nev;
    const int total = cpre[n_ev];
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < total; f += gridDim.x * blockDim.x) {
        const int e = event_of(cpre, n_ev, f);
        const int k = peaks[(size_t)e * cap + (f - cpre[e])].k_phi0;
        const int it = e * ngroups + k / kGroupCols;
        if (gcur) order[atomicAdd(&gcur[it], 1)] = f;
        else atomicAdd(&gcnt[it], 1);
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

size_t scan_tmp_bytes(int n_cap);
cudaError_t scan_exclusive(const int *in, int *out, int *out2, int n_cap, const int *d_n,
                           int *total, void *tmp, cudaStream_t st);

namespace {

struct CfWs {
    int *cpre, *head, *gcnt, *gofs, *gcur, *order;
    unsigned long long *gbest;
    void *tmp;
    HitIndex idx;
};

int cf_groups(const DevGeom &G) { return (G.n_phi0 + kGroupCols - 1) / kGroupCols; }

// Carves (p non-null) or sizes the confirmation workspace.
size_t cf_layout(const DevGeom &G, int max_events, int max_hits, int cap, char *p, CfWs *w)
{
    const size_t ni = (size_t)max_events * cf_groups(G);
    const size_t parts[] = {(size_t)(max_events + 1) * 4, 64, (size_t)(max_hits > 0 ? max_hits : 1) * 8,
                            ni * 4, (ni + 1) * 4, (ni + 1) * 4,
                            (size_t)max_events * (cap > 0 ? cap : 1) * 4,
                            scan_tmp_bytes((int)ni), hit_index_bytes(max_events, max_hits)};
    size_t at = 0;
    char *q[9];
    for (int i = 0; i < 9; ++i) {
        q[i] = p ? p + at : nullptr;
        at += align256(parts[i]);
    }
    if (w) {
        w->cpre = reinterpret_cast<int *>(q[0]);
        w->head = reinterpret_cast<int *>(q[1]);
        w->gbest = reinterpret_cast<unsigned long long *>(q[2]);
        w->gcnt = reinterpret_cast<int *>(q[3]);
        w->gofs = reinterpret_cast<int *>(q[4]);
        w->gcur = reinterpret_cast<int *>(q[5]);
        w->order = reinterpret_cast<int *>(q[6]);
        w->tmp = q[7];
        if (p) w->idx = carve_hit_index(max_events, max_hits, q[8]);
    }
    return at;
}

}  // namespace

cudaError_t prepare_confirm_kernels() { return cudaSuccess; }

// Confirmation and final assignment of a batch (device offsets and event
// count).  ws: confirm_workspace_bytes(G, max_events, max_hits, cap).
size_t confirm_workspace_bytes(const DevGeom &G, int max_events, int max_hits, int cap)
{
    return cf_layout(G, max_events, max_hits, cap, nullptr, nullptr);
}

cudaError_t launch_confirm_batch(const DevGeom &G, const ConfirmDev &P, const float *x,
                                 const float *y, const uint8_t *layer, const int *off,
                                 const int *d_nev, int max_events, int max_hits,
                                 const ht_peak *peaks, const int *counts, int cap, int *score,
                                 int *inl, int *assign, void *ws, int sms, cudaStream_t st,
                                 const HitBuckets *hb)
{
    (void)hb;
    CfWs w;
    cf_layout(G, max_events, max_hits, cap, reinterpret_cast<char *>(ws), &w);
    const int ng = cf_groups(G), ni = max_events * ng;
    cudaError_t e = cudaMemsetAsync(w.head, 0, 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.gbest, 0, (size_t)max_hits * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.gcnt, 0, (size_t)ni * 4, st);
    if (e != cudaSuccess) return e;
    k_cand_prefix<<<1, 1024, 0, st>>>(counts, d_nev, cap, w.cpre);
    // candidates by (event, column group): counts, offsets, positions
    k_cf_group<<<sms * 4, 256, 0, st>>>(d_nev, w.cpre, peaks, cap, ng, w.gcnt, nullptr, nullptr);
    e = scan_exclusive(w.gcnt, w.gofs, w.gcur, ni, nullptr, w.gofs + ni, w.tmp, st);
    if (e != cudaSuccess) return e;
    k_cf_group<<<sms * 4, 256, 0, st>>>(d_nev, w.cpre, peaks, cap, ng, nullptr, w.gcur, w.order);
    e = launch_hit_index(x, y, layer, off, d_nev, max_events, max_hits, w.idx, sms, st);
    if (e != cudaSuccess) return e;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_confirm, kCfThreads, 0);
    k_confirm<<<sms * (occ > 0 ? occ : 1), kCfThreads, 0, st>>>(
        G, P, w.idx, d_nev, peaks, cap, w.cpre, w.order, score, inl, w.head);
    k_confirm_offer<<<sms * 8, 256, 0, st>>>(off, d_nev, w.cpre, cap, score, inl, w.gbest);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_assoc_final_batch(w.gbest, off, d_nev, assign, max_hits, st);
}

// One event (host hit count n, device candidate count d_count).
size_t confirm_workspace_bytes_single(const DevGeom &G, int n, int cap)
{
    return align256(16) + confirm_workspace_bytes(G, 1, n, cap);
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


// ------------------------------------------------------------ compaction
// The confirmed candidates (score > 0) of every event, in candidate order,
// as a compact list of found tracks, and each hit's assignment as an index
// into its event's tracks (ht_batch_run_tracks_host).
namespace {

__global__ void k_track_flags(const int *__restrict__ d_nev, const int *__restrict__ cpre,
                              int cap, const int *__restrict__ score, int *__restrict__ flag)
{
    const int n_ev = *d_nev, total = cpre[n_ev];
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < total; f += gridDim.x * blockDim.x) {
        const int e = event_of(cpre, n_ev, f);
        flag[f] = score[(size_t)e * cap + (f - cpre[e])] > 0 ? 1 : 0;
    }
}

// tfirst[e] = the compact index of event e's first track (e <= n_ev)
__global__ void k_track_first(const int *__restrict__ d_nev, const int *__restrict__ cpre,
                              const int *__restrict__ pos, const int *__restrict__ ntot,
                              int *__restrict__ tfirst)
{
    const int n_ev = *d_nev, total = cpre[n_ev];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e <= n_ev; e += gridDim.x * blockDim.x)
        tfirst[e] = cpre[e] < total ? pos[cpre[e]] : *ntot;
}

__global__ void k_track_write(const int *__restrict__ d_nev, const int *__restrict__ cpre,
                              int cap, const int *__restrict__ flag, const int *__restrict__ pos,
                              const int *__restrict__ tfirst, const ht_peak *__restrict__ peaks,
                              const int *__restrict__ score, const ht_zres *__restrict__ zres,
                              ht_track_out *__restrict__ tracks, int tcap, int *__restrict__ map)
{
    const int n_ev = *d_nev, total = cpre[n_ev];
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < total; f += gridDim.x * blockDim.x) {
        if (!flag[f]) continue;
        const int e = event_of(cpre, n_ev, f);
        const size_t slot = (size_t)e * cap + (f - cpre[e]);
        const int t = pos[f];
        map[slot] = t - tfirst[e];
        if (t < tcap) {
            const ht_peak pk = peaks[slot];
            const ht_zres zr = zres[slot];
            tracks[t] = ht_track_out{pk.i_rho, pk.j_d0, pk.k_phi0, pk.count, score[slot],
                                     zr.n_z0, zr.m_cot, zr.count};
        }
    }
}

__global__ void k_track_assign(const int *__restrict__ off, const int *__restrict__ d_nev,
                               int cap, const int *__restrict__ assign,
                               const int *__restrict__ map, int *__restrict__ out)
{
    const int n_ev = *d_nev, n = off[n_ev];
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
        int lo = 0, hi = n_ev - 1;   // the hit's event
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= h) lo = mid;
            else hi = mid - 1;
        }
        const int a = assign[h];
        out[h] = a >= 0 ? map[(size_t)lo * cap + a] : -1;
    }
}

}  // namespace

size_t track_compact_bytes(int max_events, int cap)
{
    const size_t nk = (size_t)max_events * (cap > 0 ? cap : 1);
    return align256((size_t)(max_events + 1) * 4) + 2 * align256((size_t)(max_events + 1) * 4) +
           3 * align256(nk * 4) + align256(16) + scan_tmp_bytes((int)nk);
}

cudaError_t launch_track_compact(const int *off, const int *d_nev, int max_events, int max_hits,
                                 const ht_peak *peaks, const int *counts, int cap,
                                 const int *score, const ht_zres *zres, const int *assign,
                                 ht_track_out *tracks, int tcap, int *tfirst, int *ntot,
                                 int *assign_out, void *ws, int sms, cudaStream_t st)
{
    const size_t nk = (size_t)max_events * (cap > 0 ? cap : 1);
    char *p = reinterpret_cast<char *>(ws);
    int *cpre = reinterpret_cast<int *>(p);
    p += align256((size_t)(max_events + 1) * 4);
    p += 2 * align256((size_t)(max_events + 1) * 4);
    int *flag = reinterpret_cast<int *>(p);
    p += align256(nk * 4);
    int *pos = reinterpret_cast<int *>(p);
    p += align256(nk * 4);
    int *map = reinterpret_cast<int *>(p);
    p += align256(nk * 4);
    p += align256(16);
    void *tmp = p;
    k_cand_prefix<<<1, 1024, 0, st>>>(counts, d_nev, cap, cpre);
    k_track_flags<<<sms * 4, 256, 0, st>>>(d_nev, cpre, cap, score, flag);
    cudaError_t e = scan_exclusive(flag, pos, nullptr, (int)nk, nullptr, ntot, tmp, st);
    if (e != cudaSuccess) return e;
    k_track_first<<<(max_events + 256) / 256, 256, 0, st>>>(d_nev, cpre, pos, ntot, tfirst);
    k_track_write<<<sms * 4, 256, 0, st>>>(d_nev, cpre, cap, flag, pos, tfirst, peaks, score, zres,
                                            tracks, tcap, map);
    k_track_assign<<<sms * 4, 256, 0, st>>>(off, d_nev, cap, assign, map, assign_out);
    (void)max_hits;
    return cudaGetLastError();
}

}  // namespace ht
