// tiles.cuh -- the vote tile shared by the tile kernels (k_tiles.cu) and
// the masked vote of the learned proposal (k_vote_masked.cu): Hough vote of
// Section 5 of arXiv:1309.6275 over a tile of 32 rho rows x KT phi0 columns
// x all n_d0 bins.  Each translation unit that includes it gets its own copy
// of these kernels (anonymous namespace).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "df32.cuh"
#include "ht_internal.cuh"

namespace ht {
namespace {

constexpr int kThreads = 256;

// Vote modes: the plain vote; one region mask per event (MaskCtx: only halo
// cells of the mask exact); one region set per hit (HitCtx: each hit votes
// only in the halo cells of its own regions, on the 8 x 8 grid of
// ht_internal.cuh).  Association replays votes under kModeEvent with a
// candidate-box window in MaskCtx.
constexpr int kModePlain = 0, kModeEvent = 1, kModeHit = 2;
// Flag on a mode: the distinct-layer vote.  A cell counts the distinct
// detector layers of the hits voting in it (a track leaves at most one hit
// per layer); tile words hold 16-bit layer masks (bit l = layer l), set with
// atomicOr, and the write-back stores their population counts.  An OR never
// carries, so two masks always share a word, whatever the hit count.
constexpr int kModeLayers = 4, kModeBase = 3;

__host__ __device__ constexpr int base_mode(int m) { return m & kModeBase; }
__host__ __device__ constexpr bool layer_mode(int m) { return (m & kModeLayers) != 0; }

template <typename OutT>
__device__ __forceinline__ OutT saturate(uint32_t v)
{
    if (sizeof(OutT) == 2) return (OutT)(v > 65535u ? 65535u : v);
    return (OutT)(v > 2147483647u ? 2147483647u : v);
}

// Shared work list of (hit, column) items.
struct WorkList {
    float4 *a, *b;           // Item fields {s, c, r2, eD}, {E1, E2, Qa, Qb}
    int *meta;               // hit << 6 | needB << 5 | unsure << 4 | column-in-tile
    unsigned long long *hm;  // kModeHit: the hit's region set
    unsigned char *lay;      // kModeLayers: the hit's layer
};

constexpr int kMetaUnsure = 16, kMetaNeedB = 32, kMetaCol = 15;
constexpr size_t kItemBytes = 36;

__host__ __device__ constexpr size_t item_bytes(int mode)
{
    return kItemBytes + (base_mode(mode) == kModeHit ? 8 : 0) + (layer_mode(mode) ? 1 : 0);
}

__device__ __forceinline__ WorkList carve_worklist(unsigned char *p, int cap,
                                                   int mode = kModePlain)
{
    WorkList w;
    w.a = reinterpret_cast<float4 *>(p);
    w.b = w.a + cap;
    w.meta = reinterpret_cast<int *>(w.b + cap);
    w.hm = reinterpret_cast<unsigned long long *>(w.meta + cap);   // cap is a multiple of 2
    w.lay = reinterpret_cast<unsigned char *>(w.hm + (base_mode(mode) == kModeHit ? cap : 0));
    return w;
}

// Constants of one row of a tile as a lane sees it.
struct RowCtx {
    int irow;
    bool row_ok, has_b;
    float rho, invrho, invrho_es;
    float rho2, arho;   // rho^2 and |rho| (float32), for A-form items

    __device__ __forceinline__ void init_row(const DevGeom &G, int i)
    {
        irow = i;
        row_ok = irow < G.n_rho;
        rho = row_ok ? G.rho32[irow] : 0.0f;
        invrho = row_ok ? G.invrho32[irow] : 0.0f;
        has_b = row_ok && (G.rho64[irow] != 0.0);
        invrho_es = fabsf(invrho) * G.err_scale;
        rho2 = rho * rho;
        arho = fabsf(rho);
    }
};

// Per-tile constants of the lane's rows and of the tile's columns.  A tile
// has 32 RW rows: the lane's first row (i0 + lane) is the base RowCtx, its
// second (i0 + 32 + lane, RW = 2) is r1.
template <int KT, int RW = 1>
struct TileCtx : RowCtx {
    int i0, k0;
    float rho_lo, rho_hi, rt, sB, cB;
    float sk[KT], ck[KT];
    RowCtx r1;

    __device__ __forceinline__ void init(const DevGeom &G, int lane, int tx, int ty)
    {
        k0 = tx * KT;
        i0 = ty * 32 * RW;
        init_row(G, i0 + lane);
        if (RW == 2) r1.init_row(G, i0 + 32 + lane);
        const int ilast = min(i0 + 32 * RW - 1, G.n_rho - 1);
        rho_lo = G.rho32[i0] - G.drho_f;
        rho_hi = G.rho32[ilast] + G.drho_f;
        rt = fmaxf(fabsf(G.rho32[i0]), fabsf(G.rho32[ilast])) * 1.0001f;
        // the second root q / rho can reach the axis only if |1 + rho s| <=
        // |rho| dext, i.e. |s| >= 1 / rt - dext for the rows of this tile
        // (|q| >= |b|); the float32 bound is lowered by 1e-6 relative and
        // 0.01 cm (its own rounding), and phase 1 lowers it further by the
        // error of the hit's float32 s
        sB = rt > 0.0f ? fmaf(__frcp_rn(rt) - G.dext_f, 1.0f - 1e-6f, -0.01f) : 3.0e38f;
        // |q| = |b| + sqrt(D) >= sqrt(1 - rho^2 c^2), so q / rho also needs
        // c^2 >= 1 / rho^2 - dext^2 >= 1 / rt^2 - dext^2 (same margins)
        const float ir = rt > 0.0f ? __frcp_rn(rt) : 3.0e19f;
        cB = fmaf(sqrtf(fmaxf(fmaf(ir, ir, -G.dext_f * G.dext_f), 0.0f)), 1.0f - 1e-6f, -0.05f);
#pragma unroll
        for (int kl = 0; kl < KT; ++kl) {
            sk[kl] = G.sn32[k0 + kl];
            ck[kl] = G.cs32[k0 + kl];
        }
    }
};

// The learned-proposal mask as one vote tile sees it (region helpers in
// ht_internal.cuh).  bm: d0 blocks of the lane's row whose halo the row is
// in; tile_bm: their union over the tile's rows.  Each run of consecutive
// blocks in tile_bm, widened by the one-bin halo, gives a d0 window; a
// (hit, column) pair whose circle reaches none of them within the rho span
// of the tile's allowed rows cannot vote in a halo cell of the tile.
struct MaskCtx {
    unsigned bm, tile_bm;
    int nrun;
    float wlo[4], whi[4];   // d0 windows (cm), 0.01 cm outside the bin edges
    float rho_lo, rho_hi;   // rho span of the allowed rows, one row of margin

    __device__ __forceinline__ void init(const DevGeom &G, unsigned long long mask, int i0,
                                         int irow, bool row_ok)
    {
        const int ND = G.n_d0;
        bm = row_ok ? halo_row_blocks(mask, irow, G.n_rho) : 0u;
        const unsigned rows = __ballot_sync(0xffffffffu, bm != 0u);
        tile_bm = __reduce_or_sync(0xffffffffu, bm);
        nrun = 0;
        rho_lo = rho_hi = 0.0f;
        if (!rows) return;
        rho_lo = G.rho32[i0 + __ffs(rows) - 1] - G.drho_f;
        rho_hi = G.rho32[i0 + 31 - __clz(rows)] + G.drho_f;
        unsigned rem = tile_bm;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            wlo[r] = whi[r] = 0.0f;
            if (rem) {
                const int b = __ffs(rem) - 1;
                const int e = b + __ffs(~(rem >> b)) - 2;   // last block of the run
                rem &= ~((2u << e) - 1u);
                const int lo = max(block_first(b, ND) - 1, 0);
                const int hi = min(block_first(e + 1, ND), ND - 1);
                wlo[r] = (float)(((double)lo - G.off) * G.delta) - 0.01f;
                whi[r] = (float)(((double)hi + 1.0 - G.off) * G.delta) + 0.01f;
                nrun = r + 1;
            }
        }
    }
};

// Per-hit region sets as one vote tile sees them.  Phase 1 (lane = hit)
// ORs the hit's d0-block bits over the rho blocks of the tile's rows and
// their one-row halo; a hit with none votes nowhere in the tile, the others
// get one d0 window (their blocks' span widened by the one-bin halo) for the
// curvature filter.  Phase 2 (lane = row) keeps a bin j of the lane's row
// when bm & jmask[j] != 0, bm being the hit's d0 blocks over the row's rho
// block and its neighbours' (shifts sh[]) and jmask[j] the blocks of bins
// j - 1, j, j + 1 (a shared table).
struct HitCtx {
    const unsigned long long *masks;   // the event's per-hit region sets
    const uint8_t *jmask;              // [n_d0], shared
    int rb_lo, rb_hi;                  // rho blocks of rows i0 - 1 .. i0 + 32 (clamped)
    int sh[3];                         // 8 x rho block of rows irow - 1, irow, irow + 1
    float w_lo0, w_step;               // d0 (cm) of bin 0's lower edge, bin width

    __device__ __forceinline__ unsigned row_bits(unsigned long long hm) const
    {
        return (unsigned)((hm >> sh[0]) | (hm >> sh[1]) | (hm >> sh[2])) & 0xffu;
    }
};

// ------------------------------------------------------------------ A-form items
// The vote's common case: a (hit, column) item whose second root is proven out
// of the axis, with b = 1 + rho s > 0 on every row of the tile (so the one
// root is C / q, the smaller in magnitude) and whose discriminant
// D = 1 - rho^2 c^2 stays at or above 1/64 for every |rho| <= rt.  With w = d0 + s the circle equation reads
// rho w^2 + 2 w + rho c^2 = 0; the root continuous with w = 0 at rho = 0 is the
// one with |w| < c, w = (sqrt(D) - 1) / rho = -rho c^2 / (1 + sqrt(D)), and it
// is the same real number as C / q.  Its bin coordinate is
//   u = A0 - rho c2d / (1 + sqrt(1 - rho^2 c^2)),  A0 = off - s / delta,  c2d = c^2 / delta,
// A0 and c2d per item: a row costs one rsqrt, one rcp and five FMA-pipe
// operations, and 1 + sqrt(D) >= 1 keeps every step well conditioned.
//
// Error of the float32 coordinate against the exact root of the float64
// definition's s, c, rho (first order; u = 2^-24; eS = 4e-7 R1 >= 3u R1
// bounds the float32 s and c; rsqrt.approx and rcp.approx within 4.3u, 2u):
//   A0 = fma(-s, 1/delta, off):     (eS + u|s|) / delta + u|A0|
//   c^2 relative 2 eS/c + u; c2d 2 eS/c + 3u; rho c2d 2 eS/c + 5u
//   D = fma(-rho^2, c^2, 1):        |dD| <= t (2 eS/c + 5u) + u,  t = rt^2 c^2
//   1 + D rsqrt(D) >= 1, relative:  5.3u + |dD| / sqrt(Dmin); its rcp 2u more
//   final fma: u (|A0| + |rho| c2d)
// The second term is at most |rho| c2d, so the bound is affine in |rho|:
//   e = eA + |rho| eB,  eA = kSafe ((eS + u|s|)/delta + 2u|A0|) + e64,
//                       eB = kSafe c2d (2 eS/c + 14.3u + |dD| / sqrt(Dmin)).
// e64 covers the float64 definition's own rounding against the exact root:
// its C = rho r^2 + 2s (and r^2 against s^2 + c^2) is off by a few 2^-53 of
// rho R1^2 + 2 R1, divided by |q| >= sqrt(D) >= 1/8, plus a few 2^-53 of |u|.
// Only items with c >= 4e-4 R1 take this form (the relative error of c is
// then at most 2e-3, where first order holds under kSafe; c > 0 is proven,
// the item is not unsure), only hits with R1 >= 1e-20 cm (nearer the origin
// c and c^2 underflow and the bound's float32 terms would be 0 x inf), and
// only while |u| < 2^21 everywhere on the tile, for the floor below.
constexpr float kMagic = 12582912.0f;       // 1.5 2^23: rd(x + kMagic) - kMagic = floor(x), |x| < 2^22
constexpr int kMagicBits = 0x4B400000;      // its bits

// Whether a plain item (not unsure, root B proven out) takes the A-form.  A
// plain item can have b = 1 + rho s <= 0 when its c alone keeps root B out of
// the axis; its one root is then branch B, so the A-form also needs
// rt (|s| + eS) < 1, with a margin for the float32 rt and s.
__device__ __forceinline__ bool aform_ok(const DevGeom &G, float s, float c, float R1, float rt)
{
    if (!(c >= 4e-4f * R1) || !(R1 >= 1e-20f)) return false;
    const float t = rt * rt * (c * c) * 1.001f;
    return (rt * fmaf(4e-7f, R1, fabsf(s)) < 0.99f) && (1.0f - t >= 0.015625f) &&
           fmaf(R1 + rt * c * c, G.inv_delta_f, G.off_f + 1.0f) < 2.0e6f;
}

// The A-form record {A0, c^2, c2d, eA} and eB of an item that passed aform_ok.
__device__ __forceinline__ float4 make_aform(const DevGeom &G, float s, float c, float R1,
                                             float rt, float &eB)
{
    const float eS = 4e-7f * R1;
    const float c2 = c * c;
    const float t = rt * rt * c2 * 1.001f;
    const float A0 = fmaf(-s, G.inv_delta_f, G.off_f);
    const float c2d = c2 * G.inv_delta_f;
    const float rc = 2.0f * eS * rcp_approx(c) * 1.001f;
    const float dD = fmaf(t, rc + 5.0f * kEps, kEps);
    const float isD = rsqrt_approx(1.0f - t) * 1.001f;
    const float aA = fabsf(A0);
    const float e64 = 1.6e-14f * fmaf(rt * R1, R1, 2.0f * R1) * G.inv_delta_f +
                      4e-15f * (aA + rt * c2d + G.off_f);
    const float eA = (kSafe * 1.001f) * (fmaf(kEps, fabsf(s), eS) * G.inv_delta_f +
                                         2.0f * kEps * aA) + e64;
    eB = (kSafe * 1.001f) * c2d * (rc + 14.3f * kEps + dD * isD);
    return make_float4(A0, c2, c2d, eA);
}

// Bin of an A-form item for the lane's row: vote (bin in j), redo (an
// integer lies within the bound), or neither (certainly outside the axis).
// The floors of u - e and u + e, rounded outwards, come from one round-down
// addition of kMagic each (exact integers plus kMagic): equal floors inside
// the axis prove the bin.
__device__ __forceinline__ void aform_bin(const RowCtx &T, const float4 a, float eB, float mnd,
                                          int &j, bool &vote, bool &redo)
{
    const float D = fmaf(-T.rho2, a.y, 1.0f);
    const float rs = rsqrt_approx(D);
    const float den = fmaf(D, rs, 1.0f);
    const float ir = rcp_approx(den);
    const float u = fmaf(-(T.rho * a.z), ir, a.x);
    const float e = fmaf(T.arho, eB, a.w);
    const float lo = __fadd_rd(__fsub_rd(u, e), kMagic);
    const float hi = __fadd_rd(__fadd_ru(u, e), kMagic);
    j = __float_as_int(lo) - kMagicBits;
    vote = (lo == hi) & (lo >= kMagic) & (lo < mnd);
    redo = (lo != hi) & (hi >= kMagic) & (lo < mnd);
}

// Word offset (from the lane's first word) and increment of column kl's
// counters in a tile of 32 RW rows with the layout of TileCol.
template <int KT, bool PACK, int RW = 1>
__device__ __forceinline__ void col_word(int ND, int kl, uint32_t one, uint32_t &woff,
                                         uint32_t &inc)
{
    if (PACK && KT > 1) {
        woff = (uint32_t)((kl >> 1) * ND * 32 * RW);
        inc = one << ((kl & 1) << 4);
    } else if (PACK) {
        woff = 0u;
        inc = one;
    } else {
        woff = (uint32_t)(kl * ND * 32 * RW);
        inc = one;
    }
}

// Phase 1 for the hit at position h of the tile's hit sequence (h >= n: no
// items), hit index ha, at (xh, yh).  Items record the position.  Appends
// this warp's items to the list (all 32 lanes must call): plain items
// (neither unsure nor needing root B) from the front, counted in q[0], the
// others from the back of the kThreads * KT slots, counted in q[1].
// AFORM (the vote tile): the front list takes only A-form items, with the
// A-form record and their counter word (PACK: the tile's counter layout);
// other plain items join the back list with the general record.
template <int KT, int MODE = kModePlain, bool AFORM = false, bool PACK = false, int RW = 1>
__device__ __forceinline__ void collect(const DevGeom &G, const TileCtx<KT, RW> &T, float xh,
                                        float yh, int n, int h, int ha, int lane, int *q,
                                        const WorkList &W, const MaskCtx *M = nullptr,
                                        const HitCtx *H = nullptr,
                                        const uint8_t *__restrict__ layer = nullptr)
{
    constexpr int BM = base_mode(MODE);
    float is_[KT], ic_[KT];
    int fl_[KT];
    unsigned sel = 0u, af = 0u;
    float r2 = 0.0f, R1 = 0.0f;
    unsigned long long hm = 0ull;
    float hwlo = 0.0f, hwhi = 0.0f;
    bool live = h < n;
    const unsigned char lh = (layer_mode(MODE) && live) ? __ldg(layer + ha) : 0;
    if (BM == kModeHit && live) {
        hm = H->masks[ha];
        unsigned tb = 0u;
        for (int b = H->rb_lo; b <= H->rb_hi; ++b) tb |= (unsigned)(hm >> (8 * b)) & 0xffu;
        live = tb != 0u;
        if (live) {
            const int ND = G.n_d0;
            const int lo = max(block_first(__ffs(tb) - 1, ND) - 1, 0);
            const int hi = min(block_first(32 - __clz(tb), ND), ND - 1);
            hwlo = fmaf((float)lo, H->w_step, H->w_lo0) - 0.01f;
            hwhi = fmaf((float)(hi + 1), H->w_step, H->w_lo0) + 0.01f;
        }
    }
    if (live) {
        r2 = fmaf(xh, xh, yh * yh);
        R1 = fabsf(xh) + fabsf(yh);
        const float cmin = hit_cos_window(G, r2);
        const float Ec = (kSafe * 3.0f * kEps) * R1;
        // float32 s and c are within 3 2^-24 R1 of the float64 ones (the
        // tables' and the products' rounding): 4e-7 R1 bounds it
        const float eS = 4e-7f * R1;
#pragma unroll
        for (int kl = 0; kl < KT; ++kl) {
            const float c = fmaf(xh, T.ck[kl], yh * T.sk[kl]);
            if (c < cmin || c < -Ec) continue;
            const float s = fmaf(xh, T.sk[kl], -(yh * T.ck[kl]));
            int f = 0;
            if (c <= Ec) {
                f |= kMetaUnsure;
            } else if (c > 1.0f) {
                float gmin, gmax;
                if (BM == kModeHit) {
                    rho_range_w(hwlo + s, hwhi + s, c, eS, gmin, gmax);
                    if (gmax < T.rho_lo || gmin > T.rho_hi) continue;
                } else if (BM == kModeEvent) {
                    bool reach = false;
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        if (r < M->nrun) {
                            rho_range_w(M->wlo[r] + s, M->whi[r] + s, c, eS, gmin, gmax);
                            reach |= !(gmax < M->rho_lo || gmin > M->rho_hi);
                        }
                    }
                    if (!reach) continue;
                } else {
                    rho_range(G, s, c, eS, gmin, gmax);
                    if (gmax < T.rho_lo || gmin > T.rho_hi) continue;
                }
            }
            if (fabsf(s) + eS >= T.sB && c + eS >= T.cB) f |= kMetaNeedB;
            if (AFORM && f == 0 && aform_ok(G, s, c, R1, T.rt)) af |= 1u << kl;
            sel |= 1u << kl;
            fl_[kl] = f;
            is_[kl] = s;
            ic_[kl] = c;
        }
    }
    unsigned slow = 0u;
#pragma unroll
    for (int kl = 0; kl < KT; ++kl)
        if ((sel & (1u << kl)) && (AFORM ? !(af & (1u << kl))
                                         : (fl_[kl] & (kMetaUnsure | kMetaNeedB)) != 0))
            slow |= 1u << kl;
    // one scan of both counts (plain in the low half, others in the high)
    const int mine = __popc(sel & ~slow) | (__popc(slow) << 16);
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    int wf = 0, ws = 0;
    if (lane == 31) {
        if (incl & 0xffff) wf = atomicAdd(&q[0], incl & 0xffff);
        if (incl >> 16) ws = atomicAdd(&q[1], incl >> 16);
    }
    wf = __shfl_sync(0xffffffffu, wf, 31);
    ws = __shfl_sync(0xffffffffu, ws, 31);
    const int excl = incl - mine;
    int pf = wf + (excl & 0xffff);
    int ps = ws + (excl >> 16);
#pragma unroll
    for (int kl = 0; kl < KT; ++kl) {
        if (sel & (1u << kl)) {
            const int pos = (slow & (1u << kl)) ? kThreads * KT - 1 - ps++ : pf++;
            if (AFORM && (af & (1u << kl))) {
                float eB;
                W.a[pos] = make_aform(G, is_[kl], ic_[kl], R1, T.rt, eB);
                uint32_t woff, inc;
                col_word<KT, PACK, RW>(G.n_d0, kl, layer_mode(MODE) ? 1u << lh : 1u, woff, inc);
                W.b[pos] = make_float4(__uint_as_float(woff), __uint_as_float(inc), eB, 0.0f);
            } else {
                const Item it = make_item(G, is_[kl], ic_[kl], r2, R1, T.rt);
                W.a[pos] = make_float4(it.s, it.c, it.r2, it.eD);
                W.b[pos] = make_float4(it.E1, it.E2, it.Qa, it.Qb);
            }
            W.meta[pos] = (h << 6) | fl_[kl] | kl;
            if (BM == kModeHit) W.hm[pos] = hm;
            if (layer_mode(MODE)) W.lay[pos] = lh;
        }
    }
}

// Slot of the t-th item of a list with nf plain items at the front and the
// others at the back of the kThreads * KT slots.
template <int KT>
__device__ __forceinline__ int item_slot(int t, int nf)
{
    return t < nf ? t : kThreads * KT - 1 - (t - nf);
}

// The hits a tile scans: positions 0 .. n - 1 of a list (hit index hl[p])
// or of the event itself (hl null: hit index p).
struct HitSeq {
    const int *hl;
    int n;

    __device__ __forceinline__ int hit(int p) const { return hl ? __ldg(hl + p) : p; }
};

// Hit index and coordinates of thread `threadIdx.x` in the round starting
// at base: the next round's are loaded while this round runs.
struct HitPrefetch {
    int hn;
    float xn, yn;

    __device__ __forceinline__ void load(const float *__restrict__ x,
                                         const float *__restrict__ y, const HitSeq &S, int p)
    {
        hn = p < S.n ? S.hit(p) : 0;
        xn = p < S.n ? __ldg(x + hn) : 0.0f;
        yn = p < S.n ? __ldg(y + hn) : 0.0f;
    }

    __device__ __forceinline__ void start(const float *__restrict__ x,
                                          const float *__restrict__ y, const HitSeq &S)
    {
        load(x, y, S, threadIdx.x);
    }

    // hit and (xh, yh) of round `base`; issues the loads of round base + blockDim.x
    __device__ __forceinline__ void next(const float *__restrict__ x,
                                         const float *__restrict__ y, const HitSeq &S, int base,
                                         int &ha, float &xh, float &yh)
    {
        ha = hn;
        xh = xn;
        yh = yn;
        load(x, y, S, base + (int)blockDim.x + (int)threadIdx.x);
    }
};

// Bins of work item t for the lane's row by guarded float32: the number of
// bins written to jj, or -1 when the column must be redone in float64.
template <int KT>
__device__ __forceinline__ int item_bins32(const DevGeom &G, const RowCtx &T,
                                           const WorkList &W, int t, int m, int jj[2])
{
    if (m & kMetaUnsure) return -1;
    const float4 a = W.a[t], b = W.b[t];
    const Item it{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    int jA, jB;
    // the flag is per item, so the branch is uniform over the warp; the
    // common path is compiled without root B
    if (T.has_b && (m & kMetaNeedB)) {
        if (eval32<true>(G, T.rho, T.invrho_es, T.invrho, it, jA, jB) != kDecided) return -1;
        int nv = 0;
        if (jA >= 0) jj[nv++] = jA;
        if (jB >= 0) jj[nv++] = jB;
        return nv;
    }
    if (eval32<false>(G, T.rho, T.invrho_es, T.invrho, it, jA, jB) != kDecided) return -1;
    jj[0] = jA;
    return jA >= 0 ? 1 : 0;
}

// Plain items (not unsure, root B proven out of the axis): eval32<false>'s
// arithmetic and decisions, returning kFastVote with the bin in j, kFastNone
// or kFastRedo, without the general path's bookkeeping.
enum : int { kFastNone = 0, kFastVote = 1, kFastRedo = 2 };

template <int KT>
__device__ __forceinline__ int fast_bin32(const DevGeom &G, const TileCtx<KT> &T,
                                          const WorkList &W, int t, int &j)
{
    const float4 a = W.a[t], b4 = W.b[t];   // {s, c, r2, eD}, {E1, E2, Qa, Qb}
    const float b = fmaf(T.rho, a.x, 1.0f);
    const float pc = T.rho * a.y;
    const float D = fmaf(-pc, pc, 1.0f);
    const float Dp = fmaxf(D, 1e-30f);
    const float rs = rsqrt_approx(Dp);
    const float sq = Dp * rs;
    const float q = -(b + copysignf(sq, b));
    const float C = fmaf(T.rho, a.z, a.x + a.x);
    const float iq = rcp_approx(q);
    const float u = fmaf(C * iq, G.inv_delta_f, G.off_f);
    const float e = fmaf(fabsf(iq), fmaf(b4.y, rs, b4.x), G.e3);
    const float f = floorf(u);
    const float fr = u - f;
    j = (int)f;
    // decided as predicates (no early returns): no real root -> none; sign
    // of D unproven -> redo; outside the axis -> none; else vote if the
    // coordinate is farther than e from every integer, redo if not (the
    // distances as in decide(): a root within e below the axis has
    // (f + 1) - u = -u <= e and is redone, never voted in bin -1)
    const bool none = D < -a.w, tang = D <= a.w;
    const bool out = (u + e < 0.0f) | (u - e >= (float)G.n_d0);
    const bool ok = fminf(fr, (f + 1.0f) - u) > e;
    const bool vote = !tang & !out & ok;
    const bool redo = !none & (tang | (!out & !ok));
    return vote ? kFastVote : (redo ? kFastRedo : kFastNone);
}

// Deferred redo requests: (hit, row-in-tile, column) pairs whose bins
// float32 could not prove.  Drained by all threads of the CTA at the end of
// the tile (or when half full), through the double-float tier and, rarely,
// float64 (slow on this part), so neither runs as a lone divergent lane.
constexpr int kRedoCap = 512;
constexpr size_t kRedoBytes = (size_t)kRedoCap * 8;

struct RedoQueue {
    int *hit, *rc;   // rc = row << 4 | column
};

__device__ __forceinline__ RedoQueue carve_redo(unsigned char *p)
{
    RedoQueue q;
    q.hit = reinterpret_cast<int *>(p);
    q.rc = q.hit + kRedoCap;
    return q;
}

// Push a redo request; false if the queue is full (caller redoes it now).
__device__ __forceinline__ bool push_redo(const RedoQueue &Q, int *n, int hit, int row, int col)
{
    const int slot = atomicAdd(n, 1);
    if (slot >= kRedoCap) return false;
    Q.hit[slot] = hit;
    Q.rc[slot] = (row << 4) | col;
    return true;
}

// ------------------------------------------------------------------ vote
// PACK: two 16-bit counters per shared word, which halves the tile.  With
// KT >= 2 a word holds columns 2p and 2p + 1 of one (bin, row), so the
// increment (1 or 65536) is fixed per work item and a vote costs one address
// computation; with KT = 1 it holds bins 2w and 2w + 1.  Exact while no cell
// can reach 65536 votes in the tile: a cell gets at most two votes per
// scanned hit, so it is used only for tiles scanning at most kPackMaxHits.
// LAY (the distinct-layer vote): the same words hold layer masks; a vote
// ORs the hit's layer bit lbit (1 << layer) instead of adding one.
// RW: the tile has 32 RW rows (row fastest, 32 RW words per bin); lane is
// the row within the tile.
template <int KT, bool PACK, bool LAY = false, int RW = 1>
struct TileCol {
    uint32_t *base;
    uint32_t inc;

    __device__ __forceinline__ TileCol(uint32_t *cnt, int ND, int kl, int lane,
                                       uint32_t lbit = 1u)
    {
        const uint32_t one = LAY ? lbit : 1u;
        if (PACK && KT > 1) {
            base = cnt + (kl >> 1) * ND * 32 * RW + lane;
            inc = one << ((kl & 1) << 4);
        } else if (PACK) {
            base = cnt + lane;
            inc = one;
        } else {
            base = cnt + kl * ND * 32 * RW + lane;
            inc = one;
        }
    }

    __device__ __forceinline__ void add(int j) const
    {
        uint32_t *w = (PACK && KT == 1) ? base + (j >> 1) * 32 * RW : base + j * 32 * RW;
        const uint32_t v = (PACK && KT == 1) ? inc << ((j & 1) << 4) : inc;
        if (LAY) atomicOr(w, v);
        else atomicAdd(w, v);
    }
};

// An A-form item's vote: its counter word woff (from the lane's first word
// cntl) and increment inc, as col_word gave them, in bin j.
template <int KT, bool PACK, bool LAY, int RW = 1>
__device__ __forceinline__ void add_word(uint32_t *cntl, uint32_t woff, uint32_t inc, int j)
{
    uint32_t *w = (PACK && KT == 1) ? cntl + woff + (j >> 1) * 32 * RW
                                    : cntl + woff + j * 32 * RW;
    const uint32_t v = (PACK && KT == 1) ? inc << ((j & 1) << 4) : inc;
    if (LAY) atomicOr(w, v);
    else atomicAdd(w, v);
}

template <int KT, bool PACK, int RW = 1>
__device__ __forceinline__ uint32_t tile_get(const uint32_t *cnt, int ND, int kl, int j, int il)
{
    constexpr int R = 32 * RW;
    if (PACK && KT > 1) return (cnt[((kl >> 1) * ND + j) * R + il] >> ((kl & 1) << 4)) & 0xffffu;
    if (PACK) return (cnt[(j >> 1) * R + il] >> ((j & 1) << 4)) & 0xffffu;
    return cnt[(kl * ND + j) * R + il];
}

// Keep the bins jj[0 .. nv) that the hit's region set allows in the lane's
// row (kModeHit); returns the new count.
__device__ __forceinline__ int keep_allowed(unsigned bm, const uint8_t *jmask, int nv, int jj[2])
{
    int k = 0;
    if (nv > 0 && (bm & jmask[jj[0]])) jj[k++] = jj[0];
    if (nv > 1 && (bm & jmask[jj[1]])) jj[k++] = jj[1];
    return k;
}

// kModeEvent: only halo cells of `mask` are exact (others get 0 or a partial
// count); a tile without halo cells returns at once and writes nothing.
// kModeHit: hit h's votes count only in the halo cells of hmask[h]; every
// cell is written.
// hl (optional): the tile scans only the nl hits hl[0 .. nl) of the event
// (a superset of those that can vote in its columns); otherwise all n.
// RW = 2 (the plain and distinct-layer votes only): tiles of 64 rows, each
// lane evaluating rows lane and 32 + lane of every item, so that an item's
// loads, its phase-1 work and the warp's bookkeeping serve twice the votes.
template <int KT, typename OutT, bool PACK, int MODE = kModePlain, int RW = 1>
__device__ __forceinline__ void vote_tile(const DevGeom &G, const float *__restrict__ x,
                                          const float *__restrict__ y, int n,
                                          OutT *__restrict__ acc,
                                          unsigned long long *__restrict__ stats, int tx, int ty,
                                          unsigned long long mask = ~0ull,
                                          const unsigned long long *__restrict__ hmask = nullptr,
                                          const int *__restrict__ hl = nullptr, int nl = 0,
                                          const uint8_t *__restrict__ layer = nullptr)
{
    constexpr int BM = base_mode(MODE);
    constexpr bool LAY = layer_mode(MODE);
    static_assert(RW == 1 || (RW == 2 && BM == kModePlain), "64-row tiles: plain modes only");
    constexpr int TR = 32 * RW;                            // rows per tile
    extern __shared__ __align__(16) unsigned char smem[];
    const int ND = G.n_d0;
    const int NW = PACK ? (ND >> 1) : ND;                  // words per column-row
    constexpr int QCAP = kThreads * KT;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);    // [KT][NW][TR]
    unsigned char *p = reinterpret_cast<unsigned char *>(cnt + KT * NW * TR);
    const WorkList W = carve_worklist(p, QCAP, MODE);
    const RedoQueue R = carve_redo(p + (size_t)QCAP * item_bytes(MODE));
    __shared__ int qn[2][2], rn;   // [parity][plain, others]
    __shared__ unsigned long long s_stats[2];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nwarps = kThreads / 32;
    TileCtx<KT, RW> T;
    T.init(G, lane, tx, ty);
    MaskCtx M;
    if (BM == kModeEvent) {
        M.init(G, mask, T.i0, T.irow, T.row_ok);
        if (M.tile_bm == 0u) return;   // uniform: every warp sees the same rows
    }
    HitCtx H;
    if (BM == kModeHit) {
        const int NR = G.n_rho;
        uint8_t *jm = p + (size_t)QCAP * item_bytes(MODE) + kRedoBytes;
        for (int j = threadIdx.x; j < ND; j += kThreads)
            jm[j] = (uint8_t)((1u << region_block(max(j - 1, 0), ND)) |
                              (1u << region_block(j, ND)) |
                              (1u << region_block(min(j + 1, ND - 1), ND)));
        H.masks = hmask;
        H.jmask = jm;
        H.rb_lo = region_block(max(T.i0 - 1, 0), NR);
        H.rb_hi = region_block(min(T.i0 + 32, NR - 1), NR);
        const int ir = min(T.irow, NR - 1);
        H.sh[0] = 8 * region_block(max(ir - 1, 0), NR);
        H.sh[1] = 8 * region_block(ir, NR);
        H.sh[2] = 8 * region_block(min(ir + 1, NR - 1), NR);
        H.w_step = G.delta_f;
        H.w_lo0 = -G.off_f * G.delta_f;
    }
    {
        uint4 *c4 = reinterpret_cast<uint4 *>(cnt);
        for (int t = threadIdx.x; t < KT * NW * 8 * RW; t += kThreads) c4[t] = make_uint4(0, 0, 0, 0);
    }
    if (threadIdx.x < 4) qn[threadIdx.x >> 1][threadIdx.x & 1] = 0;
    if (threadIdx.x < 2) s_stats[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) rn = 0;
    __syncthreads();

    int my_fb = 0;
    unsigned my_cast = 0;   // LAY: votes cast by this thread in the tile (< 2^32: 2 KT per hit)
    int parity = 0;
    const HitSeq S{hl, hl ? nl : n};
    HitPrefetch pf;
    pf.start(x, y, S);
    for (int base = 0; base < S.n; base += kThreads, parity ^= 1) {
        int ha;
        float xh, yh;
        pf.next(x, y, S, base, ha, xh, yh);
        collect<KT, MODE, true, PACK, RW>(G, T, xh, yh, S.n, base + threadIdx.x, ha, lane,
                                          qn[parity], W, &M, &H, layer);
        __syncthreads();
        const int nf = qn[parity][0], ns = qn[parity][1];
        if (threadIdx.x == 0) {   // last read before the previous barrier
            qn[parity ^ 1][0] = 0;
            qn[parity ^ 1][1] = 0;
        }
        if (T.row_ok) {
            // A-form items: one root, no flags to test, the counter word and
            // increment precomputed.  A warp takes two items per iteration:
            // both are loaded before either votes (a shared atomic orders
            // the loads behind it), their evaluations are independent, and
            // one warp vote covers both redo tests (rare).  With RW = 2 each
            // lane also evaluates its second row (32 + lane) of both items.
            uint32_t *const cntl = cnt + lane;
            const float mnd = kMagic + (float)ND;
            const RowCtx &T1 = T.r1;
            const bool ok1 = RW == 2 && T1.row_ok;
            auto redo_item = [&](int tt, const RowCtx &Rw, int il) {
                ++my_fb;
                const int m = W.meta[tt];
                const int hh = S.hit(m >> 6);
                if (push_redo(R, &rn, hh, il, m & kMetaCol)) return;
                const TileCol<KT, PACK, LAY, RW> col(cnt, ND, m & kMetaCol, il,
                                                     LAY ? 1u << W.lay[tt] : 1u);
                int jj[2];
                int nv = redo_bins(G, x[hh], y[hh], Rw.irow, T.k0 + (m & kMetaCol), jj);
                if (BM == kModeHit) nv = keep_allowed(H.row_bits(W.hm[tt]), H.jmask, nv, jj);
                for (int v = 0; v < nv; ++v) col.add(jj[v]);
                if (LAY) my_cast += nv;
            };
            auto vote_item = [&](int tt, const float4 &b, int j, bool vote, int r) {
                if (vote && (BM != kModeHit || (H.row_bits(W.hm[tt]) & H.jmask[j]))) {
                    add_word<KT, PACK, LAY, RW>(cntl + 32 * r, __float_as_uint(b.x),
                                                __float_as_uint(b.y), j);
                    if (LAY) ++my_cast;
                }
            };
            int t = warp;
            for (; t + nwarps < nf; t += 2 * nwarps) {
                const float4 a0 = W.a[t], b0 = W.b[t];
                const float4 a1 = W.a[t + nwarps], b1 = W.b[t + nwarps];
                int j0, j1, j2 = 0, j3 = 0;
                bool v0, v1, r0, r1, v2 = false, v3 = false, r2 = false, r3 = false;
                aform_bin(T, a0, b0.z, mnd, j0, v0, r0);
                aform_bin(T, a1, b1.z, mnd, j1, v1, r1);
                if (RW == 2) {
                    aform_bin(T1, a0, b0.z, mnd, j2, v2, r2);
                    aform_bin(T1, a1, b1.z, mnd, j3, v3, r3);
                    v2 &= ok1;
                    v3 &= ok1;
                    r2 &= ok1;
                    r3 &= ok1;
                }
                vote_item(t, b0, j0, v0, 0);
                vote_item(t + nwarps, b1, j1, v1, 0);
                if (RW == 2) {
                    vote_item(t, b0, j2, v2, 1);
                    vote_item(t + nwarps, b1, j3, v3, 1);
                }
                // lanes of rows past n_rho do not run this loop, hence the active mask
                if (!__any_sync(__activemask(), r0 | r1 | r2 | r3)) continue;
                if (r0) redo_item(t, T, lane);
                if (r1) redo_item(t + nwarps, T, lane);
                if (RW == 2) {
                    if (r2) redo_item(t, T1, 32 + lane);
                    if (r3) redo_item(t + nwarps, T1, 32 + lane);
                }
            }
            if (t < nf) {
                const float4 a0 = W.a[t], b0 = W.b[t];
                int j0;
                bool v0, r0;
                aform_bin(T, a0, b0.z, mnd, j0, v0, r0);
                vote_item(t, b0, j0, v0, 0);
                if (r0) redo_item(t, T, lane);
                if (RW == 2 && ok1) {
                    aform_bin(T1, a0, b0.z, mnd, j0, v0, r0);
                    vote_item(t, b0, j0, v0, 1);
                    if (r0) redo_item(t, T1, 32 + lane);
                }
            }
            // unsure items, items whose second root can reach the axis and the
            // other plain items
            for (int t = kThreads * KT - ns + warp; t < kThreads * KT; t += nwarps) {
                const int m = W.meta[t];
#pragma unroll
                for (int r = 0; r < RW; ++r) {
                    const RowCtx &Rw = r == 0 ? static_cast<const RowCtx &>(T) : T1;
                    if (r == 1 && !ok1) break;
                    const int il = lane + 32 * r;
                    const TileCol<KT, PACK, LAY, RW> col(cnt, ND, m & kMetaCol, il,
                                                         LAY ? 1u << W.lay[t] : 1u);
                    int jj[2];
                    int nv = item_bins32<KT>(G, Rw, W, t, m, jj);
                    if (nv < 0) {
                        ++my_fb;
                        const int hh = S.hit(m >> 6);
                        if (push_redo(R, &rn, hh, il, m & kMetaCol)) continue;
                        nv = redo_bins(G, x[hh], y[hh], Rw.irow, T.k0 + (m & kMetaCol), jj);
                    }
                    if (BM == kModeHit) nv = keep_allowed(H.row_bits(W.hm[t]), H.jmask, nv, jj);
                    if (nv > 0) col.add(jj[0]);
                    if (nv > 1) col.add(jj[1]);
                    if (LAY) my_cast += nv;
                }
            }
        }
        __syncthreads();
        // drain the deferred redos when the queue is half full or at the end
        const int nr = min(rn, kRedoCap);
        if (nr >= kRedoCap / 2 || base + kThreads >= S.n) {
            for (int t = threadIdx.x; t < nr; t += kThreads) {
                const int h = R.hit[t], rc = R.rc[t];
                const int il = rc >> 4, kl = rc & 15;
                int jj[2];
                int nv = redo_bins(G, x[h], y[h], T.i0 + il, T.k0 + kl, jj);
                if (BM == kModeHit)
                    nv = keep_allowed(halo_row_blocks(H.masks[h], T.i0 + il, G.n_rho), H.jmask, nv,
                                      jj);
                const TileCol<KT, PACK, LAY, RW> col(cnt, ND, kl, il,
                                                     LAY ? 1u << __ldg(layer + h) : 1u);
                for (int v = 0; v < nv; ++v) col.add(jj[v]);
                if (LAY) my_cast += nv;
            }
            __syncthreads();
            if (threadIdx.x == 0) rn = 0;
        }
    }
    __syncthreads();

    // write-back: thread = (row, d0 bin); the KT counts of a row go out as
    // one vector of KT * sizeof(OutT) bytes.  Votes are summed here (tile
    // counters never saturate: they hold at most 2 n).
    unsigned long long my_votes = 0;
    for (int t = threadIdx.x; t < TR * ND; t += kThreads) {
        const int il = t & (TR - 1), j = t / TR;   // il == lane (RW = 1) or lane + 32 (RW = 2)
        const int i = T.i0 + il;
        if (i >= G.n_rho) continue;
        const bool keep = BM != kModeEvent || halo_bin(M.bm, j, ND);
        __align__(16) OutT e[KT];
#pragma unroll
        for (int kl = 0; kl < KT; ++kl) {
            uint32_t v = keep ? tile_get<KT, PACK, RW>(cnt, ND, kl, j, il) : 0u;
            if (LAY) v = (uint32_t)__popc(v);
            else my_votes += v;
            e[kl] = saturate<OutT>(v);
        }
        OutT *dst = acc + ((size_t)i * ND + j) * G.n_phi0 + T.k0;
        if constexpr (KT * sizeof(OutT) == 16) {
            *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(e);
        } else if constexpr (KT * sizeof(OutT) == 8) {
            *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(e);
        } else if constexpr (KT * sizeof(OutT) == 4) {
            *reinterpret_cast<uint32_t *>(dst) = *reinterpret_cast<const uint32_t *>(e);
        } else {
#pragma unroll
            for (int kl = 0; kl < KT; ++kl) dst[kl] = e[kl];
        }
    }

    if (LAY) my_votes = my_cast;
    if (stats) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            my_votes += __shfl_xor_sync(0xffffffffu, my_votes, o);
            my_fb += __shfl_xor_sync(0xffffffffu, my_fb, o);
        }
        if (lane == 0) {
            atomicAdd(&s_stats[0], my_votes);
            atomicAdd(&s_stats[1], (unsigned long long)my_fb);
        }
        __syncthreads();
        if (threadIdx.x < 2) atomicAdd(&stats[threadIdx.x], s_stats[threadIdx.x]);
    }
}

// mask: kModeEvent one device uint64, kModeHit one per hit, else unused;
// layer: one uint8 per hit under kModeLayers, else unused.
// The distinct-layer vote's tiles of at most two columns (64-row tiles, and
// the 32-row tiles of the pile-up geometry and of the per-hit mode) take four
// CTAs per SM: their counters and two-column work list fit four in shared
// memory, and 64 registers spill about as little as 80 do.
template <int KT, typename OutT, bool PACK, int MODE, int RW = 1>
__global__ void __launch_bounds__(kThreads, (RW == 2 || (layer_mode(MODE) && KT <= 2)) ? 4 : (PACK ? 3 : 2))
k_vote(DevGeom G, const float *__restrict__ x, const float *__restrict__ y, int n,
       OutT *__restrict__ acc, unsigned long long *__restrict__ stats,
       const unsigned long long *__restrict__ mask, const uint8_t *__restrict__ layer)
{
    vote_tile<KT, OutT, PACK, MODE, RW>(G, x, y, n, acc, stats, blockIdx.x, blockIdx.y,
                                    base_mode(MODE) == kModeEvent ? *mask : ~0ull, mask,
                                    nullptr, 0, layer);
}

// Persistent vote over a batch: CTAs pop (event, tile) items from a device
// counter; items run event by event in the order given (largest events
// first), so uneven events share the GPU without per-event launch tails.
// kModeEvent: event e votes under masks[e]; kModeHit: masks holds one region
// set per hit of the batch (indexed like x).
// bk (optional, ent null for none): per-event hit lists by column group; a
// tile scans its group's list instead of the whole event.
template <int KT, typename OutT, bool PACK, int MODE, int RW = 1>
__global__ void __launch_bounds__(kThreads, (RW == 2 || (layer_mode(MODE) && KT <= 2)) ? 4 : (PACK ? 3 : 2))
k_vote_batch(DevGeom G, const float *__restrict__ x, const float *__restrict__ y,
             const int *__restrict__ off, const int *__restrict__ order,
             const int *__restrict__ d_nev,
             OutT *__restrict__ acc, size_t acc_stride, unsigned long long *__restrict__ stats,
             int *__restrict__ head, const unsigned long long *__restrict__ masks,
             BucketView bk, const uint8_t *__restrict__ layer)
{
    constexpr int BM = base_mode(MODE);
    __shared__ int s_item;
    const int ntx = G.n_phi0 / KT, nty = (G.n_rho + 32 * RW - 1) / (32 * RW), ntiles = ntx * nty;
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
        // Packed 16-bit counters take the tiles that scan at most kPackMaxHits
        // hits (a cell then holds at most 2 kPackMaxHits < 2^16 votes, so no
        // count carries into its neighbour), unpacked counters the others:
        // the two launches of a batch split every event's tiles between them
        // by the scanned list's length (uniform over the CTA).  Layer masks
        // never carry, so the distinct-layer vote packs every tile.
        if (layer_mode(MODE) ? PACK : (PACK == ((bk.ent ? nl : n) <= kPackMaxHits)))
            vote_tile<KT, OutT, PACK, MODE, RW>(G, x + a, y + a, n, acc + (size_t)e * acc_stride,
                                            stats ? stats + 2 * e : nullptr, t % ntx, t / ntx,
                                            BM == kModeEvent ? masks[e] : ~0ull,
                                            BM == kModeHit ? masks + a : nullptr, hl, nl,
                                            layer_mode(MODE) ? layer + a : nullptr);
        __syncthreads();
    }
}

template <int KT>
size_t vote_smem(const DevGeom &G, bool pack, int mode = kModePlain, int rw = 1)
{
    return (size_t)KT * 32 * rw * (pack ? G.n_d0 / 2 : G.n_d0) * 4 +
           (size_t)kThreads * KT * item_bytes(mode) + kRedoBytes +
           (base_mode(mode) == kModeHit ? ((size_t)G.n_d0 + 15) / 16 * 16 : 0);
}

constexpr size_t kSmemBudget2 = 110 * 1024;   // two CTAs per SM
constexpr size_t kSmemBudget3 = 75 * 1024;    // three CTAs per SM

template <int KT, typename OutT, bool PACK, int MODE, int RW = 1>
cudaError_t launch_vote_kt(const DevGeom &G, const float *x, const float *y, int n, void *acc,
                           unsigned long long *stats, const unsigned long long *mask,
                           cudaStream_t st, const uint8_t *layer)
{
    dim3 grid(G.n_phi0 / KT, (G.n_rho + 32 * RW - 1) / (32 * RW));
    k_vote<KT, OutT, PACK, MODE, RW><<<grid, kThreads, vote_smem<KT>(G, PACK, MODE, RW), st>>>(
        G, x, y, n, reinterpret_cast<OutT *>(acc), stats, mask, layer);
    return cudaGetLastError();
}

// The distinct-layer vote's default tile: 64 rows of two columns when it
// fits in the three-CTA budget (plain base mode only).
template <int MODE>
constexpr bool tall_tiles_ok()
{
    return layer_mode(MODE) && base_mode(MODE) == kModePlain;
}

// Tile shape: packed 16-bit counters with three CTAs per SM when the output
// is uint16, n_d0 even and n <= 32767; otherwise 32-bit counters, two CTAs
// per SM.  KT is the widest tile that fits.  The distinct-layer vote
// (kModeLayers; n_d0 even) always packs, into either output type, on 64-row
// tiles of two columns (four CTAs per SM) where they fit the three-CTA
// budget, else on 32-row tiles.
template <int MODE>
cudaError_t launch_vote_t(const DevGeom &G, const float *x, const float *y, int n, void *acc,
                          unsigned long long *stats, const unsigned long long *mask,
                          cudaStream_t st, const uint8_t *layer = nullptr)
{
#define HT_V(KTV, OT, PK)                                                                     \
    return launch_vote_kt<KTV, OT, PK, MODE>(G, x, y, n, acc, stats, mask, st, layer)
    if constexpr (tall_tiles_ok<MODE>()) {
        if (vote_smem<2>(G, true, MODE, 2) <= kSmemBudget3) {
            if (G.count_bits == 16)
                return launch_vote_kt<2, uint16_t, true, MODE, 2>(G, x, y, n, acc, stats, mask,
                                                                  st, layer);
            return launch_vote_kt<2, int32_t, true, MODE, 2>(G, x, y, n, acc, stats, mask, st,
                                                             layer);
        }
    }
    if constexpr (layer_mode(MODE)) {
        if (G.count_bits == 16) {
            if (vote_smem<4>(G, true, MODE) <= kSmemBudget3) HT_V(4, uint16_t, true);
            if (vote_smem<2>(G, true, MODE) <= kSmemBudget3) HT_V(2, uint16_t, true);
            HT_V(1, uint16_t, true);
        }
        if (vote_smem<4>(G, true, MODE) <= kSmemBudget3) HT_V(4, int32_t, true);
        if (vote_smem<2>(G, true, MODE) <= kSmemBudget3) HT_V(2, int32_t, true);
        HT_V(1, int32_t, true);
    } else {
        if (G.count_bits == 16) {
            if (n <= 32767 && G.n_d0 % 2 == 0) {
                if (vote_smem<4>(G, true, MODE) <= kSmemBudget3) HT_V(4, uint16_t, true);
                if (vote_smem<2>(G, true, MODE) <= kSmemBudget3) HT_V(2, uint16_t, true);
                if (vote_smem<1>(G, true, MODE) <= kSmemBudget3) HT_V(1, uint16_t, true);
            }
            if (vote_smem<8>(G, false, MODE) <= kSmemBudget2) HT_V(8, uint16_t, false);
            if (vote_smem<4>(G, false, MODE) <= kSmemBudget2) HT_V(4, uint16_t, false);
            if (vote_smem<2>(G, false, MODE) <= kSmemBudget2) HT_V(2, uint16_t, false);
            HT_V(1, uint16_t, false);
        }
        if (vote_smem<4>(G, false, MODE) <= kSmemBudget2) HT_V(4, int32_t, false);
        if (vote_smem<2>(G, false, MODE) <= kSmemBudget2) HT_V(2, int32_t, false);
        HT_V(1, int32_t, false);
    }
#undef HT_V
}

// Persistent vote of a batch: `order` lists d_nev[0] event slots; every CTA
// slot of the GPU (SMs x resident CTAs) pops items until the queue is empty.
// kt selects the tile width (0 = default).  pack: this launch takes the
// listed events' tiles that scan at most kPackMaxHits hits (a column group's
// hit list with buckets, else the event) with 16-bit packed counters;
// otherwise it takes their other tiles with 32-bit counters.  The
// distinct-layer vote takes every tile in its packed launch (layer: the
// batch's layer array, indexed like x), by default on 64-row tiles of two
// columns (an explicit kt selects 32-row tiles of that width).  *head must
// be zero.
template <int MODE>
cudaError_t launch_vote_batch_t(const DevGeom &G, const float *x, const float *y, const int *off,
                                const int *order, const int *d_nev, uint16_t *acc,
                                size_t acc_stride, unsigned long long *stats, int *head,
                                bool pack, int kt, int sms, const unsigned long long *masks,
                                cudaStream_t st, BucketView bk = BucketView{},
                                const uint8_t *layer = nullptr)
{
#define HT_VB2(KTV, PK, RWV)                                                                  \
    do {                                                                                      \
        int occ = 0;                                                                          \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                        \
            &occ, k_vote_batch<KTV, uint16_t, PK, MODE, RWV>, kThreads,                       \
            vote_smem<KTV>(G, PK, MODE, RWV));                                                \
        k_vote_batch<KTV, uint16_t, PK, MODE, RWV><<<sms * (occ > 0 ? occ : 1), kThreads,    \
                                                     vote_smem<KTV>(G, PK, MODE, RWV), st>>>( \
            G, x, y, off, order, d_nev, acc, acc_stride, stats, head, masks, bk, layer);      \
        return cudaGetLastError();                                                            \
    } while (0)
#define HT_VB(KTV, PK) HT_VB2(KTV, PK, 1)
    // the per-hit mode's larger items would drop a tuned width to two CTAs
    // per SM: it keeps three
    const size_t budget = base_mode(MODE) == kModeHit ? kSmemBudget3 : kSmemBudget2;
    if constexpr (tall_tiles_ok<MODE>()) {
        // kt = 0 (the default): 64-row tiles of two columns where they fit
        if (pack && kt == 0 && vote_smem<2>(G, true, MODE, 2) <= kSmemBudget3) HT_VB2(2, true, 2);
    }
    if constexpr (layer_mode(MODE)) {
        if (!pack) return cudaSuccess;   // no unpacked tiles
        if (kt == 0) kt = vote_smem<4>(G, true, MODE) <= kSmemBudget3 ? 4
                        : vote_smem<2>(G, true, MODE) <= kSmemBudget3 ? 2 : 1;
        if (kt == 4 && vote_smem<4>(G, true, MODE) <= budget) HT_VB(4, true);
        if (kt >= 2 && vote_smem<2>(G, true, MODE) <= budget) HT_VB(2, true);
        HT_VB(1, true);
    } else {
        if (pack) {
            if (kt == 0) kt = vote_smem<4>(G, true, MODE) <= kSmemBudget3 ? 4
                            : vote_smem<2>(G, true, MODE) <= kSmemBudget3 ? 2 : 1;
            if (kt == 4 && vote_smem<4>(G, true, MODE) <= budget) HT_VB(4, true);
            if (kt >= 2 && vote_smem<2>(G, true, MODE) <= budget) HT_VB(2, true);
            HT_VB(1, true);
        }
        if (kt == 0) kt = vote_smem<8>(G, false, MODE) <= kSmemBudget2 ? 8
                        : vote_smem<4>(G, false, MODE) <= kSmemBudget2 ? 4
                        : vote_smem<2>(G, false, MODE) <= kSmemBudget2 ? 2 : 1;
        if (kt == 8 && vote_smem<8>(G, false, MODE) <= kSmemBudget2) HT_VB(8, false);
        if (kt >= 4 && vote_smem<4>(G, false, MODE) <= kSmemBudget2) HT_VB(4, false);
        if (kt >= 2 && vote_smem<2>(G, false, MODE) <= kSmemBudget2) HT_VB(2, false);
        HT_VB(1, false);
    }
#undef HT_VB
#undef HT_VB2
}

inline cudaError_t allow_smem(const void *const *fns, int nf, int max_smem)
{
    for (int i = 0; i < nf; ++i) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, fns[i]);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 max_smem - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Allow every vote kernel the device's opt-in shared memory (each launch
// still passes only what its tile needs).
template <int MODE>
cudaError_t prepare_vote_kernels_t(int max_smem)
{
    if constexpr (tall_tiles_ok<MODE>()) {
        const void *fns[] = {
            (const void *)k_vote<2, uint16_t, true, MODE, 2>,
            (const void *)k_vote<2, int32_t, true, MODE, 2>,
            (const void *)k_vote_batch<2, uint16_t, true, MODE, 2>};
        const cudaError_t e = allow_smem(fns, (int)(sizeof fns / sizeof fns[0]), max_smem);
        if (e != cudaSuccess) return e;
    }
    if constexpr (layer_mode(MODE)) {
        const void *fns[] = {
            (const void *)k_vote<4, uint16_t, true, MODE>,
            (const void *)k_vote<2, uint16_t, true, MODE>,
            (const void *)k_vote<1, uint16_t, true, MODE>,
            (const void *)k_vote<4, int32_t, true, MODE>,
            (const void *)k_vote<2, int32_t, true, MODE>,
            (const void *)k_vote<1, int32_t, true, MODE>,
            (const void *)k_vote_batch<4, uint16_t, true, MODE>,
            (const void *)k_vote_batch<2, uint16_t, true, MODE>,
            (const void *)k_vote_batch<1, uint16_t, true, MODE>};
        return allow_smem(fns, (int)(sizeof fns / sizeof fns[0]), max_smem);
    } else {
        const void *fns[] = {
            (const void *)k_vote<4, uint16_t, true, MODE>,
            (const void *)k_vote<2, uint16_t, true, MODE>,
            (const void *)k_vote<1, uint16_t, true, MODE>,
            (const void *)k_vote<8, uint16_t, false, MODE>,
            (const void *)k_vote<4, uint16_t, false, MODE>,
            (const void *)k_vote<2, uint16_t, false, MODE>,
            (const void *)k_vote<1, uint16_t, false, MODE>,
            (const void *)k_vote<4, int32_t, false, MODE>,
            (const void *)k_vote<2, int32_t, false, MODE>,
            (const void *)k_vote<1, int32_t, false, MODE>,
            (const void *)k_vote_batch<4, uint16_t, true, MODE>,
            (const void *)k_vote_batch<2, uint16_t, true, MODE>,
            (const void *)k_vote_batch<1, uint16_t, true, MODE>,
            (const void *)k_vote_batch<8, uint16_t, false, MODE>,
            (const void *)k_vote_batch<4, uint16_t, false, MODE>,
            (const void *)k_vote_batch<2, uint16_t, false, MODE>,
            (const void *)k_vote_batch<1, uint16_t, false, MODE>};
        return allow_smem(fns, (int)(sizeof fns / sizeof fns[0]), max_smem);
    }
}

}  // namespace
}  // namespace ht
