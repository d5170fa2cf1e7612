// ht_internal.cuh -- device-side geometry, exact and guarded cell evaluators.
//
// Shared by the kernels of libht.  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ht.h"

namespace ht {

// Streaming multiprocessors of the current device (grid sizing); 152 if the
// query fails.
inline int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
        return 152;
    return sms;
}

// ---------------------------------------------------------------------------
// Geometry as the kernels see it (passed by value).  Every float64 value is
// computed on the host with the same expression as the plain definition; the
// float32 copies are roundings of those values.
struct DevGeom {
    int n_rho, n_d0, n_phi0, n_z0, n_cot, threshold, count_bits;
    // d0 axis
    double delta, off;             // bin width, u = d0 / delta + off
    float delta_f, inv_delta_f, off_f;
    float d0lo_f, d0hi_f;          // axis limits extended by 0.01 cm (filters only)
    float err_scale;               // SAFE * 2^-24 / delta
    float dext_f;                  // |d0| of any root within half a bin of the axis, + margin
    float e3;                      // geometry part of the root bounds, in bins
    float rho_max_f, drho_f, dmax_f; // |rho| bound, row width, max |d0| (filters)
    // tables (device)
    const float *sn32, *cs32, *phi32, *rho32, *invrho32;
    const double *sn64, *cs64, *rho64;
    const float *snlo, *cslo, *rholo;  // float64 value - float32 table, as float32
    const double *esn64, *ecs64;       // column lower edges e_k = (2k - N) pi / N
    const float *esn32, *ecs32;
    float inv_delta_lo;                // 1/delta - inv_delta_f
    // z vote
    double dz, z0_max, cstep;      // dz = 2 z0_max / n_z0, cstep = cot_max / n_cot
    float inv_dz_f, z0_max_f, cstep_f;
};

constexpr float kEps = 5.9604644775390625e-8f;   // 2^-24, float32 unit roundoff
constexpr float kSafe = 4.0f;                    // slack on first-order error bounds
constexpr double kPi = 3.141592653589793;
constexpr double kHalfPi = 1.5707963267948966;

// ---------------------------------------------------------------------------
// Exact evaluation of one (hit, rho_i, phi0_k) column in float64, one
// correctly rounded operation at a time in the definition's order (the _rn
// intrinsics forbid contraction into FMA).  Writes the in-range bins to j[]
// and returns their number; *n_edge counts bin coordinates within 1e-5 of an
// integer.
static __device__ __noinline__ int cell_bins64(const DevGeom &G, float xf, float yf,
                                           int i, int k, int j[2], int *n_edge)
{
    const double x = (double)xf, y = (double)yf;
    const double sn = G.sn64[k], cs = G.cs64[k], rho = G.rho64[i];
    const double s = __dsub_rn(__dmul_rn(x, sn), __dmul_rn(y, cs));
    const double c = __dadd_rn(__dmul_rn(x, cs), __dmul_rn(y, sn));
    if (!(c > 0.0)) return 0;
    const double r2 = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
    const double b = __dadd_rn(1.0, __dmul_rn(rho, s));
    const double pc = __dmul_rn(rho, c);
    const double D = __dsub_rn(1.0, __dmul_rn(pc, pc));
    if (D < 0.0) return 0;
    const double sq = __dsqrt_rn(D);
    const double q = -__dadd_rn(b, b >= 0.0 ? sq : -sq);
    const double C = __dadd_rn(__dmul_rn(rho, r2), __dmul_rn(2.0, s));
    double root[2];
    int nr = 0;
    if (rho != 0.0) root[nr++] = __ddiv_rn(q, rho);
    if (q != 0.0 && !(D == 0.0 && rho != 0.0)) root[nr++] = __ddiv_rn(C, q);
    int nv = 0;
    for (int t = 0; t < nr; ++t) {
        const double u = __dadd_rn(__ddiv_rn(root[t], G.delta), G.off);
        if (u >= 0.0 && u < (double)G.n_d0) {
            const double fl = floor(u);
            const double fr = __dsub_rn(u, fl);
            j[nv++] = (int)fl;
            if (fr < 1e-5 || fr > 1.0 - 1e-5) ++*n_edge;
        }
    }
    return nv;
}

// ---------------------------------------------------------------------------
// Guarded float32 evaluation of one (hit, rho row, phi0 column).
//
// First-order error bounds, unit roundoff u = 2^-24 (the approximate MUFU
// reciprocal and reciprocal square root add <= 2u and <= 4.3u relative):
//   |ds|, |dc| <= 3u R1  (R1 = |x| + |y|);   |dD| <= u (10 (rho R1)^2 + 1);
//   |dq| <= u (Qa + Qb / sqrt(D)),  Qa = 6|rho|R1 + 9,  Qb = 5 (rho R1)^2 + 1/2;
//   root A = C / q:  |d dA| <= u (|1/q| (3|rho| r2 + 6 R1 + |dA| (Qa + Qb/sqrt D)) + 6 |dA|);
//   root B = q / rho: |d dB| <= u (|1/rho| (Qa + Qb/sqrt D) + 6 |dB|).
// Each is scaled by kSafe and divided by delta (bins), plus u|u| for the
// final fused multiply-add.  With |rho| bounded by the tile's largest and
// |d0| by dext (a root within half a bin of the axis), the bounds reduce to
//   eA = |1/q| (E1 + E2 / sqrt D) + E3,   eB = |1/rho| err_scale (Qa + Qb / sqrt D) + E3
// with E1, E2 (and Qa, Qb, the D bound eD) constant per (hit, column) item
// and E3 constant per geometry.  A root is decided here only if its bound is
// below 1/4 bin and its coordinate is farther than the bound from every
// integer (range edges included) or more than half a bin outside the axis;
// otherwise the whole column is redone by cell_bins64.
struct Item {
    float s, c, r2, eD;    // hit geometry in this column; D bound
    float E1, E2, Qa, Qb;  // root-A bound constants; root-B constants (scaled)
};

enum : int { kDecided = 0, kRedo = 1 };

__device__ __forceinline__ float rcp_approx(float v)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ float rsqrt_approx(float v)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// Bin of a root with coordinate u and bound e: j >= 0 (vote), -1 (certainly
// outside the axis) or -2 (undecided: redo).  Branch-free.  If u lies within
// e of the axis but outside it, its distance to the edge integer is below e,
// so it is undecided rather than misbinned; a NaN bound or coordinate is
// undecided too.  The distances to the integers below and above are u - f
// and (f + 1) - u: each is exact whenever it is the smaller one (u >= 0),
// and for f = -1 the second is -u exactly, at most e when u + e >= 0, so a
// root within e below the axis is undecided.  (1 - (u - f) would not do:
// u + 1 is rounded for u in (-1, 0) and can pass the test.)
__device__ __forceinline__ int decide(float u, float e, float nd)
{
    const float f = floorf(u);
    const float fr = u - f;
    const bool out = (u + e < 0.0f) | (u - e >= nd);
    const bool ok = fminf(fr, (f + 1.0f) - u) > e;
    return out ? -1 : (ok ? (int)f : -2);
}

// Returns kDecided with jA, jB (bin or -1) or kRedo.  NEED_B = false: the
// caller has proven root B out of the axis (jB = -1 without evaluating it).
template <bool NEED_B>
__device__ __forceinline__ int eval32(const DevGeom &G, float rho, float invrho_es,
                                      float invrho, const Item &it, int &jA, int &jB)
{
    const float b = fmaf(rho, it.s, 1.0f);
    const float pc = rho * it.c;
    const float D = fmaf(-pc, pc, 1.0f);
    const bool none = D < -it.eD;          // certainly no real root
    const bool tangent = D <= it.eD;       // sign of D not proven
    const float Dp = fmaxf(D, 1e-30f);
    const float rs = rsqrt_approx(Dp);
    const float sq = Dp * rs;
    const float q = -(b + copysignf(sq, b));
    const float C = fmaf(rho, it.r2, it.s + it.s);
    const float iq = rcp_approx(q);
    const float nd = (float)G.n_d0;
    const float uA = fmaf(C * iq, G.inv_delta_f, G.off_f);
    const float eA = fmaf(fabsf(iq), fmaf(it.E2, rs, it.E1), G.e3);
    int a = decide(uA, eA, nd);
    int bb = -1;
    if (NEED_B) {
        const float uB = fmaf(q * invrho, G.inv_delta_f, G.off_f);
        const float eB = fmaf(invrho_es, fmaf(it.Qb, rs, it.Qa), G.e3);
        bb = decide(uB, eB, nd);
    }
    jA = tangent ? -1 : a;
    jB = tangent ? -1 : bb;
    if (none) return kDecided;
    return (tangent | (a == -2) | (bb == -2)) ? kRedo : kDecided;
}

// Per-(hit, column) constants for eval32; rt = largest |rho| of the tile.
__device__ __forceinline__ Item make_item(const DevGeom &G, float s, float c, float r2,
                                          float R1, float rt)
{
    Item it;
    it.s = s;
    it.c = c;
    it.r2 = r2;
    const float P = rt * R1;
    const float Qa = fmaf(6.0f, P, 9.0f);
    const float Qb = fmaf(5.0f * P, P, 0.5f);
    it.eD = (kSafe * kEps) * fmaf(10.0f * P, P, 2.0f);
    const float Ea = fmaf(3.0f * rt, r2, 6.0f * R1);
    it.E1 = G.err_scale * fmaf(G.dext_f, Qa, Ea);
    it.E2 = G.err_scale * G.dext_f * Qb;
    it.Qa = Qa;
    it.Qb = Qb;
    return it;
}

// ---------------------------------------------------------------------------
// Phase-1 filters shared by the tile kernels.
//
// Angular window of a hit: any circle with |rho| <= rho_max through a hit at
// radius r whose perigee lies within dmax of the origin has its phi0 within
//   asin(min(1, rho_max (r + dmax) / 2)) + asin(min(1, dmax / r))
// of the hit's azimuth (half the turning angle along the chord from the
// perigee, plus the angle the chord makes with the hit's radius), and c > 0
// bounds it by pi/2.  A 1e-3 rad margin covers float32 rounding.
// Phase 1 tests it as a bound on c = r cos(phi0 - phi_hit): with
// A = asin(a), B = asin(b) the two terms above, cos(A + B) = sqrt((1 - a^2)(1 - b^2))
// - a b, and cos(w + 1e-3) >= cos(w) - 1e-3, so c < r (cos(A + B) - 1e-3)
// implies the column is outside the window (a superset of what it keeps;
// when A + B passes pi/2 the bound is negative and the c > 0 test rules).
// No trigonometric call per hit.
// r and 1/r come from one approximate reciprocal square root of r^2 (a few
// units of 2^-23 off, far inside the 1e-3 margin).
__device__ __forceinline__ float hit_cos_window(const DevGeom &G, float r2)
{
    const float ir = rsqrt_approx(fmaxf(r2, 1e-30f));
    const float r = r2 * ir;
    const float a = fminf(1.0f, G.rho_max_f * (r + G.dmax_f) * 0.5f);
    const float b = fminf(1.0f, G.dmax_f * ir);
    const float cw = sqrtf(fmaxf(fmaf(-a, a, 1.0f) * fmaf(-b, b, 1.0f), 0.0f)) - a * b;
    return r * (cw - 1e-3f);
}

// Curvature range reached by circles through a hit (s, c) with perigee d0 in
// the (extended) axis: the circle equation is rho (w^2 + c^2) + 2 w = 0 with
// w = d0 + s, so rho = g(w) = -2 w / (w^2 + c^2), which falls on |w| < c and
// rises outside; its extremes over an interval are at the ends or at w = -c
// (max 1/c) and w = c (min -1/c).  Used only to skip (hit, column) pairs
// that cannot vote in a block of rows, and widened so that it holds the
// range of the float64 s and c: e bounds the float32 error of both (the
// caller's 3 2^-24 (|x| + |y|) from the rounded tables and products), the
// window grows by e, and the range by 1.5 e / c^2 (|dg/dc| <= 1.3 / c^2)
// plus 1e-6 / c for the float32 evaluation (|g| <= 1 / c; a few ulp).
// Callers keep a one-row margin besides and skip the test for c <= 1 cm.
__device__ __forceinline__ void rho_range_w(float wlo, float whi, float c, float e, float &gmin,
                                            float &gmax)
{
    wlo -= e;
    whi += e;
    const float c2 = c * c;
    const float glo = __fdividef(-2.0f * wlo, fmaf(wlo, wlo, c2));
    const float ghi = __fdividef(-2.0f * whi, fmaf(whi, whi, c2));
    const float ic = rcp_approx(c);
    const float m = fmaf(1.5f * e, ic * ic, 1e-6f * ic);
    gmax = ((wlo <= -c && -c <= whi) ? ic : fmaxf(glo, ghi)) + m;
    gmin = ((wlo <= c && c <= whi) ? -ic : fminf(glo, ghi)) - m;
}

__device__ __forceinline__ void rho_range(const DevGeom &G, float s, float c, float e,
                                          float &gmin, float &gmax)
{
    rho_range_w(G.d0lo_f + s, G.d0hi_f + s, c, e, gmin, gmax);
}

// ---------------------------------------------------------------------------
// Regions of the learned proposal: an 8 x 8 grid of blocks over (rho row,
// d0 bin); row i lies in block i * 8 / n_rho, bin j in block j * 8 / n_d0,
// and region r = 8 * (rho block) + (d0 block) is bit r of a 64-bit mask.
// A cell is INSIDE the mask when its region's bit is set; it is in the HALO
// when some inside cell is at most one row and one bin away.  The masked
// vote gives every halo cell its full count, so every 26-neighbour of an
// inside cell is exact and the masked peaks are the full peaks inside.
__device__ __forceinline__ int region_block(int v, int n) { return (v * 8) / n; }

// First bin (or row) of block b; b = 8 gives n.
__device__ __forceinline__ int block_first(int b, int n) { return (b * n + 7) / 8; }

// d0 blocks that have an inside cell within one row of row i.
__device__ __forceinline__ unsigned halo_row_blocks(unsigned long long mask, int i, int NR)
{
    unsigned bm = 0u;
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
        const int ii = i + di;
        if (ii >= 0 && ii < NR) bm |= (unsigned)(mask >> (8 * region_block(ii, NR))) & 0xffu;
    }
    return bm;
}

// Whether bin j of a row whose halo_row_blocks are bm lies in the halo.
__device__ __forceinline__ bool halo_bin(unsigned bm, int j, int ND)
{
    unsigned b = bm >> region_block(j, ND);
    if (j > 0) b |= bm >> region_block(j - 1, ND);
    if (j < ND - 1) b |= bm >> region_block(j + 1, ND);
    return (b & 1u) != 0u;
}

// ---------------------------------------------------------------------------
// atan2 from basic float64 operations in a fixed order (three half-angle
// reductions atan t = 2 atan(t / (1 + sqrt(1 + t^2))), then the Maclaurin
// series of atan to t^21 by Horner's rule), so that any implementation that
// follows the same steps with correctly rounded operations gives the same
// bits.  (0, 0) -> 0; the sign of a zero y is ignored.
__device__ __forceinline__ double atan_unit64(double t)
{
#pragma unroll 1
    for (int h = 0; h < 3; ++h)
        t = __ddiv_rn(t, __dadd_rn(1.0, __dsqrt_rn(__dadd_rn(1.0, __dmul_rn(t, t)))));
    const double t2 = __dmul_rn(t, t);
    double p = __ddiv_rn(1.0, 21.0);
#pragma unroll 1
    for (int k = 9; k >= 0; --k)
        p = __dsub_rn(__ddiv_rn(1.0, (double)(2 * k + 1)), __dmul_rn(t2, p));
    return __dmul_rn(8.0, __dmul_rn(t, p));
}

__device__ __forceinline__ double atan2_basic64(double y, double x)
{
    if (x == 0.0 && y == 0.0) return 0.0;
    const double ax = fabs(x), ay = fabs(y);
    double a;
    if (ay <= ax)
        a = atan_unit64(__ddiv_rn(ay, ax));
    else
        a = __dsub_rn(kHalfPi, atan_unit64(__ddiv_rn(ax, ay)));
    if (x < 0.0) a = __dsub_rn(kPi, a);
    return y < 0.0 ? -a : a;
}

// ---------------------------------------------------------------------------
// Host-side launchers (one per kernel file).
cudaError_t launch_vote(const DevGeom &G, const float *x, const float *y, int n, void *acc,
                        unsigned long long *stats, cudaStream_t st);
// Masked vote: *mask (device) selects the regions; halo cells get full counts.
cudaError_t launch_vote_masked(const DevGeom &G, const float *x, const float *y, int n,
                               void *acc, unsigned long long *stats,
                               const unsigned long long *mask, cudaStream_t st);
// Per-event lists of the hits that can vote in each group of kGroupCols
// phi0 columns (k_buckets.cu): group g of event e holds cnt[e G + g] local
// hit indices at ent + start[e G + g], G = ngroups.
constexpr int kGroupCols = 8;
// Packed 16-bit tile counters are exact for tiles scanning up to this many
// hits (two votes per hit at most in a cell: 2 * 32767 < 2^16).
constexpr int kPackMaxHits = 32767;
struct HitBuckets {
    int *cnt, *start, *cursor, *ent;
    int *hg;   // per hit: first group | group count << 16
    void *tmp;
    int ngroups, ncells;
};
// What a tile kernel reads of the lists (ent null: no lists).
struct BucketView {
    const int *cnt, *start, *ent;
    int ngroups;

    __device__ __forceinline__ void list(int e, int k0, const int *&hl, int &nl) const
    {
        const int c = e * ngroups + k0 / kGroupCols;
        hl = ent + start[c];
        nl = cnt[c];
    }
};
inline BucketView bucket_view(const HitBuckets *b)
{
    return b ? BucketView{b->cnt, b->start, b->ent, b->ngroups}
             : BucketView{nullptr, nullptr, nullptr, 0};
}
size_t hit_bucket_bytes(const DevGeom &G, int max_events, int max_hits);
HitBuckets carve_hit_buckets(const DevGeom &G, int max_events, int max_hits, void *ws);
cudaError_t launch_hit_buckets(const DevGeom &G, const float *x, const float *y, const int *off,
                               const int *d_nev, int max_hits, const HitBuckets &b, int sms,
                               cudaStream_t st);

// Swept-interval vote: each (rho row, phi0 column) votes the d0 bins the
// hit's roots sweep between the column's edges (k_swept.cu).
cudaError_t launch_vote_swept(const DevGeom &G, const float *x, const float *y, int n, void *acc,
                              unsigned long long *stats, cudaStream_t st);
// Per-hit vote: hit h's votes count only in the halo cells of hit_masks[h].
cudaError_t launch_vote_hitmask(const DevGeom &G, const float *x, const float *y, int n,
                                void *acc, unsigned long long *stats,
                                const unsigned long long *hit_masks, cudaStream_t st);
// mask (device, or null for every cell): only peaks inside it are reported.
// spill (peak_spill_bytes, or null): lets the stencil run once instead of
// twice; it may be shared by launches that run one after another.
cudaError_t launch_peaks(const DevGeom &G, const void *acc, ht_peak *peaks, int cap,
                         int *d_count, void *ws, cudaStream_t st,
                         const unsigned long long *mask = nullptr, const int *d_thr = nullptr,
                         void *spill = nullptr);
size_t peaks_workspace_bytes(const DevGeom &G);
size_t peak_spill_bytes(const DevGeom &G);
cudaError_t launch_associate(const DevGeom &G, const float *x, const float *y, int n,
                             const ht_peak *peaks, const int *d_count, int cap, int *assign,
                             void *ws, cudaStream_t st);
size_t associate_workspace_bytes(const DevGeom &G, int n, int cap);
cudaError_t launch_vote_z(const DevGeom &G, const float *x, const float *y, const float *z,
                          int n, const int *assign, const ht_peak *peaks, const int *d_count,
                          int cap, ht_zres *out, void *ws, cudaStream_t st);
size_t vote_z_workspace_bytes(const DevGeom &G, int n, int cap);

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Per-event hit index by (layer, azimuth bin) (k_hitindex.cu): cell
// (e * 16 + l) * kIdxAz + b holds positions offs[cell] .. offs[cell + 1) of
// x, y (float32), h (event-local hit index) and l (layer); rmm[2 (e 16 + l)]
// and [+ 1] are the float bits of the least and largest hit radius of the
// layer (min > max: no hit).
constexpr int kIdxAz = 256;
struct HitIndex {
    int *cnt, *offs, *cur;
    unsigned *rmm;
    float *x, *y;
    int *h;
    uint8_t *l;
    void *tmp;
    int ncells;
};
size_t hit_index_bytes(int max_events, int max_hits);
HitIndex carve_hit_index(int max_events, int max_hits, void *ws);
cudaError_t launch_hit_index(const float *x, const float *y, const uint8_t *layer,
                             const int *off, const int *d_nev, int max_events, int max_hits,
                             const HitIndex &I, int sms, cudaStream_t st);

// Candidate confirmation (k_confirm.cu): parameters as ht_confirm_desc.
struct ConfirmDev {
    int pool, min_layers, n_layers;
    double tol;
};
// Batch: event e's hits at x[off[e] ..), candidates peaks[e cap ..), kept
// counts min(counts[e], cap); score (n_ev cap), inl (16 n_ev cap) and
// assign (batch hit index) written.  ws: confirm_workspace_bytes.
size_t confirm_workspace_bytes(const DevGeom &G, int max_events, int max_hits, int cap);
cudaError_t prepare_confirm_kernels();
// Compact found tracks of a batch (k_confirm.cu): tracks[tfirst[e] ..
// tfirst[e + 1]) are event e's confirmed candidates in candidate order (the
// first tcap of all written), *ntot their total, assign_out each hit's index
// into its event's tracks (-1 none).  ws: track_compact_bytes.
size_t track_compact_bytes(int max_events, int cap);
cudaError_t launch_track_compact(const int *off, const int *d_nev, int max_events, int max_hits,
                                 const ht_peak *peaks, const int *counts, int cap,
                                 const int *score, const ht_zres *zres, const int *assign,
                                 ht_track_out *tracks, int tcap, int *tfirst, int *ntot,
                                 int *assign_out, void *ws, int sms, cudaStream_t st);
cudaError_t launch_confirm_batch(const DevGeom &G, const ConfirmDev &P, const float *x,
                                 const float *y, const uint8_t *layer, const int *off,
                                 const int *d_nev, int max_events, int max_hits,
                                 const ht_peak *peaks, const int *counts, int cap, int *score,
                                 int *inl, int *assign, void *ws, int sms, cudaStream_t st,
                                 const HitBuckets *hb);
// One event of n hits (host) and *d_count candidates (device).
size_t confirm_workspace_bytes_single(const DevGeom &G, int n, int cap);
cudaError_t launch_confirm(const DevGeom &G, const ConfirmDev &P, const float *x, const float *y,
                           const uint8_t *layer, int n, const ht_peak *peaks, const int *d_count,
                           int cap, int *score, int *inl, int *assign, void *ws, cudaStream_t st);

// Records msg as this host thread's ht_last_error() text; returns s.
ht_status set_error(ht_status s, const char *msg);

size_t scan_tmp_bytes(int n_cap);
cudaError_t scan_exclusive(const int *in, int *out, int *out2, int n_cap, const int *d_n,
                           int *total, void *tmp, cudaStream_t st);

}  // namespace ht

// The geometry handle behind the opaque ht_geometry of the C ABI.
struct ht_geometry {
    ht_geometry_desc desc;
    ht::DevGeom G;
    void *d_tables;
    int device;
};
