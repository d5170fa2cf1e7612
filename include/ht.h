/*
 * ht.h -- C ABI of the GB300 Hough-transform track-finding library (libht).
 *
 * Method: Halyo, LeGresley, Lujan, "Massively Parallel Computing and the
 * Search for Jets and Black Holes at the LHC", arXiv:1309.6275.  Section 5
 * defines the transform (each input adds a vote to every parametrised
 * feature that contains it; local maxima of the vote space are candidates;
 * costlier computations then confirm them); Section 6 (Fig. 5) chains
 * transform -> peak finding -> refinement; Section 7 tunes the peak finder
 * for tracks of at least seven hits.  The paper gives no formulas or bin
 * layout; the readings used here are stated beside each call.
 *
 * Conventions shared by every call
 *  - Units: cm.  Hits are float32 structure-of-arrays (x[], y[], z[]).
 *  - Parameter space: signed curvature rho (> 0 counter-clockwise),
 *    transverse impact parameter d0, azimuth phi0 at the perigee.  A hit
 *    (x, y) lies on the circle (rho, d0, phi0) iff
 *      rho d0^2 + 2 (1 + rho s) d0 + (rho r^2 + 2 s) = 0,
 *      s = x sin phi0 - y cos phi0,  c = x cos phi0 + y sin phi0.
 *  - Axes: rho_i = (2i + 1 - n_rho) rho_max / n_rho,
 *    phi0_k = (2k + 1 - n_phi0) pi / n_phi0 (phi0 wraps),
 *    d0 bin j holds u = d0 / delta + n_d0 / 2 + 1/2 in [j, j + 1),
 *    delta = 2 d0_half / n_d0 (d0 = 0 is a bin centre).
 *  - Accumulator: n_rho x n_d0 x n_phi0 cells of uint16 (count_bits 16) or
 *    int32 (count_bits 32), logical index l = (i n_d0 + j) n_phi0 + k,
 *    counts saturate at the type maximum.
 *  - Every pointer argument is DEVICE memory owned by the caller unless
 *    marked "host".  Calls are asynchronous on `stream` (NULL = the legacy
 *    default stream), never synchronise the host and keep every count in
 *    device memory, except ht_run_event which is synchronous.
 *  - Every call returns an ht_status; no C++ exception crosses the ABI.  On
 *    failure ht_last_error() returns a description (per host thread).
 *  - Results are bit-identical to the plain fp64 CPU definition of each
 *    step: float32 arithmetic decides only votes it can prove are at least
 *    its error bound away from every decision edge; the others are redone
 *    in float64 with the definition's operation order.
 */
#ifndef HT_H
#define HT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;                       /* = cudaStream_t */
typedef struct CUstream_st *ht_stream;

typedef int32_t ht_status;
#define HT_OK 0
#define HT_ERR_ARG 1        /* invalid argument (null, size, alignment) */
#define HT_ERR_CAPACITY 2   /* a size exceeds what the call supports      */
#define HT_ERR_CUDA 3       /* a CUDA runtime call or launch failed       */
#define HT_ERR_TIMEOUT 4    /* a bounded device-side wait gave up         */

/* Geometry of the parameter space.  Requirements checked by
 * ht_geometry_create: n_rho in [1, 65535]; n_d0 in [2, 512]; n_phi0 a
 * multiple of 8 in [8, 2^20]; n_z0, n_cot in [1, 1024] with
 * n_z0 * n_cot <= 32768; n_rho * n_d0 * n_phi0 < 2^31; threshold >= 1;
 * count_bits 16 or 32; rho_max, d0_half, z0_max, cot_max > 0; the tiles
 * must fit the device's shared memory. */
typedef struct ht_geometry_desc {
    int32_t n_rho, n_d0, n_phi0;
    int32_t n_z0, n_cot;
    int32_t threshold;   /* peak threshold T (Section 7: tracks of >= 7 hits) */
    int32_t count_bits;  /* 16: uint16 cells; 32: int32 cells */
    int32_t reserved;    /* set to 0 */
    double rho_max;      /* curvature half range, 1/cm */
    double d0_half;      /* d0 half range, cm */
    double z0_max;       /* z0 axis covers [-z0_max, z0_max), cm */
    double cot_max;      /* cot(theta) axis covers [-cot_max, cot_max) */
} ht_geometry_desc;

typedef struct ht_geometry ht_geometry;   /* opaque handle */

/* A candidate track: cell indices and its vote count. */
typedef struct ht_peak { int32_t i_rho, j_d0, k_phi0, count; } ht_peak;

/* Result of the (z0, cot theta) vote of one candidate. */
typedef struct ht_zres { int32_t n_z0, m_cot, count; } ht_zres;

/* Create a geometry handle on the current CUDA device.  The library owns the
 * handle and its device tables (sin/cos phi0 and rho in float32 and float64,
 * a few KB), computed on the host in float64 and uploaded.  *out receives the
 * handle.  Errors: HT_ERR_ARG (desc or out null, a requirement above
 * violated), HT_ERR_CUDA. */
ht_status ht_geometry_create(const ht_geometry_desc *desc, ht_geometry **out);

/* Release a handle and its device tables (NULL is accepted).  The caller
 * must make sure no work using the handle is still queued. */
ht_status ht_geometry_destroy(ht_geometry *g);

/* Description of the last failure on this host thread ("" if none). */
const char *ht_last_error(void);

/* Bytes of one accumulator: n_rho * n_d0 * n_phi0 * (count_bits / 8). */
size_t ht_accumulator_bytes(const ht_geometry *g);

/* Hough vote (Section 5).  For each hit h, row i and column k with c > 0,
 * every real root d0 of the circle equation (a double root once) whose bin
 * coordinate lies in [0, n_d0) adds one vote to cell (i, j, k).  Reading:
 * c > 0 keeps the first half turn only, so a track gives one peak, not a
 * mirror pair.
 *   x, y      n_hits float32 each, 16-byte aligned (device).
 *   n_hits    >= 0 (0 writes an all-zero accumulator).
 *   acc       accumulator (device, 16-byte aligned, ht_accumulator_bytes);
 *             every cell is written, so it needs no clearing.
 *   stats     NULL or 2 device uint64: votes cast, and (hit, row, column)
 *             evaluations redone in float64 because float32 could not prove
 *             their bins.  The call zeroes them first.
 * Errors: HT_ERR_ARG (null pointer with n_hits > 0, misalignment, n_hits < 0),
 * HT_ERR_CUDA. */
ht_status ht_vote(const ht_geometry *g, const float *x, const float *y,
                  int32_t n_hits, void *acc, uint64_t *stats, ht_stream stream);

/* Peak finding (Sections 5-7).  Reading: cell l is a peak iff its count is
 * >= threshold and, for each existing 26-neighbour l' (rho and d0 do not
 * wrap, phi0 wraps), count(l) > count(l') when l' < l and count(l) >=
 * count(l') when l' > l.  Peaks are written in increasing l.
 *   acc        accumulator from ht_vote (device, 16-byte aligned).
 *   peaks      cap entries (device); the first min(total, cap) are written.
 *   cap        >= 0.
 *   d_count    one device int32: the total number of peaks (may exceed cap).
 *   workspace  ht_find_peaks_workspace_size(g) bytes of device scratch,
 *              256-byte aligned; contents need no initialisation.
 * Errors: HT_ERR_ARG, HT_ERR_CUDA. */
size_t ht_find_peaks_workspace_size(const ht_geometry *g);
ht_status ht_find_peaks(const ht_geometry *g, const void *acc, ht_peak *peaks,
                        int32_t cap, int32_t *d_count, void *workspace,
                        size_t workspace_bytes, ht_stream stream);

/* ht_find_peaks for callers that cannot allocate device memory: identical
 * results, but its scratch is a fixed array inside the library instead of a
 * caller-provided workspace.  Some callers cannot call cudaMalloc at all --
 * trigger code that must not allocate once data taking has started, or code
 * embedded in a host framework that owns every device allocation and hands
 * its plug-ins no allocator -- and this entry point is for them.  The paper
 * has no counterpart; it is an interface convenience only.
 *   Limit: n_rho * n_d0 * ceil(n_phi0 / 256) <= 524288 (about 4 MiB of
 *   scratch, held on every GPU that loads the library until the process
 *   exits); larger geometries get HT_ERR_CAPACITY.
 *   The first call on a device (made with that device current) looks up the
 *   scratch's device address; make that first call before any stream capture.
 *   A failed lookup is not remembered (the next call tries again); after a
 *   cudaDeviceReset the remembered address is stale, so restart the process.
 *   All calls share the one array: calls that overlap on the GPU (different
 *   streams, or different host threads) race and give wrong results, so
 *   serialise them.  Nothing in the array needs clearing between calls.
 *   Other arguments as ht_find_peaks.
 * Errors: HT_ERR_ARG, HT_ERR_CAPACITY, HT_ERR_CUDA. */
ht_status ht_find_peaks_noalloc(const ht_geometry *g, const void *acc, ht_peak *peaks,
                                int32_t cap, int32_t *d_count, ht_stream stream);

/* Hit association, the confirming step of Section 5.  Reading: hit h is
 * compatible with candidate m iff one of its votes (exactly as ht_vote casts
 * them) lies in a cell with |i - i_m| <= 1, |j - j_m| <= 1 and circular
 * |k - k_m| <= 1; it is assigned to the compatible candidate of largest
 * count, ties to the smallest m, else -1.  Candidates are
 * peaks[0 .. min(*d_count, cap)), in increasing l (ht_find_peaks order).
 * The candidates must be ht_find_peaks output (no two of them adjacent);
 * other lists give unspecified assignments.
 *   assign     n_hits int32 (device).
 *   workspace  ht_associate_workspace_size(g, n_hits, cap) bytes, 256-byte
 *              aligned.
 * Errors: HT_ERR_ARG, HT_ERR_CUDA. */
size_t ht_associate_workspace_size(const ht_geometry *g, int32_t n_hits, int32_t cap);
ht_status ht_associate(const ht_geometry *g, const float *x, const float *y,
                       int32_t n_hits, const ht_peak *peaks,
                       const int32_t *d_count, int32_t cap, int32_t *assign,
                       void *workspace, size_t workspace_bytes, ht_stream stream);

/* Second vote in (z0, cot theta) per candidate (reading; the paper is
 * transverse-plane only).  At the candidate's cell centres
 * (rho_i, d0_j = (j - n_d0/2) delta, phi0_k), each assigned hit has turning
 * angle theta = atan2(rho c, 1 + rho (s + d0_j)) and arc length
 * L = theta / rho (L = c if rho == 0); for each cot centre
 * t_q = (2q + 1 - n_cot) cot_max / n_cot it votes z0 = z - L t_q into bin
 * floor((z0 + z0_max) / dz), dz = 2 z0_max / n_z0, if inside [0, n_z0).
 * Output per candidate: the cell of most votes {n, q, count}, ties to the
 * smallest n n_cot + q; {-1, -1, 0} if it received none.  atan2 here is a
 * fixed sequence of basic operations (three half-angle reductions and a
 * 10-term Maclaurin series), so results are reproducible bit for bit.
 *   out        cap entries (device); the first min(*d_count, cap) are written.
 *   workspace  ht_vote_z_workspace_size(g, n_hits, cap) bytes, 256-aligned.
 * Errors: HT_ERR_ARG, HT_ERR_CUDA. */
size_t ht_vote_z_workspace_size(const ht_geometry *g, int32_t n_hits, int32_t cap);
ht_status ht_vote_z(const ht_geometry *g, const float *x, const float *y,
                    const float *z, int32_t n_hits, const int32_t *assign,
                    const ht_peak *peaks, const int32_t *d_count, int32_t cap,
                    ht_zres *out, void *workspace, size_t workspace_bytes,
                    ht_stream stream);

/* The whole path for one event from HOST buffers (Fig. 5 up to the
 * refinement step): copies the hits to the device, runs ht_vote,
 * ht_find_peaks, ht_associate and ht_vote_z on `stream`, copies the results
 * back and synchronises the stream before returning.
 *   hx, hy, hz   host float32 arrays of n_hits (pinned memory is faster).
 *   workspace    ht_event_workspace_size(g, n_hits, cap) bytes of device
 *                memory, 256-byte aligned (holds hits, accumulator, peaks,
 *                assignments, z results and scratch).
 *   h_peaks      host, cap entries; h_count host int32 (total peaks);
 *   h_assign     host, n_hits; h_zres host, cap entries;
 *   h_stats      host, 2 uint64 as ht_vote's stats (may be NULL).
 * Errors: HT_ERR_ARG, HT_ERR_CUDA. */
size_t ht_event_workspace_size(const ht_geometry *g, int32_t n_hits, int32_t cap);
ht_status ht_run_event(const ht_geometry *g, const float *hx, const float *hy,
                       const float *hz, int32_t n_hits, void *workspace,
                       size_t workspace_bytes, ht_peak *h_peaks, int32_t cap,
                       int32_t *h_count, int32_t *h_assign, ht_zres *h_zres,
                       uint64_t *h_stats, ht_stream stream);

/* Swept-interval vote (the paper samples phi0 at bin centres; this variant
 * votes, in each phi0 column, the d0 range the hit's roots sweep across the
 * column, for coarse phi0 binning).  The roots are sampled at the column's
 * lower edge e_k = (2k - N) pi / N, its centre and its upper edge
 * e_{(k+1) mod N}; at each sample they exist when c > 0 and D >= 0 and are
 * labelled by branch (+ and - sqrt D); per branch, two consecutive samples
 * with the root give every bin between their bins (roots beyond the axis
 * clamp to its ends), a sample whose neighbours lack the root gives its own
 * bin; a cell gets one vote per hit when its bin is in the union over both
 * branches.  It contains ht_vote's cells (not its double votes) and tends to
 * them as n_phi0 grows.  acc: as ht_vote (every cell written).  stats: NULL
 * or 2 uint64, stats[0] = votes cast, stats[1] = 0.  Peaks, association and
 * the z vote apply unchanged to acc.  Errors: as ht_vote; HT_ERR_ARG also
 * when n_d0 needs more shared memory than a tile has. */
ht_status ht_vote_swept(const ht_geometry *g, const float *x, const float *y, int32_t n_hits,
                        void *acc, uint64_t *stats, ht_stream stream);

/* ------------------------------------------------------------------------
 * Track finding in dense events: the distinct-layer vote and the candidate
 * confirmation (Section 5: local maxima are candidates that costlier
 * computations confirm; Fig. 5 refines them; Section 7 tunes the peak finder
 * for tracks of at least seven hits).  A track leaves at most one hit per
 * detector layer, and at thousands of hits per event the inner layers are
 * so dense that with plain counts their hits pile tens of votes into every
 * cell of the d0 band they reach; counting layers removes that pile-up.
 * ------------------------------------------------------------------------ */

/* Distinct-layer vote.  Every hit casts exactly ht_vote's votes; a cell's
 * count is the number of distinct layers among the hits voting in it.
 *   layer   n_hits uint8 (device), each in [0, 16).
 *   acc     as ht_vote (uint16 or int32 cells, every cell written).
 *   stats   NULL or 2 device uint64: votes cast, and float64 redos.
 * Requires an even n_d0.  Peaks (ht_find_peaks) apply unchanged to acc, the
 * threshold then counting layers.  Errors: as ht_vote; HT_ERR_ARG also for
 * a null layer array or an odd n_d0. */
ht_status ht_vote_layers(const ht_geometry *g, const float *x, const float *y,
                         const uint8_t *layer, int32_t n_hits, void *acc, uint64_t *stats,
                         ht_stream stream);

/* Confirmation parameters.  pool: bins of the candidate's column around its
 * bin that supply inlier hits (>= 0); min_layers: inlier layers needed
 * (>= 1); n_layers: layers 0 .. n_layers - 1 take part (1 to 16); tol: inlier
 * distance to the seed circle, cm (> 0).  The bands set, for the batched
 * track path, each event's peak threshold from its hit count: an event of n
 * hits takes band_threshold[b] for the first b < n_bands with
 * n <= band_max_hits[b], else the geometry's threshold (n_bands 0 to 8). */
typedef struct ht_confirm_desc {
    int32_t pool, min_layers, n_layers, n_bands;
    double tol;
    int32_t band_max_hits[8];
    int32_t band_threshold[8];
} ht_confirm_desc;

/* Confirmation of one event's candidates and the final hit assignment.
 * Reading, for candidate m = (i, j, k) and every hit h, with b the bins of
 * h's roots in column (rho_i, phi0_k) exactly as ht_vote casts them:
 * own(h) iff some b == j; pool(h) iff some |b - j| <= pool.  Seed layers:
 * the layers holding exactly one own hit, at least three of them; the seed
 * circle passes through the own hits of the first, the last, and the one
 * between them whose index is nearest the middle of those two (the smaller
 * on a tie).  Inliers: per layer, the pool hit closest to the circle
 * (|distance to the centre - radius|, the smaller hit index on a tie) if
 * that distance is below tol.  Confirmed iff there are at least min_layers
 * inlier layers.  Each hit is then assigned to the confirmed candidate that
 * lists it with the most inlier layers, ties to the smallest m, else -1.
 * Float32 decides a bin only where it is proven (else float64 in the
 * definition's order); the circle and the distances are float64, one
 * correctly rounded operation at a time: results are bit-identical to the
 * float64 definition.
 *   peaks, d_count, cap   candidates as ht_find_peaks wrote them.
 *   score     cap int32 (device): inlier layers of candidate m, 0 when not
 *             confirmed (only the first min(*d_count, cap) are written).
 *   inliers   16 cap int32 (device): inliers[16 m + l] = the inlier hit of
 *             layer l, -1 for none (all -1 when not confirmed).
 *   assign    n_hits int32 (device).
 *   workspace ht_confirm_workspace_size(g, n_hits, cap) bytes, 256-byte aligned.
 * Errors: HT_ERR_ARG (null pointers, parameters out of range), HT_ERR_CUDA. */
size_t ht_confirm_workspace_size(const ht_geometry *g, int32_t n_hits, int32_t cap);
ht_status ht_confirm(const ht_geometry *g, const ht_confirm_desc *c, const float *x,
                     const float *y, const uint8_t *layer, int32_t n_hits, const ht_peak *peaks,
                     const int32_t *d_count, int32_t cap, int32_t *score, int32_t *inliers,
                     int32_t *assign, void *workspace, size_t workspace_bytes, ht_stream stream);

/* ------------------------------------------------------------------------
 * Region masks (learned proposal).  The paper has no learned part; these
 * calls restrict the Section 5 vote and peak finding to regions that a
 * per-hit network proposes.  Regions: an 8 x 8 grid of blocks over (rho
 * row, d0 bin); row i is in rho block i * 8 / n_rho, bin j in d0 block
 * j * 8 / n_d0, and region 8 * (rho block) + (d0 block) is bit r of a
 * uint64 mask.  A cell is INSIDE a mask when its region's bit is set, and in
 * its HALO when an inside cell is at most one row and one bin away.
 * ------------------------------------------------------------------------ */

/* ht_vote restricted to a mask: every halo cell receives exactly the count
 * ht_vote gives it; other cells hold unspecified values, and tiles of 32
 * rows x a few columns that contain no halo cell are not written at all.
 * Work outside the halo is skipped.  mask: ONE device uint64.  stats: as
 * ht_vote, counting the votes in halo cells.  Other arguments as ht_vote.
 * Errors: as ht_vote. */
ht_status ht_vote_masked(const ht_geometry *g, const float *x, const float *y,
                         int32_t n_hits, const uint64_t *mask, void *acc, uint64_t *stats,
                         ht_stream stream);

/* The vote with one region set per hit: hit h's votes count only in the
 * halo cells of hit_masks[h] (device, n_hits uint64, 8-byte aligned); every
 * cell of acc is written (cells no allowed vote reaches hold 0).  With every
 * mask all ones this is ht_vote.  stats: as ht_vote, counting the votes
 * cast.  Other arguments as ht_vote.  Errors: as ht_vote. */
ht_status ht_vote_hit_masked(const ht_geometry *g, const float *x, const float *y,
                             int32_t n_hits, const uint64_t *hit_masks, void *acc,
                             uint64_t *stats, ht_stream stream);

/* ht_find_peaks restricted to a mask: exactly the peaks ht_find_peaks
 * reports for the full accumulator that are inside the mask, in the same
 * order.  Reads only (blocks of) inside cells and their neighbours, so acc
 * needs only its halo cells right (ht_vote_masked output is enough).
 * mask: ONE device uint64.  Other arguments as ht_find_peaks.  Errors: as
 * ht_find_peaks. */
ht_status ht_find_peaks_masked(const ht_geometry *g, const void *acc, const uint64_t *mask,
                               ht_peak *peaks, int32_t cap, int32_t *d_count, void *workspace,
                               size_t workspace_bytes, ht_stream stream);

/* ------------------------------------------------------------------------
 * Proposal network: per-hit MLP 6 -> 128 -> 128 -> 64 with ReLU and a
 * softmax over the 64 regions; the 128 x 128 and 128 x 64 layers of the
 * forward pass run on the tensor cores (tcgen05, BF16 in, float32 out).  Features of a hit (float32, then rounded
 * to BF16): x/110, y/110, z/(110 sinh 2.5), r/110, atan2(y, x)/pi,
 * layer/9.  Weights and hidden activations are BF16, sums float32.
 * Parameters: one flat array of ht_mlp_param_count() values laid out
 * W1[6][128] b1[128] W2[128][128] b2[128] W3[128][64] b3[64] (W[i][o]
 * multiplies input i into output o); the training state keeps a float32
 * master copy and the network reads the BF16 copy.
 * ------------------------------------------------------------------------ */
int32_t ht_mlp_param_count(void);

/* Forward passes that gave up waiting for their tensor-core work (bounded
 * waits; 0 in a healthy run) since the library was loaded; synchronous;
 * -1 on a CUDA error. */
int64_t ht_mlp_timeouts(void);

/* Forward pass of n hits (x, y, z float32, layer uint8 device arrays).
 * Outputs (device, each may be NULL): prob n x 64 float32 (softmax); h1, h2
 * n x 128 BF16 (hidden activations after ReLU); feat n x 8 BF16 (the six
 * features, zero padded).  h1, h2 and feat are what ht_mlp_backward needs.
 * Errors: HT_ERR_ARG, HT_ERR_CUDA. */
ht_status ht_mlp_forward(const void *params_bf16, const float *x, const float *y, const float *z,
                         const uint8_t *layer, int32_t n, float *prob, void *h1, void *h2,
                         void *feat, ht_stream stream);

/* Region masks of n_events events whose hits are concatenated at device
 * offsets off[0..n_events] (n_hits = off[n_events] total).  mass (device,
 * n_events x 64 float32) receives the per-event SUM of the hits' softmax
 * outputs; masks[e] (device) the regions whose mean mass (sum / hits) is
 * >= tau, plus, if grow is 1, the 8 neighbours of each in the region grid;
 * every region (all bits) when more than fmax * 64 are selected or the
 * event is empty.  Sums are float32 atomics, so a mean within about 1e-6 of
 * tau may fall either way.  Errors: HT_ERR_ARG, HT_ERR_CUDA. */
ht_status ht_mlp_region_mask(const void *params_bf16, const float *x, const float *y,
                             const float *z, const uint8_t *layer, const int32_t *off,
                             int32_t n_events, int32_t n_hits, float tau, float fmax,
                             int32_t grow, float *mass, uint64_t *masks, ht_stream stream);

/* Per-hit region sets (the per-hit proposal): hit_masks[h] (device, n_hits
 * uint64) gets the topk regions of largest softmax output of hit h (ties to
 * the smaller region index), or every region (all bits) when topk >= 64 or
 * those topk outputs sum to less than pmin (float32 sum; a sum within about
 * 1e-6 of pmin, or outputs within about 1e-6 of each other, may fall either
 * way).  Feed the result to ht_vote_hit_masked or ht_batch_run_hit_masked.
 * topk >= 1.  Errors: HT_ERR_ARG, HT_ERR_CUDA. */
ht_status ht_mlp_hit_masks(const void *params_bf16, const float *x, const float *y,
                           const float *z, const uint8_t *layer, int32_t n_hits, int32_t topk,
                           float pmin, uint64_t *hit_masks, ht_stream stream);

/* Gradient of the mean softmax cross entropy over the hits with label >= 0
 * (labels: device int32, region index or -1 to skip the hit), given the
 * forward pass's prob, h1, h2 and feat for the same n hits; ADDED into grad
 * (device, ht_mlp_param_count() float32, in the parameter layout).  The
 * BF16 roundings of the forward pass count as identity.  Deterministic: the
 * same inputs give the same bits (partial sums are added in a fixed order),
 * so a training run resumed from a checkpoint repeats an uninterrupted one.
 * workspace: ht_mlp_backward_workspace_size(n) bytes, 256-byte aligned.
 * Errors: HT_ERR_ARG, HT_ERR_CUDA. */
size_t ht_mlp_backward_workspace_size(int32_t n);
ht_status ht_mlp_backward(const void *params_bf16, const int32_t *labels, int32_t n,
                          const float *prob, const void *h1, const void *h2, const void *feat,
                          float *grad, void *workspace, size_t workspace_bytes, ht_stream stream);

/* One Adam step (Kingma and Ba, bias-corrected, step >= 1) on the float32
 * master parameters with moments m and v (device, ht_mlp_param_count()
 * float32 each, updated in place); also writes the BF16 copy.
 * Errors: HT_ERR_ARG, HT_ERR_CUDA. */
ht_status ht_mlp_adam(float *params, float *m, float *v, const float *grad, int32_t step,
                      float lr, float beta1, float beta2, float eps, void *params_bf16,
                      ht_stream stream);

/* ------------------------------------------------------------------------
 * Refinement of candidates (Section 5: costlier computations confirm the
 * candidates; Section 6 names a Kalman filter for it).  Without material or
 * process noise a Kalman filter over a track's hits gives the weighted
 * least-squares estimate, which this call fits directly.  Reading: p =
 * (rho, d0, phi0) starts at the candidate's cell centre (rho_i,
 * (j - n_d0/2) delta, phi0_k); the residual of hit (x, y) is F / 2 with
 * F = rho d0^2 + 2 (1 + rho s) d0 + rho r^2 + 2 s (the signed distance to
 * the circle to first order, equal weights sigma); `iters` Gauss-Newton
 * steps solve (J^T J) dp = -J^T r by Cholesky.  Float64 throughout; the sums
 * run over the hits in no fixed order, so results agree with the float64
 * definition to rounding (~1e-15 relative), not bit for bit.
 * ------------------------------------------------------------------------ */
typedef struct ht_track {
    double rho, d0, phi0;              /* fitted (the start when status 0) */
    double sig_rho, sig_d0, sig_phi0;  /* sqrt of the covariance diagonal */
    float chi2;                        /* sum (residual / sigma)^2 */
    int32_t n_hits;                    /* hits in the last fit */
    int32_t status;   /* 1 fitted, 0 fewer than min_hits hits, -1 normal
                         matrix not positive definite (last good p kept) */
    int32_t reserved;
} ht_track;

/* Fit every candidate of n_events events with at least min_hits (>= 3)
 * assigned hits.  Hits: x, y (device float32) concatenated at DEVICE offsets
 * d_off[0 .. n_events]; n_hits = the total (d_off[n_events]).  assign: per
 * hit, the candidate index within its event (ht_associate / ht_batch_run
 * output, -1 none).  Event e's candidates are peaks[e * cap ..
 * e * cap + min(d_count[e], cap)); its tracks go to out + e * cap.
 * iters, iters2 in [0, 64]; sigma > 0 (cm, the hit resolution).  Hit
 * selection: road > 0 fits only the hits within road (cm) of the cell-centre
 * circle; cut > 0 then refits, with iters2 more steps, the hits within
 * cut * sigma of the fitted circle (road, cut <= 0: off).  n_hits is the
 * number of hits in the last fit; fewer than min_hits gives status 0.
 * workspace: ht_fit_workspace_size(n_events, cap, n_hits) bytes, 256-byte
 * aligned.  Errors: HT_ERR_ARG, HT_ERR_CAPACITY (n_events * cap >= 2^31),
 * HT_ERR_CUDA. */
size_t ht_fit_workspace_size(int32_t n_events, int32_t cap, int32_t n_hits);
ht_status ht_fit_tracks(const ht_geometry *g, const float *x, const float *y, const int32_t *d_off,
                        int32_t n_events, int32_t n_hits, const int32_t *assign,
                        const ht_peak *peaks, const int32_t *d_count, int32_t cap,
                        int32_t min_hits, int32_t iters, double sigma, double road, double cut,
                        int32_t iters2, ht_track *out, void *workspace, size_t workspace_bytes,
                        ht_stream stream);

/* ------------------------------------------------------------------------
 * Second transform: displaced vertices (Section 6, Fig. 6; Section 7).
 * Tracks from one vertex lie on a sinusoid in track-parameter space; a
 * second Hough transform over the candidates finds those sinusoids and the
 * same peak finder locates them; features inside the beam pipe are dropped.
 * Readings: a candidate (i, j, k) is the straight line of its cell centre,
 * d0 = (j - n_d0/2) delta at phi0_k (the curvature is not used); a vertex
 * r (cos theta, sin theta) lies on it iff d0 = r sin(theta - phi0).  Vertex
 * space: theta_q = (2q + 1 - n_theta) pi / n_theta (wrapping) x radius bins
 * of width dr = r_max / n_r from 0.  In every theta column a candidate with
 * count >= min_count votes once, at r = d0 / (sin theta_q cos phi0_k -
 * cos theta_q sin phi0_k), in bin floor(r / dr) if 0 <= r / dr < n_r
 * (float64 definition, products then difference then two divisions; a zero
 * denominator gives no vote).  Peaks: the rule of ht_find_peaks on the
 * 1 x n_r x n_theta array (radius does not wrap, theta does), threshold
 * T2 = threshold.  Beam-pipe filter: peaks whose radius-bin centre
 * (j + 1/2) dr is below r_keep come first in peak order; d_first says
 * where the others start.
 * ------------------------------------------------------------------------ */
typedef struct ht_vertex_desc {
    int32_t n_r, n_theta;   /* n_r in [1, 4096]; n_theta a multiple of 32 */
    int32_t threshold;      /* T2: tracks through a vertex cell, >= 1 */
    int32_t min_count;      /* candidates with fewer votes do not vote */
    double r_max;           /* radius axis [0, r_max), cm */
    double r_keep;          /* beam-pipe radius, cm (Section 7: 3.0) */
} ht_vertex_desc;

typedef struct ht_vertex ht_vertex;   /* opaque; uses g's phi0 and d0 axes */

/* Create on the current device for candidates of geometry g (which must
 * outlive the handle).  Errors: HT_ERR_ARG, HT_ERR_CUDA. */
ht_status ht_vertex_create(const ht_geometry *g, const ht_vertex_desc *desc, ht_vertex **out);
ht_status ht_vertex_destroy(ht_vertex *v);

/* Bytes of one event's vertex accumulator: n_r * n_theta int32. */
size_t ht_vertex_accumulator_bytes(const ht_vertex *v);

/* Vote n_events events at once: event e's candidates are
 * cands[e * cap .. e * cap + min(d_count[e], cap)) (ht_find_peaks or
 * ht_batch_run output); its accumulator is acc + e * n_r * n_theta (device,
 * int32, [radius bin][theta], every cell written).  stats: NULL or
 * 2 * n_events uint64 (votes, float64 redos), zeroed first.
 * Errors: HT_ERR_ARG, HT_ERR_CUDA. */
ht_status ht_vertex_vote(const ht_vertex *v, const ht_peak *cands, const int32_t *d_count,
                         int32_t cap, int32_t n_events, int32_t *acc, uint64_t *stats,
                         ht_stream stream);

/* Peaks of each event's vertex accumulator into out + e * cap ({0, radius
 * bin, theta bin, count}, increasing index, first min(total, cap)), totals
 * in d_count[e] and the index of the first peak outside r_keep in
 * d_first[e].  acc 16-byte aligned; workspace: ht_vertex_workspace_size(v)
 * bytes, 256-byte aligned, reused by the events in stream order.
 * Errors: HT_ERR_ARG, HT_ERR_CUDA. */
size_t ht_vertex_workspace_size(const ht_vertex *v);
ht_status ht_vertex_find(const ht_vertex *v, const int32_t *acc, int32_t n_events,
                         ht_peak *out, int32_t cap, int32_t *d_count, int32_t *d_first,
                         void *workspace, size_t workspace_bytes, ht_stream stream);

/* ------------------------------------------------------------------------
 * Batched runtime: many events, uneven hit counts, one CUDA graph per batch.
 * The paper processes one event at a time (Fig. 5); a batch runs the same
 * four steps with identical results per event, but the vote and association
 * run as persistent kernels over a device queue of (event, tile) items,
 * largest events first, and the whole batch is captured once into a CUDA
 * graph and replayed for every later batch with the same number of events.
 * Requires count_bits 16 and an even n_d0 (two 16-bit counters per word).
 * ------------------------------------------------------------------------ */
typedef struct ht_batch ht_batch;   /* opaque */

/* Create a batch runtime on the current device for up to max_events events,
 * max_hits hits in total and cap candidates per event.  The runtime allocates
 * its scratch once here (one accumulator per event slot, candidate lists,
 * z-vote scratch; about 200 MB per slot for 256x128x512 with cap 2^21) and
 * owns it.  Errors: HT_ERR_ARG, HT_ERR_CUDA. */
ht_status ht_batch_create(const ht_geometry *g, int32_t max_events, int32_t max_hits,
                          int32_t cap, ht_batch **out);
ht_status ht_batch_destroy(ht_batch *b);

/* Enable (default) or disable CUDA-graph capture and replay. */
ht_status ht_batch_set_graphs(ht_batch *b, int32_t enable);

/* Run the path on n_events events whose hits are concatenated in x, y, z
 * (device, float32) at host offsets h_off[0..n_events] (h_off[0] == 0,
 * non-decreasing, h_off[n_events] <= max_hits).  Outputs (device, caller-owned):
 *   peaks   n_events * cap entries; event e's candidates at peaks[e * cap];
 *   counts  n_events int32 (total peaks of each event, may exceed cap);
 *   assign  h_off[n_events] int32, candidate index within the hit's event;
 *   zres    n_events * cap entries, like peaks;
 *   stats   NULL or 2 * n_events uint64 (votes, float64 redos per event).
 * Asynchronous on `stream`; the first call for a given n_events and set of
 * buffer pointers captures the graph.  Errors: HT_ERR_ARG, HT_ERR_CAPACITY,
 * HT_ERR_CUDA. */
ht_status ht_batch_run(ht_batch *b, const float *x, const float *y, const float *z,
                       const int32_t *h_off, int32_t n_events, ht_peak *peaks,
                       int32_t *counts, int32_t *assign, ht_zres *zres, uint64_t *stats,
                       ht_stream stream);

/* ht_batch_run with the vote and peak finding of event e restricted to
 * masks[e] (device, n_events uint64; see ht_vote_masked and
 * ht_find_peaks_masked): event e's candidates are its ht_batch_run
 * candidates inside masks[e], and association and the z vote run on them.
 * Errors: as ht_batch_run. */
ht_status ht_batch_run_masked(ht_batch *b, const float *x, const float *y, const float *z,
                              const int32_t *h_off, int32_t n_events, const uint64_t *masks,
                              ht_peak *peaks, int32_t *counts, int32_t *assign, ht_zres *zres,
                              uint64_t *stats, ht_stream stream);

/* The proposal used by ht_batch_run_learned. */
typedef struct ht_proposal {
    const void *params_bf16;  /* device, ht_mlp_param_count() BF16 values */
    const uint8_t *layer;     /* device, layer index of every hit (like x) */
    float tau;                /* region threshold on the mean softmax mass */
    float fmax;               /* more than fmax * 64 regions: full vote */
    int32_t grow;             /* 1: add the 8 neighbours of each region */
    int32_t reserved;         /* set to 0 */
} ht_proposal;

/* ht_batch_run_masked with the masks computed at the head of the same graph
 * by ht_mlp_region_mask (proposal *prop) and written to masks (device,
 * n_events uint64).  tau, fmax and grow are part of the captured graph: a
 * new value captures a new one.  Errors: as ht_batch_run. */
ht_status ht_batch_run_learned(ht_batch *b, const float *x, const float *y, const float *z,
                               const int32_t *h_off, int32_t n_events, const ht_proposal *prop,
                               uint64_t *masks, ht_peak *peaks, int32_t *counts,
                               int32_t *assign, ht_zres *zres, uint64_t *stats,
                               ht_stream stream);

/* ht_batch_run with the vote of each hit restricted to its region set:
 * hit_masks (device, h_off[n_events] uint64 indexed like x, 8-byte aligned)
 * as in ht_vote_hit_masked.  Peak finding, association and the z vote run
 * as in ht_batch_run on the restricted accumulator.  Errors: as
 * ht_batch_run. */
ht_status ht_batch_run_hit_masked(ht_batch *b, const float *x, const float *y, const float *z,
                                  const int32_t *h_off, int32_t n_events,
                                  const uint64_t *hit_masks, ht_peak *peaks, int32_t *counts,
                                  int32_t *assign, ht_zres *zres, uint64_t *stats,
                                  ht_stream stream);

/* The per-hit proposal used by ht_batch_run_learned_hits. */
typedef struct ht_hit_proposal {
    const void *params_bf16;  /* device, ht_mlp_param_count() BF16 values */
    const uint8_t *layer;     /* device, layer index of every hit (like x) */
    int32_t topk;             /* regions per hit, >= 1 (>= 64: every region) */
    float pmin;               /* top-k output sum below pmin: every region */
} ht_hit_proposal;

/* ht_batch_run_hit_masked with the region sets computed at the head of the
 * same graph by ht_mlp_hit_masks (proposal *prop) and written to hit_masks
 * (device, h_off[n_events] uint64).  topk and pmin are part of the captured
 * graph.  Errors: as ht_batch_run. */
ht_status ht_batch_run_learned_hits(ht_batch *b, const float *x, const float *y, const float *z,
                                    const int32_t *h_off, int32_t n_events,
                                    const ht_hit_proposal *prop, uint64_t *hit_masks,
                                    ht_peak *peaks, int32_t *counts, int32_t *assign,
                                    ht_zres *zres, uint64_t *stats, ht_stream stream);

/* Switch on the batched track path (ht_batch_run_tracks) with confirmation
 * parameters *c (see ht_confirm_desc; the bands give each event's peak
 * threshold from its hit count).  The first call allocates the path's
 * scratch: 64 bytes per candidate slot (max_events * cap) plus per-hit keys.
 * Clears the captured graphs.  Errors: HT_ERR_ARG, HT_ERR_CUDA. */
ht_status ht_batch_set_confirm(ht_batch *b, const ht_confirm_desc *c);

/* The track path on a batch: per event, the distinct-layer vote
 * (ht_vote_layers; with hit_masks each hit's votes restricted to its region
 * set as in ht_vote_hit_masked), peaks at the event's band threshold,
 * confirmation and final assignment (ht_confirm) instead of ht_associate,
 * and the (z0, cot theta) vote of each candidate over its assigned hits.
 * Results per event are those of the single-event calls.
 *   layer      device uint8 per hit (indexed like x), each in [0, 16).
 *   prop       NULL, or a per-hit proposal whose top-k region sets are
 *              computed at the head of the graph into hit_masks.
 *   hit_masks  NULL (no restriction), or device uint64 per hit: given sets
 *              (prop NULL) or the proposal's output (prop set).
 *   score      n_events * cap int32 (device): inlier layers of each
 *              candidate slot, 0 when not confirmed.
 *   peaks, counts, assign, zres, stats   as ht_batch_run; assign holds each
 *              hit's confirmed candidate within its event, -1 none.
 * Requires ht_batch_set_confirm.  Errors: as ht_batch_run. */
ht_status ht_batch_run_tracks(ht_batch *b, const float *x, const float *y, const float *z,
                              const uint8_t *layer, const int32_t *h_off, int32_t n_events,
                              const ht_hit_proposal *prop, uint64_t *hit_masks, ht_peak *peaks,
                              int32_t *counts, int32_t *score, int32_t *assign, ht_zres *zres,
                              uint64_t *stats, ht_stream stream);

/* A found track: a confirmed candidate and its (z0, cot theta) result. */
typedef struct ht_track_out {
    int32_t i_rho, j_d0, k_phi0;   /* the candidate's cell */
    int32_t count;                 /* its distinct-layer count */
    int32_t score;                 /* inlier layers of its confirmation */
    int32_t n_z0, m_cot, zcount;   /* its (z0, cot theta) vote result */
} ht_track_out;

/* ht_batch_run_tracks from HOST buffers, synchronous: copies the hits to
 * the device, runs the track path on `stream`, keeps each event's confirmed
 * candidates (score > 0, in candidate order) as its tracks, copies back only
 * the tracks and the hits' assignments to them, and synchronises the stream
 * before returning.
 *   hx, hy, hz, hlayer   host arrays of h_off[n_events] hits (float32, and
 *                        uint8 layers); pinned memory copies faster.
 *   prop        NULL or a per-hit proposal (as ht_batch_run_tracks); its
 *               params_bf16 is DEVICE memory and its layer field is ignored
 *               (the copied layers are used).
 *   h_tracks    host, track_cap entries: event e's tracks follow those of
 *               events 0 .. e - 1.
 *   h_ntracks   host, n_events int32: each event's number of tracks.
 *   h_assign    host, h_off[n_events] int32: the index of the hit's track
 *               within its event's tracks, -1 for none.
 *   h_stats     host, NULL or 2 * n_events uint64 (as ht_batch_run).
 * The first call allocates the device buffers it needs (hits for max_hits,
 * candidates for max_events * cap).  When all events' tracks exceed
 * track_cap, the first track_cap are copied, h_ntracks still gives every
 * event's total and the call returns HT_ERR_CAPACITY.  Requires
 * ht_batch_set_confirm.  Errors: as ht_batch_run_tracks. */
ht_status ht_batch_run_tracks_host(ht_batch *b, const float *hx, const float *hy,
                                   const float *hz, const uint8_t *hlayer, const int32_t *h_off,
                                   int32_t n_events, const ht_hit_proposal *prop,
                                   ht_track_out *h_tracks, int32_t track_cap,
                                   int32_t *h_ntracks, int32_t *h_assign, uint64_t *h_stats,
                                   ht_stream stream);

/* Device time of the stages of the last completed batch run, in ms: ms[0]
 * proposal (0 without one), ms[1] vote, ms[2] peak finding and candidate
 * lists, ms[3] association, ms[4] assignment decode and (z0, cot theta)
 * vote.  Call after the run's stream has completed.  Errors: HT_ERR_ARG,
 * HT_ERR_CUDA. */
ht_status ht_batch_stage_ms(const ht_batch *b, float *ms);

/* Autotune the tile widths (phi0 columns per tile of the packed and unpacked
 * vote, and of the association) by timing whole batches on the given sample
 * (arguments as ht_batch_run).  *choice = kt_pack | kt_unpacked << 8 |
 * kt_assoc << 16.  The widths apply to ht_batch_run and the masked runs; the
 * track path's distinct-layer vote keeps its own default tile.  Synchronises
 * the stream.  Errors: as ht_batch_run. */
ht_status ht_batch_autotune(ht_batch *b, const float *x, const float *y, const float *z,
                            const int32_t *h_off, int32_t n_events, ht_peak *peaks,
                            int32_t *counts, int32_t *assign, ht_zres *zres, int32_t *choice,
                            ht_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* HT_H */
