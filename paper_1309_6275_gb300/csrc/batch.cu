// batch.cu -- batched runtime (ht_batch_* in include/ht.h).
//
// A batch of events runs as one CUDA graph, captured once per batch shape and
// replayed: persistent vote and association kernels pop (event, tile) items
// from device counters (events ordered largest first, so 2k- and 60k-hit
// events share the GPU without per-event launch tails); peak finding and
// candidate lists run per event slot; the (z0, cot theta) vote runs over all
// candidates of the batch at once.  The vote and association tiles scan
// per-event lists of the hits whose angular window meets their columns
// (k_buckets.cu), built at the head of the vote stage.  Per-batch data (hit
// offsets, event order) lives in device memory, uploaded from pinned staging
// before each replay, so one graph serves every batch with the same number
// of events.  An autotuner times the tile widths on a sample batch.
//
// Masked and learned runs: the vote and the peak finding take a per-event
// region mask (given by the caller, or computed at the head of the same
// graph by the proposal MLP from the hits); association and the z vote run
// unchanged on the masked candidates.  Per-hit runs: the vote takes one
// region set per hit (given, or the proposal MLP's top-k regions of each
// hit); peak finding, association and the z vote run unchanged on the
// restricted accumulator.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "ht_internal.cuh"

namespace ht {
cudaError_t launch_vote_batch(const DevGeom &G, const float *x, const float *y, const int *off,
                              const int *order, const int *d_nev, uint16_t *acc,
                              size_t acc_stride, unsigned long long *stats, int *head, bool pack,
                              int kt, int sms, cudaStream_t st, const HitBuckets *hb);
int assoc32_kt(const DevGeom &G);
int assoc32_ntiles(const DevGeom &G, int kt);
cudaError_t launch_cand_lists(const DevGeom &G, int kt, const ht_peak *peaks, const int *d_count,
                              int cap, int *tcnt, int *toff, int *tcur, void *tmp, int *tlist,
                              cudaStream_t st);
cudaError_t launch_assoc_batch(const DevGeom &G, int kt, const float *x, const float *y,
                               const int *off, const int *order, const int *d_nev,
                               const ht_peak *peaks, int cap, const int *toff, size_t tstride,
                               const int *tlist, size_t lstride, unsigned long long *gbest,
                               int *head, int sms, cudaStream_t st, const HitBuckets *hb);
cudaError_t launch_assoc_final_batch(const unsigned long long *gbest, const int *off,
                                     const int *d_nev, int *assign, int max_hits, cudaStream_t st);
size_t vote_z_batch_workspace_bytes(int n_ev, int cap, int max_hits);
cudaError_t launch_vote_z_batch(const DevGeom &G, const float *x, const float *y, const float *z,
                                const int *assign, const int *off, const int *d_nev,
                                const ht_peak *peaks, const int *counts, int cap, int n_ev,
                                ht_zres *out, void *ws, int max_hits, cudaStream_t st);
cudaError_t prepare_batch_kernels(int max_smem);
cudaError_t launch_vote_batch_masked(const DevGeom &G, const float *x, const float *y,
                                     const int *off, const int *order, const int *d_nev,
                                     uint16_t *acc, size_t acc_stride, unsigned long long *stats,
                                     int *head, bool pack, int kt, int sms,
                                     const unsigned long long *masks, cudaStream_t st,
                                     const HitBuckets *hb);
cudaError_t launch_region_mask(const void *params_bf16, const float *x, const float *y,
                               const float *z, const uint8_t *layer, const int *off, int n_ev,
                               int max_hits, float tau, float fmax, int grow, float *mass,
                               unsigned long long *masks, cudaStream_t st);
cudaError_t launch_vote_batch_hitmask(const DevGeom &G, const float *x, const float *y,
                                      const int *off, const int *order, const int *d_nev,
                                      uint16_t *acc, size_t acc_stride,
                                      unsigned long long *stats, int *head, bool pack, int kt,
                                      int sms, const unsigned long long *hit_masks,
                                      cudaStream_t st, const HitBuckets *hb);
cudaError_t launch_hit_masks(const void *params_bf16, const float *x, const float *y,
                             const float *z, const uint8_t *layer, int n, const int *d_n,
                             int topk, float pmin, unsigned long long *hit_masks, cudaStream_t st);
cudaError_t launch_vote_batch_layers(const DevGeom &G, const float *x, const float *y,
                                     const uint8_t *layer, const int *off, const int *order,
                                     const int *d_nev, uint16_t *acc, size_t acc_stride,
                                     unsigned long long *stats, int *head, int kt, int sms,
                                     const unsigned long long *hit_masks, cudaStream_t st,
                                     const HitBuckets *hb);
}  // namespace ht

namespace {

constexpr int kGraphCache = 16;

constexpr int kStages = 5;   // proposal, vote, peaks + lists, association, z vote

struct GraphEntry {
    int n_ev;
    const void *ptr[14];
    float tau, fmax, pmin;
    int grow, topk;
    cudaGraphExec_t exec;
};

// What restricts the vote of one run (all null: the plain path), and the
// track path (layer set: distinct-layer vote, confirmation instead of the
// association, confirmation scores written to score).
struct Restrict {
    unsigned long long *masks;        // per event
    const ht_proposal *prop;          // writes masks first
    unsigned long long *hit_masks;    // per hit
    const ht_hit_proposal *hprop;     // writes hit_masks first
    const uint8_t *layer;             // per hit: the track path
    int32_t *score;                   // per candidate slot (track path)
};

}  // namespace

struct ht_batch {
    const ht_geometry *g;
    int max_events, max_hits, cap, sms;
    int kt_pack, kt_big, kt_assoc;
    size_t cells;
    uint16_t *acc;
    int *meta;          // [0] n_big [1] pad [2] n_all [3] pad, off[max_events + 1],
                        // order_big[max_events], order_all[max_events] (largest first),
                        // thr[max_events] (peak threshold of each event slot)
    int *h_meta;        // pinned staging, same layout
    size_t meta_ints;
    cudaEvent_t meta_done;
    bool meta_pending;
    int *heads;
    unsigned long long *gbest;
    char *pk_ws;
    size_t pk_stride;
    char *pk_spill;     // one spill buffer: the events' peak launches run in turn
    int ntiles;
    int *tcnt, *toff, *tcur;
    char *ttmp;
    size_t ttmp_stride;
    int *tlist;
    size_t lstride;
    char *z_ws;
    float *mass;        // per-event region masses of the learned proposal
    char *bk_ws;        // per-event hit lists by column group (k_buckets.cu)
    ht::HitBuckets bk;
    ht_confirm_desc conf;   // track path parameters (set by ht_batch_set_confirm)
    bool conf_set;
    int *inl;               // track path: 16 inlier hits per candidate slot
    char *cf_ws;            // track path: confirmation scratch
    struct HostPath {       // buffers of ht_batch_run_tracks_host (allocated on first use)
        float *x, *y, *z;
        uint8_t *layer;
        unsigned long long *hmasks;
        ht_peak *peaks;
        ht_zres *zres;
        int *counts, *score, *assign, *assign_c, *tfirst, *ntot;
        uint64_t *stats;
        ht_track_out *tracks;
        int tcap;
        char *ws;
        int *h_small;       // pinned: tfirst and the total
    } hp;
    GraphEntry cache[kGraphCache];
    int ncache;
    bool use_graph;
    cudaStream_t cap_stream;   // private stream that graphs are captured on
    cudaEvent_t stage[kStages + 1];   // recorded around the stages of every run
};

namespace {

int *off_of(int *meta) { return meta + 4; }
int *order_big_of(int *meta, int me) { return meta + 4 + me + 1; }
int *order_all_of(int *meta, int me) { return meta + 4 + 2 * me + 1; }
int *thr_of(int *meta, int me) { return meta + 4 + 3 * me + 1; }

void free_batch(ht_batch *b)
{
    if (!b) return;
    for (int i = 0; i < b->ncache; ++i) cudaGraphExecDestroy(b->cache[i].exec);
    cudaFree(b->acc);
    cudaFree(b->meta);
    cudaFree(b->heads);
    cudaFree(b->gbest);
    cudaFree(b->pk_ws);
    cudaFree(b->pk_spill);
    cudaFree(b->tcnt);
    cudaFree(b->toff);
    cudaFree(b->tcur);
    cudaFree(b->ttmp);
    cudaFree(b->tlist);
    cudaFree(b->z_ws);
    cudaFree(b->mass);
    cudaFree(b->bk_ws);
    cudaFree(b->inl);
    cudaFree(b->cf_ws);
    {
        ht_batch::HostPath &h = b->hp;
        void *bufs[] = {h.x, h.y, h.z, h.layer, h.hmasks, h.peaks, h.zres, h.counts, h.score,
                        h.assign, h.assign_c, h.tfirst, h.ntot, h.stats, h.tracks, h.ws};
        for (void *q : bufs) cudaFree(q);
        if (h.h_small) cudaFreeHost(h.h_small);
    }
    if (b->h_meta) cudaFreeHost(b->h_meta);
    if (b->meta_done) cudaEventDestroy(b->meta_done);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (int i = 0; i <= kStages; ++i)
        if (b->stage[i]) cudaEventDestroy(b->stage[i]);
    delete b;
}

void clear_graphs(ht_batch *b)
{
    for (int i = 0; i < b->ncache; ++i) cudaGraphExecDestroy(b->cache[i].exec);
    b->ncache = 0;
}

// Every launch of one batch, in order, on stream st.  R.masks: null or one
// region mask per event, written first by the proposal when R.prop is set;
// R.hit_masks: null or one region set per hit, written first by the
// proposal when R.hprop is set.
cudaError_t enqueue(ht_batch *b, const float *x, const float *y, const float *z, int n_ev,
                    ht_peak *peaks, int32_t *counts, int32_t *assign, ht_zres *zres,
                    uint64_t *stats, const Restrict &R, cudaStream_t st, bool capturing)
{
    unsigned long long *masks = R.masks;
    const ht_proposal *prop = R.prop;
    // stage timers: inside a capture they must become graph nodes
    auto mark = [&](int i) {
        return capturing ? cudaEventRecordWithFlags(b->stage[i], st, cudaEventRecordExternal)
                         : cudaEventRecord(b->stage[i], st);
    };
    const ht::DevGeom &G = b->g->G;
    const int me = b->max_events;
    int *meta = b->meta;
    const int *off = off_of(meta);
    unsigned long long *st64 = reinterpret_cast<unsigned long long *>(stats);
    cudaError_t e = cudaMemsetAsync(b->heads, 0, 4 * sizeof(int), st);
    if (e == cudaSuccess && stats) e = cudaMemsetAsync(stats, 0, (size_t)n_ev * 16, st);
    if (e == cudaSuccess) e = mark(0);
    if (e != cudaSuccess) return e;
    if (prop) {
        e = ht::launch_region_mask(prop->params_bf16, x, y, z, prop->layer, off, n_ev,
                                   b->max_hits, prop->tau, prop->fmax, prop->grow, b->mass, masks,
                                   st);
        if (e != cudaSuccess) return e;
    }
    if (R.hprop) {
        e = ht::launch_hit_masks(R.hprop->params_bf16, x, y, z, R.hprop->layer, b->max_hits,
                                 off + n_ev, R.hprop->topk, R.hprop->pmin, R.hit_masks, st);
        if (e != cudaSuccess) return e;
    }
    e = mark(1);
    if (e != cudaSuccess) return e;
    // the hits each tile scans: lists by column group (every tile width the
    // batch uses divides the group)
    e = ht::launch_hit_buckets(G, x, y, off, meta + 2, b->max_hits, b->bk, b->sms, st);
    if (e != cudaSuccess) return e;
    // vote: the tiles whose hit lists pass the packed-counter limit (only
    // events above it can have such tiles), then every other tile of every
    // event with packed counters
    auto vote = [&](const int *order, const int *d_nev, int *head, bool pack, int kt) {
        if (R.hit_masks)
            return ht::launch_vote_batch_hitmask(G, x, y, off, order, d_nev, b->acc, b->cells,
                                                 st64, head, pack, kt, b->sms, R.hit_masks, st,
                                                 &b->bk);
        return masks ? ht::launch_vote_batch_masked(G, x, y, off, order, d_nev, b->acc, b->cells,
                                                    st64, head, pack, kt, b->sms, masks, st,
                                                    &b->bk)
                     : ht::launch_vote_batch(G, x, y, off, order, d_nev, b->acc, b->cells, st64,
                                             head, pack, kt, b->sms, st, &b->bk);
    };
    const bool tracks = R.layer != nullptr;
    if (tracks) {
        // the distinct-layer vote packs every tile: one launch, always with its
        // default tile (the widths ht_batch_autotune tunes are the plain path's)
        e = ht::launch_vote_batch_layers(G, x, y, R.layer, off, order_all_of(meta, me), meta + 2,
                                         b->acc, b->cells, st64, b->heads + 1, 0, b->sms,
                                         R.hit_masks, st, &b->bk);
    } else {
        e = vote(order_big_of(meta, me), meta + 0, b->heads + 0, false, b->kt_big);
        if (e == cudaSuccess) e = vote(order_all_of(meta, me), meta + 2, b->heads + 1, true, b->kt_pack);
    }
    if (e == cudaSuccess) e = mark(2);
    if (e != cudaSuccess) return e;
    // peaks (each event slot at its staged threshold on the track path) and
    // the association's candidate tile lists per event slot
    for (int ev = 0; ev < n_ev; ++ev) {
        e = ht::launch_peaks(G, b->acc + (size_t)ev * b->cells, peaks + (size_t)ev * b->cap,
                             b->cap, counts + ev, b->pk_ws + (size_t)ev * b->pk_stride, st,
                             masks ? masks + ev : nullptr, tracks ? thr_of(meta, me) + ev : nullptr,
                             b->pk_spill);
        if (e != cudaSuccess) return e;
        if (tracks) continue;
        const size_t to = (size_t)ev * (b->ntiles + 1);
        e = ht::launch_cand_lists(G, b->kt_assoc, peaks + (size_t)ev * b->cap, counts + ev,
                                  b->cap, b->tcnt + to, b->toff + to, b->tcur + to,
                                  b->ttmp + (size_t)ev * b->ttmp_stride,
                                  b->tlist + (size_t)ev * b->lstride, st);
        if (e != cudaSuccess) return e;
    }
    if (tracks) {
        // confirmation and final assignment over the whole batch
        e = mark(3);
        const ht::ConfirmDev P{b->conf.pool, b->conf.min_layers, b->conf.n_layers, b->conf.tol};
        if (e == cudaSuccess)
            e = ht::launch_confirm_batch(G, P, x, y, R.layer, off, meta + 2, b->max_events,
                                         b->max_hits, peaks, counts, b->cap, R.score, b->inl,
                                         assign, b->cf_ws, b->sms, st, &b->bk);
        if (e == cudaSuccess) e = mark(4);
        if (e == cudaSuccess)
            e = ht::launch_vote_z_batch(G, x, y, z, assign, off, meta + 2, peaks, counts, b->cap,
                                        n_ev, zres, b->z_ws, b->max_hits, st);
        if (e == cudaSuccess) e = mark(5);
        return e;
    }
    // association over the whole batch
    e = cudaMemsetAsync(b->gbest, 0, (size_t)b->max_hits * 8, st);
    if (e == cudaSuccess) e = mark(3);
    if (e != cudaSuccess) return e;
    e = ht::launch_assoc_batch(G, b->kt_assoc, x, y, off, order_all_of(meta, me), meta + 2, peaks,
                               b->cap, b->toff, (size_t)b->ntiles + 1, b->tlist, b->lstride,
                               b->gbest, b->heads + 2, b->sms, st, &b->bk);
    if (e == cudaSuccess) e = mark(4);
    if (e != cudaSuccess) return e;
    e = ht::launch_assoc_final_batch(b->gbest, off, meta + 2, assign, b->max_hits, st);
    if (e != cudaSuccess) return e;
    e = ht::launch_vote_z_batch(G, x, y, z, assign, off, meta + 2, peaks, counts, b->cap, n_ev,
                                zres, b->z_ws, b->max_hits, st);
    if (e == cudaSuccess) e = mark(5);
    return e;
}

// Upload offsets and the largest-first event orders for this batch.
ht_status stage_meta(ht_batch *b, const int32_t *h_off, int n_ev, cudaStream_t st)
{
    if (b->meta_pending) {
        cudaError_t e = cudaEventSynchronize(b->meta_done);
        if (e != cudaSuccess) return ht::set_error(HT_ERR_CUDA, "ht_batch_run: staging wait");
        b->meta_pending = false;
    }
    const int me = b->max_events;
    int *hm = b->h_meta;
    memset(hm, 0, b->meta_ints * sizeof(int));
    std::vector<int> idx(n_ev);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) {
        return h_off[a + 1] - h_off[a] > h_off[c + 1] - h_off[c];
    });
    int nb = 0;
    for (int i = 0; i < n_ev; ++i) {
        const int ev = idx[i];
        if (h_off[ev + 1] - h_off[ev] > ht::kPackMaxHits) order_big_of(hm, me)[nb++] = ev;
        order_all_of(hm, me)[i] = ev;
    }
    hm[0] = nb;
    hm[2] = n_ev;
    // peak threshold of each event slot (track path): the first band holding
    // the event's hit count, else the geometry's threshold
    for (int ev = 0; ev < n_ev; ++ev) {
        const int nh = h_off[ev + 1] - h_off[ev];
        int t = b->g->desc.threshold;
        for (int q = 0; b->conf_set && q < b->conf.n_bands; ++q)
            if (nh <= b->conf.band_max_hits[q]) {
                t = b->conf.band_threshold[q];
                break;
            }
        thr_of(hm, me)[ev] = t;
    }
    for (int i = 0; i <= n_ev; ++i) off_of(hm)[i] = h_off[i];
    for (int i = n_ev + 1; i <= me; ++i) off_of(hm)[i] = h_off[n_ev];
    cudaError_t e = cudaMemcpyAsync(b->meta, hm, b->meta_ints * sizeof(int), cudaMemcpyHostToDevice,
                                    st);
    if (e == cudaSuccess) e = cudaEventRecord(b->meta_done, st);
    if (e != cudaSuccess) return ht::set_error(HT_ERR_CUDA, "ht_batch_run: staging upload");
    b->meta_pending = true;
    return HT_OK;
}

ht_status check_offsets(const ht_batch *b, const int32_t *h_off, int n_ev)
{
    if (!h_off || h_off[0] != 0)
        return ht::set_error(HT_ERR_ARG, "ht_batch: h_off must start at 0");
    for (int i = 0; i < n_ev; ++i)
        if (h_off[i + 1] < h_off[i])
            return ht::set_error(HT_ERR_ARG, "ht_batch: h_off must be non-decreasing");
    if (h_off[n_ev] > b->max_hits)
        return ht::set_error(HT_ERR_CAPACITY, "ht_batch: more hits than max_hits");
    return HT_OK;
}

}  // namespace

extern "C" {

ht_status ht_batch_create(const ht_geometry *g, int32_t max_events, int32_t max_hits, int32_t cap,
                          ht_batch **out)
{
    if (!g || !out) return ht::set_error(HT_ERR_ARG, "ht_batch_create: null argument");
    *out = nullptr;
    if (g->desc.count_bits != 16)
        return ht::set_error(HT_ERR_ARG, "ht_batch_create: batches need count_bits 16");
    if (max_events < 1 || max_events > 4096 || max_hits < 1 || cap < 1 ||
        (int64_t)max_events * cap > (int64_t)1 << 30)
        return ht::set_error(HT_ERR_ARG, "ht_batch_create: sizes out of range");
    if (g->desc.n_d0 % 2 != 0)
        return ht::set_error(HT_ERR_ARG, "ht_batch_create: batches need an even n_d0");
    ht_batch *b = new (std::nothrow) ht_batch();
    if (!b) return ht::set_error(HT_ERR_ARG, "ht_batch_create: out of host memory");
    b->g = g;
    b->max_events = max_events;
    b->max_hits = max_hits;
    b->cap = cap;
    b->use_graph = true;
    const ht::DevGeom &G = g->G;
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = ht::prepare_batch_kernels(max_smem);
    b->kt_pack = 0;
    b->kt_big = 0;
    b->kt_assoc = ht::assoc32_kt(G);
    b->cells = (size_t)G.n_rho * G.n_d0 * G.n_phi0;
    b->meta_ints = 4 + (size_t)max_events + 1 + 3 * (size_t)max_events;
    b->pk_stride = ht::align256(ht::peaks_workspace_bytes(G));
    b->ntiles = ht::assoc32_ntiles(G, 1);   // the most tiles any tile width gives
    b->ttmp_stride = ht::scan_tmp_bytes(b->ntiles);
    b->lstride = (size_t)6 * cap;     // a candidate's box touches at most 6 tiles
    const size_t tl = (size_t)max_events * (b->ntiles + 1) * 4;
    auto M = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    M((void **)&b->acc, b->cells * 2 * max_events);
    M((void **)&b->meta, b->meta_ints * 4);
    M((void **)&b->heads, 256);
    M((void **)&b->gbest, (size_t)max_hits * 8);
    M((void **)&b->pk_ws, b->pk_stride * max_events);
    M((void **)&b->pk_spill, ht::peak_spill_bytes(G));
    M((void **)&b->tcnt, tl);
    M((void **)&b->toff, tl);
    M((void **)&b->tcur, tl);
    M((void **)&b->ttmp, b->ttmp_stride * max_events);
    M((void **)&b->tlist, b->lstride * sizeof(int) * max_events);
    M((void **)&b->z_ws, ht::vote_z_batch_workspace_bytes(max_events, cap, max_hits));
    M((void **)&b->mass, (size_t)max_events * 64 * sizeof(float));
    M((void **)&b->bk_ws, ht::hit_bucket_bytes(G, max_events, max_hits));
    if (e == cudaSuccess) b->bk = ht::carve_hit_buckets(G, max_events, max_hits, b->bk_ws);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_meta, b->meta_ints * 4);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->meta_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    for (int i = 0; i <= kStages && e == cudaSuccess; ++i) e = cudaEventCreate(&b->stage[i]);
    if (e != cudaSuccess) {
        free_batch(b);
        return ht::set_error(HT_ERR_CUDA, "ht_batch_create: allocation or set-up failed");
    }
    *out = b;
    return HT_OK;
}

ht_status ht_batch_destroy(ht_batch *b)
{
    if (b && b->meta_pending) cudaEventSynchronize(b->meta_done);
    free_batch(b);
    return HT_OK;
}

ht_status ht_batch_set_graphs(ht_batch *b, int32_t enable)
{
    if (!b) return ht::set_error(HT_ERR_ARG, "ht_batch_set_graphs: null batch");
    b->use_graph = enable != 0;
    return HT_OK;
}

}  // extern "C"

namespace {

ht_status run_impl(ht_batch *b, const float *x, const float *y, const float *z,
                   const int32_t *h_off, int32_t n_events, const Restrict &R, ht_peak *peaks,
                   int32_t *counts, int32_t *assign, ht_zres *zres, uint64_t *stats,
                   ht_stream stream)
{
    if (!b || !x || !y || !z || !peaks || !counts || !assign || !zres)
        return ht::set_error(HT_ERR_ARG, "ht_batch_run: null argument");
    if (n_events < 1 || n_events > b->max_events)
        return ht::set_error(HT_ERR_ARG, "ht_batch_run: n_events out of range");
    const ht_proposal *prop = R.prop;
    if (prop && (!prop->params_bf16 || !prop->layer || !R.masks))
        return ht::set_error(HT_ERR_ARG, "ht_batch_run_learned: null proposal argument");
    if (R.hprop && (!R.hprop->params_bf16 || !R.hprop->layer || !R.hit_masks ||
                    R.hprop->topk < 1))
        return ht::set_error(HT_ERR_ARG, "ht_batch_run_learned_hits: bad proposal argument");
    if (R.hit_masks && (reinterpret_cast<uintptr_t>(R.hit_masks) & 7u))
        return ht::set_error(HT_ERR_ARG, "ht_batch_run_hit_masked: hit_masks not 8-byte aligned");
    if (R.layer && (!R.score || !b->conf_set))
        return ht::set_error(HT_ERR_ARG,
                             "ht_batch_run_tracks: null score, or ht_batch_set_confirm not called");
    ht_status s = check_offsets(b, h_off, n_events);
    if (s != HT_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    s = stage_meta(b, h_off, n_events, st);
    if (s != HT_OK) return s;
    if (!b->use_graph) {
        cudaError_t e = enqueue(b, x, y, z, n_events, peaks, counts, assign, zres, stats, R, st,
                                false);
        return e == cudaSuccess ? HT_OK : ht::set_error(HT_ERR_CUDA, cudaGetErrorString(e));
    }
    const void *params = prop ? prop->params_bf16 : R.hprop ? R.hprop->params_bf16 : nullptr;
    const void *layer = prop ? (const void *)prop->layer
                             : R.hprop ? (const void *)R.hprop->layer : nullptr;
    const void *key[14] = {x,     y,     z,       peaks,  counts, assign,      zres,
                           stats, R.masks, params, layer, R.hit_masks, R.layer, R.score};
    const float tau = prop ? prop->tau : 0.f, fmax = prop ? prop->fmax : 0.f;
    const int grow = prop ? prop->grow : 0;
    const int topk = R.hprop ? R.hprop->topk : 0;
    const float pmin = R.hprop ? R.hprop->pmin : 0.f;
    for (int i = 0; i < b->ncache; ++i) {
        GraphEntry &c = b->cache[i];
        if (c.n_ev == n_events && memcmp(c.ptr, key, sizeof key) == 0 && c.tau == tau &&
            c.fmax == fmax && c.grow == grow && c.topk == topk && c.pmin == pmin) {
            cudaError_t e = cudaGraphLaunch(c.exec, st);
            return e == cudaSuccess ? HT_OK : ht::set_error(HT_ERR_CUDA, cudaGetErrorString(e));
        }
    }
    // capture on the private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is launched on the caller's
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t eq = enqueue(b, x, y, z, n_events, peaks, counts, assign, zres, stats,
                                       R, b->cap_stream, true);
        e = cudaStreamEndCapture(b->cap_stream, &graph);
        if (eq != cudaSuccess) e = eq;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return ht::set_error(HT_ERR_CUDA, cudaGetErrorString(e));
    if (b->ncache == kGraphCache) {
        cudaGraphExecDestroy(b->cache[0].exec);
        memmove(&b->cache[0], &b->cache[1], sizeof(GraphEntry) * (kGraphCache - 1));
        --b->ncache;
    }
    GraphEntry &c = b->cache[b->ncache++];
    c.n_ev = n_events;
    memcpy(c.ptr, key, sizeof key);
    c.tau = tau;
    c.fmax = fmax;
    c.grow = grow;
    c.topk = topk;
    c.pmin = pmin;
    c.exec = exec;
    e = cudaGraphLaunch(exec, st);
    return e == cudaSuccess ? HT_OK : ht::set_error(HT_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace

extern "C" {

ht_status ht_batch_run(ht_batch *b, const float *x, const float *y, const float *z,
                       const int32_t *h_off, int32_t n_events, ht_peak *peaks, int32_t *counts,
                       int32_t *assign, ht_zres *zres, uint64_t *stats, ht_stream stream)
{
    return run_impl(b, x, y, z, h_off, n_events, Restrict{}, peaks, counts, assign, zres, stats,
                    stream);
}

ht_status ht_batch_run_masked(ht_batch *b, const float *x, const float *y, const float *z,
                              const int32_t *h_off, int32_t n_events, const uint64_t *masks,
                              ht_peak *peaks, int32_t *counts, int32_t *assign, ht_zres *zres,
                              uint64_t *stats, ht_stream stream)
{
    if (!masks) return ht::set_error(HT_ERR_ARG, "ht_batch_run_masked: null masks");
    Restrict R{};
    R.masks = reinterpret_cast<unsigned long long *>(const_cast<uint64_t *>(masks));
    return run_impl(b, x, y, z, h_off, n_events, R, peaks, counts, assign, zres, stats, stream);
}

ht_status ht_batch_run_learned(ht_batch *b, const float *x, const float *y, const float *z,
                               const int32_t *h_off, int32_t n_events, const ht_proposal *prop,
                               uint64_t *masks, ht_peak *peaks, int32_t *counts, int32_t *assign,
                               ht_zres *zres, uint64_t *stats, ht_stream stream)
{
    if (!prop) return ht::set_error(HT_ERR_ARG, "ht_batch_run_learned: null proposal");
    Restrict R{};
    R.masks = reinterpret_cast<unsigned long long *>(masks);
    R.prop = prop;
    return run_impl(b, x, y, z, h_off, n_events, R, peaks, counts, assign, zres, stats, stream);
}

ht_status ht_batch_run_hit_masked(ht_batch *b, const float *x, const float *y, const float *z,
                                  const int32_t *h_off, int32_t n_events,
                                  const uint64_t *hit_masks, ht_peak *peaks, int32_t *counts,
                                  int32_t *assign, ht_zres *zres, uint64_t *stats,
                                  ht_stream stream)
{
    if (!hit_masks) return ht::set_error(HT_ERR_ARG, "ht_batch_run_hit_masked: null hit_masks");
    Restrict R{};
    R.hit_masks = reinterpret_cast<unsigned long long *>(const_cast<uint64_t *>(hit_masks));
    return run_impl(b, x, y, z, h_off, n_events, R, peaks, counts, assign, zres, stats, stream);
}

ht_status ht_batch_run_learned_hits(ht_batch *b, const float *x, const float *y, const float *z,
                                    const int32_t *h_off, int32_t n_events,
                                    const ht_hit_proposal *prop, uint64_t *hit_masks,
                                    ht_peak *peaks, int32_t *counts, int32_t *assign,
                                    ht_zres *zres, uint64_t *stats, ht_stream stream)
{
    if (!prop) return ht::set_error(HT_ERR_ARG, "ht_batch_run_learned_hits: null proposal");
    Restrict R{};
    R.hit_masks = reinterpret_cast<unsigned long long *>(hit_masks);
    R.hprop = prop;
    return run_impl(b, x, y, z, h_off, n_events, R, peaks, counts, assign, zres, stats, stream);
}

ht_status ht_batch_set_confirm(ht_batch *b, const ht_confirm_desc *c)
{
    if (!b || !c) return ht::set_error(HT_ERR_ARG, "ht_batch_set_confirm: null argument");
    if (c->pool < 0 || c->min_layers < 1 || c->n_layers < 1 || c->n_layers > 16 ||
        !(c->tol > 0.0) || c->n_bands < 0 || c->n_bands > 8)
        return ht::set_error(HT_ERR_ARG, "ht_batch_set_confirm: parameters out of range");
    for (int q = 0; q < c->n_bands; ++q)
        if (c->band_threshold[q] < 1)
            return ht::set_error(HT_ERR_ARG, "ht_batch_set_confirm: band threshold below 1");
    if (b->meta_pending) {
        if (cudaEventSynchronize(b->meta_done) != cudaSuccess)
            return ht::set_error(HT_ERR_CUDA, "ht_batch_set_confirm: staging wait");
        b->meta_pending = false;
    }
    if (!b->inl) {
        cudaError_t e = cudaMalloc((void **)&b->inl, (size_t)b->max_events * b->cap * 16 * 4);
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&b->cf_ws,
                           ht::confirm_workspace_bytes(b->g->G, b->max_events, b->max_hits, b->cap));
        if (e != cudaSuccess) {
            cudaFree(b->inl);
            b->inl = nullptr;
            return ht::set_error(HT_ERR_CUDA, "ht_batch_set_confirm: allocation failed");
        }
    }
    b->conf = *c;
    b->conf_set = true;
    clear_graphs(b);   // the parameters are part of every captured track graph
    return HT_OK;
}

ht_status ht_batch_run_tracks(ht_batch *b, const float *x, const float *y, const float *z,
                              const uint8_t *layer, const int32_t *h_off, int32_t n_events,
                              const ht_hit_proposal *prop, uint64_t *hit_masks, ht_peak *peaks,
                              int32_t *counts, int32_t *score, int32_t *assign, ht_zres *zres,
                              uint64_t *stats, ht_stream stream)
{
    if (!b || !layer) return ht::set_error(HT_ERR_ARG, "ht_batch_run_tracks: null argument");
    if (prop && !hit_masks)
        return ht::set_error(HT_ERR_ARG, "ht_batch_run_tracks: a proposal needs hit_masks");
    Restrict R{};
    R.hit_masks = reinterpret_cast<unsigned long long *>(hit_masks);
    R.hprop = prop;
    R.layer = layer;
    R.score = score;
    return run_impl(b, x, y, z, h_off, n_events, R, peaks, counts, assign, zres, stats, stream);
}

ht_status ht_batch_run_tracks_host(ht_batch *b, const float *hx, const float *hy,
                                   const float *hz, const uint8_t *hlayer, const int32_t *h_off,
                                   int32_t n_events, const ht_hit_proposal *prop,
                                   ht_track_out *h_tracks, int32_t track_cap,
                                   int32_t *h_ntracks, int32_t *h_assign, uint64_t *h_stats,
                                   ht_stream stream)
{
    if (!b || !hx || !hy || !hz || !hlayer || !h_ntracks || !h_assign ||
        (track_cap > 0 && !h_tracks) || track_cap < 0)
        return ht::set_error(HT_ERR_ARG, "ht_batch_run_tracks_host: null argument");
    if (!b->conf_set)
        return ht::set_error(HT_ERR_ARG, "ht_batch_run_tracks_host: ht_batch_set_confirm not called");
    if (n_events < 1 || n_events > b->max_events)
        return ht::set_error(HT_ERR_ARG, "ht_batch_run_tracks_host: n_events out of range");
    ht_status s = check_offsets(b, h_off, n_events);
    if (s != HT_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    ht_batch::HostPath &h = b->hp;
    const size_t ne = (size_t)b->max_events, mh = (size_t)b->max_hits, nc = ne * b->cap;
    if (!h.x) {
        h.tcap = (int)std::min<size_t>(nc, ne * 16384);
        cudaError_t e = cudaSuccess;
        auto M = [&](void **q, size_t bytes) {
            if (e == cudaSuccess) e = cudaMalloc(q, bytes);
        };
        M((void **)&h.x, mh * 4);
        M((void **)&h.y, mh * 4);
        M((void **)&h.z, mh * 4);
        M((void **)&h.layer, mh);
        M((void **)&h.hmasks, mh * 8);
        M((void **)&h.peaks, nc * sizeof(ht_peak));
        M((void **)&h.zres, nc * sizeof(ht_zres));
        M((void **)&h.counts, ne * 4);
        M((void **)&h.score, nc * 4);
        M((void **)&h.assign, mh * 4);
        M((void **)&h.assign_c, mh * 4);
        M((void **)&h.tfirst, (ne + 1) * 4);
        M((void **)&h.ntot, 16);
        M((void **)&h.stats, ne * 16);
        M((void **)&h.tracks, (size_t)h.tcap * sizeof(ht_track_out));
        M((void **)&h.ws, ht::track_compact_bytes(b->max_events, b->cap));
        if (e == cudaSuccess) e = cudaMallocHost((void **)&h.h_small, (ne + 2) * 4);
        if (e != cudaSuccess) {
            void *bufs[] = {h.x, h.y, h.z, h.layer, h.hmasks, h.peaks, h.zres, h.counts,
                            h.score, h.assign, h.assign_c, h.tfirst, h.ntot, h.stats, h.tracks,
                            h.ws};
            for (void *q : bufs) cudaFree(q);
            if (h.h_small) cudaFreeHost(h.h_small);
            h = ht_batch::HostPath{};
            return ht::set_error(HT_ERR_CUDA, "ht_batch_run_tracks_host: allocation failed");
        }
    }
    const size_t n = (size_t)h_off[n_events];
    cudaError_t e = cudaSuccess;
    if (n > 0) {
        e = cudaMemcpyAsync(h.x, hx, n * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.y, hy, n * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.z, hz, n * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.layer, hlayer, n, cudaMemcpyHostToDevice, st);
    }
    if (e != cudaSuccess) return ht::set_error(HT_ERR_CUDA, "ht_batch_run_tracks_host: copy in");
    ht_hit_proposal pcopy{};
    Restrict R{};
    R.layer = h.layer;
    R.score = h.score;
    if (prop) {
        pcopy = *prop;
        pcopy.layer = h.layer;
        R.hprop = &pcopy;
        R.hit_masks = h.hmasks;
    }
    s = run_impl(b, h.x, h.y, h.z, h_off, n_events, R, h.peaks, h.counts, h.assign, h.zres,
                 h_stats ? h.stats : nullptr, stream);
    if (s != HT_OK) return s;
    e = ht::launch_track_compact(off_of(b->meta), b->meta + 2, b->max_events, b->max_hits,
                                 h.peaks, h.counts, b->cap, h.score, h.zres, h.assign, h.tracks,
                                 h.tcap, h.tfirst, h.ntot, h.assign_c, h.ws, b->sms, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.h_small, h.tfirst, (size_t)(n_events + 1) * 4,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ht::set_error(HT_ERR_CUDA, cudaGetErrorString(e));
    const int total = h.h_small[n_events];
    for (int ev = 0; ev < n_events; ++ev) h_ntracks[ev] = h.h_small[ev + 1] - h.h_small[ev];
    const int ncopy = std::min(total, std::min(track_cap, h.tcap));
    if (ncopy > 0)
        e = cudaMemcpyAsync(h_tracks, h.tracks, (size_t)ncopy * sizeof(ht_track_out),
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(h_assign, h.assign_c, n * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && h_stats)
        e = cudaMemcpyAsync(h_stats, h.stats, (size_t)n_events * 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ht::set_error(HT_ERR_CUDA, cudaGetErrorString(e));
    if (total > track_cap || total > h.tcap)
        return ht::set_error(HT_ERR_CAPACITY, "ht_batch_run_tracks_host: more tracks than track_cap");
    return HT_OK;
}

ht_status ht_batch_stage_ms(const ht_batch *b, float *ms)
{
    if (!b || !ms) return ht::set_error(HT_ERR_ARG, "ht_batch_stage_ms: null argument");
    for (int i = 0; i < kStages; ++i) {
        cudaError_t e = cudaEventElapsedTime(&ms[i], b->stage[i], b->stage[i + 1]);
        if (e != cudaSuccess) return ht::set_error(HT_ERR_CUDA, cudaGetErrorString(e));
    }
    return HT_OK;
}

ht_status ht_batch_autotune(ht_batch *b, const float *x, const float *y, const float *z,
                            const int32_t *h_off, int32_t n_events, ht_peak *peaks,
                            int32_t *counts, int32_t *assign, ht_zres *zres, int32_t *choice,
                            ht_stream stream)
{
    if (!b || !choice) return ht::set_error(HT_ERR_ARG, "ht_batch_autotune: null argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const ht::DevGeom &G = b->g->G;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    const bool graphs = b->use_graph;
    b->use_graph = false;
    auto time_run = [&](float &ms) -> ht_status {
        ht_status s = ht_batch_run(b, x, y, z, h_off, n_events, peaks, counts, assign, zres,
                                   nullptr, stream);
        if (s != HT_OK) return s;
        cudaEventRecord(t0, st);
        s = ht_batch_run(b, x, y, z, h_off, n_events, peaks, counts, assign, zres, nullptr,
                         stream);
        if (s != HT_OK) return s;
        cudaEventRecord(t1, st);
        if (cudaEventSynchronize(t1) != cudaSuccess)
            return ht::set_error(HT_ERR_CUDA, "ht_batch_autotune: timing");
        cudaEventElapsedTime(&ms, t0, t1);
        return HT_OK;
    };
    const int packs[3] = {4, 2, 1}, bigs[3] = {8, 4, 2}, assocs[3] = {4, 2, 1};
    int best_pack = 0, best_big = 0, best_assoc = ht::assoc32_kt(G);
    float best = 3.0e38f, ms = 0.f;
    ht_status s = HT_OK;
    const int assoc_default = ht::assoc32_kt(G);
    for (int ip = 0; ip < 3 && s == HT_OK; ++ip) {
        b->kt_pack = packs[ip];
        b->kt_big = bigs[ip];
        b->kt_assoc = assoc_default;
        s = time_run(ms);
        if (s == HT_OK && ms < best) { best = ms; best_pack = packs[ip]; best_big = bigs[ip]; }
    }
    b->kt_pack = best_pack;
    b->kt_big = best_big;
    best = 3.0e38f;
    for (int ia = 0; ia < 3 && s == HT_OK; ++ia) {
        if (assocs[ia] > assoc_default) continue;   // wider tiles do not fit three CTAs per SM
        b->kt_assoc = assocs[ia];
        s = time_run(ms);
        if (s == HT_OK && ms < best) { best = ms; best_assoc = assocs[ia]; }
    }
    b->kt_assoc = best_assoc;
    b->use_graph = graphs;
    clear_graphs(b);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (s != HT_OK) return s;
    *choice = b->kt_pack | (b->kt_big << 8) | (b->kt_assoc << 16);
    return HT_OK;
}

}  // extern "C"
