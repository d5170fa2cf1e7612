// k_vote_layers.cu -- the distinct-layer Hough vote: the tile kernels of
// tiles.cuh with the kModeLayers flag, in their own translation unit so that
// they compile in parallel with the others.
//
// Each hit casts exactly the votes of the plain vote (Section 5 of
// arXiv:1309.6275); a cell then counts the distinct detector layers among
// the hits voting in it, since a track leaves at most one hit per layer and
// the peak finder is tuned for tracks of at least seven hits (Section 7).
// The tile keeps a 16-bit layer mask per cell (two per shared word, set by
// atomicOr) and writes its population count.  With per-hit region sets
// (the learned proposal's per-hit mode) each hit's votes count only in the
// halo cells of its own regions, as in the plain per-hit vote.
#include "tiles.cuh"

namespace ht {

cudaError_t launch_vote_layers(const DevGeom &G, const float *x, const float *y,
                               const uint8_t *layer, int n, void *acc,
                               unsigned long long *stats, cudaStream_t st)
{
    return launch_vote_t<kModePlain | kModeLayers>(G, x, y, n, acc, stats, nullptr, st, layer);
}

cudaError_t launch_vote_batch_layers(const DevGeom &G, const float *x, const float *y,
                                     const uint8_t *layer, const int *off, const int *order,
                                     const int *d_nev, uint16_t *acc, size_t acc_stride,
                                     unsigned long long *stats, int *head, int kt, int sms,
                                     const unsigned long long *hit_masks, cudaStream_t st,
                                     const HitBuckets *hb)
{
    if (hit_masks)
        return launch_vote_batch_t<kModeHit | kModeLayers>(G, x, y, off, order, d_nev, acc,
                                                           acc_stride, stats, head, true, kt,
                                                           sms, hit_masks, st, bucket_view(hb),
                                                           layer);
    return launch_vote_batch_t<kModePlain | kModeLayers>(G, x, y, off, order, d_nev, acc,
                                                         acc_stride, stats, head, true, kt, sms,
                                                         nullptr, st, bucket_view(hb), layer);
}

cudaError_t prepare_layer_vote_kernels(int max_smem)
{
    const cudaError_t e = prepare_vote_kernels_t<kModePlain | kModeLayers>(max_smem);
    return e == cudaSuccess ? prepare_vote_kernels_t<kModeHit | kModeLayers>(max_smem) : e;
}

}  // namespace ht
