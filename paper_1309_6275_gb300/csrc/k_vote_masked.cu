// k_vote_masked.cu -- the Hough vote (Section 5 of arXiv:1309.6275)
// restricted to a learned proposal's regions: the tile kernels of tiles.cuh
// in their per-event (kModeEvent) and per-hit (kModeHit) mask modes, in their
// own translation unit so that they compile in parallel with the plain ones.
//
// Per event: a tile with no halo cell of the mask is skipped (nothing is
// written); in the other tiles phase 1 drops the (hit, column) pairs whose
// circle cannot reach a halo d0 window within the rho span of the tile's
// allowed rows, and the write-back keeps only halo cells.  Every vote that
// lands in a halo cell is still cast, so halo cells hold exactly the plain
// vote's counts.
//
// Per hit: phase 1 drops the hits with no region near the tile's rows and
// the (hit, column) pairs whose circle cannot reach the hit's d0 window; each
// remaining vote counts only in a halo cell of its hit's regions.  Every
// cell is written.
#include "tiles.cuh"

namespace ht {

cudaError_t launch_vote_masked(const DevGeom &G, const float *x, const float *y, int n,
                               void *acc, unsigned long long *stats,
                               const unsigned long long *mask, cudaStream_t st)
{
    return launch_vote_t<kModeEvent>(G, x, y, n, acc, stats, mask, st);
}

cudaError_t launch_vote_batch_masked(const DevGeom &G, const float *x, const float *y,
                                     const int *off, const int *order, const int *d_nev,
                                     uint16_t *acc, size_t acc_stride, unsigned long long *stats,
                                     int *head, bool pack, int kt, int sms,
                                     const unsigned long long *masks, cudaStream_t st,
                                     const HitBuckets *hb)
{
    return launch_vote_batch_t<kModeEvent>(G, x, y, off, order, d_nev, acc, acc_stride, stats,
                                           head, pack, kt, sms, masks, st, bucket_view(hb));
}

cudaError_t launch_vote_hitmask(const DevGeom &G, const float *x, const float *y, int n,
                                void *acc, unsigned long long *stats,
                                const unsigned long long *hit_masks, cudaStream_t st)
{
    return launch_vote_t<kModeHit>(G, x, y, n, acc, stats, hit_masks, st);
}

cudaError_t launch_vote_batch_hitmask(const DevGeom &G, const float *x, const float *y,
                                      const int *off, const int *order, const int *d_nev,
                                      uint16_t *acc, size_t acc_stride,
                                      unsigned long long *stats, int *head, bool pack, int kt,
                                      int sms, const unsigned long long *hit_masks,
                                      cudaStream_t st, const HitBuckets *hb)
{
    return launch_vote_batch_t<kModeHit>(G, x, y, off, order, d_nev, acc, acc_stride, stats,
                                         head, pack, kt, sms, hit_masks, st, bucket_view(hb));
}

cudaError_t prepare_masked_vote_kernels(int max_smem)
{
    const cudaError_t e = prepare_vote_kernels_t<kModeEvent>(max_smem);
    return e == cudaSuccess ? prepare_vote_kernels_t<kModeHit>(max_smem) : e;
}

}  // namespace ht
