// k_vote_masked.cu -- the Hough vote (Section 5 of arXiv:1309.6275)
// restricted to a learned proposal's regions: the tile kernels of tiles.cuh
// with MASKED set, in their own translation unit so that they compile in
// parallel with the plain ones.
//
// A tile with no halo cell of the mask is skipped (nothing is written); in
// the other tiles phase 1 drops the (hit, column) pairs whose circle cannot
// reach a halo d0 window within the rho span of the tile's allowed rows, and
// the write-back keeps only halo cells.  Every vote that lands in a halo
// cell is still cast, so halo cells hold exactly the plain vote's counts.
#include "tiles.cuh"

namespace ht {

cudaError_t launch_vote_masked(const DevGeom &G, const float *x, const float *y, int n,
                               void *acc, unsigned long long *stats,
                               const unsigned long long *mask, cudaStream_t st)
{
    return launch_vote_t<true>(G, x, y, n, acc, stats, mask, st);
}

cudaError_t launch_vote_batch_masked(const DevGeom &G, const float *x, const float *y,
                                     const int *off, const int *order, const int *d_nev,
                                     uint16_t *acc, size_t acc_stride, unsigned long long *stats,
                                     int *head, bool pack, int kt, int sms,
                                     const unsigned long long *masks, cudaStream_t st)
{
    return launch_vote_batch_t<true>(G, x, y, off, order, d_nev, acc, acc_stride, stats, head,
                                     pack, kt, sms, masks, st);
}

cudaError_t prepare_masked_vote_kernels(int max_smem)
{
    return prepare_vote_kernels_t<true>(max_smem);
}

}  // namespace ht
