/*
 * ht_probe.h -- microbenchmarks for the rooflines libht's kernels are measured
 * against.  Not part of the method: the paper has no counterpart.
 */
#ifndef HT_PROBE_H
#define HT_PROBE_H

#include "ht.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Conflict-free shared-memory 32-bit atomicAdd throughput of the current
 * device: every SM runs resident CTAs whose lanes each add to their own
 * shared word `iters` times.  Synchronises `stream`.  *ops_per_s receives
 * the measured atomics per second (whole GPU).  iters in [1, 1 << 20].
 * Errors: HT_ERR_ARG, HT_ERR_CUDA. */
ht_status ht_probe_shared_atomic_rate(int32_t iters, double *ops_per_s, ht_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* HT_PROBE_H */
