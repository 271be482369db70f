/*
 * rf_measure.h -- measurement entry points of librosefusion.so.  They serve the
 * roofline statements about the hot path; the paper has no counterpart for
 * either (it reports only frame rates and per-frame times).  The general rules
 * of rosefusion.h apply (status codes, *_dev device pointers, streams).
 */
#ifndef RF_MEASURE_H
#define RF_MEASURE_H

#include <stddef.h>
#include <stdint.h>

#include "rosefusion.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * rf_l2_gather_probe -- one launch of a gather microbenchmark whose bandwidth
 * bounds the fitness lookups: every thread of a grid of ctas_per_sm x (number
 * of SMs) CTAs of 256 threads issues loads_per_thread independent 16-byte
 * loads (the non-coherent path the fitness kernel's cell loads take) at
 * pseudo-random positions of buf_dev, eight in flight per thread, folds them
 * with XOR and writes one word per thread to sink_dev.
 *   mode 0  each lane loads its own random 16-byte record: a warp's load
 *           touches 32 lines (the pattern of fully scattered lookups)
 *   mode 1  each group of 8 lanes loads the 8 records of one random 128-byte
 *           line: 4 lines per warp load, every byte used (the L2's own rate)
 * With `bytes` well below the L2 size the data stays in L2, so the bytes
 * loaded (grid x 256 x loads_per_thread x 16) over the kernel time measured on
 * `stream` is the gather bandwidth of that pattern.
 *   buf_dev           device buffer of `bytes` bytes, 16-byte aligned, bytes a
 *                     multiple of 16 in [16, 2^36) (at least 128 for mode 1)
 *   loads_per_thread  multiple of 8 in [8, 2^20]; grid x 256 x loads < 2^32
 *   ctas_per_sm       1 .. 8
 *   sink_dev          device uint32[ctas_per_sm * SMs * 256], overwritten
 * Asynchronous.  RF_ERR_ARG for sizes, modes or pointers outside these ranges.
 */
rf_status rf_l2_gather_probe(const void *buf_dev, size_t bytes, int loads_per_thread, int ctas_per_sm, int mode,
                             uint32_t *sink_dev, void *stream);

/*
 * rf_volume_counters -- fusion work done on the volume since the last reset:
 * out_host[0] voxels updated by tsdf_integrate (each reads and writes its value
 * and weight: 2 x (value size + 1) bytes), out_host[1] bricks of 8^3 voxels that
 * passed the fusion kernel's frustum test (the others are skipped unread),
 * out_host[2] bricks whose packed trilinear cells were rebuilt.  reset != 0
 * zeroes the counters after reading.  Synchronises the device.
 */
rf_status rf_volume_counters(rf_volume v, long long out_host[3], int reset);

#ifdef __cplusplus
}
#endif
#endif /* RF_MEASURE_H */
