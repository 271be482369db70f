// probe.cu -- the gather microbenchmark that gives the fitness lookups their
// roofline (rf_l2_gather_probe, include/rf_measure.h).
#include "common.cuh"
#include "fitness.cuh"
#include "rf_measure.h"

namespace rf {

// One 32-bit mix of a counter (Wellons' "lowbias32" integer hash): consecutive
// counters give unrelated record indices, so a warp's loads scatter.
__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// mode 0: every lane loads its own random 16-byte record (a warp's load touches
// 32 lines); mode 1: each group of 8 lanes loads the 8 records of one random
// 128-byte line (4 lines per warp load, every byte used).  n_recs < 2^32.
__global__ void __launch_bounds__(256) l2_gather_probe_kernel(const uint4 *__restrict__ buf, uint32_t n_recs,
                                                              int loads, int mode, uint32_t *sink)
{
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    // the 8 lanes of a group draw the same counters in mode 1
    const uint32_t base = (mode ? (gtid >> 3) : gtid) * (uint32_t)loads;
    const uint32_t n_draw = mode ? n_recs >> 3 : n_recs;  // lines or records to draw from
    const uint32_t sub = mode ? (gtid & 7u) : 0u;
    uint32_t acc = 0u;
    for (int i = 0; i < loads; i += 8) {
        uint4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            // uniform in [0, n_draw): the high word of h * n_draw
            const uint32_t k = __umulhi(mix32(base + (uint32_t)(i + u)), n_draw);
            v[u] = __ldg(buf + (mode ? (size_t)k * 8 + sub : (size_t)k));
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    sink[gtid] = acc;
}

}  // namespace rf

using namespace rf;

extern "C" rf_status rf_l2_gather_probe(const void *buf_dev, size_t bytes, int loads_per_thread, int ctas_per_sm,
                                        int mode, uint32_t *sink_dev, void *stream)
{
    RF_CHECK_ARG(buf_dev && sink_dev, "null pointer");
    RF_CHECK_ARG(((uintptr_t)buf_dev & 15u) == 0, "buffer must be 16-byte aligned");
    RF_CHECK_ARG(mode == 0 || mode == 1, "mode must be 0 (16-byte records) or 1 (128-byte lines)");
    RF_CHECK_ARG(bytes % 16 == 0 && bytes >= (mode ? 128u : 16u) && bytes < ((size_t)1 << 36),
                 "bytes must be a multiple of 16 in [16 (128 for mode 1), 2^36)");
    RF_CHECK_ARG(loads_per_thread >= 8 && loads_per_thread % 8 == 0 && loads_per_thread <= (1 << 20),
                 "loads_per_thread must be a multiple of 8 in [8, 2^20]");
    RF_CHECK_ARG(ctas_per_sm >= 1 && ctas_per_sm <= 8, "ctas_per_sm must be in [1, 8]");
    const int grid = ctas_per_sm * sm_count();
    RF_CHECK_ARG((unsigned long long)grid * 256ull * (unsigned long long)loads_per_thread < (1ull << 32),
                 "grid x 256 x loads_per_thread must stay below 2^32");
    l2_gather_probe_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const uint4 *>(buf_dev),
                                                                    (uint32_t)(bytes / 16), loads_per_thread, mode,
                                                                    sink_dev);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}
