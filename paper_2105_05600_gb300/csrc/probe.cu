// probe.cu -- the L2 gather microbenchmark that gives the fitness lookups their
// roofline (rf_l2_gather_probe, include/rf_measure.h).
#include "common.cuh"
#include "fitness.cuh"
#include "rf_measure.h"

namespace rf {

// One 32-bit mix of a counter (Wellons' "lowbias32" integer hash): consecutive
// counters give unrelated record indices, so a warp's 32 loads scatter.
__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__global__ void __launch_bounds__(256) l2_gather_probe_kernel(const uint4 *__restrict__ buf, uint32_t n_recs,
                                                              uint32_t n_recs_hi, int loads, uint32_t *sink)
{
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t base = gtid * (uint32_t)loads;
    uint32_t acc = 0u;
    for (int i = 0; i < loads; i += 8) {
        uint4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t h = mix32(base + (uint32_t)(i + u));
            // record index uniform in [0, n_recs): high word of h * n_recs (64-bit for large buffers)
            const size_t idx = n_recs_hi ? (size_t)(((unsigned long long)h * ((unsigned long long)n_recs_hi << 32 |
                                                                             n_recs)) >> 32)
                                         : (size_t)__umulhi(h, n_recs);
            v[u] = __ldg(buf + idx);
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
                                        uint32_t *sink_dev, void *stream)
{
    RF_CHECK_ARG(buf_dev && sink_dev, "null pointer");
    RF_CHECK_ARG(((uintptr_t)buf_dev & 15u) == 0, "buffer must be 16-byte aligned");
    RF_CHECK_ARG(bytes >= 16 && bytes % 16 == 0 && bytes < ((size_t)1 << 36), "bytes must be a multiple of 16");
    RF_CHECK_ARG(loads_per_thread >= 8 && loads_per_thread % 8 == 0 && loads_per_thread <= (1 << 20),
                 "loads_per_thread must be a multiple of 8 in [8, 2^20]");
    RF_CHECK_ARG(ctas_per_sm >= 1 && ctas_per_sm <= 8, "ctas_per_sm must be in [1, 8]");
    const unsigned long long n = bytes / 16;
    const int grid = ctas_per_sm * sm_count();
    l2_gather_probe_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const uint4 *>(buf_dev), (uint32_t)(n & 0xffffffffu), (uint32_t)(n >> 32),
        loads_per_thread, sink_dev);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}
