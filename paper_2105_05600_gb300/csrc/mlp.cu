// mlp.cu -- the learned swarm proposal's network on the 5th-generation tensor
// cores.  Not part of the paper (Sec. 6 names learned priors as future work): a
// 4-layer MLP 832 -> 256 -> 256 -> 256 -> 16 whose output seeds the PST of a
// frame (the c_0, r_0 of the Sec. 4 initialisation).  Training (forward, loss,
// backward, Adam) and inference run only the kernels of this file.
//
// Every product is one launch of umma_gemm_kernel:
//     C[M x N] = A[M x K] . B[N x K]^T,  A, B bfloat16 row-major (K contiguous),
//     FP32 accumulation in tensor memory (TMEM), fused epilogue.
// One CTA owns a 128 x 128 tile of C and 128 TMEM columns:
//   warp 0, lane 0   TMA producer: 128-row x 64-column slabs of A and B into a
//                    4-stage shared-memory ring (mbarrier transaction counts)
//   warp 1, lane 0   MMA issuer: 4 x tcgen05.mma.kind::f16 (M 128, N 128, K 16)
//                    per slab; tcgen05.commit releases the slab
//   warps 0..3       epilogue: tcgen05.ld of the warp's 32 accumulator lanes,
//                    bias / ReLU / gradient mask, bfloat16 or FP32 stores, the
//                    bfloat16 ones optionally also transposed (the backward
//                    products reduce over the batch and need batch-contiguous
//                    operands)
// Shared-memory operand layout (no swizzle, K-major): the 8 x 8 core matrix of
// rows 8g..8g+7 and columns 8c..8c+7 of a slab is 128 contiguous bytes at
// 128 g + 2048 c; one TMA box (8 columns x 128 rows) fills one column group c.
// So the descriptors' leading-dimension (K) byte offset is 2048 and the
// stride-dimension (M/N) byte offset is 128; K step j of a slab starts at
// 4096 j.  Every wait on an mbarrier is bounded in time; on expiry the CTA
// records RF_ERR_TIMEOUT, lets its copies land, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "rf_proposal.h"

namespace rf {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int GB_M = 128, GB_N = 128, GB_K = 64, GB_STAGES = 4, GB_THREADS = 128;
constexpr int GB_CHUNK = GB_M * 16;         // one 8-column group of a slab: 128 rows x 16 B
constexpr int GB_TILE = 8 * GB_CHUNK;       // 16 KiB per operand slab (GB_M == GB_N)
constexpr int GB_STAGE = 2 * GB_TILE;
constexpr int GB_LBO = GB_CHUNK;            // K-direction core-matrix step
constexpr int GB_SBO = 128;                 // M/N-direction core-matrix step
// A margin after the ring keeps every byte that a descriptor built on these
// slabs can address inside the allocation, whatever the slab index.
constexpr int GB_GUARD = 48 * 1024;
constexpr int GB_BAR_OFF = GB_STAGES * GB_STAGE + GB_GUARD;
constexpr int GB_SMEM = GB_BAR_OFF + 128 + 1024;  // + barriers, + alignment slack
constexpr uint32_t GB_TMEM_COLS = 128;
// kind::f16 instruction descriptor: D FP32 (bits 4-5 = 1), A and B bfloat16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t GB_IDESC =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GB_N >> 3) << 17) | ((uint32_t)(GB_M >> 4) << 24);

enum { EPI_BIAS_RELU = 0, EPI_BIAS = 1, EPI_MASK = 2, EPI_PLAIN = 3 };

struct GemmEpi {
    int M, N, K;
    int mode;
    const float *bias;     // [N]                 (EPI_BIAS_RELU, EPI_BIAS)
    const bf16 *mask;      // [M x N], ld_mask    (EPI_MASK: keep where mask > 0)
    bf16 *out_h;           // [M x N] bfloat16, ld_h (may be NULL)
    bf16 *out_ht;          // [N x M] bfloat16, ld_ht (may be NULL)
    float *out_f;          // [M x N] FP32, ld_f (may be NULL)
    int ld_mask, ld_h, ld_ht, ld_f;
    int *err;
    long long timeout_ns;
};

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ long long gtimer()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Wait for the phase of `parity` to complete; false after timeout_ns.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, long long timeout_ns)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const long long t0 = gtimer();
    while (!mbar_try_wait(bar, parity))
        if (gtimer() - t0 > timeout_ns)
            return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), leading byte offset
// >> 4 (16-29), stride byte offset >> 4 (32-45), the fixed 0b001 of bits 46-48,
// base offset 0, swizzle mode 0 (none, bits 61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(GB_LBO >> 4) << 16) | ((uint64_t)(GB_SBO >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(GB_IDESC), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane; the wait
// sits in the same statement so the registers are valid when it returns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15}, [%16];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] = __uint_as_float(r[i]);
}

// Column groups of K slab kb that hold data: an even count (whole K steps of 16).
__device__ __forceinline__ int slab_groups(int K, int kb)
{
    const int rem = min(GB_K, K - kb * GB_K);
    return 2 * ((rem + 15) >> 4);
}

// ------------------------------------------------------------------ epilogue
__device__ __forceinline__ void epi_store(const GemmEpi &e, int m, int n, float v[16])
{
    if (m >= e.M)
        return;
    const bool whole = n + 16 <= e.N;
    if (e.mode == EPI_BIAS_RELU || e.mode == EPI_BIAS) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float b = (n + i < e.N) ? __ldg(&e.bias[n + i]) : 0.f;
            v[i] += b;
            if (e.mode == EPI_BIAS_RELU)
                v[i] = fmaxf(v[i], 0.f);
        }
    } else if (e.mode == EPI_MASK) {
        const bf16 *mk = e.mask + (size_t)m * e.ld_mask + n;
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (n + i >= e.N || !(__bfloat162float(mk[i]) > 0.f))
                v[i] = 0.f;
    }
    if (e.out_f) {
        float *o = e.out_f + (size_t)m * e.ld_f + n;
        if (whole) {
#pragma unroll
            for (int i = 0; i < 16; i += 4)
                *reinterpret_cast<float4 *>(o + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        } else {
            for (int i = 0; i < 16 && n + i < e.N; ++i)
                o[i] = v[i];
        }
    }
    if (e.out_h || e.out_ht) {
        bf16 h[16];
#pragma unroll
        for (int i = 0; i < 16; ++i)
            h[i] = __float2bfloat16_rn(v[i]);
        if (e.out_h) {
            bf16 *o = e.out_h + (size_t)m * e.ld_h + n;
            if (whole) {
                *reinterpret_cast<uint4 *>(o) = *reinterpret_cast<const uint4 *>(&h[0]);
                *reinterpret_cast<uint4 *>(o + 8) = *reinterpret_cast<const uint4 *>(&h[8]);
            } else {
                for (int i = 0; i < 16 && n + i < e.N; ++i)
                    o[i] = h[i];
            }
        }
        if (e.out_ht)  // lanes hold consecutive m: each column store is coalesced
            for (int i = 0; i < 16 && n + i < e.N; ++i)
                e.out_ht[(size_t)(n + i) * e.ld_ht + m] = h[i];
    }
}

// ------------------------------------------------------------------ the GEMM
__global__ void __launch_bounds__(GB_THREADS, 1)
    umma_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const GemmEpi e)
{
    extern __shared__ uint8_t gsm_raw[];
    const uint32_t raw = smem_u32(gsm_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gsm = gsm_raw + (base - raw);
    const uint32_t bar_full = base + GB_BAR_OFF;
    const uint32_t bar_empty = bar_full + 8 * GB_STAGES;
    const uint32_t bar_done = bar_empty + 8 * GB_STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gsm + GB_BAR_OFF + 16 * GB_STAGES + 8);
    volatile int *s_fail = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * GB_M, n0 = blockIdx.y * GB_N;
    const int nk = (e.K + GB_K - 1) / GB_K;

    if (threadIdx.x == 0) {
        for (int s = 0; s < GB_STAGES; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        mbar_init(bar_done, 1);
        *s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(GB_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int last[GB_STAGES];
            for (int s = 0; s < GB_STAGES; ++s)
                last[s] = -1;
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % GB_STAGES;
                if (kb >= GB_STAGES && !mbar_wait(bar_empty + 8 * s, ((kb / GB_STAGES) - 1) & 1, e.timeout_ns)) {
                    *s_fail = 1;
                    break;
                }
                const int groups = slab_groups(e.K, kb);
                mbar_expect_tx(bar_full + 8 * s, (uint32_t)(2 * groups * GB_CHUNK));
                const uint32_t a = base + s * GB_STAGE, b = a + GB_TILE;
                for (int c = 0; c < groups; ++c) {
                    tma_load_2d(a + c * GB_CHUNK, &tmA, kb * GB_K + 8 * c, m0, bar_full + 8 * s);
                    tma_load_2d(b + c * GB_CHUNK, &tmB, kb * GB_K + 8 * c, n0, bar_full + 8 * s);
                }
                last[s] = kb;
            }
            // no copy may still be landing when the CTA leaves
            for (int s = 0; s < GB_STAGES; ++s)
                if (last[s] >= 0 && !mbar_wait(bar_full + 8 * s, (last[s] / GB_STAGES) & 1, e.timeout_ns))
                    *s_fail = 1;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % GB_STAGES;
                if (!mbar_wait(bar_full + 8 * s, (kb / GB_STAGES) & 1, e.timeout_ns)) {
                    *s_fail = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t a = base + s * GB_STAGE, b = a + GB_TILE;
                const int steps = slab_groups(e.K, kb) / 2;
                for (int j = 0; j < steps; ++j)
                    umma_bf16(tmem, smem_desc(a + j * 2 * GB_CHUNK), smem_desc(b + j * 2 * GB_CHUNK),
                              (kb | j) != 0 ? 1u : 0u);
                umma_commit(bar_empty + 8 * s);
            }
            umma_commit(bar_done);  // arrives once every MMA issued above has completed
        }
        __syncwarp();
    }

    // epilogue: every warp drains its own 32 TMEM lanes
    const int ok = __syncthreads_and(mbar_wait(bar_done, 0, e.timeout_ns) ? 1 : 0) && !*s_fail;
    tc_fence_after();
    if (ok) {
        const int m = m0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int nc = 0; nc < GB_N && n0 + nc < e.N; nc += 16) {
            float v[16];
            tmem_ld16(trow + (uint32_t)nc, v);
            epi_store(e, m, n0 + nc, v);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GB_TMEM_COLS)
                     : "memory");
    }
    if (threadIdx.x == 0 && !ok)
        atomicCAS(e.err, 0, RF_ERR_TIMEOUT);
}


// ------------------------------------------------------------------ elementwise kernels
// Layout of the flat FP32 parameter vector (W1, b1, W2, b2, W3, b3, W4, b4; each W
// row-major out x in) and of the packed bfloat16 weight copies (W_l at pk_off[l],
// its transpose at the same offset of the transposed copy).
struct LayerTable {
    int w_off[4], pk_off[4], out[4], in[4];
    int total;
};

__device__ __forceinline__ int layer_of(const LayerTable &L, int p)
{
    int l = 0;
    while (l < 3 && p >= L.w_off[l + 1])
        ++l;
    return l;
}

// Adam (Kingma & Ba 2015, Algorithm 1) on the FP32 parameters when `update`,
// then the bfloat16 weights the GEMMs read, row-major and transposed.
__global__ void adam_kernel(float *theta, const float *grad, float *m, float *v, const LayerTable L, float lr,
                            float b1, float b2, float eps, float bc1, float bc2, int update, bf16 *w, bf16 *wt)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < L.total; p += gridDim.x * blockDim.x) {
        float th = theta[p];
        if (update) {
            const float g = grad[p];
            const float mm = b1 * m[p] + (1.f - b1) * g;
            const float vv = b2 * v[p] + (1.f - b2) * g * g;
            m[p] = mm;
            v[p] = vv;
            th -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
            theta[p] = th;
        }
        const int l = layer_of(L, p);
        const int q = p - L.w_off[l];
        if (q < L.out[l] * L.in[l]) {
            const int o = q / L.in[l], i = q - o * L.in[l];
            const bf16 h = __float2bfloat16_rn(th);
            w[L.pk_off[l] + q] = h;
            wt[L.pk_off[l] + i * L.out[l] + o] = h;
        }
    }
}

// Rows idx[b] (row b when idx is NULL) of a dataset into the batch buffers: the
// input row-major and transposed, the target.  Out-of-range rows raise RF_ERR_ARG.
__global__ void gather_kernel(const bf16 *x_all, const float *y_all, const int *idx, int n_all, int B, bf16 *x,
                              bf16 *xt, float *y, int *err)
{
    const int b = blockIdx.x;
    const int r = idx ? __ldg(&idx[b]) : b;
    if (r < 0 || r >= n_all) {
        if (threadIdx.x == 0)
            atomicCAS(err, 0, RF_ERR_ARG);
        return;
    }
    const bf16 *src = x_all + (size_t)r * RF_MLP_IN;
    for (int k = threadIdx.x; k < RF_MLP_IN; k += blockDim.x) {
        const bf16 v = src[k];
        x[(size_t)b * RF_MLP_IN + k] = v;
        xt[(size_t)k * B + b] = v;
    }
    if (threadIdx.x < 6)
        y[b * 6 + threadIdx.x] = y_all[(size_t)r * 6 + threadIdx.x];
}

// Loss (mean over the batch of sum_d 1/2 r^2 (1 + e^{-2s}) + s, r = y - mu,
// mu = x_v + o_mu with x_v the previous-offset inputs (columns 768..773 of the
// batch rows), s = clamp(o_s, -6, 6)) and its gradient with respect to the 16 outputs,
// computed in FP32 per sample and stored as bfloat16 (row-major and
// transposed) for the backward products; the batch sum runs in FP64 in a fixed
// order.  One CTA, one thread per sample (B <= 1024).
__global__ void loss_kernel(const float *out, const float *y, const bf16 *x, int B, bf16 *g, bf16 *gt, float *loss)
{
    __shared__ double red[32];
    const int b = threadIdx.x;
    double l = 0.0;
    if (b < B) {
        float gr[RF_MLP_OUT];
        for (int j = 0; j < RF_MLP_OUT; ++j)
            gr[j] = 0.f;
        const float inv_b = 1.f / (float)B;
        float lf = 0.f;
        for (int d = 0; d < 6; ++d) {
            const float mu = out[b * RF_MLP_OUT + d] + __bfloat162float(x[(size_t)b * RF_MLP_IN + RF_MLP_IN_USED - 6 + d]);
            const float sr = out[b * RF_MLP_OUT + 6 + d];
            const float s = fminf(fmaxf(sr, -6.f), 6.f);
            const float r = y[b * 6 + d] - mu;
            const float ex = expf(-2.f * s);
            lf += 0.5f * r * r * (1.f + ex) + s;
            gr[d] = -r * (1.f + ex) * inv_b;
            gr[6 + d] = (sr > -6.f && sr < 6.f) ? (1.f - r * r * ex) * inv_b : 0.f;
        }
        l = lf;
        for (int j = 0; j < RF_MLP_OUT; ++j) {
            const bf16 h = __float2bfloat16_rn(gr[j]);
            g[b * RF_MLP_OUT + j] = h;
            gt[(size_t)j * B + b] = h;
        }
    }
    for (int o = 16; o > 0; o >>= 1)
        l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0)
        red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            t += red[w];
        loss[0] = (float)(t / B);
    }
}

// Bias gradient db[n] = sum_b dt[n][b] over the transposed bfloat16 gradient:
// one warp per n, lane-strided FP32 partial sums, then a fixed shuffle tree.
__global__ void bias_grad_kernel(const bf16 *dt, int N, int B, float *db)
{
    const int n = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (n >= N)
        return;
    float s = 0.f;
    for (int b = lane; b < B; b += 32)
        s += __bfloat162float(dt[(size_t)n * B + b]);
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0)
        db[n] = s;
}

// ------------------------------------------------------------------ host: tensor maps and launches
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

rf_status tensor_map_encoder(EncodeTiledFn *out)
{
    static std::mutex mu;
    static EncodeTiledFn fn = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
            set_error("cuTensorMapEncodeTiled not available (%s)", cudaGetErrorString(e));
            return RF_ERR_CUDA;
        }
        fn = (EncodeTiledFn)p;
    }
    *out = fn;
    return RF_OK;
}

// TMA map of a row-major bfloat16 operand [rows x cols] with leading dimension ld:
// box of 8 columns (16 B) x 128 rows, no swizzle; reads past rows or cols fill 0.
rf_status operand_map(CUtensorMap *map, const bf16 *ptr, int rows, int cols, int ld)
{
    RF_CHECK_ARG(ptr && ((uintptr_t)ptr & 15) == 0, "operand not 16-byte aligned");
    RF_CHECK_ARG(rows >= 1 && cols >= 1 && ld >= cols && ld % 8 == 0, "operand shape");
    EncodeTiledFn enc;
    rf_status st = tensor_map_encoder(&enc);
    if (st != RF_OK)
        return st;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(bf16)};
    const cuuint32_t box[2] = {8, (cuuint32_t)GB_M};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(ptr), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return RF_ERR_CUDA;
    }
    return RF_OK;
}

rf_status gemm_smem_attr()
{
    static std::mutex mu;
    static unsigned long long done_mask = 0;
    int dev = 0;
    RF_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 64 && !(done_mask >> dev & 1ull)) {
        RF_CUDA(cudaFuncSetAttribute(umma_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, GB_SMEM));
        done_mask |= 1ull << dev;
    }
    return RF_OK;
}

// C = A . B^T with the epilogue of e (e.M, e.N, e.K set by the caller).
rf_status gemm(const bf16 *A, int lda, const bf16 *B, int ldb, GemmEpi e, cudaStream_t s)
{
    RF_CHECK_ARG(e.M >= 1 && e.N >= 1 && e.K >= 1, "empty product");
    RF_CHECK_ARG(!e.out_h || e.ld_h % 8 == 0, "ld_h");
    RF_CHECK_ARG(!e.out_f || e.ld_f % 4 == 0, "ld_f");
    CUtensorMap ta, tb;
    rf_status st = operand_map(&ta, A, e.M, e.K, lda);
    if (st == RF_OK)
        st = operand_map(&tb, B, e.N, e.K, ldb);
    if (st == RF_OK)
        st = gemm_smem_attr();
    if (st != RF_OK)
        return st;
    const dim3 grid((e.M + GB_M - 1) / GB_M, (e.N + GB_N - 1) / GB_N);
    umma_gemm_kernel<<<grid, GB_THREADS, GB_SMEM, s>>>(ta, tb, e);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

GemmEpi epi(int M, int N, int K, int mode, int *err, long long timeout_ns)
{
    GemmEpi e;
    memset(&e, 0, sizeof e);
    e.M = M;
    e.N = N;
    e.K = K;
    e.mode = mode;
    e.err = err;
    e.timeout_ns = timeout_ns;
    return e;
}

}  // namespace
// The quantities training selects and calibrates the network with, over B rows
// of a batch (outputs `out`, inputs `x`, targets `y`): mu = x_v + o_mu (x_v the
// previous-offset inputs), s = clamp(o_s, -6, 6), e = y - mu, and per row
// sum_d e_d^2, e_d^2 exp(-2 s_d), y_d^2 (13 values, FP64).  One CTA; thread t
// takes rows t, t + blockDim, ...; the per-thread sums are combined by a fixed
// shuffle tree and warp order, and thread 0 adds them to acc (the calls for the
// successive batches of a data set run in stream order, so the total is fixed).
constexpr int EVAL_STATS = 13;
__global__ void eval_kernel(const float *out, const bf16 *x, const float *y, int B, int row0, float *mu_out,
                            double *acc)
{
    __shared__ double red[EVAL_STATS][32];
    double loc[EVAL_STATS];
    for (int e = 0; e < EVAL_STATS; ++e)
        loc[e] = 0.0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        for (int d = 0; d < 6; ++d) {
            const float mu = out[b * RF_MLP_OUT + d] +
                             __bfloat162float(x[(size_t)b * RF_MLP_IN + RF_MLP_IN_USED - 6 + d]);
            const float s = fminf(fmaxf(out[b * RF_MLP_OUT + 6 + d], -6.f), 6.f);
            const double yd = (double)y[b * 6 + d];
            const double e = yd - (double)mu;
            loc[0] += e * e;
            loc[1 + d] += e * e * exp(-2.0 * (double)s);
            loc[7 + d] += yd * yd;
            if (mu_out)
                mu_out[(size_t)(row0 + b) * 6 + d] = mu;
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = 0; e < EVAL_STATS; ++e) {
        double v = loc[e];
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0)
            red[e][w] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int e = 0; e < EVAL_STATS; ++e) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
                t += red[e][q];
            acc[e] += t;
        }
}

__global__ void eval_finish_kernel(const double *acc, int n_rows, double *stats)
{
    if (threadIdx.x < EVAL_STATS)
        stats[threadIdx.x] = acc[threadIdx.x] / (double)n_rows;
}

// log k_d added to the output bias of the log-scale s_d, k_d^2 = stats[1 + d].
__global__ void calibrate_kernel(const double *stats, float *bias_s, float *k_out)
{
    const int d = threadIdx.x;
    if (d < 6) {
        const double k = sqrt(fmax(stats[1 + d], 1e-12));
        bias_s[d] += (float)log(k);
        k_out[d] = (float)k;
    }
}

}  // namespace rf

using namespace rf;

// ------------------------------------------------------------------ network handle
struct rf_mlp_s {
    int max_batch;
    LayerTable L;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    bf16 *w = nullptr, *wt = nullptr;  // packed bfloat16 weights and transposes
    bf16 *x = nullptr, *xt = nullptr;
    bf16 *h[3] = {}, *ht[3] = {};      // hidden activations h1..h3 (row-major, transposed)
    bf16 *d[3] = {}, *dt[3] = {};      // masked hidden gradients
    bf16 *g = nullptr, *gt = nullptr;  // output gradients
    float *out = nullptr, *y = nullptr, *loss = nullptr;
    double *eval_acc = nullptr;  // rf_mlp_evaluate: running sums, then the means (2 x EVAL_STATS)
    float *eval_k = nullptr;     // rf_mlp_calibrate_scale: k (6)
    int *err = nullptr;
    int step = 0;
    long long timeout_ns = 1000000000ll;
    std::vector<void *> allocs;
};

static const int kOut[4] = {RF_MLP_HIDDEN, RF_MLP_HIDDEN, RF_MLP_HIDDEN, RF_MLP_OUT};
static const int kIn[4] = {RF_MLP_IN, RF_MLP_HIDDEN, RF_MLP_HIDDEN, RF_MLP_HIDDEN};

static LayerTable layer_table()
{
    LayerTable L;
    int p = 0, k = 0;
    for (int l = 0; l < 4; ++l) {
        L.out[l] = kOut[l];
        L.in[l] = kIn[l];
        L.w_off[l] = p;
        L.pk_off[l] = k;
        p += kOut[l] * kIn[l] + kOut[l];
        k += kOut[l] * kIn[l];
    }
    L.total = p;
    return L;
}

static rf_status mlp_alloc(rf_mlp m, void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(mlp)");
    m->allocs.push_back(*p);
    return RF_OK;
}

// Refresh the bfloat16 weight copies (update = 0) or take one Adam step.
static rf_status mlp_adam(rf_mlp m, int update, float lr, cudaStream_t s)
{
    const double b1 = 0.9, b2 = 0.999;
    float bc1 = 1.f, bc2 = 1.f;
    if (update) {
        m->step += 1;
        bc1 = (float)(1.0 - pow(b1, m->step));
        bc2 = (float)(1.0 - pow(b2, m->step));
    }
    adam_kernel<<<304, 256, 0, s>>>(m->theta, m->grad, m->m, m->v, m->L, lr, (float)b1, (float)b2, 1e-8f, bc1, bc2,
                                    update, m->w, m->wt);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

// Forward pass of B rows of m->x (or of x when given): hidden activations to
// m->h (and m->ht when `train`), outputs to out (B x 16, FP32).
static rf_status mlp_forward(rf_mlp m, const bf16 *x, int B, float *out, int train, cudaStream_t s)
{
    const LayerTable &L = m->L;
    const bf16 *in = x;
    int ld_in = RF_MLP_IN;
    for (int l = 0; l < 3; ++l) {
        GemmEpi e = epi(B, RF_MLP_HIDDEN, L.in[l], EPI_BIAS_RELU, m->err, m->timeout_ns);
        e.bias = m->theta + L.w_off[l] + L.out[l] * L.in[l];
        e.out_h = m->h[l];
        e.ld_h = RF_MLP_HIDDEN;
        if (train) {
            e.out_ht = m->ht[l];
            e.ld_ht = B;
        }
        rf_status st = gemm(in, ld_in, m->w + L.pk_off[l], L.in[l], e, s);
        if (st != RF_OK)
            return st;
        in = m->h[l];
        ld_in = RF_MLP_HIDDEN;
    }
    GemmEpi e = epi(B, RF_MLP_OUT, RF_MLP_HIDDEN, EPI_BIAS, m->err, m->timeout_ns);
    e.bias = m->theta + L.w_off[3] + L.out[3] * L.in[3];
    e.out_f = out;
    e.ld_f = RF_MLP_OUT;
    return gemm(in, RF_MLP_HIDDEN, m->w + L.pk_off[3], RF_MLP_HIDDEN, e, s);
}

// Gather, forward, loss and backward of one batch: the gradient lands in m->grad.
static rf_status mlp_gradient(rf_mlp m, const bf16 *x_all, const float *y_all, const int *idx, int n_all, int B,
                              cudaStream_t s)
{
    const LayerTable &L = m->L;
    gather_kernel<<<B, 256, 0, s>>>(x_all, y_all, idx, n_all, B, m->x, m->xt, m->y, m->err);
    RF_CUDA(cudaGetLastError());
    rf_status st = mlp_forward(m, m->x, B, m->out, 1, s);
    if (st != RF_OK)
        return st;
    loss_kernel<<<1, (B + 31) / 32 * 32, 0, s>>>(m->out, m->y, m->x, B, m->g, m->gt, m->loss);
    RF_CUDA(cudaGetLastError());
    // layer 4: dW4 = g^T h3, db4 = sum_b g, dH3 = g W4 masked by h3 > 0
    const bf16 *dA = m->g, *dAt = m->gt;
    int n_out = RF_MLP_OUT;
    for (int l = 3; l >= 0; --l) {
        const bf16 *act_t = l > 0 ? m->ht[l - 1] : m->xt;  // the layer's input, transposed
        GemmEpi e = epi(L.out[l], L.in[l], B, EPI_PLAIN, m->err, m->timeout_ns);
        e.out_f = m->grad + L.w_off[l];
        e.ld_f = L.in[l];
        st = gemm(dAt, B, act_t, B, e, s);
        if (st != RF_OK)
            return st;
        bias_grad_kernel<<<(n_out + 7) / 8, 256, 0, s>>>(dAt, n_out, B, m->grad + L.w_off[l] + L.out[l] * L.in[l]);
        RF_CUDA(cudaGetLastError());
        if (l == 0)
            break;
        GemmEpi eb = epi(B, L.in[l], L.out[l], EPI_MASK, m->err, m->timeout_ns);
        eb.mask = m->h[l - 1];
        eb.ld_mask = RF_MLP_HIDDEN;
        eb.out_h = m->d[l - 1];
        eb.ld_h = RF_MLP_HIDDEN;
        eb.out_ht = m->dt[l - 1];
        eb.ld_ht = B;
        st = gemm(dA, L.out[l], m->wt + L.pk_off[l], L.out[l], eb, s);
        if (st != RF_OK)
            return st;
        dA = m->d[l - 1];
        dAt = m->dt[l - 1];
        n_out = RF_MLP_HIDDEN;
    }
    return RF_OK;
}

extern "C" {

int rf_mlp_num_params(void) { return layer_table().total; }

rf_status rf_mlp_create(int max_batch, rf_mlp *out)
{
    RF_CHECK_ARG(out != nullptr, "null output");
    *out = nullptr;
    RF_CHECK_ARG(max_batch >= 1 && max_batch <= RF_MLP_MAX_BATCH, "max_batch outside [1, RF_MLP_MAX_BATCH]");
    rf_mlp m = new rf_mlp_s();
    m->max_batch = (max_batch + 7) / 8 * 8;
    m->L = layer_table();
    const size_t P = (size_t)m->L.total, PK = (size_t)m->L.pk_off[3] + (size_t)RF_MLP_OUT * RF_MLP_HIDDEN;
    const size_t Bc = (size_t)m->max_batch;
    rf_status st = RF_OK;
    void **fl[4] = {(void **)&m->theta, (void **)&m->grad, (void **)&m->m, (void **)&m->v};
    for (int i = 0; i < 4 && st == RF_OK; ++i)
        st = mlp_alloc(m, fl[i], P * sizeof(float));
    if (st == RF_OK)
        st = mlp_alloc(m, (void **)&m->w, PK * sizeof(bf16));
    if (st == RF_OK)
        st = mlp_alloc(m, (void **)&m->wt, PK * sizeof(bf16));
    if (st == RF_OK)
        st = mlp_alloc(m, (void **)&m->x, Bc * RF_MLP_IN * sizeof(bf16));
    if (st == RF_OK)
        st = mlp_alloc(m, (void **)&m->xt, Bc * RF_MLP_IN * sizeof(bf16));
    for (int l = 0; l < 3 && st == RF_OK; ++l) {
        st = mlp_alloc(m, (void **)&m->h[l], Bc * RF_MLP_HIDDEN * sizeof(bf16));
        if (st == RF_OK)
            st = mlp_alloc(m, (void **)&m->ht[l], Bc * RF_MLP_HIDDEN * sizeof(bf16));
        if (st == RF_OK)
            st = mlp_alloc(m, (void **)&m->d[l], Bc * RF_MLP_HIDDEN * sizeof(bf16));
        if (st == RF_OK)
            st = mlp_alloc(m, (void **)&m->dt[l], Bc * RF_MLP_HIDDEN * sizeof(bf16));
    }
    if (st == RF_OK)
        st = mlp_alloc(m, (void **)&m->g, Bc * RF_MLP_OUT * sizeof(bf16));
    if (st == RF_OK)
        st = mlp_alloc(m, (void **)&m->gt, Bc * RF_MLP_OUT * sizeof(bf16));
    if (st == RF_OK)
        st = mlp_alloc(m, (void **)&m->out, Bc * RF_MLP_OUT * sizeof(float));
    if (st == RF_OK)
        st = mlp_alloc(m, (void **)&m->y, Bc * 6 * sizeof(float));
    if (st == RF_OK)
        st = mlp_alloc(m, (void **)&m->loss, sizeof(float));
    if (st == RF_OK)
        st = mlp_alloc(m, (void **)&m->err, sizeof(int));
    if (st == RF_OK)
        st = mlp_alloc(m, (void **)&m->eval_acc, 2 * EVAL_STATS * sizeof(double));
    if (st == RF_OK)
        st = mlp_alloc(m, (void **)&m->eval_k, 6 * sizeof(float));
    if (st == RF_OK) {
        cudaError_t e = cudaMemset(m->theta, 0, P * sizeof(float));
        if (e == cudaSuccess)
            e = cudaMemset(m->grad, 0, P * sizeof(float));
        if (e == cudaSuccess)
            e = cudaMemset(m->m, 0, P * sizeof(float));
        if (e == cudaSuccess)
            e = cudaMemset(m->v, 0, P * sizeof(float));
        if (e == cudaSuccess)
            e = cudaMemset(m->w, 0, PK * sizeof(bf16));
        if (e == cudaSuccess)
            e = cudaMemset(m->wt, 0, PK * sizeof(bf16));
        if (e == cudaSuccess)
            e = cudaMemset(m->err, 0, sizeof(int));
        if (e != cudaSuccess)
            st = cuda_fail(e, "cudaMemset(mlp)");
    }
    // resolve the tensor-map encoder and the kernel's shared-memory limit now, so
    // that no later call (for example inside a stream capture) does it first
    EncodeTiledFn enc;
    if (st == RF_OK)
        st = tensor_map_encoder(&enc);
    if (st == RF_OK)
        st = gemm_smem_attr();
    if (st != RF_OK) {
        rf_mlp_destroy(m);
        return st;
    }
    *out = m;
    return RF_OK;
}

void rf_mlp_destroy(rf_mlp m)
{
    if (!m)
        return;
    for (void *p : m->allocs)
        cudaFree(p);
    delete m;
}

rf_status rf_mlp_set_params(rf_mlp m, const float *theta_host)
{
    RF_CHECK_ARG(m && theta_host, "null pointer");
    const size_t P = (size_t)m->L.total;
    RF_CUDA(cudaMemcpy(m->theta, theta_host, P * sizeof(float), cudaMemcpyHostToDevice));
    RF_CUDA(cudaMemset(m->m, 0, P * sizeof(float)));
    RF_CUDA(cudaMemset(m->v, 0, P * sizeof(float)));
    m->step = 0;
    rf_status st = mlp_adam(m, 0, 0.f, 0);
    if (st != RF_OK)
        return st;
    RF_CUDA(cudaDeviceSynchronize());
    return RF_OK;
}

rf_status rf_mlp_get_params(rf_mlp m, float *theta_host)
{
    RF_CHECK_ARG(m && theta_host, "null pointer");
    RF_CUDA(cudaDeviceSynchronize());
    RF_CUDA(cudaMemcpy(theta_host, m->theta, (size_t)m->L.total * sizeof(float), cudaMemcpyDeviceToHost));
    return RF_OK;
}

rf_status rf_mlp_forward(rf_mlp m, const uint16_t *x_dev, int batch, float *out_dev, void *stream)
{
    RF_CHECK_ARG(m && x_dev && out_dev, "null pointer");
    RF_CHECK_ARG(batch >= 1 && batch <= m->max_batch, "batch outside [1, max_batch]");
    return mlp_forward(m, reinterpret_cast<const bf16 *>(x_dev), batch, out_dev, 0, (cudaStream_t)stream);
}

rf_status rf_mlp_gradient(rf_mlp m, const uint16_t *x_all_dev, const float *y_all_dev, const int *idx_dev, int n_all,
                          int batch, float *grad_dev, float *loss_dev, float *out_dev, void *stream)
{
    RF_CHECK_ARG(m && x_all_dev && y_all_dev, "null pointer");
    RF_CHECK_ARG(batch >= 8 && batch <= m->max_batch && batch % 8 == 0 && batch <= RF_MLP_MAX_TRAIN_BATCH,
                 "training batch must be a multiple of 8 in [8, min(max_batch, RF_MLP_MAX_TRAIN_BATCH)]");
    RF_CHECK_ARG(n_all >= 1 && (idx_dev || n_all >= batch), "dataset rows");
    cudaStream_t s = (cudaStream_t)stream;
    rf_status st = mlp_gradient(m, reinterpret_cast<const bf16 *>(x_all_dev), y_all_dev, idx_dev, n_all, batch, s);
    if (st != RF_OK)
        return st;
    if (grad_dev)
        RF_CUDA(cudaMemcpyAsync(grad_dev, m->grad, (size_t)m->L.total * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (loss_dev)
        RF_CUDA(cudaMemcpyAsync(loss_dev, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (out_dev)
        RF_CUDA(cudaMemcpyAsync(out_dev, m->out, (size_t)batch * RF_MLP_OUT * sizeof(float), cudaMemcpyDeviceToDevice,
                                s));
    return RF_OK;
}

rf_status rf_mlp_train_step(rf_mlp m, const uint16_t *x_all_dev, const float *y_all_dev, const int *idx_dev, int n_all,
                            int batch, float lr, float *loss_dev, void *stream)
{
    rf_status st = rf_mlp_gradient(m, x_all_dev, y_all_dev, idx_dev, n_all, batch, nullptr, loss_dev, nullptr, stream);
    if (st != RF_OK)
        return st;
    RF_CHECK_ARG(lr >= 0.f, "negative learning rate");
    return mlp_adam(m, 1, lr, (cudaStream_t)stream);
}

rf_status rf_mlp_evaluate(rf_mlp m, const uint16_t *x_all_dev, const float *y_all_dev, const int *idx_dev,
                          int n_all, int n_rows, float *mu_dev, double *stats_dev, void *stream)
{
    RF_CHECK_ARG(m && x_all_dev && y_all_dev, "null pointer");
    RF_CHECK_ARG(n_rows >= 1 && n_all >= 1 && (idx_dev || n_rows <= n_all), "dataset rows");
    cudaStream_t s = (cudaStream_t)stream;
    RF_CUDA(cudaMemsetAsync(m->eval_acc, 0, EVAL_STATS * sizeof(double), s));
    const bf16 *x_all = reinterpret_cast<const bf16 *>(x_all_dev);
    for (int r0 = 0; r0 < n_rows; r0 += m->max_batch) {
        const int B = std::min(m->max_batch, n_rows - r0);
        // rows idx[r0 ..] (or r0 ..) into the batch buffers; the transposed copy is unused here
        if (idx_dev) {
            gather_kernel<<<B, 256, 0, s>>>(x_all, y_all_dev, idx_dev + r0, n_all, B, m->x, m->xt, m->y, m->err);
        } else {
            gather_kernel<<<B, 256, 0, s>>>(x_all + (size_t)r0 * RF_MLP_IN, y_all_dev + (size_t)r0 * 6, nullptr,
                                            n_all - r0, B, m->x, m->xt, m->y, m->err);
        }
        RF_CUDA(cudaGetLastError());
        rf_status st = mlp_forward(m, m->x, B, m->out, 0, s);
        if (st != RF_OK)
            return st;
        eval_kernel<<<1, 256, 0, s>>>(m->out, m->x, m->y, B, r0, mu_dev, m->eval_acc);
        RF_CUDA(cudaGetLastError());
    }
    eval_finish_kernel<<<1, 32, 0, s>>>(m->eval_acc, n_rows, m->eval_acc + EVAL_STATS);
    RF_CUDA(cudaGetLastError());
    if (stats_dev)
        RF_CUDA(cudaMemcpyAsync(stats_dev, m->eval_acc + EVAL_STATS, EVAL_STATS * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
    return RF_OK;
}

rf_status rf_mlp_calibrate_scale(rf_mlp m, const uint16_t *x_all_dev, const float *y_all_dev, const int *idx_dev,
                                 int n_all, int n_rows, float k_host[6], void *stream)
{
    RF_CHECK_ARG(m && k_host, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    rf_status st = rf_mlp_evaluate(m, x_all_dev, y_all_dev, idx_dev, n_all, n_rows, nullptr, nullptr, stream);
    if (st != RF_OK)
        return st;
    const LayerTable &L = m->L;
    float *b4 = m->theta + L.w_off[3] + L.out[3] * L.in[3];
    calibrate_kernel<<<1, 32, 0, s>>>(m->eval_acc + EVAL_STATS, b4 + 6, m->eval_k);
    RF_CUDA(cudaGetLastError());
    RF_CUDA(cudaMemcpyAsync(k_host, m->eval_k, 6 * sizeof(float), cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaStreamSynchronize(s));
    return RF_OK;
}

rf_status rf_mlp_status(rf_mlp m)
{
    RF_CHECK_ARG(m != nullptr, "null network");
    int h = 0;
    RF_CUDA(cudaDeviceSynchronize());
    RF_CUDA(cudaMemcpy(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost));
    RF_CUDA(cudaMemset(m->err, 0, sizeof(int)));
    if (h != 0)
        set_error("rf_mlp: device status %d", h);
    return h;
}

}  // extern "C"
