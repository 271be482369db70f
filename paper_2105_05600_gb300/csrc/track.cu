// track.cu -- standalone steps of the tracking path behind the C ABI:
//
//  rf_depth_to_points   Eq. unproj + stride downsampling (Sec. 4)
//  rf_overlap_mask      Eq. validness
//  fitness_eval         Eq. normallh for one PST placement: one warp scores 32
//                       particles (one per lane) over a chunk of points staged in
//                       shared memory, then a fixed-order reduction over chunks
//  fitness_eval_noalloc the same without device allocation
//
// The persistent per-frame kernel that runs every PFO iteration is in pfo.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "fitness.cuh"

namespace rf {

template <int DT, int MODE>
__global__ void __launch_bounds__(FIT_THREADS) fitness_kernel(VolumeDesc V, const float4 *pts, int m, FitParams fp,
                                                              Split sp, double *part_S, int *part_n)
{
    extern __shared__ float4 smem_pts[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int warp_global = blockIdx.x * FIT_WARPS + w;
    fitness_units<DT, MODE, false>(V, pts, m, fp, sp, part_S, part_n, smem_pts, warp_global, gridDim.x * FIT_WARPS,
                                   lane, w);
}

__global__ void fitness_finish_kernel(int n, int n_chunks, const double *part_S, const int *part_n, int m, float tau,
                                      int normalize, float *rho, double *sumsq, int *nvalid)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    double S;
    int nv;
    particle_total(part_S, part_n, n, n_chunks, i, false, S, nv);
    rho[i] = fitness_rho(S, m, tau, normalize != 0);
    if (sumsq)
        sumsq[i] = S;
    if (nvalid)
        nvalid[i] = nv;
}

// ------------------------------------------------------------------ depth / overlap kernels
__global__ void depth_to_points_kernel(const float *depth, Intr K, int stride, int nw, int m, float4 *pts)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m)
        return;
    float4 p;
    unproject_point(depth, K, stride, nw, j, p);
    pts[j] = p;
}

__global__ void overlap_kernel(const float4 *pts, int m, const float *prev_depth, Intr K, Pose cur, Pose prev,
                               float cell_m, uint8_t *mask, int *count)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    float Rc[9], Rp[9];
    quat_rot(cur.q, Rc);
    quat_rot(prev.q, Rp);
    bool in = false;
    if (j < m) {
        in = overlap_test(pts[j], Rc, cur.t, Rp, prev.t, prev_depth, K, cell_m);
        mask[j] = in ? 1 : 0;
    }
    if (count) {
        unsigned b = __ballot_sync(0xffffffffu, in);
        if ((threadIdx.x & 31) == 0 && b)
            atomicAdd(count, __popc(b));
    }
}

// ------------------------------------------------------------------ kernel tables
using FitFn = void (*)(VolumeDesc, const float4 *, int, FitParams, Split, double *, int *);
template <int DT> static FitFn fit_fn(int mode)
{
    switch (mode) {
    case 0:
        return fitness_kernel<DT, 0>;
    case 1:
        return fitness_kernel<DT, 1>;
    case 2:
        return fitness_kernel<DT, 2>;
    default:
        return fitness_kernel<DT, 3>;
    }
}
static FitFn fit_fn(int dtype, int mode)
{
    return dtype == RF_F32 ? fit_fn<RF_F32>(mode) : dtype == RF_F16 ? fit_fn<RF_F16>(mode) : fit_fn<RF_I16>(mode);
}
static int mode_of(int flags) { return ((flags & RF_NEAREST) ? 1 : 0) | ((flags & RF_COMPENSATED) ? 0 : 2); }



}  // namespace rf

using namespace rf;

extern "C" {

rf_status rf_depth_to_points(const float *depth_dev, const rf_intrinsics *K, int stride, float *points_dev,
                             void *stream)
{
    RF_CHECK_ARG(depth_dev && K && points_dev, "null pointer");
    RF_CHECK_ARG(stride >= 1 && K->width > 0 && K->height > 0, "bad size");
    const int nw = (K->width + stride - 1) / stride, nh = (K->height + stride - 1) / stride;
    const int m = nw * nh;
    depth_to_points_kernel<<<(m + 255) / 256, 256, 0, (cudaStream_t)stream>>>(depth_dev, to_intr(*K), stride, nw, m,
                                                                             (float4 *)points_dev);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

rf_status rf_overlap_mask(const float *points_dev, int m, const float *prev_depth_dev, const rf_intrinsics *K,
                          const rf_pose *pose_cur, const rf_pose *pose_prev, float cell_extent, uint8_t *mask_dev,
                          int *count_dev, void *stream)
{
    RF_CHECK_ARG(points_dev && prev_depth_dev && K && pose_cur && pose_prev && mask_dev, "null pointer");
    RF_CHECK_ARG(m >= 0, "negative size");
    RF_CHECK_ARG(cell_extent >= 0.f && isfinite(cell_extent), "cell_extent must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    if (count_dev)
        RF_CUDA(cudaMemsetAsync(count_dev, 0, sizeof(int), s));
    if (m == 0)
        return RF_OK;
    overlap_kernel<<<(m + 255) / 256, 256, 0, s>>>((const float4 *)points_dev, m, prev_depth_dev, to_intr(*K),
                                                   to_pose(*pose_cur), to_pose(*pose_prev), cell_extent, mask_dev,
                                                   count_dev);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

rf_status fitness_eval(rf_volume v, const float *points_dev, int m, const float *pst_dev, int n,
                       const rf_pose *centre, const float scale[6], const rf_params *p, float *rho_dev,
                       double *sumsq_dev, int *nvalid_dev, void *stream)
{
    RF_CHECK_ARG(v && points_dev && pst_dev && centre && scale && p && rho_dev, "null pointer");
    RF_CHECK_ARG(m >= 1 && n >= 1, "m and n must be >= 1");
    RF_CHECK_ARG(p->tau > 0.f, "tau must be positive");
    cudaStream_t s = (cudaStream_t)stream;
    const int mode = mode_of(p->flags);
    FitFn fn = fit_fn(v->d.dtype, mode);
    const size_t smem = (size_t)FIT_WARPS * CHUNK_MAX * sizeof(float4);
    RF_CUDA(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, FIT_THREADS, smem));
    const int grid = std::max(1, per_sm) * sm_count();
    const int total_warps = grid * FIT_WARPS;
    const int max_chunks = max_chunks_for(n, m, total_warps);
    const Split sp = make_split(n, m, total_warps, max_chunks);
    const size_t need = (size_t)sp.n_chunks * n * (sizeof(double) + sizeof(int));
    if (need > v->scratch_bytes) {
        RF_CUDA(cudaStreamSynchronize(s));
        cudaFree(v->scratch);
        v->scratch = nullptr;
        v->scratch_bytes = 0;
        RF_CUDA(cudaMalloc(&v->scratch, need));
        v->scratch_bytes = need;
    }
    double *part_S = (double *)v->scratch;
    int *part_n = (int *)(part_S + (size_t)sp.n_chunks * n);
    FitParams fp;
    fp.pst = pst_dev;
    fp.n = n;
    fp.ld = n;
    fp.c = to_pose(*centre);
    for (int d = 0; d < 6; ++d)
        fp.r[d] = scale[d];
    fp.l1 = (p->flags & RF_L1) != 0;
    fp.right_mult = (p->flags & RF_RIGHT_MULT) != 0;
    fn<<<grid, FIT_THREADS, smem, s>>>(v->d, (const float4 *)points_dev, m, fp, sp, part_S, part_n);
    RF_CUDA(cudaGetLastError());
    fitness_finish_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, sp.n_chunks, part_S, part_n, m, p->tau,
                                                          (p->flags & RF_NORMALIZE) != 0, rho_dev, sumsq_dev,
                                                          nvalid_dev);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free fitness
// fitness_eval keeps its per-(chunk, particle) partial sums in a buffer that the
// volume handle grows with cudaMalloc on first use, which synchronises and
// allocates.  fitness_eval_noalloc takes them from this fixed, file-scope device
// array instead.  The array is part of the library image, so every GPU that
// loads the library holds these 32 MiB until the process exits.
namespace rf {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// In host code g_noalloc_scratch names a host-side stand-in, not device memory:
// the device address is looked up once per device (with that device current)
// and cached here.
constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_dev_ptr[NOALLOC_MAX_DEVICES];

static rf_status noalloc_scratch(void **out)
{
    int dev = 0;
    RF_CUDA(cudaGetDevice(&dev));
    RF_CHECK_ARG(dev >= 0 && dev < NOALLOC_MAX_DEVICES, "device ordinal beyond the supported range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_dev_ptr[dev] == nullptr) {
        void *p = nullptr;
        RF_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_dev_ptr[dev] = p;
    }
    *out = g_noalloc_dev_ptr[dev];
    return RF_OK;
}

}  // namespace rf

extern "C" rf_status fitness_eval_noalloc(rf_volume v, const float *points_dev, int m, const float *pst_dev, int n,
                                          const rf_pose *centre, const float scale[6], const rf_params *p,
                                          float *rho_dev, double *sumsq_dev, int *nvalid_dev, void *stream)
{
    RF_CHECK_ARG(v && points_dev && pst_dev && centre && scale && p && rho_dev, "null pointer");
    RF_CHECK_ARG(m >= 1 && n >= 1, "m and n must be >= 1");
    RF_CHECK_ARG(p->tau > 0.f, "tau must be positive");
    const size_t per_chunk = (size_t)n * (sizeof(double) + sizeof(int));
    const size_t min_chunks = ((size_t)m + CHUNK_MAX - 1) / CHUNK_MAX;
    RF_CHECK_ARG(min_chunks * per_chunk <= NOALLOC_SCRATCH_BYTES,
                 "ceil(m / 256) * n * 12 bytes exceeds the 32 MiB static scratch of fitness_eval_noalloc");
    cudaStream_t s = (cudaStream_t)stream;
    void *scratch = nullptr;
    rf_status st = noalloc_scratch(&scratch);
    if (st != RF_OK)
        return st;
    const int mode = mode_of(p->flags);
    FitFn fn = fit_fn(v->d.dtype, mode);
    const size_t smem = (size_t)FIT_WARPS * CHUNK_MAX * sizeof(float4);
    RF_CUDA(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, FIT_THREADS, smem));
    const int grid = std::max(1, per_sm) * sm_count();
    const int total_warps = grid * FIT_WARPS;
    const int cap_chunks = (int)std::min<size_t>(NOALLOC_SCRATCH_BYTES / per_chunk, 1 << 30);
    const Split sp = make_split(n, m, total_warps, std::min(max_chunks_for(n, m, total_warps), cap_chunks));
    // every (chunk, particle) slot below n_chunks * n is written by the fitness
    // kernel before the finishing kernel reads it: nothing needs clearing
    double *part_S = (double *)scratch;
    int *part_n = (int *)(part_S + (size_t)sp.n_chunks * n);
    FitParams fp;
    fp.pst = pst_dev;
    fp.n = n;
    fp.ld = n;
    fp.c = to_pose(*centre);
    for (int d = 0; d < 6; ++d)
        fp.r[d] = scale[d];
    fp.l1 = (p->flags & RF_L1) != 0;
    fp.right_mult = (p->flags & RF_RIGHT_MULT) != 0;
    fn<<<grid, FIT_THREADS, smem, s>>>(v->d, (const float4 *)points_dev, m, fp, sp, part_S, part_n);
    RF_CUDA(cudaGetLastError());
    fitness_finish_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, sp.n_chunks, part_S, part_n, m, p->tau,
                                                          (p->flags & RF_NORMALIZE) != 0, rho_dev, sumsq_dev,
                                                          nvalid_dev);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}
