// volume.cu -- TSDF volume handles and volumetric fusion (tsdf_integrate).
//
// Layout in HBM: 8x8x8 voxel bricks (512 values = 1 KiB for int16/half, 2 KiB
// for float) so that a 2x2x2 trilinear neighbourhood touches one or few 32-byte
// sectors; uint8 weights in the same layout.  A 512^3 int16 volume is 256 MiB
// of values plus 128 MiB of weights.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "rf_measure.h"

namespace rf {

static thread_local std::string g_last_error;

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

rf_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return e == cudaErrorMemoryAllocation ? RF_ERR_NOMEM : RF_ERR_CUDA;
}

static size_t dtype_size(int dt) { return dt == RF_F32 ? 4 : 2; }

// ------------------------------------------------------------------ kernels
// Fill every voxel with the unobserved sentinel and weight 0.
__global__ void reset_kernel(uint32_t *vals32, size_t n_words, uint32_t pattern, uint8_t *w, size_t n_vox)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = i; k < n_words; k += stride)
        vals32[k] = pattern;
    for (size_t k = i; k < n_vox; k += stride)
        w[k] = 0;
}

// Linear x-fastest <-> brick layout.  One thread per voxel; T is the raw code
// type (uint32_t for float, uint16_t for half / int16).  Without uploaded
// weights a voxel gets weight 1 unless its code is the unobserved sentinel.
__device__ __forceinline__ bool code_unobserved(uint32_t c, int dtype)
{
    if (dtype == RF_F32)
        return (c & 0x7f800000u) == 0x7f800000u && (c & 0x007fffffu) != 0u;
    if (dtype == RF_F16)
        return (c & 0x7c00u) == 0x7c00u && (c & 0x03ffu) != 0u;
    return (c & 0xffffu) == 0x8000u;
}

template <typename T>
__global__ void linear_to_brick(VolumeDesc V, const T *lin, const uint8_t *wlin, T *vals, uint8_t *w)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t n = (size_t)V.dim[0] * V.dim[1] * V.dim[2];
    if (i >= n)
        return;
    int x = (int)(i % V.dim[0]);
    int y = (int)((i / V.dim[0]) % V.dim[1]);
    int z = (int)(i / ((size_t)V.dim[0] * V.dim[1]));
    size_t b = brick_index(V, x, y, z);
    T v = lin[i];
    vals[b] = v;
    if (wlin)
        w[b] = wlin[i];
    else
        w[b] = code_unobserved((uint32_t)v, V.dtype) ? 0 : 1;
}

template <typename T> __global__ void brick_to_linear(VolumeDesc V, const T *vals, const uint8_t *w, T *lin, uint8_t *wlin)
{
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t n = (size_t)V.dim[0] * V.dim[1] * V.dim[2];
    if (i >= n)
        return;
    int x = (int)(i % V.dim[0]);
    int y = (int)((i / V.dim[0]) % V.dim[1]);
    int z = (int)(i / ((size_t)V.dim[0] * V.dim[1]));
    size_t b = brick_index(V, x, y, z);
    lin[i] = vals[b];
    if (wlin)
        wlin[i] = w[b];
}

template <int DT> struct Enc;
template <> struct Enc<RF_F32> {
    static __device__ __forceinline__ bool unobserved(float v) { return isnan(v); }
    static __device__ __forceinline__ bool same(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }
    static __device__ __forceinline__ float dec(float v) { return v; }
    static __device__ __forceinline__ float enc(float f) { return f; }
};
template <> struct Enc<RF_F16> {
    static __device__ __forceinline__ bool unobserved(__half v) { return __hisnan(v); }
    static __device__ __forceinline__ bool same(__half a, __half b) { return __half_as_ushort(a) == __half_as_ushort(b); }
    static __device__ __forceinline__ float dec(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half enc(float f) { return __float2half_rn(f); }
};
template <> struct Enc<RF_I16> {
    static __device__ __forceinline__ bool unobserved(int16_t v) { return v == I16_UNOBSERVED; }
    static __device__ __forceinline__ bool same(int16_t a, int16_t b) { return a == b; }
    static __device__ __forceinline__ float dec(int16_t v) { return (float)v * (1.0f / I16_SCALE); }
    static __device__ __forceinline__ int16_t enc(float f)
    {
        int c = __float2int_rn(f * I16_SCALE);
        c = max(-32767, min(32767, c));
        return (int16_t)c;
    }
};

// Conservative test of whether brick (bx, by, bz) can hold a voxel that the
// per-voxel fusion test accepts: the sphere around the brick's voxel centres
// (radius 3.5 sqrt(3) voxels, plus a margin far above FP32 rounding) must meet
// every half-space whose intersection contains the accepted voxels -- in front
// of the camera (z > 0), no deeper than z_max + trunc (sdf = D - z >= -trunc
// with D <= z_max), and re-projecting into the image (the rounded pixel lies in
// [0, W) x [0, H), i.e. -1/2 <= u < W - 1/2 and likewise v).  A brick that
// fails any test has no voxel to update, so skipping it changes nothing.
__device__ __forceinline__ bool brick_may_update(const VolumeDesc &V, int bx, int by, int bz, const float R[9],
                                                 const float t[3], const Intr &K)
{
    const float h = V.voxel;
    const float wx = V.origin[0] + h * (float)(bx * BRICK + BRICK / 2) - t[0];
    const float wy = V.origin[1] + h * (float)(by * BRICK + BRICK / 2) - t[1];
    const float wz = V.origin[2] + h * (float)(bz * BRICK + BRICK / 2) - t[2];
    const float px = R[0] * wx + R[3] * wy + R[6] * wz;
    const float py = R[1] * wx + R[4] * wy + R[7] * wz;
    const float pz = R[2] * wx + R[5] * wy + R[8] * wz;
    const float rad = h * (0.5f * (float)(BRICK - 1) * 1.7320508f + 0.05f);
    if (pz + rad <= 0.f || pz - rad > K.z_max + V.trunc)
        return false;
    const float l0 = K.cx + 0.5f, r0 = (float)K.width - 0.5f - K.cx;
    const float t0 = K.cy + 0.5f, b0 = (float)K.height - 0.5f - K.cy;
    if (K.fx * px + l0 * pz < -rad * sqrtf(K.fx * K.fx + l0 * l0))
        return false;
    if (r0 * pz - K.fx * px < -rad * sqrtf(K.fx * K.fx + r0 * r0))
        return false;
    if (K.fy * py + t0 * pz < -rad * sqrtf(K.fy * K.fy + t0 * t0))
        return false;
    if (b0 * pz - K.fy * py < -rad * sqrtf(K.fy * K.fy + b0 * b0))
        return false;
    return true;
}

// Work-list entries carry brick coordinates, so the fusion kernels index a
// brick without integer division: bx | by << 10 | bz << 20 (at most 256 bricks
// per axis).
__device__ __forceinline__ int brick_code(int bx, int by, int bz) { return bx | (by << 10) | (bz << 20); }
__device__ __forceinline__ void brick_decode(int e, int &bx, int &by, int &bz)
{
    bx = e & 1023;
    by = (e >> 10) & 1023;
    bz = e >> 20;
}

__device__ __forceinline__ void load_pose(Pose &T, const float *pose_dev)
{
    if (pose_dev) {
        for (int a = 0; a < 4; ++a)
            T.q[a] = pose_dev[a];
        for (int a = 0; a < 3; ++a)
            T.t[a] = pose_dev[4 + a];
    }
}

// Frustum culling, one thread per brick: the bricks that brick_may_update
// accepts are appended to the visible list (one atomic per warp).  The order of
// the list is immaterial: each listed brick is updated by one CTA, alone.  The
// pose comes by value, or from device memory (pose_dev != NULL, written by the
// tracker earlier on the stream); a non-zero *status_dev lists nothing, so the
// fusion that follows changes nothing.
__global__ void __launch_bounds__(256) cull_bricks_kernel(VolumeDesc V, Intr K, Pose T, const float *pose_dev,
                                                          const int *status_dev, int nbricks)
{
    if (status_dev && *((volatile const int *)status_dev) != 0)
        return;
    load_pose(T, pose_dev);
    float R[9];
    quat_rot(T.q, R);
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int bx = b % V.nb[0], by = (b / V.nb[0]) % V.nb[1], bz = b / (V.nb[0] * V.nb[1]);
    const bool vis = b < nbricks && brick_may_update(V, bx, by, bz, R, T.t, K);
    const unsigned m = __ballot_sync(0xffffffffu, vis);
    if (m == 0u)
        return;  // warp-uniform
    const int lane = threadIdx.x & 31;
    unsigned base = 0u;
    if (lane == 0) {
        base = atomicAdd(&V.fuse_count[0], (unsigned)__popc(m));
        atomicAdd(&V.counters[1], (unsigned long long)__popc(m));
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if (vis)
        V.fuse_list[base + __popc(m & ((1u << lane) - 1u))] = brick_code(bx, by, bz);
}

// Projective TSDF fusion (Sec. 3 overview; Curless & Levoy 1996, KinectFusion
// 2011) of the bricks on the visible list.  A persistent grid walks the list,
// one 8x8x8 brick per CTA step with one thread per voxel, so value and weight
// accesses are contiguous 1 KiB (or 2 KiB) runs.  Per updated voxel 2+2 B of
// value (4+4 for float) and 1+1 B of weight plus the depth read.  A brick whose
// stored value codes changed puts the bricks whose cells read it (itself and
// its lower neighbours, b - {0,1}^3) on the repack list, each once.
template <int DT>
__global__ void __launch_bounds__(512, 4) integrate_kernel(VolumeDesc V, const float *__restrict__ depth, Intr K, Pose T,
                                                        const float *pose_dev, int w_max, int nbricks)
{
    using S = typename Storage<DT>::T;
    load_pose(T, pose_dev);
    float R[9];
    quat_rot(T.q, R);
    const int l = threadIdx.x;
    const int n_visible = (int)V.fuse_count[0];
    for (int i = blockIdx.x; i < n_visible; i += gridDim.x) {
        int bx, by, bz;
        brick_decode(V.fuse_list[i], bx, by, bz);
        const int b = bx + V.nb[0] * (by + V.nb[1] * bz);
        const int x = bx * BRICK + (l & 7), y = by * BRICK + ((l >> 3) & 7), z = bz * BRICK + (l >> 6);
        bool updated = false, changed = false;
        do {
            const float pwx = V.origin[0] + V.voxel * ((float)x + 0.5f) - T.t[0];
            const float pwy = V.origin[1] + V.voxel * ((float)y + 0.5f) - T.t[1];
            const float pwz = V.origin[2] + V.voxel * ((float)z + 0.5f) - T.t[2];
            // camera frame: R^T (p - t)
            const float cx = R[0] * pwx + R[3] * pwy + R[6] * pwz;
            const float cy = R[1] * pwx + R[4] * pwy + R[7] * pwz;
            const float cz = R[2] * pwx + R[5] * pwy + R[8] * pwz;
            if (!(cz > 0.f))
                break;
            const float u = floorf(K.fx * cx / cz + K.cx + 0.5f);
            const float v = floorf(K.fy * cy / cz + K.cy + 0.5f);
            if (!(u >= 0.f && u < (float)K.width && v >= 0.f && v < (float)K.height))
                break;
            const float D = __ldg(&depth[(size_t)v * K.width + (size_t)u]);
            if (!depth_valid(D, K))
                break;
            const float sdf = D - cz;
            if (sdf < -V.trunc)
                break;
            const float f = fminf(1.f, sdf / V.trunc);
            const size_t idx = (size_t)b * BRICK_VOX + l;
            S *vals = reinterpret_cast<S *>(V.values);
            const S old = vals[idx];
            int w_old = V.weights[idx];
            float F_old = 0.f;
            if (Enc<DT>::unobserved(old))
                w_old = 0;
            else
                F_old = Enc<DT>::dec(old);
            const float F_new = ((float)w_old * F_old + f) / (float)(w_old + 1);
            const S code = Enc<DT>::enc(F_new);
            changed = !Enc<DT>::same(code, old);
            vals[idx] = code;
            V.weights[idx] = (uint8_t)min(w_old + 1, w_max);
            updated = true;
        } while (false);
        // the cells hold values only, so a weight-only update needs no repack
        const int n_updated = __syncthreads_count(updated);
        const int n_changed = __syncthreads_count(changed);
        if (n_changed && l < 8) {
            const int nx = bx - (l & 1), ny = by - ((l >> 1) & 1), nz = bz - (l >> 2);
            if (nx >= 0 && ny >= 0 && nz >= 0) {
                const int nbk = nx + V.nb[0] * (ny + V.nb[1] * nz);
                const uint32_t bit = 1u << (nbk & 31);
                if (!(atomicOr(&V.need[nbk >> 5], bit) & bit))
                    V.fuse_list[nbricks + (int)atomicAdd(&V.fuse_count[1], 1u)] = brick_code(nx, ny, nz);
            }
        }
        if (l == 0)
            atomicAdd(&V.counters[0], (unsigned long long)n_updated);
    }
}

// Packed trilinear cells of one brick (one thread per cell) and its class.
// Cell i reads voxels i + {0,1}^3; cells on the upper faces of the volume are
// never sampled and copy the nearest voxels.  The CTA first stages the 9x9x9
// voxels its cells read in shared memory: the brick itself (one contiguous
// load per thread) and the 217 voxels of its upper x, y and z faces, edges and
// corner (threads 0..216), each clamped to the volume like the corners.
constexpr int HALO = BRICK + 1;
template <int DT>
__device__ __forceinline__ void pack_brick(const VolumeDesc &V, int b, int bx, int by, int bz, int l)
{
    using S = typename Storage<DT>::T;
    __shared__ S tile[HALO * HALO * HALO];  // [z][y][x]
    const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
    const S *vals = reinterpret_cast<const S *>(V.values);
    tile[(lz * HALO + ly) * HALO + lx] = vals[(size_t)b * BRICK_VOX + l];
    if (l < 217) {
        int hx, hy, hz;
        if (l < 64) {
            hx = 8, hy = l & 7, hz = l >> 3;
        } else if (l < 128) {
            hx = l & 7, hy = 8, hz = (l - 64) >> 3;
        } else if (l < 192) {
            hx = l & 7, hy = (l - 128) >> 3, hz = 8;
        } else if (l < 200) {
            hx = 8, hy = 8, hz = l - 192;
        } else if (l < 208) {
            hx = 8, hy = l - 200, hz = 8;
        } else if (l < 216) {
            hx = l - 208, hy = 8, hz = 8;
        } else {
            hx = 8, hy = 8, hz = 8;
        }
        const int xx = min(bx * BRICK + hx, V.dim[0] - 1), yy = min(by * BRICK + hy, V.dim[1] - 1),
                  zz = min(bz * BRICK + hz, V.dim[2] - 1);
        tile[(hz * HALO + hy) * HALO + hx] = vals[brick_index(V, xx, yy, zz)];
    }
    __syncthreads();
    // (in the last brick along an axis the face holds the clamped voxel, the
    // brick's own last layer, so cells on the volume's upper faces need no test)
    S c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        c[k] = tile[((lz + (k >> 2)) * HALO + ly + ((k >> 1) & 1)) * HALO + lx + (k & 1)];
    const size_t rec = (size_t)b * BRICK_VOX + l;
    bool all_free = true, any_unobserved = false;
    if (DT == RF_F32) {
        float4 *out = reinterpret_cast<float4 *>(V.cells) + 2 * rec;
        const float *f = reinterpret_cast<const float *>(c);
        out[0] = make_float4(f[0], f[1], f[2], f[3]);
        out[1] = make_float4(f[4], f[5], f[6], f[7]);
        for (int k = 0; k < 8; ++k) {
            all_free &= f[k] == 1.0f;
            any_unobserved |= isnan(f[k]);
        }
    } else {
        const uint16_t *h = reinterpret_cast<const uint16_t *>(c);
        // int16 cells are stored biased (c + 32768) so that decoding needs no sign fix
        const uint16_t bias = DT == RF_I16 ? 0x8000u : 0u;
        const uint16_t one = DT == RF_I16 ? 32767u : 0x3C00u;
        for (int k = 0; k < 8; ++k) {
            all_free &= h[k] == one;
            any_unobserved |= DT == RF_I16 ? h[k] == 0x8000u : ((h[k] & 0x7C00u) == 0x7C00u && (h[k] & 0x03FFu));
        }
        uint4 r;
        r.x = (uint32_t)(uint16_t)(h[0] ^ bias) | ((uint32_t)(uint16_t)(h[1] ^ bias) << 16);
        r.y = (uint32_t)(uint16_t)(h[2] ^ bias) | ((uint32_t)(uint16_t)(h[3] ^ bias) << 16);
        r.z = (uint32_t)(uint16_t)(h[4] ^ bias) | ((uint32_t)(uint16_t)(h[5] ^ bias) << 16);
        r.w = (uint32_t)(uint16_t)(h[6] ^ bias) | ((uint32_t)(uint16_t)(h[7] ^ bias) << 16);
        if (DT == RF_I16 && any_unobserved)
            r = make_uint4(0u, 0u, 0u, 0u);  // one zero corner test then flags the whole cell invalid
        reinterpret_cast<uint4 *>(V.cells)[rec] = r;
    }
    // brick class: constant free space, all cells invalid, or mixed
    const bool every_free = __syncthreads_and(all_free) != 0;
    const bool every_invalid = __syncthreads_and(any_unobserved) != 0;
    if (l == 0)
        V.brick_class[b] = every_free ? CELLS_FREE : (every_invalid ? CELLS_INVALID : CELLS_MIXED);
}


// Packed cells of the bricks on the repack list, or of every brick (`all`, after
// an upload or a reset).  A persistent grid walks the list, one brick per CTA step.
template <int DT>
__global__ void __launch_bounds__(512) pack_cells_kernel(VolumeDesc V, int all, int nbricks)
{
    const int l = threadIdx.x;
    const int n = all ? nbricks : (int)V.fuse_count[1];
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        int bx, by, bz;
        if (all) {  // uniform: after an upload or a reset only
            bx = i % V.nb[0];
            by = (i / V.nb[0]) % V.nb[1];
            bz = i / (V.nb[0] * V.nb[1]);
        } else {
            brick_decode(V.fuse_list[nbricks + i], bx, by, bz);
        }
        pack_brick<DT>(V, bx + V.nb[0] * (by + V.nb[1] * bz), bx, by, bz, l);
        if (l == 0)
            atomicAdd(&V.counters[2], 1ull);
    }
}

// Bytes of the fusion bookkeeping cleared before each fusion: the two list
// counts (padded to 16 B) and the repack bit set.
static size_t fuse_flags_bytes(int nbricks) { return 16 + (size_t)((nbricks + 31) / 32) * 4; }

// Rebuild the packed cells after the values changed: every brick (all), else
// the repack list of the fusion that ran last on the stream.  Stream-ordered,
// capturable.
rf_status pack_cells(const VolumeDesc &V, int all, cudaStream_t s)
{
    const int nbricks = V.nb[0] * V.nb[1] * V.nb[2];
    const int grid = V.fuse_grid[1];
    switch (V.dtype) {
    case RF_F32:
        pack_cells_kernel<RF_F32><<<grid, 512, 0, s>>>(V, all, nbricks);
        break;
    case RF_F16:
        pack_cells_kernel<RF_F16><<<grid, 512, 0, s>>>(V, all, nbricks);
        break;
    default:
        pack_cells_kernel<RF_I16><<<grid, 512, 0, s>>>(V, all, nbricks);
        break;
    }
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

// One fusion: clear the lists, cull, update the visible bricks, repack the
// bricks that read a changed value.  Four stream-ordered operations, no host
// synchronisation (capturable).
static rf_status integrate_any(const VolumeDesc &V, const float *depth, const Intr &K, const Pose &T,
                               const float *pose_dev, const int *status_dev, cudaStream_t s)
{
    const int nbricks = V.nb[0] * V.nb[1] * V.nb[2];
    RF_CUDA(cudaMemsetAsync(V.fuse_count, 0, fuse_flags_bytes(nbricks), s));
    cull_bricks_kernel<<<(nbricks + 255) / 256, 256, 0, s>>>(V, K, T, pose_dev, status_dev, nbricks);
    RF_CUDA(cudaGetLastError());
    const int grid = V.fuse_grid[0];
    switch (V.dtype) {
    case RF_F32:
        integrate_kernel<RF_F32><<<grid, 512, 0, s>>>(V, depth, K, T, pose_dev, 255, nbricks);
        break;
    case RF_F16:
        integrate_kernel<RF_F16><<<grid, 512, 0, s>>>(V, depth, K, T, pose_dev, 255, nbricks);
        break;
    default:
        integrate_kernel<RF_I16><<<grid, 512, 0, s>>>(V, depth, K, T, pose_dev, 255, nbricks);
        break;
    }
    RF_CUDA(cudaGetLastError());
    return pack_cells(V, 0, s);
}

// Persistent grids of the fusion kernels for this device and dtype: the CTAs
// that fit at once (512 threads each), at most one per brick.
static rf_status fuse_grids(VolumeDesc &d)
{
    int dev = 0, sms = 0, oi = 0, op = 0;
    RF_CUDA(cudaGetDevice(&dev));
    RF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    switch (d.dtype) {
    case RF_F32:
        RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oi, integrate_kernel<RF_F32>, 512, 0));
        RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&op, pack_cells_kernel<RF_F32>, 512, 0));
        break;
    case RF_F16:
        RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oi, integrate_kernel<RF_F16>, 512, 0));
        RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&op, pack_cells_kernel<RF_F16>, 512, 0));
        break;
    default:
        RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oi, integrate_kernel<RF_I16>, 512, 0));
        RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&op, pack_cells_kernel<RF_I16>, 512, 0));
        break;
    }
    const int nbricks = d.nb[0] * d.nb[1] * d.nb[2];
    d.fuse_grid[0] = std::max(1, std::min(std::max(oi, 1) * sms, nbricks));
    d.fuse_grid[1] = std::max(1, std::min(std::max(op, 1) * sms, nbricks));
    return RF_OK;
}

rf_status launch_integrate(const VolumeDesc &V, const float *depth, const Intr &K, const Pose &T, cudaStream_t s)
{
    return integrate_any(V, depth, K, T, nullptr, nullptr, s);
}

rf_status launch_integrate_dev(const VolumeDesc &V, const float *depth, const Intr &K, const float *pose_dev,
                               const int *status_dev, cudaStream_t s)
{
    Pose T;
    memset(&T, 0, sizeof T);
    return integrate_any(V, depth, K, T, pose_dev, status_dev, s);
}

Pose to_pose(const rf_pose &p)
{
    Pose o;
    for (int i = 0; i < 4; ++i)
        o.q[i] = p.q[i];
    for (int i = 0; i < 3; ++i)
        o.t[i] = p.t[i];
    return o;
}

}  // namespace rf

using namespace rf;

extern "C" {

const char *rf_last_error(void) { return g_last_error.c_str(); }
const char *rf_version(void) { return "librosefusion 0.1 (sm_103a)"; }

rf_status rf_volume_create(int dx, int dy, int dz, float voxel, float trunc, const float origin[3], int dtype,
                           rf_volume *out)
{
    RF_CHECK_ARG(out != nullptr && origin != nullptr, "null pointer");
    *out = nullptr;
    RF_CHECK_ARG(dx > 0 && dy > 0 && dz > 0 && dx % 8 == 0 && dy % 8 == 0 && dz % 8 == 0 && dx <= 2048 &&
                     dy <= 2048 && dz <= 2048,
                 "dims must be positive multiples of 8 up to 2048");
    RF_CHECK_ARG(voxel > 0.f && trunc > 0.f, "voxel and trunc must be positive");
    RF_CHECK_ARG(dtype == RF_F32 || dtype == RF_F16 || dtype == RF_I16, "unknown dtype");
    RF_CHECK_ARG((size_t)dx * dy * dz < ((size_t)1 << 31), "dim_x * dim_y * dim_z must stay below 2^31");
    rf_volume v = new rf_volume_s();
    memset(v, 0, sizeof *v);
    VolumeDesc &d = v->d;
    d.dim[0] = dx;
    d.dim[1] = dy;
    d.dim[2] = dz;
    for (int a = 0; a < 3; ++a) {
        d.nb[a] = d.dim[a] / BRICK;
        d.origin[a] = origin[a];
    }
    d.voxel = voxel;
    d.inv_voxel = 1.0f / voxel;
    d.trunc = trunc;
    for (int a = 0; a < 3; ++a)
        d.goff[a] = -origin[a] / voxel - 0.5f;
    d.dtype = dtype;
    d.cell_stride[0] = BRICK_VOX;
    d.cell_stride[1] = BRICK_VOX * d.nb[0];
    d.cell_stride[2] = BRICK_VOX * d.nb[0] * d.nb[1];
    v->n_vox = (size_t)dx * dy * dz;
    cudaGetDevice(&v->device);
    cudaError_t e = cudaMalloc(&d.values, v->n_vox * dtype_size(dtype));
    if (e == cudaSuccess)
        e = cudaMalloc(&d.weights, v->n_vox);
    if (e == cudaSuccess)
        e = cudaMalloc(&d.cells, v->n_vox * 8 * dtype_size(dtype));
    const int nbricks = (int)(v->n_vox / BRICK_VOX);
    if (e == cudaSuccess)
        e = cudaMalloc(&d.fuse_count, fuse_flags_bytes(nbricks));
    if (e == cudaSuccess) {
        d.need = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(d.fuse_count) + 16);
        e = cudaMalloc(&d.fuse_list, 2 * (size_t)nbricks * sizeof(int));
    }
    if (e == cudaSuccess)
        e = cudaMalloc(&d.brick_class, v->n_vox / BRICK_VOX);
    if (e == cudaSuccess)
        e = cudaMalloc(&d.counters, 3 * sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = cudaMemset(d.counters, 0, 3 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFree(d.values);
        cudaFree(d.weights);
        cudaFree(d.cells);
        cudaFree(d.fuse_count);
        cudaFree(d.fuse_list);
        cudaFree(d.brick_class);
        cudaFree(d.counters);
        delete v;
        return cuda_fail(e, "cudaMalloc(volume)");
    }
    rf_status st = fuse_grids(d);
    if (st == RF_OK)
        st = rf_volume_reset(v, nullptr);
    if (st != RF_OK) {
        rf_volume_destroy(v);
        return st;
    }
    RF_CUDA(cudaDeviceSynchronize());
    *out = v;
    return RF_OK;
}

void rf_volume_destroy(rf_volume v)
{
    if (!v)
        return;
    cudaFree(v->d.values);
    cudaFree(v->d.weights);
    cudaFree(v->d.cells);
    cudaFree(v->d.fuse_count);
    cudaFree(v->d.fuse_list);
    cudaFree(v->d.brick_class);
    cudaFree(v->d.counters);
    cudaFree(v->scratch);
    delete v;
}

rf_status rf_volume_counters(rf_volume v, long long out_host[3], int reset)
{
    RF_CHECK_ARG(v && out_host, "null pointer");
    unsigned long long h[3];
    RF_CUDA(cudaDeviceSynchronize());
    RF_CUDA(cudaMemcpy(h, v->d.counters, sizeof h, cudaMemcpyDeviceToHost));
    for (int i = 0; i < 3; ++i)
        out_host[i] = (long long)h[i];
    if (reset)
        RF_CUDA(cudaMemset(v->d.counters, 0, sizeof h));
    return RF_OK;
}

rf_status rf_volume_reset(rf_volume v, void *stream)
{
    RF_CHECK_ARG(v != nullptr, "null volume");
    uint32_t pattern = v->d.dtype == RF_F32 ? 0x7fc00000u : (v->d.dtype == RF_F16 ? 0x7e007e00u : 0x80008000u);
    size_t words = v->n_vox * dtype_size(v->d.dtype) / 4;
    reset_kernel<<<1024, 256, 0, (cudaStream_t)stream>>>((uint32_t *)v->d.values, words, pattern, v->d.weights,
                                                         v->n_vox);
    RF_CUDA(cudaGetLastError());
    // every packed cell becomes 8 sentinel corners (biased 0 for int16), every
    // brick is classed invalid
    const uint32_t cell_pattern = v->d.dtype == RF_I16 ? 0u : pattern;
    reset_kernel<<<1024, 256, 0, (cudaStream_t)stream>>>((uint32_t *)v->d.cells, 8 * words, cell_pattern,
                                                         nullptr, 0);
    RF_CUDA(cudaGetLastError());
    RF_CUDA(cudaMemsetAsync(v->d.brick_class, CELLS_INVALID, v->n_vox / BRICK_VOX, (cudaStream_t)stream));
    return RF_OK;
}

rf_status rf_volume_info(rf_volume v, int dims[3], float *voxel, float *trunc, float origin[3], int *dtype)
{
    RF_CHECK_ARG(v != nullptr, "null volume");
    for (int a = 0; a < 3; ++a) {
        if (dims)
            dims[a] = v->d.dim[a];
        if (origin)
            origin[a] = v->d.origin[a];
    }
    if (voxel)
        *voxel = v->d.voxel;
    if (trunc)
        *trunc = v->d.trunc;
    if (dtype)
        *dtype = v->d.dtype;
    return RF_OK;
}

rf_status rf_volume_upload(rf_volume v, const void *values_host, const uint8_t *weights_host)
{
    RF_CHECK_ARG(v != nullptr && values_host != nullptr, "null pointer");
    const size_t es = dtype_size(v->d.dtype);
    void *tmp = nullptr;
    uint8_t *wtmp = nullptr;
    RF_CUDA(cudaMalloc(&tmp, v->n_vox * es));
    cudaError_t e = cudaMemcpy(tmp, values_host, v->n_vox * es, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && weights_host) {
        e = cudaMalloc(&wtmp, v->n_vox);
        if (e == cudaSuccess)
            e = cudaMemcpy(wtmp, weights_host, v->n_vox, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        const int threads = 256;
        const unsigned blocks = (unsigned)((v->n_vox + threads - 1) / threads);
        if (v->d.dtype == RF_F32)
            linear_to_brick<uint32_t><<<blocks, threads>>>(v->d, (const uint32_t *)tmp, wtmp,
                                                           (uint32_t *)v->d.values, v->d.weights);
        else
            linear_to_brick<uint16_t><<<blocks, threads>>>(v->d, (const uint16_t *)tmp, wtmp,
                                                           (uint16_t *)v->d.values, v->d.weights);
        e = cudaGetLastError();
        if (e == cudaSuccess && pack_cells(v->d, 1, nullptr) != RF_OK)
            e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaDeviceSynchronize();
    }
    cudaFree(tmp);
    cudaFree(wtmp);
    if (e != cudaSuccess)
        return cuda_fail(e, "rf_volume_upload");
    return RF_OK;
}

rf_status rf_volume_download(rf_volume v, void *values_host, uint8_t *weights_host)
{
    RF_CHECK_ARG(v != nullptr && values_host != nullptr, "null pointer");
    const size_t es = dtype_size(v->d.dtype);
    void *tmp = nullptr;
    uint8_t *wtmp = nullptr;
    RF_CUDA(cudaMalloc(&tmp, v->n_vox * es));
    cudaError_t e = cudaSuccess;
    if (weights_host)
        e = cudaMalloc(&wtmp, v->n_vox);
    if (e == cudaSuccess) {
        const int threads = 256;
        const unsigned blocks = (unsigned)((v->n_vox + threads - 1) / threads);
        if (v->d.dtype == RF_F32)
            brick_to_linear<uint32_t><<<blocks, threads>>>(v->d, (const uint32_t *)v->d.values, v->d.weights,
                                                           (uint32_t *)tmp, wtmp);
        else
            brick_to_linear<uint16_t><<<blocks, threads>>>(v->d, (const uint16_t *)v->d.values, v->d.weights,
                                                           (uint16_t *)tmp, wtmp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(values_host, tmp, v->n_vox * es, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && weights_host)
        e = cudaMemcpy(weights_host, wtmp, v->n_vox, cudaMemcpyDeviceToHost);
    cudaFree(tmp);
    cudaFree(wtmp);
    if (e != cudaSuccess)
        return cuda_fail(e, "rf_volume_download");
    return RF_OK;
}

rf_status tsdf_integrate(rf_volume v, const float *depth_dev, const rf_intrinsics *K, const rf_pose *pose,
                         void *stream)
{
    RF_CHECK_ARG(v != nullptr && depth_dev != nullptr && K != nullptr && pose != nullptr, "null pointer");
    RF_CHECK_ARG(K->width > 0 && K->height > 0, "empty depth image");
    return launch_integrate(v->d, depth_dev, to_intr(*K), to_pose(*pose), (cudaStream_t)stream);
}

rf_status tsdf_integrate_dev(rf_volume v, const float *depth_dev, const rf_intrinsics *K, const float *pose_dev,
                             const int *status_dev, void *stream)
{
    RF_CHECK_ARG(v != nullptr && depth_dev != nullptr && K != nullptr && pose_dev != nullptr, "null pointer");
    RF_CHECK_ARG(K->width > 0 && K->height > 0, "empty depth image");
    return launch_integrate_dev(v->d, depth_dev, to_intr(*K), pose_dev, status_dev, (cudaStream_t)stream);
}

}  // extern "C"
