// common.cuh -- device-side types and helpers shared by the librosefusion kernels.
// Conventions follow include/rosefusion.h: camera->world poses x_G = R(q) x + t
// (Sec. 3.1, Eq. unproj), q = (w, x, y, z) unit Hamilton quaternions; the TSDF
// holds F = sdf / trunc with an "unobserved" sentinel.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rosefusion.h"

namespace rf {

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
rf_status cuda_fail(cudaError_t e, const char *what);
#define RF_CUDA(call)                                                                                   \
    do {                                                                                                \
        cudaError_t _e = (call);                                                                        \
        if (_e != cudaSuccess)                                                                          \
            return ::rf::cuda_fail(_e, #call);                                                          \
    } while (0)
#define RF_CHECK_ARG(cond, msg)                                                                         \
    do {                                                                                                \
        if (!(cond)) {                                                                                  \
            ::rf::set_error("%s: %s", __func__, msg);                                                   \
            return RF_ERR_ARG;                                                                          \
        }                                                                                               \
    } while (0)

// ------------------------------------------------------------------ volume
constexpr int BRICK = 8;             // 8x8x8 voxels per brick
constexpr int BRICK_VOX = 512;
constexpr int16_t I16_UNOBSERVED = -32768;
constexpr float I16_SCALE = 32767.0f;

// Passed by value to every kernel that touches the TSDF.
struct VolumeDesc {
    void *values;      // brick layout: brick b = bx + nb[0]*(by + nb[1]*bz), then lx + 8*(ly + 8*lz)
    uint8_t *weights;  // same layout
    int dim[3];
    int nb[3];
    float voxel, inv_voxel, trunc;
    float origin[3];
    float goff[3];     // -origin / voxel - 0.5: g = p * inv_voxel + goff (voxel-centre coordinates)
    int dtype;
};

__host__ __device__ __forceinline__ size_t brick_index(const VolumeDesc &V, int x, int y, int z)
{
    size_t b = (size_t)(x >> 3) + (size_t)V.nb[0] * ((size_t)(y >> 3) + (size_t)V.nb[1] * (size_t)(z >> 3));
    return b * BRICK_VOX + (size_t)((x & 7) + 8 * ((y & 7) + 8 * (z & 7)));
}

struct Intr {
    float fx, fy, cx, cy;
    int width, height;
    float z_min, z_max;
};

__host__ __device__ __forceinline__ Intr to_intr(const rf_intrinsics &K)
{
    Intr k;
    k.fx = K.fx;
    k.fy = K.fy;
    k.cx = K.cx;
    k.cy = K.cy;
    k.width = K.width;
    k.height = K.height;
    k.z_min = K.z_min;
    k.z_max = K.z_max;
    return k;
}

__device__ __forceinline__ bool depth_valid(float z, const Intr &K) { return z > K.z_min && z <= K.z_max; }

// ------------------------------------------------------------------ quaternions (FP32)
struct Pose {
    float q[4];
    float t[3];
};

__device__ __forceinline__ void quat_mul(const float a[4], const float b[4], float o[4])
{
    float w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    float x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    float y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    float z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    o[0] = w;
    o[1] = x;
    o[2] = y;
    o[3] = z;
}

// Row-major R of a unit quaternion.
__device__ __forceinline__ void quat_rot(const float q[4], float R[9])
{
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y,
                wz = w * z;
    R[0] = 1.f - 2.f * (yy + zz);
    R[1] = 2.f * (xy - wz);
    R[2] = 2.f * (xz + wy);
    R[3] = 2.f * (xy + wz);
    R[4] = 1.f - 2.f * (xx + zz);
    R[5] = 2.f * (yz - wx);
    R[6] = 2.f * (xz - wy);
    R[7] = 2.f * (yz + wx);
    R[8] = 1.f - 2.f * (xx + yy);
}

// MovePST / RescalePST of one particle (Sec. 3.3): centre c (+) offset delta,
// delta = (dq_x, dq_y, dq_z, dt_x, dt_y, dt_z).  q_delta = (sqrt(1-|dq|^2), dq),
// |dq| clamped to 1; default q = q_delta (x) q_c, t = t_c + dt; RIGHT_MULT:
// q = q_c (x) q_delta, t = t_c + R_c dt.  Renormalised, w >= 0.
__device__ __forceinline__ void compose_offset(const Pose &c, const float d[6], bool right_mult, Pose &out)
{
    float dq0 = d[0], dq1 = d[1], dq2 = d[2];
    float n2 = dq0 * dq0 + dq1 * dq1 + dq2 * dq2;
    if (n2 > 1.f) {
        float s = rsqrtf(n2);
        dq0 *= s;
        dq1 *= s;
        dq2 *= s;
        n2 = 1.f;
    }
    float qd[4] = {sqrtf(fmaxf(0.f, 1.f - n2)), dq0, dq1, dq2};
    float q[4];
    if (right_mult) {
        float Rc[9];
        quat_rot(c.q, Rc);
        quat_mul(c.q, qd, q);
        for (int r = 0; r < 3; ++r)
            out.t[r] = c.t[r] + Rc[3 * r] * d[3] + Rc[3 * r + 1] * d[4] + Rc[3 * r + 2] * d[5];
    } else {
        quat_mul(qd, c.q, q);
        out.t[0] = c.t[0] + d[3];
        out.t[1] = c.t[1] + d[4];
        out.t[2] = c.t[2] + d[5];
    }
    float inv = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (q[0] < 0.f)
        inv = -inv;
    for (int i = 0; i < 4; ++i)
        out.q[i] = q[i] * inv;
}

// Neumaier-compensated accumulation (Sec. 4: Kahan/Neumaier summation of the TSDF terms).
__device__ __forceinline__ void neumaier_add(float &sum, float &comp, float x)
{
    float t = sum + x;
    if (fabsf(sum) >= fabsf(x))
        comp += (sum - t) + x;
    else
        comp += (x - t) + sum;
    sum = t;
}

// ------------------------------------------------------------------ TSDF value decode
template <int DT> struct Storage;
template <> struct Storage<RF_F32> {
    using T = float;
    static __device__ __forceinline__ float decode(float v) { return v; }
};
template <> struct Storage<RF_F16> {
    using T = __half;
    static __device__ __forceinline__ float decode(__half v) { return __half2float(v); }
};
template <> struct Storage<RF_I16> {
    using T = int16_t;
    // -32768 (unobserved) decodes to NaN so that it poisons any interpolation.
    static __device__ __forceinline__ float decode(int16_t v)
    {
        return v == I16_UNOBSERVED ? __int_as_float(0x7fc00000) : (float)v * (1.0f / I16_SCALE);
    }
};

// psi at world point p (reading: trilinear on voxel centres, all 8 corners inside
// the volume and observed; NEAREST: closest voxel centre).  Returns false when
// the sample is invalid.
template <int DT, bool NEAREST>
__device__ __forceinline__ bool sample_tsdf(const VolumeDesc &V, float px, float py, float pz, float &psi)
{
    using T = typename Storage<DT>::T;
    const T *vals = reinterpret_cast<const T *>(V.values);
    const float gx = fmaf(px, V.inv_voxel, V.goff[0]);
    const float gy = fmaf(py, V.inv_voxel, V.goff[1]);
    const float gz = fmaf(pz, V.inv_voxel, V.goff[2]);
    if (NEAREST) {
        const float rx = floorf(gx + 0.5f), ry = floorf(gy + 0.5f), rz = floorf(gz + 0.5f);
        if (!(rx >= 0.f && rx <= (float)(V.dim[0] - 1) && ry >= 0.f && ry <= (float)(V.dim[1] - 1) && rz >= 0.f &&
              rz <= (float)(V.dim[2] - 1)))
            return false;
        float v = Storage<DT>::decode(__ldg(&vals[brick_index(V, (int)rx, (int)ry, (int)rz)]));
        psi = v;
        return !isnan(v);
    }
    const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
    if (!(fx0 >= 0.f && fx0 <= (float)(V.dim[0] - 2) && fy0 >= 0.f && fy0 <= (float)(V.dim[1] - 2) && fz0 >= 0.f &&
          fz0 <= (float)(V.dim[2] - 2)))
        return false;
    const int ix = (int)fx0, iy = (int)fy0, iz = (int)fz0;
    const float fx = gx - fx0, fy = gy - fy0, fz = gz - fz0;
    // per-axis offsets of the two corners inside the brick layout
    const size_t sy = (size_t)V.nb[0] * BRICK_VOX, sz = sy * (size_t)V.nb[1];
    const size_t ox0 = (size_t)(ix >> 3) * BRICK_VOX + (ix & 7), ox1 = (size_t)((ix + 1) >> 3) * BRICK_VOX + ((ix + 1) & 7);
    const size_t oy0 = (size_t)(iy >> 3) * sy + 8 * (iy & 7), oy1 = (size_t)((iy + 1) >> 3) * sy + 8 * ((iy + 1) & 7);
    const size_t oz0 = (size_t)(iz >> 3) * sz + 64 * (iz & 7), oz1 = (size_t)((iz + 1) >> 3) * sz + 64 * ((iz + 1) & 7);
    const float v000 = Storage<DT>::decode(__ldg(&vals[ox0 + oy0 + oz0]));
    const float v100 = Storage<DT>::decode(__ldg(&vals[ox1 + oy0 + oz0]));
    const float v010 = Storage<DT>::decode(__ldg(&vals[ox0 + oy1 + oz0]));
    const float v110 = Storage<DT>::decode(__ldg(&vals[ox1 + oy1 + oz0]));
    const float v001 = Storage<DT>::decode(__ldg(&vals[ox0 + oy0 + oz1]));
    const float v101 = Storage<DT>::decode(__ldg(&vals[ox1 + oy0 + oz1]));
    const float v011 = Storage<DT>::decode(__ldg(&vals[ox0 + oy1 + oz1]));
    const float v111 = Storage<DT>::decode(__ldg(&vals[ox1 + oy1 + oz1]));
    const float c00 = fmaf(fx, v100 - v000, v000);
    const float c10 = fmaf(fx, v110 - v010, v010);
    const float c01 = fmaf(fx, v101 - v001, v001);
    const float c11 = fmaf(fx, v111 - v011, v011);
    const float c0 = fmaf(fy, c10 - c00, c00);
    const float c1 = fmaf(fy, c11 - c01, c01);
    const float v = fmaf(fz, c1 - c0, c0);
    psi = v;
    return !isnan(v);
}

}  // namespace rf

// Volume handle (host side).
struct rf_volume_s {
    rf::VolumeDesc d;
    size_t n_vox;
    int device;
    void *scratch;          // fitness_eval partial sums, grown on demand
    size_t scratch_bytes;
};
