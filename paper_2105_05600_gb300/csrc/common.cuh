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
constexpr uint8_t CELLS_MIXED = 0, CELLS_FREE = 1, CELLS_INVALID = 2;

// Passed by value to every kernel that touches the TSDF.
struct VolumeDesc {
    void *values;      // brick layout: brick b = bx + nb[0]*(by + nb[1]*bz), then lx + 8*(ly + 8*lz)
    uint8_t *weights;  // same layout
    // Packed trilinear cells: record i (same brick index as voxel i) holds the 8
    // corner codes of the cell whose lower corner is voxel i, ordered
    // (x,y,z) = 000,100,010,110,001,101,011,111: 16 B for int16/half, 32 B for
    // float.  Fusion rebuilds the cells of every brick that reads a changed value.
    // int16 cells hold the biased code c + 32768 (sentinel -> 0).
    void *cells;
    // Fusion work lists, rebuilt by every tsdf_integrate: fuse_count[0] bricks that
    // passed the frustum test, listed in fuse_list[0, nbricks); fuse_count[1] bricks
    // whose cells are to be repacked, listed in fuse_list[nbricks, 2 nbricks) and
    // marked in the bit set `need` (one bit per brick, so a brick is listed once).
    // An entry is the brick's coordinates bx | by << 10 | bz << 20.
    // fuse_count and need are one allocation, cleared together before each fusion.
    unsigned *fuse_count;
    uint32_t *need;
    int *fuse_list;
    int fuse_grid[2];  // persistent grid (CTAs) of integrate_kernel and pack_cells_kernel
    // Class of each cell brick, written with its cells: CELLS_MIXED, or every
    // cell of the brick free space (all 8 corners exactly +1: psi = 1, valid) or
    // every cell touching an unobserved voxel (invalid).  Lookups in constant
    // bricks skip the cell load.
    uint8_t *brick_class;
    // fusion counters since the last read-out: [0] voxels updated, [1] bricks that
    // passed the frustum test, [2] bricks whose cells were repacked
    unsigned long long *counters;
    int cell_stride[3];// brick-layout strides of one brick step per axis (in records)
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

// ------------------------------------------------------------------ packed-cell sampling
// floor(g) without the conversion pipe: adding 1.5 * 2^23 with round-down leaves
// floor(g) in the low mantissa bits for |g| < 2^22.  Out-of-range, huge or NaN g
// give an index that fails the unsigned bounds test of the caller.
__device__ __forceinline__ int floor_split(float g, float &frac)
{
    const float t = __fadd_rd(g, 12582912.0f);
    frac = g - (t - 12582912.0f);
    return __float_as_int(t) - 0x4B400000;
}

// Two biased int16 codes (c + 32768) of one 32-bit word as exact floats c,
// without I2F: each 16-bit half is placed in the mantissa of 2^23.
__device__ __forceinline__ void decode_i16x2(uint32_t w, float &lo, float &hi)
{
    lo = __int_as_float((int)__byte_perm(w, 0x4B00u, 0x5410)) - 8421376.0f;  // 2^23 + 32768
    hi = __int_as_float((int)__byte_perm(w, 0x4B00u, 0x5432)) - 8421376.0f;
}

// psi of a free-space cell (eight +1 corners), bit-identical to what the full
// interpolation returns for it.
template <int DT> __device__ __forceinline__ float free_psi()
{
    return DT == RF_I16 ? 32767.0f * (1.0f / I16_SCALE) : 1.0f;
}

__device__ __forceinline__ float lerp1(float a, float b, float t) { return fmaf(t, b - a, a); }

// The fields of a volume that the fitness loop reads, copied once into
// registers (a descriptor reached through a dynamic index would be reloaded).
struct CellView {
    const uint8_t *cls;
    const void *cells;
    const void *values;
    int dim[3];
    int nb0, nb1;
    __device__ __forceinline__ explicit CellView(const VolumeDesc &V)
        : cls(V.brick_class), cells(V.cells), values(V.values), nb0(V.nb[0]), nb1(V.nb[1])
    {
        dim[0] = V.dim[0];
        dim[1] = V.dim[1];
        dim[2] = V.dim[2];
    }
};

// Nearest-voxel psi at voxel-centre coordinates (flag RF_NEAREST): the voxel
// whose centre is closest, valid if inside the volume and observed.
template <int DT>
__device__ __forceinline__ bool sample_nearest_g(const CellView &V, float gx, float gy, float gz, float &psi)
{
    using T = typename Storage<DT>::T;
    float f;
    const int ix = floor_split(gx + 0.5f, f), iy = floor_split(gy + 0.5f, f), iz = floor_split(gz + 0.5f, f);
    if (!((unsigned)ix < (unsigned)V.dim[0] && (unsigned)iy < (unsigned)V.dim[1] && (unsigned)iz < (unsigned)V.dim[2]))
        return false;
    const size_t brick = (size_t)(ix >> 3) + (size_t)V.nb0 * ((size_t)(iy >> 3) + (size_t)V.nb1 * (size_t)(iz >> 3));
    const size_t idx = brick * BRICK_VOX + (size_t)((ix & 7) + 8 * ((iy & 7) + 8 * (iz & 7)));
    const float v = Storage<DT>::decode(__ldg(&reinterpret_cast<const T *>(V.values)[idx]));
    psi = v;
    return !isnan(v);
}


// Trilinear lookup from the packed cells, split into three branch-free steps so
// that a caller can issue the loads of several lookups before using any:
//   cell_locate: cell index, fractions and the brick class (one byte load);
//   cell_fetch:  the 16-byte (32 for float) record, only for mixed bricks;
//   cell_eval:   decode + interpolation, valid only inside the volume with every
//                corner observed (a cell with an unobserved corner is stored as
//                all zero codes for int16, and NaN poisons float storage).
struct CellRef {
    float fx, fy, fz;
    unsigned rec;
    unsigned cls;  // CELLS_MIXED / CELLS_FREE / CELLS_INVALID (also out of the volume)
};

template <int DT> struct CellData {
    uint4 a;
};
template <> struct CellData<RF_F32> {
    float4 a, b;
};

// RF_CELL_CLASS = 1: lookups in constant bricks skip the record (class byte
// first, then a predicated record load); 0: every lookup inside the volume loads
// its own record, which packing writes for every brick, so both give the same
// values -- the second trades L2 traffic for fewer instructions and one
// dependent load less per lookup.
#ifndef RF_CELL_CLASS
#define RF_CELL_CLASS 1
#endif

__device__ __forceinline__ void cell_locate(const CellView &V, float gx, float gy, float gz, CellRef &c)
{
    const int ix = floor_split(gx, c.fx), iy = floor_split(gy, c.fy), iz = floor_split(gz, c.fz);
    const bool inside = (unsigned)ix < (unsigned)(V.dim[0] - 1) && (unsigned)iy < (unsigned)(V.dim[1] - 1) &&
                        (unsigned)iz < (unsigned)(V.dim[2] - 1);
    const unsigned brick =
        (unsigned)(ix >> 3) + (unsigned)V.nb0 * ((unsigned)(iy >> 3) + (unsigned)V.nb1 * (unsigned)(iz >> 3));
    c.rec = brick * (unsigned)BRICK_VOX + (unsigned)((ix & 7) | ((iy & 7) << 3) | ((iz & 7) << 6));
#if RF_CELL_CLASS
    c.cls = inside ? (unsigned)__ldg(&V.cls[brick]) : (unsigned)CELLS_INVALID;
#else
    c.cls = inside ? (unsigned)CELLS_MIXED : (unsigned)CELLS_INVALID;
    c.rec = inside ? c.rec : 0u;  // any record in bounds; cell_fetch invalidates it
#endif
}

// The record of a constant brick is not loaded: the registers get a fill
// record that evaluates to the same answer (eight +1 corners for free space,
// an invalid record otherwise), and the load is predicated on a mixed brick.
// (Filling only the first word, with a free-space marker that no packed record
// holds, and leaving the other three as they were measured 22 % slower on the
// paper-scale frame; the full fill stays.)
__device__ __forceinline__ void ldg_v4_if(bool p, const void *ptr, uint32_t &x, uint32_t &y, uint32_t &z, uint32_t &w)
{
    asm("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t@p ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%5];\n\t}"
        : "+r"(x), "+r"(y), "+r"(z), "+r"(w)
        : "r"((int)p), "l"(ptr));
}

template <int DT> __device__ __forceinline__ void cell_fetch(const CellView &V, const CellRef &c, CellData<DT> &d)
{
#if !RF_CELL_CLASS
    // unconditional load of the (in-bounds) record; outside the volume the first
    // word is replaced by an invalid pattern (zero int16 codes, NaN halves/float)
    const bool inside = c.cls == CELLS_MIXED;
    if constexpr (DT == RF_F32) {
        const float4 *cp = reinterpret_cast<const float4 *>(V.cells) + 2 * (size_t)c.rec;
        d.a = __ldg(cp);
        d.b = __ldg(cp + 1);
        d.a.x = inside ? d.a.x : __int_as_float(0x7FC00000);
    } else {
        d.a = __ldg(reinterpret_cast<const uint4 *>(V.cells) + c.rec);
        d.a.x = inside ? d.a.x : (DT == RF_I16 ? 0u : 0x7E007E00u);
    }
    return;
#endif
    const bool mixed = c.cls == CELLS_MIXED, free_space = c.cls == CELLS_FREE;
    if constexpr (DT == RF_F32) {
        // +1.0f for free space, NaN (invalid) otherwise
        const uint32_t f = free_space ? 0x3F800000u : 0x7FC00000u;
        uint32_t a0 = f, a1 = f, a2 = f, a3 = f, b0 = f, b1 = f, b2 = f, b3 = f;
        const float4 *cp = reinterpret_cast<const float4 *>(V.cells) + 2 * (size_t)c.rec;
        ldg_v4_if(mixed, cp, a0, a1, a2, a3);
        ldg_v4_if(mixed, cp + 1, b0, b1, b2, b3);
        d.a = make_float4(__uint_as_float(a0), __uint_as_float(a1), __uint_as_float(a2), __uint_as_float(a3));
        d.b = make_float4(__uint_as_float(b0), __uint_as_float(b1), __uint_as_float(b2), __uint_as_float(b3));
    } else {
        // int16 (biased): 0xFFFF = code +32767, 0 = invalid; half: 1.0h pairs, NaN pairs
        const uint32_t f = DT == RF_I16 ? (free_space ? 0xFFFFFFFFu : 0u) : (free_space ? 0x3C003C00u : 0x7E007E00u);
        uint32_t x = f, y = f, z = f, w = f;
        ldg_v4_if(mixed, reinterpret_cast<const uint4 *>(V.cells) + c.rec, x, y, z, w);
        d.a = make_uint4(x, y, z, w);
    }
}

// Returns whether the lookup is valid; psi is the interpolated value when valid
// and 1 (the maximal truncated penalty) when not.
template <int DT> __device__ __forceinline__ bool cell_eval(const CellRef &c, const CellData<DT> &d, float &psi)
{
    float c00, c10, c01, c11;
    bool ok;
    if constexpr (DT == RF_I16) {
        // biased floats 2^23 + u: differences are exact, so the first lerp level
        // takes its base unbiased and its slope from the biased pair
        const float B = 8421376.0f;  // 2^23 + 32768
        const float a0 = __int_as_float((int)__byte_perm(d.a.x, 0x4B00u, 0x5410));
        const float a1 = __int_as_float((int)__byte_perm(d.a.x, 0x4B00u, 0x5432));
        const float a2 = __int_as_float((int)__byte_perm(d.a.y, 0x4B00u, 0x5410));
        const float a3 = __int_as_float((int)__byte_perm(d.a.y, 0x4B00u, 0x5432));
        const float a4 = __int_as_float((int)__byte_perm(d.a.z, 0x4B00u, 0x5410));
        const float a5 = __int_as_float((int)__byte_perm(d.a.z, 0x4B00u, 0x5432));
        const float a6 = __int_as_float((int)__byte_perm(d.a.w, 0x4B00u, 0x5410));
        const float a7 = __int_as_float((int)__byte_perm(d.a.w, 0x4B00u, 0x5432));
        c00 = fmaf(c.fx, a1 - a0, a0 - B);
        c10 = fmaf(c.fx, a3 - a2, a2 - B);
        c01 = fmaf(c.fx, a5 - a4, a4 - B);
        c11 = fmaf(c.fx, a7 - a6, a6 - B);
        ok = (d.a.x & 0xFFFFu) != 0u;  // all-zero record = some corner unobserved
    } else {
        float k[8];
        if constexpr (DT == RF_F32) {
            k[0] = d.a.x; k[1] = d.a.y; k[2] = d.a.z; k[3] = d.a.w;
            k[4] = d.b.x; k[5] = d.b.y; k[6] = d.b.z; k[7] = d.b.w;
        } else {
            const uint32_t w[4] = {d.a.x, d.a.y, d.a.z, d.a.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 f2 = __half22float2(*reinterpret_cast<const __half2 *>(&w[q]));
                k[2 * q] = f2.x;
                k[2 * q + 1] = f2.y;
            }
        }
        c00 = lerp1(k[0], k[1], c.fx);
        c10 = lerp1(k[2], k[3], c.fx);
        c01 = lerp1(k[4], k[5], c.fx);
        c11 = lerp1(k[6], k[7], c.fx);
    }
    float v = lerp1(lerp1(c00, c10, c.fy), lerp1(c01, c11, c.fy), c.fz);
    if constexpr (DT == RF_I16)
        v *= 1.0f / I16_SCALE;
    else
        ok = !isnan(v);  // a NaN corner poisons the interpolation
    psi = ok ? v : 1.f;
    return ok;
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
