// fitness.cuh -- device code shared by the standalone fitness kernels (track.cu)
// and the persistent PFO kernel (pfo.cu): point unprojection, the overlap test of
// Eq. validness, the warp-level fitness of Eq. normallh over packed TSDF cells, the
// work split into (particle group, point chunk) units and the per-particle totals.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace rf {


Pose to_pose(const rf_pose &p);

constexpr int FIT_THREADS = 256;
constexpr int FIT_WARPS = FIT_THREADS / 32;
constexpr int CHUNK_MAX = 256;        // points staged per warp (16 B each)
constexpr int MIN_CHUNK = 32;         // fewest points per work unit
#ifndef RF_UNITS_PER_WARP
#define RF_UNITS_PER_WARP 16
#endif
constexpr int UNITS_PER_WARP = RF_UNITS_PER_WARP;  // target work units per warp and iteration
constexpr int APW = 16;               // doubles per CTA in the APS partials
constexpr int MAX_CTAS_PER_SM = 2048 / FIT_THREADS;  // bound for grid-sized scratch
// CTAs of the persistent kernel resident per SM (register budget 65536 / (256 * n)).
// Measured on the paper-scale frame: groups of 6 lookups at 2 CTAs per SM 312.7 G
// lookups/s, 8 at 2: 306.5, 4 at 3: 299.1 (more loads in flight per warp beat
// more warps).
#ifndef RF_PFO_MIN_BLOCKS
#define RF_PFO_MIN_BLOCKS 2
#endif
// lookups whose loads are issued together in the trilinear loop (the default;
// the persistent kernel is also built for groups of 4 and 8, picked by the
// launch configuration)
#ifndef RF_GROUP
#define RF_GROUP 6
#endif
constexpr int GROUP = RF_GROUP;

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void unproject_point(const float *__restrict__ depth, const Intr &K, int stride, int nw,
                                                int j, float4 &out)
{
    const int a = j % nw, b = j / nw;
    const int u = a * stride, v = b * stride;
    const float z = depth[(size_t)v * K.width + u];
    if (depth_valid(z, K))
        out = make_float4(((float)u - K.cx) * z / K.fx, ((float)v - K.cy) * z / K.fy, z, 1.f);
    else
        out = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Eq. validness for one point: world with the current estimate (Rc, tc), back
// into frame t-1 with its final pose (Rp, tp), nearest pixel, valid depth.
// cell_m > 0 (RF_CELL_MARGIN: sqrt(3) voxels) also keeps the continuous pixel
// position fx cell_m / z' pixels inside the image edges, so that the TSDF cell
// the point samples lies inside frame t-1's view.
__device__ __forceinline__ bool overlap_test(const float4 &p, const float Rc[9], const float tc[3], const float Rp[9],
                                             const float tp[3], const float *__restrict__ prev_depth, const Intr &K,
                                             float cell_m)
{
    if (p.w == 0.f)
        return false;
    const float gx = Rc[0] * p.x + Rc[1] * p.y + Rc[2] * p.z + tc[0] - tp[0];
    const float gy = Rc[3] * p.x + Rc[4] * p.y + Rc[5] * p.z + tc[1] - tp[1];
    const float gz = Rc[6] * p.x + Rc[7] * p.y + Rc[8] * p.z + tc[2] - tp[2];
    const float cx = Rp[0] * gx + Rp[3] * gy + Rp[6] * gz;
    const float cy = Rp[1] * gx + Rp[4] * gy + Rp[7] * gz;
    const float cz = Rp[2] * gx + Rp[5] * gy + Rp[8] * gz;
    if (!(cz > 0.f))
        return false;
    const float uc = K.fx * cx / cz + K.cx, vc = K.fy * cy / cz + K.cy;
    const float mu = K.fx * cell_m / cz, mv = K.fy * cell_m / cz;
    if (!(uc >= mu - 0.5f && uc < (float)K.width - 0.5f - mu && vc >= mv - 0.5f && vc < (float)K.height - 0.5f - mv))
        return false;
    const float u = floorf(uc + 0.5f);
    const float v = floorf(vc + 0.5f);
    if (!(u >= 0.f && u < (float)K.width && v >= 0.f && v < (float)K.height))
        return false;
    const float d = __ldg(&prev_depth[(size_t)v * K.width + (size_t)u]);
    return depth_valid(d, K);
}

// ------------------------------------------------------------------ fitness (warp level)
// MODE bit 0: nearest sample; bit 1: plain (uncompensated) FP32 sum.
template <int MODE> struct Mode {
    static constexpr bool nearest = (MODE & 1) != 0;
    static constexpr bool plain = (MODE & 2) != 0;
};

struct FitParams {
    const float *pst;   // template, structure of arrays with leading dimension ld (pst[d * ld + i])
    int n;              // particles scored: the first n rows of the template
    int ld;
    Pose c;             // PST centre
    float r[6];         // axis lengths
    int l1, right_mult;
};

template <int DT, int MODE, bool L1, int G>
__device__ __forceinline__ void fitness_points(const CellView &V, const float4 *spts, int cnt, const float R[9],
                                               float t0, float t1, float t2, float &sum, float &comp, int &nv);

// Lane `lane` of a warp scores particle i over the points staged in `spts`
// [0, cnt): S = sum psi^2 (|psi| with L1), psi = 1 for invalid samples; G
// lookups have their loads in flight together.
template <int DT, int MODE, int G = GROUP>
__device__ __forceinline__ void fitness_lane(const VolumeDesc &V, const float4 *spts, int cnt, const FitParams &fp,
                                             int i, double &S_out, int &n_out)
{
    Pose P;
    {
        const int ii = i < fp.n ? i : 0;
        float d[6];
#pragma unroll
        for (int a = 0; a < 6; ++a)
            d[a] = fp.r[a] * __ldg(&fp.pst[(size_t)a * fp.ld + ii]);
        compose_offset(fp.c, d, fp.right_mult != 0, P);
    }
    // the rotation and translation are folded with the world -> voxel-centre map
    // g = p / voxel - origin / voxel - 1/2, so a point goes straight to grid units
    float R[9];
    quat_rot(P.q, R);
    const float s = V.inv_voxel;
    for (int a = 0; a < 9; ++a)
        R[a] *= s;
    const float t0 = fmaf(P.t[0], s, V.goff[0]), t1 = fmaf(P.t[1], s, V.goff[1]), t2 = fmaf(P.t[2], s, V.goff[2]);
    float sum = 0.f, comp = 0.f;
    int nv = 0;
    const CellView cv(V);
    if (fp.l1)
        fitness_points<DT, MODE, true, G>(cv, spts, cnt, R, t0, t1, t2, sum, comp, nv);
    else
        fitness_points<DT, MODE, false, G>(cv, spts, cnt, R, t0, t1, t2, sum, comp, nv);
    S_out = (double)sum + (double)comp;
    n_out = nv;
}

// ------------------------------------------------------------------ packed FP32 pairs
// Blackwell's FP32 pair instructions (fma/add/sub/mul .f32x2): two independent
// IEEE operations per instruction, each rounded exactly as its scalar form.  The
// packed int16 loop below pairs two points of a group and performs, for each of
// them, the same operations in the same order as the scalar loop, so its results
// are bit-identical with fewer issued instructions.
#ifndef RF_PACKED
#define RF_PACKED 0
#endif
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_pack(float a, float b)
{
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t r, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c)
{
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2_t f2_add_rd(f2_t a, f2_t b)
{
    f2_t d;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b)
{
    f2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b)
{
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// cell_locate from the biased floor words (bits of __fadd_rd(g, 1.5 * 2^23)).
__device__ __forceinline__ void cell_locate_int(const CellView &V, int ix, int iy, int iz, unsigned &rec, unsigned &cls)
{
    const bool inside = (unsigned)ix < (unsigned)(V.dim[0] - 1) && (unsigned)iy < (unsigned)(V.dim[1] - 1) &&
                        (unsigned)iz < (unsigned)(V.dim[2] - 1);
    const unsigned brick =
        (unsigned)(ix >> 3) + (unsigned)V.nb0 * ((unsigned)(iy >> 3) + (unsigned)V.nb1 * (unsigned)(iz >> 3));
    rec = brick * (unsigned)BRICK_VOX + (unsigned)((ix & 7) | ((iy & 7) << 3) | ((iz & 7) << 6));
    cls = inside ? (unsigned)__ldg(&V.cls[brick]) : (unsigned)CELLS_INVALID;
}

// The int16 trilinear group loop with two points per packed instruction (G even).
// Per point: the transform, floor and fraction, the class and record loads, the
// decode and the interpolation of the scalar loop, operation for operation.
template <int MODE, bool L1, int G>
__device__ __forceinline__ int fitness_points_i16_packed(const CellView &V, const float4 *spts, int cnt,
                                                         const float R[9], float t0, float t1, float t2, float &sum,
                                                         float &comp, int &nv)
{
    static_assert(G % 2 == 0, "the packed loop pairs the points of a group");
    const f2_t R0 = f2_pack(R[0], R[0]), R1 = f2_pack(R[1], R[1]), R2 = f2_pack(R[2], R[2]);
    const f2_t R3 = f2_pack(R[3], R[3]), R4 = f2_pack(R[4], R[4]), R5 = f2_pack(R[5], R[5]);
    const f2_t R6 = f2_pack(R[6], R[6]), R7 = f2_pack(R[7], R[7]), R8 = f2_pack(R[8], R[8]);
    const f2_t T0 = f2_pack(t0, t0), T1 = f2_pack(t1, t1), T2 = f2_pack(t2, t2);
    const f2_t MAGIC = f2_pack(12582912.0f, 12582912.0f);
    const f2_t BIAS = f2_pack(8421376.0f, 8421376.0f);  // 2^23 + 32768
    const f2_t SCALE = f2_pack(1.0f / I16_SCALE, 1.0f / I16_SCALE);
    int j = 0;
    for (; j + G <= cnt; j += G) {
        f2_t FX[G / 2], FY[G / 2], FZ[G / 2];
        CellRef c[G];
        CellData<RF_I16> d[G];
#pragma unroll
        for (int p = 0; p < G / 2; ++p) {
            const float4 xa = spts[j + 2 * p], xb = spts[j + 2 * p + 1];
            const f2_t X = f2_pack(xa.x, xb.x), Y = f2_pack(xa.y, xb.y), Z = f2_pack(xa.z, xb.z);
            const f2_t GX = f2_fma(R0, X, f2_fma(R1, Y, f2_fma(R2, Z, T0)));
            const f2_t GY = f2_fma(R3, X, f2_fma(R4, Y, f2_fma(R5, Z, T1)));
            const f2_t GZ = f2_fma(R6, X, f2_fma(R7, Y, f2_fma(R8, Z, T2)));
            const f2_t TX = f2_add_rd(GX, MAGIC), TY = f2_add_rd(GY, MAGIC), TZ = f2_add_rd(GZ, MAGIC);
            FX[p] = f2_sub(GX, f2_sub(TX, MAGIC));
            FY[p] = f2_sub(GY, f2_sub(TY, MAGIC));
            FZ[p] = f2_sub(GZ, f2_sub(TZ, MAGIC));
            float txa, txb, tya, tyb, tza, tzb;
            f2_unpack(TX, txa, txb);
            f2_unpack(TY, tya, tyb);
            f2_unpack(TZ, tza, tzb);
            cell_locate_int(V, __float_as_int(txa) - 0x4B400000, __float_as_int(tya) - 0x4B400000,
                            __float_as_int(tza) - 0x4B400000, c[2 * p].rec, c[2 * p].cls);
            cell_locate_int(V, __float_as_int(txb) - 0x4B400000, __float_as_int(tyb) - 0x4B400000,
                            __float_as_int(tzb) - 0x4B400000, c[2 * p + 1].rec, c[2 * p + 1].cls);
        }
#pragma unroll
        for (int u = 0; u < G; ++u)
            cell_fetch<RF_I16>(V, c[u], d[u]);
        float grp = 0.f;
#pragma unroll
        for (int p = 0; p < G / 2; ++p) {
            const uint4 a = d[2 * p].a, b = d[2 * p + 1].a;
            // biased corner codes as exact floats 2^23 + u, the two points side by side
            auto lo = [](uint32_t w) { return __int_as_float((int)__byte_perm(w, 0x4B00u, 0x5410)); };
            auto hi = [](uint32_t w) { return __int_as_float((int)__byte_perm(w, 0x4B00u, 0x5432)); };
            const f2_t A0 = f2_pack(lo(a.x), lo(b.x)), A1 = f2_pack(hi(a.x), hi(b.x));
            const f2_t A2 = f2_pack(lo(a.y), lo(b.y)), A3 = f2_pack(hi(a.y), hi(b.y));
            const f2_t A4 = f2_pack(lo(a.z), lo(b.z)), A5 = f2_pack(hi(a.z), hi(b.z));
            const f2_t A6 = f2_pack(lo(a.w), lo(b.w)), A7 = f2_pack(hi(a.w), hi(b.w));
            const f2_t C00 = f2_fma(FX[p], f2_sub(A1, A0), f2_sub(A0, BIAS));
            const f2_t C10 = f2_fma(FX[p], f2_sub(A3, A2), f2_sub(A2, BIAS));
            const f2_t C01 = f2_fma(FX[p], f2_sub(A5, A4), f2_sub(A4, BIAS));
            const f2_t C11 = f2_fma(FX[p], f2_sub(A7, A6), f2_sub(A6, BIAS));
            const f2_t Y0 = f2_fma(FY[p], f2_sub(C10, C00), C00);
            const f2_t Y1 = f2_fma(FY[p], f2_sub(C11, C01), C01);
            const f2_t VV = f2_mul(f2_fma(FZ[p], f2_sub(Y1, Y0), Y0), SCALE);
            float va, vb;
            f2_unpack(VV, va, vb);
            const bool oka = (a.x & 0xFFFFu) != 0u, okb = (b.x & 0xFFFFu) != 0u;
            nv += (oka ? 1 : 0) + (okb ? 1 : 0);
            va = oka ? va : 1.f;
            vb = okb ? vb : 1.f;
            grp += L1 ? fabsf(va) : va * va;
            grp += L1 ? fabsf(vb) : vb * vb;
        }
        if (Mode<MODE>::plain)
            sum += grp;
        else
            neumaier_add(sum, comp, grp);
    }
    return j;
}

// The point loop of one lane: lookups of points [0, cnt) under the grid-space
// pose (R, t), accumulated as psi^2 (|psi| with L1), psi = 1 when invalid.
template <int DT, int MODE, bool L1, int G>
__device__ __forceinline__ void fitness_points(const CellView &V, const float4 *spts, int cnt, const float R[9],
                                               float t0, float t1, float t2, float &sum, float &comp, int &nv)
{
    int j = 0;
    auto add = [&](float grp) {
        if (Mode<MODE>::plain)
            sum += grp;
        else
            neumaier_add(sum, comp, grp);
    };
    auto term = [&](bool ok, float psi) {  // psi = 1 when invalid (cell_eval, nearest below)
        nv += ok ? 1 : 0;
        return L1 ? fabsf(psi) : psi * psi;
    };
    if constexpr (RF_PACKED && DT == RF_I16 && !Mode<MODE>::nearest && G % 2 == 0)
        j = fitness_points_i16_packed<MODE, L1, G>(V, spts, cnt, R, t0, t1, t2, sum, comp, nv);
    else if (!Mode<MODE>::nearest) {
        // groups of G lookups: all class loads, then all cell loads, then the
        // arithmetic, so each group pays the load latency once; a plain FP32
        // partial of <= G terms in [0, 1] is then added with compensation
        for (; j + G <= cnt; j += G) {
            CellRef c[G];
            CellData<DT> d[G];
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const float4 x = spts[j + u];
                cell_locate(V, fmaf(R[0], x.x, fmaf(R[1], x.y, fmaf(R[2], x.z, t0))),
                            fmaf(R[3], x.x, fmaf(R[4], x.y, fmaf(R[5], x.z, t1))),
                            fmaf(R[6], x.x, fmaf(R[7], x.y, fmaf(R[8], x.z, t2))), c[u]);
            }
#pragma unroll
            for (int u = 0; u < G; ++u)
                cell_fetch<DT>(V, c[u], d[u]);
            float grp = 0.f;
#pragma unroll
            for (int u = 0; u < G; ++u) {
                float psi;
                const bool ok = cell_eval<DT>(c[u], d[u], psi);
                grp += term(ok, psi);
            }
            add(grp);
        }
    }
    for (; j < cnt; ++j) {  // the tail of the chunk (or every point in nearest mode)
        const float4 x = spts[j];
        const float gx = fmaf(R[0], x.x, fmaf(R[1], x.y, fmaf(R[2], x.z, t0)));
        const float gy = fmaf(R[3], x.x, fmaf(R[4], x.y, fmaf(R[5], x.z, t1)));
        const float gz = fmaf(R[6], x.x, fmaf(R[7], x.y, fmaf(R[8], x.z, t2)));
        float psi;
        bool ok;
        if (Mode<MODE>::nearest) {
            ok = sample_nearest_g<DT>(V, gx, gy, gz, psi);
            psi = ok ? psi : 1.f;
        } else {
            CellRef c;
            CellData<DT> d;
            cell_locate(V, gx, gy, gz, c);
            cell_fetch<DT>(V, c, d);
            ok = cell_eval<DT>(c, d, psi);
        }
        add(term(ok, psi));
    }
}

// Work decomposition shared by the standalone and the persistent kernels: unit
// u = (point chunk u / groups, particle group u % groups); consecutive units
// share a point chunk so the warps of a CTA touch neighbouring voxels.
struct Split {
    int groups, n_chunks, chunk;
};

__host__ __device__ inline Split make_split(int n, int m, int total_warps, int max_chunks)
{
    Split s;
    s.groups = (n + 31) / 32;
    int want = (UNITS_PER_WARP * total_warps + s.groups - 1) / s.groups;
    int lo = (m + CHUNK_MAX - 1) / CHUNK_MAX;   // staging capacity
    int hi = (m + MIN_CHUNK - 1) / MIN_CHUNK;   // at least MIN_CHUNK points per unit
    want = want < lo ? lo : want;
    want = want > hi ? hi : want;
    want = want > max_chunks ? max_chunks : want;
    want = want < 1 ? 1 : want;
    s.n_chunks = want;
    s.chunk = (m + want - 1) / want;
    if (s.chunk > CHUNK_MAX) {  // only when max_chunks binds
        s.chunk = CHUNK_MAX;
        s.n_chunks = (m + CHUNK_MAX - 1) / CHUNK_MAX;
    }
    return s;
}

__host__ inline int max_chunks_for(int n, int m_max, int total_warps)
{
    const int groups = (n + 31) / 32;
    const int a = (UNITS_PER_WARP * total_warps + groups - 1) / groups;
    const int b = (m_max + CHUNK_MAX - 1) / CHUNK_MAX;
    return std::max(1, std::max(std::min(a, (m_max + MIN_CHUNK - 1) / MIN_CHUNK), b));
}

// All warps of the grid walk the units; each stages its chunk of points, scores
// its 32 particles and writes one (S, n) partial per particle.  `coherent`
// selects L2-coherent loads for points written earlier in the same kernel.
// With a unit counter (`next_unit` non-null, zero at the start of the phase) the
// warps take units dynamically, one atomic per unit, fetched one unit ahead;
// otherwise warp w takes units w, w + total_warps, ...
template <int DT, int MODE, bool COHERENT>
__device__ __forceinline__ void fitness_units(const VolumeDesc &V, const float4 *pts, int m, const FitParams &fp,
                                              const Split &sp, double *part_S, int *part_n, float4 *smem_pts,
                                              int warp_global, int total_warps, int lane, int warp_in_block,
                                              int *next_unit = nullptr)
{
    float4 *spts = smem_pts + (size_t)warp_in_block * CHUNK_MAX;
    const int units = sp.groups * sp.n_chunks;
    int staged = -1;
    int u = warp_global;
    if (next_unit) {
        int t = 0;
        if (lane == 0)
            t = atomicAdd(next_unit, 1);
        u = __shfl_sync(0xffffffffu, t, 0);
    }
    while (u < units) {
        int u_next = u + total_warps;
        if (next_unit) {
            int t = 0;
            if (lane == 0)
                t = atomicAdd(next_unit, 1);
            u_next = __shfl_sync(0xffffffffu, t, 0);
        }
        const int ch = u / sp.groups, g = u - ch * sp.groups;
        const int j0 = ch * sp.chunk;
        const int cnt = min(sp.chunk, m - j0);
        if (ch != staged) {
            __syncwarp();
            for (int j = lane; j < cnt; j += 32)
                spts[j] = COHERENT ? __ldcg(&pts[j0 + j]) : __ldg(&pts[j0 + j]);
            __syncwarp();
            staged = ch;
        }
        const int i = g * 32 + lane;
        double S;
        int nv;
        fitness_lane<DT, MODE>(V, spts, cnt, fp, i, S, nv);
        if (i < fp.n) {
            part_S[(size_t)ch * fp.n + i] = S;
            part_n[(size_t)ch * fp.n + i] = nv;
        }
        u = u_next;
    }
}

// Fixed-order sum of the chunk partials of particle i, then rho (Eq. normallh,
// or Eq. ourlh without NORMALIZE).
__device__ __forceinline__ void particle_total(const double *part_S, const int *part_n, int n, int n_chunks, int i,
                                               bool coherent, double &S, int &nv)
{
    S = 0.0;
    nv = 0;
    for (int c = 0; c < n_chunks; ++c) {
        S += coherent ? __ldcg(&part_S[(size_t)c * n + i]) : part_S[(size_t)c * n + i];
        nv += coherent ? __ldcg(&part_n[(size_t)c * n + i]) : part_n[(size_t)c * n + i];
    }
}

__device__ __forceinline__ float fitness_rho(double S, int nO, float tau, bool normalize)
{
    if (nO <= 0)
        return 0.f;
    const double x = normalize ? S / ((double)tau * (double)nO) : S / (double)tau;
    return expf(-(float)x);
}


inline int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

}  // namespace rf
