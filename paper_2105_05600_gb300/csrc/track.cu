// track.cu -- the PFO/PST tracking hot path (Algorithm 1 of the paper).
//
//  depth_to_points   Eq. unproj + stride downsampling (Sec. 4)
//  overlap           Eq. validness
//  fitness           Eq. normallh, one warp scores 32 particles (one per lane)
//                    over a chunk of points staged in shared memory
//  pfo_kernel        ONE persistent cooperative kernel per frame running every
//                    PFO iteration: overlap + compaction, fitness, APS / best
//                    state / rescale (Eq. ebs, wafit, rsdir, rsinter, momentum),
//                    stop rules (Sec. 4); phases separated by a grid barrier
//                    whose waits are bounded in time.
//
// The paper streams the N fitness values to the host every iteration and
// updates the PST on the CPU (Sec. 4, GPU implementation); here the update is
// reduced on the device in a fixed order, so nothing crosses PCIe/C2C inside a
// frame.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace rf {

Pose to_pose(const rf_pose &p);

constexpr int FIT_THREADS = 256;
constexpr int FIT_WARPS = FIT_THREADS / 32;
constexpr int CHUNK_MAX = 256;        // points staged per warp (16 B each)
#ifndef RF_UNITS_PER_WARP
#define RF_UNITS_PER_WARP 16
#endif
constexpr int UNITS_PER_WARP = RF_UNITS_PER_WARP;  // target work units per warp and iteration
constexpr int APW = 16;               // doubles per CTA in the APS partials
constexpr int MAX_CTAS_PER_SM = 2048 / FIT_THREADS;  // bound for grid-sized scratch
// CTAs of the persistent kernel resident per SM (register budget 65536 / (256 * n))
#ifndef RF_PFO_MIN_BLOCKS
#define RF_PFO_MIN_BLOCKS 3
#endif

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
__device__ __forceinline__ bool overlap_test(const float4 &p, const float Rc[9], const float tc[3], const float Rp[9],
                                             const float tp[3], const float *__restrict__ prev_depth, const Intr &K)
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
    const float u = floorf(K.fx * cx / cz + K.cx + 0.5f);
    const float v = floorf(K.fy * cy / cz + K.cy + 0.5f);
    if (!(u >= 0.f && u < (float)K.width && v >= 0.f && v < (float)K.height))
        return false;
    return depth_valid(__ldg(&prev_depth[(size_t)v * K.width + (size_t)u]), K);
}

// ------------------------------------------------------------------ fitness (warp level)
// MODE bit 0: nearest sample; bit 1: plain (uncompensated) FP32 sum.
template <int MODE> struct Mode {
    static constexpr bool nearest = (MODE & 1) != 0;
    static constexpr bool plain = (MODE & 2) != 0;
};

struct FitParams {
    const float *pst;   // 6 x n SoA template
    int n;
    Pose c;             // PST centre
    float r[6];         // axis lengths
    int l1, right_mult;
};

template <int DT, int MODE, bool L1>
__device__ __forceinline__ void fitness_points(const VolumeDesc &V, const float4 *spts, int cnt, const float R[9],
                                               float t0, float t1, float t2, float &sum, float &comp, int &nv);

// Lane `lane` of a warp scores particle i over the points staged in `spts`
// [0, cnt): S = sum psi^2 (|psi| with L1), psi = 1 for invalid samples.
template <int DT, int MODE>
__device__ __forceinline__ void fitness_lane(const VolumeDesc &V, const float4 *spts, int cnt, const FitParams &fp,
                                             int i, double &S_out, int &n_out)
{
    Pose P;
    {
        const int ii = i < fp.n ? i : 0;
        float d[6];
#pragma unroll
        for (int a = 0; a < 6; ++a)
            d[a] = fp.r[a] * __ldg(&fp.pst[(size_t)a * fp.n + ii]);
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
    if (fp.l1)
        fitness_points<DT, MODE, true>(V, spts, cnt, R, t0, t1, t2, sum, comp, nv);
    else
        fitness_points<DT, MODE, false>(V, spts, cnt, R, t0, t1, t2, sum, comp, nv);
    S_out = (double)sum + (double)comp;
    n_out = nv;
}

// The point loop of one lane: lookups of points [0, cnt) under the grid-space
// pose (R, t), accumulated as psi^2 (|psi| with L1), psi = 1 when invalid.
template <int DT, int MODE, bool L1>
__device__ __forceinline__ void fitness_points(const VolumeDesc &V, const float4 *spts, int cnt, const float R[9],
                                               float t0, float t1, float t2, float &sum, float &comp, int &nv)
{
    int j = 0;
    auto add = [&](float grp) {
        if (Mode<MODE>::plain)
            sum += grp;
        else
            neumaier_add(sum, comp, grp);
    };
    auto term = [&](bool ok, float psi) {
        nv += ok ? 1 : 0;
        psi = ok ? psi : 1.f;
        return L1 ? fabsf(psi) : psi * psi;
    };
    if (!Mode<MODE>::nearest) {
        // groups of 4 lookups: all class loads, then all cell loads, then the
        // arithmetic, so each group pays the load latency once; a plain FP32
        // partial of <= 4 terms in [0, 1] is then added with compensation
        for (; j + 4 <= cnt; j += 4) {
            CellRef c[4];
            CellData<DT> d[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 x = spts[j + u];
                cell_locate(V, fmaf(R[0], x.x, fmaf(R[1], x.y, fmaf(R[2], x.z, t0))),
                            fmaf(R[3], x.x, fmaf(R[4], x.y, fmaf(R[5], x.z, t1))),
                            fmaf(R[6], x.x, fmaf(R[7], x.y, fmaf(R[8], x.z, t2))), c[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                cell_fetch<DT>(V, c[u], d[u]);
            float grp = 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
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
    int hi = (m + 15) / 16;                     // at least 16 points per unit
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
    return std::max(1, std::max(std::min(a, (m_max + 15) / 16), b));
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
                               uint8_t *mask, int *count)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    float Rc[9], Rp[9];
    quat_rot(cur.q, Rc);
    quat_rot(prev.q, Rp);
    bool in = false;
    if (j < m) {
        in = overlap_test(pts[j], Rc, cur.t, Rp, prev.t, prev_depth, K);
        mask[j] = in ? 1 : 0;
    }
    if (count) {
        unsigned b = __ballot_sync(0xffffffffu, in);
        if ((threadIdx.x & 31) == 0 && b)
            atomicAdd(count, __popc(b));
    }
}

// ------------------------------------------------------------------ grid barrier
struct GridSync {
    unsigned int count;
    unsigned int gen;
    int abort;
    int skip;  // test hook: block 0 leaves at the first barrier without arriving
};

// Sense-reversing counter barrier over all CTAs of a cooperative launch.
// Every wait is bounded: after timeout_ns the CTA sets `abort` and status =
// RF_ERR_TIMEOUT and returns false; waiters that see `abort` return false too.
__device__ bool grid_barrier(GridSync *gs, int *status, long long timeout_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int *vgen = &gs->gen;
        volatile int *vabort = &gs->abort;
        if (*vabort) {
            ok = 0;
        } else if (gs->skip && blockIdx.x == 0) {
            ok = 0;  // leave without arriving
        } else {
            const unsigned int g = *vgen;
            __threadfence();
            const unsigned int prev = atomicAdd(&gs->count, 1u);
            if (prev == gridDim.x - 1) {
                atomicExch(&gs->count, 0u);
                __threadfence();
                atomicAdd(&gs->gen, 1u);
            } else {
                const long long t0 = global_ns();
                unsigned int ns = 32;
                while (*vgen == g) {
                    if (*vabort) {
                        ok = 0;
                        break;
                    }
                    if (global_ns() - t0 > timeout_ns) {
                        atomicExch(&gs->abort, 1);
                        atomicCAS(status, 0, RF_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(ns);
                    if (ns < 256)
                        ns <<= 1;
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------------------ persistent PFO kernel
struct TrackParams {
    VolumeDesc V;
    Intr K;
    const float *depth, *prev_depth;
    int stride, nw, m;
    const float *pst;
    int n;
    const float *prev_pose;  // device float[7]
    float *out_pose;         // device float[7]
    rf_frame_stats *stats;   // nullable
    float *scale;            // device float[6]: r_0 in, r_1 out
    float4 *pts, *cpts;
    int *block_counts;
    double *part_S;
    int *part_n;
    int max_chunks;
    int *unit_ctr;           // [RF_MAX_ITERS] fitness work-unit counters, zero at launch
    double *aps;             // [grid][APW]
    GridSync *gs;
    int *status;
    float tau, beta, eps, stop_eps;
    int k_max, flags;
    long long timeout_ns;
};

struct TrackState {  // identical in every CTA (computed redundantly in a fixed order)
    Pose c;
    Pose prev;
    float r[6];
    float r1[6];
    float rho_carry;
    float rho_ref;
    int empty_run;
    int nO;
    int stop;
    int offset;  // this CTA's first slot in the compacted point array
    long long lookups;
};

// Block-wide exclusive scan of 0/1 flags over blockDim.x threads; returns the
// prefix of this thread and writes the block total to *total.
__device__ __forceinline__ int block_scan_flag(int flag, int *warp_tot, int *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned b = __ballot_sync(0xffffffffu, flag);
    const int in_warp = __popc(b & ((1u << lane) - 1u));
    if (lane == 0)
        warp_tot[w] = __popc(b);
    __syncthreads();
    int before = 0, tot = 0;
    for (int k = 0; k < nw; ++k) {
        if (k < w)
            before += warp_tot[k];
        tot += warp_tot[k];
    }
    __syncthreads();
    *total = tot;
    return before + in_warp;
}

template <int DT, int MODE>
__global__ void __launch_bounds__(FIT_THREADS, RF_PFO_MIN_BLOCKS) pfo_kernel(TrackParams P)
{
    extern __shared__ float4 smem_pts[];
    __shared__ TrackState st;
    __shared__ int warp_tot[FIT_WARPS];
    __shared__ double red_d[FIT_WARPS][9];
    __shared__ float red_f[FIT_WARPS][2];
    __shared__ int red_i[FIT_WARPS][2];

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int G = gridDim.x, b = blockIdx.x;
    const int total_warps = G * FIT_WARPS;
    const bool overlap_on = (P.flags & RF_OVERLAP) != 0;
    const bool normalize = (P.flags & RF_NORMALIZE) != 0;

    // ---- prologue: unproject the frame (a1) and load the initial PST state
    for (int j = b * blockDim.x + tid; j < P.m; j += G * blockDim.x) {
        float4 p;
        unproject_point(P.depth, P.K, P.stride, P.nw, j, p);
        P.pts[j] = p;
    }
    if (tid == 0) {
        for (int a = 0; a < 4; ++a) {
            st.c.q[a] = __ldcg(&P.prev_pose[a]);
            st.prev.q[a] = st.c.q[a];
        }
        for (int a = 0; a < 3; ++a) {
            st.c.t[a] = __ldcg(&P.prev_pose[4 + a]);
            st.prev.t[a] = st.c.t[a];
        }
        for (int d = 0; d < 6; ++d) {
            st.r[d] = __ldcg(&P.scale[d]);
            st.r1[d] = st.r[d];
        }
        st.rho_carry = 0.f;
        st.empty_run = 0;
        st.stop = 0;
        st.lookups = 0;
    }
    if (!grid_barrier(P.gs, P.status, P.timeout_ns))
        return;

    // contiguous point range of this CTA for the overlap compaction
    const int seg = (P.m + G - 1) / G;
    const int jb = min(P.m, b * seg), je = min(P.m, jb + seg);
    int k = 0;
    for (k = 1; k <= P.k_max; ++k) {
        // ---- phase A: overlap set O_k with s*_{k-1} (Eq. validness), count per CTA
        float Rc[9], Rp[9];
        quat_rot(st.c.q, Rc);
        quat_rot(st.prev.q, Rp);
        int cnt = 0;
        for (int j0 = jb; j0 < je; j0 += blockDim.x) {
            const int j = j0 + tid;
            int f = 0;
            if (j < je) {
                const float4 p = __ldcg(&P.pts[j]);
                f = overlap_on ? overlap_test(p, Rc, st.c.t, Rp, st.prev.t, P.prev_depth, P.K) : (p.w != 0.f);
            }
            int tot;
            block_scan_flag(f, warp_tot, &tot);
            cnt += tot;
        }
        if (tid == 0)
            P.block_counts[b] = cnt;
        if (!grid_barrier(P.gs, P.status, P.timeout_ns))
            return;
        // ---- phase A': offsets and order-preserving compaction
        if (w == 0) {
            int before = 0, tot = 0;
            for (int q = lane; q < G; q += 32) {
                const int c = __ldcg(&P.block_counts[q]);
                tot += c;
                before += (q < b) ? c : 0;
            }
            for (int o = 16; o > 0; o >>= 1) {
                tot += __shfl_xor_sync(0xffffffffu, tot, o);
                before += __shfl_xor_sync(0xffffffffu, before, o);
            }
            if (lane == 0) {
                st.nO = tot;
                st.offset = before;
            }
        }
        __syncthreads();
        const int nO = st.nO;
        if (nO == 0) {  // identical decision in every CTA
            if (b == 0 && tid == 0) {
                atomicCAS(P.status, 0, RF_ERR_EMPTY);
                if (P.stats) {
                    rf_iter_stats &row = P.stats->it[k - 1];
                    memset(&row, 0, sizeof row);
                    row.k = k;
                    row.stop = 4;
                }
            }
            break;
        }
        {
            int base = st.offset;
            for (int j0 = jb; j0 < je; j0 += blockDim.x) {
                const int j = j0 + tid;
                int f = 0;
                float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < je) {
                    p = __ldcg(&P.pts[j]);
                    f = overlap_on ? overlap_test(p, Rc, st.c.t, Rp, st.prev.t, P.prev_depth, P.K) : (p.w != 0.f);
                }
                int tot;
                const int pos = block_scan_flag(f, warp_tot, &tot);
                if (f)
                    P.cpts[base + pos] = p;
                base += tot;
            }
        }
        if (!grid_barrier(P.gs, P.status, P.timeout_ns))
            return;
        // ---- phase B: fitness of every particle (Eq. normallh), partial sums per chunk
        FitParams fp;
        fp.pst = P.pst;
        fp.n = P.n;
        fp.c = st.c;
        for (int d = 0; d < 6; ++d)
            fp.r[d] = st.r[d];
        fp.l1 = (P.flags & RF_L1) != 0;
        fp.right_mult = (P.flags & RF_RIGHT_MULT) != 0;
        const Split sp = make_split(P.n, nO, total_warps, P.max_chunks);
        fitness_units<DT, MODE, true>(P.V, P.cpts, nO, fp, sp, P.part_S, P.part_n, smem_pts, b * FIT_WARPS + w,
                                      total_warps, lane, w, P.unit_ctr + (k - 1));
        if (!grid_barrier(P.gs, P.status, P.timeout_ns))
            return;
        // ---- phase B': per-particle totals, rho, APS partial sums (Eq. ebs, wafit)
        if (tid == 0) {
            double S0;
            int n0;
            particle_total(P.part_S, P.part_n, P.n, sp.n_chunks, 0, true, S0, n0);
            const float rho0 = fitness_rho(S0, nO, P.tau, normalize);
            st.rho_ref = (k == 1 || (P.flags & RF_RHO_REF_CENTER)) ? rho0 : st.rho_carry;
        }
        __syncthreads();
        const float rho_ref = st.rho_ref;
        double sw = 0.0, swr = 0.0, swd[6] = {0, 0, 0, 0, 0, 0};
        int naps = 0, amax = -1, a2 = -1;
        float rmax = -1.f, r2 = -1.f;
        for (int i = b * blockDim.x + tid; i < P.n; i += G * blockDim.x) {
            double S;
            int nv;
            particle_total(P.part_S, P.part_n, P.n, sp.n_chunks, i, true, S, nv);
            const float rho = fitness_rho(S, nO, P.tau, normalize);
            if (rho > rmax) {
                r2 = rmax;
                a2 = amax;
                rmax = rho;
                amax = i;
            } else if (rho > r2) {
                r2 = rho;
                a2 = i;
            }
            if (rho > rho_ref) {
                const double wgt = (double)(rho - rho_ref);
                ++naps;
                sw += wgt;
                swr += wgt * (double)rho;
#pragma unroll
                for (int d = 0; d < 6; ++d)
                    swd[d] += wgt * (double)(st.r[d] * __ldg(&P.pst[(size_t)d * P.n + i]));
            }
        }
        (void)a2;
        // block reduction in a fixed order: xor-shuffle tree, then warps in order
        for (int o = 16; o > 0; o >>= 1) {
            sw += __shfl_xor_sync(0xffffffffu, sw, o);
            swr += __shfl_xor_sync(0xffffffffu, swr, o);
#pragma unroll
            for (int d = 0; d < 6; ++d)
                swd[d] += __shfl_xor_sync(0xffffffffu, swd[d], o);
            naps += __shfl_xor_sync(0xffffffffu, naps, o);
            const float om = __shfl_xor_sync(0xffffffffu, rmax, o);
            const int oa = __shfl_xor_sync(0xffffffffu, amax, o);
            const float o2 = __shfl_xor_sync(0xffffffffu, r2, o);
            // merge (rmax, amax, r2) with (om, oa, o2); lowest index wins ties
            float n2 = fmaxf(r2, o2);
            if (om > rmax || (om == rmax && oa >= 0 && (amax < 0 || oa < amax))) {
                n2 = fmaxf(n2, rmax);
                rmax = om;
                amax = oa;
            } else {
                n2 = fmaxf(n2, om);
            }
            r2 = n2;
        }
        if (lane == 0) {
            red_d[w][0] = sw;
            red_d[w][1] = swr;
            for (int d = 0; d < 6; ++d)
                red_d[w][2 + d] = swd[d];
            red_i[w][0] = naps;
            red_i[w][1] = amax;
            red_f[w][0] = rmax;
            red_f[w][1] = r2;
        }
        __syncthreads();
        if (tid == 0) {
            double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            int na = 0, am = -1;
            float rm = -1.f, rs = -1.f;
            for (int q = 0; q < FIT_WARPS; ++q) {
                for (int e = 0; e < 8; ++e)
                    acc[e] += red_d[q][e];
                na += red_i[q][0];
                const float om = red_f[q][0];
                const int oa = red_i[q][1];
                float n2 = fmaxf(rs, red_f[q][1]);
                if (om > rm || (om == rm && oa >= 0 && (am < 0 || oa < am))) {
                    n2 = fmaxf(n2, rm);
                    rm = om;
                    am = oa;
                } else {
                    n2 = fmaxf(n2, om);
                }
                rs = n2;
            }
            double *out = P.aps + (size_t)b * APW;
            for (int e = 0; e < 8; ++e)
                out[e] = acc[e];
            out[8] = (double)na;
            out[9] = (double)rm;
            out[10] = (double)am;
            out[11] = (double)rs;
        }
        if (!grid_barrier(P.gs, P.status, P.timeout_ns))
            return;
        // ---- phase C: every CTA reduces the APS partials in the same order and
        // updates the PST state (Eq. ebs, wafit, rsdir, rsinter, momentum)
        if (w == 0) {
            double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            double na = 0.0;
            float rm = -1.f, rs = -1.f;
            int am = -1;
            for (int q = lane; q < G; q += 32) {
                const double *in = P.aps + (size_t)q * APW;
                for (int e = 0; e < 8; ++e)
                    acc[e] += __ldcg(&in[e]);
                na += __ldcg(&in[8]);
                const float om = (float)__ldcg(&in[9]);
                const int oa = (int)__ldcg(&in[10]);
                float n2 = fmaxf(rs, (float)__ldcg(&in[11]));
                if (om > rm || (om == rm && oa >= 0 && (am < 0 || oa < am))) {
                    n2 = fmaxf(n2, rm);
                    rm = om;
                    am = oa;
                } else {
                    n2 = fmaxf(n2, om);
                }
                rs = n2;
            }
            for (int o = 16; o > 0; o >>= 1) {
                for (int e = 0; e < 8; ++e)
                    acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
                na += __shfl_xor_sync(0xffffffffu, na, o);
                const float om = __shfl_xor_sync(0xffffffffu, rm, o);
                const int oa = __shfl_xor_sync(0xffffffffu, am, o);
                const float o2 = __shfl_xor_sync(0xffffffffu, rs, o);
                float n2 = fmaxf(rs, o2);
                if (om > rm || (om == rm && oa >= 0 && (am < 0 || oa < am))) {
                    n2 = fmaxf(n2, rm);
                    rm = om;
                    am = oa;
                } else {
                    n2 = fmaxf(n2, om);
                }
                rs = n2;
            }
            if (lane == 0) {
                const int n_aps = (int)na;
                float dbar[6], rhat[6];
                float rho_t;
                Pose s_new;
                if (n_aps > 0) {
                    double nv2 = 0.0;
                    double db[6];
                    for (int d = 0; d < 6; ++d) {
                        db[d] = acc[2 + d] / acc[0];
                        nv2 += db[d] * db[d];
                    }
                    const double nv = sqrt(nv2);
                    rho_t = (float)(acc[1] / acc[0]);
                    for (int d = 0; d < 6; ++d) {
                        dbar[d] = (float)db[d];
                        const double dir = nv < 1e-12 ? 0.40824829046386302 : fabs(db[d]) / nv;
                        rhat[d] = (float)((1.0 - (double)rho_t) * dir + (double)P.eps);
                    }
                    compose_offset(st.c, dbar, (P.flags & RF_RIGHT_MULT) != 0, s_new);
                    st.empty_run = 0;
                } else {
                    rho_t = rho_ref;
                    for (int d = 0; d < 6; ++d) {
                        dbar[d] = 0.f;
                        rhat[d] = (float)(2.0 * (1.0 - (double)rho_ref) * 0.40824829046386302 + (double)P.eps);
                    }
                    s_new = st.c;
                    st.empty_run += 1;
                }
                for (int d = 0; d < 6; ++d)
                    st.r[d] = P.beta * st.r[d] + (1.f - P.beta) * rhat[d];
                st.rho_carry = rho_t;
                st.c = s_new;
                if (k == 1)
                    for (int d = 0; d < 6; ++d)
                        st.r1[d] = st.r[d];
                float step = 0.f;
                for (int d = 0; d < 6; ++d)
                    step = fmaxf(step, fabsf(dbar[d]));
                int stop = 0;
                if (st.empty_run >= 2)
                    stop = 1;
                else if (n_aps > 0 && step < P.stop_eps)
                    stop = 2;
                else if (k == P.k_max)
                    stop = 3;
                st.stop = stop;
                st.lookups += (long long)nO * (long long)P.n;
                if (b == 0 && P.stats) {
                    rf_iter_stats &row = P.stats->it[k - 1];
                    row.k = k;
                    row.n_overlap = nO;
                    row.n_aps = n_aps;
                    row.argmax = am;
                    row.rho_ref = rho_ref;
                    row.rho_tilde = rho_t;
                    row.rho_max = rm;
                    row.rho_second = rs;
                    for (int a = 0; a < 4; ++a)
                        row.pose[a] = st.c.q[a];
                    for (int a = 0; a < 3; ++a)
                        row.pose[4 + a] = st.c.t[a];
                    for (int d = 0; d < 6; ++d) {
                        row.scale[d] = st.r[d];
                        row.offset[d] = dbar[d];
                    }
                    row.stop = stop;
                }
            }
        }
        __syncthreads();
        if (st.stop)
            break;
    }
    // ---- epilogue (CTA 0): final pose, r_1 for the next frame, summary
    if (b == 0 && tid == 0) {
        for (int a = 0; a < 4; ++a)
            P.out_pose[a] = st.c.q[a];
        for (int a = 0; a < 3; ++a)
            P.out_pose[4 + a] = st.c.t[a];
        for (int d = 0; d < 6; ++d)
            P.scale[d] = st.r1[d];
        if (P.stats) {
            P.stats->iters = k > P.k_max ? P.k_max : k;
            P.stats->status = *((volatile int *)P.status);
            P.stats->n_points = P.m;
            P.stats->lookups = st.lookups;
            for (int d = 0; d < 6; ++d)
                P.stats->r1[d] = st.r1[d];
        }
    }
}

__global__ void set_int_kernel(int *dst, int v) { *dst = v; }

__global__ void set_pose_kernel(float *dst, Pose p)
{
    for (int a = 0; a < 4; ++a)
        dst[a] = p.q[a];
    for (int a = 0; a < 3; ++a)
        dst[4 + a] = p.t[a];
}

// Projective fusion at a pose held on the device (sequence mode); skipped if
// the tracker reported an error for this frame.
rf_status launch_integrate_dev(const VolumeDesc &V, const float *depth, const Intr &K, const float *pose_dev,
                               const int *status_dev, cudaStream_t s);

// ------------------------------------------------------------------ kernel tables
using FitFn = void (*)(VolumeDesc, const float4 *, int, FitParams, Split, double *, int *);
using PfoFn = void (*)(TrackParams);

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
template <int DT> static PfoFn pfo_fn(int mode)
{
    switch (mode) {
    case 0:
        return pfo_kernel<DT, 0>;
    case 1:
        return pfo_kernel<DT, 1>;
    case 2:
        return pfo_kernel<DT, 2>;
    default:
        return pfo_kernel<DT, 3>;
    }
}
static PfoFn pfo_fn(int dtype, int mode)
{
    return dtype == RF_F32 ? pfo_fn<RF_F32>(mode) : dtype == RF_F16 ? pfo_fn<RF_F16>(mode) : pfo_fn<RF_I16>(mode);
}
static int mode_of(int flags) { return ((flags & RF_NEAREST) ? 1 : 0) | ((flags & RF_COMPENSATED) ? 0 : 2); }

static rf_status check_params(const rf_params *p)
{
    RF_CHECK_ARG(p != nullptr, "null params");
    RF_CHECK_ARG(p->k_max >= 1 && p->k_max <= RF_MAX_ITERS, "k_max out of range");
    RF_CHECK_ARG(p->stride >= 1, "stride must be >= 1");
    RF_CHECK_ARG(p->tau > 0.f, "tau must be positive");
    RF_CHECK_ARG(p->beta >= 0.f && p->beta <= 1.f, "beta must lie in [0, 1]");
    return RF_OK;
}

static int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

}  // namespace rf

// ------------------------------------------------------------------ tracker handle
struct rf_tracker_s {
    rf_volume vol;
    const float *pst;
    int n;
    rf_params p;
    int max_w, max_h, m_max;
    int grid;          // cooperative grid size (CTAs)
    int max_chunks;
    size_t smem;
    // device scratch
    float4 *pts, *cpts;
    int *block_counts;
    int *unit_ctr;     // RF_MAX_ITERS work-unit counters of the fitness phase
    double *part_S;
    int *part_n;
    double *aps;
    rf::GridSync *gs;
    int *status;
    float *scale;
    float *pose_ring;  // 2 x 7
    float *depth_ring; // 2 x max_w * max_h
    int cur;           // ring slot of the previous frame
    int debug_skip;
    long long timeout_ns;
    int grid_mode;     // kernel variant the grid was sized for
};

using namespace rf;

static rf_status size_grid(rf_tracker tr)
{
    const int mode = mode_of(tr->p.flags);
    PfoFn fn = pfo_fn(tr->vol->d.dtype, mode);
    const size_t smem = (size_t)FIT_WARPS * CHUNK_MAX * sizeof(float4);
    RF_CUDA(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, FIT_THREADS, smem));
    if (per_sm < 1) {
        set_error("pfo kernel cannot be resident");
        return RF_ERR_CUDA;
    }
    tr->grid = std::min(per_sm, MAX_CTAS_PER_SM) * sm_count();
    tr->smem = smem;
    tr->grid_mode = mode;
    return RF_OK;
}

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
                          const rf_pose *pose_cur, const rf_pose *pose_prev, uint8_t *mask_dev, int *count_dev,
                          void *stream)
{
    RF_CHECK_ARG(points_dev && prev_depth_dev && K && pose_cur && pose_prev && mask_dev, "null pointer");
    RF_CHECK_ARG(m >= 0, "negative size");
    cudaStream_t s = (cudaStream_t)stream;
    if (count_dev)
        RF_CUDA(cudaMemsetAsync(count_dev, 0, sizeof(int), s));
    if (m == 0)
        return RF_OK;
    overlap_kernel<<<(m + 255) / 256, 256, 0, s>>>((const float4 *)points_dev, m, prev_depth_dev, to_intr(*K),
                                                   to_pose(*pose_cur), to_pose(*pose_prev), mask_dev, count_dev);
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

void rf_tracker_destroy(rf_tracker tr)
{
    if (!tr)
        return;
    cudaFree(tr->pts);
    cudaFree(tr->cpts);
    cudaFree(tr->block_counts);
    cudaFree(tr->part_S);
    cudaFree(tr->part_n);
    cudaFree(tr->aps);
    cudaFree(tr->unit_ctr);
    cudaFree(tr->gs);
    cudaFree(tr->status);
    cudaFree(tr->scale);
    cudaFree(tr->pose_ring);
    cudaFree(tr->depth_ring);
    delete tr;
}

rf_status rf_tracker_create(rf_volume v, const float *pst_dev, int n, const rf_params *p, int max_width,
                            int max_height, rf_tracker *out)
{
    RF_CHECK_ARG(out != nullptr, "null output");
    *out = nullptr;
    RF_CHECK_ARG(v && pst_dev, "null pointer");
    RF_CHECK_ARG(n >= 1, "n must be >= 1");
    RF_CHECK_ARG(max_width > 0 && max_height > 0, "bad frame size");
    rf_status cs = check_params(p);
    if (cs != RF_OK)
        return cs;
    rf_tracker tr = new rf_tracker_s();
    memset(tr, 0, sizeof *tr);
    tr->vol = v;
    tr->pst = pst_dev;
    tr->n = n;
    tr->p = *p;
    tr->max_w = max_width;
    tr->max_h = max_height;
    tr->timeout_ns = 1000000000ll;
    // points for the finest stride 1 so that the stride may change later
    tr->m_max = max_width * max_height;
    rf_status st = size_grid(tr);
    if (st != RF_OK) {
        delete tr;
        return st;
    }
    // the grid can only shrink with other modes; size scratch for the largest
    tr->max_chunks = max_chunks_for(n, tr->m_max, tr->grid * FIT_WARPS);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess)
            e = cudaMalloc(ptr, bytes);
    };
    alloc((void **)&tr->pts, sizeof(float4) * tr->m_max);
    alloc((void **)&tr->cpts, sizeof(float4) * tr->m_max);
    alloc((void **)&tr->block_counts, sizeof(int) * (size_t)MAX_CTAS_PER_SM * sm_count());
    alloc((void **)&tr->part_S, sizeof(double) * (size_t)tr->max_chunks * n);
    alloc((void **)&tr->part_n, sizeof(int) * (size_t)tr->max_chunks * n);
    alloc((void **)&tr->aps, sizeof(double) * APW * (size_t)MAX_CTAS_PER_SM * sm_count());
    alloc((void **)&tr->unit_ctr, sizeof(int) * RF_MAX_ITERS);
    alloc((void **)&tr->gs, sizeof(GridSync));
    alloc((void **)&tr->status, sizeof(int));
    alloc((void **)&tr->scale, sizeof(float) * 6);
    alloc((void **)&tr->pose_ring, sizeof(float) * 14);
    alloc((void **)&tr->depth_ring, sizeof(float) * 2 * (size_t)tr->m_max);
    if (e != cudaSuccess) {
        rf_tracker_destroy(tr);
        return cuda_fail(e, "rf_tracker_create");
    }
    const float ones[6] = {1, 1, 1, 1, 1, 1};
    e = cudaMemcpy(tr->scale, ones, sizeof ones, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemset(tr->status, 0, sizeof(int));
    if (e != cudaSuccess) {
        rf_tracker_destroy(tr);
        return cuda_fail(e, "rf_tracker_create");
    }
    *out = tr;
    return RF_OK;
}

rf_status rf_tracker_get_scale(rf_tracker tr, float r_host[6])
{
    RF_CHECK_ARG(tr && r_host, "null pointer");
    RF_CUDA(cudaMemcpy(r_host, tr->scale, sizeof(float) * 6, cudaMemcpyDeviceToHost));
    return RF_OK;
}

rf_status rf_tracker_set_scale(rf_tracker tr, const float r_host[6])
{
    RF_CHECK_ARG(tr && r_host, "null pointer");
    RF_CUDA(cudaMemcpy(tr->scale, r_host, sizeof(float) * 6, cudaMemcpyHostToDevice));
    return RF_OK;
}

rf_status rf_tracker_set_params(rf_tracker tr, const rf_params *p)
{
    RF_CHECK_ARG(tr != nullptr, "null tracker");
    rf_status cs = check_params(p);
    if (cs != RF_OK)
        return cs;
    tr->p = *p;
    return RF_OK;
}

rf_status rf_tracker_debug_skip_barrier(rf_tracker tr, int enable, int timeout_ms)
{
    RF_CHECK_ARG(tr != nullptr, "null tracker");
    RF_CHECK_ARG(timeout_ms >= 1 && timeout_ms <= 10000, "timeout_ms must be in [1, 10000]");
    tr->debug_skip = enable ? 1 : 0;
    tr->timeout_ns = (long long)timeout_ms * 1000000ll;
    return RF_OK;
}

rf_status rf_tracker_last_status(rf_tracker tr)
{
    RF_CHECK_ARG(tr != nullptr, "null tracker");
    int h = 0;
    RF_CUDA(cudaMemcpy(&h, tr->status, sizeof(int), cudaMemcpyDeviceToHost));
    return h;
}

rf_status pfo_track_frame_async(rf_tracker tr, const float *depth_dev, const float *prev_depth_dev,
                                const rf_intrinsics *K, const float *prev_pose_dev, float *out_pose_dev,
                                rf_frame_stats *stats_dev, void *stream)
{
    RF_CHECK_ARG(tr && depth_dev && prev_depth_dev && K && prev_pose_dev && out_pose_dev, "null pointer");
    RF_CHECK_ARG(K->width > 0 && K->height > 0 && K->width <= tr->max_w && K->height <= tr->max_h,
                 "frame larger than the tracker was created for");
    cudaStream_t s = (cudaStream_t)stream;
    const int mode = mode_of(tr->p.flags);
    if (mode != tr->grid_mode) {
        rf_status st = size_grid(tr);
        if (st != RF_OK)
            return st;
    }
    TrackParams P;
    memset(&P, 0, sizeof P);
    P.V = tr->vol->d;
    P.K = to_intr(*K);
    P.depth = depth_dev;
    P.prev_depth = prev_depth_dev;
    P.stride = tr->p.stride;
    P.nw = (K->width + P.stride - 1) / P.stride;
    P.m = P.nw * ((K->height + P.stride - 1) / P.stride);
    P.pst = tr->pst;
    P.n = tr->n;
    P.prev_pose = prev_pose_dev;
    P.out_pose = out_pose_dev;
    P.stats = stats_dev;
    P.scale = tr->scale;
    P.pts = tr->pts;
    P.cpts = tr->cpts;
    P.block_counts = tr->block_counts;
    P.part_S = tr->part_S;
    P.part_n = tr->part_n;
    P.max_chunks = tr->max_chunks;
    P.aps = tr->aps;
    P.unit_ctr = tr->unit_ctr;
    P.gs = tr->gs;
    P.status = tr->status;
    P.tau = tr->p.tau;
    P.beta = tr->p.beta;
    P.eps = tr->p.eps;
    P.stop_eps = tr->p.stop_eps;
    P.k_max = tr->p.k_max;
    P.flags = tr->p.flags;
    P.timeout_ns = tr->timeout_ns;
    // barrier state and status word are reset on the stream (memsets and a
    // one-thread kernel), so the launch sequence stays capturable
    RF_CUDA(cudaMemsetAsync(tr->status, 0, sizeof(int), s));
    RF_CUDA(cudaMemsetAsync(tr->gs, 0, sizeof(GridSync), s));
    RF_CUDA(cudaMemsetAsync(tr->unit_ctr, 0, sizeof(int) * RF_MAX_ITERS, s));
    if (tr->debug_skip) {
        set_int_kernel<<<1, 1, 0, s>>>(&tr->gs->skip, 1);
        RF_CUDA(cudaGetLastError());
    }
    if (stats_dev)
        RF_CUDA(cudaMemsetAsync(stats_dev, 0, sizeof(rf_frame_stats), s));
    void *args[] = {&P};
    PfoFn fn = pfo_fn(tr->vol->d.dtype, mode);
    RF_CUDA(cudaLaunchCooperativeKernel((const void *)fn, dim3(tr->grid), dim3(FIT_THREADS), args, tr->smem, s));
    if (tr->debug_skip) {
        RF_CUDA(cudaStreamSynchronize(s));
        tr->debug_skip = 0;
        tr->timeout_ns = 1000000000ll;
    }
    return RF_OK;
}

rf_status pfo_track_frame(rf_tracker tr, const float *depth_dev, const float *prev_depth_dev, const rf_intrinsics *K,
                          const rf_pose *prev_pose, rf_pose *out_pose, rf_frame_stats *stats_host, void *stream)
{
    RF_CHECK_ARG(tr && prev_pose && out_pose, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    float *pp = tr->pose_ring, *po = tr->pose_ring + 7;
    set_pose_kernel<<<1, 1, 0, s>>>(pp, to_pose(*prev_pose));
    RF_CUDA(cudaGetLastError());
    rf_frame_stats *sd = nullptr;
    if (stats_host)
        RF_CUDA(cudaMallocAsync((void **)&sd, sizeof(rf_frame_stats), s));
    rf_status st = pfo_track_frame_async(tr, depth_dev, prev_depth_dev, K, pp, po, sd, s);
    if (st != RF_OK) {
        if (sd)
            cudaFreeAsync(sd, s);
        return st;
    }
    float h[7];
    int hs = 0;
    RF_CUDA(cudaMemcpyAsync(h, po, sizeof h, cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaMemcpyAsync(&hs, tr->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (sd) {
        RF_CUDA(cudaMemcpyAsync(stats_host, sd, sizeof(rf_frame_stats), cudaMemcpyDeviceToHost, s));
        RF_CUDA(cudaFreeAsync(sd, s));
    }
    RF_CUDA(cudaStreamSynchronize(s));
    for (int a = 0; a < 4; ++a)
        out_pose->q[a] = h[a];
    for (int a = 0; a < 3; ++a)
        out_pose->t[a] = h[4 + a];
    if (hs != 0)
        set_error("pfo_track_frame: device status %d", hs);
    return hs;
}

rf_status rf_sequence_start(rf_tracker tr, const float *depth, int depth_on_host, const rf_intrinsics *K,
                            const rf_pose *pose, void *stream)
{
    RF_CHECK_ARG(tr && depth && K && pose, "null pointer");
    RF_CHECK_ARG(K->width > 0 && K->height > 0 && K->width <= tr->max_w && K->height <= tr->max_h, "bad frame size");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t px = (size_t)K->width * K->height;
    tr->cur = 0;
    float *slot = tr->depth_ring;
    RF_CUDA(cudaMemcpyAsync(slot, depth, px * sizeof(float),
                            depth_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    set_pose_kernel<<<1, 1, 0, s>>>(tr->pose_ring, to_pose(*pose));
    RF_CUDA(cudaGetLastError());
    RF_CUDA(cudaMemsetAsync(tr->status, 0, sizeof(int), s));
    return launch_integrate_dev(tr->vol->d, slot, to_intr(*K), tr->pose_ring, nullptr, s);
}

rf_status rf_sequence_step(rf_tracker tr, const float *depth, int depth_on_host, const rf_intrinsics *K,
                           rf_pose *out_pose_host, float *out_pose_dev, rf_frame_stats *stats_dev, void *stream)
{
    RF_CHECK_ARG(tr && depth && K, "null pointer");
    RF_CHECK_ARG(K->width > 0 && K->height > 0 && K->width <= tr->max_w && K->height <= tr->max_h, "bad frame size");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t px = (size_t)K->width * K->height;
    const int prev = tr->cur, nxt = 1 - tr->cur;
    float *dprev = tr->depth_ring + (size_t)prev * tr->m_max, *dnext = tr->depth_ring + (size_t)nxt * tr->m_max;
    float *pprev = tr->pose_ring + 7 * prev, *pnext = tr->pose_ring + 7 * nxt;
    RF_CUDA(cudaMemcpyAsync(dnext, depth, px * sizeof(float),
                            depth_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    rf_status st = pfo_track_frame_async(tr, dnext, dprev, K, pprev, pnext, stats_dev, s);
    if (st != RF_OK)
        return st;
    st = launch_integrate_dev(tr->vol->d, dnext, to_intr(*K), pnext, tr->status, s);
    if (st != RF_OK)
        return st;
    tr->cur = nxt;
    if (out_pose_dev)
        RF_CUDA(cudaMemcpyAsync(out_pose_dev, pnext, 7 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (out_pose_host) {
        float h[7];
        int hs = 0;
        RF_CUDA(cudaMemcpyAsync(h, pnext, sizeof h, cudaMemcpyDeviceToHost, s));
        RF_CUDA(cudaMemcpyAsync(&hs, tr->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        RF_CUDA(cudaStreamSynchronize(s));
        for (int a = 0; a < 4; ++a)
            out_pose_host->q[a] = h[a];
        for (int a = 0; a < 3; ++a)
            out_pose_host->t[a] = h[4 + a];
        if (hs != 0)
            set_error("rf_sequence_step: device status %d", hs);
        return hs;
    }
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
