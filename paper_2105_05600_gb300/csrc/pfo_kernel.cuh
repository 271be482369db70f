// pfo_kernel.cuh -- the persistent PFO kernel (Algorithm 1 for one frame of one or
// several sequences) and its launch descriptors, shared by the host code in pfo.cu
// and the per-storage-type translation units that instantiate the kernel
// (pfo_kernels_f32.cu, pfo_kernels_f16.cu, pfo_kernels_i16.cu, compiled in parallel).
#pragma once
#include <math.h>
#include <string.h>

#include <algorithm>

#include "fitness.cuh"

namespace rf {

constexpr int MAX_BATCH = RF_MAX_BATCH;
constexpr int MAX_LEVELS = RF_MAX_LEVELS;
// The fitness split of a sequence is computed for this warp count (not for the
// actual grid), so a sequence's results do not depend on the launch shape or on
// the other sequences of a batch.
constexpr int WORK_WARPS_DEFAULT = 3648;
constexpr int WORK_WARPS_MAX = 7296;

rf_status launch_integrate_dev(const VolumeDesc &V, const float *depth, const Intr &K, const float *pose_dev,
                               const int *status_dev, cudaStream_t s);

// ------------------------------------------------------------------ launch descriptors
struct ProblemDesc {
    VolumeDesc V;
    Intr K;
    const float *depth, *prev_depth;
    const float *pst;  // template, structure of arrays, leading dimension n_tmpl
    int n_tmpl;
    int n_levels;
    int lvl_n[MAX_LEVELS], lvl_stride[MAX_LEVELS], lvl_nw[MAX_LEVELS], lvl_m[MAX_LEVELS], lvl_off[MAX_LEVELS];
    int m_all;  // points of all levels (concatenated in pts at lvl_off)
    const float *prev_pose;
    const float *init_pose;  // c_0 (NULL: prev_pose)
    const int *run_flag;     // NULL, or skip the frame when *run_flag == 0 at launch
    float *out_pose;
    rf_frame_stats *stats;
    float *scale;  // r_0 in, r_1 out
    float4 *pts, *cpts;
    double *part_S;
    int *part_n;
    int max_chunks;
    int *status;
    float tau, beta, eps, stop_eps;
    int k_max, flags;
};

struct GridSync {
    unsigned int count;
    unsigned int gen;
    int abort;
    int skip;  // test hook: block 0 leaves at the first barrier without arriving
};

struct BatchParams {
    ProblemDesc prob[MAX_BATCH];
    int B;
    int k_max_all;
    int work_warps;
    GridSync *gs;
    int *unit_ctr;      // [RF_MAX_ITERS], zero at launch
    int *block_counts;  // [grid][MAX_BATCH]
    double *aps;        // [grid][MAX_BATCH][APW]
    long long timeout_ns;
};

// ------------------------------------------------------------------ grid barrier
// Sense-reversing counter barrier over all CTAs of the cooperative launch.  Every
// wait is bounded: after timeout_ns the CTA sets `abort`, marks every sequence's
// status RF_ERR_TIMEOUT and returns false; waiters that see `abort` return false.
static __device__ bool grid_barrier(const BatchParams &P)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        GridSync *gs = P.gs;
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
                    if (global_ns() - t0 > P.timeout_ns) {
                        atomicExch(&gs->abort, 1);
                        for (int p = 0; p < P.B; ++p)
                            atomicCAS(P.prob[p].status, 0, RF_ERR_TIMEOUT);
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

// Block-wide exclusive scan of 0/1 flags; returns this thread's prefix and the total.
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

// Merge (max, argmax, second) with another triple; the lowest index wins ties.
__device__ __forceinline__ void merge_max(float &rm, int &am, float &rs, float om, int oa, float os)
{
    float n2 = fmaxf(rs, os);
    if (om > rm || (om == rm && oa >= 0 && (am < 0 || oa < am))) {
        n2 = fmaxf(n2, rm);
        rm = om;
        am = oa;
    } else {
        n2 = fmaxf(n2, om);
    }
    rs = n2;
}

// Total over the chunk partials of particle i (stored [particle][chunk], coherent
// loads): lane l sums chunks l, l + 32, ... and a fixed butterfly combines the
// lanes; lane 0's result is the total.  The order is fixed, so the same particle
// always gets the same value.
__device__ __forceinline__ void warp_particle_total(const double *part_S, const int *part_n, int n_chunks, int i,
                                                    int lane, double &S, int &nv)
{
    const size_t row = (size_t)i * n_chunks;
    double s = 0.0;
    int c = 0;
    for (int ch = lane; ch < n_chunks; ch += 32) {
        s += __ldcg(&part_S[row + ch]);
        c += __ldcg(&part_n[row + ch]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    S = s;
    nv = c;
}

// Per-sequence state, identical in every CTA (computed redundantly in a fixed order).
struct PState {
    Pose c, prev;
    float r[6], r1[6];
    float rho_carry, rho_ref;
    int empty_run, stop, active, iters;
    int level, n_lvl, m_lvl, off_lvl;
    int nO, offset;
    int groups, n_chunks, chunk, unit_base;
    long long lookups;
};

// ------------------------------------------------------------------ the persistent kernel
template <int DT, int MODE, int LG>
__global__ void __launch_bounds__(FIT_THREADS, RF_PFO_MIN_BLOCKS) pfo_batch_kernel(const __grid_constant__ BatchParams P)
{
    extern __shared__ float4 smem_pts[];
    __shared__ PState st[MAX_BATCH];
    __shared__ int warp_tot[FIT_WARPS];
    __shared__ double red_d[FIT_WARPS][8];
    __shared__ float red_f[FIT_WARPS][2];
    __shared__ int red_i[FIT_WARPS][2];
    __shared__ long long red_v[FIT_WARPS];
    __shared__ int s_total_units;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int G = gridDim.x, b = blockIdx.x;
    const int B = P.B;

    // ---- prologue: unproject the points of every level of every sequence (Eq. unproj)
    {
        long long total = 0;
        for (int p = 0; p < B; ++p)
            total += P.prob[p].m_all;
        for (long long g = (long long)b * blockDim.x + tid; g < total; g += (long long)G * blockDim.x) {
            int p = 0;
            long long base = 0;
            while (g >= base + P.prob[p].m_all) {
                base += P.prob[p].m_all;
                ++p;
            }
            const ProblemDesc &pd = P.prob[p];
            const int j = (int)(g - base);
            int l = 0;
            while (l + 1 < pd.n_levels && j >= pd.lvl_off[l + 1])
                ++l;
            float4 pt;
            unproject_point(pd.depth, pd.K, pd.lvl_stride[l], pd.lvl_nw[l], j - pd.lvl_off[l], pt);
            pd.pts[j] = pt;
        }
    }
    if (tid < B) {
        const ProblemDesc &pd = P.prob[tid];
        PState &s = st[tid];
        const float *c0 = pd.init_pose ? pd.init_pose : pd.prev_pose;
        for (int a = 0; a < 4; ++a) {
            s.c.q[a] = __ldcg(&c0[a]);
            s.prev.q[a] = __ldcg(&pd.prev_pose[a]);
        }
        for (int a = 0; a < 3; ++a) {
            s.c.t[a] = __ldcg(&c0[4 + a]);
            s.prev.t[a] = __ldcg(&pd.prev_pose[4 + a]);
        }
        for (int d = 0; d < 6; ++d)
            s.r[d] = s.r1[d] = __ldcg(&pd.scale[d]);
        s.rho_carry = 0.f;
        s.rho_ref = 0.f;
        s.empty_run = 0;
        // stop code 5: skipped by the caller's run flag (never active, writes nothing)
        s.stop = (pd.run_flag && __ldcg(pd.run_flag) == 0) ? 5 : 0;
        s.iters = 0;
        s.lookups = 0;
    }
    if (!grid_barrier(P))
        return;

    for (int k = 1; k <= P.k_max_all; ++k) {
        if (tid < B) {
            const ProblemDesc &pd = P.prob[tid];
            PState &s = st[tid];
            s.active = (s.stop == 0 && k <= pd.k_max) ? 1 : 0;
            const int l = (k - 1) % pd.n_levels;
            s.level = l;
            s.n_lvl = pd.lvl_n[l];
            s.m_lvl = pd.lvl_m[l];
            s.off_lvl = pd.lvl_off[l];
            if (s.active)
                s.iters = k;
        }
        __syncthreads();
        int T = 0;
        bool any = false;
        for (int p = 0; p < B; ++p)
            if (st[p].active) {
                any = true;
                T += st[p].m_lvl;
            }
        if (!any)
            break;  // identical decision in every CTA
        // ---- phase A: overlap counts per (CTA, sequence) over the concatenated point sets
        const int seg = (T + G - 1) / G;
        const int jb = min(T, b * seg), je = min(T, jb + seg);
        {
            int base = 0;
            for (int p = 0; p < B; ++p) {
                if (!st[p].active)
                    continue;
                const ProblemDesc &pd = P.prob[p];
                const int lo = max(jb, base), hi = min(je, base + st[p].m_lvl);
                int cnt = 0;
                if (lo < hi) {
                    float Rc[9], Rp[9];
                    quat_rot(st[p].c.q, Rc);
                    quat_rot(st[p].prev.q, Rp);
                    const bool overlap_on = (pd.flags & RF_OVERLAP) != 0;
                    const float cell_m = (pd.flags & RF_CELL_MARGIN) ? 1.7320508f * pd.V.voxel : 0.f;
                    for (int j0 = lo; j0 < hi; j0 += blockDim.x) {
                        const int j = j0 + tid;
                        int f = 0;
                        if (j < hi) {
                            const float4 pt = __ldcg(&pd.pts[st[p].off_lvl + (j - base)]);
                            f = overlap_on ? overlap_test(pt, Rc, st[p].c.t, Rp, st[p].prev.t, pd.prev_depth, pd.K, cell_m)
                                           : (pt.w != 0.f);
                        }
                        int tot;
                        block_scan_flag(f, warp_tot, &tot);
                        cnt += tot;
                    }
                }
                if (tid == 0)
                    P.block_counts[(size_t)b * MAX_BATCH + p] = cnt;
                base += st[p].m_lvl;
            }
        }
        if (!grid_barrier(P))
            return;
        // ---- phase A': per-sequence offsets and |O_k|, then the compaction
        for (int p = w; p < B; p += FIT_WARPS) {
            if (!st[p].active)
                continue;
            int before = 0, tot = 0;
            for (int q = lane; q < G; q += 32) {
                const int c = __ldcg(&P.block_counts[(size_t)q * MAX_BATCH + p]);
                tot += c;
                before += (q < b) ? c : 0;
            }
            for (int o = 16; o > 0; o >>= 1) {
                tot += __shfl_xor_sync(0xffffffffu, tot, o);
                before += __shfl_xor_sync(0xffffffffu, before, o);
            }
            if (lane == 0) {
                st[p].nO = tot;
                st[p].offset = before;
            }
        }
        __syncthreads();
        if (tid < B && st[tid].active && st[tid].nO == 0) {  // empty overlap: this sequence stops
            PState &s = st[tid];
            s.stop = 4;
            s.active = 0;
            if (b == 0) {
                atomicCAS(P.prob[tid].status, 0, RF_ERR_EMPTY);
                if (P.prob[tid].stats) {
                    rf_iter_stats &row = P.prob[tid].stats->it[k - 1];
                    memset(&row, 0, sizeof row);
                    row.k = k;
                    row.stop = 4;
                    row.level = s.level;
                    row.n_particles = s.n_lvl;
                }
            }
        }
        __syncthreads();
        {
            int base = 0;
            for (int p = 0; p < B; ++p) {
                if (!(st[p].active || (st[p].stop == 4 && st[p].nO == 0 && st[p].iters == k)))
                    continue;  // only sequences that took part in phase A (their points count in T)
                const ProblemDesc &pd = P.prob[p];
                const int lo = max(jb, base), hi = min(je, base + st[p].m_lvl);
                if (lo < hi && st[p].active) {
                    float Rc[9], Rp[9];
                    quat_rot(st[p].c.q, Rc);
                    quat_rot(st[p].prev.q, Rp);
                    const bool overlap_on = (pd.flags & RF_OVERLAP) != 0;
                    const float cell_m = (pd.flags & RF_CELL_MARGIN) ? 1.7320508f * pd.V.voxel : 0.f;
                    int out = st[p].offset;
                    for (int j0 = lo; j0 < hi; j0 += blockDim.x) {
                        const int j = j0 + tid;
                        int f = 0;
                        float4 pt = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (j < hi) {
                            pt = __ldcg(&pd.pts[st[p].off_lvl + (j - base)]);
                            f = overlap_on ? overlap_test(pt, Rc, st[p].c.t, Rp, st[p].prev.t, pd.prev_depth, pd.K, cell_m)
                                           : (pt.w != 0.f);
                        }
                        int tot;
                        const int pos = block_scan_flag(f, warp_tot, &tot);
                        if (f)
                            pd.cpts[out + pos] = pt;
                        out += tot;
                    }
                }
                base += st[p].m_lvl;
            }
        }
        if (!grid_barrier(P))
            return;
        // ---- phase B: fitness of every particle of every active sequence (Eq. normallh)
        if (tid == 0) {
            int units = 0;
            for (int p = 0; p < B; ++p) {
                PState &s = st[p];
                if (!s.active)
                    continue;
                const Split sp = make_split(s.n_lvl, s.nO, P.work_warps, P.prob[p].max_chunks);
                s.groups = sp.groups;
                s.n_chunks = sp.n_chunks;
                s.chunk = sp.chunk;
                s.unit_base = units;
                units += sp.groups * sp.n_chunks;
            }
            s_total_units = units;
        }
        __syncthreads();
        {
            const int total_units = s_total_units;
            float4 *spts = smem_pts + (size_t)w * CHUNK_MAX;
            int *ctr = P.unit_ctr + (k - 1);
            int t = 0;
            if (lane == 0)
                t = atomicAdd(ctr, 1);
            int u = __shfl_sync(0xffffffffu, t, 0);
            while (u < total_units) {
                if (lane == 0)
                    t = atomicAdd(ctr, 1);
                const int u_next = __shfl_sync(0xffffffffu, t, 0);
                // the last active sequence whose first unit is <= u (active bases increase)
                int p = 0;
                for (int q = 0; q < B; ++q)
                    if (st[q].active && st[q].unit_base <= u)
                        p = q;
                const PState &s = st[p];
                const ProblemDesc &pd = P.prob[p];
                const int local = u - s.unit_base;
                const int ch = local / s.groups, g = local - ch * s.groups;
                const int j0 = ch * s.chunk;
                const int cnt = min(s.chunk, s.nO - j0);
                __syncwarp();
                for (int j = lane; j < cnt; j += 32)
                    spts[j] = __ldcg(&pd.cpts[j0 + j]);
                __syncwarp();
                FitParams fp;
                fp.pst = pd.pst;
                fp.n = s.n_lvl;
                fp.ld = pd.n_tmpl;
                fp.c = s.c;
                for (int d = 0; d < 6; ++d)
                    fp.r[d] = s.r[d];
                fp.l1 = (pd.flags & RF_L1) != 0;
                fp.right_mult = (pd.flags & RF_RIGHT_MULT) != 0;
                const int i = g * 32 + lane;
                double S;
                int nv;
                fitness_lane<DT, MODE, LG>(pd.V, spts, cnt, fp, i, S, nv);
                if (i < s.n_lvl) {  // partials stored [particle][chunk]: phase B' reads a particle's row
                    pd.part_S[(size_t)i * s.n_chunks + ch] = S;
                    pd.part_n[(size_t)i * s.n_chunks + ch] = nv;
                }
                u = u_next;
            }
        }
        if (!grid_barrier(P))
            return;
        // ---- phase B': per-particle totals, rho, per-CTA APS sums (Eq. ebs, Eq. wafit)
        for (int p = 0; p < B; ++p) {
            if (!st[p].active)
                continue;
            const ProblemDesc &pd = P.prob[p];
            const bool normalize = (pd.flags & RF_NORMALIZE) != 0;
            if (w == 0) {  // the centre particle's total, by the same code as every particle's below
                double S0;
                int n0;
                warp_particle_total(pd.part_S, pd.part_n, st[p].n_chunks, 0, lane, S0, n0);
                if (lane == 0) {
                    const float rho0 = fitness_rho(S0, st[p].nO, pd.tau, normalize);
                    const bool centre = k == 1 || (pd.flags & RF_RHO_REF_CENTER) || pd.n_levels > 1;
                    st[p].rho_ref = centre ? rho0 : st[p].rho_carry;
                }
            }
            __syncthreads();
            const float rho_ref = st[p].rho_ref;
            // particle 0 is the centre s*_{k-1} itself: an APS candidate only with RF_APS_WITH_CENTRE
            const int first = (pd.flags & RF_APS_WITH_CENTRE) ? 0 : 1;
            double sw = 0.0, swr = 0.0, swd[6] = {0, 0, 0, 0, 0, 0};
            int naps = 0, amax = -1;
            long long valid = 0;  // valid TSDF samples of all particles (first corner case of Sec. 4)
            float rmax = -1.f, r2 = -1.f;
            // one warp per particle: its lanes sum the chunk partials, lane 0 takes the particle
            for (int i = b * FIT_WARPS + w; i < st[p].n_lvl; i += G * FIT_WARPS) {
                double S;
                int nv;
                warp_particle_total(pd.part_S, pd.part_n, st[p].n_chunks, i, lane, S, nv);
                if (lane != 0)
                    continue;
                valid += nv;
                const float rho = fitness_rho(S, st[p].nO, pd.tau, normalize);
                merge_max(rmax, amax, r2, rho, i, -1.f);
                if (i >= first && rho > rho_ref) {
                    const double wgt = (double)(rho - rho_ref);
                    ++naps;
                    sw += wgt;
                    swr += wgt * (double)rho;
#pragma unroll
                    for (int d = 0; d < 6; ++d)
                        swd[d] += wgt * (double)(st[p].r[d] * __ldg(&pd.pst[(size_t)d * pd.n_tmpl + i]));
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                sw += __shfl_xor_sync(0xffffffffu, sw, o);
                swr += __shfl_xor_sync(0xffffffffu, swr, o);
#pragma unroll
                for (int d = 0; d < 6; ++d)
                    swd[d] += __shfl_xor_sync(0xffffffffu, swd[d], o);
                naps += __shfl_xor_sync(0xffffffffu, naps, o);
                valid += __shfl_xor_sync(0xffffffffu, valid, o);
                const float om = __shfl_xor_sync(0xffffffffu, rmax, o);
                const int oa = __shfl_xor_sync(0xffffffffu, amax, o);
                const float o2 = __shfl_xor_sync(0xffffffffu, r2, o);
                merge_max(rmax, amax, r2, om, oa, o2);
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
                red_v[w] = valid;
            }
            __syncthreads();
            if (tid == 0) {
                double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                int na = 0, am = -1;
                long long nv_all = 0;
                float rm = -1.f, rs = -1.f;
                for (int q = 0; q < FIT_WARPS; ++q) {
                    for (int e = 0; e < 8; ++e)
                        acc[e] += red_d[q][e];
                    na += red_i[q][0];
                    nv_all += red_v[q];
                    merge_max(rm, am, rs, red_f[q][0], red_i[q][1], red_f[q][1]);
                }
                double *out = P.aps + ((size_t)b * MAX_BATCH + p) * APW;
                for (int e = 0; e < 8; ++e)
                    out[e] = acc[e];
                out[8] = (double)na;
                out[9] = (double)rm;
                out[10] = (double)am;
                out[11] = (double)rs;
                out[12] = (double)nv_all;  // exact: far below 2^53
            }
            __syncthreads();
        }
        if (!grid_barrier(P))
            return;
        // ---- phase C: fixed-order reduction of the APS sums and the PST update
        for (int p = w; p < B; p += FIT_WARPS) {
            if (!st[p].active)
                continue;
            const ProblemDesc &pd = P.prob[p];
            PState &s = st[p];
            double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            double na = 0.0, nvalid = 0.0;
            float rm = -1.f, rs = -1.f;
            int am = -1;
            for (int q = lane; q < G; q += 32) {
                const double *in = P.aps + ((size_t)q * MAX_BATCH + p) * APW;
                for (int e = 0; e < 8; ++e)
                    acc[e] += __ldcg(&in[e]);
                na += __ldcg(&in[8]);
                nvalid += __ldcg(&in[12]);
                merge_max(rm, am, rs, (float)__ldcg(&in[9]), (int)__ldcg(&in[10]), (float)__ldcg(&in[11]));
            }
            for (int o = 16; o > 0; o >>= 1) {
                for (int e = 0; e < 8; ++e)
                    acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
                na += __shfl_xor_sync(0xffffffffu, na, o);
                nvalid += __shfl_xor_sync(0xffffffffu, nvalid, o);
                const float om = __shfl_xor_sync(0xffffffffu, rm, o);
                const int oa = __shfl_xor_sync(0xffffffffu, am, o);
                const float o2 = __shfl_xor_sync(0xffffffffu, rs, o);
                merge_max(rm, am, rs, om, oa, o2);
            }
            if (lane == 0) {
                // first corner case of Sec. 4: no particle found a single TSDF sample, so the
                // likelihood cannot be evaluated: rho = 0.5, v = 1, r_hat = 0.5 v + eps, s* kept
                const int corner = nvalid == 0.0 ? 1 : (na == 0.0 ? 2 : 0);
                const int n_aps = corner == 1 ? 0 : (int)na;
                const float rho_ref = s.rho_ref;
                float dbar[6], rhat[6];
                float rho_t;
                Pose s_new;
                if (corner == 1) {
                    rho_t = 0.5f;
                    for (int d = 0; d < 6; ++d) {
                        dbar[d] = 0.f;
                        rhat[d] = (float)(0.5 + (double)pd.eps);
                    }
                    s_new = s.c;
                    s.empty_run += 1;
                } else if (n_aps > 0) {
                    double nv2 = 0.0, db[6];
                    for (int d = 0; d < 6; ++d) {
                        db[d] = acc[2 + d] / acc[0];
                        nv2 += db[d] * db[d];
                    }
                    const double nv = sqrt(nv2);
                    rho_t = (float)(acc[1] / acc[0]);
                    for (int d = 0; d < 6; ++d) {
                        dbar[d] = (float)db[d];
                        const double dir = nv < 1e-12 ? 0.40824829046386302 : fabs(db[d]) / nv;
                        rhat[d] = (float)((1.0 - (double)rho_t) * dir + (double)pd.eps);
                    }
                    compose_offset(s.c, dbar, (pd.flags & RF_RIGHT_MULT) != 0, s_new);
                    s.empty_run = 0;
                } else {
                    rho_t = rho_ref;
                    for (int d = 0; d < 6; ++d) {
                        dbar[d] = 0.f;
                        rhat[d] = (float)(2.0 * (1.0 - (double)rho_ref) * 0.40824829046386302 + (double)pd.eps);
                    }
                    s_new = s.c;
                    s.empty_run += 1;
                }
                for (int d = 0; d < 6; ++d)
                    s.r[d] = pd.beta * s.r[d] + (1.f - pd.beta) * rhat[d];
                s.rho_carry = rho_t;
                s.c = s_new;
                if (k == 1)
                    for (int d = 0; d < 6; ++d)
                        s.r1[d] = s.r[d];
                float step = 0.f;
                for (int d = 0; d < 6; ++d)
                    step = fmaxf(step, fabsf(dbar[d]));
                int stop = 0;
                if (s.empty_run >= 2)
                    stop = 1;
                else if (n_aps > 0 && step < pd.stop_eps)
                    stop = 2;
                else if (k == pd.k_max)
                    stop = 3;
                s.stop = stop;
                s.lookups += (long long)s.nO * (long long)s.n_lvl;
                if (b == 0 && pd.stats) {
                    rf_iter_stats &row = pd.stats->it[k - 1];
                    row.k = k;
                    row.n_overlap = s.nO;
                    row.n_aps = n_aps;
                    row.argmax = am;
                    row.rho_ref = rho_ref;
                    row.rho_tilde = rho_t;
                    row.rho_max = rm;
                    row.rho_second = rs;
                    for (int a = 0; a < 4; ++a)
                        row.pose[a] = s.c.q[a];
                    for (int a = 0; a < 3; ++a)
                        row.pose[4 + a] = s.c.t[a];
                    for (int d = 0; d < 6; ++d) {
                        row.scale[d] = s.r[d];
                        row.offset[d] = dbar[d];
                    }
                    row.stop = stop;
                    row.level = s.level;
                    row.n_particles = s.n_lvl;
                    row.corner = corner;
                }
            }
        }
        __syncthreads();
    }
    // ---- epilogue (CTA 0): final poses, r_1 for the next frame, summaries
    if (b == 0 && tid < B && st[tid].stop != 5) {
        const ProblemDesc &pd = P.prob[tid];
        const PState &s = st[tid];
        for (int a = 0; a < 4; ++a)
            pd.out_pose[a] = s.c.q[a];
        for (int a = 0; a < 3; ++a)
            pd.out_pose[4 + a] = s.c.t[a];
        for (int d = 0; d < 6; ++d)
            pd.scale[d] = s.r1[d];
        if (pd.stats) {
            pd.stats->iters = s.iters;
            pd.stats->status = *((volatile int *)pd.status);
            pd.stats->n_points = pd.lvl_m[0];
            pd.stats->lookups = s.lookups;
            for (int d = 0; d < 6; ++d)
                pd.stats->r1[d] = s.r1[d];
        }
    }
}

// ------------------------------------------------------------------ kernel table
// The trilinear modes are built for groups of 4, 6 and 8 lookups in flight (the
// group regroups the FP32 partial sums, so results differ in rounding only);
// nearest-voxel modes sample one point at a time and have one variant.  Each
// storage type's variants live in their own translation unit.
using PfoFn = void (*)(BatchParams);
constexpr int GROUP_CHOICES[3] = {4, 6, 8};
template <int DT, int MODE> PfoFn pfo_fn_group(int group)
{
    if constexpr ((MODE & 1) != 0) {
        return pfo_batch_kernel<DT, MODE, GROUP>;
    } else {
        switch (group) {
        case 4:
            return pfo_batch_kernel<DT, MODE, 4>;
        case 8:
            return pfo_batch_kernel<DT, MODE, 8>;
        default:
            return pfo_batch_kernel<DT, MODE, GROUP>;
        }
    }
}
template <int DT> PfoFn pfo_fn_dtype(int mode, int group)
{
    switch (mode) {
    case 0:
        return pfo_fn_group<DT, 0>(group);
    case 1:
        return pfo_fn_group<DT, 1>(group);
    case 2:
        return pfo_fn_group<DT, 2>(group);
    default:
        return pfo_fn_group<DT, 3>(group);
    }
}
PfoFn pfo_fn_f32(int mode, int group);
PfoFn pfo_fn_f16(int mode, int group);
PfoFn pfo_fn_i16(int mode, int group);

}  // namespace rf
