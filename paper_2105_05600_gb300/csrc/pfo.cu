// pfo.cu -- Algorithm 1 (PFO with PST) for one frame of one or several
// sequences in ONE persistent cooperative kernel.
//
// Per iteration k, for every active sequence p (its level l = (k-1) mod L_p of the
// multi-resolution schedule, Sec. 4):
//   A   overlap set O_k with s*_{k-1} (Eq. validness), counted per CTA
//   A'  order-preserving compaction of O_k
//   B   fitness of the level's particles (Eq. normallh): (sequence, particle
//       group, point chunk) work units handed out through an atomic counter
//   B'  per-particle totals, rho, per-CTA APS sums (Eq. ebs, Eq. wafit)
//   C   every CTA reduces the APS sums in the same fixed order and applies the
//       best-state / axis-length update and the stop rules (Eq. rsdir, rsinter,
//       momentum; Sec. 4) redundantly, so the decision is identical everywhere
// separated by a grid barrier whose waits are bounded in time.  The paper streams
// the fitness values to the host every iteration (Sec. 4, GPU implementation);
// here nothing leaves the device inside a frame.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

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
__device__ bool grid_barrier(const BatchParams &P)
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
template <int DT, int MODE>
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
                fitness_lane<DT, MODE>(pd.V, spts, cnt, fp, i, S, nv);
                if (i < s.n_lvl) {
                    pd.part_S[(size_t)ch * s.n_lvl + i] = S;
                    pd.part_n[(size_t)ch * s.n_lvl + i] = nv;
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
            if (tid == 0) {
                double S0;
                int n0;
                particle_total(pd.part_S, pd.part_n, st[p].n_lvl, st[p].n_chunks, 0, true, S0, n0);
                const float rho0 = fitness_rho(S0, st[p].nO, pd.tau, normalize);
                const bool centre = k == 1 || (pd.flags & RF_RHO_REF_CENTER) || pd.n_levels > 1;
                st[p].rho_ref = centre ? rho0 : st[p].rho_carry;
            }
            __syncthreads();
            const float rho_ref = st[p].rho_ref;
            // particle 0 is the centre s*_{k-1} itself: an APS candidate only with RF_APS_WITH_CENTRE
            const int first = (pd.flags & RF_APS_WITH_CENTRE) ? 0 : 1;
            double sw = 0.0, swr = 0.0, swd[6] = {0, 0, 0, 0, 0, 0};
            int naps = 0, amax = -1;
            long long valid = 0;  // valid TSDF samples of all particles (first corner case of Sec. 4)
            float rmax = -1.f, r2 = -1.f;
            for (int i = b * blockDim.x + tid; i < st[p].n_lvl; i += G * blockDim.x) {
                double S;
                int nv;
                particle_total(pd.part_S, pd.part_n, st[p].n_lvl, st[p].n_chunks, i, true, S, nv);
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

__global__ void set_int_kernel(int *dst, int v) { *dst = v; }

__global__ void set_pose_kernel(float *dst, Pose p)
{
    for (int a = 0; a < 4; ++a)
        dst[a] = p.q[a];
    for (int a = 0; a < 3; ++a)
        dst[4 + a] = p.t[a];
}

// ------------------------------------------------------------------ kernel table
using PfoFn = void (*)(BatchParams);
template <int DT> static PfoFn pfo_fn(int mode)
{
    switch (mode) {
    case 0:
        return pfo_batch_kernel<DT, 0>;
    case 1:
        return pfo_batch_kernel<DT, 1>;
    case 2:
        return pfo_batch_kernel<DT, 2>;
    default:
        return pfo_batch_kernel<DT, 3>;
    }
}
static PfoFn pfo_fn(int dtype, int mode)
{
    return dtype == RF_F32 ? pfo_fn<RF_F32>(mode) : dtype == RF_F16 ? pfo_fn<RF_F16>(mode) : pfo_fn<RF_I16>(mode);
}
static int mode_of(int flags) { return ((flags & RF_NEAREST) ? 1 : 0) | ((flags & RF_COMPENSATED) ? 0 : 2); }
static size_t pfo_smem() { return (size_t)FIT_WARPS * CHUNK_MAX * sizeof(float4); }

// Largest cooperative grid of the kernel variant (CTAs per SM x SMs).
static rf_status max_ctas_per_sm(int dtype, int mode, int *per_sm)
{
    PfoFn fn = pfo_fn(dtype, mode);
    RF_CUDA(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pfo_smem()));
    *per_sm = 0;
    RF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, (const void *)fn, FIT_THREADS, pfo_smem()));
    if (*per_sm < 1) {
        set_error("the PFO kernel cannot be resident on this device");
        return RF_ERR_CUDA;
    }
    return RF_OK;
}

static rf_status check_params(const rf_params *p)
{
    RF_CHECK_ARG(p != nullptr, "null params");
    RF_CHECK_ARG(p->k_max >= 1 && p->k_max <= RF_MAX_ITERS, "k_max out of range");
    RF_CHECK_ARG(p->stride >= 1, "stride must be >= 1");
    RF_CHECK_ARG(p->tau > 0.f, "tau must be positive");
    RF_CHECK_ARG(p->beta >= 0.f && p->beta <= 1.f, "beta must lie in [0, 1]");
    return RF_OK;
}

// Scratch shared by the CTAs of one launch (per tracker or per batch).
struct LaunchScratch {
    GridSync *gs = nullptr;
    int *unit_ctr = nullptr;
    int *block_counts = nullptr;
    double *aps = nullptr;
    rf_status alloc()
    {
        const size_t max_grid = (size_t)MAX_CTAS_PER_SM * sm_count();
        cudaError_t e = cudaMalloc(&gs, sizeof(GridSync));
        if (e == cudaSuccess)
            e = cudaMalloc(&unit_ctr, sizeof(int) * RF_MAX_ITERS);
        if (e == cudaSuccess)
            e = cudaMalloc(&block_counts, sizeof(int) * MAX_BATCH * max_grid);
        if (e == cudaSuccess)
            e = cudaMalloc(&aps, sizeof(double) * APW * MAX_BATCH * max_grid);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(launch scratch)");
        return RF_OK;
    }
    void release()
    {
        cudaFree(gs);
        cudaFree(unit_ctr);
        cudaFree(block_counts);
        cudaFree(aps);
        gs = nullptr;
        unit_ctr = block_counts = nullptr;
        aps = nullptr;
    }
};

}  // namespace rf

using namespace rf;

// ------------------------------------------------------------------ tracker handle
struct rf_tracker_s {
    rf_volume vol;
    const float *pst;
    int n;  // template size
    rf_params p;
    int n_levels;
    int lvl_n[MAX_LEVELS], lvl_stride[MAX_LEVELS];
    int max_w, max_h;
    int m_cap;       // points the buffers hold (all levels at max_w x max_h)
    int max_chunks;  // per level, for WORK_WARPS_MAX
    // device scratch
    float4 *pts, *cpts;
    double *part_S;
    int *part_n;
    int *status;
    float *scale;
    float *pose_ring;   // 2 x 7
    float *depth_ring;  // 2 x max_w * max_h
    int cur;            // ring slot of the previous frame (sequence mode)
    LaunchScratch ls;
    int debug_skip;
    long long timeout_ns;
};

static void level_geometry(const rf_tracker tr, int W, int H, int nw[MAX_LEVELS], int m[MAX_LEVELS],
                           int off[MAX_LEVELS], int *m_all)
{
    int o = 0;
    for (int l = 0; l < tr->n_levels; ++l) {
        const int s = tr->lvl_stride[l];
        nw[l] = (W + s - 1) / s;
        m[l] = nw[l] * ((H + s - 1) / s);
        off[l] = o;
        o += m[l];
    }
    *m_all = o;
}

// (Re)allocate the point and partial-sum buffers for the current schedule.
static rf_status alloc_schedule_buffers(rf_tracker tr)
{
    int nw[MAX_LEVELS], m[MAX_LEVELS], off[MAX_LEVELS], m_all;
    level_geometry(tr, tr->max_w, tr->max_h, nw, m, off, &m_all);
    int max_chunks = 1;
    size_t part = 0;
    for (int l = 0; l < tr->n_levels; ++l) {
        const int c = max_chunks_for(tr->lvl_n[l], m[l], WORK_WARPS_MAX);
        max_chunks = std::max(max_chunks, c);
        part = std::max(part, (size_t)c * tr->lvl_n[l]);
    }
    cudaFree(tr->pts);
    cudaFree(tr->cpts);
    cudaFree(tr->part_S);
    cudaFree(tr->part_n);
    tr->pts = tr->cpts = nullptr;
    tr->part_S = nullptr;
    tr->part_n = nullptr;
    cudaError_t e = cudaMalloc(&tr->pts, sizeof(float4) * (size_t)m_all);
    if (e == cudaSuccess)
        e = cudaMalloc(&tr->cpts, sizeof(float4) * (size_t)m_all);
    if (e == cudaSuccess)
        e = cudaMalloc(&tr->part_S, sizeof(double) * part);
    if (e == cudaSuccess)
        e = cudaMalloc(&tr->part_n, sizeof(int) * part);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(tracker buffers)");
    tr->m_cap = m_all;
    tr->max_chunks = max_chunks;
    return RF_OK;
}

// The launch descriptor of one tracker for one frame.
static rf_status fill_problem(rf_tracker tr, const float *depth, const float *prev_depth, const rf_intrinsics *K,
                              const float *prev_pose, float *out_pose, rf_frame_stats *stats, ProblemDesc &pd)
{
    RF_CHECK_ARG(K->width > 0 && K->height > 0 && K->width <= tr->max_w && K->height <= tr->max_h,
                 "frame larger than the tracker was created for");
    memset(&pd, 0, sizeof pd);
    pd.V = tr->vol->d;
    pd.K = to_intr(*K);
    pd.depth = depth;
    pd.prev_depth = prev_depth;
    pd.pst = tr->pst;
    pd.n_tmpl = tr->n;
    pd.n_levels = tr->n_levels;
    for (int l = 0; l < tr->n_levels; ++l) {
        pd.lvl_n[l] = tr->lvl_n[l];
        pd.lvl_stride[l] = tr->lvl_stride[l];
    }
    level_geometry(tr, K->width, K->height, pd.lvl_nw, pd.lvl_m, pd.lvl_off, &pd.m_all);
    pd.prev_pose = prev_pose;
    pd.out_pose = out_pose;
    pd.stats = stats;
    pd.scale = tr->scale;
    pd.pts = tr->pts;
    pd.cpts = tr->cpts;
    pd.part_S = tr->part_S;
    pd.part_n = tr->part_n;
    pd.max_chunks = tr->max_chunks;
    pd.status = tr->status;
    pd.tau = tr->p.tau;
    pd.beta = tr->p.beta;
    pd.eps = tr->p.eps;
    pd.stop_eps = tr->p.stop_eps;
    pd.k_max = tr->p.k_max;
    pd.flags = tr->p.flags;
    return RF_OK;
}

// Enqueue one persistent launch for B prepared problems: resets of the barrier,
// counters, statuses and stats, then the cooperative kernel.  Capturable.
static rf_status launch_batch(BatchParams &P, const LaunchScratch &ls, int dtype, int mode, int ctas_per_sm,
                              int debug_skip, cudaStream_t s)
{
    int per_sm = 0;
    rf_status st = max_ctas_per_sm(dtype, mode, &per_sm);
    if (st != RF_OK)
        return st;
    const int use = ctas_per_sm > 0 ? std::min(per_sm, ctas_per_sm) : per_sm;
    const int grid = std::min(use, MAX_CTAS_PER_SM) * sm_count();
    P.gs = ls.gs;
    P.unit_ctr = ls.unit_ctr;
    P.block_counts = ls.block_counts;
    P.aps = ls.aps;
    P.k_max_all = 0;
    for (int p = 0; p < P.B; ++p) {
        P.k_max_all = std::max(P.k_max_all, P.prob[p].k_max);
        RF_CUDA(cudaMemsetAsync(P.prob[p].status, 0, sizeof(int), s));
        if (P.prob[p].stats)
            RF_CUDA(cudaMemsetAsync(P.prob[p].stats, 0, sizeof(rf_frame_stats), s));
    }
    RF_CUDA(cudaMemsetAsync(ls.gs, 0, sizeof(GridSync), s));
    RF_CUDA(cudaMemsetAsync(ls.unit_ctr, 0, sizeof(int) * RF_MAX_ITERS, s));
    if (debug_skip) {
        set_int_kernel<<<1, 1, 0, s>>>(&ls.gs->skip, 1);
        RF_CUDA(cudaGetLastError());
    }
    void *args[] = {&P};
    RF_CUDA(cudaLaunchCooperativeKernel((const void *)pfo_fn(dtype, mode), dim3(grid), dim3(FIT_THREADS), args,
                                       pfo_smem(), s));
    return RF_OK;
}

extern "C" {

void rf_tracker_destroy(rf_tracker tr)
{
    if (!tr)
        return;
    cudaFree(tr->pts);
    cudaFree(tr->cpts);
    cudaFree(tr->part_S);
    cudaFree(tr->part_n);
    cudaFree(tr->status);
    cudaFree(tr->scale);
    cudaFree(tr->pose_ring);
    cudaFree(tr->depth_ring);
    tr->ls.release();
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
    tr->n_levels = 1;
    tr->lvl_n[0] = n;
    tr->lvl_stride[0] = p->stride;
    rf_status st = alloc_schedule_buffers(tr);
    if (st == RF_OK)
        st = tr->ls.alloc();
    cudaError_t e = cudaSuccess;
    if (st == RF_OK) {
        e = cudaMalloc(&tr->status, sizeof(int));
        if (e == cudaSuccess)
            e = cudaMalloc(&tr->scale, sizeof(float) * 6);
        if (e == cudaSuccess)
            e = cudaMalloc(&tr->pose_ring, sizeof(float) * 14);
        if (e == cudaSuccess)
            e = cudaMalloc(&tr->depth_ring, sizeof(float) * 2 * (size_t)max_width * max_height);
        const float ones[6] = {1, 1, 1, 1, 1, 1};
        if (e == cudaSuccess)
            e = cudaMemcpy(tr->scale, ones, sizeof ones, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemset(tr->status, 0, sizeof(int));
        if (e != cudaSuccess)
            st = cuda_fail(e, "rf_tracker_create");
    }
    if (st != RF_OK) {
        rf_tracker_destroy(tr);
        return st;
    }
    *out = tr;
    return RF_OK;
}

rf_status rf_tracker_set_schedule(rf_tracker tr, int n_levels, const int *n, const int *stride)
{
    RF_CHECK_ARG(tr && n && stride, "null pointer");
    RF_CHECK_ARG(n_levels >= 1 && n_levels <= MAX_LEVELS, "n_levels out of range");
    for (int l = 0; l < n_levels; ++l) {
        RF_CHECK_ARG(n[l] >= 1 && n[l] <= tr->n, "level particle count out of range");
        RF_CHECK_ARG(stride[l] >= 1, "level stride must be >= 1");
    }
    RF_CUDA(cudaDeviceSynchronize());
    tr->n_levels = n_levels;
    for (int l = 0; l < n_levels; ++l) {
        tr->lvl_n[l] = n[l];
        tr->lvl_stride[l] = stride[l];
    }
    return alloc_schedule_buffers(tr);
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
    const bool stride_changed = tr->n_levels == 1 && p->stride != tr->lvl_stride[0];
    tr->p = *p;
    if (stride_changed) {
        RF_CUDA(cudaDeviceSynchronize());
        tr->lvl_stride[0] = p->stride;
        return alloc_schedule_buffers(tr);
    }
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
    cudaStream_t s = (cudaStream_t)stream;
    BatchParams P;
    memset(&P, 0, sizeof P);
    rf_status st = fill_problem(tr, depth_dev, prev_depth_dev, K, prev_pose_dev, out_pose_dev, stats_dev, P.prob[0]);
    if (st != RF_OK)
        return st;
    P.B = 1;
    P.work_warps = WORK_WARPS_DEFAULT;
    P.timeout_ns = tr->timeout_ns;
    st = launch_batch(P, tr->ls, tr->vol->d.dtype, mode_of(tr->p.flags), 0, tr->debug_skip, s);
    if (st != RF_OK)
        return st;
    if (tr->debug_skip) {
        RF_CUDA(cudaStreamSynchronize(s));
        tr->debug_skip = 0;
        tr->timeout_ns = 1000000000ll;
    }
    return RF_OK;
}

rf_status pfo_track_frame_ex_async(rf_tracker tr, const float *depth_dev, const float *prev_depth_dev,
                                   const rf_intrinsics *K, const float *prev_pose_dev, float *out_pose_dev,
                                   rf_frame_stats *stats_dev, const rf_track_options *opt, void *stream)
{
    RF_CHECK_ARG(tr && depth_dev && prev_depth_dev && K && prev_pose_dev && out_pose_dev && opt, "null pointer");
    RF_CHECK_ARG(opt->k_max >= 0 && opt->k_max <= RF_MAX_ITERS, "k_max outside [0, RF_MAX_ITERS]");
    cudaStream_t s = (cudaStream_t)stream;
    BatchParams P;
    memset(&P, 0, sizeof P);
    rf_status st = fill_problem(tr, depth_dev, prev_depth_dev, K, prev_pose_dev, out_pose_dev, stats_dev, P.prob[0]);
    if (st != RF_OK)
        return st;
    ProblemDesc &pd = P.prob[0];
    pd.init_pose = opt->init_pose_dev;
    pd.run_flag = opt->run_flag_dev;
    if (opt->scale_dev)
        pd.scale = opt->scale_dev;
    if (opt->k_max > 0)
        pd.k_max = opt->k_max;
    P.B = 1;
    P.work_warps = WORK_WARPS_DEFAULT;
    P.timeout_ns = tr->timeout_ns;
    return launch_batch(P, tr->ls, tr->vol->d.dtype, mode_of(tr->p.flags), 0, 0, s);
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
    const size_t slot = (size_t)tr->max_w * tr->max_h;
    const int prev = tr->cur, nxt = 1 - tr->cur;
    float *dprev = tr->depth_ring + (size_t)prev * slot, *dnext = tr->depth_ring + (size_t)nxt * slot;
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

// ------------------------------------------------------------------ batch handle
struct rf_batch_s {
    int n;
    rf_tracker tr[MAX_BATCH];
    rf_intrinsics K[MAX_BATCH];
    int dtype, mode;
    LaunchScratch ls;
    rf_frame_stats *stats;  // device [n]
    rf_launch_config cfg;
    cudaStream_t capture_stream;
    cudaGraphExec_t graph[2];
    rf_launch_config graph_cfg[2];
};

static rf_status batch_params(rf_batch b, int parity, BatchParams &P)
{
    memset(&P, 0, sizeof P);
    P.B = b->n;
    P.work_warps = b->cfg.work_warps;
    P.timeout_ns = 1000000000ll;
    for (int i = 0; i < b->n; ++i) {
        rf_tracker tr = b->tr[i];
        const size_t slot = (size_t)tr->max_w * tr->max_h;
        const float *cur = tr->depth_ring + (size_t)parity * slot, *prv = tr->depth_ring + (size_t)(1 - parity) * slot;
        rf_status st = fill_problem(tr, cur, prv, &b->K[i], tr->pose_ring + 7 * (1 - parity),
                                    tr->pose_ring + 7 * parity, b->stats + i, P.prob[i]);
        if (st != RF_OK)
            return st;
    }
    return RF_OK;
}

// One batch step: the persistent PFO launch, then fusion of every tracked frame.
static rf_status batch_enqueue(rf_batch b, int parity, cudaStream_t s)
{
    BatchParams P;
    rf_status st = batch_params(b, parity, P);
    if (st != RF_OK)
        return st;
    st = launch_batch(P, b->ls, b->dtype, b->mode, b->cfg.ctas_per_sm, 0, s);
    if (st != RF_OK)
        return st;
    for (int i = 0; i < b->n; ++i) {
        rf_tracker tr = b->tr[i];
        st = launch_integrate_dev(tr->vol->d, P.prob[i].depth, to_intr(b->K[i]), P.prob[i].out_pose, tr->status, s);
        if (st != RF_OK)
            return st;
    }
    return RF_OK;
}

extern "C" {

void rf_batch_destroy(rf_batch b)
{
    if (!b)
        return;
    for (int p = 0; p < 2; ++p)
        if (b->graph[p])
            cudaGraphExecDestroy(b->graph[p]);
    if (b->capture_stream)
        cudaStreamDestroy(b->capture_stream);
    cudaFree(b->stats);
    b->ls.release();
    delete b;
}

rf_status rf_batch_create(const rf_tracker *trackers, int n, const rf_intrinsics *K, rf_batch *out)
{
    RF_CHECK_ARG(out != nullptr, "null output");
    *out = nullptr;
    RF_CHECK_ARG(trackers && K, "null pointer");
    RF_CHECK_ARG(n >= 1 && n <= MAX_BATCH, "n must be in [1, RF_MAX_BATCH]");
    for (int i = 0; i < n; ++i) {
        RF_CHECK_ARG(trackers[i] != nullptr, "null tracker");
        RF_CHECK_ARG(trackers[i]->vol->d.dtype == trackers[0]->vol->d.dtype, "trackers must share the volume dtype");
        RF_CHECK_ARG(mode_of(trackers[i]->p.flags) == mode_of(trackers[0]->p.flags),
                     "trackers must share the RF_NEAREST and RF_COMPENSATED flags");
        RF_CHECK_ARG(K[i].width > 0 && K[i].height > 0 && K[i].width <= trackers[i]->max_w &&
                         K[i].height <= trackers[i]->max_h,
                     "frame size exceeds a tracker's maximum");
        for (int j = 0; j < i; ++j)
            RF_CHECK_ARG(trackers[j] != trackers[i], "a tracker appears twice");
    }
    rf_batch b = new rf_batch_s();
    memset(b, 0, sizeof *b);
    b->n = n;
    for (int i = 0; i < n; ++i) {
        b->tr[i] = trackers[i];
        b->K[i] = K[i];
    }
    b->dtype = trackers[0]->vol->d.dtype;
    b->mode = mode_of(trackers[0]->p.flags);
    b->cfg.ctas_per_sm = 0;  // as many as fit
    b->cfg.work_warps = WORK_WARPS_DEFAULT;
    rf_status st = b->ls.alloc();
    cudaError_t e = cudaSuccess;
    if (st == RF_OK) {
        e = cudaMalloc(&b->stats, sizeof(rf_frame_stats) * n);
        if (e == cudaSuccess)
            e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess)
            st = cuda_fail(e, "rf_batch_create");
    }
    if (st != RF_OK) {
        rf_batch_destroy(b);
        return st;
    }
    *out = b;
    return RF_OK;
}

rf_status rf_batch_depth_slot(rf_batch b, int i, int parity, float **depth_dev)
{
    RF_CHECK_ARG(b && depth_dev, "null pointer");
    RF_CHECK_ARG(i >= 0 && i < b->n && (parity == 0 || parity == 1), "index out of range");
    rf_tracker tr = b->tr[i];
    *depth_dev = tr->depth_ring + (size_t)parity * tr->max_w * tr->max_h;
    return RF_OK;
}

rf_status rf_batch_pose_dev(rf_batch b, int i, int parity, float **pose_dev)
{
    RF_CHECK_ARG(b && pose_dev, "null pointer");
    RF_CHECK_ARG(i >= 0 && i < b->n && (parity == 0 || parity == 1), "index out of range");
    *pose_dev = b->tr[i]->pose_ring + 7 * parity;
    return RF_OK;
}

rf_status rf_batch_stats_dev(rf_batch b, rf_frame_stats **stats_dev)
{
    RF_CHECK_ARG(b && stats_dev, "null pointer");
    *stats_dev = b->stats;
    return RF_OK;
}

rf_status rf_batch_start(rf_batch b, const rf_pose *poses_host, void *stream)
{
    RF_CHECK_ARG(b && poses_host, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < b->n; ++i) {
        rf_tracker tr = b->tr[i];
        set_pose_kernel<<<1, 1, 0, s>>>(tr->pose_ring, to_pose(poses_host[i]));
        RF_CUDA(cudaGetLastError());
        RF_CUDA(cudaMemsetAsync(tr->status, 0, sizeof(int), s));
        rf_status st = launch_integrate_dev(tr->vol->d, tr->depth_ring, to_intr(b->K[i]), tr->pose_ring, nullptr, s);
        if (st != RF_OK)
            return st;
    }
    return RF_OK;
}

rf_status rf_batch_set_config(rf_batch b, const rf_launch_config *cfg)
{
    RF_CHECK_ARG(b && cfg, "null pointer");
    RF_CHECK_ARG(cfg->ctas_per_sm >= 0 && cfg->ctas_per_sm <= MAX_CTAS_PER_SM, "ctas_per_sm out of range");
    RF_CHECK_ARG(cfg->work_warps >= 1 && cfg->work_warps <= WORK_WARPS_MAX, "work_warps out of range");
    b->cfg = *cfg;
    return RF_OK;
}

rf_status rf_batch_step(rf_batch b, int parity, int use_graph, void *stream)
{
    RF_CHECK_ARG(b != nullptr, "null batch");
    RF_CHECK_ARG(parity == 0 || parity == 1, "parity must be 0 or 1");
    cudaStream_t s = (cudaStream_t)stream;
    if (!use_graph)
        return batch_enqueue(b, parity, s);
    const bool stale = b->graph[parity] && (b->graph_cfg[parity].ctas_per_sm != b->cfg.ctas_per_sm ||
                                            b->graph_cfg[parity].work_warps != b->cfg.work_warps);
    if (stale) {
        cudaGraphExecDestroy(b->graph[parity]);
        b->graph[parity] = nullptr;
    }
    if (!b->graph[parity]) {
        // capture on the internal stream (the caller's may be the legacy stream)
        cudaStream_t cs = b->capture_stream;
        RF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        rf_status st = batch_enqueue(b, parity, cs);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (st != RF_OK) {
            if (g)
                cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaStreamEndCapture(batch step)");
        e = cudaGraphInstantiate(&b->graph[parity], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaGraphInstantiate(batch step)");
        b->graph_cfg[parity] = b->cfg;
    }
    RF_CUDA(cudaGraphLaunch(b->graph[parity], s));
    return RF_OK;
}

rf_status rf_batch_autotune(rf_batch b, int parity, rf_launch_config *chosen, void *stream)
{
    RF_CHECK_ARG(b != nullptr, "null batch");
    RF_CHECK_ARG(parity == 0 || parity == 1, "parity must be 0 or 1");
    cudaStream_t s = (cudaStream_t)stream;
    int per_sm = 0;
    rf_status st = max_ctas_per_sm(b->dtype, b->mode, &per_sm);
    if (st != RF_OK)
        return st;
    // the PFO launch rewrites each tracker's r_0 and output pose: keep and restore them
    std::vector<float> saved_scale(6 * b->n), saved_pose(7 * b->n);
    for (int i = 0; i < b->n; ++i) {
        RF_CUDA(cudaMemcpyAsync(&saved_scale[6 * i], b->tr[i]->scale, 6 * sizeof(float), cudaMemcpyDeviceToHost, s));
        RF_CUDA(cudaMemcpyAsync(&saved_pose[7 * i], b->tr[i]->pose_ring + 7 * parity, 7 * sizeof(float),
                                cudaMemcpyDeviceToHost, s));
    }
    RF_CUDA(cudaStreamSynchronize(s));
    cudaEvent_t e0, e1;
    RF_CUDA(cudaEventCreate(&e0));
    RF_CUDA(cudaEventCreate(&e1));
    rf_launch_config best = b->cfg;
    best.ms = 1e30f;
    const int warps_opts[3] = {WORK_WARPS_DEFAULT / 2, WORK_WARPS_DEFAULT, WORK_WARPS_MAX};
    for (int c = 1; c <= std::min(per_sm, MAX_CTAS_PER_SM); ++c) {
        for (int wi = 0; wi < 3; ++wi) {
            rf_launch_config cand;
            cand.ctas_per_sm = c;
            cand.work_warps = warps_opts[wi];
            float best_t = 1e30f;
            for (int rep = 0; rep < 2; ++rep) {  // first run warms the caches
                for (int i = 0; i < b->n; ++i)
                    RF_CUDA(cudaMemcpyAsync(b->tr[i]->scale, &saved_scale[6 * i], 6 * sizeof(float),
                                            cudaMemcpyHostToDevice, s));
                BatchParams P;
                st = batch_params(b, parity, P);
                if (st != RF_OK)
                    break;
                P.work_warps = cand.work_warps;
                RF_CUDA(cudaEventRecord(e0, s));
                st = launch_batch(P, b->ls, b->dtype, b->mode, cand.ctas_per_sm, 0, s);
                if (st != RF_OK)
                    break;
                RF_CUDA(cudaEventRecord(e1, s));
                RF_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                RF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                best_t = std::min(best_t, ms);
            }
            if (st != RF_OK)
                break;
            if (best_t < best.ms) {
                best = cand;
                best.ms = best_t;
            }
        }
        if (st != RF_OK)
            break;
    }
    for (int i = 0; i < b->n; ++i) {
        cudaMemcpyAsync(b->tr[i]->scale, &saved_scale[6 * i], 6 * sizeof(float), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(b->tr[i]->pose_ring + 7 * parity, &saved_pose[7 * i], 7 * sizeof(float),
                        cudaMemcpyHostToDevice, s);
    }
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != RF_OK)
        return st;
    b->cfg = best;
    if (chosen)
        *chosen = best;
    return RF_OK;
}

}  // extern "C"
