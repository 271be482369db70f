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

#include "pfo_kernel.cuh"

namespace rf {

static PfoFn pfo_fn(int dtype, int mode, int group)
{
    return dtype == RF_F32 ? pfo_fn_f32(mode, group) : dtype == RF_F16 ? pfo_fn_f16(mode, group) : pfo_fn_i16(mode, group);
}

__global__ void set_int_kernel(int *dst, int v) { *dst = v; }

__global__ void set_pose_kernel(float *dst, Pose p)
{
    for (int a = 0; a < 4; ++a)
        dst[a] = p.q[a];
    for (int a = 0; a < 3; ++a)
        dst[4 + a] = p.t[a];
}

static int mode_of(int flags) { return ((flags & RF_NEAREST) ? 1 : 0) | ((flags & RF_COMPENSATED) ? 0 : 2); }
static size_t pfo_smem() { return (size_t)FIT_WARPS * CHUNK_MAX * sizeof(float4); }

// Largest cooperative grid of the kernel variant (CTAs per SM x SMs).
static rf_status max_ctas_per_sm(int dtype, int mode, int group, int *per_sm)
{
    PfoFn fn = pfo_fn(dtype, mode, group);
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
    rf_launch_config cfg;  // launch of this tracker's own frames
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
                              int group, int debug_skip, cudaStream_t s)
{
    int per_sm = 0;
    rf_status st = max_ctas_per_sm(dtype, mode, group, &per_sm);
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
    RF_CUDA(cudaLaunchCooperativeKernel((const void *)pfo_fn(dtype, mode, group), dim3(grid), dim3(FIT_THREADS), args,
                                       pfo_smem(), s));
    return RF_OK;
}

// Validated copy of a launch configuration (group 0 means the default).
static rf_status normalise_config(const rf_launch_config *cfg, rf_launch_config *out)
{
    RF_CHECK_ARG(cfg->ctas_per_sm >= 0 && cfg->ctas_per_sm <= MAX_CTAS_PER_SM, "ctas_per_sm out of range");
    RF_CHECK_ARG(cfg->work_warps >= 1 && cfg->work_warps <= WORK_WARPS_MAX, "work_warps out of range");
    RF_CHECK_ARG(cfg->group == 0 || cfg->group == 4 || cfg->group == 6 || cfg->group == 8,
                 "group must be 0, 4, 6 or 8");
    *out = *cfg;
    if (out->group == 0)
        out->group = GROUP;
    return RF_OK;
}

// Kernel time of one candidate: the faster of two runs (the first warms the caches),
// the launch's mutable inputs restored before each.
template <class Run, class Restore>
static rf_status time_candidate(const rf_launch_config &cand, Run &run, Restore &restore, cudaStream_t s,
                                cudaEvent_t e0, cudaEvent_t e1, float *ms_out)
{
    float best_t = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
        rf_status st = restore();
        if (st != RF_OK)
            return st;
        RF_CUDA(cudaEventRecord(e0, s));
        st = run(cand);
        if (st != RF_OK)
            return st;
        RF_CUDA(cudaEventRecord(e1, s));
        RF_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        RF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        best_t = std::min(best_t, ms);
    }
    *ms_out = best_t;
    return RF_OK;
}

// The candidate search shared by the tracker and batch autotuners: CTAs per SM x
// work warps {1824, 3648, 7296} with the default group of 6, then groups of 4 and
// 8 at the best work split (with the best CTAs per SM where that group fits it,
// and at its own maximum).
template <class Run, class Restore>
static rf_status autotune_search(int dtype, int mode, Run &run, Restore &restore, cudaStream_t s,
                                 rf_launch_config *best_out)
{
    cudaEvent_t e0, e1;
    RF_CUDA(cudaEventCreate(&e0));
    RF_CUDA(cudaEventCreate(&e1));
    rf_launch_config best;
    best.ctas_per_sm = 0;
    best.work_warps = WORK_WARPS_DEFAULT;
    best.group = GROUP;
    best.ms = 1e30f;
    rf_status st = RF_OK;
    auto consider = [&](const rf_launch_config &cand) -> rf_status {
        float ms = 0.f;
        rf_status r = time_candidate(cand, run, restore, s, e0, e1, &ms);
        if (r == RF_OK && ms < best.ms) {
            best = cand;
            best.ms = ms;
        }
        return r;
    };
    int per_sm = 0;
    st = max_ctas_per_sm(dtype, mode, GROUP, &per_sm);
    const int warps_opts[3] = {WORK_WARPS_DEFAULT / 2, WORK_WARPS_DEFAULT, WORK_WARPS_MAX};
    for (int c = 1; st == RF_OK && c <= std::min(per_sm, MAX_CTAS_PER_SM); ++c)
        for (int wi = 0; st == RF_OK && wi < 3; ++wi) {
            rf_launch_config cand;
            cand.ctas_per_sm = c;
            cand.work_warps = warps_opts[wi];
            cand.group = GROUP;
            cand.ms = 0.f;
            st = consider(cand);
        }
    if ((mode & 1) == 0) {  // trilinear: the other lookup groups
        const rf_launch_config base = best;
        for (int gi = 0; st == RF_OK && gi < 3; ++gi) {
            const int g = GROUP_CHOICES[gi];
            if (g == GROUP)
                continue;
            int g_per_sm = 0;
            st = max_ctas_per_sm(dtype, mode, g, &g_per_sm);
            const int top = std::min(g_per_sm, MAX_CTAS_PER_SM);
            const int opts[2] = {std::min(base.ctas_per_sm, top), top};
            for (int k = 0; st == RF_OK && k < (opts[0] == opts[1] ? 1 : 2); ++k) {
                rf_launch_config cand = base;
                cand.ctas_per_sm = opts[k];
                cand.group = g;
                st = consider(cand);
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != RF_OK)
        return st;
    *best_out = best;
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
    tr->cfg.ctas_per_sm = 0;
    tr->cfg.work_warps = WORK_WARPS_DEFAULT;
    tr->cfg.group = GROUP;
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
    P.work_warps = tr->cfg.work_warps;
    P.timeout_ns = tr->timeout_ns;
    st = launch_batch(P, tr->ls, tr->vol->d.dtype, mode_of(tr->p.flags), tr->cfg.ctas_per_sm, tr->cfg.group,
                      tr->debug_skip, s);
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
    P.work_warps = tr->cfg.work_warps;
    P.timeout_ns = tr->timeout_ns;
    return launch_batch(P, tr->ls, tr->vol->d.dtype, mode_of(tr->p.flags), tr->cfg.ctas_per_sm, tr->cfg.group, 0, s);
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
    st = launch_batch(P, b->ls, b->dtype, b->mode, b->cfg.ctas_per_sm, b->cfg.group, 0, s);
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
    b->cfg.group = GROUP;
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
    rf_launch_config c;
    rf_status st = normalise_config(cfg, &c);
    if (st != RF_OK)
        return st;
    b->cfg = c;
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
                                            b->graph_cfg[parity].work_warps != b->cfg.work_warps ||
                                            b->graph_cfg[parity].group != b->cfg.group);
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
    // the PFO launch rewrites each tracker's r_0 and output pose: keep and restore them
    std::vector<float> saved_scale(6 * b->n), saved_pose(7 * b->n);
    for (int i = 0; i < b->n; ++i) {
        RF_CUDA(cudaMemcpyAsync(&saved_scale[6 * i], b->tr[i]->scale, 6 * sizeof(float), cudaMemcpyDeviceToHost, s));
        RF_CUDA(cudaMemcpyAsync(&saved_pose[7 * i], b->tr[i]->pose_ring + 7 * parity, 7 * sizeof(float),
                                cudaMemcpyDeviceToHost, s));
    }
    RF_CUDA(cudaStreamSynchronize(s));
    auto restore = [&]() -> rf_status {
        for (int i = 0; i < b->n; ++i)
            RF_CUDA(cudaMemcpyAsync(b->tr[i]->scale, &saved_scale[6 * i], 6 * sizeof(float), cudaMemcpyHostToDevice,
                                    s));
        return RF_OK;
    };
    auto run = [&](const rf_launch_config &cand) -> rf_status {
        BatchParams P;
        rf_status st = batch_params(b, parity, P);
        if (st != RF_OK)
            return st;
        P.work_warps = cand.work_warps;
        return launch_batch(P, b->ls, b->dtype, b->mode, cand.ctas_per_sm, cand.group, 0, s);
    };
    rf_launch_config best;
    rf_status st = autotune_search(b->dtype, b->mode, run, restore, s, &best);
    for (int i = 0; i < b->n; ++i) {
        cudaMemcpyAsync(b->tr[i]->scale, &saved_scale[6 * i], 6 * sizeof(float), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(b->tr[i]->pose_ring + 7 * parity, &saved_pose[7 * i], 7 * sizeof(float),
                        cudaMemcpyHostToDevice, s);
    }
    cudaStreamSynchronize(s);
    if (st != RF_OK)
        return st;
    b->cfg = best;
    if (chosen)
        *chosen = best;
    return RF_OK;
}

rf_status rf_tracker_set_config(rf_tracker tr, const rf_launch_config *cfg)
{
    RF_CHECK_ARG(tr && cfg, "null pointer");
    rf_launch_config c;
    rf_status st = normalise_config(cfg, &c);
    if (st != RF_OK)
        return st;
    tr->cfg = c;
    return RF_OK;
}

rf_status rf_tracker_get_config(rf_tracker tr, rf_launch_config *cfg)
{
    RF_CHECK_ARG(tr && cfg, "null pointer");
    *cfg = tr->cfg;
    return RF_OK;
}

rf_status rf_tracker_autotune(rf_tracker tr, const float *depth_dev, const float *prev_depth_dev,
                              const rf_intrinsics *K, const float *prev_pose_dev, rf_launch_config *chosen,
                              void *stream)
{
    RF_CHECK_ARG(tr && depth_dev && prev_depth_dev && K && prev_pose_dev, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    float saved_scale[6];
    RF_CUDA(cudaMemcpyAsync(saved_scale, tr->scale, sizeof saved_scale, cudaMemcpyDeviceToHost, s));
    RF_CUDA(cudaStreamSynchronize(s));
    float *out_pose = nullptr;
    RF_CUDA(cudaMalloc(&out_pose, 7 * sizeof(float)));
    auto restore = [&]() -> rf_status {
        RF_CUDA(cudaMemcpyAsync(tr->scale, saved_scale, sizeof saved_scale, cudaMemcpyHostToDevice, s));
        return RF_OK;
    };
    auto run = [&](const rf_launch_config &cand) -> rf_status {
        BatchParams P;
        memset(&P, 0, sizeof P);
        rf_status st = fill_problem(tr, depth_dev, prev_depth_dev, K, prev_pose_dev, out_pose, nullptr, P.prob[0]);
        if (st != RF_OK)
            return st;
        P.B = 1;
        P.work_warps = cand.work_warps;
        P.timeout_ns = tr->timeout_ns;
        return launch_batch(P, tr->ls, tr->vol->d.dtype, mode_of(tr->p.flags), cand.ctas_per_sm, cand.group, 0, s);
    };
    rf_launch_config best;
    rf_status st = autotune_search(tr->vol->d.dtype, mode_of(tr->p.flags), run, restore, s, &best);
    restore();
    cudaStreamSynchronize(s);
    cudaFree(out_pose);
    if (st != RF_OK)
        return st;
    tr->cfg = best;
    if (chosen)
        *chosen = best;
    return RF_OK;
}

}  // extern "C"
