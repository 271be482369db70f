// learned.cu -- the learned swarm proposal around the PFO tracker: network
// features of a frame pair, training targets, the proposal (c_0, r_0) that
// replaces the Sec. 4 PST initialisation, and the per-frame driver with the
// plain-PFO fallback.  Definitions are in include/rf_proposal.h.
#include <math.h>
#include <string.h>

#include <cuda_bf16.h>

#include "common.cuh"
#include "rf_proposal.h"

namespace rf {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int GRID_W = 32, GRID_H = 24, N_RES = GRID_W * GRID_H;
constexpr double S_Z = 0.1, RES_CLIP = 8.0, S_CLAMP = 6.0;
__constant__ double c_units[6] = {0.05, 0.05, 0.05, 0.1, 0.1, 0.1};

// offset(a, b): b = a (+) d under the left-multiplied MovePST composition
// (Sec. 3.3); d[0..2] = vector part of q_b q_a^-1 (scalar part >= 0), d[3..5] =
// t_b - t_a.  FP64 from the FP32 poses.
__device__ void pose_offset(const float *a, const float *b, double d[6])
{
    double qa[4], qb[4], na = 0.0, nb = 0.0;
    for (int i = 0; i < 4; ++i) {
        qa[i] = a[i];
        qb[i] = b[i];
        na += qa[i] * qa[i];
        nb += qb[i] * qb[i];
    }
    nb = sqrt(nb);
    for (int i = 0; i < 4; ++i)
        qb[i] /= nb;
    const double ia[4] = {qa[0] / na, -qa[1] / na, -qa[2] / na, -qa[3] / na};
    double q[4];
    q[0] = qb[0] * ia[0] - qb[1] * ia[1] - qb[2] * ia[2] - qb[3] * ia[3];
    q[1] = qb[0] * ia[1] + qb[1] * ia[0] + qb[2] * ia[3] - qb[3] * ia[2];
    q[2] = qb[0] * ia[2] - qb[1] * ia[3] + qb[2] * ia[0] + qb[3] * ia[1];
    q[3] = qb[0] * ia[3] + qb[1] * ia[2] - qb[2] * ia[1] + qb[3] * ia[0];
    const double sg = q[0] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < 3; ++i) {
        d[i] = sg * q[1 + i];
        d[3 + i] = (double)b[4 + i] - (double)a[4 + i];
    }
}

constexpr int FEAT_WARPS = 8;                             // cells per CTA (one warp each)
constexpr int FEAT_CTAS = N_RES / FEAT_WARPS + 1;          // + one CTA for the offset / padding entries

// One warp per grid cell (i, j): the lanes stride over the cell's pixels, sum
// the valid depths of both frames in FP64 and reduce in a fixed shuffle order;
// lane 0 writes the clipped residual.  The last CTA writes the offset features
// and the zero padding.  (FP64 is spread over the grid: GB300's per-SM FP64
// rate is low, one CTA of FP64 sums would serialise on one SM.)
__global__ void __launch_bounds__(FEAT_WARPS * 32) features_kernel(const float *depth, const float *prev_depth,
                                                                   Intr K, const float *pose_prev2,
                                                                   const float *pose_prev, bf16 *x)
{
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == FEAT_CTAS - 1) {
        const int t = N_RES + threadIdx.x;
        if (t < RF_MLP_IN) {
            double v = 0.0;
            if (t < RF_MLP_IN_USED) {
                double d[6];
                pose_offset(pose_prev2, pose_prev, d);
                v = d[t - N_RES] / c_units[t - N_RES];
            }
            x[t] = __double2bfloat16(v);
        }
        return;
    }
    const int cell = blockIdx.x * FEAT_WARPS + (threadIdx.x >> 5);
    const int i = cell % GRID_W, j = cell / GRID_W;
    const int c0 = (i * K.width) / GRID_W, c1 = ((i + 1) * K.width) / GRID_W;
    const int r0 = (j * K.height) / GRID_H, r1 = ((j + 1) * K.height) / GRID_H;
    const int cw = c1 - c0, npix = cw * (r1 - r0);
    double sc = 0.0, sp = 0.0;
    int nc = 0, np = 0;
    for (int p = lane; p < npix; p += 32) {
        const int r = r0 + p / cw, c = c0 + p % cw;
        const size_t o = (size_t)r * K.width + c;
        const float zc = __ldg(&depth[o]), zp = __ldg(&prev_depth[o]);
        if (zc > K.z_min && zc <= K.z_max) {
            sc += zc;
            ++nc;
        }
        if (zp > K.z_min && zp <= K.z_max) {
            sp += zp;
            ++np;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
        sp += __shfl_xor_sync(0xffffffffu, sp, o);
        nc += __shfl_xor_sync(0xffffffffu, nc, o);
        np += __shfl_xor_sync(0xffffffffu, np, o);
    }
    if (lane == 0) {
        double f = 0.0;
        if (nc > 0 && np > 0)
            f = fmin(fmax((sc / nc - sp / np) / S_Z, -RES_CLIP), RES_CLIP);
        x[cell] = __double2bfloat16(f);
    }
}

__global__ void target_kernel(const float *pose_prev, const float *pose_cur, float *y)
{
    double d[6];
    pose_offset(pose_prev, pose_cur, d);
    for (int i = 0; i < 6; ++i)
        y[i] = (float)(d[i] / c_units[i]);
}

struct PropParams {
    float kappa;
    float r_min[6], r_max[6];
};

// c_0 = s*_{t-1} (+) mu * units with mu = x_v + o_mu (x_v: the previous-offset
// inputs of the network), r_0 = clip(kappa e^s units, r_min, r_max).
__device__ void proposal(const float *o, const bf16 *x, const float *prev, const PropParams &p, float *c0, float *r0)
{
    Pose c;
    for (int a = 0; a < 4; ++a)
        c.q[a] = prev[a];
    for (int a = 0; a < 3; ++a)
        c.t[a] = prev[4 + a];
    float d[6];
    for (int i = 0; i < 6; ++i)
        d[i] = (__bfloat162float(x[N_RES + i]) + o[i]) * (float)c_units[i];
    Pose out;
    compose_offset(c, d, false, out);
    for (int a = 0; a < 4; ++a)
        c0[a] = out.q[a];
    for (int a = 0; a < 3; ++a)
        c0[4 + a] = out.t[a];
    for (int i = 0; i < 6; ++i) {
        const float s = fminf(fmaxf(o[6 + i], -(float)S_CLAMP), (float)S_CLAMP);
        r0[i] = fminf(fmaxf(p.kappa * expf(s) * (float)c_units[i], p.r_min[i]), p.r_max[i]);
    }
}

__global__ void apply_kernel(const float *o, const bf16 *x, const float *prev, PropParams p, float *c0, float *r0,
                             float *r0_copy)
{
    proposal(o, x, prev, p, c0, r0);
    if (r0_copy)
        for (int i = 0; i < 6; ++i)
            r0_copy[i] = r0[i];
}

// Final rho_tilde of a run (0 when it made no iteration).
__device__ float final_rho(const rf_frame_stats *s)
{
    return s->iters > 0 ? s->it[s->iters - 1].rho_tilde : 0.f;
}

// Per-frame state of a learned tracker on the device.
struct LearnedState {
    float hist[2][7];       // s*_{t-2}, s*_{t-1}
    float c0[7];            // proposal centre
    float r0[6];            // proposal axis lengths
    float r_learned[6];     // r_0 of the learned run, r_1 after it
    float r_carry[6];       // r_1 carried for the plain fallback (Sec. 4)
    float r_fb[6];          // second run's r_0 in / r_1 out
    float c_fb[7];          // second run's centre: s*_{t-1} (restart) or the learned s* (resume)
    float pose_l[7], pose_f[7];
    float rho_prev;
    int run_flag;           // 0 no second run, 1 plain restart, 2 resume of the learned run
    int status;             // final status of the frame (fusion skips when != 0)
    rf_frame_stats st_l, st_f;
};

// Second run of a frame: a plain restart from s*_{t-1} with the carried r_1 when
// the learned run failed, its final rho_tilde fell below theta x the previous
// frame's, or its first iteration found no TSDF sample for any particle (the
// first corner case of Sec. 4: the proposal lies off the map, where every
// particle scores alike and PFO cannot leave c_0, so keeping it would let the
// next proposal extrapolate the jump); otherwise, with `resume`, a continuation
// from the learned run's state (its s* and axis lengths) when that run used all
// k_learned iterations without meeting a convergence criterion of Sec. 4 (stop
// reason k_max).
__global__ void judge_kernel(LearnedState *S, float theta, int resume, int stuck)
{
    const rf_frame_stats &l = S->st_l;
    const float rho = final_rho(&l);
    const int last = min(l.iters, RF_MAX_ITERS) - 1;
    const bool off_map = l.iters > 0 && l.it[0].corner == 1;
    const bool bad = l.status != 0 || l.iters == 0 || rho < theta * S->rho_prev || off_map;
    const bool open = last >= 0 && l.it[last].stop == 3;
    bool moved = false;  // some iteration had a non-empty APS, i.e. s* left c_0
    for (int k = 0; k <= last; ++k)
        moved |= l.it[k].n_aps > 0;
    // 1 plain restart, 2 resume of the learned run, 3 resume from c_0 with the carried r_1
    int mode = 0;
    if (theta >= 0.f) {
        if (bad || (!moved && stuck == 2))
            mode = 1;
        else if (!moved && stuck == 1)
            mode = 3;
        else if (resume && open)
            mode = 2;
    }
    S->run_flag = mode;
    for (int a = 0; a < 7; ++a)
        S->c_fb[a] = mode == 2 ? S->pose_l[a] : (mode == 3 ? S->c0[a] : S->hist[1][a]);
    for (int i = 0; i < 6; ++i)
        S->r_fb[i] = mode == 2 ? l.it[last].scale[i] : S->r_carry[i];
}

__global__ void select_kernel(LearnedState *S, rf_learned_stats *out_stats, float *out_pose)
{
    const rf_frame_stats &l = S->st_l, &f = S->st_f;
    const float rl = final_rho(&l), rfb = final_rho(&f);
    const bool ran = S->run_flag != 0 && f.iters > 0;
    // the higher final rho_tilde wins; a tie goes to a plain restart (the method's
    // own tracker from s*_{t-1}), otherwise to the learned run
    const bool take_f = ran && f.status == 0 && (l.status != 0 || rfb > rl || (S->run_flag == 1 && rfb == rl));
    const float *p = take_f ? S->pose_f : S->pose_l;
    if (out_stats) {
        out_stats->status = take_f ? f.status : l.status;
        out_stats->used_fallback = ran ? S->run_flag : 0;
        out_stats->chose_fallback = take_f ? 1 : 0;
        out_stats->iters_learned = l.iters;
        out_stats->iters_fallback = ran ? f.iters : 0;
        out_stats->rho_learned = rl;
        out_stats->rho_fallback = ran ? rfb : 0.f;
        out_stats->rho_prev = S->rho_prev;
        for (int a = 0; a < 7; ++a)
            out_stats->init_pose[a] = S->c0[a];
        for (int i = 0; i < 6; ++i)
            out_stats->r0[i] = S->r0[i];
        out_stats->lookups = l.lookups + (ran ? f.lookups : 0);
    }
    S->status = take_f ? f.status : l.status;
    S->rho_prev = take_f ? rfb : rl;
    for (int i = 0; i < 6; ++i)
        S->r_carry[i] = take_f ? S->r_fb[i] : S->r_learned[i];
    for (int a = 0; a < 7; ++a) {
        const float v = p[a];
        S->hist[0][a] = S->hist[1][a];
        S->hist[1][a] = v;
        if (out_pose)
            out_pose[a] = v;
    }
}

__global__ void start_kernel(LearnedState *S, Pose p, const float *r)
{
    for (int a = 0; a < 4; ++a)
        S->hist[0][a] = S->hist[1][a] = p.q[a];
    for (int a = 0; a < 3; ++a)
        S->hist[0][4 + a] = S->hist[1][4 + a] = p.t[a];
    for (int i = 0; i < 6; ++i)
        S->r_carry[i] = r[i];
    S->rho_prev = 0.f;
    S->status = 0;
}

PropParams to_params(const rf_proposal_params &p)
{
    PropParams q;
    q.kappa = p.kappa;
    for (int i = 0; i < 6; ++i) {
        q.r_min[i] = p.r_min[i];
        q.r_max[i] = p.r_max[i];
    }
    return q;
}

rf_status check_params(const rf_proposal_params *p)
{
    RF_CHECK_ARG(p != nullptr, "null parameters");
    RF_CHECK_ARG(p->k_learned >= 1 && p->k_learned <= RF_MAX_ITERS, "k_learned outside [1, RF_MAX_ITERS]");
    RF_CHECK_ARG(p->k_fallback >= 1 && p->k_fallback <= RF_MAX_ITERS, "k_fallback outside [1, RF_MAX_ITERS]");
    RF_CHECK_ARG(p->kappa > 0.f, "kappa must be positive");
    RF_CHECK_ARG(p->resume == 0 || p->resume == 1, "resume must be 0 or 1");
    RF_CHECK_ARG(p->stuck >= 0 && p->stuck <= 2, "stuck must be 0, 1 or 2");
    for (int i = 0; i < 6; ++i)
        RF_CHECK_ARG(p->r_min[i] > 0.f && p->r_max[i] >= p->r_min[i], "r_min / r_max");
    return RF_OK;
}

}  // namespace
}  // namespace rf

using namespace rf;

struct rf_learned_s {
    rf_tracker tr;
    rf_volume vol;
    rf_mlp net;
    rf_proposal_params p;
    int max_w, max_h;
    float *depth_cur = nullptr, *depth_prev = nullptr;
    uint16_t *x = nullptr;
    float *out = nullptr;
    LearnedState *S = nullptr;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    rf_intrinsics graph_K;  // what the graph was captured for
    rf_learned_stats *graph_stats = nullptr;
    float *graph_pose = nullptr;
};

// The kernels of one frame (after the depth is in depth_cur).  Capturable.
static rf_status learned_enqueue(rf_learned lp, const rf_intrinsics *K, rf_learned_stats *stats_dev, float *out_pose,
                                 cudaStream_t s)
{
    LearnedState *S = lp->S;
    features_kernel<<<FEAT_CTAS, FEAT_WARPS * 32, 0, s>>>(lp->depth_cur, lp->depth_prev, to_intr(*K), S->hist[0],
                                                          S->hist[1], reinterpret_cast<bf16 *>(lp->x));
    RF_CUDA(cudaGetLastError());
    rf_status st = rf_mlp_forward(lp->net, lp->x, 1, lp->out, s);
    if (st != RF_OK)
        return st;
    apply_kernel<<<1, 1, 0, s>>>(lp->out, reinterpret_cast<const bf16 *>(lp->x), S->hist[1], to_params(lp->p), S->c0,
                                 S->r_learned, S->r0);
    RF_CUDA(cudaGetLastError());
    rf_track_options o;
    memset(&o, 0, sizeof o);
    o.init_pose_dev = S->c0;
    o.scale_dev = S->r_learned;
    o.k_max = lp->p.k_learned;
    st = pfo_track_frame_ex_async(lp->tr, lp->depth_cur, lp->depth_prev, K, S->hist[1], S->pose_l, &S->st_l, &o, s);
    if (st != RF_OK)
        return st;
    judge_kernel<<<1, 1, 0, s>>>(S, lp->p.theta, lp->p.resume, lp->p.stuck);
    RF_CUDA(cudaGetLastError());
    memset(&o, 0, sizeof o);
    o.init_pose_dev = S->c_fb;
    o.scale_dev = S->r_fb;
    o.run_flag_dev = &S->run_flag;
    o.k_max = lp->p.k_fallback;
    st = pfo_track_frame_ex_async(lp->tr, lp->depth_cur, lp->depth_prev, K, S->hist[1], S->pose_f, &S->st_f, &o, s);
    if (st != RF_OK)
        return st;
    select_kernel<<<1, 1, 0, s>>>(S, stats_dev, out_pose);
    RF_CUDA(cudaGetLastError());
    st = tsdf_integrate_dev(lp->vol, lp->depth_cur, K, S->hist[1], &S->status, s);
    if (st != RF_OK)
        return st;
    RF_CUDA(cudaMemcpyAsync(lp->depth_prev, lp->depth_cur, (size_t)K->width * K->height * sizeof(float),
                            cudaMemcpyDeviceToDevice, s));
    return RF_OK;
}

extern "C" {

void rf_proposal_default_params(rf_proposal_params *p)
{
    if (!p)
        return;
    p->k_learned = 5;
    p->k_fallback = 20;
    p->kappa = 0.25f;
    p->theta = 0.95f;
    p->resume = 1;
    p->stuck = 1;
    for (int i = 0; i < 6; ++i) {
        p->r_min[i] = i < 3 ? 2e-3f : 4e-3f;
        p->r_max[i] = i < 3 ? 0.2f : 0.4f;
    }
}

rf_status rf_proposal_features(const float *depth_dev, const float *prev_depth_dev, const rf_intrinsics *K,
                               const float *pose_prev2_dev, const float *pose_prev_dev, uint16_t *x_dev, void *stream)
{
    RF_CHECK_ARG(depth_dev && prev_depth_dev && K && pose_prev2_dev && pose_prev_dev && x_dev, "null pointer");
    RF_CHECK_ARG(K->width >= 1 && K->height >= 1, "bad frame size");
    features_kernel<<<FEAT_CTAS, FEAT_WARPS * 32, 0, (cudaStream_t)stream>>>(
        depth_dev, prev_depth_dev, to_intr(*K), pose_prev2_dev, pose_prev_dev, reinterpret_cast<bf16 *>(x_dev));
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

rf_status rf_proposal_target(const float *pose_prev_dev, const float *pose_cur_dev, float *y_dev, void *stream)
{
    RF_CHECK_ARG(pose_prev_dev && pose_cur_dev && y_dev, "null pointer");
    target_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(pose_prev_dev, pose_cur_dev, y_dev);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

rf_status rf_proposal_apply(const float *out_dev, const uint16_t *x_dev, const float *pose_prev_dev,
                            const rf_proposal_params *p, float *init_pose_dev, float *scale_dev, void *stream)
{
    RF_CHECK_ARG(out_dev && x_dev && pose_prev_dev && init_pose_dev && scale_dev, "null pointer");
    rf_status st = check_params(p);
    if (st != RF_OK)
        return st;
    apply_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(out_dev, reinterpret_cast<const bf16 *>(x_dev), pose_prev_dev,
                                                    to_params(*p), init_pose_dev, scale_dev, nullptr);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

rf_status rf_learned_create(rf_tracker tr, rf_volume vol, rf_mlp net, const rf_proposal_params *p, int max_width,
                            int max_height, rf_learned *out)
{
    RF_CHECK_ARG(out != nullptr, "null output");
    *out = nullptr;
    RF_CHECK_ARG(tr && vol && net, "null handle");
    RF_CHECK_ARG(max_width >= 1 && max_height >= 1, "bad frame size");
    rf_status st = check_params(p);
    if (st != RF_OK)
        return st;
    rf_learned lp = new rf_learned_s();
    lp->tr = tr;
    lp->vol = vol;
    lp->net = net;
    lp->p = *p;
    lp->max_w = max_width;
    lp->max_h = max_height;
    const size_t px = (size_t)max_width * max_height;
    cudaError_t e = cudaMalloc(&lp->depth_cur, px * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&lp->depth_prev, px * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&lp->x, RF_MLP_IN * sizeof(uint16_t));
    if (e == cudaSuccess)
        e = cudaMalloc(&lp->out, RF_MLP_OUT * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&lp->S, sizeof(LearnedState));
    if (e == cudaSuccess)
        e = cudaMemset(lp->S, 0, sizeof(LearnedState));
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&lp->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        rf_learned_destroy(lp);
        return cuda_fail(e, "rf_learned_create");
    }
    *out = lp;
    return RF_OK;
}

void rf_learned_destroy(rf_learned lp)
{
    if (!lp)
        return;
    if (lp->graph)
        cudaGraphExecDestroy(lp->graph);
    if (lp->capture_stream)
        cudaStreamDestroy(lp->capture_stream);
    cudaFree(lp->depth_cur);
    cudaFree(lp->depth_prev);
    cudaFree(lp->x);
    cudaFree(lp->out);
    cudaFree(lp->S);
    delete lp;
}

rf_status rf_learned_start(rf_learned lp, const float *depth, int depth_on_host, const rf_intrinsics *K,
                           const rf_pose *pose, void *stream)
{
    RF_CHECK_ARG(lp && depth && K && pose, "null pointer");
    RF_CHECK_ARG(K->width >= 1 && K->height >= 1 && K->width <= lp->max_w && K->height <= lp->max_h,
                 "bad frame size");
    cudaStream_t s = (cudaStream_t)stream;
    float r[6];
    rf_status st = rf_tracker_get_scale(lp->tr, r);
    if (st != RF_OK)
        return st;
    float *r_dev = lp->out;  // staging for the carried axis lengths
    RF_CUDA(cudaMemcpyAsync(r_dev, r, sizeof r, cudaMemcpyHostToDevice, s));
    RF_CUDA(cudaMemcpyAsync(lp->depth_prev, depth, (size_t)K->width * K->height * sizeof(float),
                            depth_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    Pose p;
    for (int a = 0; a < 4; ++a)
        p.q[a] = pose->q[a];
    for (int a = 0; a < 3; ++a)
        p.t[a] = pose->t[a];
    start_kernel<<<1, 1, 0, s>>>(lp->S, p, r_dev);
    RF_CUDA(cudaGetLastError());
    st = tsdf_integrate(lp->vol, lp->depth_prev, K, pose, s);
    if (st != RF_OK)
        return st;
    RF_CUDA(cudaStreamSynchronize(s));  // the staging buffer and host r are reused
    return RF_OK;
}

rf_status rf_learned_step(rf_learned lp, const float *depth, int depth_on_host, const rf_intrinsics *K, int use_graph,
                          rf_pose *out_pose_host, float *out_pose_dev, rf_learned_stats *stats_dev, void *stream)
{
    RF_CHECK_ARG(lp && depth && K, "null pointer");
    RF_CHECK_ARG(K->width >= 1 && K->height >= 1 && K->width <= lp->max_w && K->height <= lp->max_h,
                 "bad frame size");
    cudaStream_t s = (cudaStream_t)stream;
    RF_CUDA(cudaMemcpyAsync(lp->depth_cur, depth, (size_t)K->width * K->height * sizeof(float),
                            depth_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    if (!use_graph) {
        rf_status st = learned_enqueue(lp, K, stats_dev, out_pose_dev, s);
        if (st != RF_OK)
            return st;
    } else {
        if (lp->graph && (memcmp(&lp->graph_K, K, sizeof *K) != 0 || lp->graph_stats != stats_dev ||
                          lp->graph_pose != out_pose_dev)) {
            cudaGraphExecDestroy(lp->graph);
            lp->graph = nullptr;
        }
        if (!lp->graph) {
            cudaStream_t cs = lp->capture_stream;
            RF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            rf_status st = learned_enqueue(lp, K, stats_dev, out_pose_dev, cs);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(cs, &g);
            if (st != RF_OK) {
                if (g)
                    cudaGraphDestroy(g);
                return st;
            }
            if (e != cudaSuccess)
                return cuda_fail(e, "cudaStreamEndCapture(learned step)");
            e = cudaGraphInstantiate(&lp->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess)
                return cuda_fail(e, "cudaGraphInstantiate(learned step)");
            lp->graph_K = *K;
            lp->graph_stats = stats_dev;
            lp->graph_pose = out_pose_dev;
        }
        RF_CUDA(cudaGraphLaunch(lp->graph, s));
    }
    if (out_pose_host) {
        float h[7];
        int hs = 0;
        RF_CUDA(cudaMemcpyAsync(h, lp->S->hist[1], sizeof h, cudaMemcpyDeviceToHost, s));
        RF_CUDA(cudaMemcpyAsync(&hs, &lp->S->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        RF_CUDA(cudaStreamSynchronize(s));
        for (int a = 0; a < 4; ++a)
            out_pose_host->q[a] = h[a];
        for (int a = 0; a < 3; ++a)
            out_pose_host->t[a] = h[4 + a];
        if (hs != 0)
            set_error("rf_learned_step: device status %d", hs);
        return hs;
    }
    return RF_OK;
}

}  // extern "C"
