/*
 * rf_oracle.c -- plain FP64 CPU oracle for the ROSEFusion depth-only tracking path
 * (Zhang, Zhu, Zheng, Xu, "ROSEFusion: Random Optimization for Online Dense
 * Reconstruction under Fast Camera Motion", ACM TOG 40(4), 2021).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg load it.  It shares no code, header, table or helper with the CUDA
 * library; it is written to be read against the paper line by line, so every
 * loop is the literal definition: no blocking, no fusion, no reordering, all
 * arithmetic in double precision.
 *
 * Conventions (shared with the CUDA path only through the paper and the
 * readings listed in the design notes):
 *   pose  = double[7]: q = (w, x, y, z) unit Hamilton quaternion, w >= 0,
 *           then t = (x, y, z); camera -> world: x_G = R(q) x + t  (Sec. 3.1, Eq. unproj)
 *   state offset = double[6]: (q_x, q_y, q_z, x, y, z)             (Sec. 3.3)
 *   volume = dense x-fastest array F[dx*dy*dz] of normalised TSDF values
 *           (NaN = never observed) plus integer weights W; voxel (i,j,k) has
 *           its centre at origin + voxel*(i+0.5, j+0.5, k+0.5).
 *   points = double[4*M]: camera-frame (x, y, z, flag), flag 1 = valid depth.
 *
 * Flags (same bit values as the library's parameter block):
 *   1 OVERLAP      normalise over the overlap set O_k (Eq. validness); else over all valid points
 *   2 NORMALIZE    divide the sum by |O_k| (Eq. normallh); else Eq. ourlh
 *   4 COMPENSATED  (GPU summation only; the oracle always sums in FP64)
 *   8 NEAREST      nearest-voxel sample instead of trilinear
 *  16 RHO_REF_CENTER  APS threshold = fitness of the current centre particle
 *  32 L1           sum |psi| instead of psi^2
 *  64 RIGHT_MULT   particle offset applied in the camera frame (T_c * T_delta)
 * 128 CELL_MARGIN  overlap set: the re-projected point must lie inside frame
 *                  t-1's image by the footprint of one TSDF cell (sqrt(3) voxels)
 * 256 APS_WITH_CENTRE  the centre particle (particle 0, s*_{k-1} itself) is an
 *                  APS candidate like every other particle
 *
 * Threads: or_fitness_particles, the *_mt frame functions and
 * or_tsdf_integrate_mt may split independent items (particles, voxel slices)
 * over threads for speed; every item is computed by the same plain loop and
 * every reduction stays sequential, so the results do not depend on the
 * thread count.
 *
 * Functions whose result has no independent pin say so in their comment;
 * every other function is pinned by tests/test_oracle_*.py.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OVERLAP 1
#define OR_NORMALIZE 2
#define OR_COMPENSATED 4
#define OR_NEAREST 8
#define OR_RHO_REF_CENTER 16
#define OR_L1 32
#define OR_RIGHT_MULT 64
#define OR_CELL_MARGIN 128
#define OR_APS_WITH_CENTRE 256

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_EMPTY -4

/* ------------------------------------------------------------------------- */
/* Quaternion algebra (Sec. 3.3 parameterises rotation by a unit quaternion). */
/* ------------------------------------------------------------------------- */

/* Hamilton product o = a (x) b. */
void or_quat_mul(const double a[4], const double b[4], double o[4])
{
    double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    o[0] = w;
    o[1] = x;
    o[2] = y;
    o[3] = z;
}

/* Row-major rotation matrix of a unit quaternion (w, x, y, z). */
void or_quat_to_rot(const double q[4], double R[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

static void normalise_quat_wpos(double q[4])
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i)
        q[i] /= n;
    if (q[0] < 0.0)
        for (int i = 0; i < 4; ++i)
            q[i] = -q[i];
}

/* y = R x + t */
static void apply_pose(const double R[9], const double t[3], const double x[3], double y[3])
{
    for (int r = 0; r < 3; ++r)
        y[r] = R[3 * r + 0] * x[0] + R[3 * r + 1] * x[1] + R[3 * r + 2] * x[2] + t[r];
}

/* y = R^T (x - t): world -> camera for a camera -> world pose. */
static void apply_pose_inverse(const double R[9], const double t[3], const double x[3], double y[3])
{
    double d[3] = {x[0] - t[0], x[1] - t[1], x[2] - t[2]};
    for (int c = 0; c < 3; ++c)
        y[c] = R[0 * 3 + c] * d[0] + R[1 * 3 + c] * d[1] + R[2 * 3 + c] * d[2];
}

/*
 * MovePST for one particle (Sec. 3.3 "PST move"; Algorithm 1; the exact
 * transform is in the paper's missing supplement).  Reading: the state offset
 * delta = (dq_x, dq_y, dq_z, dt_x, dt_y, dt_z) about the centre pose c is the
 * imaginary part of a unit quaternion (real part sqrt(1 - |dq|^2), |dq|
 * clamped to 1) and a translation.  Default: q = q_delta (x) q_c, t = t_c + dt
 * (rotation about the camera centre in world axes).  RIGHT_MULT: the SE(3)
 * product T_c * T_delta.  The result is renormalised with w >= 0.
 */
void or_compose_offset(const double c[7], const double delta[6], int flags, double out[7])
{
    double dq[3] = {delta[0], delta[1], delta[2]};
    double n2 = dq[0] * dq[0] + dq[1] * dq[1] + dq[2] * dq[2];
    if (n2 > 1.0) {
        double s = 1.0 / sqrt(n2);
        dq[0] *= s;
        dq[1] *= s;
        dq[2] *= s;
        n2 = 1.0;
    }
    double qd[4] = {sqrt(1.0 - n2), dq[0], dq[1], dq[2]};
    double q[4];
    if (flags & OR_RIGHT_MULT) {
        double Rc[9];
        or_quat_to_rot(c, Rc);
        or_quat_mul(c, qd, q);
        for (int r = 0; r < 3; ++r)
            out[4 + r] = c[4 + r] + Rc[3 * r + 0] * delta[3] + Rc[3 * r + 1] * delta[4] + Rc[3 * r + 2] * delta[5];
    } else {
        or_quat_mul(qd, c, q);
        for (int r = 0; r < 3; ++r)
            out[4 + r] = c[4 + r] + delta[3 + r];
    }
    normalise_quat_wpos(q);
    for (int i = 0; i < 4; ++i)
        out[i] = q[i];
}

/* RescalePST: particle i of the template omega (6 x N, structure of arrays)
 * at centre c and axis lengths r is c (+) (r (.) omega_i)  (Sec. 3.3, Sec. 4
 * "GPU implementation": the original unit-ball PST is moved and rescaled). */
void or_particle_pose(const double c[7], const double r[6], const double omega6[6], int flags, double out[7])
{
    double delta[6];
    for (int d = 0; d < 6; ++d)
        delta[d] = r[d] * omega6[d];
    or_compose_offset(c, delta, flags, out);
}

/* ------------------------------------------------------------------------- */
/* Depth preprocessing (Eq. unproj; Sec. 4 stride-based downsampling).        */
/* ------------------------------------------------------------------------- */

/* Points are taken at full-resolution pixels (a*stride, b*stride), row-major
 * over (b, a).  Returns the number of points written (ceil(H/s)*ceil(W/s)). */
int or_unproject(const float *depth, int W, int H, double fx, double fy, double cx, double cy,
                 double z_min, double z_max, int stride, double *pts)
{
    if (stride < 1)
        return OR_ERR_ARG;
    int nw = (W + stride - 1) / stride, nh = (H + stride - 1) / stride;
    for (int b = 0; b < nh; ++b)
        for (int a = 0; a < nw; ++a) {
            int u = a * stride, v = b * stride;
            double z = depth[(size_t)v * W + u];
            double *p = pts + 4 * ((size_t)b * nw + a);
            if (z > z_min && z <= z_max) {
                p[0] = ((double)u - cx) * z / fx;
                p[1] = ((double)v - cy) * z / fy;
                p[2] = z;
                p[3] = 1.0;
            } else {
                p[0] = p[1] = p[2] = p[3] = 0.0;
            }
        }
    return nw * nh;
}

/*
 * Overlap set O_k (Eq. validness, Sec. 4 "TSDF normalization"): a valid point
 * is unprojected with the current estimate s*_{k-1}, re-projected into frame
 * t-1 with its final pose, and kept if it lands in front of that camera, the
 * nearest pixel lies inside the image and frame t-1 has a valid depth there.
 * With cell_m > 0 (flag CELL_MARGIN, cell_m = sqrt(3) voxels) the continuous
 * pixel position must also lie at least fx cell_m / z' (fy cell_m / z'
 * vertically) pixels inside the image edges (-0.5 and W - 0.5), z' the
 * point's depth in frame t-1: the TSDF cell the point samples then lies
 * inside that frame's view, i.e. the pixel is observed by both frames at the
 * volume's resolution.
 * margin[j] (optional) is the distance of the continuous pixel coordinate to
 * the nearest rounding boundary or (inset) image border, in pixels; tests use
 * it to skip decisions that FP32 and FP64 may legitimately take differently.
 * Returns |O_k|.
 */
int or_overlap(const double *pts, int M, const float *prev_depth, int W, int H, double fx, double fy,
               double cx, double cy, double z_min, double z_max, const double pose_cur[7],
               const double pose_prev[7], double cell_m, int *mask, double *margin)
{
    double Rc[9], Rp[9];
    or_quat_to_rot(pose_cur, Rc);
    or_quat_to_rot(pose_prev, Rp);
    int count = 0;
    for (int j = 0; j < M; ++j) {
        const double *p = pts + 4 * (size_t)j;
        mask[j] = 0;
        if (margin)
            margin[j] = INFINITY;
        if (p[3] == 0.0)
            continue;
        double pg[3], pc[3];
        apply_pose(Rc, pose_cur + 4, p, pg);
        apply_pose_inverse(Rp, pose_prev + 4, pg, pc);
        if (!(pc[2] > 0.0))
            continue;
        double u = fx * pc[0] / pc[2] + cx;
        double v = fy * pc[1] / pc[2] + cy;
        double ur = floor(u + 0.5), vr = floor(v + 0.5);
        double bu = fx * cell_m / pc[2], bv = fy * cell_m / pc[2]; /* cell footprint in pixels */
        if (margin) {
            double mu = fabs((u + 0.5) - ur), mu2 = fabs((u + 0.5) - (ur + 1.0));
            double mv = fabs((v + 0.5) - vr), mv2 = fabs((v + 0.5) - (vr + 1.0));
            double m = fmin(fmin(mu, mu2), fmin(mv, mv2));
            if (cell_m > 0.0) {
                m = fmin(m, fmin(fabs(u - (bu - 0.5)), fabs(((double)W - 0.5 - bu) - u)));
                m = fmin(m, fmin(fabs(v - (bv - 0.5)), fabs(((double)H - 0.5 - bv) - v)));
            }
            margin[j] = m;
        }
        if (ur < 0.0 || ur >= (double)W || vr < 0.0 || vr >= (double)H)
            continue;
        if (u < bu - 0.5 || u >= (double)W - 0.5 - bu || v < bv - 0.5 || v >= (double)H - 0.5 - bv)
            continue;
        double d = prev_depth[(size_t)vr * W + (size_t)ur];
        if (d > z_min && d <= z_max) {
            mask[j] = 1;
            ++count;
        }
    }
    return count;
}

/* ------------------------------------------------------------------------- */
/* TSDF sampling (Sec. 3.1: psi queried at R x + t).                          */
/* ------------------------------------------------------------------------- */

static double vox(const double *F, const int dim[3], int i, int j, int k)
{
    return F[(size_t)i + (size_t)dim[0] * ((size_t)j + (size_t)dim[1] * (size_t)k)];
}

/*
 * psi at world point p.  Trilinear interpolation of the voxel-centre samples;
 * the sample is valid only if all 8 corners lie inside the volume and have
 * been observed (readings 2-3).  NEAREST takes the closest voxel centre.
 * Returns 1 if valid.
 */
int or_tsdf_sample(const double *F, const int dim[3], double voxel, const double origin[3], const double p[3],
                   int flags, double *psi)
{
    double g[3];
    for (int a = 0; a < 3; ++a)
        g[a] = (p[a] - origin[a]) / voxel - 0.5;
    if (flags & OR_NEAREST) {
        int i[3];
        for (int a = 0; a < 3; ++a) {
            double r = floor(g[a] + 0.5);
            if (r < 0.0 || r > (double)(dim[a] - 1))
                return 0;
            i[a] = (int)r;
        }
        double v = vox(F, dim, i[0], i[1], i[2]);
        if (isnan(v))
            return 0;
        *psi = v;
        return 1;
    }
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(g[a]);
        if (fl < 0.0 || fl > (double)(dim[a] - 2))
            return 0;
        i0[a] = (int)fl;
        f[a] = g[a] - fl;
    }
    double sum = 0.0;
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                double v = vox(F, dim, i0[0] + a, i0[1] + b, i0[2] + c);
                if (isnan(v))
                    return 0;
                double w = (a ? f[0] : 1.0 - f[0]) * (b ? f[1] : 1.0 - f[1]) * (c ? f[2] : 1.0 - f[2]);
                sum += w * v;
            }
    *psi = sum;
    return 1;
}

/*
 * Fitness of one pose (Eq. normallh; Eq. ourlh without NORMALIZE).
 * Sums psi^2 (|psi| with L1) over the points with in_set[j] != 0; a point
 * whose sample is invalid contributes psi = 1, the largest truncated value
 * (reading 2).  Outputs S = the sum, n = number of valid samples, nO = |O|,
 * rho.  |O| = 0 gives rho = 0.
 */
void or_fitness(const double *F, const int dim[3], double voxel, const double origin[3], const double *pts,
                const int *in_set, int M, const double pose[7], double tau, int flags, double *S_out,
                int *n_out, int *nO_out, double *rho_out)
{
    double R[9];
    or_quat_to_rot(pose, R);
    double S = 0.0;
    int n = 0, nO = 0;
    for (int j = 0; j < M; ++j) {
        if (!in_set[j])
            continue;
        ++nO;
        double pg[3], psi;
        apply_pose(R, pose + 4, pts + 4 * (size_t)j, pg);
        if (or_tsdf_sample(F, dim, voxel, origin, pg, flags, &psi))
            ++n;
        else
            psi = 1.0;
        S += (flags & OR_L1) ? fabs(psi) : psi * psi;
    }
    double rho;
    if (nO == 0)
        rho = 0.0;
    else if (flags & OR_NORMALIZE)
        rho = exp(-S / (tau * (double)nO));
    else
        rho = exp(-S / tau);
    *S_out = S;
    *n_out = n;
    *nO_out = nO;
    *rho_out = rho;
}

/* ------------------------------------------------------------------------- */
/* PST state update: APS, CompBestState, CompAxisLength (Sec. 3.3, Sec. 4).   */
/* ------------------------------------------------------------------------- */

/*
 * One PST update from the N fitness values rho[i] of particles with state
 * offsets delta[6*i..] about the centre c_{k-1}:
 *   APS = { i : rho_i > rho_ref }                                (Sec. 3.3)
 *   w_i = rho_i - rho_ref,  wbar_i = w_i / sum w                 (Eq. ebs)
 *   delta_bar = sum wbar_i delta_i  (s*_k = c_{k-1} (+) delta_bar)
 *   rho_tilde = sum wbar_i rho_i                                 (Eq. wafit)
 *   v = delta_bar                                                (Eq. rsdir)
 *   rhat = (1 - rho_tilde) |v| / ||v|| + eps                     (Eq. rsinter, reading 6)
 *   r_k  = beta r_{k-1} + (1 - beta) rhat                        (Eq. momentum)
 * Empty APS (Sec. 4 "PST update", second corner case): delta_bar = 0,
 *   rhat = 2 (1 - rho_ref) / sqrt(6) + eps  (v = 1, eps added: reading 6).
 * Returns |APS|.
 */
int or_pst_update(int N, const double *rho, const double *delta, double rho_ref, const double r_prev[6],
                  double beta, double eps, double delta_bar[6], double *rho_tilde, double r_out[6])
{
    double sw = 0.0, swr = 0.0, swd[6] = {0, 0, 0, 0, 0, 0};
    int n_aps = 0;
    for (int i = 0; i < N; ++i) {
        if (rho[i] > rho_ref) {
            double w = rho[i] - rho_ref;
            ++n_aps;
            sw += w;
            swr += w * rho[i];
            for (int d = 0; d < 6; ++d)
                swd[d] += w * delta[6 * (size_t)i + d];
        }
    }
    double rhat[6];
    if (n_aps == 0) {
        for (int d = 0; d < 6; ++d) {
            delta_bar[d] = 0.0;
            rhat[d] = 2.0 * (1.0 - rho_ref) / sqrt(6.0) + eps;
        }
        *rho_tilde = rho_ref;
    } else {
        double nv2 = 0.0;
        for (int d = 0; d < 6; ++d) {
            delta_bar[d] = swd[d] / sw;
            nv2 += delta_bar[d] * delta_bar[d];
        }
        *rho_tilde = swr / sw;
        double nv = sqrt(nv2);
        for (int d = 0; d < 6; ++d) {
            double dir = (nv < 1e-12) ? 1.0 / sqrt(6.0) : fabs(delta_bar[d]) / nv;
            rhat[d] = (1.0 - *rho_tilde) * dir + eps;
        }
    }
    for (int d = 0; d < 6; ++d)
        r_out[d] = beta * r_prev[d] + (1.0 - beta) * rhat[d];
    return n_aps;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1: per-frame pose optimisation by PFO with PST.                  */
/* ------------------------------------------------------------------------- */

#define OR_TRACE_STRIDE 40
/* trace row per iteration k (doubles):
 *  0 k, 1 |O_k|, 2 |APS|, 3 rho_ref, 4 rho_tilde, 5 rho_max, 6 argmax,
 *  7..13 s*_k (pose), 14..19 r_k, 20..25 delta_bar, 26 min_i |rho_i - rho_ref|
 *  over the APS candidates, 27 min overlap rounding margin (px), 28 stop reason
 *  (0 running, 1 empty twice, 2 small step, 3 k_max, 4 empty overlap),
 *  29 second-largest rho, 30 level, 31 particles scored, 32 corner case of
 *  Sec. 4 "PST update" (0 none, 1 no TSDF yet, 2 empty APS), 33 valid samples
 *  summed over all particles, 34 consecutive empty APS after this iteration,
 *  35 points whose overlap decision lies within OR_TIE_PX of its threshold,
 *  36 candidates whose fitness lies within OR_TIE_RHO of the APS threshold,
 *  37 sensitivity of delta_bar to the weights: sum_APS max_d |delta_i,d -
 *  delta_bar_d| / sum_APS w_i (so an error e in every weight moves delta_bar by
 *  at most e times this), 38 max_d |delta_bar_d| (the small-step statistic),
 *  39 the same sensitivity for independent weight errors: sqrt(sum_APS max_d
 *  |delta_i,d - delta_bar_d|^2) / sum_APS w_i                                */
#define OR_TIE_PX 1e-3
#define OR_TIE_RHO 1e-5

/* State of Algorithm 1 between two iterations (doubles):
 *  0..6 c_{k-1} = s*_{k-1}, 7..12 r_{k-1}, 13 rho(s*_{k-1}) by Eq. wafit (the
 *  carried APS threshold), 14 consecutive empty APS so far, 15 k, the iteration
 *  about to run (1-based). */
#define OR_STATE_LEN 16

/* Fitness of particles [0, Nl) of the template about centre c with axes r:
 * delta_i = r . omega_i, pose_i = c (+) delta_i, rho_i and the valid-sample
 * count by or_fitness over the points with mask != 0.  Particles are
 * independent, so the work may be split over threads (each thread runs the
 * plain per-particle loop on its own particles); the results do not depend on
 * the thread count. */
typedef struct {
    const double *F;
    const int *dim;
    double voxel;
    const double *origin;
    const double *pts;
    const int *mask;
    int M;
    const double *c, *r;
    const float *omega;
    int N, i0, i1;
    double tau;
    int flags;
    double *rho, *delta;
    int *nval;
} or_fit_job;

static void *or_fit_worker(void *arg)
{
    or_fit_job *j = (or_fit_job *)arg;
    for (int i = j->i0; i < j->i1; ++i) {
        double pose[7], S;
        int n, nO;
        for (int d = 0; d < 6; ++d)
            j->delta[6 * (size_t)i + d] = j->r[d] * j->omega[(size_t)d * j->N + i];
        or_compose_offset(j->c, j->delta + 6 * (size_t)i, j->flags, pose);
        or_fitness(j->F, j->dim, j->voxel, j->origin, j->pts, j->mask, j->M, pose, j->tau, j->flags, &S, &n, &nO,
                   &j->rho[i]);
        j->nval[i] = n;
    }
    return NULL;
}

/* rho[i], nval[i] and delta[6i..6i+5] for i in [i_begin, i_end). */
void or_fitness_particles(const double *F, const int dim[3], double voxel, const double origin[3], const double *pts,
                          const int *mask, int M, const double c[7], const double r[6], const float *omega, int N,
                          int i_begin, int i_end, double tau, int flags, int nthreads, double *rho, int *nval,
                          double *delta)
{
    int nt = nthreads < 1 ? 1 : nthreads;
    int count = i_end - i_begin;
    if (count <= 0)
        return;
    if (nt > count)
        nt = count;
    or_fit_job jobs[256];
    pthread_t th[256];
    if (nt > 256)
        nt = 256;
    for (int t = 0; t < nt; ++t) {
        or_fit_job *j = &jobs[t];
        j->F = F;
        j->dim = dim;
        j->voxel = voxel;
        j->origin = origin;
        j->pts = pts;
        j->mask = mask;
        j->M = M;
        j->c = c;
        j->r = r;
        j->omega = omega;
        j->N = N;
        j->i0 = i_begin + (int)((long long)count * t / nt);
        j->i1 = i_begin + (int)((long long)count * (t + 1) / nt);
        j->tau = tau;
        j->flags = flags;
        j->rho = rho;
        j->delta = delta;
        j->nval = nval;
    }
    if (nt == 1) {
        or_fit_worker(&jobs[0]);
        return;
    }
    int started = 0;
    for (int t = 1; t < nt; ++t) {
        if (pthread_create(&th[t], NULL, or_fit_worker, &jobs[t]) != 0)
            break;
        started = t;
    }
    or_fit_worker(&jobs[0]);
    for (int t = started + 1; t < nt; ++t) /* threads that could not start run here */
        or_fit_worker(&jobs[t]);
    for (int t = 1; t <= started; ++t)
        pthread_join(th[t], NULL);
}

/*
 * One iteration k of Algorithm 1 (state layout above), on Nl <= N particles
 * (the first Nl rows of the template omega, 6 x N structure of arrays, row 0 =
 * origin) and M points (or_unproject output):
 *  1. O_k with s*_{k-1} = c_{k-1} (Eq. validness; all valid points without OVERLAP)
 *  2. fitness of every particle c_{k-1} (+) (r_{k-1} . omega_i) (Eq. normallh)
 *  3. APS threshold rho(s*_{k-1}): particle 0 when k = 1, RHO_REF_CENTER or
 *     centre_ref != 0, else the carried Eq. wafit value (readings 7-8)
 *  4. APS = candidates strictly above it (particles 1..Nl-1, plus particle 0
 *     with APS_WITH_CENTRE); or_pst_update: Eq. ebs, wafit, rsdir, rsinter,
 *     momentum, and the empty-APS corner case of Sec. 4
 *  5. first corner case of Sec. 4 ("TSDF has not been built"): when no
 *     particle has a single valid TSDF sample the likelihood cannot be
 *     evaluated; the iteration then keeps s*, uses rho = 0.5 and the isotropic
 *     attractor v = 1, r_hat = 0.5 v + eps, and counts as an empty APS
 *  6. stop rules of Sec. 4: two consecutive empty APS, a step below stop_eps
 *     in all six dimensions, or k = k_max; an empty O_k stops with code 4.
 * Updates `state` (unless O_k is empty) and writes the trace row tr (may be
 * NULL).  Returns the stop code (0 = continue), or OR_ERR_ARG.
 */
int or_pfo_step(const double *F, const int dim[3], double voxel, const double origin[3], const double *pts, int M,
                int Nl, const float *prev_depth, int W, int H, double fx, double fy, double cx, double cy,
                double z_min, double z_max, const double pose_prev[7], const float *omega, int N, double tau,
                double beta, double eps, double stop_eps, int k_max, int flags, int centre_ref, int nthreads,
                double *state, double *tr)
{
    if (Nl < 1 || Nl > N || M < 0)
        return OR_ERR_ARG;
    for (int d = 0; d < 6; ++d)
        if (omega[(size_t)d * N] != 0.0f)
            return OR_ERR_ARG; /* row 0 must be the origin (reading 8) */
    double c[7], r[6];
    memcpy(c, state, sizeof c);
    memcpy(r, state + 7, sizeof r);
    const double rho_carry = state[13];
    int empty_run = (int)state[14];
    const int k = (int)state[15];
    int *mask = (int *)malloc(sizeof(int) * (size_t)(M > 0 ? M : 1));
    double *margin = (double *)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1));
    double *rho = (double *)malloc(sizeof(double) * (size_t)Nl);
    int *nval = (int *)malloc(sizeof(int) * (size_t)Nl);
    double *delta = (double *)malloc(sizeof(double) * 6 * (size_t)Nl);
    /* 1. O_k */
    int nO = 0, fragile_px = 0;
    double min_margin = INFINITY;
    if (flags & OR_OVERLAP) {
        nO = or_overlap(pts, M, prev_depth, W, H, fx, fy, cx, cy, z_min, z_max, c, pose_prev,
                        (flags & OR_CELL_MARGIN) ? sqrt(3.0) * voxel : 0.0, mask, margin);
        for (int j = 0; j < M; ++j)
            if (pts[4 * (size_t)j + 3] != 0.0) {
                if (margin[j] < min_margin)
                    min_margin = margin[j];
                if (margin[j] < OR_TIE_PX)
                    ++fragile_px;
            }
    } else {
        for (int j = 0; j < M; ++j) {
            mask[j] = pts[4 * (size_t)j + 3] != 0.0;
            nO += mask[j];
        }
    }
    int stop = 0;
    if (nO == 0) {
        stop = 4;
        if (tr) {
            memset(tr, 0, sizeof(double) * OR_TRACE_STRIDE);
            tr[0] = k;
            tr[28] = 4;
            tr[31] = Nl;
            tr[34] = empty_run;
        }
    } else {
        /* 2. fitness of every particle */
        or_fitness_particles(F, dim, voxel, origin, pts, mask, M, c, r, omega, N, 0, Nl, tau, flags, nthreads, rho,
                             nval, delta);
        double rho_max = -1.0, rho_2nd = -1.0, valid = 0.0;
        int argmax = 0;
        for (int i = 0; i < Nl; ++i) {
            valid += (double)nval[i];
            if (rho[i] > rho_max) {
                rho_2nd = rho_max;
                rho_max = rho[i];
                argmax = i;
            } else if (rho[i] > rho_2nd) {
                rho_2nd = rho[i];
            }
        }
        /* 3. threshold */
        const double rho_ref = (k == 1 || (flags & OR_RHO_REF_CENTER) || centre_ref) ? rho[0] : rho_carry;
        /* 4. APS over the candidates: particles 1..Nl-1 (particle 0 is s*_{k-1} itself) */
        const int first = (flags & OR_APS_WITH_CENTRE) ? 0 : 1;
        double min_gap = INFINITY;
        int ties = 0;
        for (int i = first; i < Nl; ++i) {
            double g = fabs(rho[i] - rho_ref);
            if (g < min_gap)
                min_gap = g;
            if (g < OR_TIE_RHO)
                ++ties;
        }
        double dbar[6], rho_tilde, r_new[6];
        int n_aps, corner;
        if (valid == 0.0) {
            /* 5. no TSDF sample anywhere: rho = 0.5, v = 1 (not normalised) */
            n_aps = 0;
            corner = 1;
            rho_tilde = 0.5;
            for (int d = 0; d < 6; ++d) {
                dbar[d] = 0.0;
                r_new[d] = beta * r[d] + (1.0 - beta) * (0.5 * 1.0 + eps);
            }
        } else {
            n_aps = or_pst_update(Nl - first, rho + first, delta + 6 * (size_t)first, rho_ref, r, beta, eps, dbar,
                                  &rho_tilde, r_new);
            corner = n_aps == 0 ? 2 : 0;
        }
        double sens = 0.0, sens2 = 0.0;
        if (n_aps > 0) {
            double sw = 0.0;
            for (int i = first; i < Nl; ++i)
                if (rho[i] > rho_ref) {
                    double dev = 0.0;
                    for (int d = 0; d < 6; ++d)
                        dev = fmax(dev, fabs(delta[6 * (size_t)i + d] - dbar[d]));
                    sens += dev;
                    sens2 += dev * dev;
                    sw += rho[i] - rho_ref;
                }
            sens /= sw;
            sens2 = sqrt(sens2) / sw;
        }
        double s_new[7];
        if (n_aps > 0) {
            or_compose_offset(c, dbar, flags, s_new);
            empty_run = 0;
        } else {
            memcpy(s_new, c, sizeof s_new);
            ++empty_run;
        }
        /* 6. stop rules */
        double step = 0.0;
        for (int d = 0; d < 6; ++d)
            step = fmax(step, fabs(dbar[d]));
        if (empty_run >= 2)
            stop = 1;
        else if (n_aps > 0 && step < stop_eps)
            stop = 2;
        else if (k == k_max)
            stop = 3;
        memcpy(state, s_new, sizeof(double) * 7);
        memcpy(state + 7, r_new, sizeof(double) * 6);
        state[13] = rho_tilde;
        state[14] = empty_run;
        if (tr) {
            tr[0] = k;
            tr[1] = nO;
            tr[2] = n_aps;
            tr[3] = rho_ref;
            tr[4] = rho_tilde;
            tr[5] = rho_max;
            tr[6] = argmax;
            for (int a = 0; a < 7; ++a)
                tr[7 + a] = s_new[a];
            for (int d = 0; d < 6; ++d) {
                tr[14 + d] = r_new[d];
                tr[20 + d] = dbar[d];
            }
            tr[26] = min_gap;
            tr[27] = min_margin;
            tr[28] = stop;
            tr[29] = rho_2nd;
            tr[31] = Nl;
            tr[32] = corner;
            tr[33] = valid;
            tr[34] = empty_run;
            tr[35] = fragile_px;
            tr[36] = ties;
            tr[37] = sens;
            tr[38] = step;
            tr[39] = sens2;
        }
    }
    if (tr)
        tr[35] = fragile_px;
    state[15] = k + 1;
    free(mask);
    free(margin);
    free(rho);
    free(nval);
    free(delta);
    return stop;
}

/*
 * Algorithm 1 with L (particle count, depth stride) levels used in turn (Sec. 4
 * "Multi-resolution PST"; L = 1 is the plain algorithm): iteration k runs
 * or_pfo_step on level l = (k - 1) mod L, i.e. the first level_n[l] rows of the
 * template and the points level_pts[l] (level_M[l] of them).  With L > 1 the
 * fitness of consecutive iterations is normalised over different point sets,
 * so the APS threshold is the centre particle's fitness in the current
 * iteration (reading 17).  The PST starts at c0 with axes r0 (Sec. 4 "PST
 * initialization").  Outputs: the final pose s*, the axis lengths after
 * iteration 1 (r_1, handed to the next frame; r0 if O_1 is empty), the trace
 * (k_max rows of OR_TRACE_STRIDE, may be NULL) and the iteration count.
 * Returns 0, OR_ERR_EMPTY if some |O_k| = 0 (the pose then stays s*_{k-1}), or
 * OR_ERR_ARG.
 */
int or_pfo_frame_sched_mt(const double *F, const int dim[3], double voxel, const double origin[3], int L,
                          const int *level_n, const double *const *level_pts, const int *level_M,
                          const float *prev_depth, int W, int H, double fx, double fy, double cx, double cy,
                          double z_min, double z_max, const double pose_prev[7], const double c0[7],
                          const double r0[6], const float *omega, int N, double tau, double beta, double eps,
                          double stop_eps, int k_max, int flags, int nthreads, double pose_out[7], double r1_out[6],
                          double *trace, int *iters_out)
{
    if (L < 1 || N < 1 || k_max < 1)
        return OR_ERR_ARG;
    for (int l = 0; l < L; ++l)
        if (level_n[l] < 1 || level_n[l] > N)
            return OR_ERR_ARG;
    double state[OR_STATE_LEN];
    memcpy(state, c0, sizeof(double) * 7);
    memcpy(state + 7, r0, sizeof(double) * 6);
    state[13] = 0.0;
    state[14] = 0.0;
    state[15] = 1.0;
    memcpy(r1_out, r0, sizeof(double) * 6);
    int status = OR_OK, k;
    for (k = 1; k <= k_max; ++k) {
        const int l = (k - 1) % L;
        double *tr = trace ? trace + OR_TRACE_STRIDE * (size_t)(k - 1) : NULL;
        int stop = or_pfo_step(F, dim, voxel, origin, level_pts[l], level_M[l], level_n[l], prev_depth, W, H, fx,
                               fy, cx, cy, z_min, z_max, pose_prev, omega, N, tau, beta, eps, stop_eps, k_max, flags,
                               L > 1, nthreads, state, tr);
        if (stop < 0)
            return stop;
        if (tr)
            tr[30] = l;
        if (stop == 4) {
            status = OR_ERR_EMPTY;
            break;
        }
        if (k == 1)
            memcpy(r1_out, state + 7, sizeof(double) * 6);
        if (stop)
            break;
    }
    if (k > k_max)
        k = k_max;
    memcpy(pose_out, state, sizeof(double) * 7);
    *iters_out = k;
    return status;
}

/* Single-threaded multi-resolution frame (see or_pfo_frame_sched_mt). */
int or_pfo_frame_sched(const double *F, const int dim[3], double voxel, const double origin[3], int L,
                       const int *level_n, const double *const *level_pts, const int *level_M,
                       const float *prev_depth, int W, int H, double fx, double fy, double cx, double cy,
                       double z_min, double z_max, const double pose_prev[7], const double c0[7], const double r0[6],
                       const float *omega, int N, double tau, double beta, double eps, double stop_eps, int k_max,
                       int flags, double pose_out[7], double r1_out[6], double *trace, int *iters_out)
{
    return or_pfo_frame_sched_mt(F, dim, voxel, origin, L, level_n, level_pts, level_M, prev_depth, W, H, fx, fy, cx,
                                 cy, z_min, z_max, pose_prev, c0, r0, omega, N, tau, beta, eps, stop_eps, k_max,
                                 flags, 1, pose_out, r1_out, trace, iters_out);
}

/*
 * Algorithm 1 for one frame on one point set and the whole template:
 * or_pfo_frame_sched_mt with a single level (see there for inputs, outputs and
 * the readings).  nthreads splits the per-particle fitness loop only.
 */
int or_pfo_frame_mt(const double *F, const int dim[3], double voxel, const double origin[3], const double *pts, int M,
                    const float *prev_depth, int W, int H, double fx, double fy, double cx, double cy, double z_min,
                    double z_max, const double pose_prev[7], const double c0[7], const double r0[6],
                    const float *omega, int N, double tau, double beta, double eps, double stop_eps, int k_max,
                    int flags, int nthreads, double pose_out[7], double r1_out[6], double *trace, int *iters_out)
{
    const int level_n[1] = {N}, level_M[1] = {M};
    const double *level_pts[1] = {pts};
    return or_pfo_frame_sched_mt(F, dim, voxel, origin, 1, level_n, level_pts, level_M, prev_depth, W, H, fx, fy, cx,
                                 cy, z_min, z_max, pose_prev, c0, r0, omega, N, tau, beta, eps, stop_eps, k_max,
                                 flags, nthreads, pose_out, r1_out, trace, iters_out);
}

int or_pfo_frame(const double *F, const int dim[3], double voxel, const double origin[3], const double *pts, int M,
                 const float *prev_depth, int W, int H, double fx, double fy, double cx, double cy, double z_min,
                 double z_max, const double pose_prev[7], const double c0[7], const double r0[6],
                 const float *omega, int N, double tau, double beta, double eps, double stop_eps, int k_max,
                 int flags, double pose_out[7], double r1_out[6], double *trace, int *iters_out)
{
    return or_pfo_frame_mt(F, dim, voxel, origin, pts, M, prev_depth, W, H, fx, fy, cx, cy, z_min, z_max, pose_prev,
                           c0, r0, omega, N, tau, beta, eps, stop_eps, k_max, flags, 1, pose_out, r1_out, trace,
                           iters_out);
}

/* ------------------------------------------------------------------------- */
/* Volumetric fusion (Sec. 3 overview: Curless-Levoy / KinectFusion).         */
/* ------------------------------------------------------------------------- */

/* Storage rounding of a fused value: 0 none, 1 float32, 2 float16,
 * 3 int16 code round(F * 32767) (reading 14). */
double or_quantize(double F, int qmode)
{
    switch (qmode) {
    case 1:
        return (double)(float)F;
    case 2:
        return (double)(_Float16)F;
    case 3: {
        double code = nearbyint(F * 32767.0);
        if (code > 32767.0)
            code = 32767.0;
        if (code < -32767.0)
            code = -32767.0;
        return code / 32767.0;
    }
    default:
        return F;
    }
}

/*
 * Projective TSDF update of every voxel (reading 14): the voxel centre is
 * moved into the camera with the inverse pose and projected to the nearest
 * pixel; with a valid depth D there, sdf = D - z_cam; voxels with sdf < -trunc
 * are untouched; otherwise f = min(1, sdf / trunc) and
 *   F <- (W F + f) / (W + 1),   W <- min(W + 1, w_max).
 * F is rounded to the storage type after every update (qmode).  Slices z in
 * [z0, z1) only (the whole volume: 0, dim[2]).
 */
typedef struct {
    double *F;
    int *Wt;
    const int *dim;
    double voxel;
    const double *origin;
    double trunc;
    int w_max, qmode;
    const float *depth;
    int W, H;
    double fx, fy, cx, cy, z_min, z_max;
    const double *pose;
    int z0, z1;
} or_integrate_job;

static void *or_integrate_slices(void *arg)
{
    const or_integrate_job *j = (const or_integrate_job *)arg;
    const int *dim = j->dim;
    double R[9];
    or_quat_to_rot(j->pose, R);
    for (int k = j->z0; k < j->z1; ++k)
        for (int jy = 0; jy < dim[1]; ++jy)
            for (int i = 0; i < dim[0]; ++i) {
                double pw[3] = {j->origin[0] + j->voxel * (i + 0.5), j->origin[1] + j->voxel * (jy + 0.5),
                                j->origin[2] + j->voxel * (k + 0.5)};
                double pc[3];
                apply_pose_inverse(R, j->pose + 4, pw, pc);
                if (!(pc[2] > 0.0))
                    continue;
                double u = floor(j->fx * pc[0] / pc[2] + j->cx + 0.5);
                double v = floor(j->fy * pc[1] / pc[2] + j->cy + 0.5);
                if (u < 0.0 || u >= (double)j->W || v < 0.0 || v >= (double)j->H)
                    continue;
                double D = j->depth[(size_t)v * j->W + (size_t)u];
                if (!(D > j->z_min && D <= j->z_max))
                    continue;
                double sdf = D - pc[2];
                if (sdf < -j->trunc)
                    continue;
                double f = sdf / j->trunc;
                if (f > 1.0)
                    f = 1.0;
                size_t idx = (size_t)i + (size_t)dim[0] * ((size_t)jy + (size_t)dim[1] * (size_t)k);
                int w_old = j->Wt[idx];
                double F_old = isnan(j->F[idx]) ? 0.0 : j->F[idx];
                if (isnan(j->F[idx]))
                    w_old = 0;
                double F_new = ((double)w_old * F_old + f) / (double)(w_old + 1);
                j->F[idx] = or_quantize(F_new, j->qmode);
                j->Wt[idx] = (w_old + 1 < j->w_max) ? w_old + 1 : j->w_max;
            }
    return NULL;
}

/* The update of every voxel, the z slices split over nthreads threads (each
 * voxel is updated by the same plain code whatever the split). */
void or_tsdf_integrate_mt(double *F, int *Wt, const int dim[3], double voxel, const double origin[3], double trunc,
                          int w_max, int qmode, const float *depth, int W, int H, double fx, double fy, double cx,
                          double cy, double z_min, double z_max, const double pose[7], int nthreads)
{
    int nt = nthreads < 1 ? 1 : (nthreads > 256 ? 256 : nthreads);
    if (nt > dim[2])
        nt = dim[2];
    or_integrate_job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < nt; ++t) {
        or_integrate_job *j = &jobs[t];
        j->F = F;
        j->Wt = Wt;
        j->dim = dim;
        j->voxel = voxel;
        j->origin = origin;
        j->trunc = trunc;
        j->w_max = w_max;
        j->qmode = qmode;
        j->depth = depth;
        j->W = W;
        j->H = H;
        j->fx = fx;
        j->fy = fy;
        j->cx = cx;
        j->cy = cy;
        j->z_min = z_min;
        j->z_max = z_max;
        j->pose = pose;
        j->z0 = (int)((long long)dim[2] * t / nt);
        j->z1 = (int)((long long)dim[2] * (t + 1) / nt);
    }
    int started = 0;
    for (int t = 1; t < nt; ++t) {
        if (pthread_create(&th[t], NULL, or_integrate_slices, &jobs[t]) != 0)
            break;
        started = t;
    }
    or_integrate_slices(&jobs[0]);
    for (int t = started + 1; t < nt; ++t)
        or_integrate_slices(&jobs[t]);
    for (int t = 1; t <= started; ++t)
        pthread_join(th[t], NULL);
}

void or_tsdf_integrate(double *F, int *Wt, const int dim[3], double voxel, const double origin[3], double trunc,
                       int w_max, int qmode, const float *depth, int W, int H, double fx, double fy, double cx,
                       double cy, double z_min, double z_max, const double pose[7])
{
    or_tsdf_integrate_mt(F, Wt, dim, voxel, origin, trunc, w_max, qmode, depth, W, H, fx, fy, cx, cy, z_min, z_max,
                         pose, 1);
}

/* ------------------------------------------------------------------------- */
/* PST pre-sampling (Sec. 4 "PST pre-sampling").                              */
/* ------------------------------------------------------------------------- */

/* Philox4x32-10 counter-based generator, from its published definition
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC 2011): ten rounds of two 32x32->64 multiplies with the round constants
 * 0xD2511F53 / 0xCD9E8D57 and a Weyl key schedule 0x9E3779B9 / 0xBB67AE85. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/*
 * Uniform PST in the closed unit 6D ball by rejection from the cube.
 * Row 0 is the origin (reading 8).  Particle i >= 1, attempt a: key = seed,
 * counters (i, a, 0, 0) and (i, a, 1, 0) give eight 32-bit words; the first
 * six give m_d = word >> 8 and the coordinate (2 m_d + 1 - 2^24) / 2^24, which
 * is exact in float32.  The candidate is accepted iff
 * sum_d (2 m_d + 1 - 2^24)^2 <= 2^48, an exact integer test.
 * out is 6 x N, structure of arrays (out[d*N + i]).  Returns 0 or -1.
 */
int or_pst_uniform(int N, uint64_t seed, float *out)
{
    if (N < 1)
        return OR_ERR_ARG;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int d = 0; d < 6; ++d)
        out[(size_t)d * N] = 0.0f;
    for (int i = 1; i < N; ++i) {
        int ok = 0;
        for (uint32_t a = 0; a < 100000u && !ok; ++a) {
            uint32_t c0[4] = {(uint32_t)i, a, 0u, 0u}, c1[4] = {(uint32_t)i, a, 1u, 0u};
            uint32_t w[8];
            or_philox4x32_10(c0, key, w);
            or_philox4x32_10(c1, key, w + 4);
            int64_t v[6];
            int64_t s2 = 0;
            for (int d = 0; d < 6; ++d) {
                v[d] = 2 * (int64_t)(w[d] >> 8) + 1 - ((int64_t)1 << 24);
                s2 += v[d] * v[d];
            }
            if (s2 <= ((int64_t)1 << 48)) {
                for (int d = 0; d < 6; ++d)
                    out[(size_t)d * N + i] = (float)((double)v[d] / 16777216.0);
                ok = 1;
            }
        }
        if (!ok)
            return OR_ERR_ARG;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* Evaluation: ATE (Sec. 5.1, mean after rigid alignment) and TE (Eq. te).    */
/* ------------------------------------------------------------------------- */

/* Largest-eigenvalue eigenvector of a symmetric 4x4 matrix by cyclic Jacobi
 * rotations (Golub & Van Loan, Sec. 8.5). */
static void sym4_top_eigvec(double A[4][4], double vec[4])
{
    double V[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 4; ++q)
                off += A[p][q] * A[p][q];
        if (off < 1e-30)
            break;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 4; ++q) {
                if (fabs(A[p][q]) < 1e-300)
                    continue;
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 4; ++k) { /* A <- J^T A J */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 4; ++k) {
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 4; ++k) {
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    int best = 0;
    for (int i = 1; i < 4; ++i)
        if (A[i][i] > A[best][best])
            best = i;
    for (int k = 0; k < 4; ++k)
        vec[k] = V[k][best];
}

/*
 * ATE over T frames: the estimated camera positions are aligned to the
 * ground truth by the rotation + translation that minimises the squared
 * error (Horn 1987, closed form through the unit quaternion of the largest
 * eigenvector of the 4x4 matrix N), then the mean and RMS of the position
 * errors are returned (reading 15).  est/gt are T x 7 poses.
 */
void or_ate(const double *est, const double *gt, int T, double *mean_out, double *rmse_out)
{
    double ce[3] = {0, 0, 0}, cg[3] = {0, 0, 0};
    for (int f = 0; f < T; ++f)
        for (int a = 0; a < 3; ++a) {
            ce[a] += est[7 * (size_t)f + 4 + a] / T;
            cg[a] += gt[7 * (size_t)f + 4 + a] / T;
        }
    double S[3][3] = {{0}};
    for (int f = 0; f < T; ++f)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                S[a][b] += (est[7 * (size_t)f + 4 + a] - ce[a]) * (gt[7 * (size_t)f + 4 + b] - cg[b]);
    double Nm[4][4] = {
        {S[0][0] + S[1][1] + S[2][2], S[1][2] - S[2][1], S[2][0] - S[0][2], S[0][1] - S[1][0]},
        {S[1][2] - S[2][1], S[0][0] - S[1][1] - S[2][2], S[0][1] + S[1][0], S[2][0] + S[0][2]},
        {S[2][0] - S[0][2], S[0][1] + S[1][0], -S[0][0] + S[1][1] - S[2][2], S[1][2] + S[2][1]},
        {S[0][1] - S[1][0], S[2][0] + S[0][2], S[1][2] + S[2][1], -S[0][0] - S[1][1] + S[2][2]}};
    double q[4], R[9];
    sym4_top_eigvec(Nm, q);
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int a = 0; a < 4; ++a)
        q[a] /= nq;
    or_quat_to_rot(q, R);
    double sum = 0.0, sum2 = 0.0;
    for (int f = 0; f < T; ++f) {
        double d[3], e[3];
        for (int a = 0; a < 3; ++a)
            d[a] = est[7 * (size_t)f + 4 + a] - ce[a];
        for (int a = 0; a < 3; ++a)
            e[a] = R[3 * a + 0] * d[0] + R[3 * a + 1] * d[1] + R[3 * a + 2] * d[2] + cg[a] -
                   gt[7 * (size_t)f + 4 + a];
        double n2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
        sum += sqrt(n2);
        sum2 += n2;
    }
    *mean_out = sum / T;
    *rmse_out = sqrt(sum2 / T);
}

/* TE of one frame (Eq. te): the norm of the translation of T_G^-1 T_E. */
double or_te(const double est[7], const double gt[7])
{
    double Rg[9], d[3], y[3];
    or_quat_to_rot(gt, Rg);
    for (int a = 0; a < 3; ++a)
        d[a] = est[4 + a];
    apply_pose_inverse(Rg, gt + 4, d, y);
    return sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
}

/* ------------------------------------------------------------------------- */
/* Brute force for tiny inputs: the best pose on a regular 6D grid of offsets  */
/* about c, steps^6 candidates spanning [-half[d], +half[d]] per dimension.    */
/* Used by the tests to bound Algorithm 1 from below on small problems.        */
/* ------------------------------------------------------------------------- */
double or_grid_search(const double *F, const int dim[3], double voxel, const double origin[3], const double *pts,
                      const int *in_set, int M, const double c[7], const double half[6], int steps, double tau,
                      int flags, double best_pose[7])
{
    double best = -1.0;
    int idx[6];
    long total = 1;
    for (int d = 0; d < 6; ++d)
        total *= steps;
    for (long g = 0; g < total; ++g) {
        long r = g;
        for (int d = 0; d < 6; ++d) {
            idx[d] = (int)(r % steps);
            r /= steps;
        }
        double delta[6], pose[7], S, rho;
        int n, nO;
        for (int d = 0; d < 6; ++d)
            delta[d] = steps > 1 ? -half[d] + 2.0 * half[d] * idx[d] / (steps - 1) : 0.0;
        or_compose_offset(c, delta, flags, pose);
        or_fitness(F, dim, voxel, origin, pts, in_set, M, pose, tau, flags, &S, &n, &nO, &rho);
        if (rho > best) {
            best = rho;
            memcpy(best_pose, pose, sizeof(double) * 7);
        }
    }
    return best;
}

/* ------------------------------------------------------------------------- */
/* Decisions that FP32 and FP64 may legitimately take differently.            */
/* ------------------------------------------------------------------------- */

/*
 * Same sum as or_fitness, plus the number of points whose sample validity (or,
 * in NEAREST mode, whose chosen voxel) changes when the sample position moves
 * by +-delta_g voxels along any axis.  Each such point can move S by at most 1
 * (psi^2 and |psi| lie in [0, 1]), which bounds the admissible gap between an
 * FP32 evaluation and this one.
 */
void or_fitness_fragile(const double *F, const int dim[3], double voxel, const double origin[3], const double *pts,
                        const int *in_set, int M, const double pose[7], double tau, int flags, double delta_g,
                        double *S_out, int *n_out, int *nO_out, double *rho_out, int *fragile_out)
{
    double R[9];
    or_quat_to_rot(pose, R);
    int fragile = 0;
    for (int j = 0; j < M; ++j) {
        if (!in_set[j])
            continue;
        double pg[3], psi;
        apply_pose(R, pose + 4, pts + 4 * (size_t)j, pg);
        int base = or_tsdf_sample(F, dim, voxel, origin, pg, flags, &psi);
        int moved = 0;
        for (int a = 0; a < 3 && !moved; ++a)
            for (int s = -1; s <= 1; s += 2) {
                double q[3] = {pg[0], pg[1], pg[2]};
                q[a] += s * delta_g * voxel;
                double g0 = (pg[a] - origin[a]) / voxel - 0.5, g1 = (q[a] - origin[a]) / voxel - 0.5;
                double psi2;
                int v2 = or_tsdf_sample(F, dim, voxel, origin, q, flags, &psi2);
                int cell_change = (flags & OR_NEAREST) ? floor(g0 + 0.5) != floor(g1 + 0.5) : 0;
                if (v2 != base || (base && cell_change)) {
                    moved = 1;
                    break;
                }
            }
        fragile += moved;
    }
    or_fitness(F, dim, voxel, origin, pts, in_set, M, pose, tau, flags, S_out, n_out, nO_out, rho_out);
    *fragile_out = fragile;
}

/*
 * Ambiguity map of one projective fusion step: ambig[v] = 1 where a decision of
 * or_tsdf_integrate for voxel v lies within tol of its threshold (pixel
 * rounding in u or v, the image border, the valid-depth range, sdf >= -trunc,
 * z > 0), so that an FP32 implementation may decide it the other way.
 */
void or_tsdf_integrate_ambiguity(const int dim[3], double voxel, const double origin[3], double trunc,
                                 const float *depth, int W, int H, double fx, double fy, double cx, double cy,
                                 double z_min, double z_max, const double pose[7], double tol, int *ambig)
{
    double R[9];
    or_quat_to_rot(pose, R);
    for (int k = 0; k < dim[2]; ++k)
        for (int j = 0; j < dim[1]; ++j)
            for (int i = 0; i < dim[0]; ++i) {
                size_t idx = (size_t)i + (size_t)dim[0] * ((size_t)j + (size_t)dim[1] * (size_t)k);
                double pw[3] = {origin[0] + voxel * (i + 0.5), origin[1] + voxel * (j + 0.5),
                                origin[2] + voxel * (k + 0.5)};
                double pc[3];
                apply_pose_inverse(R, pose + 4, pw, pc);
                int a = 0;
                if (fabs(pc[2]) < tol)
                    a = 1;
                if (pc[2] > 0.0) {
                    double uc = fx * pc[0] / pc[2] + cx + 0.5, vc = fy * pc[1] / pc[2] + cy + 0.5;
                    double du = fabs(uc - nearbyint(uc)), dv = fabs(vc - nearbyint(vc));
                    if (du < tol || dv < tol)
                        a = 1;
                    double u = floor(uc), v = floor(vc);
                    if (u >= 0.0 && u < (double)W && v >= 0.0 && v < (double)H) {
                        double D = depth[(size_t)v * W + (size_t)u];
                        if (fabs(D - z_min) < tol || fabs(D - z_max) < tol)
                            a = 1;
                        if (D > z_min && D <= z_max && fabs((D - pc[2]) + trunc) < tol)
                            a = 1;
                    }
                }
                ambig[idx] = a;
            }
}
