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
 *
 * Functions whose result has no independent pin say so in their comment;
 * every other function is pinned by tests/test_oracle_*.py.
 */
#include <math.h>
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
 *  7..13 s*_k (pose), 14..19 r_k, 20..25 delta_bar, 26 min_i |rho_i - rho_ref|,
 *  27 min overlap rounding margin, 28 stop reason (0 running, 1 empty twice,
 *  2 small step, 3 k_max, 4 empty overlap), 29 second-largest rho            */

/*
 * Inputs: the volume, the frame's points (or_unproject output, M of them), the
 * previous frame's full-resolution depth and final pose (for Eq. validness),
 * the initial centre c0 and axis lengths r0 (Sec. 4 "PST initialization"),
 * the template omega (6 x N, structure of arrays, row 0 = origin), the
 * parameters.  Outputs: final pose s*, the axis lengths after iteration 1
 * (r_1, handed to the next frame), the trace, the number of iterations.
 * Loop order follows Algorithm 1 with the readings: iteration k evaluates the
 * PST centred at c_{k-1} with axes r_{k-1}; rho_ref = rho of particle 0 at
 * k = 1 (and with RHO_REF_CENTER), else the carried Eq. wafit value; the APS
 * is drawn from particles 1..N-1 (particle 0 is s*_{k-1} itself); stop on
 * two consecutive empty APS, a step below stop_eps in all six dimensions, or
 * k = k_max (Sec. 4 "Convergence criteria").
 * Returns 0, or OR_ERR_EMPTY if |O_k| = 0 (the pose then stays s*_{k-1}).
 */
int or_pfo_frame(const double *F, const int dim[3], double voxel, const double origin[3], const double *pts, int M,
                 const float *prev_depth, int W, int H, double fx, double fy, double cx, double cy, double z_min,
                 double z_max, const double pose_prev[7], const double c0[7], const double r0[6],
                 const float *omega, int N, double tau, double beta, double eps, double stop_eps, int k_max,
                 int flags, double pose_out[7], double r1_out[6], double *trace, int *iters_out)
{
    if (N < 1 || k_max < 1)
        return OR_ERR_ARG;
    for (int d = 0; d < 6; ++d)
        if (omega[(size_t)d * N] != 0.0f)
            return OR_ERR_ARG; /* row 0 must be the origin (reading 8) */
    int *mask = (int *)malloc(sizeof(int) * (size_t)(M > 0 ? M : 1));
    double *margin = (double *)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1));
    double *rho = (double *)malloc(sizeof(double) * (size_t)N);
    double *delta = (double *)malloc(sizeof(double) * 6 * (size_t)N);
    double c[7], r[6], rho_carry = 0.0;
    memcpy(c, c0, sizeof c);
    memcpy(r, r0, sizeof r);
    int empty_run = 0, status = OR_OK, k = 0;
    for (k = 1; k <= k_max; ++k) {
        /* O_k with s*_{k-1} = c_{k-1} */
        int nO = 0;
        double min_margin = INFINITY;
        if (flags & OR_OVERLAP) {
            nO = or_overlap(pts, M, prev_depth, W, H, fx, fy, cx, cy, z_min, z_max, c, pose_prev,
                            (flags & OR_CELL_MARGIN) ? sqrt(3.0) * voxel : 0.0, mask, margin);
            for (int j = 0; j < M; ++j)
                if (pts[4 * (size_t)j + 3] != 0.0 && margin[j] < min_margin)
                    min_margin = margin[j];
        } else {
            for (int j = 0; j < M; ++j) {
                mask[j] = pts[4 * (size_t)j + 3] != 0.0;
                nO += mask[j];
            }
        }
        double *tr = trace ? trace + OR_TRACE_STRIDE * (size_t)(k - 1) : NULL;
        if (nO == 0) {
            status = OR_ERR_EMPTY;
            if (tr) {
                memset(tr, 0, sizeof(double) * OR_TRACE_STRIDE);
                tr[0] = k;
                tr[28] = 4;
            }
            break;
        }
        /* fitness of every particle (Eq. normallh) */
        double rho_max = -1.0, rho_2nd = -1.0;
        int argmax = 0;
        for (int i = 0; i < N; ++i) {
            double om[6], pose[7], S;
            int n, nOi;
            for (int d = 0; d < 6; ++d) {
                om[d] = omega[(size_t)d * N + i];
                delta[6 * (size_t)i + d] = r[d] * om[d];
            }
            or_compose_offset(c, delta + 6 * (size_t)i, flags, pose);
            or_fitness(F, dim, voxel, origin, pts, mask, M, pose, tau, flags, &S, &n, &nOi, &rho[i]);
            if (rho[i] > rho_max) {
                rho_2nd = rho_max;
                rho_max = rho[i];
                argmax = i;
            } else if (rho[i] > rho_2nd) {
                rho_2nd = rho[i];
            }
        }
        double rho_ref = (k == 1 || (flags & OR_RHO_REF_CENTER)) ? rho[0] : rho_carry;
        double min_gap = INFINITY;
        for (int i = 0; i < N; ++i)
            if (fabs(rho[i] - rho_ref) < min_gap && i != 0)
                min_gap = fabs(rho[i] - rho_ref);
        double dbar[6], rho_tilde, r_new[6];
        /* the APS holds particles better than s*_{k-1}; particle 0 (zero offset) is
         * s*_{k-1} itself, so it is no candidate (it only passes rho_ref when that is
         * the Eq. wafit approximation) */
        int n_aps = or_pst_update(N - 1, rho + 1, delta + 6, rho_ref, r, beta, eps, dbar, &rho_tilde, r_new);
        double s_new[7];
        if (n_aps > 0) {
            or_compose_offset(c, dbar, flags, s_new);
            empty_run = 0;
        } else {
            memcpy(s_new, c, sizeof s_new);
            ++empty_run;
        }
        rho_carry = rho_tilde;
        memcpy(c, s_new, sizeof c);
        memcpy(r, r_new, sizeof r);
        if (k == 1)
            memcpy(r1_out, r, sizeof r);
        double step = 0.0;
        for (int d = 0; d < 6; ++d)
            step = fmax(step, fabs(dbar[d]));
        int stop = 0;
        if (empty_run >= 2)
            stop = 1;
        else if (n_aps > 0 && step < stop_eps)
            stop = 2;
        else if (k == k_max)
            stop = 3;
        if (tr) {
            tr[0] = k;
            tr[1] = nO;
            tr[2] = n_aps;
            tr[3] = rho_ref;
            tr[4] = rho_tilde;
            tr[5] = rho_max;
            tr[6] = argmax;
            for (int a = 0; a < 7; ++a)
                tr[7 + a] = c[a];
            for (int d = 0; d < 6; ++d) {
                tr[14 + d] = r[d];
                tr[20 + d] = dbar[d];
            }
            tr[26] = min_gap;
            tr[27] = min_margin;
            tr[28] = stop;
            tr[29] = rho_2nd;
        }
        if (stop)
            break;
    }
    if (k > k_max)
        k = k_max;
    memcpy(pose_out, c, sizeof c);
    if (k == 1 && status == OR_ERR_EMPTY)
        memcpy(r1_out, r0, sizeof r);
    *iters_out = k;
    free(mask);
    free(margin);
    free(rho);
    free(delta);
    return status;
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
 * F is rounded to the storage type after every update (qmode).
 */
void or_tsdf_integrate(double *F, int *Wt, const int dim[3], double voxel, const double origin[3], double trunc,
                       int w_max, int qmode, const float *depth, int W, int H, double fx, double fy, double cx,
                       double cy, double z_min, double z_max, const double pose[7])
{
    double R[9];
    or_quat_to_rot(pose, R);
    for (int k = 0; k < dim[2]; ++k)
        for (int j = 0; j < dim[1]; ++j)
            for (int i = 0; i < dim[0]; ++i) {
                double pw[3] = {origin[0] + voxel * (i + 0.5), origin[1] + voxel * (j + 0.5),
                                origin[2] + voxel * (k + 0.5)};
                double pc[3];
                apply_pose_inverse(R, pose + 4, pw, pc);
                if (!(pc[2] > 0.0))
                    continue;
                double u = floor(fx * pc[0] / pc[2] + cx + 0.5);
                double v = floor(fy * pc[1] / pc[2] + cy + 0.5);
                if (u < 0.0 || u >= (double)W || v < 0.0 || v >= (double)H)
                    continue;
                double D = depth[(size_t)v * W + (size_t)u];
                if (!(D > z_min && D <= z_max))
                    continue;
                double sdf = D - pc[2];
                if (sdf < -trunc)
                    continue;
                double f = sdf / trunc;
                if (f > 1.0)
                    f = 1.0;
                size_t idx = (size_t)i + (size_t)dim[0] * ((size_t)j + (size_t)dim[1] * (size_t)k);
                int w_old = Wt[idx];
                double F_old = isnan(F[idx]) ? 0.0 : F[idx];
                if (isnan(F[idx]))
                    w_old = 0;
                double F_new = ((double)w_old * F_old + f) / (double)(w_old + 1);
                F[idx] = or_quantize(F_new, qmode);
                Wt[idx] = (w_old + 1 < w_max) ? w_old + 1 : w_max;
            }
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

/* ------------------------------------------------------------------------- */
/* Multi-resolution PST alternation (Sec. 4 "Multi-resolution PST").          */
/* ------------------------------------------------------------------------- */

/*
 * Algorithm 1 with L (particle count, depth stride) levels used in turn:
 * iteration k uses level l = (k - 1) mod L, i.e. the first level_n[l] rows of
 * the template and the points unprojected at that level's stride
 * (level_pts[l], level_M[l] points).  Readings: with L > 1 the fitness of
 * consecutive iterations is normalised over different point sets, so the APS
 * threshold is the fitness of the centre particle in the current iteration
 * (particle 0); with L = 1 the rule of or_pfo_frame applies.  Everything else
 * (overlap with s*_{k-1}, Eq. ebs / wafit / rsdir / rsinter / momentum, the
 * corner cases and stop rules) is that of or_pfo_frame.  Same outputs.
 */
int or_pfo_frame_sched(const double *F, const int dim[3], double voxel, const double origin[3], int L,
                       const int *level_n, const double *const *level_pts, const int *level_M,
                       const float *prev_depth, int W, int H, double fx, double fy, double cx, double cy,
                       double z_min, double z_max, const double pose_prev[7], const double c0[7], const double r0[6],
                       const float *omega, int N, double tau, double beta, double eps, double stop_eps, int k_max,
                       int flags, double pose_out[7], double r1_out[6], double *trace, int *iters_out)
{
    if (L < 1 || N < 1 || k_max < 1)
        return OR_ERR_ARG;
    int M_max = 1, N_lev_max = 1;
    for (int l = 0; l < L; ++l) {
        if (level_n[l] < 1 || level_n[l] > N)
            return OR_ERR_ARG;
        if (level_M[l] > M_max)
            M_max = level_M[l];
        if (level_n[l] > N_lev_max)
            N_lev_max = level_n[l];
    }
    for (int d = 0; d < 6; ++d)
        if (omega[(size_t)d * N] != 0.0f)
            return OR_ERR_ARG;
    int *mask = (int *)malloc(sizeof(int) * (size_t)M_max);
    double *margin = (double *)malloc(sizeof(double) * (size_t)M_max);
    double *rho = (double *)malloc(sizeof(double) * (size_t)N_lev_max);
    double *delta = (double *)malloc(sizeof(double) * 6 * (size_t)N_lev_max);
    double c[7], r[6], rho_carry = 0.0;
    memcpy(c, c0, sizeof c);
    memcpy(r, r0, sizeof r);
    int empty_run = 0, status = OR_OK, k = 0;
    for (k = 1; k <= k_max; ++k) {
        const int l = (k - 1) % L;
        const int Nl = level_n[l], M = level_M[l];
        const double *pts = level_pts[l];
        int nO = 0;
        double min_margin = INFINITY;
        if (flags & OR_OVERLAP) {
            nO = or_overlap(pts, M, prev_depth, W, H, fx, fy, cx, cy, z_min, z_max, c, pose_prev,
                            (flags & OR_CELL_MARGIN) ? sqrt(3.0) * voxel : 0.0, mask, margin);
            for (int j = 0; j < M; ++j)
                if (pts[4 * (size_t)j + 3] != 0.0 && margin[j] < min_margin)
                    min_margin = margin[j];
        } else {
            for (int j = 0; j < M; ++j) {
                mask[j] = pts[4 * (size_t)j + 3] != 0.0;
                nO += mask[j];
            }
        }
        double *tr = trace ? trace + OR_TRACE_STRIDE * (size_t)(k - 1) : NULL;
        if (nO == 0) {
            status = OR_ERR_EMPTY;
            if (tr) {
                memset(tr, 0, sizeof(double) * OR_TRACE_STRIDE);
                tr[0] = k;
                tr[28] = 4;
            }
            break;
        }
        double rho_max = -1.0, rho_2nd = -1.0;
        int argmax = 0;
        for (int i = 0; i < Nl; ++i) {
            double pose[7], S;
            int n, nOi;
            for (int d = 0; d < 6; ++d)
                delta[6 * (size_t)i + d] = r[d] * omega[(size_t)d * N + i];
            or_compose_offset(c, delta + 6 * (size_t)i, flags, pose);
            or_fitness(F, dim, voxel, origin, pts, mask, M, pose, tau, flags, &S, &n, &nOi, &rho[i]);
            if (rho[i] > rho_max) {
                rho_2nd = rho_max;
                rho_max = rho[i];
                argmax = i;
            } else if (rho[i] > rho_2nd) {
                rho_2nd = rho[i];
            }
        }
        const int centre_ref = (k == 1) || (flags & OR_RHO_REF_CENTER) || (L > 1);
        double rho_ref = centre_ref ? rho[0] : rho_carry;
        double min_gap = INFINITY;
        for (int i = 1; i < Nl; ++i)
            if (fabs(rho[i] - rho_ref) < min_gap)
                min_gap = fabs(rho[i] - rho_ref);
        double dbar[6], rho_tilde, r_new[6];
        int n_aps = or_pst_update(Nl - 1, rho + 1, delta + 6, rho_ref, r, beta, eps, dbar, &rho_tilde, r_new);
        double s_new[7];
        if (n_aps > 0) {
            or_compose_offset(c, dbar, flags, s_new);
            empty_run = 0;
        } else {
            memcpy(s_new, c, sizeof s_new);
            ++empty_run;
        }
        rho_carry = rho_tilde;
        memcpy(c, s_new, sizeof c);
        memcpy(r, r_new, sizeof r);
        if (k == 1)
            memcpy(r1_out, r, sizeof r);
        double step = 0.0;
        for (int d = 0; d < 6; ++d)
            step = fmax(step, fabs(dbar[d]));
        int stop = 0;
        if (empty_run >= 2)
            stop = 1;
        else if (n_aps > 0 && step < stop_eps)
            stop = 2;
        else if (k == k_max)
            stop = 3;
        if (tr) {
            tr[0] = k;
            tr[1] = nO;
            tr[2] = n_aps;
            tr[3] = rho_ref;
            tr[4] = rho_tilde;
            tr[5] = rho_max;
            tr[6] = argmax;
            for (int a = 0; a < 7; ++a)
                tr[7 + a] = c[a];
            for (int d = 0; d < 6; ++d) {
                tr[14 + d] = r[d];
                tr[20 + d] = dbar[d];
            }
            tr[26] = min_gap;
            tr[27] = min_margin;
            tr[28] = stop;
            tr[29] = rho_2nd;
            tr[30] = l;
            tr[31] = Nl;
        }
        if (stop)
            break;
    }
    if (k > k_max)
        k = k_max;
    memcpy(pose_out, c, sizeof c);
    if (k == 1 && status == OR_ERR_EMPTY)
        memcpy(r1_out, r0, sizeof r);
    *iters_out = k;
    free(mask);
    free(margin);
    free(rho);
    free(delta);
    return status;
}
