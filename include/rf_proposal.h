/*
 * rf_proposal.h -- C ABI of the learned swarm proposal in librosefusion.so.
 *
 * The paper has no learned component.  Sec. 4 starts the PST of frame t at the
 * previous frame's best state (c_0 = s*_{t-1}) with the previous frame's axis
 * lengths (r_0 = r_1 of frame t-1), and Sec. 6 names combining the random
 * optimisation with learned priors as future work.  This API replaces that
 * initialisation with the output of a small network: the network predicts the
 * offset of frame t from frame t-1 and a per-axis uncertainty; c_0 and r_0 come
 * from them, a short PFO run (Algorithm 1) refines the swarm, and plain PFO
 * (the Sec. 4 initialisation, full iteration budget) stays as the fallback.
 * Everything runs in the library's kernels: feature extraction, the network's
 * forward and backward products on the tensor cores (bfloat16 operands, FP32
 * accumulation), the loss, Adam (Kingma & Ba 2015, Algorithm 1) and the
 * proposal.  The general rules of rosefusion.h apply (status codes, *_dev
 * device pointers, streams, poses as 7 floats q then t).
 *
 * Definitions
 *  features  x (RF_MLP_IN bfloat16 values, stored as uint16 bit patterns):
 *            a 32 x 24 grid of cells over the frame, cell (i, j) covering
 *            columns [floor(i W / 32), floor((i + 1) W / 32)) and rows
 *            [floor(j H / 24), floor((j + 1) H / 24)); m(i, j) = mean of the
 *            valid depths (z_min < z <= z_max) of a cell;
 *              x[32 j + i] = clip((m_t(i, j) - m_{t-1}(i, j)) / 0.1 m, -8, 8)
 *            where both cells hold valid depth, else 0;
 *              x[768..773] = offset(s*_{t-2}, s*_{t-1}) / units;  x[774..831] = 0.
 *  offset    offset(a, b) = d with b = a (+) d under the MovePST composition of
 *            Sec. 3.3 (left-multiplied rotation, world-frame translation):
 *            d[0..2] = vector part of q_b q_a^-1 (scalar part >= 0),
 *            d[3..5] = t_b - t_a.  units = (0.05, 0.05, 0.05, 0.1 m, 0.1 m, 0.1 m).
 *  network   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3),
 *            o = W4 h3 + b4; W1 256 x 832, W2 and W3 256 x 256, W4 16 x 256.
 *            Weights, x and h are rounded to bfloat16 (nearest even) before each
 *            product; products accumulate in FP32.  Parameters: one flat float
 *            vector W1 (row-major), b1, W2, b2, W3, b3, W4, b4.  Columns 774..831
 *            of W1 and rows 12..15 of W4 / entries 12..15 of b4 are padding.
 *  output    mu = x[768..773] + o[0..5]: the offset from s*_{t-1} to s*_t over
 *            units, as the previous offset plus the network's correction;
 *            s = clamp(o[6..11], -6, 6) (log scale per axis).
 *  loss      mean over the batch of sum_d 1/2 r_d^2 (1 + exp(-2 s_d)) + s_d,
 *            r = y - mu (squared error plus a Gaussian negative log-likelihood);
 *            the target y = offset(s*_{t-1}, s*_t) / units of the plain tracker.
 *  proposal  c_0 = s*_{t-1} (+) mu * units;
 *            r_0 = clip(kappa * exp(s) * units, r_min, r_max), per axis.
 */
#ifndef RF_PROPOSAL_H
#define RF_PROPOSAL_H

#include "rosefusion.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RF_MLP_IN 832
#define RF_MLP_IN_USED 774
#define RF_MLP_HIDDEN 256
#define RF_MLP_OUT 16
#define RF_MLP_OUT_USED 12
#define RF_MLP_MAX_BATCH 4096
#define RF_MLP_MAX_TRAIN_BATCH 1024

/* ------------------------------------------------------------- network --- */
typedef struct rf_mlp_s *rf_mlp;

/* Number of floats in the flat parameter vector (348944). */
int rf_mlp_num_params(void);
/*
 * rf_mlp_create -- device storage for the parameters, the Adam moments, the
 * bfloat16 weight copies and the activations of up to max_batch rows
 * (1 .. RF_MLP_MAX_BATCH).  Parameters start at zero.  Synchronous.
 */
rf_status rf_mlp_create(int max_batch, rf_mlp *out);
void rf_mlp_destroy(rf_mlp m);
/* Upload / download the flat parameter vector (host float[rf_mlp_num_params()]).
 * set_params also zeroes the Adam moments and step count.  Synchronous. */
rf_status rf_mlp_set_params(rf_mlp m, const float *theta_host);
rf_status rf_mlp_get_params(rf_mlp m, float *theta_host);
/*
 * rf_mlp_forward -- o for `batch` input rows.
 *   x_dev    device uint16[batch * RF_MLP_IN] (bfloat16 bit patterns), row-major
 *   out_dev  device float[batch * RF_MLP_OUT]
 */
rf_status rf_mlp_forward(rf_mlp m, const uint16_t *x_dev, int batch, float *out_dev, void *stream);
/*
 * rf_mlp_gradient -- loss and gradient of one batch (no update).  The batch is
 * rows idx_dev[0..batch) of a dataset (rows 0..batch-1 when idx_dev is NULL).
 *   x_all_dev  device uint16[n_all * RF_MLP_IN]   inputs (bfloat16 bits)
 *   y_all_dev  device float[n_all * 6]            targets (over units)
 *   idx_dev    device int[batch] or NULL; a row outside [0, n_all) sets
 *              RF_ERR_ARG in rf_mlp_status and skips that row
 *   batch      multiple of 8, 8 .. min(max_batch, RF_MLP_MAX_TRAIN_BATCH)
 *   grad_dev   device float[rf_mlp_num_params()] or NULL
 *   loss_dev   device float[1] or NULL
 *   out_dev    device float[batch * RF_MLP_OUT] or NULL: the forward outputs
 */
rf_status rf_mlp_gradient(rf_mlp m, const uint16_t *x_all_dev, const float *y_all_dev, const int *idx_dev, int n_all,
                          int batch, float *grad_dev, float *loss_dev, float *out_dev, void *stream);
/* rf_mlp_gradient followed by one Adam step (beta1 0.9, beta2 0.999, eps 1e-8)
 * with learning rate lr on the FP32 parameters. */
rf_status rf_mlp_train_step(rf_mlp m, const uint16_t *x_all_dev, const float *y_all_dev, const int *idx_dev, int n_all,
                            int batch, float lr, float *loss_dev, void *stream);
/*
 * rf_mlp_evaluate -- the network over dataset rows (forward passes of at most
 * max_batch rows at a time) and the quantities its training selects and
 * calibrates with.  Per row: mu = x[768..773] + o[0..5], s = clamp(o[6..11],
 * -6, 6), e = y - mu.  The rows are idx_dev[0..n_rows) of the data set (rows
 * 0..n_rows-1 when idx_dev is NULL); a row outside [0, n_all) sets RF_ERR_ARG in
 * rf_mlp_status and is skipped.
 *   mu_dev     device float[n_rows * 6] or NULL: mu of every row
 *   stats_dev  device double[RF_MLP_EVAL_STATS] or NULL, means over the rows:
 *              [0] sum_d e_d^2 (the squared offset error), [1 + d] e_d^2
 *              exp(-2 s_d) (the calibration moments), [7 + d] y_d^2 (the error
 *              of the zero offset, i.e. of the Sec. 4 initialisation, per axis)
 * The row sums run in FP64 in a fixed order.  Asynchronous.
 */
#define RF_MLP_EVAL_STATS 13
rf_status rf_mlp_evaluate(rf_mlp m, const uint16_t *x_all_dev, const float *y_all_dev, const int *idx_dev,
                          int n_all, int n_rows, float *mu_dev, double *stats_dev, void *stream);
/*
 * rf_mlp_calibrate_scale -- per-axis calibration of the log-scale head on dataset
 * rows (same row selection as rf_mlp_evaluate): with k_d^2 the mean of e_d^2
 * exp(-2 s_d) over the rows, log k_d is added to the output bias of s_d, so that
 * the predicted variances exp(2 s_d) match the rows' squared errors.  k_host
 * (host float[6]) receives k.  Synchronous.
 */
rf_status rf_mlp_calibrate_scale(rf_mlp m, const uint16_t *x_all_dev, const float *y_all_dev, const int *idx_dev,
                                 int n_all, int n_rows, float k_host[6], void *stream);
/* Device status of the network's kernels since the last call (bounded waits in
 * the tensor-core products report RF_ERR_TIMEOUT); resets it.  Synchronous. */
rf_status rf_mlp_status(rf_mlp m);

/* ------------------------------------------------------------ proposal --- */
/*
 * rf_proposal_features -- x of one frame pair (definition above).
 *   depth_dev, prev_depth_dev  device float[H * W] frames t and t-1
 *   pose_prev2_dev, pose_prev_dev  device float[7]: s*_{t-2}, s*_{t-1}
 *   x_dev                      device uint16[RF_MLP_IN]
 */
rf_status rf_proposal_features(const float *depth_dev, const float *prev_depth_dev, const rf_intrinsics *K,
                               const float *pose_prev2_dev, const float *pose_prev_dev, uint16_t *x_dev,
                               void *stream);
/* rf_proposal_target -- y = offset(s*_{t-1}, s*_t) / units (device float[6]). */
rf_status rf_proposal_target(const float *pose_prev_dev, const float *pose_cur_dev, float *y_dev, void *stream);

typedef struct {
    int k_learned;   /* PFO iterations after the proposal (default 5) */
    int k_fallback;  /* iterations of the plain fallback run (default 20) */
    float kappa;     /* r_0 = kappa * exp(s) * units (default 0.25) */
    float theta;     /* fallback runs when the learned run's final rho_tilde <
                        theta * the previous frame's, on any error status, or
                        when its first iteration found no TSDF sample for any
                        particle (Sec. 4's first corner case: the proposal is off
                        the map); theta < 0: never (default 0.95) */
    float r_min[6];  /* default 2e-3 (rotation axes), 4e-3 m (translation) */
    float r_max[6];  /* default 0.2, 0.4 m */
    int resume;      /* 1 (default): when the learned run used all k_learned
                        iterations without meeting a convergence criterion of
                        Sec. 4 (and the fallback rule did not fire), PFO resumes
                        from its s* and axis lengths for up to k_fallback more
                        iterations; 0: no second run in that case */
    int stuck;       /* a learned run whose every iteration had an empty APS never
                        left c_0 (its result is the proposal itself): 0 keep it,
                        1 (default) resume PFO from c_0 with the carried r_1 of the
                        Sec. 4 initialisation for up to k_fallback iterations,
                        2 plain restart from s*_{t-1} */
} rf_proposal_params;

/* Fills *p with the defaults above. */
void rf_proposal_default_params(rf_proposal_params *p);
/*
 * rf_proposal_apply -- c_0 and r_0 (definition above) from one network output.
 *   out_dev        device float[RF_MLP_OUT]
 *   x_dev          device uint16[RF_MLP_IN]: the input row the output came from
 *                  (its previous-offset entries are the base of mu)
 *   pose_prev_dev  device float[7], s*_{t-1}
 *   init_pose_dev  device float[7] receives c_0;  scale_dev device float[6] r_0
 */
rf_status rf_proposal_apply(const float *out_dev, const uint16_t *x_dev, const float *pose_prev_dev,
                            const rf_proposal_params *p, float *init_pose_dev, float *scale_dev, void *stream);

/* -------------------------------------------------- learned tracking --- */
/*
 * A learned tracker drives an rf_tracker (its template, parameters and scratch)
 * and the rf_volume it fuses into, with a trained rf_mlp:
 *   per frame t: features of (D_t, D_{t-1}, s*_{t-2}, s*_{t-1}) -> network ->
 *   proposal (c_0, r_0) -> PFO with at most k_learned iterations from c_0
 *   (pfo_track_frame_ex_async; the overlap set still uses s*_{t-1}) -> if the
 *   fallback rule fires, plain PFO from s*_{t-1} with the carried r_1 and
 *   k_fallback iterations; else if the run never left c_0, the `stuck` rule;
 *   else, with `resume`, if the learned run stopped at k_learned unconverged,
 *   PFO continues from its s* and axis lengths for up to k_fallback
 *   iterations; the result with the higher final rho_tilde is kept (a tie goes
 *   to a plain restart, else to the learned run) -> fusion
 *   (tsdf_integrate) of D_t at the kept pose.
 * Frames are at most max_width x max_height.  The tracker and network must not
 * be used by other calls while a step runs.
 */
typedef struct rf_learned_s *rf_learned;
typedef struct {
    int status;          /* final status of the frame (0 = OK) */
    int used_fallback;   /* second run: 0 none, 1 plain restart, 2 resumed, 3 resumed
                            from a proposal the learned run never left */
    int chose_fallback;  /* its result was kept */
    int iters_learned;
    int iters_fallback;
    float rho_learned;   /* final rho_tilde of the learned run */
    float rho_fallback;  /* final rho_tilde of the fallback run (0 if none) */
    float rho_prev;      /* kept rho_tilde of frame t-1 */
    float init_pose[7];  /* c_0 */
    float r0[6];         /* r_0 */
    long long lookups;   /* particle x point lookups of both runs */
} rf_learned_stats;

rf_status rf_learned_create(rf_tracker tr, rf_volume vol, rf_mlp net, const rf_proposal_params *p, int max_width,
                            int max_height, rf_learned *out);
void rf_learned_destroy(rf_learned lp);
/* Fuse frame 0 at `pose`; s*_{-1} = s*_0 (zero previous motion), the carried
 * r_1 is the tracker's current r_0. */
rf_status rf_learned_start(rf_learned lp, const float *depth, int depth_on_host, const rf_intrinsics *K,
                           const rf_pose *pose, void *stream);
/*
 * rf_learned_step -- track and fuse the next frame.
 *   depth          float[H * W], on the host if depth_on_host != 0
 *   use_graph      != 0: the frame's kernels run as a CUDA graph, captured on
 *                  first use (on an internal stream) and again whenever K,
 *                  out_pose_dev or stats_dev differ from the captured ones
 *   out_pose_host  host rf_pose or NULL (when given the call synchronises)
 *   out_pose_dev   device float[7] or NULL
 *   stats_dev      device rf_learned_stats or NULL
 */
rf_status rf_learned_step(rf_learned lp, const float *depth, int depth_on_host, const rf_intrinsics *K, int use_graph,
                          rf_pose *out_pose_host, float *out_pose_dev, rf_learned_stats *stats_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RF_PROPOSAL_H */
