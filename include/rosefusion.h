/*
 * rosefusion.h -- C ABI of librosefusion.so, the GB300 (sm_103a) implementation of
 * the depth-only tracking hot path of ROSEFusion (Zhang, Zhu, Zheng, Xu,
 * "ROSEFusion: Random Optimization for Online Dense Reconstruction under Fast
 * Camera Motion", ACM TOG 40(4), 2021): particle filter optimisation (PFO)
 * with a particle swarm template (PST) scored against a TSDF volume, and the
 * volumetric fusion of each tracked frame.
 *
 * General rules
 *  - Every entry point returns an rf_status (0 = RF_OK, < 0 = error) and never
 *    throws.  rf_last_error() returns a thread-local message for the last
 *    failure on the calling thread.
 *  - Pointers named *_dev are device pointers owned by the caller (for
 *    example torch CUDA tensors' data_ptr()); pointers named *_host are host
 *    pointers owned by the caller.  Handles (rf_volume, rf_tracker) own their
 *    device storage and scratch; destroy them with the matching *_destroy.
 *  - `stream` is a cudaStream_t passed as void* (0 = legacy default stream).
 *    Calls are asynchronous on that stream unless stated otherwise.  Calls
 *    that share a handle must be ordered by the caller (same stream or
 *    events); two calls on one handle that overlap on the GPU race on its
 *    scratch.
 *  - Poses are camera->world, x_G = R(q) x + t (Sec. 3.1, Eq. unproj), with q =
 *    (w, x, y, z) a unit Hamilton quaternion, w >= 0.  On the device a pose
 *    is 7 contiguous floats (q then t).
 *  - The TSDF stores the normalised truncated distance F = sdf / trunc in
 *    [-1, 1]; unobserved voxels hold a sentinel (NaN for float storage,
 *    -32768 for int16).  Voxel (i, j, k) has its centre at
 *    origin + voxel * (i + 0.5, j + 0.5, k + 0.5).
 */
#ifndef ROSEFUSION_H
#define ROSEFUSION_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int rf_status;
#define RF_OK 0
#define RF_ERR_ARG (-1)     /* invalid argument (null pointer, size, alignment) */
#define RF_ERR_CUDA (-2)    /* a CUDA runtime call failed                      */
#define RF_ERR_TIMEOUT (-3) /* a bounded device-side wait gave up               */
#define RF_ERR_EMPTY (-4)   /* the overlap set O_k was empty                    */
#define RF_ERR_NOMEM (-5)   /* device allocation failed                         */

/* Pinhole camera; depth values outside (z_min, z_max] are invalid. */
typedef struct {
    float fx, fy, cx, cy;
    int width, height;
    float z_min, z_max;
} rf_intrinsics;

typedef struct {
    float q[4]; /* w, x, y, z */
    float t[3];
} rf_pose;

/* Flags of rf_params.flags (ablations of Sec. 5.2 and the readings of the
 * paper's silent points). */
#define RF_OVERLAP 1         /* normalise over the overlap set O_k (Eq. validness)      */
#define RF_NORMALIZE 2       /* divide by |O_k| (Eq. normallh); off = Eq. ourlh          */
#define RF_COMPENSATED 4     /* Neumaier-compensated FP32 sums (Sec. 4, Kahan summation) */
#define RF_NEAREST 8         /* nearest-voxel sample instead of trilinear               */
#define RF_RHO_REF_CENTER 16 /* APS threshold = fitness of the centre particle          */
#define RF_L1 32             /* sum |psi| instead of psi^2                               */
#define RF_RIGHT_MULT 64     /* particle offset applied in the camera frame              */
#define RF_CELL_MARGIN 128   /* O_k: re-projection inside frame t-1 by one cell footprint */
#define RF_APS_WITH_CENTRE 256 /* the centre particle (s*_{k-1} itself) may join the APS */
#define RF_DEFAULT_FLAGS (RF_OVERLAP | RF_NORMALIZE | RF_COMPENSATED | RF_CELL_MARGIN)

/* Parameters of Algorithm 1; the defaults of the paper are tau = 1 (Sec. 3.2),
 * beta = 0.1 (Eq. momentum), eps = 1e-3 (Eq. rsinter), stop_eps = 1e-6 and
 * k_max = 20 (Sec. 4, convergence criteria). */
typedef struct {
    float tau, beta, eps, stop_eps;
    int k_max; /* 1 .. RF_MAX_ITERS */
    int flags;
    int stride; /* depth downsampling stride (Sec. 4, multi-resolution PST) */
    int reserved;
} rf_params;

#define RF_MAX_ITERS 64

/* One row per PFO iteration k (all on the device; copied out by the caller). */
typedef struct {
    int k, n_overlap, n_aps, argmax;
    float rho_ref, rho_tilde, rho_max, rho_second;
    float pose[7];  /* s*_k                                  */
    float scale[6]; /* r_k                                   */
    float offset[6];/* delta_bar_k = s*_k - s*_{k-1} (local) */
    int stop;       /* 0 running, 1 empty twice, 2 small step, 3 k_max, 4 empty overlap */
    int level;      /* multi-resolution level used by this iteration          */
    int n_particles;/* particles scored (the level's prefix of the template)  */
    int corner;     /* Sec. 4 "PST update" corner case taken: 0 none, 1 no TSDF
                       sample for any particle (rho = 0.5, v = 1, r_hat = 0.5 + eps,
                       s* kept), 2 empty APS (r_hat = 2 (1 - rho) / sqrt(6) + eps) */
} rf_iter_stats;

typedef struct {
    int iters, status, n_points, reserved;
    long long lookups; /* particle x point TSDF lookups performed: sum_k N * |O_k| */
    float r1[6];       /* axis lengths after iteration 1 (next frame's r_0)        */
    float pad[2];
    rf_iter_stats it[RF_MAX_ITERS];
} rf_frame_stats;

typedef enum { RF_F32 = 0, RF_F16 = 1, RF_I16 = 2 } rf_dtype;

typedef struct rf_volume_s *rf_volume;
typedef struct rf_tracker_s *rf_tracker;

/* Thread-local text of the last error on this thread ("" if none). */
const char *rf_last_error(void);
/* Library version string. */
const char *rf_version(void);

/* ---------------------------------------------------------------- PST --- */
/*
 * pst_create -- pre-sample a particle swarm template in the closed unit 6D
 * ball (Sec. 4, "PST pre-sampling"; Sec. 3.3: c_0 = 0, r_0 = 1).
 *   n           number of particles, n >= 1.  Row 0 is always the origin, so
 *               particle 0 sits on the PST centre.
 *   seed        Philox4x32-10 key (Salmon et al., SC 2011).
 *   method      0 = uniform by rejection from the cube (GPU kernel); the
 *               candidate coordinates are exact multiples of 2^-24 and the
 *               acceptance test is an exact integer test, so the template is
 *               bit-reproducible on any machine.  1 = Poisson-disk (Bridson,
 *               SIGGRAPH 2007 sketch) computed on the host and copied in.
 *   out_dev     device float[6 * n], structure of arrays: out_dev[d * n + i].
 * Errors: RF_ERR_ARG for n < 1 or a null pointer.  Asynchronous for method 0.
 */
rf_status pst_create(int n, uint64_t seed, int method, float *out_dev, void *stream);

/* ------------------------------------------------------------- volume --- */
/*
 * rf_volume_create -- allocate a dim_x * dim_y * dim_z TSDF (each a multiple
 * of 8, up to 2048) in 8x8x8 voxel bricks, storage type dtype, plus uint8
 * weights, all unobserved.  voxel and trunc are in metres; origin is the
 * world position of the volume's lower corner.  The handle owns the memory.
 */
rf_status rf_volume_create(int dim_x, int dim_y, int dim_z, float voxel, float trunc, const float origin[3],
                           int dtype, rf_volume *out);
void rf_volume_destroy(rf_volume v);
/* Set every voxel unobserved (value sentinel, weight 0). */
rf_status rf_volume_reset(rf_volume v, void *stream);
/*
 * rf_volume_upload / rf_volume_download -- copy the whole volume from / to
 * host arrays in plain x-fastest order (index x + dim_x * (y + dim_y * z)):
 * values_host holds storage codes of the volume's dtype (float, IEEE half,
 * or int16 round(F * 32767) with -32768 = unobserved); weights_host holds
 * uint8 (may be NULL on upload: weight 1 where observed, 0 elsewhere; may be
 * NULL on download).  Synchronous.
 */
rf_status rf_volume_upload(rf_volume v, const void *values_host, const uint8_t *weights_host);
rf_status rf_volume_download(rf_volume v, void *values_host, uint8_t *weights_host);
/* Query the geometry: dims[3], voxel, trunc, origin[3], dtype. */
rf_status rf_volume_info(rf_volume v, int dims[3], float *voxel, float *trunc, float origin[3], int *dtype);

/*
 * tsdf_integrate -- fuse one depth frame into the volume (Sec. 3 overview:
 * volumetric fusion after Curless & Levoy 1996 / KinectFusion 2011).  Every
 * voxel centre in front of the camera is projected to its nearest pixel; with
 * a valid depth D there and sdf = D - z_cam >= -trunc, f = min(1, sdf/trunc)
 * is averaged in: F <- (W F + f) / (W + 1), W <- min(W + 1, 255).
 *   depth_dev   device float[K->height * K->width], metres, row-major.
 *   K, pose     host structs.
 * Asynchronous: four stream-ordered operations (list reset, frustum culling,
 * update of the visible bricks, repacking of the cells that read a changed
 * value).  The volume holds one set of work lists, so fusions into the same
 * volume must not run concurrently on different streams.
 */
rf_status tsdf_integrate(rf_volume v, const float *depth_dev, const rf_intrinsics *K, const rf_pose *pose,
                         void *stream);
/*
 * tsdf_integrate_dev -- tsdf_integrate with the pose read from device memory
 * (pose_dev: float[7], for example a tracker's output) when the kernel runs;
 * if status_dev (device int, may be NULL) is non-zero at that time the frame
 * is skipped, so a failed track is never fused.  Asynchronous; capturable.
 */
rf_status tsdf_integrate_dev(rf_volume v, const float *depth_dev, const rf_intrinsics *K, const float *pose_dev,
                             const int *status_dev, void *stream);

/* ------------------------------------------------------ depth + overlap --- */
/*
 * rf_depth_to_points -- stride downsampling and unprojection of a depth map
 * (Eq. unproj; Sec. 4 stride-based downsampling).  Point (a, b) comes from
 * full-resolution pixel (a*stride, b*stride), row-major over b then a, so
 * there are ceil(H/stride) * ceil(W/stride) points.
 *   points_dev  device float4[ceil(H/s) * ceil(W/s)]: camera-frame (x, y, z)
 *               and w = 1 for a valid depth, all zeros for an invalid one.
 * Asynchronous.
 */
rf_status rf_depth_to_points(const float *depth_dev, const rf_intrinsics *K, int stride, float *points_dev,
                             void *stream);

/*
 * rf_overlap_mask -- the overlap set of Eq. validness: point j (w != 0) is in
 * O if, moved to the world with pose_cur and into frame t-1 with pose_prev,
 * it lies in front of that camera, rounds to a pixel inside the image and
 * frame t-1's depth there is valid.  With cell_extent > 0 its continuous
 * pixel position (u, v) must also satisfy
 *   fx c / z' - 1/2 <= u < W - 1/2 - fx c / z'   (and likewise v with fy, H),
 * c = cell_extent in metres, z' the point's depth in frame t-1: the TSDF cell
 * the point samples then lies inside frame t-1's view.  The tracker uses
 * c = sqrt(3) voxels under RF_CELL_MARGIN; 0 gives the plain test.
 *   points_dev      device float4[m] (rf_depth_to_points layout)
 *   prev_depth_dev  device float[H * W], full resolution
 *   mask_dev        device uint8[m] (1 = in O)
 *   count_dev       device int[1] receiving |O| (may be NULL)
 * Asynchronous.  RF_ERR_ARG for a negative or non-finite cell_extent.
 */
rf_status rf_overlap_mask(const float *points_dev, int m, const float *prev_depth_dev, const rf_intrinsics *K,
                          const rf_pose *pose_cur, const rf_pose *pose_prev, float cell_extent, uint8_t *mask_dev,
                          int *count_dev, void *stream);

/* ------------------------------------------------------------- fitness --- */
/*
 * fitness_eval -- score n PST particles on m points (Eq. normallh): particle i
 * has the pose centre (+) (scale . omega_i) (Sec. 3.3, Sec. 4 "GPU
 * implementation": the original PST is moved and rescaled on the fly), and
 *   S_i = sum_j psi(R_i x_j + t_i)^2,  rho_i = exp(-S_i / (tau m))
 * with psi the trilinear TSDF sample and psi = 1 where the sample is invalid
 * (out of the volume or an unobserved corner).  Every one of the m points
 * counts as a member of O (pass the compacted overlap set).  Flags NEAREST,
 * L1, NORMALIZE, COMPENSATED and RIGHT_MULT apply.
 *   points_dev  device float4[m] (x, y, z, ignored), camera frame; m >= 1
 *   pst_dev     device float[6 * n], structure of arrays, n >= 1
 *   centre      host pose; scale: host float[6]
 *   rho_dev     device float[n]; sumsq_dev device double[n] (may be NULL);
 *   nvalid_dev  device int[n] (may be NULL): number of valid samples
 * Scratch lives in the volume handle (grown on demand with cudaMalloc, which
 * synchronises the device the first time).  Asynchronous.
 */
rf_status fitness_eval(rf_volume v, const float *points_dev, int m, const float *pst_dev, int n,
                       const rf_pose *centre, const float scale[6], const rf_params *p, float *rho_dev,
                       double *sumsq_dev, int *nvalid_dev, void *stream);
/*
 * fitness_eval_noalloc -- fitness_eval without any device allocation (the
 * paper has no counterpart; this is a library service).  fitness_eval grows a
 * scratch buffer with cudaMalloc the first time a size needs it, and that call
 * synchronises the device and allocates.  Callers that cannot do either --
 * real-time loops that must never stall on a device-wide synchronisation or
 * on the allocator, plug-in hosts that own a fixed memory budget and forbid
 * their plug-ins to allocate -- use this entry point instead.  Arguments,
 * layouts and results are those of
 * fitness_eval; the caller still provides every input and output buffer.
 *   Scratch: the per-chunk partial sums live in a 32 MiB static device array
 *   inside the library, which every GPU that loads the library holds until
 *   the process exits.  Sizes with ceil(m / 256) * n * 12 bytes above 32 MiB
 *   are rejected with RF_ERR_ARG: n particles allow up to
 *   floor(32 MiB / (12 n)) * 256 points (n = 20,000: 139 chunks, m up to
 *   35,584).
 *   Set-up: the first call on each device (with that device current) looks
 *   up the array's device address with cudaGetSymbolAddress and caches it;
 *   make that first call before any stream capture.
 *   Sharing: all calls use the same array and leave their partial sums in
 *   it.  Every slot a call reads is written by that call first, so nothing
 *   needs clearing, but two calls that overlap on the GPU (different streams
 *   without ordering) race on the array.
 * No cudaMalloc, cudaFree or other allocating call is made.  Asynchronous.
 */
rf_status fitness_eval_noalloc(rf_volume v, const float *points_dev, int m, const float *pst_dev, int n,
                               const rf_pose *centre, const float scale[6], const rf_params *p, float *rho_dev,
                               double *sumsq_dev, int *nvalid_dev, void *stream);

/* ------------------------------------------------------------- tracker --- */
/*
 * rf_tracker_create -- a PFO tracker bound to a volume and a PST template
 * (pst_dev, n particles, row 0 = origin; the template is read, not copied,
 * and must outlive the tracker), for depth frames up to max_width x
 * max_height.  Allocates all scratch up front.  The axis lengths r start at 1
 * (Sec. 3.3).
 */
rf_status rf_tracker_create(rf_volume v, const float *pst_dev, int n, const rf_params *p, int max_width,
                            int max_height, rf_tracker *out);
void rf_tracker_destroy(rf_tracker tr);
/* Read / overwrite the axis lengths r_0 used by the next frame (host float[6]). */
rf_status rf_tracker_get_scale(rf_tracker tr, float r_host[6]);
rf_status rf_tracker_set_scale(rf_tracker tr, const float r_host[6]);
/* Replace the parameter block (k_max <= RF_MAX_ITERS). */
rf_status rf_tracker_set_params(rf_tracker tr, const rf_params *p);
/*
 * rf_tracker_set_schedule -- multi-resolution PST alternation (Sec. 4,
 * "Multi-resolution PST"): iteration k uses level (k - 1) mod n_levels, i.e.
 * the first n[level] particles of the template and the depth points at
 * stride[level].  1 <= n_levels <= RF_MAX_LEVELS, 1 <= n[l] <= template size,
 * stride[l] >= 1.  With more than one level the APS threshold of every
 * iteration is the fitness of the centre particle (consecutive iterations
 * normalise over different point sets).  The default schedule is one level:
 * the whole template at rf_params.stride.  Reallocates the tracker's point
 * and partial-sum buffers (synchronous).
 */
#define RF_MAX_LEVELS 4
rf_status rf_tracker_set_schedule(rf_tracker tr, int n_levels, const int *n, const int *stride);

/*
 * pfo_track_frame_async -- Algorithm 1 for one frame in ONE persistent kernel
 * (all iterations, no host round trip): per iteration the overlap set O_k is
 * built with s*_{k-1} (Eq. validness), every particle is scored (Eq.
 * normallh), the APS, best state and axis lengths are updated (Eq. ebs, wafit,
 * rsdir, rsinter, momentum; empty-APS corner case of Sec. 4) and the stop
 * rules of Sec. 4 are applied.  PST initialisation (Sec. 4): the centre
 * starts at prev_pose and the axis lengths at the tracker's r_0; r_0 is then
 * replaced by r_1 of this frame.
 *   depth_dev       device float[H * W] current frame
 *   prev_depth_dev  device float[H * W] frame t-1 (for the overlap set)
 *   prev_pose_dev   device float[7], the final pose of frame t-1
 *   out_pose_dev    device float[7], receives s*
 *   stats_dev       device rf_frame_stats (may be NULL)
 * Asynchronous.  Uses a bounded grid barrier: if a barrier wait exceeds about
 * one second the kernel stops and reports RF_ERR_TIMEOUT in stats->status
 * and through rf_tracker_last_status().
 */
rf_status pfo_track_frame_async(rf_tracker tr, const float *depth_dev, const float *prev_depth_dev,
                                const rf_intrinsics *K, const float *prev_pose_dev, float *out_pose_dev,
                                rf_frame_stats *stats_dev, void *stream);
/*
 * pfo_track_frame_ex_async -- pfo_track_frame_async with the Sec. 4 PST
 * initialisation supplied by the caller (e.g. a learned proposal):
 *   init_pose_dev  device float[7]: the swarm centre c_0 (NULL: prev_pose_dev).
 *                  prev_pose_dev stays the pose of frame t-1 for the overlap set.
 *   scale_dev      device float[6]: r_0 in, r_1 of this frame out (NULL: the
 *                  tracker's own r_0 / r_1 buffer)
 *   run_flag_dev   device int (may be NULL): read when the kernel starts; zero
 *                  means the frame is skipped (no iteration; out_pose_dev and
 *                  scale_dev untouched, stats_dev zeroed).  Lets a conditional
 *                  second run sit in a stream or CUDA graph.
 *   k_max          > 0: iteration cap of this call (<= RF_MAX_ITERS); 0: the
 *                  tracker's
 */
typedef struct {
    const float *init_pose_dev;
    float *scale_dev;
    const int *run_flag_dev;
    int k_max;
    int reserved;
} rf_track_options;
rf_status pfo_track_frame_ex_async(rf_tracker tr, const float *depth_dev, const float *prev_depth_dev,
                                   const rf_intrinsics *K, const float *prev_pose_dev, float *out_pose_dev,
                                   rf_frame_stats *stats_dev, const rf_track_options *opt, void *stream);
/*
 * pfo_track_frame -- pfo_track_frame_async with host poses: copies
 * prev_pose in, runs, synchronises the stream and writes out_pose (host) and
 * stats_host (may be NULL).  Returns the frame's device status.
 */
rf_status pfo_track_frame(rf_tracker tr, const float *depth_dev, const float *prev_depth_dev,
                          const rf_intrinsics *K, const rf_pose *prev_pose, rf_pose *out_pose,
                          rf_frame_stats *stats_host, void *stream);
/* Status written by the last finished frame (synchronises the tracker's state copy). */
rf_status rf_tracker_last_status(rf_tracker tr);

/*
 * Launch configuration of the persistent PFO kernel (a tracker's own frames, or a
 * batch).  The work split and the lookup group regroup the FP32 partial sums of
 * the fitness, so different configurations agree to rounding, not bit for bit;
 * one configuration always gives the same results.
 */
typedef struct {
    int ctas_per_sm;  /* resident CTAs of 256 threads per SM, 0 = as many as fit      */
    int work_warps;   /* warp count the work split targets (about 16 units per warp):
                         1 .. 7296; the default 3648                                   */
    int group;        /* lookups per lane whose loads are in flight together: 4, 6 or 8
                         (0 = 6); nearest-voxel sampling ignores it                     */
    float ms;         /* measured PFO kernel time of the chosen configuration (autotune) */
} rf_launch_config;
/* Set / read the configuration of a tracker's own frames (default {0, 3648, 6}). */
rf_status rf_tracker_set_config(rf_tracker tr, const rf_launch_config *cfg);
rf_status rf_tracker_get_config(rf_tracker tr, rf_launch_config *cfg);
/*
 * rf_tracker_autotune -- times the persistent kernel on one frame
 * (pfo_track_frame_async's inputs) for candidate configurations -- first CTAs
 * per SM x work warps {1824, 3648, 7296} with groups of 6, then groups of 4
 * and 8 at the best of those -- keeps the fastest as the tracker's
 * configuration and returns it (ms = its kernel time).  The tracker's r_0 is
 * restored; nothing else of the tracker's state changes.  Synchronous.
 */
rf_status rf_tracker_autotune(rf_tracker tr, const float *depth_dev, const float *prev_depth_dev,
                              const rf_intrinsics *K, const float *prev_pose_dev, rf_launch_config *chosen,
                              void *stream);

/* ------------------------------------------------------------ sequence --- */
/*
 * Sequence mode: the tracker keeps the previous depth frame and pose on the
 * device.  rf_sequence_start fuses frame 0 at the given pose; each
 * rf_sequence_step tracks the next frame against the previous one
 * (pfo_track_frame_async), fuses it at the tracked pose (tsdf_integrate) and
 * makes it the previous frame.
 *   depth          float[H * W]; on the host if depth_on_host != 0 (copied in
 *                  on `stream` from the caller's buffer, ideally pinned), else
 *                  on the device
 *   out_pose_host  host rf_pose (may be NULL); when given the call
 *                  synchronises the stream before returning
 *   out_pose_dev   device float[7] (may be NULL)
 *   stats_dev      device rf_frame_stats (may be NULL)
 */
rf_status rf_sequence_start(rf_tracker tr, const float *depth, int depth_on_host, const rf_intrinsics *K,
                            const rf_pose *pose, void *stream);
rf_status rf_sequence_step(rf_tracker tr, const float *depth, int depth_on_host, const rf_intrinsics *K,
                           rf_pose *out_pose_host, float *out_pose_dev, rf_frame_stats *stats_dev, void *stream);

/* ------------------------------------------------------------------ batch --- */
/*
 * A batch steps up to RF_MAX_BATCH independent sequences (trackers in sequence
 * mode, each with its own volume, template, schedule and frame size) by one
 * frame per rf_batch_step: ONE persistent kernel runs the PFO iterations of
 * every sequence (work units of all sequences share the grid; a sequence that
 * has stopped takes no further work), then each frame is fused.  All trackers
 * must use the same volume dtype and the same RF_NEAREST / RF_COMPENSATED
 * flags.  The trackers' depth and pose rings (two slots) hold the frames:
 * frame f of sequence i lives in slot f % 2.
 *   rf_batch_depth_slot  device address where the caller writes frame f of
 *                        sequence i (float[H_i * W_i]) before the step for f
 *   rf_batch_start       fuse the slot-0 frames at the given host poses
 *   rf_batch_step        track the frames of slot `parity` against slot
 *                        1 - parity and fuse them; use_graph != 0 replays a
 *                        CUDA graph captured on first use for this parity and
 *                        launch configuration (capture happens on an internal
 *                        stream; the graph is launched on `stream`)
 *   rf_batch_pose_dev    device float[7]: the pose of sequence i in slot parity
 *   rf_batch_autotune    times the PFO kernel of the frames currently in slot
 *                        `parity` for the candidate configurations of
 *                        rf_tracker_autotune (CTAs per SM, work warps, lookup
 *                        group), keeps the fastest and returns it (ms); inputs
 *                        and tracker state are restored, the volumes are not
 *                        touched
 * Asynchronous except rf_batch_create / rf_batch_autotune.
 */
#define RF_MAX_BATCH 16
typedef struct rf_batch_s *rf_batch;
rf_status rf_batch_create(const rf_tracker *trackers, int n, const rf_intrinsics *K, rf_batch *out);
void rf_batch_destroy(rf_batch b);
rf_status rf_batch_depth_slot(rf_batch b, int i, int parity, float **depth_dev);
rf_status rf_batch_pose_dev(rf_batch b, int i, int parity, float **pose_dev);
rf_status rf_batch_start(rf_batch b, const rf_pose *poses_host, void *stream);
rf_status rf_batch_step(rf_batch b, int parity, int use_graph, void *stream);
rf_status rf_batch_autotune(rf_batch b, int parity, rf_launch_config *chosen, void *stream);
rf_status rf_batch_set_config(rf_batch b, const rf_launch_config *cfg);
/* Per-sequence frame statistics of the last step (device rf_frame_stats[n]). */
rf_status rf_batch_stats_dev(rf_batch b, rf_frame_stats **stats_dev);

/* Test hook: make block 0 of the next persistent launch leave without arriving
 * at its first grid barrier, with barrier waits limited to timeout_ms; the
 * other blocks then give up and the frame reports RF_ERR_TIMEOUT.  Exercises
 * the failure path without faulting or hanging the GPU. */
rf_status rf_tracker_debug_skip_barrier(rf_tracker tr, int enable, int timeout_ms);

#ifdef __cplusplus
}
#endif
#endif /* ROSEFUSION_H */
