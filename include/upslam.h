/*
 * upslam.h -- C ABI of the GB300 (sm_103a) UPSLAM per-sweep hot path.
 *
 * The library implements the data-parallel path of UPSLAM: Union of Panoramas
 * SLAM (Cowley, Miller, Taylor; arXiv 2101.00585):
 *   1. spherical projection of a lidar sweep into a panoramic depth image with a
 *      deterministic z-buffer                                  (Sec. III-A)
 *   2. per-pixel normals from two image neighbours             (Sec. III-A)
 *   3. point-to-plane ICP over projective correspondences
 *      filtered by the similarity test Omega_{d,theta}         (Sec. III-B, Eq. 1)
 *   4. keyframe update: weighted per-pixel average with a
 *      sample count saturated at 10, gated by registration quality (Sec. III-C)
 *
 * Conventions
 * -----------
 * - Every pointer named d_* is DEVICE memory owned by the caller.  The library
 *   allocates nothing and keeps no state between calls.  Host pointers (the
 *   parameter structs) are read during the call only.
 * - "float4" arrays are 16-byte aligned arrays of 4 floats; "half4" arrays are
 *   8-byte aligned arrays of 4 IEEE binary16 values.
 * - Panoramas are row-major [rows][cols].  Row 0 is the top edge (elevation
 *   el_top); column 0 starts at azimuth +pi and columns advance clockwise.
 *   A point p falls in pixel (row, col) by the FP32 binning rule below.
 * - A pose is 12 doubles, row-major [R | t] (3x4), mapping sweep coordinates
 *   to keyframe coordinates (T = T_kf<-sweep, the T of Eq. 1 that acts on the
 *   sweep point s2).
 * - Calls are asynchronous and ordered on the given CUDA stream (a
 *   cudaStream_t passed as void*; NULL = the legacy default stream).  Results
 *   that the device decides (pose, convergence, inlier counts) stay in device
 *   memory so a sequence of calls can be captured in a CUDA graph.
 * - Errors: argument errors are found on the host before any launch and
 *   return UPSLAM_ERR_INVALID_ARG; a failed launch returns UPSLAM_ERR_CUDA.
 *   Conditions found on the device (degenerate normal equations, a wait that
 *   timed out) are written to the stats record.  No C++ exception crosses this
 *   boundary.
 *
 * FP32 binning rule (shared definition; the kernels and any checker must apply
 * these IEEE round-to-nearest operations in this order, without fused
 * multiply-add):
 *   xy2 = x*x + y*y;  r = sqrt(xy2 + z*z);  reject unless r_min <= r <= r_max
 *   az = atan2p(y, x);  el = atan2p(z, sqrt(xy2))
 *   fc = (PI_F - az) * s_az;  fr = (el_top - el) * s_el
 *   reject unless 0 <= fr < rows;  row = floor(fr);  col = floor(fc) (col == cols -> 0)
 * where atan2p reduces atan2 to atan(t), t = min/max in [0,1], evaluated as
 * t * P(t*t) with the 8-term polynomial of Abramowitz & Stegun 4.4.49
 * (Horner, separate multiply and add), then a = pi/2 - a if |y| > |x|,
 * a = pi - a if x < 0, a = -a if y < 0 (-0 counts as +0; atan2p(0,0) = 0).
 * A transformed point is p = ((r00*x + r01*y) + r02*z) + t0 (etc.) with the
 * pose rounded to FP32; the inverse is q = (r00*dx + r10*dy) + r20*dz with
 * d = s - t.  The z-buffer key of point i is (bits(r) << 32) | i and the
 * smallest key wins, so winners are unique and independent of thread order.
 */
#ifndef UPSLAM_H
#define UPSLAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    UPSLAM_OK = 0,
    UPSLAM_ERR_INVALID_ARG = 1,
    UPSLAM_ERR_CUDA = 2,
    UPSLAM_ERR_DEGENERATE = 3,   /* too few inliers or a Cholesky pivot <= pivot_eps * max diag */
    UPSLAM_ERR_NOT_CONVERGED = 4,
    UPSLAM_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    UPSLAM_ERR_UNSUPPORTED = 6,  /* e.g. a cooperative launch the device cannot host */
    UPSLAM_ERR_CAPACITY = 7      /* the request needs more than a fixed-size scratch array holds */
} upslam_status;

/* Storage precision of normals and sample counts. */
typedef enum {
    UPSLAM_F32 = 0, /* float4 (nx, ny, nz, w) */
    UPSLAM_F16 = 1  /* half4  (nx, ny, nz, w) */
} upslam_precision;

/* Panorama geometry.  The FP32 values are the definition (computed once by the
 * caller, e.g. s_az = cols / 2pi rounded to FP32). */
typedef struct {
    int32_t rows, cols;
    float el_top; /* elevation of the top edge of row 0, radians */
    float s_az;   /* columns per radian of azimuth */
    float s_el;   /* rows per radian of elevation */
    float r_min, r_max; /* accepted range interval, metres */
} upslam_pano;

/* Normal estimation (Sec. III-A).  A neighbour is unusable when
 * |r_nb - r| > jump_rel * r + jump_abs (FP32); a normal is invalid when
 * |a x b| < min_cross * |a| |b|. */
typedef struct {
    float jump_rel, jump_abs, min_cross;
} upslam_normal_params;

/* Point-to-plane error of Eq. 1: squared (Gauss-Newton on sum r^2), or the
 * absolute value printed in Eq. 1, minimised by iteratively reweighted least
 * squares: each correspondence weighs w = 1 / max(|r|, loss_delta). */
typedef enum { UPSLAM_LOSS_L2 = 0, UPSLAM_LOSS_L1 = 1 } upslam_loss;

/* ICP (Sec. III-B, Eq. 1).  Omega keeps a correspondence when the points are
 * within d_max metres and the normals' cosine is >= cos_theta_max.  The paper
 * gives no threshold; a coarse-to-fine gate (wide while a large initial error
 * is taken out, then narrow) is selected by coarse_iters > 0: Gauss-Newton
 * steps 0 .. coarse_iters - 1 of one multi-step call gate with d_max, later
 * steps with d_max_fine.  coarse_iters = 0 gates every step with d_max.  A
 * single upslam_icp_step always gates with d_max. */
typedef struct {
    float d_max, cos_theta_max;
    int32_t max_iters;   /* iterations of upslam_icp */
    int32_t min_inliers; /* fewer inliers -> degenerate */
    double eps_rot, eps_trans; /* converged when |omega| < eps_rot and |v| < eps_trans */
    double pivot_eps;          /* Cholesky pivot threshold relative to the largest diagonal */
    int32_t loss;              /* upslam_loss */
    float loss_delta;          /* metres; > 0 with UPSLAM_LOSS_L1 */
    int32_t coarse_iters;      /* >= 0; steps gated with d_max before switching to d_max_fine */
    float d_max_fine;          /* metres; > 0 when coarse_iters > 0 */
} upslam_icp_params;

/* Keyframe update (Sec. III-C). */
typedef struct {
    float d_max, cos_theta_max; /* similarity gate for averaging a sample in */
    float w_max;                /* sample count saturation (10 in the paper) */
    float accept_quality;       /* fuse only when inliers / valid >= accept_quality */
} upslam_fuse_params;

/* ICP result record, written by the device. */
typedef struct {
    double A[21];   /* upper triangle of sum w J^T J at the last linearisation, row-major */
    double b[6];    /* sum w J^T r */
    double sse;     /* sum w r^2 (w = 1 for UPSLAM_LOSS_L2) */
    int64_t inliers;
    int64_t valid;  /* sweep pixels holding a point */
    int32_t status; /* upslam_status of the last step */
    int32_t converged;
    double xi[6];   /* last update (omega, v) */
    int32_t iters;  /* Gauss-Newton steps taken by upslam_icp */
    int32_t accepted; /* set by upslam_fuse: 1 when the sweep was fused */
} upslam_icp_stats;

/* A sweep after projection and normal estimation. */
typedef struct {
    upslam_pano pano;
    const float *d_pix;  /* float4 [rows*cols]: the pixel's point (x, y, z, valid) */
    const void *d_nrm;   /* float4 or half4 [rows*cols]: (nx, ny, nz, valid) */
    int32_t nrm_precision; /* upslam_precision of d_nrm */
} upslam_sweep;

/* A keyframe panorama (Sec. III: depth plus surface normals, and the
 * per-pixel sample count of Sec. III-C).  Empty pixels have depth 0, w 0. */
typedef struct {
    upslam_pano pano;
    float *d_depth;      /* float [rows*cols]: range along the pixel-centre ray */
    void *d_nw;          /* float4 or half4 [rows*cols]: (nx, ny, nz, w) */
    int32_t precision;   /* upslam_precision of d_nw */
    const float *d_dirs; /* direction table from upslam_pano_dirs */
} upslam_keyframe;

/* Size in floats of a panorama's direction table (Sec. III-A panoramas): 2*rows + 2*cols. */
size_t upslam_pano_dirs_floats(const upslam_pano *pp);

/*
 * Direction table of a panorama (Sec. III-A): cos/sin of every row-centre elevation and
 * column-centre azimuth, computed in FP64 and rounded to FP32
 * (d_dirs[2v], d_dirs[2v+1] = cos, sin of el_v; then d_dirs[2*rows + 2u],
 * [.. + 1] = cos, sin of az_u).  The FP32 point of pixel (v, u) at depth d is
 * d * (ce*ca, ce*sa, se).  Call once per panorama geometry.
 */
upslam_status upslam_pano_dirs(const upslam_pano *pp, float *d_dirs, void *stream);

/*
 * Spherical projection with a deterministic z-buffer (Sec. III-A).
 * d_pts: float4 [n] points (x, y, z, valid); invalid (valid == 0) points are skipped.
 * d_pose12: optional transform applied first (NULL = identity).
 * d_zbuf: uint64 [rows*cols] scratch that must hold all-ones on entry; it is
 *   left all-ones on return (each pixel is reset as it is resolved).
 * Outputs: d_depth [rows*cols] range of the nearest point (0 if empty),
 *   d_idx [rows*cols] its index (-1 if empty), and, if d_pix != NULL,
 *   d_pix float4 [rows*cols] = (x, y, z, 1) of that input point as given.
 */
upslam_status upslam_project(const float *d_pts, int32_t n, const double *d_pose12, const upslam_pano *pp,
                             uint64_t *d_zbuf, float *d_depth, int32_t *d_idx, float *d_pix, void *stream);

/* Keyframe pixel points (Sec. III: a keyframe is a depth panorama) d_pix float4 [rows*cols] = depth * dir
 * (valid = depth > 0). */
upslam_status upslam_unproject(const float *d_depth, const upslam_pano *pp, const float *d_dirs, float *d_pix,
                               void *stream);

/*
 * Per-pixel normals (Sec. III-A): n = a x b, a toward column + 1 (wrapping),
 * b toward row + 1; an unusable neighbour is replaced by the opposite one with
 * the vector's sign flipped.  Normalised, oriented toward the sensor.
 * d_pix float4 [rows*cols] pixel points, d_depth [rows*cols] their ranges.
 * d_nrm float4 or half4 [rows*cols] = (nx, ny, nz, valid).
 */
upslam_status upslam_normals(const float *d_pix, const float *d_depth, const upslam_pano *pp,
                             const upslam_normal_params *np, void *d_nrm, int32_t nrm_precision, void *stream);

/*
 * Edge-avoiding a-trous smoothing of a normal image (Sec. III-A names the
 * a-trous wavelet filter of Dammertz et al. 2010 for the noisy cross-product
 * normals; Sec. III-B notes the smoothing aids ICP convergence).  Level
 * l = 0 .. levels-1 sets each valid pixel p to the normalised sum over the 5 x 5
 * taps q = p + 2^l (dy, dx), dy, dx in -2..2, of
 *   h(dy) h(dx) exp(-|N_p - N_q|^2 / sigma_n^2 - (N_p . (P_q - P_p))^2 / (sigma_x |P_p|)^2) N_q,
 * h = [1, 4, 6, 4, 1] / 16, over valid taps; columns wrap, rows outside the
 * image are skipped; invalid pixels stay invalid (written as zeros).
 */
typedef struct {
    int32_t levels; /* 0 .. 6, with 2^levels <= cols; 0 copies the input */
    float sigma_n;  /* normal-difference scale, > 0 */
    float sigma_x;  /* tangent-plane distance scale relative to the range, > 0 */
} upslam_atrous_params;

/*
 * A-trous smoothing arguments (Sec. III-A).
 * d_pix float4 [rows*cols] pixel points (16-byte aligned); d_nrm_in and
 * d_nrm_out float4 or half4 [rows*cols] = (nx, ny, nz, valid) in `precision`;
 * d_tmp a scratch image of the same size, needed when levels >= 2 (else may be
 * NULL).  The three normal buffers must not alias.  One launch per level on
 * `stream`; the result is in d_nrm_out.  Invalid arguments return
 * UPSLAM_ERR_INVALID_ARG before any launch.
 */
upslam_status upslam_atrous_normals(const upslam_pano *pp, const float *d_pix, const void *d_nrm_in,
                                    void *d_nrm_out, void *d_tmp, int32_t precision,
                                    const upslam_atrous_params *ap, void *stream);

/* Workspace bytes that upslam_icp_step / upslam_icp (Sec. III-B, Eq. 1) need for this keyframe. */
size_t upslam_icp_workspace_bytes(const upslam_keyframe *kf);

/*
 * One Gauss-Newton step of Eq. 1 (squared point-to-plane error).  Every
 * keyframe pixel holding a sample is put at d * dir, taken into the sweep frame
 * by T^-1 and binned into the sweep panorama; the sweep pixel's point s2 and the
 * keyframe point s1 form a correspondence kept by Omega.  The normal equations
 * J^T J xi = -J^T r (J = [p x n, n], p = T s2, left update) are reduced on the
 * device, solved by an FP64 Cholesky, and d_pose12 <- exp(xi^) d_pose12.
 * A degenerate system leaves d_pose12 unchanged (stats.status = 3).
 * d_ws: workspace of upslam_icp_workspace_bytes(kf) bytes; it must be zeroed
 * once before its first use and is left reusable.
 */
upslam_status upslam_icp_step(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_pose12,
                              const upslam_icp_params *ip, upslam_icp_stats *d_stats, void *d_ws, size_t ws_bytes,
                              void *stream);

/*
 * Up to ip->max_iters Gauss-Newton steps of Eq. 1 (Sec. III-B) in ONE persistent cooperative launch
 * (one CTA per SM; a bounded grid-wide barrier per step).  Each CTA adds its
 * share of the step's J^T J, J^T r and counts into integer accumulators in the
 * workspace as exact fixed-point numbers, so the totals do not depend on the
 * order of the CTAs; every CTA reads them and solves in FP64, getting the same
 * pose.  Stops early on convergence or a degenerate system.  stats.iters counts
 * the steps taken.  A barrier that waits longer than about a second gives up and
 * sets stats.status = 5; the workspace must then be zeroed again before reuse.
 */
upslam_status upslam_icp(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_pose12,
                         const upslam_icp_params *ip, upslam_icp_stats *d_stats, void *d_ws, size_t ws_bytes,
                         void *stream);

/*
 * Test support for the bounded grid-barrier waits of the persistent launch
 * (the paper has no counterpart).  Runs upslam_icp with every barrier wait
 * limited to wait_cycles SM clock cycles (1000 .. 4e9) and with CTA 0 not
 * arriving at the first Gauss-Newton barrier, so that barrier cannot complete:
 * every CTA's wait gives up, the launch ends, and stats.status becomes
 * UPSLAM_ERR_TIMEOUT; the pose is left unchanged.  This is how the tests show
 * that a wait that never completes ends in a status instead of a hang, and that
 * the device stays usable afterwards.  Zero the workspace again before its next
 * use (its barrier counter is left mid-count).
 */
upslam_status upslam_icp_wait_probe(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_pose12,
                                    const upslam_icp_params *ip, upslam_icp_stats *d_stats, void *d_ws,
                                    size_t ws_bytes, long long wait_cycles, void *stream);

/*
 * Registration of one sweep in one launch: the motion prior (Sec. IV-F
 * footnote), then upslam_icp, then the motion update.
 * prior = 0: start from d_pose12 as given (d_prev, d_motion unused);
 *         1: zero-velocity prior, start from d_prev;
 *         2: zero-acceleration prior, start from d_prev * d_motion (rotation
 *            re-orthonormalised).
 * With prior >= 1, on return d_motion = d_prev^-1 * pose and d_prev = pose
 * (the registered pose), so the next sweep's call needs no host step; to
 * start a new keyframe at this sweep set d_prev to the identity.
 * d_pose12 receives the registered pose in every mode.  Workspace, stats and
 * stopping rules as upslam_icp.
 */
upslam_status upslam_register(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_prev, double *d_motion,
                              double *d_pose12, int32_t prior, const upslam_icp_params *ip,
                              upslam_icp_stats *d_stats, void *d_ws, size_t ws_bytes, void *stream);

/*
 * The whole registration and keyframe update of one sweep (Sec. III-B, III-C) in ONE persistent
 * launch: upslam_register followed by upslam_fuse with the registered pose
 * (gated by the same acceptance test), reusing the keyframe samples the ICP
 * staged in shared memory.  Arguments as those two calls; ip->max_iters >= 1.
 * stats.accepted records whether the sweep was fused.
 */
upslam_status upslam_track(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_prev, double *d_motion,
                           double *d_pose12, int32_t prior, const upslam_icp_params *ip,
                           const upslam_fuse_params *fp, upslam_icp_stats *d_stats, void *d_ws, size_t ws_bytes,
                           uint64_t *d_zbuf_kf, void *stream);

/*
 * Keyframe update (Sec. III-C) with T = d_pose12.  Runs only when d_stats is
 * NULL or the registration was accepted (status 0 and inliers / valid >=
 * accept_quality); stats.accepted records the outcome.  Averaging: every
 * keyframe pixel with w > 0 is projected onto the sweep image and, if Omega
 * keeps the pair, d <- (w d + |T s2|)/(w + 1), n <- unit(w n + R m),
 * w <- min(w + 1, w_max).  Hole fill: every sweep pixel with a point and a
 * normal is binned (with T) into the keyframe; each empty keyframe pixel takes
 * its nearest sample (z-buffer on (range, sweep pixel index)) with w = 1.
 * d_zbuf_kf: uint64 [kf rows*cols] scratch, all-ones on entry and on return.
 */
upslam_status upslam_fuse(const upslam_keyframe *kf, const upslam_sweep *sw, const double *d_pose12,
                          const upslam_fuse_params *fp, upslam_icp_stats *d_stats, uint64_t *d_zbuf_kf,
                          void *stream);

/*
 * Allocation-free ICP.  The paper has no counterpart: this exists for callers
 * that cannot allocate device memory once they are running, such as a robot's
 * real-time control loop (a cudaMalloc can block on a driver lock and miss the
 * sweep deadline), a plugin whose host runtime owns the device allocator, or
 * code that may only use memory fixed at load time.  It runs exactly what
 * upslam_icp runs, but its workspace is a static device array inside the
 * library (upslam_icp_noalloc_capacity_bytes() = 561152 bytes, 548 KiB: the
 * control block plus 2048 per-CTA records, enough for devices of up to 1024
 * SMs) instead of d_ws.  The caller still provides the keyframe, sweep, pose
 * and stats buffers.
 * - Allocates nothing: no cudaMalloc / cudaFree, no allocating library call.
 *   The scratch's barrier counters are cleared with cudaMemsetAsync on the
 *   stream at every call.
 * - The first call on a device is a warm-up: it looks up the array's device
 *   address (cudaGetSymbolAddress) with that device current, and under lazy
 *   module loading (the CUDA default) that lookup is what loads the library's
 *   device code and its array onto the device, which can allocate and take a
 *   driver lock.  Make that first call during set-up, before the real-time
 *   loop and before any stream capture; later calls allocate nothing.  The
 *   array then stays on every GPU the library was used on until the process
 *   exits.
 * - Returns UPSLAM_ERR_CAPACITY when the launch this device needs would not fit
 *   the array (more than 1024 SMs).
 * - Every call shares the one array: calls that overlap on the GPU (other
 *   streams, other threads) race and corrupt each other's results; serialise
 *   them on one stream.
 */
size_t upslam_icp_noalloc_capacity_bytes(void);
upslam_status upslam_icp_noalloc(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_pose12,
                                 const upslam_icp_params *ip, upslam_icp_stats *d_stats, void *stream);

/*
 * Motion prior for the ICP initial guess (Sec. IV-F footnote: a zero-velocity
 * prior by default, a zero-acceleration prior as the alternative).
 * upslam_predict_pose: d_T_out = d_T_prev * d_motion (d_motion NULL: the
 *   zero-velocity prior, d_T_out = d_T_prev).  Poses are 12 doubles [R | t];
 *   the product's rotation is re-orthonormalised.  d_T_out may alias d_T_prev.
 * upslam_update_motion: d_motion = d_T_prev^-1 * d_T (the last inter-sweep motion).
 * One thread each, FP64, stream-ordered.
 */
upslam_status upslam_predict_pose(const double *d_T_prev, const double *d_motion, double *d_T_out, void *stream);
upslam_status upslam_update_motion(const double *d_T_prev, const double *d_T, double *d_motion, void *stream);

/*
 * Batched persistent ICP (the grid search of Sec. III-C carried to full
 * registrations): one sweep against n_kf keyframes of any sizes, with n_hyp
 * initial poses per keyframe, i.e. n_kf * n_hyp problems (problem
 * p = kf * n_hyp + h), all in ONE cooperative launch.  Every problem follows
 * upslam_icp (Eq. 1, FP64 solve, same stopping rules); all active problems
 * advance one Gauss-Newton step at a time and a keyframe sample is evaluated
 * for all hypotheses of its keyframe at once.
 * d_kfs: device array [n_kf] of keyframe views; kfs: the same array on the host
 *   (sizes and validation).  n_kf <= 256, n_kf * n_hyp <= 1024.
 * d_poses: [n_kf * n_hyp][12] FP64, initial poses in, registered poses out.
 * d_stats: [n_kf * n_hyp] records.
 * d_ws: upslam_icp_batched_workspace_bytes(...) bytes (256-byte aligned); its
 *   first 8 bytes must be zero before the first use (arrival counter).
 * tiles: CTA width (256 or 512) and keyframe chunk (a multiple of it), or NULL
 *   for 512 / 512; the package's autotuner picks them per device and shape.
 */
typedef struct {
    int32_t threads; /* threads per CTA: 256 or 512 */
    int32_t chunk;   /* keyframe pixels per chunk, a multiple of threads */
} upslam_batch_tiles;

size_t upslam_icp_batched_workspace_bytes(const upslam_keyframe *kfs, int32_t n_kf, int32_t n_hyp,
                                          const upslam_batch_tiles *tiles);
upslam_status upslam_icp_batched(const upslam_keyframe *d_kfs, const upslam_keyframe *kfs, int32_t n_kf,
                                 const upslam_sweep *sw, int32_t n_hyp, double *d_poses, const upslam_icp_params *ip,
                                 upslam_icp_stats *d_stats, void *d_ws, size_t ws_bytes,
                                 const upslam_batch_tiles *tiles, void *stream);

/* Sweep buffers written by upslam_track_scan (the outputs of upslam_project and
 * upslam_normals).  d_zbuf is all ones at rest and left so. */
typedef struct {
    upslam_pano pano;
    uint64_t *d_zbuf;      /* [rows*cols], 8-byte aligned */
    float *d_depth;        /* [rows*cols] */
    int32_t *d_idx;        /* [rows*cols] */
    float *d_pix;          /* float4 [rows*cols], 16-byte aligned */
    void *d_nrm;           /* float4 or half4 [rows*cols] */
    int32_t nrm_precision; /* UPSLAM_F32 or UPSLAM_F16 */
} upslam_sweep_buffers;

/*
 * One whole sweep (Sec. III-A to III-C) in ONE persistent cooperative launch: projection with the
 * z-buffer, resolve and normals of the scan d_pts4 (float4 [n_pts], 16-byte
 * aligned) into the sweep buffers (as upslam_project with no pose followed by
 * upslam_normals, with the same results), then everything upslam_track does.
 * Three extra grid barriers separate projection, resolve and normals; the
 * keyframe staging runs before the last so its wait is hidden.  Arguments and
 * errors as upslam_project, upslam_normals and upslam_track.
 */
upslam_status upslam_track_scan(const upslam_keyframe *kf, const float *d_pts4, int32_t n_pts,
                                const upslam_sweep_buffers *sb, const upslam_normal_params *np, double *d_prev,
                                double *d_motion, double *d_pose12, int32_t prior, const upslam_icp_params *ip,
                                const upslam_fuse_params *fp, upslam_icp_stats *d_stats, void *d_ws,
                                size_t ws_bytes, uint64_t *d_zbuf_kf, void *stream);

/*
 * Loop-closure grid search (Sec. III-C): each candidate pose gets a cheap
 * projective score on a subsampled keyframe, and the winner is refined by ICP
 * at full resolution afterwards.  A candidate's score is its number of
 * inliers of the ICP association (keyframe pixel -> sweep pixel under T^-1,
 * the FP32 binning rule, Omega with ip->d_max and ip->cos_theta_max) over the
 * keyframe pixels (stride i, stride j).
 *
 * d_poses: FP64 [n][12] candidates, row-major [R | t] (keyframe <- sweep).
 * d_scores: u64 [n] (overwritten; 8-byte aligned).  d_best: int32 [1], the
 * first candidate with the largest score.  d_best_pose12: FP64 [12] copy of
 * that candidate, or NULL.  Two launches (scores, winner) after a memset of
 * d_scores, all on `stream`; n <= 2097120.  Invalid arguments return
 * UPSLAM_ERR_INVALID_ARG before any launch.
 */
upslam_status upslam_grid_score(const upslam_keyframe *kf, const upslam_sweep *sw, const double *d_poses, int32_t n,
                                int32_t stride, const upslam_icp_params *ip, uint64_t *d_scores, int32_t *d_best,
                                double *d_best_pose12, void *stream);

/* Grid-search candidates (Sec. III-C): d_poses[i] = exp(xi_i^) * center (FP64 [n][12]) for FP32 twists
 * d_xi [n][6] = (omega, v), e.g. a grid of offsets around the current estimate. */
upslam_status upslam_grid_candidates(const double *d_center12, const float *d_xi, int32_t n, double *d_poses,
                                     void *stream);

/*
 * Keyframe mutual consistency check (Sec. III-C: run whenever keyframes are
 * switched, it filters moving objects from the map).  A sample of keyframe A
 * is removed when keyframe B saw through it: binned into B (FP32 rule, T_ab =
 * pose of B in A rounded to FP32, range r), B holds a depth there and every
 * depth-holding pixel of the 3 x 3 neighbourhood (columns wrapped, rows
 * clipped) lies beyond (rel * r + abs_m) + r (FP32).  B's samples are checked
 * against A with T_ba = [R^T | -R^T t] (FP64, t' summed in the order
 * -((R_0i t_0 + R_1i t_1) + R_2i t_2)).  Both directions read the unmodified
 * depths; then the flagged pixels of both keyframes are emptied (depth 0,
 * normal and count 0).
 *
 * d_ws: upslam_consistency_workspace_bytes(kf_a, kf_b) bytes, 256-byte aligned;
 * it keeps the flags (one byte per pixel: A's at offset 0, B's at the next
 * multiple of 256 after A's).  d_removed2: int64 [2] = samples removed from A and
 * B (overwritten), or NULL.  The keyframes must be distinct buffers.  Two
 * launches on `stream`; invalid arguments return UPSLAM_ERR_INVALID_ARG before
 * any launch.
 */
size_t upslam_consistency_workspace_bytes(const upslam_keyframe *kf_a, const upslam_keyframe *kf_b);
upslam_status upslam_keyframe_consistency(const upslam_keyframe *kf_a, const upslam_keyframe *kf_b,
                                          const double *d_T_ab12, float rel, float abs_m, void *d_ws, size_t ws_bytes,
                                          int64_t *d_removed2, void *stream);

/*
 * Pose-proposal network (learned initial guess).  The paper has no learned
 * component: it relies on a zero-velocity or zero-acceleration prior (Sec. IV-F
 * footnote), and a large motion is left to the registration itself.  This
 * network is a design addition that predicts the relative pose of a
 * keyframe/sweep pair so ICP (Sec. III-B) can start near it; the caller gates
 * the result by the ICP residual and falls back to the plain prior.
 *
 * Input: BF16 NHWC [batch][64][256][8]: keyframe (depth / scale, nx, ny, nz)
 * then sweep (the same), each from upslam_downsample.  Output: FP32 [batch][6]
 * xi = (omega, v), the keyframe-from-sweep pose as exp(xi^).
 * Parameters: one FP32 array of upslam_cnn_param_count() values in the order
 * w0 b0 w1 b1 w2 b2 w3 b3 wf bf (conv weights [C_out][3][3][C_in] for
 * 8->32->64->128->128 channels, head wf [6][128]).  Convolutions run as BF16
 * tensor-core GEMMs (tcgen05.mma, FP32 accumulators in tensor memory).
 * d_ws: upslam_cnn_workspace_bytes(batch) bytes, 256-byte aligned; it keeps
 *   the activations of the last forward call, which upslam_cnn_backward reads.
 * d_x must be 16-byte aligned.  A null pointer, batch <= 0, a short or
 * misaligned workspace returns UPSLAM_ERR_INVALID_ARG before any launch.
 * Every wait of the tensor-core kernels is bounded: one that gives up (the
 * tensor cores never signalled) stops its CTA, leaves that call's outputs
 * incomplete and stores a nonzero int32 at byte upslam_cnn_error_offset(batch)
 * of d_ws.  The library never clears that word: zero the workspace once after
 * allocating it and read the word at the caller's next synchronisation.
 */
size_t upslam_cnn_param_count(void);
size_t upslam_cnn_workspace_bytes(int32_t batch);
/*
 * Where the pose network (not in the paper) keeps its tensors inside a workspace for `batch` pairs, so a
 * caller can inspect them after upslam_cnn_forward / upslam_cnn_backward (e.g. to check one layer at a
 * time).  Writes 16 byte offsets and returns upslam_cnn_workspace_bytes(batch) (0 for batch <= 0 or a
 * null array):
 *   [l]      BF16 conv weights of layer l, [C_out][3 * 3 * C_in] ((ky * 3 + kx) * C_in + ci), l = 0..3;
 *   [4 + l]  BF16 output of layer l after its ReLU, NHWC [batch][64 >> (l+1)][256 >> (l+1)][C_out];
 *   [8 + l]  BF16 gradient of the loss at layer l's pre-activation (ReLU mask applied), same shape;
 *   [12]     FP32 pooled features [batch][128]; [13] their gradient; [14] FP32 outputs [batch][6];
 *   [15]     the int32 error word (upslam_cnn_error_offset).
 */
size_t upslam_cnn_workspace_layout(int32_t batch, size_t *offsets16);
size_t upslam_cnn_error_offset(int32_t batch);
upslam_status upslam_cnn_forward(const float *d_params, const void *d_x, int32_t batch, float *d_out, void *d_ws,
                                 size_t ws_bytes, void *stream);
/*
 * Test support for the bounded tensor-core waits (the paper has no
 * counterpart): upslam_cnn_forward with every mbarrier wait of the first
 * layer's GEMM limited to timeout_ns nanoseconds (1000 .. 2e9) and its MMA
 * thread not signalling its first accumulator as full, so the epilogue's wait
 * cannot end: the CTAs give up, drain the copies and MMAs they issued, free
 * their tensor memory and stop, and the error word at
 * upslam_cnn_error_offset(batch) becomes nonzero.  The outputs of the call are
 * incomplete; the device stays usable.
 */
upslam_status upslam_cnn_forward_wait_probe(const float *d_params, const void *d_x, int32_t batch, float *d_out,
                                            void *d_ws, size_t ws_bytes, unsigned long long timeout_ns,
                                            void *stream);
/* Pose network (not in the paper), backward: loss sum_b sum_i w_i (out - target)^2 / batch into *d_loss and
 * every parameter's gradient into d_grads
 * (overwritten), for the activations of the preceding upslam_cnn_forward on the same workspace. */
upslam_status upslam_cnn_backward(const float *d_params, const void *d_x, int32_t batch, const float *d_out,
                                  const float *d_target, const float *d_wloss6, float *d_grads, float *d_loss,
                                  void *d_ws, size_t ws_bytes, void *stream);
/* Pose network (not in the paper): one Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected for step >= 1)
 * on the FP32 master parameters. */
upslam_status upslam_cnn_adam(float *d_params, const float *d_grads, float *d_m, float *d_v, int32_t step, float lr,
                              void *stream);
/*
 * Pose-network input (not in the paper): downsample a panorama to out_rows x out_cols cells (rows and cols must
 * divide evenly): per cell the mean over pixels holding a sample of
 * (depth / depth_scale, nx, ny, nz), zeros where none, written as BF16 to
 * d_out[cell * c_stride + c_off + 0..3].  d_nrm: float4 or half4
 * (nx, ny, nz, w-or-valid).
 */
upslam_status upslam_downsample(const float *d_depth, const void *d_nrm, int32_t precision, const upslam_pano *pp,
                                int32_t out_rows, int32_t out_cols, float depth_scale, void *d_out, int32_t c_stride,
                                int32_t c_off, void *stream);

/* Poses exp(xi^) (FP64 [n][12], row-major [R | t]) of n FP32 twists xi = (omega, v), e.g. the pose
 * network's outputs (not in the paper), with the left update of the ICP step (Sec. III-B). */
upslam_status upslam_se3_exp(const float *d_xi, int32_t n, double *d_poses, void *stream);

/* Human-readable name of a status code (static storage). */
const char *upslam_status_string(upslam_status s);

/* Library version string. */
const char *upslam_version(void);

#ifdef __cplusplus
}
#endif

#endif /* UPSLAM_H */
