/*
 * rimg.h -- C ABI of the B300 range-image registration library (librimg.so).
 *
 * The library registers LiDAR scans stored as cylindrical range images by
 * multi-scale projective point-to-plane Gauss-Newton, the method of
 * "Revisiting LiDAR Registration and Reconstruction: A Range Image
 * Perspective" (arXiv 2112.02779), Sections 3 and 4.1.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Images are float32, row-major [H][W]; row v is the beam (elevation)
 *    index, column u the azimuth index (Section 3).  Batches of images are
 *    stacked as [n][H][W].  A range <= 0 or not finite marks an invalid pixel.
 *  - All image, table, pose and workspace pointers are DEVICE pointers owned
 *    by the caller, except where a parameter says "host".  The library never
 *    allocates device memory (entry points that need scratch take a caller
 *    workspace whose size is returned by the matching *_workspace_bytes call).
 *  - Poses are float64 row-major 4x4 matrices T that map source-frame points
 *    into the target frame, x = R p + t (Eq. 5).
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream) unless stated otherwise.  Calls return RIMG_OK (0) or a
 *    negative rimg_status; nothing is thrown across the ABI.  On an error no
 *    kernel has been launched unless the code is RIMG_ERR_CUDA.
 *  - Thread safety: calls may be made from several host threads on different
 *    streams if they use different workspaces.
 */
#ifndef RIMG_H
#define RIMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RIMG_MAX_LEVELS 8

typedef enum rimg_status {
  RIMG_OK = 0,
  RIMG_ERR_INVALID_ARG = -1,      /* null pointer, negative count, bad parameter */
  RIMG_ERR_LUT = -2,              /* elevation table not strictly monotone / out of range */
  RIMG_ERR_SIZE = -3,             /* image size incompatible with the pyramid (see rimg_sensor_build) */
  RIMG_ERR_WORKSPACE = -4,        /* workspace too small or not 256-byte aligned */
  RIMG_ERR_CUDA = -5,             /* a CUDA runtime call failed; see rimg_last_error() */
  RIMG_ERR_MISMATCH = -6          /* source and target sensors disagree where they must agree */
} rimg_status;

/* Per-pair status bits written by rimg_icp_step / rimg_register. */
#define RIMG_FLAG_DEGENERATE 1    /* an iteration had < 6 correspondences or an LDL^T pivot
                                     <= 1e-12 * trace(J^T W J); its update was skipped */

/* One pyramid level of a sensor's device tables (filled by rimg_sensor_build;
 * callers treat it as read-only). */
typedef struct rimg_level {
  int H, W;                 /* level size: H >> l, W >> l */
  int n_bins;               /* entries of the inverse elevation table (<= 64 H) */
  int tie_up;               /* 1 when elevation decreases with the row index */
  int bins_exact;           /* 1 when every bin holds at most one row boundary */
  int has_theta;            /* 0 when theta_lut is identically zero */
  float s_lo, s_hi;         /* vertical field of view as sin(elevation) */
  float bin_scale;          /* n_bins / (s_hi - s_lo) */
  float w_over_2pi;         /* W / (2 pi) */
  size_t off_rows;          /* float4[H]: cos phi, sin phi, cos theta_lut, sin theta_lut */
  size_t off_cols;          /* float[W] cos, then (at off_cols + 4W) float[W] sin of 2 pi u / W */
  size_t off_thu;           /* float[H]:  theta_lut[v] * W / (2 pi) */
  size_t off_rank;          /* int[H]:    row of the j-th smallest elevation */
  size_t off_bnd;           /* float[H-1]: sin of the mid-elevation between ranks j, j+1 */
  size_t off_bins;          /* int4[n_bins]: row below / row above the bin's boundary, the
                               boundary (float bits, +inf if none; with tie_up the largest
                               float below it, so that one "s > boundary" test applies the
                               lower-row tie rule), rank at the lower edge */
} rimg_level;

/* A sensor's intrinsics in device form: the elevation table phi_lut and the
 * azimuth-offset table theta_lut of Section 3 (Eq. 1-2), the receiver radius
 * r0, and per-level tables for the strided pyramid of Section 4.1. */
typedef struct rimg_sensor {
  int H, W, levels;
  float r0;
  void* d_tables;           /* device, caller-owned, rimg_sensor_table_bytes() long */
  size_t table_bytes;
  rimg_level level[RIMG_MAX_LEVELS];
} rimg_sensor;

/* Method parameters.  Defaults (rimg_default_params): huber_delta 0.5 m (the
 * outdoor kernel size of Section 6.1), no distance gate, normal_rel_jump 0.1,
 * proj_iters 3, kahan 1, streams 2.  Pairs are independent: each sub-batch of
 * at least 32 pairs runs on its own internal stream forked from and joined
 * back into the caller's stream, and `streams` changes results only through
 * the FP32 summation order (a small sub-batch may split each pair over more
 * blocks to fill the GPU). */
typedef struct rimg_params {
  float huber_delta;        /* pseudo-Huber kernel size (m); <= 0: plain least squares */
  float max_corr_dist;      /* reject pairs with |x - q| > max_corr_dist; <= 0: off */
  float normal_rel_jump;    /* a normal needs |r_nb - r_c| <= normal_rel_jump * r_c, in [0, 0.5) */
  int proj_iters;           /* receiver-offset fixed-point steps when r0 != 0 (1..16) */
  int kahan;                /* 1: Kahan-compensated FP32 accumulation of J^T W J / J^T W e */
  int streams;              /* rimg_register: concurrent sub-batches (internal streams), 1..4 */
  int normal_method;        /* 0: cross product of neighbour pixels (default); 1: PCA of the 3x3
                               window -- Section 4.1 names both (see rimg_normals) */
} rimg_params;

/* Fill *p with the defaults above.  Host only. */
int rimg_default_params(rimg_params* p);

/* Human-readable text of a status code; never NULL. */
const char* rimg_status_string(int code);

/* Text of the last RIMG_ERR_CUDA (per host thread); "" if none. */
const char* rimg_last_error(void);

/* ---------------------------------------------------------------------------
 * Sensor tables (step A1: host, once per sensor).
 *
 * Section 3.1-3.2: the elevation table phi_lut[H] and azimuth offsets
 * theta_lut[H] (radians, HOST float64 arrays) come from the manufacturer.
 * The library precomputes, per pyramid level l (rows 2^l v of the finest
 * tables, W_l = W >> l), separable cos/sin tables for Eq. 1 and an inverse
 * elevation table in sin(elevation) space (the inverse table of Section 3.2,
 * sized so that each bin holds at most one row boundary, which makes one
 * comparison give the exact Eq. 4 argmin; for tables too uneven for 64 H
 * bins the device walks across the row boundaries instead).
 *
 * Requirements: levels in [1, RIMG_MAX_LEVELS]; H >> (levels-1) >= 2;
 * W divisible by 4 << (levels-1); phi_lut finite, strictly monotone, inside
 * (-pi/2, pi/2); |theta_lut| < pi; r0 finite and >= 0.  Otherwise
 * RIMG_ERR_SIZE / RIMG_ERR_LUT / RIMG_ERR_INVALID_ARG.
 *
 * rimg_sensor_build copies the tables into d_tables SYNCHRONOUSLY (blocking
 * cudaMemcpy) and fills *out; it is not meant for the hot path.
 * ------------------------------------------------------------------------- */
int rimg_sensor_table_bytes(int H, int W, int levels, size_t* bytes);
int rimg_sensor_build(int H, int W, int levels, const double* phi_lut, const double* theta_lut,
                      double r0, void* d_tables, size_t table_bytes, rimg_sensor* out);

/* ---------------------------------------------------------------------------
 * Unprojection Pi^-1 (step A2), Eq. 1-2: for each pixel of level `level` of
 * n_images range images range[n][H_l][W_l],
 *   x = r cos(theta) cos(phi) + r0 cos(2 pi u / W_l)
 *   y = r sin(theta) cos(phi) + r0 sin(2 pi u / W_l)
 *   z = r sin(phi),  theta = 2 pi u / W_l + theta_lut[v], phi = phi_lut[v]
 * xyz: float32 [n][3][H_l][W_l] (three planes); invalid pixels get the point of
 * r = 0.  mask (nullable): uint8 [n][H_l][W_l], 1 = valid range.
 * ------------------------------------------------------------------------- */
int rimg_unproject(const rimg_sensor* s, int level, int n_images, const float* range,
                   float* xyz, uint8_t* mask, void* stream);

/* ---------------------------------------------------------------------------
 * Pyramid (step A3), Section 4.1: level l is the finest image strided by 2^l
 * in rows and columns, Omega_l(u, v) = Omega_0(2^l u, 2^l v) (an exact copy;
 * intrinsics stay those of the finest level).
 * in: [n][H][W][channels] float32 with channels 1 (ranges) or 4 (planes);
 * out_levels: HOST array of `levels` device pointers; entry l (l >= 1) receives
 * [n][H >> l][W >> l][channels]; entry 0 is ignored (level 0 is `in`).
 * H and W must be divisible by 2^(levels-1).
 * ------------------------------------------------------------------------- */
int rimg_pyramid(int n_images, int H, int W, int levels, int channels, const float* in,
                 float* const* out_levels, void* stream);

/* ---------------------------------------------------------------------------
 * Normals (step A4), Section 4.1 ("cross product of two neighbor pixels"):
 * at finest-level pixel (u, v) with points P from Eq. 1,
 *   a = P(u+1, v) - P(u-1, v)   (u wraps around the 360 degree image)
 *   b = P(u, v+1) - P(u, v-1)
 *   n = a x b / |a x b|, flipped so that n . P(u, v) <= 0 (facing the sensor).
 * Invalid (plane = 0) on rows 0 and H-1, when any of the five ranges is invalid,
 * when |r_nb - r_c| > normal_rel_jump * r_c for a neighbour (decided exactly),
 * or when |a x b| <= 1e-4 |a| |b|.
 * With p->normal_method = 1 (PCA, the eigen-decomposition alternative of
 * Section 4.1): the 3x3 window's points whose range passes the same jump test
 * (at least 5 of the nine, the centre included) give the scatter matrix
 * sum (p - mean)(p - mean)^T; n is the eigenvector of its smallest eigenvalue,
 * flipped as above; invalid on rows 0 and H-1, at an invalid centre, with
 * fewer points, or when lambda_1 <= 1e-4 lambda_2 (collinear points).
 * Output is a plane image per level: planes_levels (HOST array of s->levels
 * device pointers) entry l receives float4 [n][H_l][W_l] = (n_x, n_y, n_z, d)
 * with d = n . P, strided from the finest level like rimg_pyramid (normals are
 * strided, not recomputed, Section 4.1).  mask0 (nullable): uint8 [n][H][W],
 * 1 = valid normal at the finest level.  range and every planes_levels[l]:
 * device, 16-byte aligned (RIMG_ERR_INVALID_ARG otherwise).
 * ------------------------------------------------------------------------- */
int rimg_normals(const rimg_sensor* s, int n_images, const float* range, const rimg_params* p,
                 float* const* planes_levels, uint8_t* mask0, void* stream);

/* ---------------------------------------------------------------------------
 * One projective-association Gauss-Newton step (steps A5-A8), Section 4.1,
 * Eq. 5-7, for n_pairs independent pairs at pyramid level `level`.
 *
 * For every source pixel i of level l (src_range_l [n][H_l][W_l] of sensor
 * `src`): p = Pi^-1(u, v, r) (Eq. 1), x = R p + t with T = pose[pair]; the
 * target pixel (u', v') = Pi(x) at level l of sensor `dst` (Eq. 3-4 with the
 * receiver-offset fixed point, rows by the exact Eq. 4 argmin, columns
 * rounded half up and wrapped); the pair is valid when the source range is
 * valid, the elevation lies within half an edge-row spacing of the table,
 * the target plane (n, d) at (u', v') is valid and, if max_corr_dist > 0,
 * |x - q| <= max_corr_dist.  Then e = n . x - d (= n^T (x - q)), weight
 * w = 1/sqrt(1 + (e/delta)^2) (pseudo-Huber IRLS), J = [x cross n, n] for the
 * left perturbation x <- Exp(xi) x, and the library reduces
 *   J^T W J (21 upper-triangle terms, row-major), J^T W e (6), sum w e^2, count
 * (29 values, FP32 per thread with optional Kahan compensation, FP64 across
 * blocks).  With `update` != 0 it solves (J^T W J) xi = -J^T W e by an FP64
 * LDL^T (Cholesky-type) factorisation and sets T <- Exp(xi) T in place; a degenerate system
 * (count < 6 or pivot <= 1e-12 trace) leaves T unchanged and sets
 * RIMG_FLAG_DEGENERATE in status[pair] (status is OR-ed, never cleared here).
 *
 * dst_planes_l: float4 [n][H_l][W_l] from rimg_normals; dst_range_l
 * ([n][H_l][W_l]) is read only when max_corr_dist > 0 (may be NULL otherwise).
 * pose: float64 [n][16] device.  out29 (nullable): float64 [n][29] device.
 * assoc (nullable): int32 [n][H_l][W_l] device, v' * W_l + u' or -1.
 * status (nullable): int32 [n] device.  Source and target must have the same
 * number of levels (RIMG_ERR_MISMATCH otherwise).
 * workspace: device, 256-byte aligned, >= rimg_icp_workspace_bytes(); its
 * first bytes hold per-pair counters that every call leaves at zero (the call
 * zeroes them with cudaMemsetAsync before its kernel).
 * ------------------------------------------------------------------------- */
int rimg_icp_workspace_bytes(const rimg_sensor* src, int n_pairs, size_t* bytes);
int rimg_icp_step(const rimg_sensor* src, const rimg_sensor* dst, int level, int n_pairs,
                  const float* src_range_l, const float* dst_planes_l, const float* dst_range_l,
                  double* pose, const rimg_params* p, int update, double* out29, int32_t* assoc,
                  int* status, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * The Gauss-Newton update alone (step A8), Section 4.1: for each pair, solve
 * the normal equations of Eq. 7, H xi = -g, in FP64 (LDL^T; not applied when
 * a pivot is <= 1e-12 trace(H) or with fewer than 6 correspondences) and
 * apply T <- Exp(xi) T, xi = (omega, tau).  It is the update rimg_icp_step
 * applies with update = 1, for sums that the caller combined itself (for
 * instance the out29 records of partial images or of several devices, added).
 *
 * sums: float64 [n_pairs][32] device, 8-byte aligned, in place.  Entries
 * 0..28 are read: the 29 reduced quantities in out29's order (21 upper-
 * triangle entries of J^T W J row-major, 6 of J^T W e, sum w e^2, count).
 * Entries 29..31 are written: |omega| (rad) and |tau| (m) of the step, to
 * FP32 precision, and 1 if it was applied (0, 0, 0 otherwise).
 * pose: float64 [n_pairs][16] device, row-major 4x4, updated in place
 * (unchanged when the update is not applied).  status (nullable): int32
 * [n_pairs] device; RIMG_FLAG_DEGENERATE is OR-ed in when it is not applied.
 * ------------------------------------------------------------------------- */
int rimg_gn_update(int n_pairs, double* sums, double* pose, int* status, void* stream);

/* ---------------------------------------------------------------------------
 * rimg_icp_step without a caller workspace.  The paper has no counterpart:
 * this is a library convenience for callers that cannot allocate device
 * memory when they run the step (allocation-free real-time loops, plug-ins
 * that may only touch the buffers they are handed).
 *
 * Same arguments, semantics and results as rimg_icp_step, minus the
 * workspace.  The step's scratch (per-pair completion counters and per-block
 * partial sums) lives in a fixed device array of RIMG_STATIC_SCRATCH_BYTES
 * inside the library; every GPU that loads the library holds one such array
 * until the process exits.  The call allocates nothing.
 *  - Limit: rimg_icp_workspace_bytes(src, n_pairs) must not exceed
 *    RIMG_STATIC_SCRATCH_BYTES (about n_pairs * (H * 128 + 260) bytes for a
 *    sensor with H rows: e.g. up to 124 pairs of 64-row images per call); larger
 *    batches return RIMG_ERR_WORKSPACE before anything is launched.
 *  - The first call on a device looks up the array's device address (with
 *    that device current) and caches it; make that first call before any
 *    stream capture.  The cached address lasts for the process: it does not
 *    survive cudaDeviceReset or any other teardown of the device's primary
 *    context, after which this entry point must not be called on that device
 *    again.
 *  - All calls share the one array and it keeps the previous call's
 *    contents: the counters are cleared on `stream` before every kernel, but
 *    calls that overlap on the GPU (other streams, other host threads) race
 *    on the scratch and must be serialised by the caller.
 * ------------------------------------------------------------------------- */
#define RIMG_STATIC_SCRATCH_BYTES (1u << 20)
int rimg_icp_step_static(const rimg_sensor* src, const rimg_sensor* dst, int level, int n_pairs,
                         const float* src_range_l, const float* dst_planes_l, const float* dst_range_l,
                         double* pose, const rimg_params* p, int update, double* out29, int32_t* assoc,
                         int* status, void* stream);

/* ---------------------------------------------------------------------------
 * Initial pose by centre alignment (Section 4.1, problem statement: the
 * rotation is typically initialised to the identity and the translation
 * estimated by aligning the centres of the two point sets).  For each pair,
 * with P_src / P_dst the valid pixels of the level-l images unprojected by
 * Eq. 1-2 (src_range_l / dst_range_l: float32 [n][H_l][W_l] device, 16-byte
 * aligned, of sensors src / dst at pyramid level `level`):
 *   T_out[pair] = [I | mean(P_dst) - mean(P_src)]
 * so that x = p + t maps the source centre onto the target centre.  Points are
 * unprojected and summed in FP32 four pixels at a time, the sums carried in
 * FP64.  T_out: float64 [n][16] device, row-major, overwritten (a valid
 * T_init for rimg_register).  status (nullable): int32 [n] device;
 * RIMG_FLAG_DEGENERATE is OR-ed in (and T_out = I) when either image has no
 * valid pixel.  The two sensors may differ (each set uses its own tables).
 * ------------------------------------------------------------------------- */
int rimg_center_init(const rimg_sensor* src, const rimg_sensor* dst, int level, int n_pairs, const float* src_range_l,
                     const float* dst_range_l, double* T_out, int* status, void* stream);

/* ---------------------------------------------------------------------------
 * Multi-scale registration (step A9), Section 4.1 with the coarse-to-fine
 * schedule of Section 6.1: normals of every target at the finest level, the
 * strided source-range and target-plane pyramids, then for each level from the
 * coarsest (levels-1) to the finest (0) iters[k] Gauss-Newton steps
 * (iters is a HOST array listed coarse -> fine); the pose carries over between
 * levels unchanged.  All n_pairs pairs share the two sensors and are
 * registered together (one kernel per step covers every pair).
 *
 * src_range, dst_range: float32 [n][H][W] device.  T_init, T_out: float64
 * [n][16] device (they may alias).  status (nullable): int32 [n] device, set
 * to 0 and then OR-ed with RIMG_FLAG_* bits.  workspace: device, 256-byte
 * aligned, >= rimg_register_workspace_bytes().  1 <= levels <= each sensor's
 * levels; both sensors must agree on H, W.
 * ------------------------------------------------------------------------- */
int rimg_register_workspace_bytes(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs,
                                  int levels, size_t* bytes);
int rimg_register(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs,
                  const float* src_range, const float* dst_range, const double* T_init,
                  double* T_out, int levels, const int* iters, const rimg_params* p, int* status,
                  void* workspace, size_t workspace_bytes, void* stream);

/* The last Gauss-Newton step of the most recent rimg_register call on
 * `workspace` (same sensors, n_pairs and levels): out32 float64 [n][32]
 * device.  Entries 0-28 are that step's reduced sums in rimg_icp_step's
 * out29 layout (21 entries of J^T W J, 6 of J^T W e, sum w e^2,
 * correspondence count), evaluated at the pose before the update; 29 and 30
 * are the sizes |omega| (rad) and |tau| (m) of the update xi = (omega, tau)
 * that was applied, 31 is 1 if it was applied (0: degenerate, skipped).
 * A caller judges convergence from them.  Ordered on `stream` after the
 * registration if both use the same stream. */
int rimg_register_last_sums(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs, int levels,
                            const void* workspace, size_t workspace_bytes, double* out32, void* stream);

/* ---------------------------------------------------------------------------
 * Uneven batches: several groups, each a batch of pairs of one sensor pair
 * (one image size) with its own schedule and parameters, registered in one
 * call.  Every group splits into params->streams sub-batches of >= 32 pairs;
 * all sub-batches of all groups are spread over eight internal streams
 * (largest first, to the least-loaded stream) forked from and joined back
 * into `stream`, so the groups run concurrently.
 *
 * The leading small levels of the schedule (the coarsest levels whose pair
 * fits one 256-thread block, when the target projects with the branch-free
 * form and no distance gate is set) of all groups run in ONE persistent
 * launch per kernel form (receiver offset or not, Kahan or not): its blocks
 * take pairs from an atomic work queue ordered by cost, largest groups
 * first, and run each pair's queued levels with all their iterations and
 * FP64 updates; no block waits for another.  The finer levels then run per
 * sub-batch on the internal streams.  rimg_autotune may move a level out of
 * the queue (per-iteration launches) where that measured faster.
 *
 * The call queues work only (no synchronisation, no allocation) and can be
 * captured in a CUDA graph once the library has been used on the device (the
 * first call creates the internal streams and events).  Semantics per group
 * are those of rimg_register.  workspace: device, 256-byte aligned, >=
 * rimg_register_groups_workspace_bytes().
 * ------------------------------------------------------------------------- */
typedef struct rimg_group {
  const rimg_sensor* src;
  const rimg_sensor* dst;
  int n_pairs;
  int levels;
  const int* iters;           /* HOST, coarse -> fine, `levels` entries */
  const rimg_params* params;
  const float* src_range;     /* device [n_pairs][H][W] */
  const float* dst_range;     /* device [n_pairs][H][W] */
  const double* T_init;       /* device [n_pairs][16] */
  double* T_out;              /* device [n_pairs][16] (may alias T_init) */
  int* status;                /* device [n_pairs], nullable */
} rimg_group;

int rimg_register_groups_workspace_bytes(int n_groups, const rimg_group* groups, size_t* bytes);
int rimg_register_groups(int n_groups, const rimg_group* groups, void* workspace, size_t workspace_bytes,
                         void* stream);

/* Autotuner of the per-level schedule and launch shapes, for the sub-batch
 * sizes rimg_register_groups will use.  It builds each group's pyramids in the
 * workspace and, on the group's own data, for every level:
 *  - times every candidate shape of the association kernel (threads per
 *    block, blocks per pair) without updating poses;
 *  - where the level's pair fits one block, and on every level of
 *    sub-batches of at most 64 pairs, times its whole iteration count each
 *    way -- all iterations in one block per pair (where the pair fits one
 *    block: the persistent queue of rimg_register_groups / the one-launch
 *    level of rimg_register), one association launch of the best shape plus
 *    one FP64 solve launch per iteration, and all iterations on a
 *    thread-block cluster of 2, 4 or 8 blocks per pair (one launch; the
 *    blocks exchange their sums through distributed shared memory, one
 *    cluster barrier per iteration) -- and records the fastest schedule;
 *  - for levels that run as per-iteration launches, times the default shape
 *    and the three fastest shapes of the sweep over whole calls and records
 *    the fastest (or no entry, where the default wins).
 * The choices go to a process-wide table keyed by (level size, pairs) that
 * later rimg_register / rimg_register_groups calls use.  Last, the whole call
 * is timed with the new table and with the table as rimg_autotune found it
 * (twice each, alternately); the new entries stay only if they are faster,
 * otherwise the table is left as it was and the return value is 0.  T_out ends
 * as a copy of T_init.  SYNCHRONOUS; returns the number of entries set (>= 0)
 * or a negative status.  rimg_autotune_clear empties the table.
 *
 * rimg_autotune_register: the same tuning for a batch registered with
 * rimg_register (arguments as for rimg_register, workspace >=
 * rimg_register_workspace_bytes()), every timing taken through
 * rimg_register itself. */
int rimg_autotune(int n_groups, const rimg_group* groups, void* workspace, size_t workspace_bytes, void* stream);
int rimg_autotune_register(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs, const float* src_range,
                           const float* dst_range, const double* T_init, double* T_out, int levels,
                           const int* iters, const rimg_params* p, void* workspace, size_t workspace_bytes,
                           void* stream);
int rimg_autotune_clear(void);
/* One entry of the same table set by hand (a saved tuning, or a test that
 * pins a candidate): for levels of H_l x W_l pixels registered in launches of
 * n_pairs pairs, the association launch shape -- threads per block (128 or
 * 256; 0 removes the shape entry) and blocks per pair (1 .. H_l, rounded as
 * the tuner rounds: whole rows per block) -- and the schedule: 1 all
 * iterations in one block per pair (taken only where the pair fits one
 * block, else 0), 2, 4 or 8 all iterations on a cluster of that many
 * 128-thread blocks per pair (any level; with the distance gate a cluster
 * schedule runs as 1 where the pair fits one block, else as 0), 0 one
 * association launch and one FP64 solve launch per iteration, -1 leaves the
 * schedule entry as it is.  A cluster of C blocks gives the same poses and
 * sums, bit for bit, as per-iteration launches with 128 threads and C blocks
 * per pair.  Returns RIMG_OK or RIMG_ERR_INVALID_ARG (non-positive sizes,
 * other thread counts, blocks per pair outside 1 .. H_l, schedule not one of
 * -1, 0, 1, 2, 4, 8). */
int rimg_autotune_set(int H_l, int W_l, int n_pairs, int threads, int blocks_per_pair, int schedule);

/* ---------------------------------------------------------------------------
 * rimg_register with HOST inputs and outputs: copies src_range/dst_range
 * ([n][H][W] float32) and T_init ([n][16] float64) from host memory (pinned
 * memory is needed for the copies to overlap computation) into the
 * workspace, registers, copies T_out (host, [n][16]) and status (host int32
 * [n], nullable) back, and SYNCHRONISES the stream before returning.
 * workspace >= rimg_register_host_workspace_bytes() (it stages the whole
 * batch).  The batch is uploaded in chunks of chunk_pairs pairs (<= 0: one
 * chunk; at most 64 chunks) on an internal copy stream; each chunk is
 * registered on one of four internal compute streams as soon as its own
 * upload has landed, so uploads overlap registrations and registrations of
 * successive chunks overlap each other.  All internal work starts after the
 * work already queued on `stream` and is joined back into it.
 * ------------------------------------------------------------------------- */
int rimg_register_host_workspace_bytes(const rimg_sensor* src, const rimg_sensor* dst,
                                       int n_pairs, int levels, int chunk_pairs, size_t* bytes);
int rimg_register_host(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs,
                       const float* src_range_host, const float* dst_range_host,
                       const double* T_init_host, double* T_out_host, int levels, const int* iters,
                       const rimg_params* p, int* status_host, int chunk_pairs, void* workspace,
                       size_t workspace_bytes, void* stream);

/* The same without the final synchronisation: all copies and kernels are
 * queued and joined into `stream`; the caller must synchronise `stream` (or
 * wait on an event recorded after the call) before reading T_out_host /
 * status_host and before reusing the workspace or the host input buffers.
 * A streaming caller alternating two workspaces and two streams overlaps the
 * upload of batch k+1 with the registration of batch k.  The internal copy
 * and compute streams are shared by all calls on a device, so calls are
 * ordered with each other there. */
int rimg_register_host_async(const rimg_sensor* src, const rimg_sensor* dst, int n_pairs,
                             const float* src_range_host, const float* dst_range_host,
                             const double* T_init_host, double* T_out_host, int levels, const int* iters,
                             const rimg_params* p, int* status_host, int chunk_pairs, void* workspace,
                             size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Point clouds without scan structure (Section 3.2, last paragraph: clouds
 * such as KITTI's enter the same path through a synthetic sensor, theta_lut
 * = 0 and rows evenly spread over the field of view -- any rimg_sensor works).
 * Each point x (optionally moved by T_cloud_to_sensor, float64 [n][16]
 * device, nullable = identity) is projected by Pi at pyramid level `level`;
 * pixel (u, v) keeps the smallest range r = |x - o| of the points that land on
 * it inside the vertical field of view (an exact, order-independent minimum).
 * Pixels without a point are set to +inf, which is an invalid range for every
 * entry point of this library.
 *
 * xyz: float32 [n_clouds][max_points][3] device; counts (nullable): int32
 * [n_clouds] device, points used per cloud (NULL: all max_points); points
 * with a non-finite coordinate are skipped.  range_l: float32
 * [n_clouds][H_l][W_l] device, overwritten.  p (nullable): only proj_iters is
 * used.  n_clouds <= 65535.
 * ------------------------------------------------------------------------- */
int rimg_points_to_range(const rimg_sensor* sensor, int level, int n_clouds, int max_points, const float* xyz,
                         const int* counts, const double* T_cloud_to_sensor, float* range_l, const rimg_params* p,
                         void* stream);

/* ---------------------------------------------------------------------------
 * Projective SDF integration, Section 4.2 (Eq. 8-10), on a dense voxel grid.
 *
 * For each voxel centre x = origin + voxel * (i + 1/2, j + 1/2, k + 1/2) and
 * each scan s: [u v r] = Pi(R_s x + t_s) at pyramid level `level` (Eq. 8; the
 * projection of rimg_icp_step), and, when the point is inside the vertical
 * field of view and the scan's range at (u, v) is valid, the signed distance
 * along the ray d_s = range(u, v) - r (Eq. 9).  With trunc > 0 a scan with
 * d_s < -trunc does not observe the voxel (it lies behind the surface) and
 * d_s is clipped to trunc; trunc <= 0 keeps Eq. 9 as is.  The observations are
 * merged into the voxel's least-squares estimate (Eq. 10) incrementally:
 * sdf <- (sdf * weight + sum_s d_s) / (weight + count), weight += count.
 *
 * range_l: float32 [n_scans][H_l][W_l] device (level-l images, e.g. from
 * rimg_pyramid).  T_world_to_sensor: float64 [n_scans][16] device, mapping
 * world points into each scan's sensor frame.  sdf, weight: float32
 * [nz][ny][nx] device (x fastest), read and updated in place (start from
 * zeros).  p (nullable): only proj_iters is used.  n_scans = 0 or an empty
 * grid is a no-op.
 * ------------------------------------------------------------------------- */
typedef struct rimg_grid {
  int nx, ny, nz;
  float voxel;              /* edge length, > 0 */
  float origin[3];          /* world position of the outer corner of voxel (0, 0, 0) */
} rimg_grid;

int rimg_sdf_integrate(const rimg_sensor* sensor, int level, int n_scans, const float* range_l,
                       const double* T_world_to_sensor, const rimg_grid* grid, float trunc, float* sdf,
                       float* weight, const rimg_params* p, void* stream);

/* ---------------------------------------------------------------------------
 * Dense BF16 GEMM on the tcgen05 tensor cores (the contraction of the learned
 * pose proposal's convolutions; the registration itself uses no tensor
 * cores):  C[M x N] = A[M x K] * B[N x K]^T (+ bias[N]) (ReLU), FP32
 * accumulation in tensor memory.  A and B are BF16, K-major (row i of A is K
 * contiguous elements at A + i * lda), device, 16-byte aligned, lda and ldb
 * multiples of 8 elements; K must be a multiple of 64 (zero-pad).  C: FP32
 * row-major [M][ldc]; C_bf16 (nullable): a BF16 copy with the same leading
 * dimension.  splits > 1 divides K into `splits` ranges (multiples of 64)
 * computed by separate CTAs, each writing its own partial result at
 * C + z * M * ldc (the caller sums them; bias, ReLU and C_bf16 must then be
 * unset).  err (nullable, device int): set to 1 if a CTA gave up waiting for
 * its tensor-core work (it then skips its epilogue).
 * ------------------------------------------------------------------------- */
int rimg_gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, float* C, int ldc,
                   void* C_bf16, const float* bias, int relu, int splits, int* err, void* stream);

/* ---------------------------------------------------------------------------
 * Learned pose proposal (an extension: the paper starts Gauss-Newton from a
 * given initial pose and names learned range-image features only as future
 * work, Section 7).  A BF16 convolutional network reads the coarsest pyramid
 * level (Section 4.1; every 8th row and column of a 64 x 1024 scan) of a
 * source and a target scan and regresses T0, the init pose of rimg_register;
 * the registration stays the judge of its result.
 *
 * Network: input [n][8][128][2] = (source, target) range * RIMG_CNN_RANGE_SCALE
 * (0 for invalid ranges), BF16; five 3x3 stride-2 convolutions with ReLU,
 * rows zero-padded, columns wrapped around (360 degrees of azimuth), channels
 * 2 -> 32 -> 64 -> 64 -> 128 -> 128 (8x128 -> 4x64 -> 2x32 -> 1x16 -> 1x8 ->
 * 1x4); a linear layer 512 -> 6 on the (w, c)-flattened activations gives
 * p = (omega / RIMG_CNN_OMEGA_SCALE, t / RIMG_CNN_T_SCALE) and
 * T0 = [Exp(omega), t] (Exp: Rodrigues).  BF16 operands, FP32 accumulation on
 * the tcgen05 tensor cores (rimg_gemm_bf16's kernel), FP32 master weights.
 *
 * Parameters (FP32, rimg_cnn_param_count of them, in this order): for each
 * convolution W [C_out][9 C_in] (column (kh * 3 + kw) * C_in + c) and
 * b [C_out]; then the linear W [6][512] (column w * 128 + c) and b [6].
 *
 * State: one device buffer (256-byte aligned, rimg_cnn_state_bytes long)
 * holding the master parameters (its first param_count floats), the Adam
 * moments and BF16 copies of the weights.  Workspace: per batch size n,
 * rimg_cnn_workspace_bytes(n), 256-byte aligned; one call at a time per
 * workspace.
 *
 * Inputs: src_range, dst_range float32 [*][H][W] device with
 * H = 8 * stride and W = 128 * stride (stride 8 reads the coarsest level of
 * a 4-level 64 x 1024 pyramid straight from the full images; stride 1 reads
 * stored 8 x 128 images).  index (nullable, device int32 [n]): pair i of the
 * batch is image index[i] (and label index[i]); NULL means i.  T_label
 * float64 [*][16]: the training target poses.  err (nullable, device int):
 * set to 1 if a tensor-core wait timed out (that GEMM tile's output is then
 * not written).  Sizes: 0 <= n <= RIMG_CNN_MAX_BATCH.
 * ------------------------------------------------------------------------- */
#define RIMG_CNN_IN_H 8
#define RIMG_CNN_IN_W 128
#define RIMG_CNN_RANGE_SCALE 0.03125f
#define RIMG_CNN_OMEGA_SCALE 0.25
#define RIMG_CNN_T_SCALE 3.0
#define RIMG_CNN_MAX_BATCH 65536

typedef struct rimg_adam {
  float lr, beta1, beta2, eps;
} rimg_adam;

int rimg_cnn_param_count(size_t* n_params);
int rimg_cnn_state_bytes(size_t* bytes);
int rimg_cnn_workspace_bytes(int n, size_t* bytes);

/* Seeded initialisation: He-uniform convolution weights U(+-sqrt(6 / fan_in)),
 * linear weights U(+-0.1 sqrt(3 / 512)), zero biases, zero moments. */
int rimg_cnn_init(void* state, size_t state_bytes, uint64_t seed, void* stream);

/* Master parameters from `params` (device FP32 [param_count]; may be the
 * state's own first floats), Adam moments cleared, BF16 copies rebuilt. */
int rimg_cnn_load(void* state, size_t state_bytes, const float* params, void* stream);

/* Inference: pred (nullable) float32 [n][6] network outputs p; T_out
 * (nullable) float64 [n][16] proposals T0 = [Exp(0.25 p[0:3]), 3 p[3:6]]. */
int rimg_propose(const void* state, int n, int H, int W, int stride, const float* src_range, const float* dst_range,
                 const int32_t* index, float* pred, double* T_out, int* err, void* workspace, size_t workspace_bytes,
                 void* stream);

/* Loss and gradient without an update: loss (nullable, device double)
 * = 1 / (2 n) sum_i |p_i - y_i|^2 with y = (Log R / 0.25, t / 3) of the
 * label pose [R, t]; grad: device FP32 [param_count] in the parameter order;
 * pred (nullable) as in rimg_propose.  Backpropagation treats the BF16
 * roundings as identities. */
int rimg_cnn_grad(const void* state, int n, int H, int W, int stride, const float* src_range, const float* dst_range,
                  const int32_t* index, const double* T_label, double* loss, float* grad, float* pred, int* err,
                  void* workspace, size_t workspace_bytes, void* stream);

/* One training step: the gradient of rimg_cnn_grad, then Adam (step >= 1:
 * bias corrections 1 - beta^step) on the master parameters and a rebuild of
 * the BF16 copies. */
int rimg_cnn_train_step(void* state, size_t state_bytes, int n, int H, int W, int stride, const float* src_range,
                        const float* dst_range, const int32_t* index, const double* T_label, const rimg_adam* opt,
                        int step, double* loss, int* err, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Launch timing (tracing).  rimg_profile_begin(max) makes subsequent library
 * launches on any stream record a CUDA event pair around each kernel (at most
 * `max` launches; later ones are not recorded).  rimg_profile_end waits for
 * the recorded events, writes up to `cap` records (kernel id, level, n_pairs,
 * start in ms after the first record's start, duration in ms; any output
 * pointer may be NULL) and stops recording; it returns the number of records.
 * Launches on concurrent streams overlap in time: the start offsets let a
 * caller take the union of intervals.
 * Kernel ids: 0 unproject, 1 pyramid, 2 normals (+ plane pyramid),
 * 3 icp step (association + reduction), 4 source-range pyramid, 5 FP64
 * solve + pose update, 6 SDF integration, 7 point-cloud projection, 8 all
 * iterations of a small pyramid level (one block per pair), 9 the persistent
 * small-level queue of rimg_register_groups (level -1, n_pairs = items).  Not
 * for use during stream capture.
 * ------------------------------------------------------------------------- */
int rimg_profile_begin(int max_launches);
int rimg_profile_end(int cap, int* kernel_id, int* level, int* n_pairs, float* start_ms, float* ms);

#ifdef __cplusplus
}
#endif
#endif /* RIMG_H */
