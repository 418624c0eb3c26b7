/*
 * dtsdf.h - C ABI of the Directional TSDF render + ICP library (libdtsdf.so).
 *
 * The library implements the data-parallel hot path of Splietker & Behnke,
 * "Rendering the Directional TSDF for Tracking and Multi-Sensor Registration with
 * Point-To-Plane Scale ICP": fusing RGB-D frames into a Directional TSDF (six
 * per-axis TSDFs in one voxel-block hash keyed by block and direction), ray-cast
 * rendering of depth, normal and colour images from it, and the point-to-plane
 * ICP normal-equation reduction and solve in SE(3) and Sim(3), with the optional
 * frame-to-keyframe photometric term.
 *
 * Conventions shared by every call
 *   - Pointers documented as "device" are CUDA device pointers owned by the caller;
 *     "host" pointers are ordinary CPU memory read or written before the call returns.
 *   - Images are row-major, pixel (u, v) at index v * width + u; pixel centres sit
 *     at integer (u, v). Camera frame: x right, y down, z forward.
 *   - Poses are row-major 4x4 double matrices. T_wc maps camera to world.
 *   - Depth is z-depth in metres; 0 marks an invalid or missing value.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     All device work is ordered on it. Calls returning host results synchronise it.
 *   - Errors are reported only through dtsdf_status; dtsdf_last_error() returns a
 *     message for the calling thread's most recent failure. Nothing throws.
 *   - A map or ICP context may be used by one host thread at a time.
 */
#ifndef DTSDF_H
#define DTSDF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DTSDF_API __attribute__((visibility("default")))
#else
#define DTSDF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dtsdf_map_s* dtsdf_map;
typedef struct dtsdf_icp_s* dtsdf_icp;

typedef enum {
  DTSDF_OK = 0,
  DTSDF_ERR_INVALID_ARG = 1, /* null pointer, bad size, bad parameter */
  DTSDF_ERR_OOM = 2,         /* device allocation failed */
  DTSDF_ERR_MAP_FULL = 3,    /* block pool, directory or hash table exhausted */
  DTSDF_ERR_CUDA = 4,        /* a CUDA runtime error (message in dtsdf_last_error) */
  DTSDF_ERR_DEGENERATE = 5,  /* ICP normal equations not positive definite / too few rows */
  DTSDF_ERR_TIMEOUT = 6      /* a bounded device wait ran out */
} dtsdf_status;

typedef enum { DTSDF_STORE_FP32 = 0, DTSDF_STORE_FP16 = 1 } dtsdf_storage;

/* Map parameters (Sec. 3, 4 and 7 of the paper; constants the paper leaves open take the stated defaults). */
typedef struct {
  float voxel_size;     /* h, metres */
  float truncation;     /* tau, metres (Eq. point-to-plane normalises by it) */
  float theta;          /* angular threshold of Eq. angular_threshold, radians, in (acos(1/sqrt3), pi/2] */
  float w_max;          /* cap of the accumulated depth and colour weights */
  float w_carve;        /* constant weight of a free-space carving update (Sec. 3) */
  float z_min, z_max;   /* valid depth range, metres; z_min also enters Eq. ICP_weight */
  float delta_sup;      /* outlier filter: neighbour supports a depth if |dz| <= delta_sup (Sec. 7) */
  int32_t carve_radius; /* carving needs no depth jump > tau within this many pixels (Sec. 3: 2) */
  int32_t dense_dim;    /* > 0: dense grid of dense_dim^3 voxels (multiple of 8), every block
                           allocated at creation; 0: sparse voxel-block hash */
  float dense_origin[3];/* world position of voxel (0,0,0); voxel (i,j,k) of block b is at
                           origin + (8 b + (i,j,k)) * h */
  uint32_t max_blocks;  /* pool capacity in (block, direction) bricks of 8^3 voxels */
  int32_t storage;      /* dtsdf_storage: FP32 sdf+weight (8 B) or FP16 sdf + u16 weight (4 B) */
  int32_t color;        /* 1: integrate and render colour */
} dtsdf_params;

typedef struct {
  int32_t width, height;
  float fx, fy, cx, cy;
} dtsdf_intrinsics;

/* One RGB-D frame in device memory. */
typedef struct {
  const float* depth;  /* device, height*width float32 z-depth, 0 = invalid */
  const uint8_t* rgb;  /* device, height*width*3 uint8, or NULL */
  dtsdf_intrinsics K;
} dtsdf_frame;

/* Render output buffers, device memory owned by the caller, sized height*width*(1|4). */
typedef struct {
  float* depth;   /* z-depth of the first positive-to-negative crossing, 0 = miss */
  float* normals; /* float4 per pixel: camera-frame unit normal (x, y, z) and w = depth; 0 on a miss */
  float* color;   /* float4 per pixel: r, g, b in [0, 255] and w = 1 where colour is defined; or NULL */
} dtsdf_render_out;

/* Map statistics (dtsdf_map_stats synchronises the stream). */
typedef struct {
  int64_t bricks;          /* allocated (block, direction) bricks (recycled ones not counted) */
  int64_t blocks;          /* distinct allocated block coordinates */
  int64_t bricks_per_dir[6];
  int64_t capacity;        /* max_blocks */
  uint32_t error_flags;    /* bit 0: pool full, bit 1: directory full, bit 2: hash probe limit,
                              bit 3: allocation work list full, bit 4: a bounded device wait
                              of the combine pass ran out (that pass stopped early; the next
                              dtsdf_integrate returns DTSDF_ERR_TIMEOUT) */
  int32_t frames;          /* frames integrated */
} dtsdf_map_stats_t;

/* ----------------------------------------------------------------- map ---- */

/* Create an empty map. Allocates max_blocks bricks of device memory up front
 * (FP32: 24 B per voxel with colour, 8 B without; FP16: 8 / 4 B). */
DTSDF_API dtsdf_status dtsdf_create(const dtsdf_params* params, void* stream, dtsdf_map* out);
DTSDF_API dtsdf_status dtsdf_destroy(dtsdf_map map);

/* Fuse one frame taken at pose T_wc (Sec. 3 voxel-projection fusion): outlier filter and
 * cross-product normals (Sec. 7), allocation of the (block, direction) bricks that the
 * segment [p - tau r, p + tau r] of every pixel with a normal crosses, for each direction
 * of Eq. angular_threshold, then the weighted running average of Eq. point-to-plane with
 * the weights of Eq. combined_fusion_weight and Eq. color_weight, and free-space carving.
 * Asynchronous. Pool exhaustion sets an error flag reported by dtsdf_map_stats and by the
 * next dtsdf_integrate call (DTSDF_ERR_MAP_FULL); so does a bounded device wait of the combine
 * pass that ran out (DTSDF_ERR_TIMEOUT). Flags are read back without stalling the stream, so
 * they surface one or two calls after the launch that set them. The first call with a new frame
 * size allocates scratch memory. */
DTSDF_API dtsdf_status dtsdf_integrate(dtsdf_map map, const dtsdf_frame* frame, const double T_wc[16], void* stream);

/* Same as dtsdf_integrate with the pose read from device memory (16 doubles, row-major),
 * so a tracking loop can fuse at the pose its ICP produced without a host round trip. */
DTSDF_API dtsdf_status dtsdf_integrate_dev(dtsdf_map map, const dtsdf_frame* frame, const double* T_wc_dev,
                                           void* stream);

/* Ray-cast depth, normals and colour at pose T_wc with intrinsics K (Sec. 4): per pixel,
 * march the combined SDF of Eq. combine_weight (fallback Eq. combine_tsdf_weight) along
 * the ray from z_min to z_max, find the first positive-to-negative crossing between
 * consecutive samples of the h/2 grid and refine it by 16 bisection steps on the sign of the
 * continuous combined SDF (an undefined point counts as free space): the depth is the final
 * bracket's midpoint, normal and colour are taken at its non-positive end. A pre-pass records
 * per tile of 32 rays the depth range of the allocated blocks in view, and each ray marches
 * only that range (outside it no sample can be defined). Asynchronous; the scratch (8 bytes per
 * ray tile for the pre-pass, 8 bytes per ray for the crossings the march hands to the
 * refinement) is stream-ordered memory from a pool the map keeps cached. */
DTSDF_API dtsdf_status dtsdf_render(dtsdf_map map, const dtsdf_intrinsics* K, const double T_wc[16],
                          const dtsdf_render_out* out, void* stream);

/* Same as dtsdf_render with the pose read from device memory (16 doubles, row-major). */
DTSDF_API dtsdf_status dtsdf_render_dev(dtsdf_map map, const dtsdf_intrinsics* K, const double* T_wc_dev,
                                        const dtsdf_render_out* out, void* stream);

/* Render from the view-dependent combined TSDF (Sec. 4; Sec. 7: combination at integer voxel
 * positions): the combined value of every voxel of the blocks in the view frustum grown by 1/8
 * of the image on each side is formed with the weights of Eq. combine_weight (6-neighbour
 * gradients, view ray from the camera centre of the combination pose; fallback of
 * Eq. combine_tsdf_weight), and the result is ray-cast like a regular TSDF with the rules of
 * dtsdf_render (sample grid, first crossing, refinement, outputs), the normal from the central
 * differences of the trilinear combined field. Conditional combination (Sec. 4): the whole
 * frustum is recombined at this pose while fewer than 5 combined renders were made, after more
 * than 50 without recombination, or when the pose moved by more than 0.05 m or turned by more
 * than 0.05 pi/2 since the last combination; otherwise only blocks that received bricks since
 * the previous call, and the 26 blocks around each of them, are combined (at the last combination
 * pose) and the render uses the stored field. The decision is taken on the device. The first call
 * allocates the combined field: per directory entry 729 voxels x 8 B (+ 729 x 8 B with colour)
 * and 5 B of state. Asynchronous. */
DTSDF_API dtsdf_status dtsdf_render_combined(dtsdf_map map, const dtsdf_intrinsics* K, const double T_wc[16],
                                             const dtsdf_render_out* out, void* stream);

/* Same with the pose read from device memory (16 doubles, row-major). */
DTSDF_API dtsdf_status dtsdf_render_combined_dev(dtsdf_map map, const dtsdf_intrinsics* K, const double* T_wc_dev,
                                                 const dtsdf_render_out* out, void* stream);

/* The next combined render recombines the whole frustum at its pose. */
DTSDF_API dtsdf_status dtsdf_combined_reset(dtsdf_map map);

/* The combination step of dtsdf_render_combined alone (conditional as there, or the whole
 * padded frustum at T_wc when force != 0), for callers that precompute the combined TSDF
 * ahead of their renders. Asynchronous. */
DTSDF_API dtsdf_status dtsdf_combine(dtsdf_map map, const dtsdf_intrinsics* K, const double T_wc[16], int32_t force,
                                     void* stream);
DTSDF_API dtsdf_status dtsdf_combine_dev(dtsdf_map map, const dtsdf_intrinsics* K, const double* T_wc_dev,
                                         int32_t force, void* stream);

/* Blocks of the current combination and the (block, direction) bricks they hold (host
 * outputs); 0 before the first combination. Synchronous. */
DTSDF_API dtsdf_status dtsdf_combined_blocks(dtsdf_map map, int64_t* blocks, int64_t* bricks, void* stream);

/* Launch shape of the map's renders (no counterpart in the paper: scheduling only; every
 * shape computes the same samples, decisions and outputs). ctas: CTAs of the persistent
 * render grid, 0 = one wave of resident CTAs. tile_w: width of the pixel tiles of 32 rays
 * that the work is handed out in, 1, 2, 4, 8, 16 or 32 (0 = 4), the height being 32 / tile_w; a
 * tile's rays go to the lanes of a warp row by row. refill: lanes per refill group, 1, 2, 4,
 * 8, 16 or 32 (0 = 32): a group of `refill` consecutive lanes takes its next `refill` rays
 * once all of its lanes have finished (32: the warp takes a whole tile; 1: a lane takes a ray
 * as soon as it is free). Defaults {0, 0, 0}. DTSDF_ERR_INVALID_ARG for other values. */
typedef struct {
  int32_t ctas;
  int32_t refill;
  int32_t tile_w;
} dtsdf_render_opts;

DTSDF_API dtsdf_status dtsdf_set_render_opts(dtsdf_map map, const dtsdf_render_opts* opts);

/* Autotuner of the render launch shape (no counterpart in the paper): times a render at T_wc
 * (intrinsics K, outputs `out`, as dtsdf_render) with tile widths 2 to 32 and refill groups
 * of 8, 16 or 32 lanes (ctas 0), keeps the fastest as the map's shape and returns it in *best
 * and its time in *best_ms (host, may be NULL). Synchronous. */
DTSDF_API dtsdf_status dtsdf_render_tune(dtsdf_map map, const dtsdf_intrinsics* K, const double T_wc[16],
                                         const dtsdf_render_out* out, dtsdf_render_opts* best, float* best_ms,
                                         void* stream);

/* Instrumented render at T_wc that counts the distinct bricks the march reads: geometry
 * bricks (sdf + weight) and colour bricks. Defines the algorithmic bytes of a render for
 * roofline accounting. counters (host, 8 int64, or NULL) receives totals over all rays:
 * samples, full combinations, cells entered, allocated cells entered, hits, cells jumped
 * because every allocated direction is positive throughout them. Synchronous;
 * allocates scratch. */
DTSDF_API dtsdf_status dtsdf_render_touched(dtsdf_map map, const dtsdf_intrinsics* K, const double T_wc[16],
                                            int64_t* geom_bricks, int64_t* color_bricks, int64_t* counters,
                                            void* stream);

/* C = A B, or A^-1 B when invert_a != 0, for 4x4 affine transforms (rigid or similarity) in
 * device memory; one thread, asynchronous. Chains poses in a device-resident tracking loop. */
DTSDF_API dtsdf_status dtsdf_pose_compose(const double* A_dev, int32_t invert_a, const double* B_dev, double* C_dev,
                                          void* stream);

DTSDF_API dtsdf_status dtsdf_map_stats(dtsdf_map map, dtsdf_map_stats_t* stats, void* stream);

/* Copy the map to host memory: coords (n x 4 int32: bx, by, bz, D) and voxels
 * (n x 512 x 6 float: sdf, w, r, g, b, wc, voxel index i + 8 j + 64 k), one entry per pool
 * brick. At most `cap` bricks are written; *n_out receives the pool count. Entries of bricks
 * that dtsdf_recycle returned to the pool (and that were not handed out again) have D = -1;
 * dtsdf_map_import rejects them. Synchronous. */
DTSDF_API dtsdf_status dtsdf_map_export(dtsdf_map map, int32_t* coords, float* voxels, int64_t cap, int64_t* n_out,
                              void* stream);

/* Load bricks from host memory, in the layout dtsdf_map_export writes: coords (n x 4:
 * bx, by, bz, D) and voxels (n x 512 x 6: sdf, w, r, g, b, wc). Missing bricks are
 * allocated (sparse maps); existing ones are overwritten. Restores a saved map or loads a
 * map built elsewhere. Synchronous. DTSDF_ERR_MAP_FULL if the pool cannot hold them. */
DTSDF_API dtsdf_status dtsdf_map_import(dtsdf_map map, const int32_t* coords, const float* voxels, int64_t n,
                                        void* stream);

/* ----------------------------------------------------------------- ICP ---- */

typedef struct {
  int32_t levels;       /* pyramid levels used, 1..4 (level 0 = full resolution) */
  int32_t iters[4];     /* iteration cap per level, index = level (0 finest) */
  float eps[4];         /* distance outlier threshold per level, metres (Sec. 8: 0.005 fine / 0.05 coarse) */
  float photo_thr[4];   /* intensity outlier threshold per level (Sec. 8: 0.05 fine / 0.175 coarse) */
  float lambda;         /* photometric weight of Eq. combined_icp (0.1); 0 disables the term */
  float z_min;          /* z_min of Eq. ICP_weight */
  double stop_norm;     /* stop a level when ||xi|| < stop_norm (Sec. 8: 1e-6) */
  int32_t min_rows;     /* fewer rows than this -> DTSDF_ERR_DEGENERATE */
  int32_t kahan;        /* 1: Kahan-compensated FP32 accumulation of the per-pixel sums */
  int32_t lm;           /* 1: Levenberg-Marquardt with Madsen's damping update (Sec. 7) instead of
                         * Gauss-Newton; dtsdf_icp_solve only (one LM state per level: the first
                         * evaluation is accepted, mu = 1e-3 max diag(H), nu = 2; a step whose gain
                         * ratio is not positive is undone and mu grows by nu, nu doubles). The
                         * single-step, batch, server and no-alloc entry points need 0 here
                         * (DTSDF_ERR_INVALID_ARG otherwise). */
} dtsdf_icp_opts;

/* Result of one Gauss-Newton iteration. H (row-major, dim x dim in the top-left of 7x7
 * storage) and g are the normal equations of Eq. ICP_Hessian without the factor 2, for
 * xi = (nu, omega) or (nu, omega, sigma). */
typedef struct {
  double H[49];
  double g[7];
  double xi[7];
  double error;        /* sum of w r^2 */
  int64_t rows;        /* geometric + photometric rows used */
  int64_t rows_photo;
  double step_norm;    /* ||xi|| */
  int32_t dim;         /* 6 or 7 */
  int32_t status;      /* 0 ok, DTSDF_ERR_DEGENERATE */
  int32_t converged;   /* step_norm < stop_norm */
  int32_t iterations;  /* iterations run (dtsdf_icp_solve) */
} dtsdf_icp_stats;

/* ICP context: current-frame pyramid, keyframe pyramid, reduction scratch, device pose. */
DTSDF_API dtsdf_status dtsdf_icp_create(int32_t max_width, int32_t max_height, int32_t levels, dtsdf_icp* out);
DTSDF_API dtsdf_status dtsdf_icp_destroy(dtsdf_icp icp);

/* Current frame: outlier filter (Sec. 7), then the depth pyramid (2x2 mean of valid depths,
 * f/2, (c - 0.5)/2) and, if rgb is given, the intensity pyramid I = (0.299 R + 0.587 G +
 * 0.114 B) / 255. Asynchronous. */
DTSDF_API dtsdf_status dtsdf_icp_set_frame(dtsdf_icp icp, const dtsdf_frame* cur, float z_min, float z_max,
                                 float delta_sup, void* stream);

/* Keyframe of the frame-to-keyframe photometric term (Eq. keyframe_icp): intensity pyramid
 * and central-difference gradients of its rgb. Asynchronous. */
DTSDF_API dtsdf_status dtsdf_icp_set_keyframe(dtsdf_icp icp, const dtsdf_frame* kf, void* stream);

/* One Gauss-Newton iteration on pyramid `level` against the render `ref` (intrinsics K_ref):
 * point-to-plane rows of Eq. geometric_ICP / Eq. ICP_geometric_dx with weights of
 * Eq. ICP_weight, plus photometric rows against the keyframe when T_rs (render camera ->
 * keyframe camera, host, row-major) is non-NULL and opts->lambda > 0; deterministic
 * reduction, Cholesky solve of Eq. ICP_solution and the update of Eq. deltaT_update.
 * T_rel (host, row-major, current camera -> render camera) is read and, unless the system
 * is degenerate, overwritten. Synchronous (returns stats). */
DTSDF_API dtsdf_status dtsdf_icp_step(dtsdf_icp icp, const dtsdf_render_out* ref, const dtsdf_intrinsics* K_ref,
                            int32_t level, double T_rel[16], const double* T_rs, const dtsdf_icp_opts* opts,
                            dtsdf_icp_stats* stats, void* stream);

/* Same in Sim(3) (Sec. 6, Eq. sim3_derivative): T_rel = [s R | t], 7x7 normal equations. */
DTSDF_API dtsdf_status dtsdf_icp_sim3_step(dtsdf_icp icp, const dtsdf_render_out* ref, const dtsdf_intrinsics* K_ref,
                                 int32_t level, double T_rel[16], const double* T_rs,
                                 const dtsdf_icp_opts* opts, dtsdf_icp_stats* stats, void* stream);

/* Whole coarse-to-fine schedule (levels-1 .. 0, opts->iters[l] iterations, early stop per
 * level), entirely on the device: T_rel_dev (device, 16 doubles) is read and updated in
 * place; T_rs_dev (device, 16 doubles, or NULL: no photometric term) is the render ->
 * keyframe camera transform; stats_dev (device, one dtsdf_icp_stats, or NULL) receives the
 * last iteration's statistics. Asynchronous and free of host synchronisation, so it can be
 * captured in a CUDA graph. sim3 = 0: SE(3), 1: Sim(3). */
DTSDF_API dtsdf_status dtsdf_icp_solve(dtsdf_icp icp, const dtsdf_render_out* ref, const dtsdf_intrinsics* K_ref,
                                       int32_t sim3, double* T_rel_dev, const double* T_rs_dev,
                                       const dtsdf_icp_opts* opts, dtsdf_icp_stats* stats_dev, void* stream);

/* One Gauss-Newton iteration of geometric point-to-plane ICP (SE(3) or Sim(3)) that allocates
 * no device memory. The paper has no counterpart: this serves callers that cannot allocate when
 * they run ICP - real-time loops where cudaMalloc's implicit device synchronisation would stall
 * other streams, or a host application that owns all device memory. Every input and output is a caller-owned device
 * buffer: depth (K_cur->height x K_cur->width float32, already outlier-filtered, 0 invalid),
 * ref (the render's normals, float4 with the depth in w; K_ref its intrinsics), T_rel_dev
 * (16 doubles, current -> render camera, read and updated in place unless degenerate) and
 * stats_dev (one dtsdf_icp_stats, overwritten). The reduction's scratch is a fixed file-scope
 * device array of 256 KB that every GPU loading the library keeps until exit; images of more
 * than 1048576 pixels are rejected (DTSDF_ERR_INVALID_ARG). The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress) and keeps it, so that first call should be
 * made before any stream capture, and the library must not be used across cudaDeviceReset. All
 * calls share the scratch and it keeps the last call's contents; calls that overlap on the GPU
 * race on it. Asynchronous on `stream`. */
DTSDF_API dtsdf_status dtsdf_icp_step_noalloc(const float* depth, const dtsdf_intrinsics* K_cur,
                                              const dtsdf_render_out* ref, const dtsdf_intrinsics* K_ref,
                                              int32_t sim3, float eps, float z_min, int32_t min_rows,
                                              double stop_norm, double* T_rel_dev, dtsdf_icp_stats* stats_dev,
                                              void* stream);

/* ------------------------------------------------------------- batches ---- */

/* One registration problem of a batch: the current frame held by `icp` (prepared with
 * dtsdf_icp_set_frame; its pyramid must have at least opts->levels levels), the reference
 * render `ref` (device; its normals carry the depth in w) with intrinsics K_ref, the pose
 * T_rel_dev (device, 16 doubles, current camera -> render camera, read and updated) and
 * stats_dev (device, one dtsdf_icp_stats, or NULL). sim3 = 1: Sim(3) (Sec. 6, 7x7 system),
 * 0: SE(3). Problems of one batch may have different image sizes. */
typedef struct {
  dtsdf_icp icp;
  dtsdf_render_out ref;
  dtsdf_intrinsics K_ref;
  double* T_rel_dev;
  dtsdf_icp_stats* stats_dev;
  int32_t sim3;
} dtsdf_icp_problem;

/* Launch shape of a batched registration (no counterpart in the paper): CTAs per problem
 * (a thread-block cluster: 1, 2, 4, 8 or 16) and threads per CTA (128, 256 or 512). */
typedef struct {
  int32_t cluster;
  int32_t threads;
} dtsdf_batch_shape;

/* Whole geometric coarse-to-fine schedule of dtsdf_icp_solve for n problems in one launch per
 * 64 problems: each problem is one thread-block cluster that runs opts->levels levels of
 * opts->iters[l] Gauss-Newton iterations (early stop per level at ||xi|| < opts->stop_norm),
 * with the deterministic reduction (rank order, FP64), the FP64 Cholesky solve and the pose
 * update on the device (Eqs. geometric_ICP, ICP_weight, ICP_Hessian, ICP_solution,
 * deltaT_update; Sim(3) exponential of Sec. 6). No photometric term (opts->lambda is ignored);
 * opts->kahan selects compensated summation. shape NULL: {8, 256}. Asynchronous, allocates
 * nothing and synchronises nothing: can be captured in a CUDA graph. DTSDF_ERR_INVALID_ARG
 * for a bad problem, option or shape; DTSDF_ERR_CUDA if the cluster cannot be scheduled. */
DTSDF_API dtsdf_status dtsdf_icp_batch(const dtsdf_icp_problem* problems, int32_t n, const dtsdf_icp_opts* opts,
                                       const dtsdf_batch_shape* shape, void* stream);

/* Autotuner of dtsdf_icp_batch: times every supported shape on these problems (scratch copies
 * of the poses; the problems' poses and stats are left unchanged) and returns the fastest in
 * *best and its time in *best_ms (host). Synchronous; allocates scratch. */
DTSDF_API dtsdf_status dtsdf_icp_batch_tune(const dtsdf_icp_problem* problems, int32_t n,
                                            const dtsdf_icp_opts* opts, dtsdf_batch_shape* best, float* best_ms,
                                            void* stream);

/* One frame of a batched render: intrinsics, pose (device, 16 doubles, camera -> world) and
 * caller-owned outputs as for dtsdf_render. */
typedef struct {
  dtsdf_intrinsics K;
  const double* T_wc_dev;
  dtsdf_render_out out;
} dtsdf_render_job;

/* Ray-cast n frames of any sizes (Sec. 4, as dtsdf_render) in one persistent launch per 64
 * frames: the pixels of all frames form one work list that the CTAs take in 8x4 tiles, so
 * uneven frames share the GPU without a tail per frame. Asynchronous; its scratch (as for
 * dtsdf_render) is stream-ordered memory from the map's pool, so the call can be captured in a
 * CUDA graph. */
DTSDF_API dtsdf_status dtsdf_render_batch(dtsdf_map map, const dtsdf_render_job* jobs, int32_t n, void* stream);

/* ------------------------------------------------------------- serving ---- */

/* A request server over device-resident maps (no counterpart in the paper: it schedules the
 * paper's tracking step - preprocessing and pyramid of a depth frame (Sec. 7), a render of
 * the map at a prior pose (Sec. 4), coarse-to-fine point-to-plane registration in SE(3) or
 * Sim(3) (Secs. 5, 6) - for many sensors at once). A worker thread owned by the server admits
 * requests in arrival order when their device working set fits in a fixed arena of
 * hbm_budget bytes (allocated at creation) and a host slot is free, and keeps up to `streams`
 * batches on the device: whenever a stream is idle, every pending request that fits (at most
 * max_batch) is launched as one batch - per-request copy, preprocessing and pyramid, one
 * render launch per map over the batch's frames of any sizes, one batched registration launch
 * (opts: levels, iterations, eps, stop; no photometric term) - so requests arriving while
 * others run join the next batch and batches overlap on the device. A request's result does
 * not depend on the batch it was served in. The maps stay owned by the caller and must not be
 * modified or destroyed while the server exists. */
typedef struct dtsdf_server_s* dtsdf_server;

typedef struct {
  int64_t hbm_budget;       /* bytes of device memory for request working sets (the admission limit) */
  int32_t max_inflight;     /* requests admitted at once, 1..4096 (pinned host slots are allocated for them) */
  int32_t max_batch;        /* requests per batch, 1..64 */
  int32_t streams;          /* batches on the device at once (one CUDA stream each), 1..16 */
  int32_t max_width, max_height; /* largest accepted frame */
  float z_min, z_max, delta_sup; /* preprocessing of request depth (outlier filter, Sec. 7) */
  dtsdf_icp_opts opts;      /* registration schedule of every request (lambda ignored) */
  dtsdf_batch_shape shape;  /* launch shape of the batched registration */
} dtsdf_server_params;

typedef struct {
  int32_t map;              /* index into the maps given to dtsdf_server_create */
  int32_t sim3;             /* 0: SE(3), 1: Sim(3) */
  dtsdf_intrinsics K;       /* frame size (<= max_width x max_height) and intrinsics */
  const float* depth;       /* host, K.height * K.width float32 z-depth; read when the request is
                               admitted, so it must stay valid until its result is returned; page-
                               locked memory is copied directly, other memory through a pinned slot */
  double T_prior[16];       /* camera -> world prior pose (row-major); the map is rendered there */
  uint64_t tag;             /* caller's tag, returned with the result */
} dtsdf_request;

typedef struct {
  uint64_t tag;
  uint64_t seq;             /* submission order */
  int32_t status;           /* DTSDF_OK, or DTSDF_ERR_DEGENERATE from the last iteration */
  int32_t batch_size;       /* requests in the batch that served it */
  double T_rel[16];         /* current camera -> render camera after registration */
  double T_wc[16];          /* refined camera -> world pose, T_prior T_rel */
  dtsdf_icp_stats stats;    /* last iteration's statistics */
  double t_submit, t_admit, t_done; /* seconds on the server clock: submission, launch, completion seen */
} dtsdf_result;

typedef struct {
  int64_t submitted, admitted, completed, batches, pending, inflight, peak_inflight;
  int64_t bytes_in_use, peak_bytes; /* arena bytes held by admitted requests */
} dtsdf_server_stats_t;

/* Create a server over n_maps maps of the current device. DTSDF_ERR_INVALID_ARG for bad
 * parameters, DTSDF_ERR_OOM if the arena or host slots cannot be allocated. */
DTSDF_API dtsdf_status dtsdf_server_create(const dtsdf_map* maps, int32_t n_maps, const dtsdf_server_params* params,
                                           dtsdf_server* out);

/* Queue one request (thread-safe, returns at once; *seq, if given, receives its submission
 * number). DTSDF_ERR_INVALID_ARG for a bad request or one whose working set exceeds the
 * whole budget. */
DTSDF_API dtsdf_status dtsdf_server_submit(dtsdf_server s, const dtsdf_request* r, uint64_t* seq);

/* Move up to cap completed results, oldest completion first, into out (host); *n receives the
 * count. Waits up to wait_us microseconds when none is ready; DTSDF_ERR_TIMEOUT (with *n = 0)
 * when that wait runs out with no result (wait_us = 0 never waits and returns DTSDF_OK).
 * DTSDF_ERR_CUDA if a batch failed on the device (message in dtsdf_last_error). */
DTSDF_API dtsdf_status dtsdf_server_poll(dtsdf_server s, dtsdf_result* out, int32_t cap, int32_t* n,
                                         int32_t wait_us);

DTSDF_API dtsdf_status dtsdf_server_stats(dtsdf_server s, dtsdf_server_stats_t* st);

/* Seconds since the server was created (the clock of the result time stamps). */
DTSDF_API double dtsdf_server_clock(dtsdf_server s);

/* Finish every submitted request, stop the worker and free the server's memory. Results not
 * yet polled are dropped. */
DTSDF_API dtsdf_status dtsdf_server_destroy(dtsdf_server s);

/* Voxel recycling (Sec. 3: bricks that repeated carving turned into free space go back to the
 * pool). Every brick of a hash map whose core voxels with weight > 0 all have sdf >= free_sdf
 * (0 < free_sdf <= 1; e.g. 0.75: at least 3/4 of the truncation range in front of any surface)
 * is detached: its slot leaves the block's directory entry and hash mask, its copies in the
 * neighbours' aprons and its own voxels return to the empty value (sdf 1, weight 0), and the
 * allocator hands it out again before growing the pool. Stream-ordered with the map's other
 * work: run it on the map's stream between frames (or on another stream after an event), never
 * concurrently with dtsdf_integrate* or a render of the same map. recycled (host, or NULL)
 * receives the number of bricks detached; then the call waits for the stream. Dense maps:
 * DTSDF_ERR_INVALID_ARG. */
DTSDF_API dtsdf_status dtsdf_recycle(dtsdf_map map, float free_sdf, int64_t* recycled, void* stream);

/* Quality-reference render with the free-space combination of Sec. 4, Alg. 1 ("Compute
 * Combined TSDF"): at every sample the point is first classified as free space or occupied -
 * free if some direction with Phi^D > 0 has no zero transition between the point and the camera,
 * or if at its first such transition q no direction has Phi^D~(q) < 0 with a gradient normal
 * facing the camera - and the value is the fused-weight average of the directions on that side
 * (a direction whose gradient normal lies outside its angular range is ignored; a flat field
 * keeps its information). Same sample grid, refinement and output layout as dtsdf_render (depth,
 * normal with the depth in w); the normal is the normalised fused-weight sum of the chosen
 * directions' normals; no colour (out->color, if given, is zeroed). One thread per pixel, a
 * march that walks every sample in allocated block cells: slower than dtsdf_render, meant for
 * quality comparison on synthetic maps. Asynchronous. */
DTSDF_API dtsdf_status dtsdf_render_freespace(dtsdf_map map, const dtsdf_intrinsics* K, const double T_wc[16],
                                              const dtsdf_render_out* out, void* stream);

/* Same with the pose in device memory (16 doubles, row-major camera-to-world). */
DTSDF_API dtsdf_status dtsdf_render_freespace_dev(dtsdf_map map, const dtsdf_intrinsics* K, const double* T_wc_dev,
                                                  const dtsdf_render_out* out, void* stream);

/* ------------------------------------------------------------ input filters ---- */

/* Bilateral input filters (Sec. 8 settings: depth sigma_d = 5.0 px, sigma_r = 0.025 m, radius 5;
 * normals sigma_d = 2.5 px, sigma_r = 5.0, radius 5). The paper gives no formula; the filters
 * are the usual ones. Depth: after the outlier filter, each survivor becomes the mean of the
 * survivors in its (2r+1)^2 window weighted by exp(-(du^2+dv^2)/(2 sigma_d^2)) *
 * exp(-(z_j - z_i)^2/(2 sigma_r^2)), then is back-projected. Normals: after the normal
 * estimate, each normal becomes the normalised weighted sum of the window's normals with the
 * range term exp(-a^2/(2 sigma_r^2)), a the angle between the normals in DEGREES. radius 0 turns
 * a filter off (the default of a new map or ICP context). Radii 0..8; sigmas > 0 where used. */
typedef struct {
  int32_t depth_radius;
  float depth_sigma_d;   /* pixels */
  float depth_sigma_r;   /* metres */
  int32_t normal_radius;
  float normal_sigma_d;  /* pixels */
  float normal_sigma_r;  /* degrees */
} dtsdf_filter_opts;

/* Filters applied by the map's fusion preprocessing (NULL: both off). Takes effect at the next
 * dtsdf_integrate*. */
DTSDF_API dtsdf_status dtsdf_set_filters(dtsdf_map map, const dtsdf_filter_opts* f);

/* Filters applied by dtsdf_icp_set_frame (only the depth filter changes what ICP uses: the
 * pyramid is built from the filtered depth). NULL: both off. */
DTSDF_API dtsdf_status dtsdf_icp_set_filters(dtsdf_icp icp, const dtsdf_filter_opts* f);

/* Preprocessing of one frame as fusion runs it (Sec. 7): outlier filter, optional bilateral
 * depth filter, normals, optional bilateral normal filter (f may be NULL). points and normals:
 * device float4 arrays of width x height, (x, y, z, 1) / (nx, ny, nz, 1) in the camera frame where
 * present, zeros elsewhere. Asynchronous; allocates stream-ordered scratch when a filter is on. */
DTSDF_API dtsdf_status dtsdf_preprocess(const dtsdf_frame* frame, float z_min, float z_max, float delta_sup,
                                        const dtsdf_filter_opts* f, float* points, float* normals, void* stream);

/* Post-fusion error (Sec. 8.2): sum of |rendered - measured| over the n pixels where both depths
 * are positive, and that pixel count, as out_dev[0], out_dev[1] (device, 2 doubles; the MAE is
 * their ratio). rendered, measured: device float32 (may be NULL when n = 0). FP64 sums in a
 * fixed order (deterministic).
 * Asynchronous; uses 4 KB of stream-ordered scratch. */
DTSDF_API dtsdf_status dtsdf_depth_mae(const float* rendered, const float* measured, int64_t n, double* out_dev,
                                       void* stream);

/* ------------------------------------------------------ multi-sensor scale ---- */

/* Multi-sensor scale anchoring (Sec. 6, Eq. scale_anchor). n frames in time order (host
 * arrays): log_scale_est[k] = log of the scale of frame k's Sim(3) estimate against the model,
 * sensor[k] = its sensor. The anchor sensor's scale is held at exp(anchor_log_scale); a drift of
 * the model's scale shows as a common offset of every sensor's estimate, which the anchor
 * sensor's estimate measures. Output: anchor_log_scale for the anchor's frames; for the others
 * est[k] - (est[j] - anchor_log_scale), j the anchor's latest frame before k (est[k] itself
 * before the anchor's first frame). With anchor_log_scale = 0 this is the paper's
 * s_i = s^_i - s^_0 in the log domain. log_scale_out may alias log_scale_est. Host arithmetic
 * only: no device is used. DTSDF_ERR_INVALID_ARG for null arrays or n < 0. */
DTSDF_API dtsdf_status dtsdf_scale_anchor(const double* log_scale_est, const int32_t* sensor, int64_t n,
                                          int32_t anchor_sensor, double anchor_log_scale, double* log_scale_out);

/* depth_out[i] = scale * depth_in[i] (float32, device, n pixels; invalid 0 stays 0): a sensor's
 * depth brought to the model's metric before fusion (Sec. 6: with the scale known, the images
 * are scaled and SE(3) poses serve the rest of the pipeline). depth_out may equal depth_in.
 * Asynchronous on `stream`. DTSDF_ERR_INVALID_ARG for null pointers, n < 0 or a scale that is
 * not finite and positive. */
DTSDF_API dtsdf_status dtsdf_depth_scale(const float* depth_in, float* depth_out, int64_t n, float scale,
                                         void* stream);

/* Exponential map of se(3) (sim3 = 0, xi[6]) or sim(3) (sim3 = 1, xi[7]) evaluated by the
 * library's device code (the closed form of the matrix exponential of the 4x4 generator);
 * out: host 16 doubles. Synchronous; exposed for verification. */
DTSDF_API dtsdf_status dtsdf_exp(int32_t sim3, const double* xi, double out[16]);

/* Message of the calling thread's most recent error ("" if none). */
DTSDF_API const char* dtsdf_last_error(void);

/* Library version string. */
DTSDF_API const char* dtsdf_version(void);

/* Device and pinned host allocations the library holds right now (maps, registration contexts,
 * servers and their buffers; stream-ordered scratch is not counted). The paper has no
 * counterpart: a diagnostic for error paths. Every create call that fails (for instance under
 * the allocation-failure injection: with the environment variable DTSDF_FAIL_ALLOC set to N,
 * the N-th allocation of a dtsdf_create, dtsdf_icp_create or dtsdf_server_create call, counted
 * from 0, and every later one fails as if the device were out of memory, and the call returns
 * DTSDF_ERR_OOM) leaves this count where it was. */
DTSDF_API int64_t dtsdf_live_allocations(void);

#ifdef __cplusplus
}
#endif
#endif /* DTSDF_H */
