// Host-side declarations shared by the translation units of libdtsdf.
#pragma once

#include "common.cuh"

namespace dtsdf {

// Levenberg-Marquardt state of one pyramid level (device memory; zero = no evaluation yet).
struct LmState {
  double mu, nu, E, pred;
  double pose[16];  // accepted pose
  double H[49];     // accepted system (row-major 7x7) and right-hand side
  double g[7];
  int have;
};

struct IcpLaunch {
  const float* depth;
  const float* inten;
  Intr K;
  const float4* ref;
  Intr Kr;
  float eps, zmin;
  const float4* kf;
  Intr Kk;
  float Rrs[9], trs[3];
  const double* Trs_dev;
  float thr, lambda;
  double* pose;
  float* partials;
  uint32_t* ticket;
  int32_t* stop;
  dtsdf_icp_stats* stats;
  int min_rows;
  double stop_norm;
  int kahan;
  LmState* lm = nullptr;  // Levenberg-Marquardt state, or null for Gauss-Newton
};

// Record a message for dtsdf_last_error() and return the status.
dtsdf_status set_error(dtsdf_status s, const char* msg);

// Device and pinned host allocations of the library go through these. Failure injection for
// tests of the error paths: with the environment variable DTSDF_FAIL_ALLOC set to N, the N-th
// allocation (counted from 0) after alloc_hook_begin() on the calling thread, and every later
// one, fails with cudaErrorMemoryAllocation without allocating.
// dt_free / dt_free_host release them (null is a no-op), and the library keeps the count of its
// live allocations for dtsdf_live_allocations().
void alloc_hook_begin();
cudaError_t dt_malloc(void** p, size_t bytes);
cudaError_t dt_malloc_host(void** p, size_t bytes);
cudaError_t dt_free(void* p);
cudaError_t dt_free_host(void* p);
int64_t live_allocations();

// Bilateral input filters (radius 0 = off); layout of dtsdf_filter_opts.
struct FilterOpts {
  int depth_radius;
  float depth_sigma_d, depth_sigma_r;
  int normal_radius;
  float normal_sigma_d, normal_sigma_r;
};

// Outlier filter and normals; with f (and a scratch image tmp of W x H float4) the bilateral depth
// filter runs between them and the bilateral normal filter after them.
void launch_preprocess(const float* depth, const Intr& K, float zmin, float zmax, float dsup, float4* P, float4* N,
                       cudaStream_t s, const FilterOpts* f = nullptr, float4* tmp = nullptr);
void launch_alloc(const MapView& m, const float4* P, const float4* N, int npix, const Pose32& T, const double* Tdev,
                  int num_sms, cudaStream_t s);
void launch_dense_fill(const MapView& m, int nb, cudaStream_t s);
void launch_pool_init(const MapView& m, int with_color, int num_sms, cudaStream_t s);
// Fusion of one frame followed by the apron refresh of the bricks near the changed ones.
void launch_fuse(const MapView& m, const Intr& K, const Pose32& T, const double* Tdev, const float4* P,
                 const float4* N, const uint8_t* rgb, uint8_t* J, int num_sms, cudaStream_t s);
// Apron refresh and bound of every brick (after an import).
void launch_apron_refresh_all(const MapView& m, int num_sms, cudaStream_t s);
void launch_pose_compose(const double* A, int invert_a, const double* B, double* C, cudaStream_t s);
void launch_recycle(const MapView& m, float free_sdf, int32_t* list, uint32_t* nlist, int num_sms, cudaStream_t s);
cudaError_t launch_render_freespace(const MapView& m, const Intr& K, const Pose32& T, const double* Tdev, float* depth,
                                    float4* normals, float4* color, cudaStream_t s);
constexpr int MAE_PARTIAL_DOUBLES = 2 * 256;
void launch_mae(const float* a, const float* b, int64_t n, double* part, double* out, cudaStream_t s);
void launch_depth_scale(const float* in, float* out, int64_t n, float scale, cudaStream_t s);
void launch_import(const MapView& m, const int32_t* coords, const float* vox, int64_t n, bool allocate, int num_sms,
                   cudaStream_t s);
void launch_export(const MapView& m, int64_t cap, int32_t* coords, float* vox, int num_sms, cudaStream_t s);
// One frame of a render launch: intrinsics, camera -> world pose (device pointer, else T) and
// caller-owned outputs. tiles_x / start are filled in by launch_render_jobs.
struct RenderJob {
  Intr K;
  const double* Tdev;
  Pose32 T;
  double T64[12];  // the host pose in double precision (rotation rows, then translation); unused with Tdev
  float* depth;
  float4* normals;
  float4* color;
  int tiles_x;
  int start;
};

constexpr int MAX_RENDER_JOBS = 64;

// Kernel arguments of a render launch over NJ frames. The work items are the pixels of the
// frames' 8x4 tiles, frame after frame; `queue` counts the items handed out and must be
// zero when the launch starts.
template <int NJ>
struct RenderBatch {
  RenderJob job[NJ];
  int njobs;
  int total;
  unsigned* queue;
  uint8_t* touched;  // instrumentation build only (brick flags + counters), else null
  int max_samples;
  int refill;        // lanes per refill group (1 .. 32): a group takes new rays when all its lanes finish
  int tile_w;        // pixel tile of 32 rays: tile_w x (32 / tile_w)
  // camera-depth range per ray tile (bit patterns of non-negative floats) of the allocated
  // blocks whose box covers one of the tile's pixels; zlo = 0xFFFFFFFF: no block. Null: none.
  const uint32_t* zlo;
  const uint32_t* zhi;
  // crossings found by the march, refined by the second pass: (pixel, k << 6 | job) per ray
  // with a crossing between samples k - 1 and k; nhits counts them (zero at launch)
  int2* hits;
  unsigned* nhits;
};

// Launch shape of a render: persistent CTAs (0 = one wave of resident CTAs), the lanes per
// refill group (a group of consecutive lanes takes new rays when all of them have finished)
// and the width of the 32-ray pixel tiles (1, 2, 4, 8, 16 or 32).
struct RenderShape {
  int ctas = 0;
  int refill = 32;
  int tile_w = 4;
};

// Combined TSDF: device state of the conditional combination (combined.cu).
struct CombState {
  double pose[16];     // camera -> world pose of the current combination
  uint32_t gen;        // generation of the current combination (comb_gen of its blocks)
  uint32_t frames;     // combined renders so far
  uint32_t since;      // combined renders since the last full combination
  uint32_t full;       // this call recombines every block in view
  uint32_t pool_mark;  // brick count at the previous call
  uint32_t pool_from;  // bricks from this index on were allocated since the previous call
  uint32_t taken_mark; // recycled bricks handed out again, at the previous call
};
struct Pose64 {
  double T[16];
};
struct CombFrame {
  float pl[4][3];  // inward unit normals of the padded frustum's side planes (camera frame)
  // Failure-detection test hook (environment variable DTSDF_TEST_COMBINE_STALL set and not 0):
  // the combine pass's producer warp issues no stage, so the consumers' bounded waits run out.
  int stall;
};
// Conditional combination and the combine pass for a render at T (device pose, else host).
void launch_combine(const MapView& m, CombState* st, const Intr& K, const double* Tdev, const double* Thost, int force,
                    int num_sms, cudaStream_t s);

// Render njobs (1..MAX_RENDER_JOBS) frames in one persistent launch. With a memory pool, a
// pre-pass first records per ray tile the depth range of the allocated blocks in view
// (stream-ordered scratch from `pool`), so rays start and end their march there.
cudaError_t launch_render_jobs(const MapView& m, const RenderJob* jobs, int njobs, unsigned* queue, cudaStream_t s,
                               uint8_t* touched, const RenderShape& shape, cudaMemPool_t pool, bool combined = false);
void launch_frame_pyramid(const float4* P, const uint8_t* rgb, int levels, const Intr* K, float* const* depth,
                          float* const* inten, cudaStream_t s);
void launch_keyframe_pyramid(const uint8_t* rgb, int levels, const Intr* K, float* const* tmpI, float4* const* kf,
                             cudaStream_t s);
constexpr int ICP_CTA_THREADS = 256;  // threads per CTA of one ICP iteration
void launch_icp(const IcpLaunch& L, int sim3, bool photo, int grid, cudaStream_t s);
void launch_exp(int dim, const double* xi, double* T, cudaStream_t s);

// One problem of a batched registration: current-frame pyramid (levels of the batch),
// reference render, pose (device, 16 doubles, read and written) and optional stats.
constexpr int ICP_MAX_LEVELS = 4;
struct IcpProblemDev {
  const float* depth[ICP_MAX_LEVELS];
  Intr K[ICP_MAX_LEVELS];
  const float4* ref;
  Intr Kr;
  double* pose;
  dtsdf_icp_stats* stats;
  int sim3;
};

constexpr int ICP_BATCH_MAX = 64;
struct IcpBatchArgs {
  IcpProblemDev p[ICP_BATCH_MAX];
  int n, levels;
  int iters[ICP_MAX_LEVELS];
  float eps[ICP_MAX_LEVELS];
  float zmin;
  int min_rows;
  double stop_norm;
};

// Batched registration, one cluster of `cluster` CTAs (threads each) per problem.
void launch_icp_batch(const IcpBatchArgs& a, int kahan, int cluster, int threads, cudaStream_t s, cudaError_t* err);

}  // namespace dtsdf
