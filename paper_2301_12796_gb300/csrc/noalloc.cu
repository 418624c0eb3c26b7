// dtsdf_icp_step_noalloc: one Gauss-Newton iteration of point-to-plane ICP that never
// allocates device memory.
//
// Who needs this: callers that cannot call cudaMalloc at the moment they want an ICP
// iteration - real-time loops where cudaMalloc's implicit synchronisation would stall every
// other stream on the device, and host applications that hand out all device memory from
// their own pool and forbid libraries from allocating behind their back. They pass in device
// buffers for every input and output; the only memory this entry point uses beyond them is
// the fixed scratch below, which exists as soon as the library is loaded.
//
// Scratch: the per-CTA partial sums of the reduction, the completion ticket and the stop
// flag live in one file-scope __device__ array. Every device that loads the library holds
// it (NOALLOC_SCRATCH_BYTES) until the process exits. All calls share it and it keeps the
// last call's contents; calls whose work overlaps on the GPU (different streams, no ordering
// between them) race on it and must not be issued.
#include <mutex>

#include "internal.h"

namespace dtsdf {

// One CTA per 1024 pixels (256 threads x 4 pixels); at most NOALLOC_MAX_CTAS CTAs, i.e. at most
// NOALLOC_MAX_PIXELS pixels in the current image.
constexpr int NOALLOC_MAX_CTAS = 1024;
constexpr int NOALLOC_PIXELS_PER_CTA = 1024;
constexpr int64_t NOALLOC_MAX_PIXELS = (int64_t)NOALLOC_MAX_CTAS * NOALLOC_PIXELS_PER_CTA;
constexpr int NOALLOC_PARTIAL_FLOATS = 64;  // per CTA, >= the 38 sums of the 7x7 system
// layout: [0, MAX_CTAS * 64) floats of partials, then 2 words: ticket (uint32), stop flag (int32)
constexpr size_t NOALLOC_SCRATCH_WORDS = (size_t)NOALLOC_MAX_CTAS * NOALLOC_PARTIAL_FLOATS + 64;
constexpr size_t NOALLOC_SCRATCH_BYTES = NOALLOC_SCRATCH_WORDS * 4;  // 256 KB + 256 B

static __device__ __align__(256) uint32_t g_noalloc_scratch[NOALLOC_SCRATCH_WORDS];
static_assert(sizeof(g_noalloc_scratch) == NOALLOC_SCRATCH_BYTES, "scratch size");

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (set up once per device, with
// that device current, and kept for the life of the library: after cudaDeviceReset the module
// may load at another address, so the library must not be used across a reset). The host-side
// symbol is only a stand-in and must never reach a kernel.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace dtsdf

using namespace dtsdf;

extern "C" {

dtsdf_status dtsdf_icp_step_noalloc(const float* depth, const dtsdf_intrinsics* K_cur, const dtsdf_render_out* ref,
                                    const dtsdf_intrinsics* K_ref, int32_t sim3, float eps, float z_min,
                                    int32_t min_rows, double stop_norm, double* T_rel_dev,
                                    dtsdf_icp_stats* stats_dev, void* stream) {
  if (!depth || !K_cur || !ref || !ref->normals || !K_ref || !T_rel_dev || !stats_dev || (sim3 != 0 && sim3 != 1) ||
      !(eps > 0) || !(z_min > 0) || min_rows < 0 || !(stop_norm >= 0) || K_cur->width <= 0 || K_cur->height <= 0 ||
      K_ref->width <= 0 || K_ref->height <= 0 || !(K_cur->fx > 0) || !(K_cur->fy > 0) || !(K_ref->fx > 0) ||
      !(K_ref->fy > 0))
    return set_error(DTSDF_ERR_INVALID_ARG, "dtsdf_icp_step_noalloc: bad argument");
  const int64_t npix = (int64_t)K_cur->width * K_cur->height;
  if (npix > NOALLOC_MAX_PIXELS)
    return set_error(DTSDF_ERR_INVALID_ARG,
                     "dtsdf_icp_step_noalloc: the current image exceeds the fixed scratch (at most 1048576 pixels)");
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return set_error(DTSDF_ERR_CUDA, "dtsdf_icp_step_noalloc: cudaGetSymbolAddress failed");
  cudaStream_t s = (cudaStream_t)stream;
  float* partials = (float*)base;
  uint32_t* ticket = (uint32_t*)base + (size_t)NOALLOC_MAX_CTAS * NOALLOC_PARTIAL_FLOATS;
  int32_t* stop = (int32_t*)(ticket + 1);
  // the ticket and the stop flag must start at zero; the caller's stats accumulate an
  // iteration count and are cleared too. The partials are fully rewritten by every call.
  e = cudaMemsetAsync(ticket, 0, 2 * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(stats_dev, 0, sizeof(dtsdf_icp_stats), s);
  if (e != cudaSuccess) return set_error(DTSDF_ERR_CUDA, "dtsdf_icp_step_noalloc: scratch reset failed");
  IcpLaunch L;
  L.depth = depth;
  L.inten = nullptr;
  L.K.W = K_cur->width;
  L.K.H = K_cur->height;
  L.K.fx = K_cur->fx;
  L.K.fy = K_cur->fy;
  L.K.cx = K_cur->cx;
  L.K.cy = K_cur->cy;
  L.ref = (const float4*)ref->normals;
  L.Kr.W = K_ref->width;
  L.Kr.H = K_ref->height;
  L.Kr.fx = K_ref->fx;
  L.Kr.fy = K_ref->fy;
  L.Kr.cx = K_ref->cx;
  L.Kr.cy = K_ref->cy;
  L.eps = eps;
  L.zmin = z_min;
  L.kf = nullptr;
  L.Kk = L.K;
  for (int i = 0; i < 9; ++i) L.Rrs[i] = 0.f;
  for (int i = 0; i < 3; ++i) L.trs[i] = 0.f;
  L.Trs_dev = nullptr;
  L.thr = 0.f;
  L.lambda = 0.f;
  L.pose = T_rel_dev;
  L.partials = partials;
  L.ticket = ticket;
  L.stop = stop;
  L.stats = stats_dev;
  L.min_rows = min_rows;
  L.stop_norm = stop_norm;
  L.kahan = 0;
  const int grid = (int)((npix + NOALLOC_PIXELS_PER_CTA - 1) / NOALLOC_PIXELS_PER_CTA);
  launch_icp(L, sim3, false, grid < 1 ? 1 : grid, s);
  if (cudaGetLastError() != cudaSuccess) return set_error(DTSDF_ERR_CUDA, "dtsdf_icp_step_noalloc: launch failed");
  return DTSDF_OK;
}

}  // extern "C"
