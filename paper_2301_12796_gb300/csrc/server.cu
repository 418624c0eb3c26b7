// Serving: a request loop over device-resident maps that admits render + registration
// requests by device-memory footprint and runs them in continuous batches.
//
// A request carries one depth frame (host memory), its intrinsics, a prior camera -> world
// pose and the map it is to be registered against. Serving it is the tracking step of the
// paper without fusion: preprocessing and the depth pyramid of the frame (Sec. 7), a render
// of the map at the prior (Sec. 4), and the coarse-to-fine point-to-plane registration of the
// frame against that render in SE(3) or Sim(3) (Secs. 5 and 6), then T_wc = T_prior T_rel.
//
// Scheduling (no counterpart in the paper):
//   * Memory: every admitted request takes its working set (input depth, preprocessing
//     scratch, pyramid, render outputs, poses, statistics) from one device arena of a fixed
//     budget, first fit; a request is admitted only when its footprint fits. Maps are the
//     caller's and stay resident; they are not part of the budget.
//   * Continuous batching: the loop keeps up to `streams` batches on the device, one per
//     stream. As soon as a stream is idle and the head of the queue fits, everything pending
//     that fits (up to max_batch requests, in arrival order) is launched as one batch: per
//     request H2D copy, preprocessing and pyramid; one persistent render launch per map over
//     the batch's frames of any sizes; one batched registration launch (a thread-block
//     cluster per request, SE(3) and Sim(3) mixed); one pose composition; one D2H copy per
//     request. Requests that arrive while batches run wait only for the next free stream,
//     and batches on different streams overlap on the device.
//   * Every kernel of a request computes the same values whatever else shares its launch (the
//     render is per pixel, each registration owns its cluster and reduces in a fixed order),
//     so a result does not depend on the mix it was served in.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string.h>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace dtsdf {
namespace {

constexpr size_t ALIGN = 256;
constexpr int SERVE_MAX_STREAMS = 16;

size_t align_up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

// First-fit allocator over [0, size) of a device arena, with coalescing of free ranges.
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = 0;
    peak_ = 0;
  }
  // offset of a block of `bytes` (a multiple of ALIGN), or SIZE_MAX
  size_t alloc(size_t bytes) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > bytes) free_[off + bytes] = len - bytes;
      used_ += bytes;
      if (used_ > peak_) peak_ = used_;
      return off;
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t bytes) {
    used_ -= bytes;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0, peak_ = 0;
};

// Device working set of one request, carved from its arena block.
struct ReqDev {
  float* depth_in;
  float4* P;
  float4* N;
  float* pyr[ICP_MAX_LEVELS];
  float* ref_depth;
  float4* ref_normals;
  double* io;  // 16 prior, 16 T_rel (in: identity), then out: 16 T_rel, 16 T_wc, stats
};

// Layout of the pose/statistics block shared by the device working set and the pinned host
// slot, so one copy moves each direction.
constexpr size_t IO_IN_DOUBLES = 32;                                           // prior, T_rel
constexpr size_t IO_OUT_BYTES = sizeof(double) * 32 + sizeof(dtsdf_icp_stats);  // T_rel, T_wc, stats
constexpr size_t IO_BYTES = sizeof(double) * IO_IN_DOUBLES + IO_OUT_BYTES;

struct Req {
  dtsdf_request r;
  uint64_t seq;
  double t_submit, t_admit;
  int levels;
  Intr K[ICP_MAX_LEVELS];
  size_t bytes, off;
  int host_slot;
  bool pinned_input;
  ReqDev d;
};

struct Batch {
  std::vector<Req*> reqs;
  int stream;
  cudaEvent_t done;
};

// Per-request pose composition of a batch: T_wc = T_prior T_rel.
struct ComposeArgs {
  const double* io[64];
  double* out[64];
  int n;
};

__global__ void k_serve_compose(ComposeArgs a) {
  const int i = blockIdx.x;
  const int e = threadIdx.x;
  if (i >= a.n || e >= 16) return;
  const double* prior = a.io[i];
  const double* rel = a.io[i] + 16;
  const int r = e >> 2, c = e & 3;
  double acc = 0.0;
  for (int q = 0; q < 4; ++q) acc += prior[4 * r + q] * rel[4 * q + c];
  a.out[i][16 + e] = acc;                    // T_wc
  a.out[i][e] = rel[e];                      // T_rel after the registration
}

Intr to_intr_s(const dtsdf_intrinsics& K) {
  Intr k;
  k.W = K.width;
  k.H = K.height;
  k.fx = K.fx;
  k.fy = K.fy;
  k.cx = K.cx;
  k.cy = K.cy;
  return k;
}

Intr half_intr(const Intr& k) {
  Intr n;
  n.W = k.W / 2;
  n.H = k.H / 2;
  n.fx = k.fx / 2.0f;
  n.fy = k.fy / 2.0f;
  n.cx = (k.cx - 0.5f) / 2.0f;
  n.cy = (k.cy - 0.5f) / 2.0f;
  return n;
}

}  // namespace
}  // namespace dtsdf

using namespace dtsdf;

struct dtsdf_server_s {
  dtsdf_server_params p;
  std::vector<dtsdf_map> maps;
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  // device arena
  char* arena_base = nullptr;
  Arena arena;
  // pinned host slots: staging of a pageable input depth + the pose/statistics block
  char* host_base = nullptr;
  size_t host_slot_bytes = 0;
  std::vector<int> free_slots;
  cudaStream_t streams[SERVE_MAX_STREAMS] = {};
  Batch* running[SERVE_MAX_STREAMS] = {};
  std::vector<cudaEvent_t> events;
  // queues
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::deque<dtsdf_result> done;
  uint64_t next_seq = 0;
  bool stop = false;
  std::string error;
  dtsdf_server_stats_t st;
  std::thread worker;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

size_t request_bytes(const dtsdf_server_s* s, const Intr* K, int levels) {
  const size_t n0 = (size_t)K[0].W * K[0].H;
  size_t b = align_up(sizeof(float) * n0) + 2 * align_up(sizeof(float4) * n0);
  for (int l = 0; l < levels; ++l) b += align_up(sizeof(float) * (size_t)K[l].W * K[l].H);
  b += align_up(sizeof(float) * n0) + align_up(sizeof(float4) * n0);
  b += align_up(IO_BYTES);
  (void)s;
  return b;
}

void carve(Req* q, char* base) {
  char* p = base + q->off;
  const size_t n0 = (size_t)q->K[0].W * q->K[0].H;
  auto take = [&](size_t bytes) {
    char* r = p;
    p += align_up(bytes);
    return r;
  };
  q->d.depth_in = (float*)take(sizeof(float) * n0);
  q->d.P = (float4*)take(sizeof(float4) * n0);
  q->d.N = (float4*)take(sizeof(float4) * n0);
  for (int l = 0; l < ICP_MAX_LEVELS; ++l)
    q->d.pyr[l] = l < q->levels ? (float*)take(sizeof(float) * (size_t)q->K[l].W * q->K[l].H) : nullptr;
  q->d.ref_depth = (float*)take(sizeof(float) * n0);
  q->d.ref_normals = (float4*)take(sizeof(float4) * n0);
  q->d.io = (double*)take(IO_BYTES);
}

char* host_slot(dtsdf_server_s* s, int i) { return s->host_base + (size_t)i * s->host_slot_bytes; }
double* host_io(dtsdf_server_s* s, int i) { return (double*)host_slot(s, i); }
float* host_stage(dtsdf_server_s* s, int i) { return (float*)(host_slot(s, i) + align_up(IO_BYTES)); }

// Launch one batch on stream `si`. Called by the worker only.
cudaError_t launch_batch(dtsdf_server_s* s, Batch* b) {
  cudaStream_t st = s->streams[b->stream];
  cudaError_t e = cudaSuccess;
  const dtsdf_server_params& P = s->p;
  for (Req* q : b->reqs) {
    const size_t n0 = (size_t)q->K[0].W * q->K[0].H;
    double* hio = host_io(s, q->host_slot);
    memcpy(hio, q->r.T_prior, sizeof(double) * 16);
    for (int i = 0; i < 16; ++i) hio[16 + i] = (i % 5 == 0) ? 1.0 : 0.0;
    const float* src = q->r.depth;
    if (!q->pinned_input) {
      memcpy(host_stage(s, q->host_slot), q->r.depth, sizeof(float) * n0);
      src = host_stage(s, q->host_slot);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(q->d.depth_in, src, sizeof(float) * n0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(q->d.io, hio, sizeof(double) * IO_IN_DOUBLES, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    launch_preprocess(q->d.depth_in, q->K[0], P.z_min, P.z_max, P.delta_sup, q->d.P, q->d.N, st);
    launch_frame_pyramid(q->d.P, nullptr, q->levels, q->K, q->d.pyr, nullptr, st);
  }
  // one render launch per map over the batch's frames
  std::vector<dtsdf_render_job> jobs;
  for (size_t mi = 0; mi < s->maps.size() && e == cudaSuccess; ++mi) {
    jobs.clear();
    for (Req* q : b->reqs) {
      if (q->r.map != (int)mi) continue;
      dtsdf_render_job j;
      memset(&j, 0, sizeof(j));
      j.K = q->r.K;
      j.T_wc_dev = q->d.io;
      j.out.depth = q->d.ref_depth;
      j.out.normals = (float*)q->d.ref_normals;
      j.out.color = nullptr;
      jobs.push_back(j);
    }
    if (jobs.empty()) continue;
    if (dtsdf_render_batch(s->maps[mi], jobs.data(), (int32_t)jobs.size(), st) != DTSDF_OK) return cudaErrorUnknown;
  }
  // batched registration
  IcpBatchArgs a;
  memset(&a, 0, sizeof(a));
  a.n = (int)b->reqs.size();
  a.levels = P.opts.levels;
  for (int l = 0; l < P.opts.levels; ++l) {
    a.iters[l] = P.opts.iters[l];
    a.eps[l] = P.opts.eps[l];
  }
  a.zmin = P.opts.z_min;
  a.min_rows = P.opts.min_rows;
  a.stop_norm = P.opts.stop_norm;
  ComposeArgs ca;
  memset(&ca, 0, sizeof(ca));
  ca.n = a.n;
  for (int i = 0; i < a.n; ++i) {
    Req* q = b->reqs[(size_t)i];
    IcpProblemDev& d = a.p[i];
    for (int l = 0; l < q->levels; ++l) {
      d.depth[l] = q->d.pyr[l];
      d.K[l] = q->K[l];
    }
    d.ref = q->d.ref_normals;
    d.Kr = q->K[0];
    d.pose = q->d.io + 16;
    d.stats = (dtsdf_icp_stats*)(q->d.io + IO_IN_DOUBLES + 32);
    d.sim3 = q->r.sim3;
    ca.io[i] = q->d.io;
    ca.out[i] = q->d.io + IO_IN_DOUBLES;
  }
  launch_icp_batch(a, P.opts.kahan, P.shape.cluster, P.shape.threads, st, &e);
  if (e != cudaSuccess) return e;
  k_serve_compose<<<a.n, 16, 0, st>>>(ca);
  e = cudaGetLastError();
  for (Req* q : b->reqs) {
    if (e != cudaSuccess) break;
    e = cudaMemcpyAsync(host_io(s, q->host_slot) + IO_IN_DOUBLES, q->d.io + IO_IN_DOUBLES, IO_OUT_BYTES,
                        cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->done, st);
  return e;
}

void retire(dtsdf_server_s* s, Batch* b, double t_done) {
  std::lock_guard<std::mutex> lk(s->mu);
  for (Req* q : b->reqs) {
    dtsdf_result r;
    memset(&r, 0, sizeof(r));
    const double* hio = host_io(s, q->host_slot);
    r.tag = q->r.tag;
    r.seq = q->seq;
    memcpy(r.T_rel, hio + IO_IN_DOUBLES, sizeof(double) * 16);
    memcpy(r.T_wc, hio + IO_IN_DOUBLES + 16, sizeof(double) * 16);
    memcpy(&r.stats, hio + IO_IN_DOUBLES + 32, sizeof(dtsdf_icp_stats));
    r.status = r.stats.status;
    r.batch_size = (int32_t)b->reqs.size();
    r.t_submit = q->t_submit;
    r.t_admit = q->t_admit;
    r.t_done = t_done;
    s->done.push_back(r);
    s->arena.release(q->off, q->bytes);
    s->free_slots.push_back(q->host_slot);
    s->st.completed++;
    s->st.inflight--;
    delete q;
  }
  s->st.bytes_in_use = (int64_t)s->arena.used();
  s->cv_done.notify_all();
}

void worker_main(dtsdf_server_s* s) {
  cudaSetDevice(s->device);
  const int ns = s->p.streams;
  int rr = 0;
  for (;;) {
    bool progressed = false;
    // 1. retire finished batches
    for (int i = 0; i < ns; ++i) {
      Batch* b = s->running[i];
      if (!b) continue;
      const cudaError_t q = cudaEventQuery(b->done);
      if (q == cudaErrorNotReady) continue;
      const double t = s->now();
      if (q != cudaSuccess) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->error = std::string("batch failed: ") + cudaGetErrorString(q);
      }
      retire(s, b, t);
      s->events.push_back(b->done);
      delete b;
      s->running[i] = nullptr;
      progressed = true;
    }
    // 2. admit: the next idle stream takes everything pending that fits, in arrival order
    int idle = -1;
    for (int k = 0; k < ns; ++k) {
      const int i = (rr + k) % ns;
      if (!s->running[i]) {
        idle = i;
        break;
      }
    }
    Batch* nb = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (idle >= 0) {
        while (!s->pending.empty() && (!nb || (int)nb->reqs.size() < s->p.max_batch) &&
               s->st.inflight < s->p.max_inflight && !s->free_slots.empty()) {
          Req* q = s->pending.front();
          const size_t off = s->arena.alloc(q->bytes);
          if (off == SIZE_MAX) break;  // head of the queue waits for memory (no overtaking)
          q->off = off;
          q->host_slot = s->free_slots.back();
          s->free_slots.pop_back();
          carve(q, s->arena_base);
          s->pending.pop_front();
          if (!nb) {
            nb = new Batch();
            nb->stream = idle;
            nb->done = s->events.back();
            s->events.pop_back();
          }
          nb->reqs.push_back(q);
          s->st.inflight++;
          if (s->st.inflight > s->st.peak_inflight) s->st.peak_inflight = s->st.inflight;
        }
        if (nb) {
          s->st.admitted += (int64_t)nb->reqs.size();
          s->st.batches++;
          s->st.bytes_in_use = (int64_t)s->arena.used();
          s->st.peak_bytes = (int64_t)s->arena.peak();
        }
      }
      if (!nb && !progressed) {
        bool busy = false;
        for (int i = 0; i < ns; ++i) busy |= s->running[i] != nullptr;
        if (s->stop && !busy && s->pending.empty()) return;
        // idle: sleep until a submission; busy: poll the running batches every few microseconds
        if (busy)
          s->cv_work.wait_for(lk, std::chrono::microseconds(20));
        else
          s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        continue;
      }
    }
    if (nb) {
      const double t = s->now();
      for (Req* q : nb->reqs) q->t_admit = t;
      const cudaError_t e = launch_batch(s, nb);
      if (e != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(s->mu);
        s->error = std::string("batch launch failed: ") + cudaGetErrorString(e);
      }
      s->running[nb->stream] = nb;
      rr = (nb->stream + 1) % ns;
    }
  }
}

bool opts_valid(const dtsdf_icp_opts& o) {
  if (o.levels < 1 || o.levels > ICP_MAX_LEVELS || !(o.z_min > 0) || !(o.stop_norm >= 0) || o.min_rows < 0 ||
      o.lm != 0)
    return false;
  for (int l = 0; l < o.levels; ++l)
    if (o.iters[l] < 0 || o.iters[l] > 1000 || !(o.eps[l] > 0)) return false;
  return true;
}

}  // namespace

extern "C" {

dtsdf_status dtsdf_server_create(const dtsdf_map* maps, int32_t n_maps, const dtsdf_server_params* params,
                                 dtsdf_server* out) {
  alloc_hook_begin();
  if (!maps || n_maps < 1 || !params || !out) return set_error(DTSDF_ERR_INVALID_ARG, "server: bad argument");
  *out = nullptr;
  const dtsdf_server_params& p = *params;
  for (int i = 0; i < n_maps; ++i)
    if (!maps[i]) return set_error(DTSDF_ERR_INVALID_ARG, "server: null map");
  if (p.hbm_budget <= 0 || p.max_inflight < 1 || p.max_inflight > 4096 || p.max_batch < 1 ||
      p.max_batch > ICP_BATCH_MAX || p.streams < 1 || p.streams > SERVE_MAX_STREAMS || p.max_width < 16 ||
      p.max_height < 16 || p.max_width > 16384 || p.max_height > 16384 || !opts_valid(p.opts) || !(p.z_min > 0) ||
      !(p.z_max > p.z_min) || !(p.delta_sup > 0) ||
      !(p.shape.cluster == 1 || p.shape.cluster == 2 || p.shape.cluster == 4 || p.shape.cluster == 8 ||
        p.shape.cluster == 16) ||
      !(p.shape.threads == 128 || p.shape.threads == 256 || p.shape.threads == 512))
    return set_error(DTSDF_ERR_INVALID_ARG, "server: invalid parameters");
  dtsdf_server_s* s = new (std::nothrow) dtsdf_server_s();
  if (!s) return set_error(DTSDF_ERR_OOM, "server: host allocation");
  s->p = p;
  s->maps.assign(maps, maps + n_maps);
  memset(&s->st, 0, sizeof(s->st));
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaGetDevice(&s->device);
  const size_t npix = (size_t)p.max_width * p.max_height;
  s->host_slot_bytes = align_up(IO_BYTES) + align_up(sizeof(float) * npix);
  if (e == cudaSuccess) e = dt_malloc((void**)&s->arena_base, (size_t)p.hbm_budget);
  if (e == cudaSuccess) e = dt_malloc_host((void**)&s->host_base, s->host_slot_bytes * (size_t)p.max_inflight);
  for (int i = 0; i < p.streams && e == cudaSuccess; ++i)
    e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
  for (int i = 0; i < p.streams && e == cudaSuccess; ++i) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) s->events.push_back(ev);
  }
  if (e != cudaSuccess) {
    for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
    for (int i = 0; i < p.streams; ++i)
      if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
    dt_free(s->arena_base);
    if (s->host_base) dt_free_host(s->host_base);
    delete s;
    return set_error(e == cudaErrorMemoryAllocation ? DTSDF_ERR_OOM : DTSDF_ERR_CUDA, "server: allocation failed");
  }
  s->arena.reset((size_t)p.hbm_budget);
  for (int i = p.max_inflight - 1; i >= 0; --i) s->free_slots.push_back(i);
  s->worker = std::thread(worker_main, s);
  *out = s;
  return DTSDF_OK;
}

dtsdf_status dtsdf_server_submit(dtsdf_server s, const dtsdf_request* r, uint64_t* seq) {
  if (!s || !r || !r->depth || r->map < 0 || r->map >= (int)s->maps.size() || (r->sim3 != 0 && r->sim3 != 1) ||
      r->K.width < 16 || r->K.height < 16 || r->K.width > s->p.max_width || r->K.height > s->p.max_height ||
      !(r->K.fx > 0) || !(r->K.fy > 0))
    return set_error(DTSDF_ERR_INVALID_ARG, "server: bad request");
  for (int i = 0; i < 16; ++i)
    if (!(r->T_prior[i] == r->T_prior[i])) return set_error(DTSDF_ERR_INVALID_ARG, "server: bad prior pose");
  Req* q = new (std::nothrow) Req();
  if (!q) return set_error(DTSDF_ERR_OOM, "server: host allocation");
  q->r = *r;
  q->levels = s->p.opts.levels;
  q->K[0] = to_intr_s(r->K);
  for (int l = 1; l < q->levels; ++l) q->K[l] = half_intr(q->K[l - 1]);
  q->bytes = request_bytes(s, q->K, q->levels);
  if (q->bytes > (size_t)s->p.hbm_budget) {
    delete q;
    return set_error(DTSDF_ERR_INVALID_ARG, "server: request larger than the memory budget");
  }
  cudaPointerAttributes at;
  q->pinned_input = cudaPointerGetAttributes(&at, r->depth) == cudaSuccess && at.type == cudaMemoryTypeHost;
  cudaGetLastError();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete q;
      return set_error(DTSDF_ERR_INVALID_ARG, "server: shutting down");
    }
    q->seq = s->next_seq++;
    q->t_submit = s->now();
    s->pending.push_back(q);
    s->st.submitted++;
    if (seq) *seq = q->seq;
  }
  s->cv_work.notify_one();
  return DTSDF_OK;
}

dtsdf_status dtsdf_server_poll(dtsdf_server s, dtsdf_result* out, int32_t cap, int32_t* n, int32_t wait_us) {
  if (!s || !n || cap < 0 || (cap > 0 && !out) || wait_us < 0) return set_error(DTSDF_ERR_INVALID_ARG, "server: bad argument");
  std::unique_lock<std::mutex> lk(s->mu);
  bool waited_out = false;
  if (s->done.empty() && wait_us > 0)
    waited_out = !s->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return !s->done.empty(); });
  int32_t k = 0;
  while (k < cap && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *n = k;
  if (!s->error.empty()) return set_error(DTSDF_ERR_CUDA, s->error.c_str());
  if (waited_out) return set_error(DTSDF_ERR_TIMEOUT, "server: no result within the wait");
  return DTSDF_OK;
}

dtsdf_status dtsdf_server_stats(dtsdf_server s, dtsdf_server_stats_t* st) {
  if (!s || !st) return set_error(DTSDF_ERR_INVALID_ARG, "server: bad argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *st = s->st;
  st->pending = (int64_t)s->pending.size();
  return DTSDF_OK;
}

double dtsdf_server_clock(dtsdf_server s) { return s ? s->now() : 0.0; }

dtsdf_status dtsdf_server_destroy(dtsdf_server s) {
  if (!s) return set_error(DTSDF_ERR_INVALID_ARG, "server: null");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (Req* q : s->pending) delete q;
  for (int i = 0; i < s->p.streams; ++i) {
    if (s->running[i]) {
      cudaEventSynchronize(s->running[i]->done);
      s->events.push_back(s->running[i]->done);
      for (Req* q : s->running[i]->reqs) delete q;
      delete s->running[i];
    }
    if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
  }
  for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
  dt_free(s->arena_base);
  if (s->host_base) dt_free_host(s->host_base);
  delete s;
  return DTSDF_OK;
}

}  // extern "C"
