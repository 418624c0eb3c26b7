// View-dependent combined TSDF (Sec. 4) at integer voxel positions (Sec. 7), and the
// conditional combination that decides when to recompute it (Sec. 4, conditions 1-4).
//
// For the camera centre c of the combination pose, every voxel v of a block in the padded view
// frustum (the image grown by 1/8 of its size on each side) gets the combined value of
// Eq. combine_weight: each direction D with weight W^D(v) > 0 takes part; its gradient is the
// central difference of its 6 axis neighbours (all with weight > 0, norm > 1e-12; with the
// padded bricks every neighbour of a voxel in [0, 8]^3 is in the same brick); the view ray is
// r = (x_v - c) / |x_v - c|; w^D = w_dir(<n^D, v^D>) max(0, <n^D, -r>) W^D; when every w^D
// vanishes the weights W^D max(0, <v^D, -r>) of Eq. combine_tsdf_weight apply; otherwise the
// voxel is undefined. The colour combines the colours of the directions with a combination
// weight and a colour weight > 0. The result is then ray-cast like a regular TSDF (render.cu,
// STORE_COMBINED) from any pose near the combination pose.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>

#include "internal.h"

namespace dtsdf {

// Eq. direction_weight as read; the clamped ranges (angle <= pi/2 - theta: 1, >= theta: 0)
// are decided on the cosine (cos_hi = sin theta, cos_lo = cos theta) without the arc cosine;
// inv_span = 1 / (2 theta - pi/2).
__device__ __forceinline__ float w_dir_c(float c, float theta, float cos_lo, float cos_hi, float inv_span) {
  if (c >= cos_hi) return 1.0f;
  if (c <= cos_lo) return 0.0f;
  const float alpha = acosf(c);
  return fminf(fmaxf((theta - alpha) * inv_span, 0.0f), 1.0f);
}

// Conditional combination (Sec. 4): recombine while fewer than 5 frames were rendered, after
// more than 50 frames without an update, or when the camera moved by more than 0.05 m or
// turned by more than 0.05 pi/2 since the last combination; otherwise only the blocks that
// received bricks since then, and the blocks around them, are combined, at the last combination
// pose. Recycled bricks handed out again keep old pool indices, so a change of the recycled-brick
// count also recombines all.
__global__ void k_comb_policy(CombState* st, const double* Tdev, Pose64 Tv, const uint32_t* counters, int force) {
  double T[16];
  for (int i = 0; i < 16; ++i) T[i] = Tdev ? Tdev[i] : Tv.T[i];
  const uint32_t taken = counters[C_FREE_TAKEN];
  bool full = force || st->frames < 5 || st->since > 50 || taken != st->taken_mark;
  st->taken_mark = taken;
  const uint32_t* pool_count = counters + C_POOL;
  if (!full) {
    const double* L = st->pose;
    const double dx = T[3] - L[3], dy = T[7] - L[7], dz = T[11] - L[11];
    double tr = 0.0;  // trace(R_last^T R)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) tr += L[4 * b + a] * T[4 * b + a];
    const double ang = acos(fmin(fmax((tr - 1.0) / 2.0, -1.0), 1.0));
    full = sqrt(dx * dx + dy * dy + dz * dz) > 0.05 || ang > 0.05 * 1.57079632679489662;
  }
  st->frames += 1;
  st->pool_from = st->pool_mark;
  st->pool_mark = *pool_count;
  st->full = full ? 1u : 0u;
  if (full) {
    st->gen += 1;
    st->since = 0;
    for (int i = 0; i < 16; ++i) st->pose[i] = T[i];
  } else {
    st->since += 1;
  }
}

// Incremental combination: every block around a block that received bricks since the last call
// (pool indices [pool_from, pool_mark)) is marked for recombination, since its stored voxels next
// to that block - the layer the two share at local 8, and the gradient stencils that reach into it -
// depend on the new bricks. A full combination marks nothing.
__global__ void k_comb_mark(MapView m, const CombState* st) {
  if (st->full) return;
  const uint32_t from = st->pool_from, to = min(st->pool_mark, m.pool_cap);
  for (uint32_t p = from + blockIdx.x * blockDim.x + threadIdx.x; p < to; p += gridDim.x * blockDim.x) {
    const int bd = m.brick_dir[p];
    if (bd < 0) continue;
    const int d = bd >> 3;
    const int bx = m.dir_coord[4 * d], by = m.dir_coord[4 * d + 1], bz = m.dir_coord[4 * d + 2];
#pragma unroll 1
    for (int q = 0; q < 27; ++q) {
      if (q == 13) continue;
      const int dd = hash_find(m, bx + q % 3 - 1, by + (q / 3) % 3 - 1, bz + q / 9 - 1);
      if (dd >= 0) m.comb_dirty[dd] = 1;
    }
  }
}

// Bricks of the blocks {0, 1}^3 from block d for the 6 directions (src[D][j], -1: none): voxel
// (x, y, z) of [0, 8]^3 belongs to block (x >> 3, y >> 3, z >> 3) and is combined from that
// block's directions (a voxel's data is its own block's). One thread per neighbour j.
__device__ __forceinline__ void comb_sources(const MapView& m, uint32_t d, int j, int (*src)[8]) {
  const int bx = m.dir_coord[4 * d], by = m.dir_coord[4 * d + 1], bz = m.dir_coord[4 * d + 2];
  const int dd = j == 0 ? (int)d : hash_find(m, bx + (j & 1), by + ((j >> 1) & 1), bz + (j >> 2));
  const uint32_t mask = dd >= 0 ? (uint32_t)m.dir_slots[(size_t)dd * 8 + SLOT_MASK] : 0u;
#pragma unroll
  for (int D = 0; D < ND; ++D) src[D][j] = ((mask >> D) & 1u) ? m.dir_slots[(size_t)dd * 8 + D] : -1;
}

// ---- the block cache (Sec. 7: a block's bricks are held in shared memory while it is combined).
// A stage is one (block, direction): the block's padded geometry brick of that direction and its
// colour brick, fetched by two bulk copies (cp.async.bulk) that complete on the stage's "full"
// mbarrier. One producer warp walks the blocks, looks up each block's upper neighbours and issues
// the copies into a ring of COMB_NS stage buffers; the consumer warps combine the stages in order
// and free each buffer on its "empty" mbarrier. No CTA-wide barrier couples the two sides, so the
// producer's hash probes and the copies of the next stages overlap the combination.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// orders the CTA's earlier generic-proxy accesses of shared memory before later bulk copies into it
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared bulk copy: both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Waits for the completion of the barrier's phase of the given parity (the current phase or the
// one before it); gives up after 2^31 clock cycles (about a second) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}

// Element types of the source bricks per storage form, and the size of one stage buffer.
template <int STORE>
struct CombSrc {
  using G = float2;  // (sdf, weight)
  using C = float4;  // (r, g, b, colour weight)
};
template <>
struct CombSrc<DTSDF_STORE_FP16> {
  using G = uint32_t;  // half sdf | half-coded weight
  using C = uint32_t;  // u8 r, g, b | log colour-weight code
};
template <int STORE, bool COLOR>
struct CombLayout {
  static constexpr uint32_t GBYTES = (uint32_t)sizeof(typename CombSrc<STORE>::G) * PVOX;
  // a padded brick copied from the 16-byte boundary at or below it: at most GBYTES + 15 bytes,
  // rounded up to 16
  static constexpr uint32_t GBUF = (GBYTES + 30) / 16 * 16;
  static constexpr uint32_t CBUF = COLOR ? (uint32_t)sizeof(typename CombSrc<STORE>::C) * BVOX : 0u;
  static constexpr uint32_t STAGE = GBUF + CBUF;
};
__device__ __forceinline__ float2 geom_val(float2 v) { return v; }
__device__ __forceinline__ float2 geom_val(uint32_t v) { return unpack_geom16(v); }
__device__ __forceinline__ float4 col_val(float4 v) { return v; }
__device__ __forceinline__ float4 col_val(uint32_t v) { return unpack_col8(v); }

// Running sums of one voxel's combination.
struct CombAcc {
  float ws, acc;  // sum of w^D, sum of w^D phi^D (Eq. combine_weight)
  float wf, af;   // fallback weights of Eq. combine_tsdf_weight and their weighted sum
  float cw, cr, cg, cb;
  bool any;       // some direction has weight at the voxel
};

// Contribution of direction D at one voxel: v(o) is the (sdf, weight) at offset o (in padded-brick
// elements) from the voxel, col() its colour; r is the unit view ray to the voxel.
template <bool COLOR, typename GF, typename CF>
__device__ __forceinline__ void comb_dir(CombAcc& a, int D, const GF& v, const CF& col, float r0, float r1, float r2,
                                         float inv2h, float theta, float cos_lo, float cos_hi, float inv_span) {
  const float2 v0 = v(0);
  if (!(v0.y > 0.0f)) return;
  a.any = true;
  const float vr = (D & 1) ? ((D >> 1) == 0 ? r0 : (D >> 1) == 1 ? r1 : r2)
                           : -((D >> 1) == 0 ? r0 : (D >> 1) == 1 ? r1 : r2);
  const float w_f = v0.y * fmaxf(vr, 0.0f);
  if (w_f > 0.0f) {
    a.wf += w_f;
    a.af += w_f * v0.x;
  }
  const float2 xp = v(1), xm = v(-1), yp = v(PAD), ym = v(-PAD), zp = v(PAD * PAD), zm = v(-PAD * PAD);
  if (!(xp.y > 0.f && xm.y > 0.f && yp.y > 0.f && ym.y > 0.f && zp.y > 0.f && zm.y > 0.f)) return;
  const float g0 = (xp.x - xm.x) * inv2h, g1 = (yp.x - ym.x) * inv2h, g2 = (zp.x - zm.x) * inv2h;
  const float gg = g0 * g0 + g1 * g1 + g2 * g2;
  if (!(gg > 1e-24f)) return;  // |g| > 1e-12
  const float ig = rsqrtf(gg);
  const float n0 = g0 * ig, n1 = g1 * ig, n2 = g2 * ig;
  const float facing = -(n0 * r0 + n1 * r1 + n2 * r2);
  if (!(facing > 0.0f)) return;  // the weight of Eq. combine_weight vanishes
  const float cosv = (D == 0) ? n0 : (D == 1) ? -n0 : (D == 2) ? n1 : (D == 3) ? -n1 : (D == 4) ? n2 : -n2;
  const float wc = w_dir_c(cosv, theta, cos_lo, cos_hi, inv_span) * facing * v0.y;
  if (!(wc > 0.0f)) return;
  a.ws += wc;
  a.acc += wc * v0.x;
  if (COLOR) {
    const float4 c = col();
    if (c.w > 0.0f) {
      a.cw += wc;
      a.cr += wc * c.x;
      a.cg += wc * c.y;
      a.cb += wc * c.z;
    }
  }
}

// A stage as the producer hands it to the consumers.
struct CombStageDesc {
  int d;       // directory index of the block
  int D;       // direction, -1: none (a block without stages, whose voxels are all undefined)
  int slot;    // the block's brick of D, staged in the buffer; -1: only upper neighbours have D
  int flags;   // COMB_FIRST | COMB_LAST | COMB_END
  int bc[3];   // block coordinates
  int src[8];  // brick of D of the blocks {0, 1}^3 from this one (j = x | y << 1 | z << 2), -1: none
};
enum { COMB_FIRST = 1, COMB_LAST = 2, COMB_END = 4 };

// One CTA combines one block at a time, the resident CTAs walking the directory. A block's stages
// are its directions D = 0..5 that it has (staged: every voxel of [0, 8]^3 whose own block has D
// reads its 7 stencil values from the staged padded brick, whose apron mirrors the upper
// neighbours' voxels at local 8 and 9; the colour of a voxel of [0, 7]^3 from the staged colour
// brick, of the upper layer from its own block's colour brick), and the directions only upper
// neighbours have (combined at the upper layer's voxels from those blocks' bricks in global
// memory). Every voxel sums its directions in the order D = 0..5.
// Launch shape (paired A/B on the forced whole-frustum pass of the 300-frame Kinect map): 23
// consumer warps, one voxel of [0, 8]^3 per thread, 2 CTAs per SM at 40 registers and a ring of 5
// stages (94 KB) ran at 0.65 ms; 8 consumer warps (3 voxels per thread) at 3 CTAs 0.85 ms, 12 at 3
// CTAs 0.81 ms, 31 warps with a ring of 8 at 1 CTA 0.82 ms; rings of 3 / 4 stages 0.71 / 0.67 ms.
#ifndef DTSDF_COMB_CWARPS
#define DTSDF_COMB_CWARPS 23
#endif
constexpr int COMB_CWARPS = DTSDF_COMB_CWARPS;       // consumer warps
constexpr int COMB_CT = 32 * COMB_CWARPS;            // consumer threads
constexpr int COMB_T = COMB_CT + 32;                 // + the producer warp
constexpr int COMB_VPT = (CVOX + COMB_CT - 1) / COMB_CT;  // voxels per consumer thread
#ifndef DTSDF_COMB_STAGES
#define DTSDF_COMB_STAGES 5  // stage buffers in the ring
#endif
#ifndef DTSDF_COMB_MINB
#define DTSDF_COMB_MINB 2    // resident CTAs per SM the register allocation is sized for
#endif
constexpr int COMB_NS = DTSDF_COMB_STAGES;

template <int STORE, bool COLOR>
__global__ void __launch_bounds__(COMB_T, DTSDF_COMB_MINB) k_combine(MapView m, const CombState* st, CombFrame f) {
  using G = typename CombSrc<STORE>::G;
  using C = typename CombSrc<STORE>::C;
  using L = CombLayout<STORE, COLOR>;
  extern __shared__ __align__(128) unsigned char s_buf[];  // COMB_NS x L::STAGE bytes
  __shared__ __align__(8) uint64_t s_fullbar[COMB_NS], s_emptybar[COMB_NS];
  __shared__ CombStageDesc s_desc[COMB_NS];
  __shared__ float s_c[3];
  __shared__ float s_R[9];
  __shared__ uint32_t s_full, s_gen, s_from;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    s_full = st->full;
    s_gen = st->gen;
    s_from = st->pool_from;
    for (int a = 0; a < 3; ++a) {
      s_c[a] = (float)st->pose[4 * a + 3];
      for (int b = 0; b < 3; ++b) s_R[3 * a + b] = (float)st->pose[4 * a + b];
    }
    for (int q = 0; q < COMB_NS; ++q) {
      mbar_init(&s_fullbar[q], 1);
      mbar_init(&s_emptybar[q], COMB_CWARPS);
    }
    mbar_init_fence();
  }
  __syncthreads();  // the last CTA-wide barrier: from here on the two sides meet on mbarriers only
  const G* gpool = reinterpret_cast<const G*>(STORE == DTSDF_STORE_FP16 ? (const void*)m.geom16 : (const void*)m.geom);
  const C* cpool = reinterpret_cast<const C*>(STORE == DTSDF_STORE_FP16 ? (const void*)m.col8 : (const void*)m.col);
  const uint32_t ndir = min(*((volatile uint32_t*)(m.counters + C_DIR)), m.dir_cap);
  const float h = m.h;

  if (warp == COMB_CWARPS) {
    // ------------------------------------------------------------------ producer warp
    if (f.stall) return;  // test hook: no stage is issued
    // the next block from d on (stride gridDim.x) that this pass combines (ndir if none)
    auto next_taken = [&](uint32_t d) -> uint32_t {
      for (; d < ndir; d += gridDim.x) {
        const uint32_t mask = (uint32_t)m.dir_slots[(size_t)d * 8 + SLOT_MASK];
        bool take = mask != 0;
        if (take && !s_full) {
          // incremental: blocks with a brick allocated since the last combination, and the blocks
          // around them (marked by k_comb_mark)
          bool fresh = m.comb_dirty[d] != 0;
          for (uint32_t mm = mask; mm; mm &= mm - 1)
            fresh |= (uint32_t)m.dir_slots[(size_t)d * 8 + __ffs(mm) - 1] >= s_from;
          take = fresh;
        }
        if (!take) continue;
        // padded frustum of the combination pose: bounding sphere of the block against the four
        // side planes (image grown by 1/8) and the camera's half-space
        const int bx = m.dir_coord[4 * d], by = m.dir_coord[4 * d + 1], bz = m.dir_coord[4 * d + 2];
        const float rad = 0.8660254f * 8.0f * h + h;
        const float p0 = m.ox + (8.0f * bx + 3.5f) * h - s_c[0];
        const float p1 = m.oy + (8.0f * by + 3.5f) * h - s_c[1];
        const float p2 = m.oz + (8.0f * bz + 3.5f) * h - s_c[2];
        const float cx = s_R[0] * p0 + s_R[3] * p1 + s_R[6] * p2;
        const float cy = s_R[1] * p0 + s_R[4] * p1 + s_R[7] * p2;
        const float cz = s_R[2] * p0 + s_R[5] * p1 + s_R[8] * p2;
        take = cz > -rad;
#pragma unroll
        for (int q = 0; q < 4; ++q) take &= (f.pl[q][0] * cx + f.pl[q][1] * cy + f.pl[q][2] * cz) >= -rad;
        if (take) return d;
      }
      return ndir;
    };
    int q = 0;
    uint32_t pe = (1u << COMB_NS) - 1u;  // parity to wait for per empty barrier: a fresh ring is free
    uint32_t issued = 0u, pfull = 0u;    // slots that received copies; parity of each slot's last use
    bool fail = false;
    uint32_t d = next_taken(blockIdx.x);
    for (;;) {
      const bool end = d >= ndir;
      int bc[3] = {0, 0, 0};
      int bsl[ND];  // lanes 0..7: bricks of block j = lane of {0, 1}^3 from this one
#pragma unroll
      for (int D = 0; D < ND; ++D) bsl[D] = -1;
      uint32_t stages;
      if (!end) {
        bc[0] = m.dir_coord[4 * d];
        bc[1] = m.dir_coord[4 * d + 1];
        bc[2] = m.dir_coord[4 * d + 2];
        if (lane < 8) {
          const int dd = lane == 0 ? (int)d : hash_find(m, bc[0] + (lane & 1), bc[1] + ((lane >> 1) & 1), bc[2] + (lane >> 2));
          const uint32_t mask = dd >= 0 ? (uint32_t)m.dir_slots[(size_t)dd * 8 + SLOT_MASK] : 0u;
#pragma unroll
          for (int D = 0; D < ND; ++D) bsl[D] = ((mask >> D) & 1u) ? m.dir_slots[(size_t)dd * 8 + D] : -1;
        }
        stages = 0u;
#pragma unroll
        for (int D = 0; D < ND; ++D) {
          const bool own = __shfl_sync(0xffffffffu, bsl[D], 0) >= 0;
          const bool up = __ballot_sync(0xffffffffu, lane >= 1 && lane < 8 && bsl[D] >= 0) != 0u;
          if (own || up) stages |= 1u << D;
        }
        if (!stages) stages = 1u << ND;  // no stage: one empty stage writes the block's undefined voxels
      } else {
        stages = 1u << 7;  // the end marker
      }
      bool first = true;
      while (stages) {
        const int bit = __ffs(stages) - 1;
        stages &= stages - 1;
        bool ok = true;
        if (lane == 0) ok = mbar_wait_bounded(&s_emptybar[q], (pe >> q) & 1u);
        if (!__shfl_sync(0xffffffffu, (int)ok, 0)) {
          fail = true;
          break;
        }
        pe ^= 1u << q;
        const int D = bit < ND ? bit : -1;
        int mine = -1;
#pragma unroll
        for (int E = 0; E < ND; ++E)
          if (E == D) mine = bsl[E];
        int src[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) src[j] = __shfl_sync(0xffffffffu, mine, j);
        if (lane == 0) {
          CombStageDesc& sd = s_desc[q];
          const int slot = D >= 0 ? src[0] : -1;
          sd.d = (int)d;
          sd.D = D;
          sd.slot = slot;
          sd.flags = (first ? COMB_FIRST : 0) | (stages == 0u ? COMB_LAST : 0) | (end ? COMB_END : 0);
          sd.bc[0] = bc[0];
          sd.bc[1] = bc[1];
          sd.bc[2] = bc[2];
#pragma unroll
          for (int j = 0; j < 8; ++j) sd.src[j] = src[j];
          if (slot >= 0) {
            const uintptr_t a = reinterpret_cast<uintptr_t>(gpool + (size_t)slot * PVOX);
            const uintptr_t a16 = a & ~(uintptr_t)15;
            const uint32_t gb = (uint32_t)((a - a16 + L::GBYTES + 15) & ~(uintptr_t)15);
            unsigned char* buf = s_buf + (size_t)q * L::STAGE;
            fence_proxy_async_smem();
            mbar_arrive_expect(&s_fullbar[q], gb + L::CBUF);
            bulk_g2s(buf, (const void*)a16, gb, &s_fullbar[q]);
            if (COLOR) bulk_g2s(buf + L::GBUF, cpool + (size_t)slot * BVOX, L::CBUF, &s_fullbar[q]);
          } else {
            mbar_arrive(&s_fullbar[q]);
          }
        }
        __syncwarp();
        issued |= 1u << q;
        pfull ^= 1u << q;
        first = false;
        q = q + 1 == COMB_NS ? 0 : q + 1;
      }
      if (end || fail) break;
      d = next_taken(d + gridDim.x);
    }
    if (fail) {
      // the consumers stopped: flag it and let this warp's copies in flight land before leaving
      if (lane == 0) {
        atomicOr(m.counters + C_ERR, ERR_TIMEOUT);
        for (int s = 0; s < COMB_NS; ++s)
          if ((issued >> s) & 1u) mbar_wait_bounded(&s_fullbar[s], ((pfull >> s) & 1u) ^ 1u);
      }
    }
    return;
  }

  // -------------------------------------------------------------------- consumer warps
  const float inv2h = 0.5f / h;
  const float theta = m.theta, cos_lo = m.costh, cos_hi = m.sinth;
  const float inv_span = 1.0f / (2.0f * theta - 1.57079632679489662f);
  // this thread's voxels of [0, 8]^3: vi = tid + i COMB_CT, packed as x | y << 4 | z << 8 (-1 if
  // none), and their stage indices: padded-brick index p | owner block j << 11 | index ci of the
  // voxel in its owner's brick << 14
  int vx[COMB_VPT], vp[COMB_VPT];
#pragma unroll
  for (int i = 0; i < COMB_VPT; ++i) {
    const int vi = tid + i * COMB_CT;
    const int x = vi % CEDGE, y = (vi / CEDGE) % CEDGE, z = vi / (CEDGE * CEDGE);
    vx[i] = vi < CVOX ? x | (y << 4) | (z << 8) : -1;
    vp[i] = pad_index(x, y, z) | (((x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2)) << 11) |
            ((((z & 7) * 8 + (y & 7)) * 8 + (x & 7)) << 14);
  }
  CombAcc A[COMB_VPT];
  float ray[COMB_VPT][3];
  int q = 0;
  uint32_t pf = 0u;  // parity to wait for per full barrier
  for (;;) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&s_fullbar[q], (pf >> q) & 1u));
    if (!ok) {
      if (lane == 0) atomicOr(m.counters + C_ERR, ERR_TIMEOUT);
      return;
    }
    pf ^= 1u << q;
    const CombStageDesc& sd = s_desc[q];
    const int flags = sd.flags;
    if (flags & COMB_END) break;
    const int d = sd.d, D = sd.D, slot = sd.slot;
    if (flags & COMB_FIRST) {
      const int bx = sd.bc[0], by = sd.bc[1], bz = sd.bc[2];
#pragma unroll
      for (int i = 0; i < COMB_VPT; ++i) {
        A[i].ws = A[i].acc = A[i].wf = A[i].af = A[i].cw = A[i].cr = A[i].cg = A[i].cb = 0.f;
        A[i].any = false;
        const int x = vx[i] & 15, y = (vx[i] >> 4) & 15, z = (vx[i] >> 8) & 15;
        float r0 = m.ox + (float)(8 * bx + x) * h - s_c[0];
        float r1 = m.oy + (float)(8 * by + y) * h - s_c[1];
        float r2 = m.oz + (float)(8 * bz + z) * h - s_c[2];
        const float rinv = 1.0f / sqrtf(r0 * r0 + r1 * r1 + r2 * r2);
        ray[i][0] = r0 * rinv;
        ray[i][1] = r1 * rinv;
        ray[i][2] = r2 * rinv;
      }
    }
    if (D >= 0 && slot >= 0) {
      const uint32_t off = (uint32_t)((reinterpret_cast<uintptr_t>(gpool + (size_t)slot * PVOX) & 15) / sizeof(G));
      const unsigned char* buf = s_buf + (size_t)q * L::STAGE;
      const G* sg = reinterpret_cast<const G*>(buf) + off;
      const C* sc = reinterpret_cast<const C*>(buf + L::GBUF);
#pragma unroll
      for (int i = 0; i < COMB_VPT; ++i) {
        if (vx[i] < 0) continue;
        const int p = vp[i] & 2047, j = (vp[i] >> 11) & 7, ci = vp[i] >> 14;
        const int osl = sd.src[j];  // the brick of D of the voxel's own block
        if (osl < 0) continue;
        comb_dir<COLOR>(
            A[i], D, [&](int o) { return geom_val(sg[p + o]); },
            [&]() { return col_val(j == 0 ? sc[ci] : __ldg(cpool + (size_t)osl * BVOX + ci)); }, ray[i][0],
            ray[i][1], ray[i][2], inv2h, theta, cos_lo, cos_hi, inv_span);
      }
    } else if (D >= 0) {
      // only upper neighbours have D: their voxels on this block's upper layer, from their bricks
#pragma unroll
      for (int i = 0; i < COMB_VPT; ++i) {
        if (vx[i] < 0) continue;
        const int x = vx[i] & 15, y = (vx[i] >> 4) & 15, z = (vx[i] >> 8) & 15;
        const int j = (x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2);
        const int osl = j ? sd.src[j] : -1;
        if (osl < 0) continue;
        const G* gb = gpool + (size_t)osl * PVOX + pad_index(x & 7, y & 7, z & 7);
        const int ci = ((z & 7) * 8 + (y & 7)) * 8 + (x & 7);
        comb_dir<COLOR>(
            A[i], D, [&](int o) { return geom_val(__ldg(gb + o)); },
            [&]() { return col_val(__ldg(cpool + (size_t)osl * BVOX + ci)); }, ray[i][0], ray[i][1], ray[i][2], inv2h,
            theta, cos_lo, cos_hi, inv_span);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&s_emptybar[q]);  // this warp is done with the buffer and the descriptor
    q = q + 1 == COMB_NS ? 0 : q + 1;
    if (flags & COMB_LAST) {
#pragma unroll
      for (int i = 0; i < COMB_VPT; ++i) {
        if (vx[i] < 0) continue;
        const int vi = tid + i * COMB_CT;
        float2 out = make_float2(0.f, 0.f);
        uint2 oc = make_uint2(0u, 0u);
        if (A[i].any && A[i].ws > 0.0f) {
          out = make_float2(A[i].acc / A[i].ws, 1.0f);
          if (COLOR && A[i].cw > 0.0f)
            oc = pack_comb_col(A[i].cr / A[i].cw, A[i].cg / A[i].cw, A[i].cb / A[i].cw, true);
        } else if (A[i].any && A[i].wf > 0.0f) {
          out = make_float2(A[i].af / A[i].wf, 1.0f);
        }
        m.comb[(size_t)d * CVOX + vi] = out;
        if (COLOR) m.comb_col[(size_t)d * CVOX + vi] = oc;
      }
      if (tid == 0) {
        m.comb_gen[d] = s_gen;
        m.comb_dirty[d] = 0;
      }
    }
  }
}

template <int STORE, bool COLOR>
void launch_k_combine(const MapView& m, CombState* st, const CombFrame& f, int num_sms, cudaStream_t s) {
  auto kern = k_combine<STORE, COLOR>;
  constexpr size_t smem = (size_t)COMB_NS * CombLayout<STORE, COLOR>::STAGE;
  // the ring exceeds the default 48 KB of dynamic shared memory: raise the limit once per device
  // (callers on several host threads may race here; setting the attribute twice is harmless)
  static std::atomic<uint64_t> opted{0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64 || !((opted.load(std::memory_order_relaxed) >> dev) & 1u)) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess && dev < 64)
      opted.fetch_or(1ull << dev, std::memory_order_relaxed);
  }
  // one wave of resident CTAs walks the directory
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, COMB_T, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  kern<<<num_sms * per_sm, COMB_T, smem, s>>>(m, st, f);
}

void launch_combine(const MapView& m, CombState* st, const Intr& K, const double* Tdev, const double* Thost, int force,
                    int num_sms, cudaStream_t s) {
  Pose64 Tv;
  for (int i = 0; i < 16; ++i) Tv.T[i] = Thost ? Thost[i] : 0.0;
  k_comb_policy<<<1, 1, 0, s>>>(st, Tdev, Tv, m.counters, force);
  k_comb_mark<<<num_sms * 2, 256, 0, s>>>(m, st);
  CombFrame f;
  // inward unit normals of the four side planes of the image grown by 1/8 of its size
  const float pu = 0.125f * (float)K.W, pv = 0.125f * (float)K.H;
  auto set = [&](int q, float a, float b, float c) {
    const float l = sqrtf(a * a + b * b + c * c);
    f.pl[q][0] = a / l;
    f.pl[q][1] = b / l;
    f.pl[q][2] = c / l;
  };
  set(0, K.fx, 0.f, K.cx + 0.5f + pu);
  set(1, -K.fx, 0.f, (float)K.W - 0.5f + pu - K.cx);
  set(2, 0.f, K.fy, K.cy + 0.5f + pv);
  set(3, 0.f, -K.fy, (float)K.H - 0.5f + pv - K.cy);
  const char* stall = getenv("DTSDF_TEST_COMBINE_STALL");
  f.stall = stall && *stall && atoi(stall) != 0;
  const bool col = m.color && m.comb_col;
  if (m.storage == DTSDF_STORE_FP16) {
    if (col) launch_k_combine<DTSDF_STORE_FP16, true>(m, st, f, num_sms, s);
    else launch_k_combine<DTSDF_STORE_FP16, false>(m, st, f, num_sms, s);
  } else {
    if (col) launch_k_combine<DTSDF_STORE_FP32, true>(m, st, f, num_sms, s);
    else launch_k_combine<DTSDF_STORE_FP32, false>(m, st, f, num_sms, s);
  }
}

}  // namespace dtsdf
