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
#include <string.h>

#include "internal.h"

namespace dtsdf {

// Eq. direction_weight as read; the clamped ranges (angle <= pi/2 - theta: 1, >= theta: 0)
// are decided on the cosine (cos_hi = sin theta, cos_lo = cos theta) without the arc cosine.
__device__ __forceinline__ float w_dir_c(float c, float theta, float cos_lo, float cos_hi) {
  if (c >= cos_hi) return 1.0f;
  if (c <= cos_lo) return 0.0f;
  const float alpha = acosf(c);
  return fminf(fmaxf((theta - alpha) / (2.0f * theta - 1.57079632679489662f), 0.0f), 1.0f);
}

template <int STORE>
__device__ __forceinline__ float2 src_geom(const MapView& m, size_t i) {
  if (STORE == DTSDF_STORE_FP16) return unpack_geom16(__ldg(m.geom16 + i));
  return __ldg(m.geom + i);
}

// Conditional combination (Sec. 4): recombine while fewer than 5 frames were rendered, after
// more than 50 frames without an update, or when the camera moved by more than 0.05 m or
// turned by more than 0.05 pi/2 since the last combination; otherwise only the blocks that
// received bricks since then are combined, at the last combination pose. Recycled bricks handed
// out again keep old pool indices, so a change of the recycled-brick count also recombines all.
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

// Register budget for 8 resident CTAs per SM (32 registers, a few spilled bytes): the pass is
// bound by the latency of its dependent reads, and more warps in flight beat fewer spills
// (forced whole-frustum pass on the 300-frame Kinect map: 1.00 ms at 5 CTAs per SM, 0.93 ms at
// 6, 0.86 ms at 8). The CTA walks its blocks with the bricks of the next block looked up (hash
// probes of its 7 neighbours) by 8 threads of its last warp while the others combine the
// current one.
constexpr int COMB_PREFETCH_T0 = 224;  // threads 224..231: 2 voxels each instead of 3

template <int STORE, bool COLOR>
__global__ void __launch_bounds__(256, 8) k_combine(MapView m, const CombState* st, CombFrame f) {
  __shared__ int s_src[2][ND][8];
  __shared__ float s_c[3];
  __shared__ float s_R[9];
  __shared__ uint32_t s_full, s_gen, s_from;
  if (threadIdx.x == 0) {
    s_full = st->full;
    s_gen = st->gen;
    s_from = st->pool_from;
    for (int a = 0; a < 3; ++a) {
      s_c[a] = (float)st->pose[4 * a + 3];
      for (int b = 0; b < 3; ++b) s_R[3 * a + b] = (float)st->pose[4 * a + b];
    }
  }
  __syncthreads();
  const uint32_t ndir = min(*((volatile uint32_t*)(m.counters + C_DIR)), m.dir_cap);
  const float h = m.h;
  const float cos_lo = m.costh, cos_hi = m.sinth;
  // the next block from d on (stride gridDim.x) that this pass combines (ndir if none); uniform
  auto next_taken = [&](uint32_t d) -> uint32_t {
    for (; d < ndir; d += gridDim.x) {
      const uint32_t mask = (uint32_t)m.dir_slots[(size_t)d * 8 + SLOT_MASK];
      bool take = mask != 0;
      if (take && !s_full) {  // incremental: blocks with a brick allocated since the last combination
        bool fresh = false;
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
  const int pj = (int)threadIdx.x - COMB_PREFETCH_T0;  // 0..7 on the prefetching threads
  uint32_t d = next_taken(blockIdx.x);
  if (d < ndir && pj >= 0 && pj < 8) comb_sources(m, d, pj, s_src[0]);
  __syncthreads();
  int cb = 0;
  while (d < ndir) {
    const uint32_t dn = next_taken(d + gridDim.x);
    if (dn < ndir && pj >= 0 && pj < 8) comb_sources(m, dn, pj, s_src[cb ^ 1]);
    const int bx = m.dir_coord[4 * d], by = m.dir_coord[4 * d + 1], bz = m.dir_coord[4 * d + 2];
    int (*src)[8] = s_src[cb];
    const float inv2h = 0.5f / h;
    for (int vi = threadIdx.x; vi < CVOX; vi += blockDim.x) {
      const int x = vi % CEDGE, y = (vi / CEDGE) % CEDGE, z = vi / (CEDGE * CEDGE);
      float r0 = m.ox + (float)(8 * bx + x) * h - s_c[0];
      float r1 = m.oy + (float)(8 * by + y) * h - s_c[1];
      float r2 = m.oz + (float)(8 * bz + z) * h - s_c[2];
      const float rinv = 1.0f / sqrtf(r0 * r0 + r1 * r1 + r2 * r2);
      r0 *= rinv;
      r1 *= rinv;
      r2 *= rinv;
      float ws = 0.f, acc = 0.f, wf = 0.f, af = 0.f, cw = 0.f, cr = 0.f, cg = 0.f, cb = 0.f;
      bool any = false;
#pragma unroll 1
      const int own = (x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2);
      for (int D = 0; D < ND; ++D) {
        const int sl = src[D][own];
        if (sl < 0) continue;
        const size_t base = (size_t)sl * PVOX + pad_index(x & 7, y & 7, z & 7);
        const float2 v0 = src_geom<STORE>(m, base);
        if (!(v0.y > 0.0f)) continue;
        any = true;
        const float vr = (D & 1) ? ((D >> 1) == 0 ? r0 : (D >> 1) == 1 ? r1 : r2)
                                 : -((D >> 1) == 0 ? r0 : (D >> 1) == 1 ? r1 : r2);
        const float w_f = v0.y * fmaxf(vr, 0.0f);
        if (w_f > 0.0f) {
          wf += w_f;
          af += w_f * v0.x;
        }
        const float2 xp = src_geom<STORE>(m, base + 1), xm = src_geom<STORE>(m, base - 1);
        const float2 yp = src_geom<STORE>(m, base + PAD), ym = src_geom<STORE>(m, base - PAD);
        const float2 zp = src_geom<STORE>(m, base + PAD * PAD), zm = src_geom<STORE>(m, base - PAD * PAD);
        if (!(xp.y > 0.f && xm.y > 0.f && yp.y > 0.f && ym.y > 0.f && zp.y > 0.f && zm.y > 0.f)) continue;
        const float g0 = (xp.x - xm.x) * inv2h, g1 = (yp.x - ym.x) * inv2h, g2 = (zp.x - zm.x) * inv2h;
        const float gn = sqrtf(g0 * g0 + g1 * g1 + g2 * g2);
        if (!(gn > 1e-12f)) continue;
        const float n0 = g0 / gn, n1 = g1 / gn, n2 = g2 / gn;
        const float facing = -(n0 * r0 + n1 * r1 + n2 * r2);
        if (!(facing > 0.0f)) continue;  // the weight of Eq. combine_weight vanishes
        const float cosv = (D == 0) ? n0 : (D == 1) ? -n0 : (D == 2) ? n1 : (D == 3) ? -n1 : (D == 4) ? n2 : -n2;
        const float wc = w_dir_c(cosv, m.theta, cos_lo, cos_hi) * facing * v0.y;
        if (!(wc > 0.0f)) continue;
        ws += wc;
        acc += wc * v0.x;
        if (COLOR) {
          {
            const size_t ci = (size_t)sl * BVOX + ((z & 7) * 8 + (y & 7)) * 8 + (x & 7);
            const float4 c = STORE == DTSDF_STORE_FP16 ? unpack_col8(__ldg(m.col8 + ci)) : __ldg(m.col + ci);
            if (c.w > 0.0f) {
              cw += wc;
              cr += wc * c.x;
              cg += wc * c.y;
              cb += wc * c.z;
            }
          }
        }
      }
      float2 out = make_float2(0.f, 0.f);
      uint2 oc = make_uint2(0u, 0u);
      if (any && ws > 0.0f) {
        out = make_float2(acc / ws, 1.0f);
        if (COLOR && cw > 0.0f) oc = pack_comb_col(cr / cw, cg / cw, cb / cw, true);
      } else if (any && wf > 0.0f) {
        out = make_float2(af / wf, 1.0f);
      }
      m.comb[(size_t)d * CVOX + vi] = out;
      if (COLOR) m.comb_col[(size_t)d * CVOX + vi] = oc;
    }
    if (threadIdx.x == 0) m.comb_gen[d] = s_gen;
    __syncthreads();  // the next block's sources are in place; this block's may be overwritten
    cb ^= 1;
    d = dn;
  }
}

void launch_combine(const MapView& m, CombState* st, const Intr& K, const double* Tdev, const double* Thost, int force,
                    int num_sms, cudaStream_t s) {
  Pose64 Tv;
  for (int i = 0; i < 16; ++i) Tv.T[i] = Thost ? Thost[i] : 0.0;
  k_comb_policy<<<1, 1, 0, s>>>(st, Tdev, Tv, m.counters, force);
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
  const bool col = m.color && m.comb_col;
  // one wave of resident CTAs walks the directory
  auto go = [&](auto kern) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess || per_sm < 1) per_sm = 4;
    kern<<<num_sms * per_sm, 256, 0, s>>>(m, st, f);
  };
  if (m.storage == DTSDF_STORE_FP16) {
    if (col) go(k_combine<DTSDF_STORE_FP16, true>);
    else go(k_combine<DTSDF_STORE_FP16, false>);
  } else {
    if (col) go(k_combine<DTSDF_STORE_FP32, true>);
    else go(k_combine<DTSDF_STORE_FP32, false>);
  }
}

}  // namespace dtsdf
