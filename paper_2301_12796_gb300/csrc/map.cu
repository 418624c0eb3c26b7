// Map construction: frame preprocessing (Sec. 7), voxel-block allocation in the
// (block, direction) hash (Sec. 7), and voxel-projection fusion of depth and colour
// with free-space carving (Sec. 3).
//
// HBM layout of a map (all allocated once at creation, sized by max_blocks):
//   keys/vals   open-addressing hash, block coordinate (21 bits per axis) -> directory index
//   dir_slots   8 int32 per block coordinate: brick index of each of the 6 directions
//               (-1 absent) and the bitmask of allocated directions; one probe of the
//               hash yields all six directions, which is what the ray marcher needs
//   geom        one padded brick per (block, direction): float2 (sdf, weight), x fastest, the
//               8^3 voxels of the block plus an apron (local coordinates -1, 8, 9) that
//               mirrors the neighbouring blocks and is refreshed after every fusion
//   col         matching unpadded float4 (r, g, b, colour weight) 8^3 bricks when colour is enabled
//   bound       per brick: minimum sdf of the weighted voxels at local coordinates [0, 8]^3
//               (the trilinear corners of every sample whose base voxel is in the block)
// The voxel (i, j, k) of block b sits at origin + (8 b + (i, j, k)) h.
#include <math.h>
#include <string.h>

#include "internal.h"
#include "dsfloat.cuh"

namespace dtsdf {

// ------------------------------------------------------------ preprocessing
// Depth outlier filter: a depth in [z_min, z_max] survives if at least two of its eight
// neighbours are in range and within delta_sup of it. Survivors are back-projected with
// Eq. reprojection: P = (z (u - cx)/fx, z (v - cy)/fy, z). P.w = 1 marks a survivor. The
// back-projection runs in double-single arithmetic (u - cx exact, then times 1/fx and z, about
// 48 bits) and is rounded once. ifx, ify: 1/fx, 1/fy split into two floats.
__global__ void k_filter(const float* __restrict__ depth, Intr K, float zmin, float zmax, float dsup, dsf ifx,
                         dsf ify, float4* __restrict__ P) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= K.W || v >= K.H) return;
  const int i = v * K.W + u;
  const float z = depth[i];
  float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
  if (depth_in_range(z, zmin, zmax)) {
    int support = 0;
    for (int dv = -1; dv <= 1; ++dv)
      for (int du = -1; du <= 1; ++du) {
        if (!du && !dv) continue;
        const int uu = u + du, vv = v + dv;
        if (uu < 0 || vv < 0 || uu >= K.W || vv >= K.H) continue;
        const float zn = depth[vv * K.W + uu];
        if (!depth_in_range(zn, zmin, zmax)) continue;
        if (fabsf(rsub(zn, z)) <= dsup) ++support;
      }
    if (support >= 2) {
      const dsf x = ds_mul_f(ds_mul(ds_two_sum((float)u, -K.cx), ifx), z);
      const dsf y = ds_mul_f(ds_mul(ds_two_sum((float)v, -K.cy), ify), z);
      out = make_float4(ds_to_float(x), ds_to_float(y), z, 1.0f);
    }
  }
  P[i] = out;
}

// Normals: cross product of the central differences of the back-projected x and y
// neighbours (Sec. 7), normalised and turned toward the camera. N.w = 1 marks a normal. The
// cross product of nearby points cancels most of their digits (at grazing incidence a single-
// precision normal is off by up to ~5e-4 rad), so the points are re-formed from the exact input
// depths and the normal computed in double-single arithmetic (about 48 bits), then rounded once;
// it feeds the direction membership and the band tests of allocation and fusion. The
// orientation is decided on the unnormalised double-single normal: n . P has the sign of
// n . (a, b, 1) since z > 0. ifx, ify: 1/fx, 1/fy split into two floats.
__global__ void k_normals(const float4* __restrict__ P, Intr K, dsf ifx, dsf ify, float4* __restrict__ N) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= K.W || v >= K.H) return;
  const int i = v * K.W + u;
  float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
  if (u >= 1 && v >= 1 && u < K.W - 1 && v < K.H - 1) {
    const float4 c = P[i], l = P[i - 1], r = P[i + 1], t = P[i - K.W], b = P[i + K.W];
    if (c.w > 0 && l.w > 0 && r.w > 0 && t.w > 0 && b.w > 0) {
      // ray slopes (u - cx)/fx and (v - cy)/fy of the centre and its four neighbours
      const dsf am = ds_mul(ds_two_sum((float)(u - 1), -K.cx), ifx);
      const dsf a0 = ds_mul(ds_two_sum((float)u, -K.cx), ifx);
      const dsf ap = ds_mul(ds_two_sum((float)(u + 1), -K.cx), ifx);
      const dsf bm = ds_mul(ds_two_sum((float)(v - 1), -K.cy), ify);
      const dsf b0 = ds_mul(ds_two_sum((float)v, -K.cy), ify);
      const dsf bp = ds_mul(ds_two_sum((float)(v + 1), -K.cy), ify);
      // central differences P(u+1) - P(u-1) and P(v+1) - P(v-1)
      const dsf dx2 = ds_two_sum(r.z, -l.z), dy2 = ds_two_sum(b.z, -t.z);
      const dsf dx0 = ds_sub(ds_mul_f(ap, r.z), ds_mul_f(am, l.z)), dx1 = ds_mul(dx2, b0);
      const dsf dy0 = ds_mul(dy2, a0), dy1 = ds_sub(ds_mul_f(bp, b.z), ds_mul_f(bm, t.z));
      dsf n0 = ds_sub(ds_mul(dx1, dy2), ds_mul(dx2, dy1));
      dsf n1 = ds_sub(ds_mul(dx2, dy0), ds_mul(dx0, dy2));
      dsf n2 = ds_sub(ds_mul(dx0, dy1), ds_mul(dx1, dy0));
      const dsf len = ds_sqrt(ds_add(ds_add(ds_mul(n0, n0), ds_mul(n1, n1)), ds_mul(n2, n2)));
      if (len.hi > 0.0f) {
        const dsf il = ds_recip(len);
        const dsf facing = ds_add(ds_add(ds_mul(n0, a0), ds_mul(n1, b0)), n2);
        const float sg = facing.hi > 0.0f ? -1.0f : 1.0f;
        out = make_float4(sg * ds_to_float(ds_mul(n0, il)), sg * ds_to_float(ds_mul(n1, il)),
                          sg * ds_to_float(ds_mul(n2, il)), 1.0f);
      }
    }
  }
  N[i] = out;
}

// Bilateral depth filter (Sec. 8 settings): for a survivor of the outlier filter, the mean of the
// survivors in the (2r+1)^2 window weighted by exp(-(du^2 + dv^2) / (2 sd^2)) in pixels times
// exp(-(z_j - z_i)^2 / (2 sr^2)) in depth; the result is back-projected again. Non-survivors
// stay empty. Fixed tap order (dv, then du), FP32.
__global__ void k_bilateral_depth(const float4* __restrict__ Pin, Intr K, int r, float sd, float sr,
                                  float4* __restrict__ Pout) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= K.W || v >= K.H) return;
  const int i = v * K.W + u;
  const float4 c = Pin[i];
  float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
  if (c.w > 0.f) {
    const float ks = -0.5f / (sd * sd), kr = -0.5f / (sr * sr);
    float num = 0.f, den = 0.f;
    for (int dv = -r; dv <= r; ++dv) {
      const int vv = v + dv;
      if (vv < 0 || vv >= K.H) continue;
      for (int du = -r; du <= r; ++du) {
        const int uu = u + du;
        if (uu < 0 || uu >= K.W) continue;
        const float4 q = Pin[vv * K.W + uu];
        if (!(q.w > 0.f)) continue;
        const float dz = q.z - c.z;
        const float w = expf(ks * (float)(du * du + dv * dv) + kr * dz * dz);
        num += w * q.z;
        den += w;
      }
    }
    const float z = num / den;  // den >= 1 (the centre tap)
    const float a = rdiv(rsub((float)u, K.cx), K.fx);
    const float b = rdiv(rsub((float)v, K.cy), K.fy);
    out = make_float4(rmul(z, a), rmul(z, b), z, 1.0f);
  }
  Pout[i] = out;
}

// Bilateral normal filter (Sec. 8 settings): for a pixel with a normal, the normalised sum of the
// normals in the (2r+1)^2 window weighted by exp(-(du^2 + dv^2) / (2 sd^2)) in pixels times
// exp(-a^2 / (2 sr^2)), a the angle between the two normals in degrees. Fixed tap order, FP32.
__global__ void k_bilateral_normals(const float4* __restrict__ Nin, Intr K, int r, float sd, float sr_deg,
                                    float4* __restrict__ Nout) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= K.W || v >= K.H) return;
  const int i = v * K.W + u;
  const float4 c = Nin[i];
  float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
  if (c.w > 0.f) {
    const float ks = -0.5f / (sd * sd), kr = -0.5f / (sr_deg * sr_deg);
    const float deg = 57.29577951308232f;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int dv = -r; dv <= r; ++dv) {
      const int vv = v + dv;
      if (vv < 0 || vv >= K.H) continue;
      for (int du = -r; du <= r; ++du) {
        const int uu = u + du;
        if (uu < 0 || uu >= K.W) continue;
        const float4 q = Nin[vv * K.W + uu];
        if (!(q.w > 0.f)) continue;
        const float d = fminf(1.f, fmaxf(-1.f, c.x * q.x + c.y * q.y + c.z * q.z));
        const float a = acosf(d) * deg;
        const float w = expf(ks * (float)(du * du + dv * dv) + kr * a * a);
        s0 += w * q.x;
        s1 += w * q.y;
        s2 += w * q.z;
      }
    }
    const float len = sqrtf(s0 * s0 + s1 * s1 + s2 * s2);
    if (len > 0.f) out = make_float4(s0 / len, s1 / len, s2 / len, 1.0f);
  }
  Nout[i] = out;
}

// Post-fusion error (Sec. 8.2): per CTA, the sum of |rendered - measured| and the count over the
// pixels where both depths are positive, in FP64; the CTA partials are summed in a fixed order by
// k_mae_final, so the result does not depend on scheduling.
constexpr int MAE_CTAS = 256;
__global__ void __launch_bounds__(256) k_mae_partial(const float* __restrict__ a, const float* __restrict__ b,
                                                     int64_t n, double* __restrict__ part) {
  __shared__ double ss[256];
  __shared__ double sc[256];
  double s = 0.0, c = 0.0;
  for (int64_t i = blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)MAE_CTAS * 256) {
    const float x = a[i], y = b[i];
    if (x > 0.f && y > 0.f) {
      s += fabs((double)x - (double)y);
      c += 1.0;
    }
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      ss[threadIdx.x] += ss[threadIdx.x + o];
      sc[threadIdx.x] += sc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ss[0];
    part[2 * blockIdx.x + 1] = sc[0];
  }
}

__global__ void k_mae_final(const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s = 0.0, c = 0.0;
  for (int k = 0; k < MAE_CTAS; ++k) {
    s += part[2 * k];
    c += part[2 * k + 1];
  }
  out[0] = s;
  out[1] = c;
}

// ---------------------------------------------------------------- allocation
// Record that block (bx, by, bz) needs the directions in `mask`.
__device__ void request_block(const MapView& m, int bx, int by, int bz, uint32_t mask) {
  const unsigned long long k = pack_block(bx, by, bz);
  uint32_t i = hash_slot(k, m.hmask);
  int p = 0;
  for (; p < MAX_PROBE; ++p) {
    unsigned long long kk = *((volatile unsigned long long*)(m.keys + i));
    if (kk == EMPTY_KEY) {
      kk = atomicCAS(m.keys + i, EMPTY_KEY, k);
      if (kk == EMPTY_KEY) kk = k;
    }
    if (kk == k) break;
    i = (i + 1) & m.hmask;
  }
  if (p == MAX_PROBE) {
    atomicOr(m.counters + C_ERR, ERR_HASH_FULL);
    return;
  }
  const uint32_t v = *((volatile uint32_t*)(m.vals + i));
  if (v != VAL_EMPTY && (mask & ~val_mask(v)) == 0) return;
  const uint32_t old = atomicOr(m.req + i, mask);
  if (old == 0) {
    const uint32_t w = atomicAdd(m.counters + C_WORK, 1u);
    if (w < m.work_cap)
      m.work[w] = (int32_t)i;
    else
      atomicOr(m.counters + C_ERR, ERR_WORK_FULL);
  }
}

// Per pixel with a normal: directions of Eq. angular_threshold (<n_w, v^D> > cos theta),
// then every block the segment [p - tau r, p + tau r] crosses, by a 3D DDA in block
// units (ties broken x, y, z).
__global__ void k_alloc_request(MapView m, const float4* __restrict__ P, const float4* __restrict__ N, int npix,
                                Pose32 Tv, const double* __restrict__ Tdev) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  const Pose32 T = Tdev ? pose_from_device(Tdev) : Tv;
  const float4 n = N[i];
  if (!(n.w > 0)) return;
  float nw[3];
  rrot(T.R, n.x, n.y, n.z, nw[0], nw[1], nw[2]);
  uint32_t mask = 0;
#pragma unroll
  for (int D = 0; D < ND; ++D) {
    const float c = (D & 1) ? -nw[D >> 1] : nw[D >> 1];
    if (c > m.costh) mask |= 1u << D;
  }
  if (!mask) return;
  const float4 p = P[i];
  float rv[3], pw[3], rh[3], A[3], B[3];
  rrot(T.R, p.x, p.y, p.z, rv[0], rv[1], rv[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) pw[a] = radd(rv[a], T.t[a]);
  const float len = rsqrt_exact(rdot3(rv[0], rv[1], rv[2], rv[0], rv[1], rv[2]));
  const float org[3] = {m.ox, m.oy, m.oz};
  const float bs = rmul(8.0f, m.h);
  float d[3], tmax[3], tdel[3];
  int c[3], e[3], st[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    rh[a] = rdiv(rv[a], len);
    A[a] = rsub(pw[a], rmul(m.tau, rh[a]));
    B[a] = radd(pw[a], rmul(m.tau, rh[a]));
    const float Ab = rdiv(rsub(A[a], org[a]), bs);
    const float Bb = rdiv(rsub(B[a], org[a]), bs);
    d[a] = rsub(Bb, Ab);
    c[a] = (int)floorf(Ab);
    e[a] = (int)floorf(Bb);
    if (d[a] > 0.0f) {
      st[a] = 1;
      tdel[a] = rdiv(1.0f, d[a]);
      tmax[a] = rdiv(rsub((float)(c[a] + 1), Ab), d[a]);
    } else if (d[a] < 0.0f) {
      st[a] = -1;
      tdel[a] = rdiv(-1.0f, d[a]);
      tmax[a] = rdiv(rsub((float)c[a], Ab), d[a]);
    } else {
      st[a] = 0;
      tdel[a] = INFINITY;
      tmax[a] = INFINITY;
    }
  }
  for (int it = 0; it < 64; ++it) {
    request_block(m, c[0], c[1], c[2], mask);
    if (c[0] == e[0] && c[1] == e[1] && c[2] == e[2]) break;
    int ax = 0;
    if (tmax[1] < tmax[ax]) ax = 1;
    if (tmax[2] < tmax[ax]) ax = 2;
    if (tmax[ax] > 1.0f) break;
    c[ax] += st[ax];
    tmax[ax] = radd(tmax[ax], tdel[ax]);
  }
}

// Assign directory entries and bricks to the requests of this frame (one thread per
// requested hash slot, so each directory entry has a single writer).
__global__ void k_alloc_assign(MapView m) {
  const uint32_t nwork = min(*((volatile uint32_t*)(m.counters + C_WORK)), m.work_cap);
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwork; w += gridDim.x * blockDim.x) {
    const int i = m.work[w];
    int d = val_dir(m.vals[i]);
    if (d < 0) {
      const uint32_t nd = atomicAdd(m.counters + C_DIR, 1u);
      if (nd >= m.dir_cap) {
        atomicOr(m.counters + C_ERR, ERR_DIR_FULL);
        m.req[i] = 0;
        continue;
      }
      d = (int)nd;
      int bx, by, bz;
      unpack_block(m.keys[i], bx, by, bz);
      occ_set(m, bx, by, bz);
      m.dir_coord[4 * d] = bx;
      m.dir_coord[4 * d + 1] = by;
      m.dir_coord[4 * d + 2] = bz;
      m.dir_coord[4 * d + 3] = 0;
      __threadfence();
      *((volatile uint32_t*)(m.vals + i)) = pack_val(d, 0u);
    }
    const uint32_t want = m.req[i];
    m.req[i] = 0;
    int32_t* slots = m.dir_slots + (size_t)d * 8;
    uint32_t have = (uint32_t)slots[SLOT_MASK];
    for (int D = 0; D < ND; ++D) {
      if (!(want & (1u << D)) || (have & (1u << D))) continue;
      // a recycled brick first (the ring holds C_FREE_N - C_FREE_TAKEN of them; a take past
      // the end falls back to the pool and the count is clamped after this kernel)
      uint32_t s;
      const uint32_t t = m.free_ring ? atomicAdd(m.counters + C_FREE_TAKEN, 1u) : 0xFFFFFFFFu;
      if (m.free_ring && t < *((volatile uint32_t*)(m.counters + C_FREE_N))) {
        s = (uint32_t)m.free_ring[t % m.pool_cap];
      } else {
        s = atomicAdd(m.counters + C_POOL, 1u);
        if (s >= m.pool_cap) {
          atomicOr(m.counters + C_ERR, ERR_POOL_FULL);
          continue;
        }
      }
      m.brick_dir[s] = d * 8 + D;
      // a new brick's apron may already hold data: no bound until it is recomputed
      m.bound[s] = -INFINITY;
      m.stamp[s] = m.frame;
      slots[D] = (int32_t)s;
      have |= 1u << D;
    }
    __threadfence();
    slots[SLOT_MASK] = (int32_t)have;
    *((volatile uint32_t*)(m.vals + i)) = pack_val(d, have);
  }
}

// Takes past the ring's end fell back to the pool: bring the taken count back to the end.
__global__ void k_free_clamp(uint32_t* counters) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && counters[C_FREE_TAKEN] > counters[C_FREE_N])
    counters[C_FREE_TAKEN] = counters[C_FREE_N];
}

// Dense mode: every (block, direction) of an n^3-block grid, directory index = linear block
// index, brick = 6 * index + D.
__global__ void k_dense_fill(MapView m, int nb) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nb * nb * nb) return;
  const int bx = idx % nb, by = (idx / nb) % nb, bz = idx / (nb * nb);
  const unsigned long long k = pack_block(bx, by, bz);
  uint32_t i = hash_slot(k, m.hmask);
  for (int p = 0; p < MAX_PROBE; ++p) {
    const unsigned long long kk = atomicCAS(m.keys + i, EMPTY_KEY, k);
    if (kk == EMPTY_KEY || kk == k) break;
    i = (i + 1) & m.hmask;
  }
  m.vals[i] = pack_val(idx, 0x3Fu);
  occ_set(m, bx, by, bz);
  m.dir_coord[4 * idx] = bx;
  m.dir_coord[4 * idx + 1] = by;
  m.dir_coord[4 * idx + 2] = bz;
  m.dir_coord[4 * idx + 3] = 0;
  for (int D = 0; D < ND; ++D) {
    m.dir_slots[(size_t)idx * 8 + D] = idx * ND + D;
    m.brick_dir[idx * ND + D] = idx * 8 + D;
  }
  m.dir_slots[(size_t)idx * 8 + SLOT_MASK] = 0x3F;
  m.dir_slots[(size_t)idx * 8 + 7] = 0;
}

// Every voxel starts at sdf 1, weight 0 (geometry including the aprons), colour 0.
__global__ void k_pool_init(MapView m, int with_color) {
  const size_t n = (size_t)m.pool_cap * PVOX;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (m.storage == DTSDF_STORE_FP16)
      m.geom16[i] = pack_geom16(1.0f, 0.0f);
    else
      m.geom[i] = make_float2(1.0f, 0.0f);
    if (i < m.pool_cap) m.bound[i] = INFINITY;
    if (with_color && i < (size_t)m.pool_cap * BVOX) {
      if (m.storage == DTSDF_STORE_FP16)
        m.col8[i] = 0u;
      else
        m.col[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// ------------------------------------------------------------------ fusion
struct FuseFrame {
  const uint8_t* J;    // per pixel: a valid depth within the carving radius differs by more than tau
  Intr K;
  Pose32 T;            // camera -> world (unless Tdev is given)
  const double* Tdev;  // camera -> world in device memory, or null
  const float4* P;
  const float4* N;
  const uint8_t* rgb;
  // conservative frustum planes through the camera centre (camera frame, unit normals)
  float pl[4][3];
};

__device__ __forceinline__ float w_dir_of(float c, float theta) {
  const float alpha = acosf(fminf(fmaxf(c, -1.0f), 1.0f));
  return fminf(fmaxf((theta - alpha) / (2.0f * theta - 1.57079632679489662f), 0.0f), 1.0f);
}

template <int STORE>
__device__ __forceinline__ float2 load_geom(const MapView& m, size_t i) {
  if (STORE == DTSDF_STORE_FP16) return unpack_geom16(m.geom16[i]);
  return m.geom[i];
}

template <int STORE>
__device__ __forceinline__ void store_geom(const MapView& m, size_t i, float sdf, float w) {
  if (STORE == DTSDF_STORE_FP16)
    m.geom16[i] = pack_geom16(sdf, w);
  else
    m.geom[i] = make_float2(sdf, w);
}

// Carving test of every pixel with a back-projected point: 1 if a valid pixel within the
// carving radius has a depth differing from it by more than tau (Sec. 3, free-space carving
// only where no depth discontinuity is near).
__global__ void k_carve_flags(const float4* __restrict__ P, Intr K, int rad, float tau, uint8_t* __restrict__ J) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= K.W || v >= K.H) return;
  const float4 p = P[v * K.W + u];
  bool jump = false;
  if (p.w > 0) {
    for (int dv = -rad; dv <= rad && !jump; ++dv)
      for (int du = -rad; du <= rad; ++du) {
        const int uu = u + du, vv = v + dv;
        if (uu < 0 || vv < 0 || uu >= K.W || vv >= K.H) continue;
        const float4 q = P[vv * K.W + uu];
        if (!(q.w > 0)) continue;
        if (fabsf(rsub(q.z, p.z)) > tau) {
          jump = true;
          break;
        }
      }
  }
  J[v * K.W + u] = jump ? 1 : 0;
}

// Conservative frustum test of block (bx, by, bz): its bounding sphere, grown by `margin`,
// reaches the camera's half-space z > 0 and the four side planes.
__device__ __forceinline__ bool block_visible(const MapView& m, const FuseFrame& f, int bx, int by, int bz,
                                              float margin) {
  const float h = m.h;
  const float r = 0.8660254f * 8.0f * h + h + margin;
  const float cw0 = m.ox + (8.0f * bx + 3.5f) * h - f.T.t[0];
  const float cw1 = m.oy + (8.0f * by + 3.5f) * h - f.T.t[1];
  const float cw2 = m.oz + (8.0f * bz + 3.5f) * h - f.T.t[2];
  const float cz = f.T.R[2] * cw0 + f.T.R[5] * cw1 + f.T.R[8] * cw2;
  if (cz <= -r) return false;
  const float cx = f.T.R[0] * cw0 + f.T.R[3] * cw1 + f.T.R[6] * cw2;
  const float cy = f.T.R[1] * cw0 + f.T.R[4] * cw1 + f.T.R[7] * cw2;
  bool out = false;
#pragma unroll
  for (int q = 0; q < 4; ++q) out |= (f.pl[q][0] * cx + f.pl[q][1] * cy + f.pl[q][2] * cz) < -r;
  return !out;
}

// One CTA per brick at a time (grid-stride over the pool): cull the block against the
// frustum, then every voxel is projected to its nearest pixel and updated with the
// weighted running average (Sec. 3). A voxel has one writer, so fusion is deterministic.
// A brick with an updated voxel is stamped with the frame id for the apron refresh.
// Apron maintenance by the brick that changed: brick b (block (bx, by, bz), direction D)
// copies its core voxels into the aprons of its 26 neighbours. The apron voxel at local
// coordinate x of the neighbour at block offset -e comes from this brick's core voxel x - 8 e
// (e = floor(x / 8) per axis). It reads only its own core, which no other CTA writes, and
// writes only aprons, which nobody reads during fusion, so bricks push concurrently. The
// brick and the neighbours whose bound region [0, 8]^3 holds its voxels (offsets -e with e in
// {0, 1}^3) are stamped with the frame for the exact bound pass.
template <int STORE>
__device__ void push_borders(const MapView& m, int b, int bx, int by, int bz, int D) {
  __shared__ int s_nb[27];
  if (threadIdx.x < 27) {
    const int q = threadIdx.x;  // neighbour at block offset (q % 3 - 1, q / 3 % 3 - 1, q / 9 - 1)
    int sl = -1;
    if (q != 13) {
      const int dd = hash_find(m, bx + q % 3 - 1, by + (q / 3) % 3 - 1, bz + q / 9 - 1);
      sl = dd >= 0 ? m.dir_slots[(size_t)dd * 8 + D] : -1;
    }
    s_nb[q] = sl;
    // bound regions that contain this brick's voxels: its own and those at offsets in {-1, 0}^3
    if (q == 13)
      m.stamp[b] = m.frame;
    else if (sl >= 0 && q % 3 != 2 && (q / 3) % 3 != 2 && q / 9 != 2)
      m.stamp[sl] = m.frame;
  }
  __syncthreads();
  const size_t src = (size_t)b * PVOX;
  for (int vi = threadIdx.x; vi < PVOX; vi += blockDim.x) {
    const int x = vi % PAD - 1, y = (vi / PAD) % PAD - 1, z = vi / (PAD * PAD) - 1;
    const int ex = x >> 3, ey = y >> 3, ez = z >> 3;
    if ((ex | ey | ez) == 0) continue;  // core position: no neighbour holds it in an apron
    const int sl = s_nb[(1 - ez) * 9 + (1 - ey) * 3 + (1 - ex)];
    if (sl < 0) continue;
    const size_t from = src + pad_index(x & 7, y & 7, z & 7);
    if (STORE == DTSDF_STORE_FP16)
      m.geom16[(size_t)sl * PVOX + vi] = m.geom16[from];
    else
      m.geom[(size_t)sl * PVOX + vi] = m.geom[from];
  }
  __syncthreads();
}

template <int STORE>
__global__ void __launch_bounds__(128, 16) k_fuse(MapView m, FuseFrame f) {
  const uint32_t nb = min(*((volatile uint32_t*)(m.counters + C_POOL)), m.pool_cap);
  if (f.Tdev) f.T = pose_from_device(f.Tdev);
  const float h = m.h;
  for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const int bd = __ldg(m.brick_dir + b);
    if (bd < 0) continue;  // a recycled brick in the free ring
    const int d = bd >> 3, D = bd & 7;
    const int bx = __ldg(m.dir_coord + 4 * d), by = __ldg(m.dir_coord + 4 * d + 1),
              bz = __ldg(m.dir_coord + 4 * d + 2);
    if (!block_visible(m, f, bx, by, bz, 0.0f)) continue;
    bool updated = false;
    for (int vi = threadIdx.x; vi < BVOX; vi += blockDim.x) {
      const int i = vi & 7, j = (vi >> 3) & 7, k = vi >> 6;
      // single-precision decision path: voxel centre, camera frame, projection
      const float x0 = radd(rmul((float)(8 * bx + i), h), m.ox);
      const float x1 = radd(rmul((float)(8 * by + j), h), m.oy);
      const float x2 = radd(rmul((float)(8 * bz + k), h), m.oz);
      float xc0, xc1, xc2;
      rrotT(f.T.R, rsub(x0, f.T.t[0]), rsub(x1, f.T.t[1]), rsub(x2, f.T.t[2]), xc0, xc1, xc2);
      if (!(xc2 > 0.0f)) continue;
      const float uf = radd(rmul(rdiv(xc0, xc2), f.K.fx), f.K.cx);
      const float vf = radd(rmul(rdiv(xc1, xc2), f.K.fy), f.K.cy);
      const float ur = floorf(radd(uf, 0.5f)), vr = floorf(radd(vf, 0.5f));
      if (!(ur >= 0.0f && vr >= 0.0f && ur < (float)f.K.W && vr < (float)f.K.H)) continue;
      const int u = (int)ur, v = (int)vr;
      const int pi = v * f.K.W + u;
      const float4 n = __ldg(f.N + pi);
      if (!(n.w > 0)) continue;
      const float4 P = __ldg(f.P + pi);
      const float e0 = rsub(xc0, P.x), e1 = rsub(xc1, P.y), e2 = rsub(xc2, P.z);
      const float draw = rdot3(e0, e1, e2, n.x, n.y, n.z);
      if (draw < -m.tau) continue;
      const size_t gi = (size_t)b * PVOX + pad_index(i, j, k);  // geometry (padded brick)
      const size_t ci = (size_t)b * BVOX + vi;                  // colour
      if (draw > m.tau) {
        // free-space carving, unless a depth jump > tau lies within the carving radius of the
        // pixel (a property of the pixel alone, flagged once per frame by k_carve_flags)
        if (__ldg(f.J + pi)) continue;
        const float2 g = load_geom<STORE>(m, gi);
        const float wn = g.y + m.wcarve;
        const float nsdf = (g.y * g.x + m.wcarve) / wn;
        store_geom<STORE>(m, gi, nsdf, fminf(wn, m.wmax));
        updated = true;
        continue;
      }
      // membership of the pixel normal in direction D, and a camera-facing normal
      float nw0, nw1, nw2;
      rrot(f.T.R, n.x, n.y, n.z, nw0, nw1, nw2);
      const float cd = (D == 0) ? nw0 : (D == 1) ? -nw0 : (D == 2) ? nw1 : (D == 3) ? -nw1 : (D == 4) ? nw2 : -nw2;
      if (!(cd > m.costh)) continue;
      const float ndp = rdot3(n.x, n.y, n.z, P.x, P.y, P.z);
      if (!(ndp < 0.0f)) continue;
      // values (Eq. point-to-plane, Eq. combined_fusion_weight)
      const float sd = fminf(fmaxf(draw / m.tau, -1.0f), 1.0f);
      const float zz = P.z + 1.0f - m.zmin;
      const float w_depth = 1.0f / (zz * zz);
      const float plen = sqrtf(P.x * P.x + P.y * P.y + P.z * P.z);
      const float w_angle = fmaxf(-ndp / plen, 0.0f);
      float w_d = w_depth * w_angle * w_dir_of(cd, m.theta);
      if (!(w_d > 1e-12f)) w_d = 1e-12f;
      const float2 g = load_geom<STORE>(m, gi);
      const float wn = g.y + w_d;
      const float nsdf = (g.y * g.x + w_d * sd) / wn;
      store_geom<STORE>(m, gi, nsdf, fminf(wn, m.wmax));
      updated = true;
      if (m.color && f.rgb) {
        const float dist = rsqrt_exact(rdot3(e0, e1, e2, e0, e1, e2));
        if (dist < m.tau) {
          float w_c = w_d * (1.0f - fminf(1.0f, dist / m.tau));
          if (!(w_c > 1e-12f)) w_c = 1e-12f;
          const uint8_t* c = f.rgb + 3 * pi;
          if (STORE == DTSDF_STORE_FP16) {
            const float4 cv = unpack_col8(m.col8[ci]);
            const float wcn = cv.w + w_c;
            m.col8[ci] = pack_col8((cv.w * cv.x + w_c * c[0]) / wcn, (cv.w * cv.y + w_c * c[1]) / wcn,
                                   (cv.w * cv.z + w_c * c[2]) / wcn, fminf(wcn, m.wmax));
          } else {
            float4 cv = m.col[ci];
            const float wcn = cv.w + w_c;
            cv.x = (cv.w * cv.x + w_c * c[0]) / wcn;
            cv.y = (cv.w * cv.y + w_c * c[1]) / wcn;
            cv.z = (cv.w * cv.z + w_c * c[2]) / wcn;
            cv.w = fminf(wcn, m.wmax);
            m.col[ci] = cv;
          }
        }
      }
    }
    if (!__syncthreads_or(updated)) continue;
    push_borders<STORE>(m, (int)b, bx, by, bz, D);
  }
}

// Exact bound of a brick: minimum sdf over its voxels at local coordinates [0, 8]^3 with
// weight > 0 (+inf if none), reduced over the CTA.
template <int STORE>
__device__ void exact_bound(const MapView& m, uint32_t b) {
  __shared__ float s_red[8];
  const size_t base = (size_t)b * PVOX;
  float mn = INFINITY;
  for (int vi = threadIdx.x; vi < 729; vi += blockDim.x) {
    const int x = vi % 9, y = (vi / 9) % 9, z = vi / 81;
    const float2 g = load_geom<STORE>(m, base + pad_index(x, y, z));
    if (g.y > 0.0f) mn = fminf(mn, g.x);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = mn;
  __syncthreads();
  if (threadIdx.x == 0) {
    float x = INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x = fminf(x, s_red[w]);
    m.bound[b] = x;
  }
  __syncthreads();
}

// Apron pull: the bricks [C_POOL_BEFORE, C_POOL) allocated this frame (every brick when `all`)
// copy their neighbours' voxels at local coordinates -1, 8 and 9 into their apron (an
// unallocated neighbour reads as sdf 1, weight 0, the initial value, so it stays absent for
// presence tests). Runs before fusion for new bricks (fusion then pushes what it changes) and
// after an import for every brick; reads touch only cores and writes only aprons. With `all`
// the exact bound follows.
template <int STORE>
__global__ void __launch_bounds__(256) k_apron_pull(MapView m, int all) {
  __shared__ int s_nb[27];
  const uint32_t nb = min(*((volatile uint32_t*)(m.counters + C_POOL)), m.pool_cap);
  const uint32_t b0 = all ? 0u : min(*((volatile uint32_t*)(m.counters + C_POOL_BEFORE)), nb);
  // recycled bricks handed out again this frame: ring positions [C_FREE_BEFORE, C_FREE_TAKEN)
  const uint32_t r0 = all || !m.free_ring ? 0u : *((volatile uint32_t*)(m.counters + C_FREE_BEFORE));
  const uint32_t r1 = all || !m.free_ring ? 0u : *((volatile uint32_t*)(m.counters + C_FREE_TAKEN));
  const uint32_t nitems = (nb - b0) + (r1 > r0 ? r1 - r0 : 0u);
  for (uint32_t it = blockIdx.x; it < nitems; it += gridDim.x) {
    const uint32_t b = it < nb - b0 ? b0 + it : (uint32_t)m.free_ring[(r0 + (it - (nb - b0))) % m.pool_cap];
    const int bd = m.brick_dir[b];
    if (bd < 0) continue;
    const int d = bd >> 3, D = bd & 7;
    const int bx = m.dir_coord[4 * d], by = m.dir_coord[4 * d + 1], bz = m.dir_coord[4 * d + 2];
    if (threadIdx.x < 27) {
      const int q = threadIdx.x;
      int sl = (int)b;
      if (q != 13) {
        const int dd = hash_find(m, bx + q % 3 - 1, by + (q / 3) % 3 - 1, bz + q / 9 - 1);
        sl = dd >= 0 ? m.dir_slots[(size_t)dd * 8 + D] : -1;
      }
      s_nb[q] = sl;
    }
    __syncthreads();
    const size_t base = (size_t)b * PVOX;
    for (int vi = threadIdx.x; vi < PVOX; vi += blockDim.x) {
      const int x = vi % PAD - 1, y = (vi / PAD) % PAD - 1, z = vi / (PAD * PAD) - 1;
      if ((unsigned)x < 8u && (unsigned)y < 8u && (unsigned)z < 8u) continue;
      const int sl = s_nb[((z >> 3) + 1) * 9 + ((y >> 3) + 1) * 3 + ((x >> 3) + 1)];
      const size_t src = (size_t)sl * PVOX + pad_index(x & 7, y & 7, z & 7);
      if (STORE == DTSDF_STORE_FP16)
        m.geom16[base + vi] = sl >= 0 ? m.geom16[src] : pack_geom16(1.0f, 0.0f);
      else
        m.geom[base + vi] = sl >= 0 ? m.geom[src] : make_float2(1.0f, 0.0f);
    }
    __syncthreads();
    if (all) exact_bound<STORE>(m, b);
  }
}

// Exact bounds of the bricks whose bound region changed this frame (stamped by fusion): one warp
// per brick (23 voxels of [0, 8]^3 per lane, a shuffle reduction), without CTA barriers.
template <int STORE>
__global__ void __launch_bounds__(256) k_bounds_exact(MapView m) {
  const uint32_t nb = min(*((volatile uint32_t*)(m.counters + C_POOL)), m.pool_cap);
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nb; b += warps) {
    if (!(m.stamp[b] == m.frame && m.brick_dir[b] >= 0)) continue;  // uniform over the warp
    const size_t base = (size_t)b * PVOX;
    float mn = INFINITY;
    for (int vi = lane; vi < 729; vi += 32) {
      const int x = vi % 9, y = (vi / 9) % 9, z = vi / 81;
      const float2 g = load_geom<STORE>(m, base + pad_index(x, y, z));
      if (g.y > 0.0f) mn = fminf(mn, g.x);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    if (lane == 0) m.bound[b] = mn;
  }
}

// ------------------------------------------------------------------ import
// Request the (block, direction) bricks of an imported map (same hash path as allocation).
__global__ void k_import_request(MapView m, const int32_t* __restrict__ coords, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int D = coords[4 * i + 3];
  if (D < 0 || D >= ND) return;
  request_block(m, coords[4 * i], coords[4 * i + 1], coords[4 * i + 2], 1u << D);
}

// Write imported voxel data (sdf, w, r, g, b, wc per voxel) into the bricks.
__global__ void k_import_write(MapView m, const int32_t* __restrict__ coords, const float* __restrict__ vox,
                               int64_t n) {
  for (int64_t b = blockIdx.x; b < n; b += gridDim.x) {
    const int D = coords[4 * b + 3];
    if (D < 0 || D >= ND) continue;
    const int d = hash_find(m, coords[4 * b], coords[4 * b + 1], coords[4 * b + 2]);
    if (d < 0) continue;
    const int slot = m.dir_slots[(size_t)d * 8 + D];
    if (slot < 0) continue;
    for (int vi = threadIdx.x; vi < BVOX; vi += blockDim.x) {
      const float* in = vox + ((size_t)b * BVOX + vi) * 6;
      const size_t gi = (size_t)slot * PVOX + pad_index(vi & 7, (vi >> 3) & 7, vi >> 6);
      const size_t ci = (size_t)slot * BVOX + vi;
      if (m.storage == DTSDF_STORE_FP16)
        m.geom16[gi] = pack_geom16(in[0], in[1]);
      else
        m.geom[gi] = make_float2(in[0], in[1]);
      if (m.color) {
        if (m.storage == DTSDF_STORE_FP16) {
          m.col8[ci] = pack_col8(in[2], in[3], in[4], in[5]);
        } else {
          m.col[ci] = make_float4(in[2], in[3], in[4], in[5]);
        }
      }
    }
  }
}

// ------------------------------------------------------------------- poses
// C = op(A) B for 4x4 affine transforms in device memory (op(A) = A or A^-1).
__global__ void k_pose_compose(const double* A, int invert_a, const double* B, double* C) {
  double M[16];
  if (invert_a) {
    const double a = A[0], b = A[1], c = A[2], d = A[4], e = A[5], f = A[6], g = A[8], h = A[9], k = A[10];
    const double co0 = e * k - f * h, co1 = f * g - d * k, co2 = d * h - e * g;
    const double det = a * co0 + b * co1 + c * co2;
    const double id = 1.0 / det;
    const double inv[9] = {co0 * id, (c * h - b * k) * id, (b * f - c * e) * id,
                           co1 * id, (a * k - c * g) * id, (c * d - a * f) * id,
                           co2 * id, (b * g - a * h) * id, (a * e - b * d) * id};
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) M[4 * i + j] = inv[3 * i + j];
      M[4 * i + 3] = -(inv[3 * i] * A[3] + inv[3 * i + 1] * A[7] + inv[3 * i + 2] * A[11]);
    }
    M[12] = M[13] = M[14] = 0.0;
    M[15] = 1.0;
  } else {
    for (int i = 0; i < 16; ++i) M[i] = A[i];
  }
  double out[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double acc = 0;
      for (int q = 0; q < 4; ++q) acc += M[4 * i + q] * B[4 * q + j];
      out[4 * i + j] = acc;
    }
  for (int i = 0; i < 16; ++i) C[i] = out[i];
}

// depth brought to the model's metric: out = scale * in, 0 (invalid) stays 0
__global__ void k_depth_scale(const float* __restrict__ in, float* __restrict__ out, int64_t n, float scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __fmul_rn(in[i], scale);
}

void launch_depth_scale(const float* in, float* out, int64_t n, float scale, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t blocks = (n + 255) / 256;
  k_depth_scale<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(in, out, n, scale);
}

void launch_pose_compose(const double* A, int invert_a, const double* B, double* C, cudaStream_t s) {
  k_pose_compose<<<1, 1, 0, s>>>(A, invert_a, B, C);
}

// ------------------------------------------------------------------ export
__global__ void k_export(MapView m, int64_t cap, int32_t* coords, float* vox) {
  const uint32_t nb = min(*((volatile uint32_t*)(m.counters + C_POOL)), m.pool_cap);
  for (uint32_t b = blockIdx.x; b < nb && b < cap; b += gridDim.x) {
    const int bd = m.brick_dir[b];
    const int d = bd >> 3;
    if (threadIdx.x < 4) {  // a recycled brick: (0, 0, 0, -1)
      coords[4 * (size_t)b + threadIdx.x] =
          bd < 0 ? (threadIdx.x < 3 ? 0 : -1) : (threadIdx.x < 3 ? m.dir_coord[4 * d + threadIdx.x] : (bd & 7));
    }
    for (int vi = threadIdx.x; vi < BVOX; vi += blockDim.x) {
      const size_t ci = (size_t)b * BVOX + vi;
      const size_t gi = (size_t)b * PVOX + pad_index(vi & 7, (vi >> 3) & 7, vi >> 6);
      float* o = vox + ci * 6;
      float2 g = (m.storage == DTSDF_STORE_FP16) ? unpack_geom16(m.geom16[gi]) : m.geom[gi];
      o[0] = g.x;
      o[1] = g.y;
      if (m.color) {
        if (m.storage == DTSDF_STORE_FP16) {
          const float4 c = unpack_col8(m.col8[ci]);
          o[2] = c.x;
          o[3] = c.y;
          o[4] = c.z;
          o[5] = c.w;
        } else {
          const float4 c = m.col[ci];
          o[2] = c.x;
          o[3] = c.y;
          o[4] = c.z;
          o[5] = c.w;
        }
      } else {
        o[2] = o[3] = o[4] = o[5] = 0.f;
      }
    }
  }
}

// --------------------------------------------------------------- launchers
void launch_preprocess(const float* depth, const Intr& K, float zmin, float zmax, float dsup, float4* P, float4* N,
                       cudaStream_t s, const FilterOpts* f, float4* tmp) {
  dim3 blk(32, 8), grd((K.W + 31) / 32, (K.H + 7) / 8);
  const bool fd = f && f->depth_radius > 0 && tmp, fn = f && f->normal_radius > 0 && tmp;
  const dsf ifx = ds_from_double(1.0 / (double)K.fx), ify = ds_from_double(1.0 / (double)K.fy);
  if (fd) {
    k_filter<<<grd, blk, 0, s>>>(depth, K, zmin, zmax, dsup, ifx, ify, tmp);
    k_bilateral_depth<<<grd, blk, 0, s>>>(tmp, K, f->depth_radius, f->depth_sigma_d, f->depth_sigma_r, P);
  } else {
    k_filter<<<grd, blk, 0, s>>>(depth, K, zmin, zmax, dsup, ifx, ify, P);
  }
  if (fn) {
    k_normals<<<grd, blk, 0, s>>>(P, K, ifx, ify, tmp);
    k_bilateral_normals<<<grd, blk, 0, s>>>(tmp, K, f->normal_radius, f->normal_sigma_d, f->normal_sigma_r, N);
  } else {
    k_normals<<<grd, blk, 0, s>>>(P, K, ifx, ify, N);
  }
}

void launch_mae(const float* a, const float* b, int64_t n, double* part, double* out, cudaStream_t s) {
  k_mae_partial<<<MAE_CTAS, 256, 0, s>>>(a, b, n, part);
  k_mae_final<<<1, 32, 0, s>>>(part, out);
}

void launch_alloc(const MapView& m, const float4* P, const float4* N, int npix, const Pose32& T, const double* Tdev,
                  int num_sms, cudaStream_t s) {
  k_alloc_request<<<(npix + 255) / 256, 256, 0, s>>>(m, P, N, npix, T, Tdev);
  k_alloc_assign<<<num_sms * 2, 256, 0, s>>>(m);
  if (m.free_ring) k_free_clamp<<<1, 32, 0, s>>>(m.counters);
}

// ------------------------------------------------------------------ recycling
// A brick is recycled when every core voxel with weight > 0 has sdf >= free_sdf: repeated
// carving (running averages toward 1) left only free space in it (Sec. 3). The list of such
// bricks is built first; then each is detached: its slot leaves the directory and the hash
// mask, its copies in the 26 neighbours' aprons return to the empty value (1, 0), its voxels
// are reset and it is pushed to the free ring for the allocator.
template <int STORE>
__global__ void __launch_bounds__(256) k_recycle_mark(MapView m, float free_sdf, int32_t* list, uint32_t* nlist) {
  const uint32_t nb = min(*((volatile uint32_t*)(m.counters + C_POOL)), m.pool_cap);
  for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
    if (m.brick_dir[b] < 0) continue;
    bool free_only = true;
    for (int vi = threadIdx.x; vi < BVOX; vi += blockDim.x) {
      const size_t gi = (size_t)b * PVOX + pad_index(vi & 7, (vi >> 3) & 7, vi >> 6);
      const float2 g = STORE == DTSDF_STORE_FP16 ? unpack_geom16(m.geom16[gi]) : m.geom[gi];
      if (g.y > 0.0f && !(g.x >= free_sdf)) free_only = false;
    }
    free_only = __syncthreads_and(free_only);
    if (free_only && threadIdx.x == 0) list[atomicAdd(nlist, 1u)] = (int32_t)b;
  }
}

template <int STORE>
__global__ void __launch_bounds__(256) k_recycle_apply(MapView m, const int32_t* list, const uint32_t* nlist) {
  __shared__ int s_nb[27];
  const uint32_t n = *nlist;
  for (uint32_t it = blockIdx.x; it < n; it += gridDim.x) {
    const int b = list[it];
    const int bd = m.brick_dir[b];
    const int d = bd >> 3, D = bd & 7;
    const int bx = m.dir_coord[4 * d], by = m.dir_coord[4 * d + 1], bz = m.dir_coord[4 * d + 2];
    if (threadIdx.x < 27) {
      const int q = threadIdx.x;
      int sl = -1;
      if (q != 13) {
        const int dd = hash_find(m, bx + q % 3 - 1, by + (q / 3) % 3 - 1, bz + q / 9 - 1);
        sl = dd >= 0 ? m.dir_slots[(size_t)dd * 8 + D] : -1;
      }
      s_nb[q] = sl;
    }
    __syncthreads();
    // the neighbours' apron positions that mirror this brick's voxels (as the apron push writes them)
    for (int vi = threadIdx.x; vi < PVOX; vi += blockDim.x) {
      const int x = vi % PAD - 1, y = (vi / PAD) % PAD - 1, z = vi / (PAD * PAD) - 1;
      const int ex = x >> 3, ey = y >> 3, ez = z >> 3;
      if ((ex | ey | ez) == 0) continue;
      const int sl = s_nb[(1 - ez) * 9 + (1 - ey) * 3 + (1 - ex)];
      if (sl < 0) continue;
      if (STORE == DTSDF_STORE_FP16)
        m.geom16[(size_t)sl * PVOX + vi] = pack_geom16(1.0f, 0.0f);
      else
        m.geom[(size_t)sl * PVOX + vi] = make_float2(1.0f, 0.0f);
    }
    // the brick itself, core and apron, and its colour
    for (int vi = threadIdx.x; vi < PVOX; vi += blockDim.x) {
      if (STORE == DTSDF_STORE_FP16)
        m.geom16[(size_t)b * PVOX + vi] = pack_geom16(1.0f, 0.0f);
      else
        m.geom[(size_t)b * PVOX + vi] = make_float2(1.0f, 0.0f);
    }
    if (m.color) {
      for (int vi = threadIdx.x; vi < BVOX; vi += blockDim.x) {
        if (STORE == DTSDF_STORE_FP16)
          m.col8[(size_t)b * BVOX + vi] = 0u;
        else
          m.col[(size_t)b * BVOX + vi] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    if (threadIdx.x == 0) {
      // leave the directory and the hash mask
      m.dir_slots[(size_t)d * 8 + D] = -1;
      atomicAnd((unsigned*)(m.dir_slots + (size_t)d * 8 + SLOT_MASK), ~(1u << D));
      const unsigned long long k = pack_block(bx, by, bz);
      uint32_t i = hash_slot(k, m.hmask);
      for (int p = 0; p < MAX_PROBE; ++p) {
        const unsigned long long kk = m.keys[i];
        if (kk == k) {
          atomicAnd(m.vals + i, ~(1u << (26 + D)));
          break;
        }
        if (kk == EMPTY_KEY) break;
        i = (i + 1) & m.hmask;
      }
      m.bound[b] = INFINITY;
      m.brick_dir[b] = -1;
      const uint32_t pos = atomicAdd(m.counters + C_FREE_N, 1u);
      m.free_ring[pos % m.pool_cap] = b;
    }
    __syncthreads();
  }
}

void launch_recycle(const MapView& m, float free_sdf, int32_t* list, uint32_t* nlist, int num_sms, cudaStream_t s) {
  if (m.storage == DTSDF_STORE_FP16) {
    k_recycle_mark<DTSDF_STORE_FP16><<<num_sms * 8, 256, 0, s>>>(m, free_sdf, list, nlist);
    k_recycle_apply<DTSDF_STORE_FP16><<<num_sms * 4, 256, 0, s>>>(m, list, nlist);
  } else {
    k_recycle_mark<DTSDF_STORE_FP32><<<num_sms * 8, 256, 0, s>>>(m, free_sdf, list, nlist);
    k_recycle_apply<DTSDF_STORE_FP32><<<num_sms * 4, 256, 0, s>>>(m, list, nlist);
  }
}

void launch_dense_fill(const MapView& m, int nb, cudaStream_t s) {
  const int n = nb * nb * nb;
  k_dense_fill<<<(n + 127) / 128, 128, 0, s>>>(m, nb);
}

void launch_pool_init(const MapView& m, int with_color, int num_sms, cudaStream_t s) {
  k_pool_init<<<num_sms * 8, 256, 0, s>>>(m, with_color);
}

void launch_fuse(const MapView& m, const Intr& K, const Pose32& T, const double* Tdev, const float4* P,
                 const float4* N, const uint8_t* rgb, uint8_t* J, int num_sms, cudaStream_t s) {
  {
    dim3 blk(32, 8), grd((K.W + 31) / 32, (K.H + 7) / 8);
    k_carve_flags<<<grd, blk, 0, s>>>(P, K, m.carve_r, m.tau, J);
  }
  FuseFrame f;
  f.J = J;
  f.K = K;
  f.T = T;
  f.Tdev = Tdev;
  f.P = P;
  f.N = N;
  f.rgb = rgb;
  // inward unit normals of the four side planes (pixel edges at -0.5 and W-0.5)
  auto set = [&](int q, float a, float b, float c) {
    const float l = sqrtf(a * a + b * b + c * c);
    f.pl[q][0] = a / l;
    f.pl[q][1] = b / l;
    f.pl[q][2] = c / l;
  };
  set(0, K.fx, 0.f, K.cx + 0.5f);
  set(1, -K.fx, 0.f, (float)K.W - 0.5f - K.cx);
  set(2, 0.f, K.fy, K.cy + 0.5f);
  set(3, 0.f, -K.fy, (float)K.H - 0.5f - K.cy);
  const bool sparse = m.dense_dim <= 0;
  // fusion: CTAs of 128 threads (4 voxels each), so that twice as many bricks are in flight per
  // SM as with 256 (each brick's update is a chain of dependent gathers and barriers), with a
  // register budget for 16 of them per SM (32 registers, a few spilled bytes); the grid-stride
  // loop runs as one wave of the CTAs that fit on the device at once (a grid of 16 per SM at 48
  // registers, 10 of them resident, ran its last 6 as a second, under-filled wave)
  auto fuse_grid = [&](auto kern) {
    static thread_local int cached_dev = -1, per_sm = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_dev) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0) != cudaSuccess || per_sm < 1) per_sm = 8;
      cached_dev = dev;
    }
    return num_sms * per_sm;
  };
  if (m.storage == DTSDF_STORE_FP16) {
    if (sparse) k_apron_pull<DTSDF_STORE_FP16><<<num_sms * 4, 256, 0, s>>>(m, 0);
    k_fuse<DTSDF_STORE_FP16><<<fuse_grid(k_fuse<DTSDF_STORE_FP16>), 128, 0, s>>>(m, f);
    k_bounds_exact<DTSDF_STORE_FP16><<<num_sms * 8, 256, 0, s>>>(m);
  } else {
    if (sparse) k_apron_pull<DTSDF_STORE_FP32><<<num_sms * 4, 256, 0, s>>>(m, 0);
    k_fuse<DTSDF_STORE_FP32><<<fuse_grid(k_fuse<DTSDF_STORE_FP32>), 128, 0, s>>>(m, f);
    k_bounds_exact<DTSDF_STORE_FP32><<<num_sms * 8, 256, 0, s>>>(m);
  }
}

void launch_apron_refresh_all(const MapView& m, int num_sms, cudaStream_t s) {
  if (m.storage == DTSDF_STORE_FP16)
    k_apron_pull<DTSDF_STORE_FP16><<<num_sms * 8, 256, 0, s>>>(m, 1);
  else
    k_apron_pull<DTSDF_STORE_FP32><<<num_sms * 8, 256, 0, s>>>(m, 1);
}

void launch_import(const MapView& m, const int32_t* coords, const float* vox, int64_t n, bool allocate, int num_sms,
                   cudaStream_t s) {
  if (allocate && n > 0) {
    k_import_request<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m, coords, n);
    k_alloc_assign<<<num_sms * 2, 256, 0, s>>>(m);
    if (m.free_ring) k_free_clamp<<<1, 32, 0, s>>>(m.counters);
  }
  if (n > 0) k_import_write<<<num_sms * 4, 256, 0, s>>>(m, coords, vox, n);
}

void launch_export(const MapView& m, int64_t cap, int32_t* coords, float* vox, int num_sms, cudaStream_t s) {
  k_export<<<num_sms * 4, 256, 0, s>>>(m, cap, coords, vox);
}

}  // namespace dtsdf
