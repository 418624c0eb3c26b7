// Direct ray-cast rendering of the Directional TSDF (Sec. 4).
//
// One thread per pixel. The ray is probed at regular intervals, on a global grid of
// samples t_k = k h/2 from z_min to z_max (Sec. 4: regular probing until the SDF turns
// negative, then small SDF-sized steps). Per block cell the hash is probed once; the
// directory entry gives the bricks of all six directions, and cells with no allocated
// direction are skipped whole (no sample in them can be defined). At a sample, the
// combined SDF Phi of Eq. combine_weight is a convex combination of the present
// directions' trilinear values Phi^D, so its sign follows from min/max of those alone
// whenever they agree (8 voxel reads per direction); the full combination with
// central-difference gradients (32 voxel reads per direction) is computed only where
// the signs disagree and for the outputs. The reported crossing is the first pair of
// consecutive defined samples with Phi > 0 >= Phi; it is refined by two scans of 8
// regular sub-steps to the first sign change and linear interpolation over the final
// h/128-wide bracket.
#include <math.h>

#include "internal.h"

namespace dtsdf {

constexpr int RT_X = 16, RT_Y = 8, RT_N = RT_X * RT_Y;
constexpr int UNPROBED = -2;

struct RenderArgs {
  Intr K;
  Pose32 T;        // camera -> world
  float* depth;
  float4* normals;
  float4* color;
  int max_samples;
};

// Per-thread cache of the directory indices of the 27 blocks around the current cell,
// held in shared memory (transposed so a warp's accesses are conflict free).
struct NbCache {
  int* s;
  int cx, cy, cz;
  __device__ __forceinline__ void reset(int x, int y, int z) {
    cx = x;
    cy = y;
    cz = z;
#pragma unroll
    for (int j = 0; j < 27; ++j) s[j * RT_N] = UNPROBED;
  }
  __device__ __forceinline__ int dir(const MapView& m, int dx, int dy, int dz) {
    if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) return hash_find(m, cx + dx, cy + dy, cz + dz);
    const int j = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
    int v = s[j * RT_N];
    if (v == UNPROBED) {
      v = hash_find(m, cx + dx, cy + dy, cz + dz);
      s[j * RT_N] = v;
    }
    return v;
  }
};

template <int STORE>
__device__ __forceinline__ float2 ld_geom(const MapView& m, size_t i) {
  if (STORE == DTSDF_STORE_FP16) return unpack_geom16(__ldg(m.geom16 + i));
  return __ldg(m.geom + i);
}

// Voxel (gx, gy, gz) of direction D; false if its brick is absent or its weight is 0.
template <int STORE>
__device__ __forceinline__ bool voxel(const MapView& m, NbCache& c, int D, int gx, int gy, int gz, float2& out) {
  const int bx = gx >> 3, by = gy >> 3, bz = gz >> 3;
  const int d = c.dir(m, bx - c.cx, by - c.cy, bz - c.cz);
  if (d < 0) return false;
  const int slot = __ldg(m.dir_slots + (size_t)d * 8 + D);
  if (slot < 0) return false;
  out = ld_geom<STORE>(m, (size_t)slot * BVOX + ((gz & 7) * 8 + (gy & 7)) * 8 + (gx & 7));
  return out.y > 0.0f;
}

__device__ __forceinline__ float tri(const float v[8], float fx, float fy, float fz) {
  const float a = v[0] + fx * (v[1] - v[0]);
  const float b = v[2] + fx * (v[3] - v[2]);
  const float c = v[4] + fx * (v[5] - v[4]);
  const float d = v[6] + fx * (v[7] - v[6]);
  const float e = a + fy * (b - a);
  const float f = c + fy * (d - c);
  return e + fz * (f - e);
}

// The 8 trilinear corners (corner c = (c&1, c>>1&1, c>>2&1)) of direction D at base voxel g.
template <int STORE>
__device__ __forceinline__ bool corners(const MapView& m, NbCache& c, int D, int g0, int g1, int g2, float sdf[8],
                                        float w[8]) {
  const int l0 = g0 & 7, l1 = g1 & 7, l2 = g2 & 7;
  if (l0 < 7 && l1 < 7 && l2 < 7 && (g0 >> 3) == c.cx && (g1 >> 3) == c.cy && (g2 >> 3) == c.cz) {
    // all corners inside the current cell's brick
    const int d = c.dir(m, 0, 0, 0);
    const int slot = __ldg(m.dir_slots + (size_t)d * 8 + D);
    if (slot < 0) return false;
    const size_t base = (size_t)slot * BVOX + (l2 * 8 + l1) * 8 + l0;
    bool ok = true;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float2 v = ld_geom<STORE>(m, base + ((q >> 2) & 1) * 64 + ((q >> 1) & 1) * 8 + (q & 1));
      sdf[q] = v.x;
      w[q] = v.y;
      ok &= v.y > 0.0f;
    }
    return ok;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float2 v;
    if (!voxel<STORE>(m, c, D, g0 + (q & 1), g1 + ((q >> 1) & 1), g2 + ((q >> 2) & 1), v)) return false;
    sdf[q] = v.x;
    w[q] = v.y;
  }
  return true;
}

__device__ __forceinline__ float w_dir_r(float c, float theta) {
  const float alpha = acosf(fminf(fmaxf(c, -1.0f), 1.0f));
  return fminf(fmaxf((theta - alpha) / (2.0f * theta - 1.57079632679489662f), 0.0f), 1.0f);
}

struct Combined {
  int defined;   // 0 undefined, 1 defined
  float phi;
  float wsum;    // sum of combination weights (0 when the fallback was used)
  float n[3];    // sum of w_comb n^D (world)
  float rgb[3];
  float cw;      // sum of w_comb over directions with colour
};

// Full combination of Eq. combine_weight at voxel coordinate g (fallback Eq. combine_tsdf_weight).
template <int STORE, bool COLOR>
__device__ Combined combine_full(const MapView& m, NbCache& c, uint32_t dmask, const float g[3], const float r[3]) {
  Combined out;
  out.defined = 0;
  out.phi = 0.f;
  out.wsum = 0.f;
  out.n[0] = out.n[1] = out.n[2] = 0.f;
  out.rgb[0] = out.rgb[1] = out.rgb[2] = 0.f;
  out.cw = 0.f;
  const float f0 = floorf(g[0]), f1 = floorf(g[1]), f2 = floorf(g[2]);
  const int g0 = (int)f0, g1 = (int)f1, g2 = (int)f2;
  const float fx = g[0] - f0, fy = g[1] - f1, fz = g[2] - f2;
  float acc = 0.f, facc = 0.f, fw = 0.f;
  bool any = false;
  const float inv2h = 0.5f / m.h;
#pragma unroll 1
  for (int D = 0; D < ND; ++D) {
    if (!(dmask & (1u << D))) continue;
    float s[8], w[8];
    if (!corners<STORE>(m, c, D, g0, g1, g2, s, w)) continue;
    any = true;
    const float phiD = tri(s, fx, fy, fz);
    const float WD = tri(w, fx, fy, fz);
    // fallback weight W^D max(0, <v^D, -r>)
    const float vr = (D & 1) ? r[D >> 1] : -r[D >> 1];
    const float wf = WD * fmaxf(vr, 0.0f);
    fw += wf;
    facc += wf * phiD;
    // central differences of the trilinear field at +-h along each axis
    float grad[3];
    bool gok = true;
#pragma unroll
    for (int a = 0; a < 3 && gok; ++a) {
      float sp[8], wp[8], sm[8], wm[8];
      const int p0 = g0 + (a == 0), p1 = g1 + (a == 1), p2 = g2 + (a == 2);
      const int m0 = g0 - (a == 0), m1 = g1 - (a == 1), m2 = g2 - (a == 2);
      if (!corners<STORE>(m, c, D, p0, p1, p2, sp, wp) || !corners<STORE>(m, c, D, m0, m1, m2, sm, wm)) {
        gok = false;
        break;
      }
      grad[a] = (tri(sp, fx, fy, fz) - tri(sm, fx, fy, fz)) * inv2h;
    }
    if (!gok) continue;
    const float gn = sqrtf(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]);
    if (!(gn > 1e-12f)) continue;
    const float n0 = grad[0] / gn, n1 = grad[1] / gn, n2 = grad[2] / gn;
    const float nD[3] = {n0, n1, n2};
    const float cosv = (D & 1) ? -nD[D >> 1] : nD[D >> 1];
    const float facing = fmaxf(-(n0 * r[0] + n1 * r[1] + n2 * r[2]), 0.0f);
    const float wc = w_dir_r(cosv, m.theta) * facing * WD;
    if (!(wc > 0.0f)) continue;
    out.wsum += wc;
    acc += wc * phiD;
    out.n[0] += wc * n0;
    out.n[1] += wc * n1;
    out.n[2] += wc * n2;
    if (COLOR) {
      // trilinear colour of the 8 corners; contributes where the trilinear colour weight > 0
      const int gq[3] = {g0, g1, g2};
      float cr[8], cg[8], cb[8], cwt[8];
      bool cok = true;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int x0 = gq[0] + (q & 1), x1 = gq[1] + ((q >> 1) & 1), x2 = gq[2] + ((q >> 2) & 1);
        const int d = c.dir(m, (x0 >> 3) - c.cx, (x1 >> 3) - c.cy, (x2 >> 3) - c.cz);
        const int slot = d >= 0 ? __ldg(m.dir_slots + (size_t)d * 8 + D) : -1;
        if (slot < 0) {
          cok = false;
          break;
        }
        const size_t vi = (size_t)slot * BVOX + ((x2 & 7) * 8 + (x1 & 7)) * 8 + (x0 & 7);
        if (STORE == DTSDF_STORE_FP16) {
          const uint32_t cv = __ldg(m.col8 + vi);
          cr[q] = (float)(cv & 0xFF);
          cg[q] = (float)((cv >> 8) & 0xFF);
          cb[q] = (float)((cv >> 16) & 0xFF);
          cwt[q] = (float)(cv >> 24);
        } else {
          const float4 cv = __ldg(m.col + vi);
          cr[q] = cv.x;
          cg[q] = cv.y;
          cb[q] = cv.z;
          cwt[q] = cv.w;
        }
      }
      if (cok && tri(cwt, fx, fy, fz) > 0.0f) {
        out.cw += wc;
        out.rgb[0] += wc * tri(cr, fx, fy, fz);
        out.rgb[1] += wc * tri(cg, fx, fy, fz);
        out.rgb[2] += wc * tri(cb, fx, fy, fz);
      }
    }
  }
  if (!any) return out;
  if (out.wsum > 0.0f) {
    out.defined = 1;
    out.phi = acc / out.wsum;
  } else if (fw > 0.0f) {
    out.defined = 1;
    out.phi = facc / fw;
  }
  return out;
}

// Sign of Phi from the present directions' trilinear values.
// Returns 0 undefined, 1 positive, -1 non-positive, 2 undecided (needs the full combination).
template <int STORE>
__device__ __forceinline__ int sign_fast(const MapView& m, NbCache& c, uint32_t dmask, const float g[3],
                                         const float r[3], float& lo) {
  const float f0 = floorf(g[0]), f1 = floorf(g[1]), f2 = floorf(g[2]);
  const int g0 = (int)f0, g1 = (int)f1, g2 = (int)f2;
  const float fx = g[0] - f0, fy = g[1] - f1, fz = g[2] - f2;
  float mn = 2.f, mx = -2.f;
  bool any = false, facing = false;
#pragma unroll 1
  for (int D = 0; D < ND; ++D) {
    if (!(dmask & (1u << D))) continue;
    float s[8], w[8];
    if (!corners<STORE>(m, c, D, g0, g1, g2, s, w)) continue;
    const float phiD = tri(s, fx, fy, fz);
    any = true;
    mn = fminf(mn, phiD);
    mx = fmaxf(mx, phiD);
    const float vr = (D & 1) ? r[D >> 1] : -r[D >> 1];
    facing |= vr > 0.0f;
  }
  lo = mn;
  if (!any) return 0;
  if (!facing) return 2;
  if (mn > 0.0f) return 1;
  if (mx <= 0.0f) return -1;
  return 2;
}

template <int STORE, bool COLOR>
__global__ void __launch_bounds__(RT_N) k_render(MapView m, RenderArgs a) {
  __shared__ int s_cache[27 * RT_N];
  const int tid = threadIdx.y * RT_X + threadIdx.x;
  const int u = blockIdx.x * RT_X + threadIdx.x;
  const int v = blockIdx.y * RT_Y + threadIdx.y;
  if (u >= a.K.W || v >= a.K.H) return;
  const int pix = v * a.K.W + u;
  NbCache cache;
  cache.s = s_cache + tid;
  cache.cx = cache.cy = cache.cz = 0x7fffffff;

  // unit ray in camera and world frame
  const float rc0 = (u - a.K.cx) / a.K.fx, rc1 = (v - a.K.cy) / a.K.fy;
  const float rl = sqrtf(rc0 * rc0 + rc1 * rc1 + 1.0f);
  const float q0 = rc0 / rl, q1 = rc1 / rl, q2 = 1.0f / rl;
  float r[3];
  r[0] = a.T.R[0] * q0 + a.T.R[1] * q1 + a.T.R[2] * q2;
  r[1] = a.T.R[3] * q0 + a.T.R[4] * q1 + a.T.R[5] * q2;
  r[2] = a.T.R[6] * q0 + a.T.R[7] * q1 + a.T.R[8] * q2;
  const float o[3] = {a.T.t[0], a.T.t[1], a.T.t[2]};
  const float org[3] = {m.ox, m.oy, m.oz};
  const float inv_h = 1.0f / m.h;
  const float step = 0.5f * m.h;
  const int k0 = (int)ceilf(m.zmin * rl / step);
  const int k1 = (int)floorf(m.zmax * rl / step);
  const float bsz = 8.0f * m.h;

  uint32_t cmask = 0;
  bool prev_def = false;
  float prev_phi = 0.f;
  int hit_k = -1;
  int k = k0;
  for (int it = 0; it < a.max_samples && k <= k1; ++it) {
    const float t = (float)k * step;
    float g[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) g[q] = (o[q] + t * r[q] - org[q]) * inv_h;
    const int cx = ((int)floorf(g[0])) >> 3, cy = ((int)floorf(g[1])) >> 3, cz = ((int)floorf(g[2])) >> 3;
    if (cx != cache.cx || cy != cache.cy || cz != cache.cz) {
      cache.reset(cx, cy, cz);
      const int d0 = cache.dir(m, 0, 0, 0);
      cmask = d0 >= 0 ? (uint32_t)__ldg(m.dir_slots + (size_t)d0 * 8 + SLOT_MASK) : 0u;
    }
    if (cmask == 0) {
      // no direction allocated in this cell: no sample in it can be defined; jump past it
      float tex = 3.4e38f;
      const int cc[3] = {cx, cy, cz};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (r[q] > 0.f)
          tex = fminf(tex, (org[q] + (cc[q] + 1) * bsz - o[q]) / r[q]);
        else if (r[q] < 0.f)
          tex = fminf(tex, (org[q] + cc[q] * bsz - o[q]) / r[q]);
      }
      const int kn = (int)ceilf(tex / step);
      prev_def = false;
      k = max(k + 1, kn);
      continue;
    }
    float lo = 0.f;
    int sg = sign_fast<STORE>(m, cache, cmask, g, r, lo);
    if (sg == 2) {
      const Combined cb = combine_full<STORE, false>(m, cache, cmask, g, r);
      sg = cb.defined ? (cb.phi > 0.f ? 1 : -1) : 0;
      lo = cb.phi;
    }
    if (sg == 0) {
      prev_def = false;
      ++k;
      continue;
    }
    if (sg < 0 && prev_def && prev_phi > 0.f) {
      hit_k = k;
      break;
    }
    prev_def = true;
    prev_phi = sg > 0 ? lo : -1.f;
    ++k;
  }

  float out_depth = 0.f;
  float4 out_n = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 out_c = make_float4(0.f, 0.f, 0.f, 0.f);
  if (hit_k >= 0) {
    // bracket [t_a, t_b] with Phi(t_a) > 0 >= Phi(t_b)
    float ta = (float)(hit_k - 1) * step, tb = (float)hit_k * step;
    auto eval = [&](float t) -> Combined {
      float g[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) g[q] = (o[q] + t * r[q] - org[q]) * inv_h;
      const int cx = ((int)floorf(g[0])) >> 3, cy = ((int)floorf(g[1])) >> 3, cz = ((int)floorf(g[2])) >> 3;
      if (cx != cache.cx || cy != cache.cy || cz != cache.cz) {
        cache.reset(cx, cy, cz);
        const int d0 = cache.dir(m, 0, 0, 0);
        cmask = d0 >= 0 ? (uint32_t)__ldg(m.dir_slots + (size_t)d0 * 8 + SLOT_MASK) : 0u;
      }
      Combined cb;
      if (cmask == 0) {
        cb.defined = 0;
        cb.wsum = 0.f;
        return cb;
      }
      return combine_full<STORE, false>(m, cache, cmask, g, r);
    };
    // small regular steps: two scans of 8 sub-steps keep the first sub-interval where
    // Phi turns <= 0 (an undefined probe counts as free space); sign tests only
#pragma unroll 1
    for (int lvl = 0; lvl < 2; ++lvl) {
      const float a0 = ta, dt = (tb - ta) * 0.125f;
      float prev = ta;
#pragma unroll 1
      for (int j = 1; j < 8; ++j) {
        const float tj = a0 + (float)j * dt;
        float g[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) g[q] = (o[q] + tj * r[q] - org[q]) * inv_h;
        const int cx = ((int)floorf(g[0])) >> 3, cy = ((int)floorf(g[1])) >> 3, cz = ((int)floorf(g[2])) >> 3;
        if (cx != cache.cx || cy != cache.cy || cz != cache.cz) {
          cache.reset(cx, cy, cz);
          const int d0 = cache.dir(m, 0, 0, 0);
          cmask = d0 >= 0 ? (uint32_t)__ldg(m.dir_slots + (size_t)d0 * 8 + SLOT_MASK) : 0u;
        }
        int sg = 0;
        if (cmask) {
          float lo;
          sg = sign_fast<STORE>(m, cache, cmask, g, r, lo);
          if (sg == 2) {
            const Combined cb = combine_full<STORE, false>(m, cache, cmask, g, r);
            sg = cb.defined ? (cb.phi > 0.f ? 1 : -1) : 0;
          }
        }
        if (sg < 0) {
          tb = tj;
          break;
        }
        prev = tj;
      }
      ta = prev;
    }
    // root: linear interpolation of Phi over the final bracket
    const Combined A = eval(ta), B = eval(tb);
    float ts = 0.5f * (ta + tb);
    if (A.defined && A.phi > 0.f && B.defined && B.phi <= 0.f) ts = ta + (tb - ta) * A.phi / (A.phi - B.phi);
    // normal and colour at the first grid sample behind the crossing (the sample that
    // decided the hit), else at the sample in front of it, else at the refined root
    const float ends[3] = {(float)hit_k * step, (float)(hit_k - 1) * step, ts};
#pragma unroll 1
    for (int e = 0; e < 3; ++e) {
      float g[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) g[q] = (o[q] + ends[e] * r[q] - org[q]) * inv_h;
      const int cx = ((int)floorf(g[0])) >> 3, cy = ((int)floorf(g[1])) >> 3, cz = ((int)floorf(g[2])) >> 3;
      if (cx != cache.cx || cy != cache.cy || cz != cache.cz) {
        cache.reset(cx, cy, cz);
        const int d0 = cache.dir(m, 0, 0, 0);
        cmask = d0 >= 0 ? (uint32_t)__ldg(m.dir_slots + (size_t)d0 * 8 + SLOT_MASK) : 0u;
      }
      if (!cmask) continue;
      const Combined H = combine_full<STORE, COLOR>(m, cache, cmask, g, r);
      const float nl = sqrtf(H.n[0] * H.n[0] + H.n[1] * H.n[1] + H.n[2] * H.n[2]);
      if (!(H.defined && H.wsum > 0.f && nl > 0.f)) continue;
      const float n0 = H.n[0] / nl, n1 = H.n[1] / nl, n2 = H.n[2] / nl;
      // world -> camera: R^T n
      const float c0 = a.T.R[0] * n0 + a.T.R[3] * n1 + a.T.R[6] * n2;
      const float c1 = a.T.R[1] * n0 + a.T.R[4] * n1 + a.T.R[7] * n2;
      const float c2 = a.T.R[2] * n0 + a.T.R[5] * n1 + a.T.R[8] * n2;
      out_depth = ts / rl;
      out_n = make_float4(c0, c1, c2, out_depth);
      if (COLOR && H.cw > 0.f) out_c = make_float4(H.rgb[0] / H.cw, H.rgb[1] / H.cw, H.rgb[2] / H.cw, 1.0f);
      break;
    }
  }
  a.depth[pix] = out_depth;
  a.normals[pix] = out_n;
  if (COLOR && a.color) a.color[pix] = out_c;
}

void launch_render(const MapView& m, const Intr& K, const Pose32& T, float* depth, float4* normals, float4* color,
                   cudaStream_t s) {
  RenderArgs a;
  a.K = K;
  a.T = T;
  a.depth = depth;
  a.normals = normals;
  a.color = color;
  a.max_samples = 1 << 16;
  dim3 blk(RT_X, RT_Y), grd((K.W + RT_X - 1) / RT_X, (K.H + RT_Y - 1) / RT_Y);
  const bool col = m.color && color;
  if (m.storage == DTSDF_STORE_FP16) {
    if (col)
      k_render<DTSDF_STORE_FP16, true><<<grd, blk, 0, s>>>(m, a);
    else
      k_render<DTSDF_STORE_FP16, false><<<grd, blk, 0, s>>>(m, a);
  } else {
    if (col)
      k_render<DTSDF_STORE_FP32, true><<<grd, blk, 0, s>>>(m, a);
    else
      k_render<DTSDF_STORE_FP32, false><<<grd, blk, 0, s>>>(m, a);
  }
}

}  // namespace dtsdf
