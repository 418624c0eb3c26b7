// Free-space combination render (Sec. 4, Alg. 1 "Compute Combined TSDF"): the quality
// reference mode that decides, per sample of the view ray, whether the point is free or
// occupied before combining the directions, instead of the weighting of Eq. combine_weight.
//
// At a point p on the ray from the camera centre c with unit direction r, a direction D takes
// part where its trilinear field is present, unless it has a gradient whose normal lies outside
// the direction's angular range (w_dir = 0): the paper's first implementation remark drops
// information whose gradient does not belong to the direction, while a flat (truncated) field
// keeps its free-space or interior information. Among those, F holds
// the directions with Phi^D(p) > 0 and O those with Phi^D(p) <= 0. p is free space if some D in F
// has no zero transition of Phi^D between p and the camera, or if at its first such transition q
// (walking from p toward c) no taking-part direction D~ has Phi^D~(q) < 0 with a normal facing the
// camera (<n^D~(q), -r> > 0; a gradient is needed). The value is the fused-weight average of Phi^D over F when p is free
// space, else over O; undefined when that set is empty.
//
// The march samples t_k = k h/2 as the direct render does. Walking back from a grid sample over
// the grid finds the latest transition among the sample pairs behind it, so the march keeps, per
// direction, whether a transition (Phi^D <= 0 at t_{k-1}, > 0 at t_k, both present) was seen and
// whether its point q (the linear root in that pair) was blocked. A refinement point p between
// t_{k-1} and t_k first checks the pair (t_{k-1}, p), then falls back to the state at t_{k-1}.
// The crossing is refined as in the direct render (bisection on the sign of the value, linear
// root of the final bracket) and the normal is the normalised fused-weight sum of the chosen
// set's normals at the final bracket's non-positive end; a miss where that sum vanishes. No
// colour.
#include "internal.h"

namespace dtsdf {

namespace {

constexpr int FS_THREADS = 128;

template <int STORE>
__device__ __forceinline__ float2 fs_ld(const MapView& m, size_t i) {
  if (STORE == DTSDF_STORE_FP16) return unpack_geom16(__ldg(m.geom16 + i));
  return __ldg(m.geom + i);
}

__host__ __device__ __forceinline__ constexpr int fs_coff(int q) {
  return (q & 1) + PAD * ((q >> 1) & 1) + PAD * PAD * (q >> 2);
}

__device__ __forceinline__ float fs_lerp(float a, float b, float t) { return __fmaf_rn(t, b - a, a); }

__device__ __forceinline__ float fs_tri(const float* v, float fx, float fy, float fz) {
  const float s00 = fs_lerp(v[0], v[1], fx), s10 = fs_lerp(v[2], v[3], fx);
  const float s01 = fs_lerp(v[4], v[5], fx), s11 = fs_lerp(v[6], v[7], fx);
  return fs_lerp(fs_lerp(s00, s10, fy), fs_lerp(s01, s11, fy), fz);
}

__device__ __forceinline__ float fs_wdir(float c, const MapView& m) {
  if (c >= m.sinth) return 1.0f;
  if (c <= m.costh) return 0.0f;
  const float alpha = acosf(c);
  return fminf(fmaxf((m.theta - alpha) / (2.0f * m.theta - 1.57079632679489662f), 0.0f), 1.0f);
}

// Per-direction sample: trilinear value and fused weight (all 8 corners weighted), and the
// normal of the central-difference gradient at +-1 voxel (all 24 further taps weighted).
struct DirSample {
  float phi, W, n[3];
  bool part;  // takes part: present, and no gradient or a normal within the direction's range
  bool grad;
};

// Brick slots of the six directions in block cell (x, y, z); returns the allocated mask.
__device__ uint32_t fs_cell(const MapView& m, int x, int y, int z, int slot[6]) {
  const unsigned long long k = pack_block(x, y, z);
  uint32_t i = hash_slot(k, m.hmask);
  uint32_t v = VAL_EMPTY;
#pragma unroll 1
  for (int p = 0; p < MAX_PROBE; ++p) {
    const unsigned long long kk = __ldg(m.keys + i);
    if (kk == k) {
      v = __ldg(m.vals + i);
      break;
    }
    if (kk == EMPTY_KEY) break;
    i = (i + 1) & m.hmask;
  }
  const int d = val_dir(v);
  uint32_t mask = 0;
#pragma unroll
  for (int D = 0; D < 6; ++D) {
    slot[D] = -1;
    if (d >= 0 && ((val_mask(v) >> D) & 1u)) {
      slot[D] = __ldg(m.dir_slots + (size_t)d * 8 + D);
      if (slot[D] >= 0) mask |= 1u << D;
    }
  }
  return mask;
}

// Samples of every allocated direction at voxel coordinate g (cell (cx, cy, cz) of g).
// Returns the mask of present directions; part flags the ones that take part.
template <int STORE>
__device__ uint32_t fs_sample(const MapView& m, const int slot[6], uint32_t amask, int cx, int cy, int cz,
                              const float g[3], DirSample S[6]) {
  const float f0 = floorf(g[0]), f1 = floorf(g[1]), f2 = floorf(g[2]);
  const int g0 = (int)f0, g1 = (int)f1, g2 = (int)f2;
  const float fx = g[0] - f0, fy = g[1] - f1, fz = g[2] - f2;
  const int lofs = pad_index(g0 - 8 * cx, g1 - 8 * cy, g2 - 8 * cz);
  const float inv2h = 0.5f / m.h;
  uint32_t pres = 0;
#pragma unroll 1
  for (int D = 0; D < 6; ++D) {
    S[D].part = false;
    S[D].grad = false;
    S[D].n[0] = S[D].n[1] = S[D].n[2] = 0.f;
    if (!((amask >> D) & 1u)) continue;
    const size_t base = (size_t)slot[D] * PVOX + lofs;
    float s[8], w[8];
    bool ok = true;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float2 v = fs_ld<STORE>(m, base + fs_coff(q));
      ok &= v.y > 0.0f;
      s[q] = v.x;
      w[q] = v.y;
    }
    if (!ok) continue;
    pres |= 1u << D;
    S[D].part = true;
    S[D].phi = fs_tri(s, fx, fy, fz);
    S[D].W = fs_tri(w, fx, fy, fz);
    bool gok = true;
    float gr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int St = a == 0 ? 1 : (a == 1 ? PAD : PAD * PAD);
      const int bit = 1 << a;
      float dv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float2 t = fs_ld<STORE>(m, (q & bit) ? base + St + fs_coff(q) : base - St + fs_coff(q));
        gok &= t.y > 0.0f;
        dv[q] = (q & bit) ? t.x - s[q & ~bit] : s[q | bit] - t.x;
      }
      gr[a] = fs_tri(dv, fx, fy, fz) * inv2h;
    }
    if (!gok) continue;
    const float gn = sqrtf(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
    if (!(gn > 1e-12f)) continue;
    S[D].grad = true;
    S[D].n[0] = gr[0] / gn;
    S[D].n[1] = gr[1] / gn;
    S[D].n[2] = gr[2] / gn;
    const float cosv = (D & 1) ? -S[D].n[D >> 1] : S[D].n[D >> 1];
    S[D].part = fs_wdir(cosv, m) > 0.0f;
  }
  return pres;
}

struct Ray {
  float o[3], r[3], org[3], inv_h;
};

__device__ __forceinline__ void fs_point(const Ray& R, float t, float g[3]) {
#pragma unroll
  for (int q = 0; q < 3; ++q) g[q] = (R.o[q] + t * R.r[q] - R.org[q]) * R.inv_h;
}

// Is the transition point at ray parameter tq inside the occupied space of a visible surface?
template <int STORE>
__device__ bool fs_blocked(const MapView& m, const Ray& R, float tq) {
  float g[3];
  fs_point(R, tq, g);
  const int cx = ((int)floorf(g[0])) >> 3, cy = ((int)floorf(g[1])) >> 3, cz = ((int)floorf(g[2])) >> 3;
  int slot[6];
  const uint32_t am = fs_cell(m, cx, cy, cz, slot);
  if (!am) return false;
  DirSample S[6];
  fs_sample<STORE>(m, slot, am, cx, cy, cz, g, S);
#pragma unroll 1
  for (int D = 0; D < 6; ++D) {
    if (!S[D].part || !S[D].grad || !(S[D].phi < 0.0f)) continue;
    const float f = -(S[D].n[0] * R.r[0] + S[D].n[1] * R.r[1] + S[D].n[2] * R.r[2]);
    if (f > 0.0f) return true;
  }
  return false;
}

struct Value {
  bool defined;
  float phi;
  float n[3];  // fused-weight sum of the chosen set's normals (world)
};

// Alg. 1 at a point with direction samples S; hasq / blk: per direction, a transition was
// found walking back from the point / its point is blocked.
__device__ Value fs_value(const DirSample S[6], uint32_t pres, uint32_t hasq, uint32_t blk) {
  uint32_t F = 0, O = 0;
#pragma unroll
  for (int D = 0; D < 6; ++D) {
    if (!((pres >> D) & 1u) || !S[D].part) continue;
    if (S[D].phi > 0.0f)
      F |= 1u << D;
    else
      O |= 1u << D;
  }
  const bool free_space = (F & ~(hasq & blk)) != 0;
  const uint32_t set = free_space ? F : O;
  Value v;
  v.defined = false;
  v.phi = 0.f;
  v.n[0] = v.n[1] = v.n[2] = 0.f;
  if (!set) return v;
  float ws = 0.f, acc = 0.f, n0 = 0.f, n1 = 0.f, n2 = 0.f;
#pragma unroll
  for (int D = 0; D < 6; ++D) {
    if (!((set >> D) & 1u)) continue;
    ws += S[D].W;
    acc += S[D].W * S[D].phi;
    n0 += S[D].W * S[D].n[0];
    n1 += S[D].W * S[D].n[1];
    n2 += S[D].W * S[D].n[2];
  }
  if (!(ws > 0.0f)) return v;
  v.defined = true;
  v.phi = acc / ws;
  v.n[0] = n0;
  v.n[1] = n1;
  v.n[2] = n2;
  return v;
}

// Alg. 1 at a refinement point at parameter t (t_{k-1} < t < t_k), given the march state at
// t_{k-1}: the previous samples and the transition flags.
template <int STORE>
__device__ Value fs_subpoint(const MapView& m, const Ray& R, float t, float tprev, const float* pphi, uint32_t ppres,
                             uint32_t hasq, uint32_t blk) {
  float g[3];
  fs_point(R, t, g);
  const int cx = ((int)floorf(g[0])) >> 3, cy = ((int)floorf(g[1])) >> 3, cz = ((int)floorf(g[2])) >> 3;
  int slot[6];
  const uint32_t am = fs_cell(m, cx, cy, cz, slot);
  Value none;
  none.defined = false;
  none.phi = 0.f;
  none.n[0] = none.n[1] = none.n[2] = 0.f;
  if (!am) return none;
  DirSample S[6];
  const uint32_t pres = fs_sample<STORE>(m, slot, am, cx, cy, cz, g, S);
#pragma unroll 1
  for (int D = 0; D < 6; ++D) {
    if (((ppres & pres) >> D) & 1u) {
      if (pphi[D] <= 0.0f && S[D].phi > 0.0f) {
        const float tq = tprev + (t - tprev) * (-pphi[D] / (S[D].phi - pphi[D]));
        hasq |= 1u << D;
        if (fs_blocked<STORE>(m, R, tq))
          blk |= 1u << D;
        else
          blk &= ~(1u << D);
      }
    }
  }
  return fs_value(S, pres, hasq, blk);
}

template <int STORE>
__global__ void __launch_bounds__(FS_THREADS) k_render_freespace(MapView m, Intr K, Pose32 T, const double* Tdev,
                                                                 float* depth, float4* normals, float4* color) {
  const int pix = blockIdx.x * FS_THREADS + threadIdx.x;
  if (pix >= K.W * K.H) return;
  if (Tdev) T = pose_from_device(Tdev);
  const int u = pix % K.W, v = pix / K.W;
  const float rc0 = (u - K.cx) / K.fx, rc1 = (v - K.cy) / K.fy;
  const float rl = sqrtf(rc0 * rc0 + rc1 * rc1 + 1.0f);
  const float q0 = rc0 / rl, q1 = rc1 / rl, q2 = 1.0f / rl;
  Ray R;
  R.r[0] = T.R[0] * q0 + T.R[1] * q1 + T.R[2] * q2;
  R.r[1] = T.R[3] * q0 + T.R[4] * q1 + T.R[5] * q2;
  R.r[2] = T.R[6] * q0 + T.R[7] * q1 + T.R[8] * q2;
  R.o[0] = T.t[0];
  R.o[1] = T.t[1];
  R.o[2] = T.t[2];
  R.org[0] = m.ox;
  R.org[1] = m.oy;
  R.org[2] = m.oz;
  R.inv_h = 1.0f / m.h;
  const float step = 0.5f * m.h;
  const int k0 = (int)ceilf(m.zmin * rl / step), k1 = (int)floorf(m.zmax * rl / step);
  // march state
  float pphi[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  uint32_t ppres = 0, hasq = 0, blk = 0;
  bool prev_def = false;
  Value prev_val;
  prev_val.defined = false;
  int ccx = 0x7fffffff, ccy = 0, ccz = 0;
  int slot[6];
  uint32_t am = 0;
  float out_depth = 0.f;
  float4 out_n = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
  for (int k = k0; k <= k1; ++k) {
    const float t = (float)k * step;
    float g[3];
    fs_point(R, t, g);
    const int cx = ((int)floorf(g[0])) >> 3, cy = ((int)floorf(g[1])) >> 3, cz = ((int)floorf(g[2])) >> 3;
    if (cx != ccx || cy != ccy || cz != ccz) {
      ccx = cx;
      ccy = cy;
      ccz = cz;
      am = fs_cell(m, cx, cy, cz, slot);
    }
    if (!am) {  // no brick: every direction absent here
      ppres = 0;
      prev_def = false;
      continue;
    }
    DirSample S[6];
    const uint32_t pres = fs_sample<STORE>(m, slot, am, cx, cy, cz, g, S);
    const uint32_t hasq0 = hasq, blk0 = blk;
    const float tprev = (float)(k - 1) * step;
#pragma unroll 1
    for (int D = 0; D < 6; ++D) {
      if ((((ppres & pres) >> D) & 1u) && pphi[D] <= 0.0f && S[D].phi > 0.0f) {
        const float tq = tprev + step * (-pphi[D] / (S[D].phi - pphi[D]));
        hasq |= 1u << D;
        if (fs_blocked<STORE>(m, R, tq))
          blk |= 1u << D;
        else
          blk &= ~(1u << D);
      }
    }
    const Value cur = fs_value(S, pres, hasq, blk);
    if (prev_def && cur.defined && prev_val.phi > 0.0f && cur.phi <= 0.0f) {
      // the root in [t_{k-1}, t_k]: bisection (an undefined point counts as free space), then
      // the linear root of the final bracket
      float lo = tprev, hi = t;
      Value vlo = prev_val, vhi = cur;
#pragma unroll 1
      for (int j = 0; j < REFINE_HALVINGS; ++j) {
        const float tm = 0.5f * (lo + hi);
        const Value vm = fs_subpoint<STORE>(m, R, tm, tprev, pphi, ppres, hasq0, blk0);
        if (vm.defined && vm.phi <= 0.0f) {
          hi = tm;
          vhi = vm;
        } else {
          lo = tm;
          vlo = vm;
        }
      }
      const bool da = vlo.defined && vlo.phi > 0.0f, db = vhi.defined && vhi.phi <= 0.0f;
      const float ts = (da && db) ? lo + (hi - lo) * (vlo.phi / (vlo.phi - vhi.phi)) : 0.5f * (lo + hi);
      // normal at the root's non-positive side (the final bracket's end hi)
      const float* nn = nullptr;
      const Value vr = fs_subpoint<STORE>(m, R, hi, tprev, pphi, ppres, hasq0, blk0);
      if (vr.defined && (vr.n[0] != 0.f || vr.n[1] != 0.f || vr.n[2] != 0.f)) nn = vr.n;
      if (nn) {
        const float ln = sqrtf(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        const float w0 = nn[0] / ln, w1 = nn[1] / ln, w2 = nn[2] / ln;
        out_depth = ts / rl;
        out_n = make_float4(T.R[0] * w0 + T.R[3] * w1 + T.R[6] * w2, T.R[1] * w0 + T.R[4] * w1 + T.R[7] * w2,
                            T.R[2] * w0 + T.R[5] * w1 + T.R[8] * w2, out_depth);
      }
      break;
    }
#pragma unroll
    for (int D = 0; D < 6; ++D) pphi[D] = S[D].phi;
    ppres = pres;
    prev_def = cur.defined;
    prev_val = cur;
  }
  depth[pix] = out_depth;
  normals[pix] = out_n;
  if (color) color[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace

cudaError_t launch_render_freespace(const MapView& m, const Intr& K, const Pose32& T, const double* Tdev, float* depth,
                                    float4* normals, float4* color, cudaStream_t s) {
  const int n = K.W * K.H;
  if (n <= 0) return cudaSuccess;
  const int blocks = (n + FS_THREADS - 1) / FS_THREADS;
  if (m.storage == DTSDF_STORE_FP16)
    k_render_freespace<DTSDF_STORE_FP16><<<blocks, FS_THREADS, 0, s>>>(m, K, T, Tdev, depth, normals, color);
  else
    k_render_freespace<DTSDF_STORE_FP32><<<blocks, FS_THREADS, 0, s>>>(m, K, T, Tdev, depth, normals, color);
  return cudaGetLastError();
}

}  // namespace dtsdf
