// Direct ray-cast rendering of the Directional TSDF (Sec. 4).
//
// One thread per pixel. The ray is probed at regular intervals, on a global grid of
// samples t_k = k h/2 from z_min to z_max (Sec. 4: regular probing until the SDF turns
// negative, then small SDF-sized steps). Per block cell the hash is probed once; the
// directory entry gives the bricks of all six directions, and cells with no allocated
// direction are skipped whole (no sample in them can be defined). Geometry bricks are
// padded with an apron that mirrors the neighbouring blocks, so every voxel a sample in the
// cell reads (trilinear corners and gradient taps) is at a fixed offset from one index. At a sample, the
// combined SDF Phi of Eq. combine_weight is a convex combination of the present
// directions' trilinear values Phi^D, so its sign follows from min/max of those alone
// whenever they agree (8 voxel reads per direction); the full combination with
// central-difference gradients (7 trilinear gathers per direction) is computed only where
// the signs disagree and for the outputs. The reported crossing is the first pair of
// consecutive defined samples with Phi > 0 >= Phi; the hit is the root of Phi(t) in that
// bracket, found by REFINE_HALVINGS bisection steps on the sign of Phi (an undefined point
// counts as free space): the depth is the final bracket's midpoint (h / 2^17 wide, so within
// 2e-8 m of the root at h = 5 mm); normal and colour are evaluated at the bracket's
// non-positive end, where Phi is defined.
// The refinement places its samples from the bracket's first sample computed in double
// precision from the pose, so its positions carry the rounding of a small offset only.
// The per-block occupancy filters let empty space be crossed without probes, and per-brick
// lower bounds let cells whose present directions are all positive be jumped.
#include <math.h>

#include "internal.h"

namespace dtsdf {

constexpr int RT_N = 128;  // threads per CTA of the persistent render grid
#ifndef DTSDF_RENDER_MINB
#define DTSDF_RENDER_MINB 4   // resident CTAs per SM the register allocation is sized for (128 registers, no spills)
#endif

// Out-of-line hash probe over explicit pointers (keeps callers' state in registers).
__device__ __noinline__ uint32_t probe_block(const unsigned long long* __restrict__ keys,
                                             const uint32_t* __restrict__ vals, uint32_t hmask, int bx, int by,
                                             int bz) {
  const unsigned long long k = pack_block(bx, by, bz);
  uint32_t i = hash_slot(k, hmask);
  for (int p = 0; p < MAX_PROBE; ++p) {
    const unsigned long long kk = __ldg(keys + i);
    if (kk == k) return __ldg(vals + i);
    if (kk == EMPTY_KEY) return VAL_EMPTY;
    i = (i + 1) & hmask;
  }
  return VAL_EMPTY;
}

// Per-thread state of the block cell the ray is in. The brick slots of the directions
// allocated in the cell are kept in shared memory (strided by RT_N so a warp's accesses hit
// distinct banks); every voxel that a sample in the cell reads lies in those padded bricks.
struct Cell {
  int* slot;        // 6 brick slots: slot[D * RT_N], valid for the allocated directions
  int cx, cy, cz;
  uint32_t cmask;   // directions allocated in the cell with weighted voxels among [0, 8]^3
  bool positive;    // every active direction's brick bound is > 0
  bool jumped;      // the march already jumped over this cell's positive samples
};

__device__ __forceinline__ void cell_enter(const MapView& m, Cell& c, int x, int y, int z) {
  c.cx = x;
  c.cy = y;
  c.cz = z;
  c.jumped = false;
  const uint32_t v = probe_block(m.keys, m.vals, m.hmask, x, y, z);
  const int d0 = val_dir(v);
  uint32_t active = 0;
  bool positive = true;
#pragma unroll 1
  for (uint32_t mm = val_mask(v); mm; mm &= mm - 1) {
    const int E = __ffs(mm) - 1;
    const int sl = __ldg(m.dir_slots + (size_t)d0 * 8 + E);
    c.slot[E * RT_N] = sl;
    const float lb = sl >= 0 ? __ldg(m.bound + sl) : INFINITY;
    // a bound of +inf: no weighted voxel among the corners, the direction is never present here
    if (lb < INFINITY) active |= 1u << E;
    positive &= lb > 0.0f;
  }
  c.cmask = active;
  c.positive = positive;
}

// COUNT: instrumentation build of the marcher that flags every brick it reads
// (touched[brick] for geometry, touched[pool_cap + brick] for colour); off in normal use.
template <int STORE, bool COUNT>
__device__ __forceinline__ float2 ld_geom(const MapView& m, size_t i, uint8_t* touched) {
  if (COUNT) touched[i / PVOX] = 1;
  if (STORE == DTSDF_STORE_FP16) return unpack_geom16(__ldg(m.geom16 + i));
  return __ldg(m.geom + i);
}

// Offset of trilinear corner q = (q&1, q>>1&1, q>>2&1) in a padded brick.
__host__ __device__ __forceinline__ constexpr int coff(int q) {
  return (q & 1) + PAD * ((q >> 1) & 1) + PAD * PAD * (q >> 2);
}

// Trilinear weight of corner q (colour interpolation).
__device__ __forceinline__ float corner_w(int q, float fx, float fy, float fz) {
  return ((q & 1) ? fx : 1.0f - fx) * ((q & 2) ? fy : 1.0f - fy) * ((q & 4) ? fz : 1.0f - fz);
}

// Trilinear interpolation as nested linear interpolations (x, then y, then z) with explicit
// fused multiply-adds, so a constant field interpolates to exactly its value: the central
// differences of a flat (truncated) region are exactly zero, as in the double-precision
// definition, instead of a rounding residue that would pass the gradient test.
__device__ __forceinline__ float lerp_rn(float a, float b, float t) { return __fmaf_rn(t, b - a, a); }

__device__ __forceinline__ float tri(const float* v, float fx, float fy, float fz) {
  const float s00 = lerp_rn(v[0], v[1], fx), s10 = lerp_rn(v[2], v[3], fx);
  const float s01 = lerp_rn(v[4], v[5], fx), s11 = lerp_rn(v[6], v[7], fx);
  return lerp_rn(lerp_rn(s00, s10, fy), lerp_rn(s01, s11, fy), fz);
}

// Eq. direction_weight as read; the clamped ranges (angle <= pi/2 - theta: 1, >= theta: 0) are
// decided on the cosine (sin theta, cos theta) without the arc cosine; inv_span = 1 / (2 theta - pi/2).
__device__ __forceinline__ float w_dir_r(float c, float theta, float cos_lo, float cos_hi, float inv_span) {
  if (c >= cos_hi) return 1.0f;
  if (c <= cos_lo) return 0.0f;
  const float alpha = acosf(c);
  return fminf(fmaxf((theta - alpha) * inv_span, 0.0f), 1.0f);
}

// component a (0..2) of a 3-vector held in registers, by selects: every index stays in range
// even where the compiler evaluates it ahead of the branch that guards it
__device__ __forceinline__ float ray_comp(const float v[3], int a) { return a == 0 ? v[0] : (a == 1 ? v[1] : v[2]); }

struct Combined {
  int defined;   // 0 undefined, 1 defined
  float phi;
  float wsum;    // sum of combination weights (0 when the fallback was used)
  float n[3];    // sum of w_comb n^D (world)
  float rgb[3];
  float cw;      // sum of w_comb over directions with colour
};

// Colour brick of direction D holding voxel (gx, gy, gz): the cell's brick, else a hash probe
// (colour bricks are unpadded and read only for the outputs).
__device__ __forceinline__ int col_slot(const MapView& m, const Cell& c, int D, int gx, int gy, int gz) {
  const int bx = gx >> 3, by = gy >> 3, bz = gz >> 3;
  if (bx == c.cx && by == c.cy && bz == c.cz) return c.slot[D * RT_N];
  const int d = val_dir(probe_block(m.keys, m.vals, m.hmask, bx, by, bz));
  return d >= 0 ? __ldg(m.dir_slots + (size_t)d * 8 + D) : -1;
}

// Full combination of Eq. combine_weight at voxel coordinate g (fallback Eq. combine_tsdf_weight).
// Per present direction: trilinear value and weight from the 8 corners, and the gradient as
// the central differences (phi(+h) - phi(-h)) / 2h of the trilinear field along each axis,
// whose further 24 taps (4 per side and axis) lie in the same padded brick.
template <int STORE, bool COLOR, bool COUNT>
__device__ __forceinline__ Combined combine_full(const MapView& m, Cell& c, const int gi[3], const float fr[3],
                                                 const float r[3], uint8_t* touched, bool want_color) {
  Combined out;
  out.defined = 0;
  out.phi = 0.f;
  out.wsum = 0.f;
  out.n[0] = out.n[1] = out.n[2] = 0.f;
  out.rgb[0] = out.rgb[1] = out.rgb[2] = 0.f;
  out.cw = 0.f;
  const int g0 = gi[0], g1 = gi[1], g2 = gi[2];
  const float fx = fr[0], fy = fr[1], fz = fr[2];
  const int lofs = pad_index(g0 - 8 * c.cx, g1 - 8 * c.cy, g2 - 8 * c.cz);
  float acc = 0.f, facc = 0.f, fw = 0.f;
  bool any = false;
  const float inv2h = 0.5f / m.h;
  const float inv_span = 1.0f / (2.0f * m.theta - 1.57079632679489662f);
#pragma unroll 1
  for (uint32_t mm = c.cmask; mm; mm &= mm - 1) {
    const int D = __ffs(mm) - 1;
    const size_t base = (size_t)c.slot[D * RT_N] * PVOX + lofs;
    float2 cv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) cv[q] = ld_geom<STORE, COUNT>(m, base + coff(q), touched);
    bool ok = true;
    float s[8], w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      ok &= cv[q].y > 0.0f;
      s[q] = cv[q].x;
      w[q] = cv[q].y;
    }
    if (!ok) continue;
    const float phiD = tri(s, fx, fy, fz);
    const float WD = tri(w, fx, fy, fz);
    any = true;
    // fallback weight W^D max(0, <v^D, -r>)
    const float rc = ray_comp(r, D >> 1);
    const float vr = (D & 1) ? rc : -rc;
    const float wf = WD * fmaxf(vr, 0.0f);
    fw += wf;
    facc += wf * phiD;
    // axis a: phi(+h) - phi(-h) is the trilinear interpolation, with the sample's fractions,
    // of the voxel differences v(c + e_a) - v(c - e_a) at the 8 corners c (the interpolation
    // is linear in the values). Differencing first keeps the gradient accurate in single
    // precision where the field is nearly flat (nearby values subtract exactly), and a flat
    // field still gives exactly zero. For corners with bit a set, c + e_a lies one voxel
    // beyond the base cube and c - e_a is the base corner without bit a; for the others,
    // c + e_a is the base corner with bit a and c - e_a lies one voxel before the cube.
    bool gok = true;
    float gr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int S = a == 0 ? 1 : (a == 1 ? PAD : PAD * PAD);
      const int bit = 1 << a;
      float2 t[8];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        t[q] = ld_geom<STORE, COUNT>(m, (q & bit) ? base + S + coff(q) : base - S + coff(q), touched);
      float dv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        gok &= t[q].y > 0.0f;
        dv[q] = (q & bit) ? t[q].x - s[q & ~bit] : s[q | bit] - t[q].x;
      }
      gr[a] = tri(dv, fx, fy, fz) * inv2h;
    }
    if (!gok) continue;
    const float gg = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
    if (!(gg > 1e-24f)) continue;  // |gradient| > 1e-12
    const float ig = rsqrtf(gg);
    const float n0 = gr[0] * ig, n1 = gr[1] * ig, n2 = gr[2] * ig;
    const float facing = -(n0 * r[0] + n1 * r[1] + n2 * r[2]);
    if (!(facing > 0.0f)) continue;  // the weight of Eq. combine_weight vanishes
    const float cosv = (D == 0) ? n0 : (D == 1) ? -n0 : (D == 2) ? n1 : (D == 3) ? -n1 : (D == 4) ? n2 : -n2;
    const float wc = w_dir_r(cosv, m.theta, m.costh, m.sinth, inv_span) * facing * WD;
    if (!(wc > 0.0f)) continue;
    out.wsum += wc;
    acc += wc * phiD;
    out.n[0] += wc * n0;
    out.n[1] += wc * n1;
    out.n[2] += wc * n2;
    if (COLOR && want_color) {
      // trilinear colour of the 8 corners; contributes where the trilinear colour weight > 0
      float cr = 0.f, cg = 0.f, cb = 0.f, cwt = 0.f;
      bool cok = true;
#pragma unroll 1
      for (int q = 0; q < 8; ++q) {
        const int x0 = g0 + (q & 1), x1 = g1 + ((q >> 1) & 1), x2 = g2 + ((q >> 2) & 1);
        const int slot = col_slot(m, c, D, x0, x1, x2);
        if (slot < 0) {
          cok = false;
          break;
        }
        const size_t vi = (size_t)slot * BVOX + ((x2 & 7) * 8 + (x1 & 7)) * 8 + (x0 & 7);
        if (COUNT) touched[m.pool_cap + (vi >> 9)] = 1;
        const float wq = corner_w(q, fx, fy, fz);
        const float4 cv4 = STORE == DTSDF_STORE_FP16 ? unpack_col8(__ldg(m.col8 + vi)) : __ldg(m.col + vi);
        cr += wq * cv4.x;
        cg += wq * cv4.y;
        cb += wq * cv4.z;
        cwt += wq * cv4.w;
      }
      if (cok && cwt > 0.0f) {
        out.cw += wc;
        out.rgb[0] += wc * cr;
        out.rgb[1] += wc * cg;
        out.rgb[2] += wc * cb;
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

// Sign of Phi from the present directions' trilinear values (Phi is their convex combination).
// Returns 0 undefined, 1 positive, -1 non-positive, 2 undecided (needs the full combination).
// npres receives the number of present directions: with one present direction that faces
// the ray (return value 1 or -1), Phi is that direction's value lo itself.
template <int STORE, bool COUNT>
__device__ __forceinline__ int sign_fast(const MapView& m, Cell& c, const int gi[3], const float fr[3], const float r[3],
                                         float& lo,
                                         int& npres, uint8_t* touched) {
  const float fx = fr[0], fy = fr[1], fz = fr[2];
  const int lofs = pad_index(gi[0] - 8 * c.cx, gi[1] - 8 * c.cy, gi[2] - 8 * c.cz);
  float mn = 2.f, mx = -2.f;
  bool any = false, facing = false;
  int np = 0;
  // two directions per step: their 16 corner loads are in flight together
#pragma unroll 1
  for (uint32_t mm = c.cmask; mm;) {
    const int D0 = __ffs(mm) - 1;
    mm &= mm - 1;
    const int D1 = mm ? __ffs(mm) - 1 : -1;
    if (mm) mm &= mm - 1;
    float2 v0[8], v1[8];
    const size_t b0 = (size_t)c.slot[D0 * RT_N] * PVOX + lofs;
#pragma unroll
    for (int q = 0; q < 8; ++q) v0[q] = ld_geom<STORE, COUNT>(m, b0 + coff(q), touched);
    if (D1 >= 0) {
      const size_t b1 = (size_t)c.slot[(D1 >= 0 ? D1 : D0) * RT_N] * PVOX + lofs;
#pragma unroll
      for (int q = 0; q < 8; ++q) v1[q] = ld_geom<STORE, COUNT>(m, b1 + coff(q), touched);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int D = k ? D1 : D0;
      if (D < 0) break;
      const float2* v = k ? v1 : v0;
      bool ok = true;
      float s[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        ok &= v[q].y > 0.0f;
        s[q] = v[q].x;
      }
      if (!ok) continue;
      const float phiD = tri(s, fx, fy, fz);
      any = true;
      ++np;
      mn = fminf(mn, phiD);
      mx = fmaxf(mx, phiD);
      const float rc = ray_comp(r, D >> 1);
      const float vr = (D & 1) ? rc : -rc;
      facing |= vr > 0.0f;
    }
  }
  lo = mn;
  npres = np;
  if (!any) return 0;
  if (!facing) return 2;
  if (mn > 0.0f) return 1;
  if (mx <= 0.0f) return -1;
  return 2;
}

// ------------------------------------------------------ combined-TSDF mode
// The same march over the view-dependent combined TSDF (combined.cu): a block cell is present
// when its combined brick belongs to the current combination; the field at a sample is the
// trilinear interpolation of the combined values (all 8 corners defined), so the sign test
// is exact and the bracket ends take its value; the outputs add the normal (central
// differences of that field at +-h, corner differences first) and the trilinear colour.
__device__ __forceinline__ void cell_enter_comb(const MapView& m, Cell& c, int x, int y, int z, uint32_t gen) {
  c.cx = x;
  c.cy = y;
  c.cz = z;
  c.jumped = false;
  c.positive = false;
  const int d = val_dir(probe_block(m.keys, m.vals, m.hmask, x, y, z));
  const bool ok = d >= 0 && __ldg(m.comb_gen + d) == gen;
  c.slot[0] = ok ? d : -1;
  c.cmask = ok ? 1u : 0u;
}

__host__ __device__ __forceinline__ constexpr int ccoff(int q) {
  return (q & 1) + CEDGE * ((q >> 1) & 1) + CEDGE * CEDGE * (q >> 2);
}

// combined value at local voxel (lx, ly, lz) of the cell, -1 <= l <= 9 (beyond [0, 8] through
// the neighbouring block); false where undefined
__device__ __forceinline__ bool comb_at(const MapView& m, const Cell& c, int lx, int ly, int lz, uint32_t gen,
                                        float& v) {
  if ((unsigned)lx <= 8u && (unsigned)ly <= 8u && (unsigned)lz <= 8u) {
    const float2 e = __ldg(m.comb + (size_t)c.slot[0] * CVOX + comb_index(lx, ly, lz));
    v = e.x;
    return e.y > 0.0f;
  }
  const int ex = lx >> 3, ey = ly >> 3, ez = lz >> 3;
  const int d = val_dir(probe_block(m.keys, m.vals, m.hmask, c.cx + ex, c.cy + ey, c.cz + ez));
  if (d < 0 || __ldg(m.comb_gen + d) != gen) return false;
  const float2 e = __ldg(m.comb + (size_t)d * CVOX + comb_index(lx & 7, ly & 7, lz & 7));
  v = e.x;
  return e.y > 0.0f;
}

__device__ __forceinline__ int sign_comb(const MapView& m, const Cell& c, const int gi[3], const float fr[3], float& val,
                                         int& npres) {
  const float fx = fr[0], fy = fr[1], fz = fr[2];
  const size_t base = (size_t)c.slot[0] * CVOX + comb_index(gi[0] - 8 * c.cx, gi[1] - 8 * c.cy, gi[2] - 8 * c.cz);
  float2 v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __ldg(m.comb + base + ccoff(q));
  bool ok = true;
  float s[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    ok &= v[q].y > 0.0f;
    s[q] = v[q].x;
  }
  npres = ok ? 1 : 0;
  if (!ok) return 0;
  val = tri(s, fx, fy, fz);
  return val > 0.0f ? 1 : -1;
}

template <bool COLOR>
__device__ __forceinline__ Combined full_comb(const MapView& m, const Cell& c, const int gi[3], const float fr[3],
                                              bool want_color, uint32_t gen) {
  Combined out;
  out.defined = 0;
  out.phi = 0.f;
  out.wsum = 0.f;
  out.n[0] = out.n[1] = out.n[2] = 0.f;
  out.rgb[0] = out.rgb[1] = out.rgb[2] = 0.f;
  out.cw = 0.f;
  int np = 0;
  float val = 0.f;
  if (sign_comb(m, c, gi, fr, val, np) == 0) return out;
  out.defined = 1;
  out.phi = val;
  const float fx = fr[0], fy = fr[1], fz = fr[2];
  const int l0 = gi[0] - 8 * c.cx, l1 = gi[1] - 8 * c.cy, l2 = gi[2] - 8 * c.cz;
  float gr[3];
  bool gok = true;
#pragma unroll 1
  for (int a = 0; a < 3 && gok; ++a) {
    float dv[8];
    for (int q = 0; q < 8 && gok; ++q) {
      const int x = l0 + (q & 1), y = l1 + ((q >> 1) & 1), z = l2 + (q >> 2);
      float vp = 0.f, vm = 0.f;
      gok = comb_at(m, c, x + (a == 0), y + (a == 1), z + (a == 2), gen, vp) &&
            comb_at(m, c, x - (a == 0), y - (a == 1), z - (a == 2), gen, vm);
      dv[q] = vp - vm;
    }
    if (gok) gr[a] = tri(dv, fx, fy, fz) * (0.5f / m.h);
  }
  if (gok) {
    const float gn = sqrtf(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
    if (gn > 1e-12f) {
      out.wsum = 1.0f;
      out.n[0] = gr[0] / gn;
      out.n[1] = gr[1] / gn;
      out.n[2] = gr[2] / gn;
    }
  }
  if (COLOR && want_color) {
    const size_t base = (size_t)c.slot[0] * CVOX + comb_index(l0, l1, l2);
    float cr = 0.f, cg = 0.f, cb = 0.f;
    bool cok = true;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 cv = unpack_comb_col(__ldg(m.comb_col + base + ccoff(q)));
      cok &= cv.w > 0.0f;
      const float wq = corner_w(q, fx, fy, fz);
      cr += wq * cv.x;
      cg += wq * cv.y;
      cb += wq * cv.z;
    }
    if (cok) {
      out.cw = 1.0f;
      out.rgb[0] = cr;
      out.rgb[1] = cg;
      out.rgb[2] = cb;
    }
  }
  return out;
}

// Two passes. The march (k_render): one lane per ray, marching the global sample grid until the
// first crossing, which it appends to the crossing list (a miss writes the zero outputs); a lane
// whose ray is finished takes the next ray from the launch's work counter at the top of the
// loop once its refill group has finished. Work items are the pixels of tiles of 32 rays
// (tile_w x 32 / tile_w pixels), handed out tile after tile. The refinement (k_refine): one
// lane per crossing, the same number of field evaluations on every lane.
enum { S_MARCH = 0, S_DONE = 1 };

template <int STORE, bool COLOR, bool COUNT, int NJ>
__global__ void __launch_bounds__(RT_N, DTSDF_RENDER_MINB) k_render(MapView m, RenderBatch<NJ> a) {
  __shared__ int s_slot[ND * RT_N];
  __shared__ Pose32 s_pose[NJ];
  uint8_t* touched = a.touched;
  // COUNT build: per-ray event counts (samples, full combinations, cells, allocated cells,
  // crossings, jumps)
  unsigned long long* ctr = COUNT ? (unsigned long long*)(touched + 2 * (size_t)m.pool_cap) : nullptr;
  uint32_t n_samples = 0, n_full = 0, n_cells = 0, n_acells = 0, n_jumps = 0, n_hits = 0;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  for (int jb = tid; jb < a.njobs; jb += RT_N) s_pose[jb] = a.job[jb].Tdev ? pose_from_device(a.job[jb].Tdev) : a.job[jb].T;
  __syncthreads();

  Cell cell;
  cell.slot = s_slot + tid;
  const uint32_t cgen = STORE == STORE_COMBINED ? __ldg(m.comb_cur) : 0u;
  const float org[3] = {m.ox, m.oy, m.oz};
  const float inv_h = 1.0f / m.h;
  const float step = 0.5f * m.h;
  const float bsz = 8.0f * m.h;

  // per-ray state
  bool alive = true;
  int state = S_DONE;
  int jb = 0, pix = 0, it = 0, k = 0, k1 = 0;
  float r[3] = {0.f, 0.f, 0.f}, o[3] = {0.f, 0.f, 0.f}, ri[3] = {0.f, 0.f, 0.f};
  bool prev_def = false;
  float prev_phi = 0.f;

  for (;;) {
    // ---- lanes without a ray take the next work items (warp-aggregated atomic). A group of
    // a.refill consecutive lanes takes new rays once all of its lanes have finished: 32 keeps
    // the warp on one 8x4 tile (coherent, but lanes wait for the slowest), smaller groups take
    // rows of a tile, 1 lets every lane take a ray as soon as it is free
    const unsigned busym = __ballot_sync(0xffffffffu, alive && state != S_DONE);
    const unsigned gmask = a.refill >= 32 ? 0xffffffffu : (((1u << a.refill) - 1u) << (lane & ~(a.refill - 1)));
    const bool need = alive && state == S_DONE && (busym & gmask) == 0;
    const unsigned nm = __ballot_sync(0xffffffffu, need);
    if (nm) {
      const int leader = __ffs(nm) - 1;
      unsigned base = 0;
      if (lane == leader) base = atomicAdd(a.queue, (unsigned)__popc(nm));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (need) {
        const unsigned item = base + (unsigned)__popc(nm & ((1u << lane) - 1u));
        if (item >= (unsigned)a.total) {
          alive = false;
        } else {
          jb = 0;
#pragma unroll 1
          while (jb + 1 < a.njobs && item >= (unsigned)a.job[jb + 1].start) ++jb;
          const RenderJob& J = a.job[jb];
          const int loc = (int)(item - (unsigned)J.start);
          const int tile = loc >> 5, w = loc & 31;
          const int u = (tile % J.tiles_x) * a.tile_w + (w & (a.tile_w - 1));
          const int v = (tile / J.tiles_x) * (32 / a.tile_w) + (w / a.tile_w);
          if (u < J.K.W && v < J.K.H) {
            pix = v * J.K.W + u;
            int zt = -1;
            if (a.zlo) zt = (J.start >> 5) + tile;
            const Pose32& T = s_pose[jb];
            // unit ray in camera and world frame
            const float rc0 = (u - J.K.cx) / J.K.fx, rc1 = (v - J.K.cy) / J.K.fy;
            const float rl = sqrtf(rc0 * rc0 + rc1 * rc1 + 1.0f);
            const float q0 = rc0 / rl, q1 = rc1 / rl, q2 = 1.0f / rl;
            r[0] = T.R[0] * q0 + T.R[1] * q1 + T.R[2] * q2;
            r[1] = T.R[3] * q0 + T.R[4] * q1 + T.R[5] * q2;
            r[2] = T.R[6] * q0 + T.R[7] * q1 + T.R[8] * q2;
            o[0] = T.t[0];
            o[1] = T.t[1];
            o[2] = T.t[2];
#pragma unroll
            for (int q = 0; q < 3; ++q) ri[q] = r[q] != 0.f ? 1.0f / r[q] : 0.f;
            k1 = (int)floorf(m.zmax * rl / step);
            k = (int)ceilf(m.zmin * rl / step);
            if (zt >= 0) {
              // no sample outside the tile's block depth range lies in a cell with an active
              // direction: start and end the march there (one sample of margin on each side)
              const uint32_t lo = a.zlo[zt], hi = a.zhi[zt];
              if (lo == 0xFFFFFFFFu) {
                k1 = k - 1;
              } else {
                k = max(k, (int)floorf(__uint_as_float(lo) * rl / step) - 1);
                k1 = min(k1, (int)ceilf(__uint_as_float(hi) * rl / step) + 1);
              }
            }
            state = S_MARCH;
            it = 0;
            prev_def = false;
            prev_phi = 0.f;
            cell.cx = cell.cy = cell.cz = 0x7fffffff;
            cell.cmask = 0;
            cell.positive = false;
            cell.jumped = true;
          }
        }
      }
    }
    if (!__any_sync(0xffffffffu, alive)) break;
    if (!alive || state == S_DONE) continue;

    // ---- samples of this lane's ray: one per pass of the refill loop, or, when the whole warp
    // refills together, every sample until the ray is finished (no warp vote per sample)
    do {
    if (++it > a.max_samples || k > k1) {
      // a miss (or the sample limit): write the zero outputs
      const RenderJob& J = a.job[jb];
      J.depth[pix] = 0.f;
      J.normals[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (COLOR && J.color) J.color[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
      state = S_DONE;
      continue;
    }
    const float t = (float)k * step;
    // sample position: voxel index and fraction from the single-precision ray (position error
    // ~1e-4 voxel at metres from the origin, which only moves a grid sample)
    int gi[3];
    float fr[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float gq = (o[q] + t * r[q] - org[q]) * inv_h;
      const float fq = floorf(gq);
      gi[q] = (int)fq;
      fr[q] = gq - fq;
    }
    const int cx = gi[0] >> 3, cy = gi[1] >> 3, cz = gi[2] >> 3;
    if (cx != cell.cx || cy != cell.cy || cz != cell.cz) {
      // occupancy filters: cross an empty super-cell (4^3 blocks) or block without a probe
      const int lv = occ_test(m, cx, cy, cz, 1) ? (occ_test(m, cx, cy, cz, 0) ? -1 : 0) : 1;
      if (lv >= 0) {
        const int sh = lv ? 2 : 0;
        const float cs = bsz * (float)(1 << sh);
        const int cc[3] = {cx >> sh, cy >> sh, cz >> sh};
        float tex = 3.4e38f;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (r[q] > 0.f)
            tex = fminf(tex, (org[q] + (cc[q] + 1) * cs - o[q]) * ri[q]);
          else if (r[q] < 0.f)
            tex = fminf(tex, (org[q] + cc[q] * cs - o[q]) * ri[q]);
        }
        if (COUNT) {
          ++n_cells;
          ++n_samples;
        }
        prev_def = false;
        k = max(k + 1, (int)ceilf(tex / step - 1e-3f));
        continue;
      }
      if constexpr (STORE == STORE_COMBINED)
        cell_enter_comb(m, cell, cx, cy, cz, cgen);
      else
        cell_enter(m, cell, cx, cy, cz);
      if (COUNT) {
        ++n_cells;
        n_acells += cell.cmask != 0;
      }
    }
    const bool empty = cell.cmask == 0;
    if (empty || (cell.positive && !cell.jumped)) {
      // an empty cell holds no defined sample; in an all-positive cell (brick bounds cover
      // the +1 apron its trilinear corners reach) no sample can end a crossing: resume two
      // samples before its exit, the first of which fixes the state
      float tex = 3.4e38f;
      const int cc[3] = {cx, cy, cz};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (r[q] > 0.f)
          tex = fminf(tex, (org[q] + (cc[q] + 1) * bsz - o[q]) * ri[q]);
        else if (r[q] < 0.f)
          tex = fminf(tex, (org[q] + cc[q] * bsz - o[q]) * ri[q]);
      }
      if (empty) {
        if (COUNT) ++n_samples;
        prev_def = false;
        k = max(k + 1, (int)ceilf(tex / step - 1e-3f));
        continue;
      }
      cell.jumped = true;
      const int kj = (int)floorf(tex / step) - 1;
      if (kj > k) {
        if (COUNT) ++n_jumps;
        k = kj;
        prev_def = false;
        continue;
      }
    }
    if (COUNT) ++n_samples;
    // ---- the sign of Phi at the sample: from the present directions' values where they agree,
    // else from the full combination
    int sg = 0;
    float val = 0.f;
    int npres = 0;
    if constexpr (STORE == STORE_COMBINED)
      sg = sign_comb(m, cell, gi, fr, val, npres);
    else
      sg = sign_fast<STORE, COUNT>(m, cell, gi, fr, r, val, npres, touched);
    if (sg == 2) {
      if (COUNT) ++n_full;
      Combined C;
      if constexpr (STORE == STORE_COMBINED)
        C = full_comb<false>(m, cell, gi, fr, false, cgen);
      else
        C = combine_full<STORE, false, COUNT>(m, cell, gi, fr, r, touched, false);
      sg = C.defined ? (C.phi > 0.f ? 1 : -1) : 0;
      val = C.phi;
    }
    // ---- transitions
    if (sg == 0) {
      prev_def = false;
      ++k;
    } else if (sg < 0 && prev_def && prev_phi > 0.f) {
      // crossing between samples k-1 and k: handed to the refinement pass
      const unsigned h = atomicAdd(a.nhits, 1u);
      a.hits[h] = make_int2(pix, (k << 6) | jb);
      if (COUNT) ++n_hits;
      state = S_DONE;
    } else {
      prev_def = true;
      prev_phi = sg > 0 ? val : -1.f;
      ++k;
    }
    } while (a.refill >= 32 && state == S_MARCH);
  }
  if (COUNT) {
    atomicAdd(ctr + 0, (unsigned long long)n_samples);
    atomicAdd(ctr + 1, (unsigned long long)n_full);
    atomicAdd(ctr + 2, (unsigned long long)n_cells);
    atomicAdd(ctr + 3, (unsigned long long)n_acells);
    atomicAdd(ctr + 4, (unsigned long long)n_hits);
    atomicAdd(ctr + 5, (unsigned long long)n_jumps);
  }
}

// The refinement of one crossing per lane (Sec. 4): REFINE_HALVINGS bisection steps of the
// bracket [t_{k-1}, t_k] on the sign of Phi (an undefined midpoint counts as free space), then
// the outputs at the final bracket's non-positive end, where Phi is defined (a miss if no
// direction has a combination weight there); the depth is the final bracket's midpoint. The samples are
// placed from the bracket's first sample, computed in double precision from the pose, plus the
// offset along the ray, so that the root and the outputs are placed to ~1e-6 voxel like the
// double-precision definition (the combined normal can turn by milliradians over 1e-4 voxel).
template <int STORE, bool COLOR, bool COUNT, int NJ>
__global__ void __launch_bounds__(RT_N, 3) k_refine(MapView m, RenderBatch<NJ> a) {
  __shared__ int s_slot[ND * RT_N];
  __shared__ Pose32 s_pose[NJ];
  uint8_t* touched = a.touched;
  const int tid = threadIdx.x;
  for (int jb = tid; jb < a.njobs; jb += RT_N) s_pose[jb] = a.job[jb].Tdev ? pose_from_device(a.job[jb].Tdev) : a.job[jb].T;
  __syncthreads();
  Cell cell;
  cell.slot = s_slot + tid;
  const uint32_t cgen = STORE == STORE_COMBINED ? __ldg(m.comb_cur) : 0u;
  const float inv_h = 1.0f / m.h;
  const float step = 0.5f * m.h;
  const unsigned n = min(*((volatile unsigned*)a.nhits), (unsigned)a.total);
  for (unsigned i = blockIdx.x * RT_N + tid; i < n; i += gridDim.x * RT_N) {
    const int2 hr = a.hits[i];
    const int pix = hr.x, k = hr.y >> 6, jb = hr.y & 63;
    const RenderJob& J = a.job[jb];
    const Pose32& T = s_pose[jb];
    const int pu = pix % J.K.W, pv = pix / J.K.W;
    // the march's single-precision ray (weights and offsets), and the bracket's first sample in
    // double precision: integer voxel coordinates and fractions
    float r[3], rl;
    {
      const float rc0 = (pu - J.K.cx) / J.K.fx, rc1 = (pv - J.K.cy) / J.K.fy;
      rl = sqrtf(rc0 * rc0 + rc1 * rc1 + 1.0f);
      const float q0 = rc0 / rl, q1 = rc1 / rl, q2 = 1.0f / rl;
      r[0] = T.R[0] * q0 + T.R[1] * q1 + T.R[2] * q2;
      r[1] = T.R[3] * q0 + T.R[4] * q1 + T.R[5] * q2;
      r[2] = T.R[6] * q0 + T.R[7] * q1 + T.R[8] * q2;
    }
    int bi[3];
    float bf[3];
    {
      double Rd[9], Od[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
#pragma unroll
        for (int e = 0; e < 3; ++e) Rd[3 * q + e] = J.Tdev ? __ldg(J.Tdev + 4 * q + e) : J.T64[3 * q + e];
        Od[q] = J.Tdev ? __ldg(J.Tdev + 4 * q + 3) : J.T64[9 + q];
      }
      const double q0 = ((double)pu - (double)J.K.cx) / (double)J.K.fx;
      const double q1 = ((double)pv - (double)J.K.cy) / (double)J.K.fy;
      const double ql = sqrt(q0 * q0 + q1 * q1 + 1.0);
      const double hd = (double)m.h;
      const double t0 = (double)(k - 1) * (0.5 * hd);
      const double org[3] = {(double)m.ox, (double)m.oy, (double)m.oz};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const double rq = (Rd[3 * q] * q0 + Rd[3 * q + 1] * q1 + Rd[3 * q + 2]) / ql;
        const double gq = (Od[q] + t0 * rq - org[q]) / hd;
        const double fq = floor(gq);
        bi[q] = (int)fq;
        bf[q] = (float)(gq - fq);
      }
    }
    cell.cx = cell.cy = cell.cz = 0x7fffffff;
    cell.cmask = 0;
    float ta = 0.f, tb = step;
    float out_depth = 0.f;
    float4 out_n = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 out_c = make_float4(0.f, 0.f, 0.f, 0.f);
    // after an evaluation that needed the full combination, the next one (a nearby point) goes
    // to it directly: the sign test's corners would be read twice (both give the same sign
    // where the sign test decides)
    bool went_full = false;
    // phases: 0 bisection (REFINE_HALVINGS steps), 3 outputs at the final bracket's end tb
#pragma unroll 1
    for (int j = 0; j <= REFINE_HALVINGS; ++j) {
      const int phase = j < REFINE_HALVINGS ? 0 : 3;
      const float t = phase == 0 ? 0.5f * (ta + tb) : tb;
      int gi[3];
      float fr[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float gq = bf[q] + t * (r[q] * inv_h);
        const float fq = floorf(gq);
        gi[q] = bi[q] + (int)fq;
        fr[q] = gq - fq;
      }
      const int cx = gi[0] >> 3, cy = gi[1] >> 3, cz = gi[2] >> 3;
      if (cx != cell.cx || cy != cell.cy || cz != cell.cz) {
        if constexpr (STORE == STORE_COMBINED)
          cell_enter_comb(m, cell, cx, cy, cz, cgen);
        else
          cell_enter(m, cell, cx, cy, cz);
      }
      // the bracket ends need Phi's value: from the sign test when one facing direction is
      // present, else from the full combination; the outputs always need the full combination
      int sg = 0;
      Combined C;
      C.defined = 0;
      C.phi = 0.f;
      C.wsum = 0.f;
      C.n[0] = C.n[1] = C.n[2] = 0.f;
      C.rgb[0] = C.rgb[1] = C.rgb[2] = 0.f;
      C.cw = 0.f;
      if (cell.cmask) {
        bool full = phase == 3 || (STORE != STORE_COMBINED && went_full);
        if (!full) {
          int npres = 0;
          float val = 0.f;
          if constexpr (STORE == STORE_COMBINED)
            sg = sign_comb(m, cell, gi, fr, val, npres);
          else
            sg = sign_fast<STORE, COUNT>(m, cell, gi, fr, r, val, npres, touched);
          full = sg == 2 || (phase >= 1 && npres > 1);
          if (!full) {
            C.defined = sg != 0;
            C.phi = val;
          }
        }
        went_full = full;
        if (full) {
          if constexpr (STORE == STORE_COMBINED)
            C = full_comb<COLOR>(m, cell, gi, fr, phase == 3, cgen);
          else
            C = combine_full<STORE, COLOR, COUNT>(m, cell, gi, fr, r, touched, phase == 3);
          sg = C.defined ? (C.phi > 0.f ? 1 : -1) : 0;
        }
      }
      if (phase == 0) {
        // an undefined midpoint counts as free space
        if (sg < 0)
          tb = t;
        else
          ta = t;
      } else {
        // the root: the final bracket's midpoint (within h / 2^(REFINE_HALVINGS + 2) of it)
        const float ts = 0.5f * (ta + tb);
        const float nl = sqrtf(C.n[0] * C.n[0] + C.n[1] * C.n[1] + C.n[2] * C.n[2]);
        if (C.defined && C.wsum > 0.f && nl > 0.f) {
          const float n0 = C.n[0] / nl, n1 = C.n[1] / nl, n2 = C.n[2] / nl;
          // world -> camera: R^T n
          const float c0 = T.R[0] * n0 + T.R[3] * n1 + T.R[6] * n2;
          const float c1 = T.R[1] * n0 + T.R[4] * n1 + T.R[7] * n2;
          const float c2 = T.R[2] * n0 + T.R[5] * n1 + T.R[8] * n2;
          out_depth = ((float)(k - 1) * step + ts) / rl;
          out_n = make_float4(c0, c1, c2, out_depth);
          if (COLOR && C.cw > 0.f) out_c = make_float4(C.rgb[0] / C.cw, C.rgb[1] / C.cw, C.rgb[2] / C.cw, 1.0f);
        }
      }
    }
    J.depth[pix] = out_depth;
    J.normals[pix] = out_n;
    if (COLOR && J.color) J.color[pix] = out_c;
  }
}

// Depth ranges of the ray tiles: every allocated block with a direction holding weighted voxels
// (brick bound < inf) projects the 8 corners of its cell box [8 b, 8 b + 8) h into each frame;
// the ray tiles covering its pixel bounding box (grown by half a pixel) take the minimum and
// maximum camera depth of its corners. A box reaching behind the camera covers the whole frame
// from depth 0. Floats are non-negative, so their bit patterns order like unsigned integers.
template <int NJ>
__global__ void __launch_bounds__(256) k_tile_range(MapView m, RenderBatch<NJ> a, uint32_t* zlo, uint32_t* zhi) {
  __shared__ Pose32 s_pose[NJ];
  for (int jb = threadIdx.x; jb < a.njobs; jb += blockDim.x)
    s_pose[jb] = a.job[jb].Tdev ? pose_from_device(a.job[jb].Tdev) : a.job[jb].T;
  __syncthreads();
  const uint32_t ndir = min(*((volatile uint32_t*)(m.counters + C_DIR)), m.dir_cap);
  const float bs = 8.0f * m.h;
  const int th = 32 / a.tile_w;
  for (uint32_t d = blockIdx.x * blockDim.x + threadIdx.x; d < ndir; d += gridDim.x * blockDim.x) {
    const uint32_t mask = (uint32_t)__ldg(m.dir_slots + (size_t)d * 8 + SLOT_MASK);
    bool act = false;
    for (uint32_t mm = mask; mm; mm &= mm - 1) {
      const int sl = __ldg(m.dir_slots + (size_t)d * 8 + (__ffs(mm) - 1));
      act |= sl >= 0 && __ldg(m.bound + sl) < INFINITY;
    }
    if (!act) continue;
    const float x0 = m.ox + (float)__ldg(m.dir_coord + 4 * d) * bs;
    const float y0 = m.oy + (float)__ldg(m.dir_coord + 4 * d + 1) * bs;
    const float z0 = m.oz + (float)__ldg(m.dir_coord + 4 * d + 2) * bs;
    for (int jb = 0; jb < a.njobs; ++jb) {
      const Pose32& T = s_pose[jb];
      const RenderJob& J = a.job[jb];
      float zmin = 3.4e38f, zmax = 0.0f, umin = 3.4e38f, umax = -3.4e38f, vmin = 3.4e38f, vmax = -3.4e38f;
      bool behind = false;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float px = x0 + ((c & 1) ? bs : 0.f) - T.t[0];
        const float py = y0 + ((c & 2) ? bs : 0.f) - T.t[1];
        const float pz = z0 + ((c & 4) ? bs : 0.f) - T.t[2];
        const float xc = T.R[0] * px + T.R[3] * py + T.R[6] * pz;
        const float yc = T.R[1] * px + T.R[4] * py + T.R[7] * pz;
        const float zc = T.R[2] * px + T.R[5] * py + T.R[8] * pz;
        zmin = fminf(zmin, zc);
        zmax = fmaxf(zmax, zc);
        if (zc < 1e-4f) {
          behind = true;
        } else {
          const float u = J.K.fx * xc / zc + J.K.cx, v = J.K.fy * yc / zc + J.K.cy;
          umin = fminf(umin, u);
          umax = fmaxf(umax, u);
          vmin = fminf(vmin, v);
          vmax = fmaxf(vmax, v);
        }
      }
      if (zmax < 1e-4f || zmin > m.zmax || zmax < m.zmin) continue;
      int u0 = 0, u1 = J.K.W - 1, v0 = 0, v1 = J.K.H - 1;
      if (behind) {
        zmin = 0.0f;
      } else {
        u0 = max(u0, (int)floorf(umin - 0.5f));
        u1 = min(u1, (int)ceilf(umax + 0.5f));
        v0 = max(v0, (int)floorf(vmin - 0.5f));
        v1 = min(v1, (int)ceilf(vmax + 0.5f));
        if (u0 > u1 || v0 > v1) continue;
      }
      const uint32_t lo = __float_as_uint(fmaxf(zmin, 0.0f)), hi = __float_as_uint(zmax);
      const int base = J.start >> 5;
      for (int ty = v0 / th; ty <= v1 / th; ++ty)
        for (int tx = u0 / a.tile_w; tx <= u1 / a.tile_w; ++tx) {
          const int i = base + ty * J.tiles_x + tx;
          atomicMin(zlo + i, lo);
          atomicMax(zhi + i, hi);
        }
    }
  }
}

namespace {

// CTAs of the persistent render grid that fit on the device at once (per kernel instance).
template <typename KernelT>
int resident_ctas(KernelT kern) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RT_N, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

template <int STORE, bool COLOR, bool COUNT, int NJ>
void launch_k_render(const MapView& m, const RenderBatch<NJ>& a, int ctas, cudaStream_t s) {
  static thread_local int cached_dev = -1, cached_ctas = 0, cached_refine = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != cached_dev) {
    cached_ctas = resident_ctas(k_render<STORE, COLOR, COUNT, NJ>);
    cached_refine = resident_ctas(k_refine<STORE, COLOR, COUNT, NJ>);
    cached_dev = dev;
  }
  int grid = ctas > 0 ? ctas : cached_ctas;
  const int need = (a.total + RT_N - 1) / RT_N;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  k_render<STORE, COLOR, COUNT, NJ><<<grid, RT_N, 0, s>>>(m, a);
  // the crossings are at most one per ray; their count is known on the device only
  int rgrid = cached_refine;
  if (rgrid > need) rgrid = need;
  if (rgrid < 1) rgrid = 1;
  k_refine<STORE, COLOR, COUNT, NJ><<<rgrid, RT_N, 0, s>>>(m, a);
}

template <int NJ>
void dispatch_render(const MapView& m, const RenderBatch<NJ>& a, bool col, int ctas, cudaStream_t s,
                     bool combined) {
  if (combined) {
    if (col && m.comb_col)
      launch_k_render<STORE_COMBINED, true, false, NJ>(m, a, ctas, s);
    else
      launch_k_render<STORE_COMBINED, false, false, NJ>(m, a, ctas, s);
    return;
  }
  const bool cnt = a.touched != nullptr;
#define DTSDF_RENDER(ST, CO, CN) launch_k_render<ST, CO, CN, NJ>(m, a, ctas, s)
  if (cnt) {
    if (m.storage == DTSDF_STORE_FP16) {
      if (col) DTSDF_RENDER(DTSDF_STORE_FP16, true, true); else DTSDF_RENDER(DTSDF_STORE_FP16, false, true);
    } else {
      if (col) DTSDF_RENDER(DTSDF_STORE_FP32, true, true); else DTSDF_RENDER(DTSDF_STORE_FP32, false, true);
    }
  } else {
    // the direct ray-cast: the per-lane march
    if (m.storage == DTSDF_STORE_FP16) {
      if (col) DTSDF_RENDER(DTSDF_STORE_FP16, true, false); else DTSDF_RENDER(DTSDF_STORE_FP16, false, false);
    } else {
      if (col) DTSDF_RENDER(DTSDF_STORE_FP32, true, false); else DTSDF_RENDER(DTSDF_STORE_FP32, false, false);
    }
  }
#undef DTSDF_RENDER
}

template <int NJ>
void fill_batch(RenderBatch<NJ>& a, const RenderJob* jobs, int njobs, unsigned* queue, uint8_t* touched,
                int refill, int tile_w) {
  a.njobs = njobs;
  a.queue = queue;
  a.touched = touched;
  a.max_samples = 1 << 17;
  a.refill = refill;
  a.tile_w = tile_w;
  const int tile_h = 32 / tile_w;
  int start = 0;
  for (int i = 0; i < njobs; ++i) {
    a.job[i] = jobs[i];
    a.job[i].tiles_x = (jobs[i].K.W + tile_w - 1) / tile_w;
    a.job[i].start = start;
    start += a.job[i].tiles_x * ((jobs[i].K.H + tile_h - 1) / tile_h) * 32;
  }
  a.total = start;
}

}  // namespace

// Depth-range pre-pass into stream-ordered scratch from the pool, then the render. The
// scratch is freed on the stream after the render, so concurrent launches never share it.
template <int NJ>
cudaError_t range_and_render(const MapView& m, RenderBatch<NJ>& a, bool col, int ctas, cudaStream_t s,
                             cudaMemPool_t pool, bool combined) {
  // scratch: the crossing list (8 bytes per ray), its counter (16 bytes), then the depth
  // ranges of the ray tiles (2 words per tile)
  const size_t ntiles = (size_t)a.total / 32;
  const size_t hit_bytes = (size_t)a.total * sizeof(int2);
  const size_t bytes = hit_bytes + 16 + 2 * ntiles * sizeof(uint32_t);
  char* buf = nullptr;
  cudaError_t e = pool ? cudaMallocFromPoolAsync((void**)&buf, bytes, pool, s) : cudaMallocAsync((void**)&buf, bytes, s);
  if (e != cudaSuccess) return e;
  a.hits = (int2*)buf;
  a.nhits = (unsigned*)(buf + hit_bytes);
  uint32_t* zr = (uint32_t*)(buf + hit_bytes + 16);
  a.zlo = a.zhi = nullptr;
  e = cudaMemsetAsync(a.nhits, 0, sizeof(unsigned), s);
  if (e == cudaSuccess && ntiles) {
    e = cudaMemsetAsync(zr, 0xFF, ntiles * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(zr + ntiles, 0, ntiles * sizeof(uint32_t), s);
    if (e == cudaSuccess) {
      static thread_local int sms = 0;
      if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 132;
      }
      k_tile_range<NJ><<<sms * 4, 256, 0, s>>>(m, a, zr, zr + ntiles);
      a.zlo = zr;
      a.zhi = zr + ntiles;
    }
  }
  if (e == cudaSuccess) {
    dispatch_render(m, a, col, ctas, s, combined);
    e = cudaGetLastError();
  }
  const cudaError_t f = cudaFreeAsync(buf, s);
  if (e == cudaSuccess) e = f;
  return e;
}

cudaError_t launch_render_jobs(const MapView& m, const RenderJob* jobs, int njobs, unsigned* queue, cudaStream_t s,
                               uint8_t* touched, const RenderShape& sh, cudaMemPool_t pool, bool combined) {
  const int ctas = sh.ctas, refill = sh.refill, tile_w = sh.tile_w;
  bool col = false;
  for (int i = 0; i < njobs; ++i) col |= jobs[i].color != nullptr;
  col &= m.color != 0;
  if (njobs == 1) {
    RenderBatch<1> a;
    fill_batch(a, jobs, njobs, queue, touched, refill, tile_w);
    return range_and_render(m, a, col, ctas, s, pool, combined);
  }
  RenderBatch<MAX_RENDER_JOBS> a;
  fill_batch(a, jobs, njobs, queue, touched, refill, tile_w);
  return range_and_render(m, a, col, ctas, s, pool, combined);
}

}  // namespace dtsdf
