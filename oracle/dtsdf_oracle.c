/*
 * FP64 CPU oracle of DTSDF fusion and rendering (test infrastructure only).
 *
 * This file is a plain, slow, obviously correct restatement of what the paper
 * computes, used only by the tests, the smoke check and the CPU baseline of the
 * benchmark. It shares no code with the CUDA path. Every value and every decision
 * (which pixel a voxel projects to, which blocks a segment crosses, whether a voxel
 * lies in the truncation band, whether a normal belongs to a direction) is taken in
 * double precision.
 *
 * A decision whose FP64 quantity lies within a stated margin of its threshold is a
 * "tie": an implementation that computes the same quantity in single precision may
 * take it the other way. The oracle records ties (per pixel, per allocated
 * (block, D) key and per voxel) so that a comparison can check that every element on
 * which two implementations disagree is a tie of the oracle. The margins bound the
 * difference between an FP32 and an FP64 evaluation of the quantity:
 *   TIE_N  2e-5    cosines between a pixel normal and an axis or the view ray: the
 *                  single-precision rounding of a normal computed in double precision
 *                  and of the pose's rotation (~1e-7), with a wide margin
 *   TIE_X  1e-5 m  camera- and world-frame coordinates and distances (FP32 keeps ~1e-6 m
 *                  at 8 m), plus TIE_N times the lever arm where a normal multiplies a
 *                  distance
 *   TIE_PX 2e-3    pixel coordinates of a projection (about 10x the FP32 rounding of
 *                  f x / z at f = 910)
 *
 * Paper references (Splietker & Behnke, "Rendering the Directional TSDF for
 * Tracking and Multi-Sensor Registration with Point-To-Plane Scale ICP"):
 *   Sec. 3  Eq. angular_threshold, Eq. direction_weight, Eq. combined_fusion_weight,
 *           Eq. color_weight, Eq. point-to-plane, free-space carving, voxel
 *           projection fusion.
 *   Sec. 4  ray-cast rendering (regular probing, then refinement of the first
 *           positive-to-negative transition), Eq. combine_weight,
 *           Eq. combine_tsdf_weight (no-gradient fallback).
 *   Sec. 7  voxel-block hashing of 8^3 blocks keyed by (x, y, z, D); depth
 *           outlier filter (two supporting neighbours) and cross-product normals.
 *   Sec. 5.1 Eq. ICP_weight, reused as the fusion depth weight.
 *
 * Readings of points the paper leaves open (the GPU path implements the same ones):
 *   direction weight  w_dir = clamp((theta - acos<n,v>) / (2 theta - pi/2), 0, 1)
 *   depth weight      w_depth = 1 / (z + 1 - z_min)^2       (the ICP weight)
 *   angle weight      w_angle = max(0, <n, -r>)             (r: unit pixel ray)
 *   SDF sign          d = <x - p, n> / tau with n facing the camera (d > 0 in front)
 *   carving           d_raw > tau and no valid depth within 2 px differs by more
 *                     than tau: sdf <- running average with value 1, weight w_carve
 *   allocation        every (block, D) whose closed 8h cube the segment
 *                     [p - tau r, p + tau r] meets, for every D the normal belongs to
 *   presence          a direction counts at x only if all 8 trilinear corners
 *                     exist and have weight > 0; its gradient (central differences
 *                     of the trilinear field at +-h) only if the 6 offset samples
 *                     are present
 *   render march      samples at t = k * h/2 along the unit ray; the first pair of
 *                     consecutive defined samples with Phi > 0 >= Phi brackets the
 *                     hit; the hit is the root of the continuous Phi(t) in that
 *                     bracket, found by bisection to 1e-10 m (an undefined midpoint
 *                     counts as free space); normal and colour are evaluated at the
 *                     root's side of Phi <= 0 (the non-positive end of the final
 *                     bracket, where Phi is defined: the root itself can sit on the
 *                     edge of the defined region); a miss if no direction has a
 *                     combination weight there
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp -ffp-contract=off (see oracle/__init__.py; no contraction,
 * so that x86 and Arm builds give the same bits).
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ND 6
#define BLK 8
#define BVOX 512
#define TIE_N 2e-5
#define TIE_X 1e-5
#define TIE_PX 2e-3
/* bisection of the crossing bracket ends when it is narrower than this (metres along the ray) */
#define ROOT_TOL 1e-10

/* Direction axis vectors v^D: X+, X-, Y+, Y-, Z+, Z- (Sec. 3). */
static const double VDIR[ND][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

typedef struct {
  double sdf, w, r, g, b, wc;
} ovox;

typedef struct {
  /* parameters: the nominal single-precision values the library takes, widened to double */
  double h, tau, theta, wmax, wcarve, zmin, zmax, dsup, costh, origin[3];
  int carve_r, dense_dim, color;
  /* hash: (bx, by, bz, D) -> brick index, open addressing, linear probing */
  uint64_t* keys;
  int32_t* vals;
  size_t cap, count;
  /* bricks */
  ovox* vox;
  uint8_t* tie;   /* per voxel: 1 once a decision about its update was a tie */
  int32_t* coord; /* 4 per brick: bx, by, bz, D */
  int32_t* first_frame;
  size_t nbricks, brick_cap;
  int frames;
  /* (block, D) keys whose allocation was a tie in some frame, with the first such frame */
  uint64_t* tkeys;
  int32_t* tvals;
  size_t tcap, tcount;
  /* view-dependent combined TSDF (om_combine): one entry per allocated block */
  uint64_t* ckeys;   /* block key -> combined block index, open addressing */
  int32_t* cvals;
  size_t ccap, nblocks;
  double* comb;      /* per block, 512 voxels x 5: phi, defined, r, g, b */
  uint8_t* comb_col; /* per block, 512 colour flags */
} omap;

#define EMPTY_KEY 0xFFFFFFFFFFFFFFFFull

static uint64_t pack_key(int bx, int by, int bz, int D) {
  return ((uint64_t)(uint32_t)(bx + (1 << 19)) & 0xFFFFFull) << 44 |
         ((uint64_t)(uint32_t)(by + (1 << 19)) & 0xFFFFFull) << 24 |
         ((uint64_t)(uint32_t)(bz + (1 << 19)) & 0xFFFFFull) << 4 | (uint64_t)D;
}

static uint64_t mix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

static int32_t hash_find(const omap* m, int bx, int by, int bz, int D) {
  uint64_t k = pack_key(bx, by, bz, D);
  size_t i = mix64(k) & (m->cap - 1);
  for (;;) {
    if (m->keys[i] == k) return m->vals[i];
    if (m->keys[i] == EMPTY_KEY) return -1;
    i = (i + 1) & (m->cap - 1);
  }
}

static void hash_put(omap* m, uint64_t k, int32_t v) {
  size_t i = mix64(k) & (m->cap - 1);
  while (m->keys[i] != EMPTY_KEY && m->keys[i] != k) i = (i + 1) & (m->cap - 1);
  if (m->keys[i] == EMPTY_KEY) m->count++;
  m->keys[i] = k;
  m->vals[i] = v;
}

static int hash_grow(omap* m) {
  size_t oc = m->cap;
  uint64_t* ok = m->keys;
  int32_t* ov = m->vals;
  m->cap = oc * 2;
  m->keys = (uint64_t*)malloc(m->cap * sizeof(uint64_t));
  m->vals = (int32_t*)malloc(m->cap * sizeof(int32_t));
  if (!m->keys || !m->vals) return -1;
  memset(m->keys, 0xFF, m->cap * sizeof(uint64_t));
  m->count = 0;
  for (size_t i = 0; i < oc; ++i)
    if (ok[i] != EMPTY_KEY) hash_put(m, ok[i], ov[i]);
  free(ok);
  free(ov);
  return 0;
}

void om_free(omap* m);

/* Record a tie of the allocation of (bx, by, bz, D) in frame `frame` (keeps the first frame). */
static int tie_key_put(omap* m, int bx, int by, int bz, int D, int frame) {
  if ((m->tcount + 1) * 2 > m->tcap) {
    size_t oc = m->tcap;
    uint64_t* ok = m->tkeys;
    int32_t* ov = m->tvals;
    m->tcap = oc * 2;
    m->tkeys = (uint64_t*)malloc(m->tcap * sizeof(uint64_t));
    m->tvals = (int32_t*)malloc(m->tcap * sizeof(int32_t));
    if (!m->tkeys || !m->tvals) return -1;
    memset(m->tkeys, 0xFF, m->tcap * sizeof(uint64_t));
    m->tcount = 0;
    for (size_t i = 0; i < oc; ++i)
      if (ok[i] != EMPTY_KEY) {
        size_t j = mix64(ok[i]) & (m->tcap - 1);
        while (m->tkeys[j] != EMPTY_KEY) j = (j + 1) & (m->tcap - 1);
        m->tkeys[j] = ok[i];
        m->tvals[j] = ov[i];
        m->tcount++;
      }
    free(ok);
    free(ov);
  }
  const uint64_t k = pack_key(bx, by, bz, D);
  size_t i = mix64(k) & (m->tcap - 1);
  while (m->tkeys[i] != EMPTY_KEY && m->tkeys[i] != k) i = (i + 1) & (m->tcap - 1);
  if (m->tkeys[i] == EMPTY_KEY) {
    m->tkeys[i] = k;
    m->tvals[i] = frame;
    m->tcount++;
  }
  return 0;
}

/* First frame in which the allocation of (bx, by, bz, D) was a tie, -1 if never. */
static int32_t tie_key_find(const omap* m, int bx, int by, int bz, int D) {
  const uint64_t k = pack_key(bx, by, bz, D);
  size_t i = mix64(k) & (m->tcap - 1);
  for (;;) {
    if (m->tkeys[i] == k) return m->tvals[i];
    if (m->tkeys[i] == EMPTY_KEY) return -1;
    i = (i + 1) & (m->tcap - 1);
  }
}

/* Allocate brick (bx, by, bz, D) if absent. Initial voxel: sdf 1, weights 0, colour 0. */
static int32_t brick_alloc(omap* m, int bx, int by, int bz, int D, int frame) {
  int32_t b = hash_find(m, bx, by, bz, D);
  if (b >= 0) return b;
  if (m->nbricks == m->brick_cap) {
    size_t nc = m->brick_cap ? m->brick_cap * 2 : 1024;
    ovox* nv = (ovox*)realloc(m->vox, nc * BVOX * sizeof(ovox));
    if (nv) m->vox = nv;
    uint8_t* nt = (uint8_t*)realloc(m->tie, nc * BVOX);
    if (nt) m->tie = nt;
    int32_t* ncd = (int32_t*)realloc(m->coord, nc * 4 * sizeof(int32_t));
    if (ncd) m->coord = ncd;
    int32_t* nff = (int32_t*)realloc(m->first_frame, nc * sizeof(int32_t));
    if (!nv || !nt || !ncd || !nff) return -1;
    m->coord = ncd;
    m->first_frame = nff;
    m->brick_cap = nc;
  }
  if ((m->count + 1) * 2 > m->cap && hash_grow(m) != 0) return -1;
  b = (int32_t)m->nbricks++;
  ovox* v = m->vox + (size_t)b * BVOX;
  for (int i = 0; i < BVOX; ++i) {
    v[i].sdf = 1.0;
    v[i].w = v[i].r = v[i].g = v[i].b = v[i].wc = 0.0;
  }
  memset(m->tie + (size_t)b * BVOX, 0, BVOX);
  m->coord[4 * b] = bx;
  m->coord[4 * b + 1] = by;
  m->coord[4 * b + 2] = bz;
  m->coord[4 * b + 3] = D;
  m->first_frame[b] = frame;
  hash_put(m, pack_key(bx, by, bz, D), b);
  return b;
}

omap* om_create(float voxel_size, float truncation, float theta, float w_max, float w_carve, float z_min,
                float z_max, float delta_sup, int carve_radius, int dense_dim, const float* origin, int color) {
  omap* m = (omap*)calloc(1, sizeof(omap));
  if (!m) return NULL;
  m->h = voxel_size;
  m->tau = truncation;
  m->theta = theta;
  m->wmax = w_max;
  m->wcarve = w_carve;
  m->zmin = z_min;
  m->zmax = z_max;
  m->dsup = delta_sup;
  m->costh = cos((double)theta);
  m->carve_r = carve_radius;
  m->dense_dim = dense_dim;
  m->color = color;
  for (int a = 0; a < 3; ++a) m->origin[a] = origin ? (double)origin[a] : 0.0;
  m->cap = 1 << 12;
  m->keys = (uint64_t*)malloc(m->cap * sizeof(uint64_t));
  m->vals = (int32_t*)malloc(m->cap * sizeof(int32_t));
  m->tcap = 1 << 10;
  m->tkeys = (uint64_t*)malloc(m->tcap * sizeof(uint64_t));
  m->tvals = (int32_t*)malloc(m->tcap * sizeof(int32_t));
  if (!m->keys || !m->vals || !m->tkeys || !m->tvals) {
    om_free(m);
    return NULL;
  }
  memset(m->keys, 0xFF, m->cap * sizeof(uint64_t));
  memset(m->tkeys, 0xFF, m->tcap * sizeof(uint64_t));
  if (dense_dim > 0) {
    /* dense grid: every (block, D) of the dense_dim^3 voxel cube exists from the start */
    int nb = dense_dim / BLK;
    for (int D = 0; D < ND; ++D)
      for (int z = 0; z < nb; ++z)
        for (int y = 0; y < nb; ++y)
          for (int x = 0; x < nb; ++x)
            if (brick_alloc(m, x, y, z, D, 0) < 0) {
              om_free(m);
              return NULL;
            }
  }
  return m;
}

void om_free(omap* m) {
  if (!m) return;
  free(m->keys);
  free(m->vals);
  free(m->vox);
  free(m->tie);
  free(m->coord);
  free(m->first_frame);
  free(m->tkeys);
  free(m->tvals);
  free(m->ckeys);
  free(m->cvals);
  free(m->comb);
  free(m->comb_col);
  free(m);
}

int64_t om_num_bricks(const omap* m) { return (int64_t)m->nbricks; }

/* Brick list: n x 5 (bx, by, bz, D, first frame). */
void om_bricks(const omap* m, int32_t* out) {
  for (size_t b = 0; b < m->nbricks; ++b) {
    for (int a = 0; a < 4; ++a) out[5 * b + a] = m->coord[4 * b + a];
    out[5 * b + 4] = m->first_frame[b];
  }
}

/* Voxel data of one brick: 512 x 6 doubles (sdf, w, r, g, b, wc), x fastest. Returns -1 if absent. */
int om_brick_data(const omap* m, int bx, int by, int bz, int D, double* out) {
  int32_t b = hash_find(m, bx, by, bz, D);
  if (b < 0) return -1;
  const ovox* v = m->vox + (size_t)b * BVOX;
  for (int i = 0; i < BVOX; ++i) {
    out[6 * i] = v[i].sdf;
    out[6 * i + 1] = v[i].w;
    out[6 * i + 2] = v[i].r;
    out[6 * i + 3] = v[i].g;
    out[6 * i + 4] = v[i].b;
    out[6 * i + 5] = v[i].wc;
  }
  return 0;
}

/* Tie flags of one brick's 512 voxels (bit 0: sdf and weight, bit 1: colour). Returns -1 if absent. */
int om_brick_ties(const omap* m, int bx, int by, int bz, int D, uint8_t* out) {
  int32_t b = hash_find(m, bx, by, bz, D);
  if (b < 0) return -1;
  memcpy(out, m->tie + (size_t)b * BVOX, BVOX);
  return 0;
}

/* Bricks [start, start + count) in map order: coordinates (n x 4: bx, by, bz, D), voxels
 * (n x 512 x 6, as om_brick_data) and tie flags (n x 512, as om_brick_ties). Returns the number
 * written. */
long om_export(const omap* m, long start, long count, int32_t* coords, double* vox, uint8_t* ties) {
  long n = 0;
  for (long b = start; b < (long)m->nbricks && n < count; ++b, ++n) {
    for (int a = 0; a < 4; ++a) coords[4 * n + a] = m->coord[4 * b + a];
    const ovox* v = m->vox + (size_t)b * BVOX;
    double* o = vox + (size_t)n * BVOX * 6;
    for (int i = 0; i < BVOX; ++i) {
      o[6 * i] = v[i].sdf;
      o[6 * i + 1] = v[i].w;
      o[6 * i + 2] = v[i].r;
      o[6 * i + 3] = v[i].g;
      o[6 * i + 4] = v[i].b;
      o[6 * i + 5] = v[i].wc;
    }
    memcpy(ties + (size_t)n * BVOX, m->tie + (size_t)b * BVOX, BVOX);
  }
  return n;
}

/* First frame in which the allocation of (bx, by, bz, D) was a tie, -1 if it never was. */
int om_alloc_tie(const omap* m, int bx, int by, int bz, int D) { return tie_key_find(m, bx, by, bz, D); }

/* ===================================================== preprocessing (A0) == */
/*
 * Depth outlier filter (Sec. 7): a pixel with depth in [z_min, z_max] is kept only
 * if at least two of its 8 neighbours are in range and differ by at most
 * delta_sup. Normals: cross product of the central differences of the
 * back-projected neighbours in x and y (Sec. 7), oriented toward the camera;
 * valid only where the centre and the 4 neighbours survived the filter.
 * Back-projection follows Eq. reprojection: (z (u - cx)/fx, z (v - cy)/fy, z).
 * The filter compares differences of input depths, which are exact in either
 * precision near the threshold (Sterbenz: the two depths are within a factor of two
 * when they differ by about delta_sup >= 0.1 m / 2), so it has no ties. The
 * orientation of a normal is a tie when <n, P> / |P| is within TIE_N of zero.
 */
typedef struct {
  int W, H;
  double fx, fy, cx, cy;
  float* z;      /* filtered depth */
  uint8_t* ok;   /* survived filter */
  uint8_t* nok;  /* has a normal */
  uint8_t* tie;  /* the normal's orientation is a tie */
  double* P;     /* camera point */
  double* n;     /* camera normal */
} oframe;

static void frame_free(oframe* f) {
  free(f->z);
  free(f->ok);
  free(f->nok);
  free(f->tie);
  free(f->P);
  free(f->n);
}

static int in_range(double z, double zmin, double zmax) { return z > 0.0 && z >= zmin && z <= zmax; }

static int frame_prepare(oframe* f, const float* depth, int W, int H, double fx, double fy, double cx, double cy,
                         double zmin, double zmax, double dsup) {
  size_t n = (size_t)W * H;
  f->W = W;
  f->H = H;
  f->fx = fx;
  f->fy = fy;
  f->cx = cx;
  f->cy = cy;
  f->z = (float*)calloc(n, sizeof(float));
  f->ok = (uint8_t*)calloc(n, 1);
  f->nok = (uint8_t*)calloc(n, 1);
  f->tie = (uint8_t*)calloc(n, 1);
  f->P = (double*)calloc(3 * n, sizeof(double));
  f->n = (double*)calloc(3 * n, sizeof(double));
  if (!f->z || !f->ok || !f->nok || !f->tie || !f->P || !f->n) return -1;
  for (int v = 0; v < H; ++v)
    for (int u = 0; u < W; ++u) {
      size_t i = (size_t)v * W + u;
      double z = depth[i];
      if (!in_range(z, zmin, zmax)) continue;
      int support = 0;
      for (int dv = -1; dv <= 1; ++dv)
        for (int du = -1; du <= 1; ++du) {
          if (!du && !dv) continue;
          int uu = u + du, vv = v + dv;
          if (uu < 0 || vv < 0 || uu >= W || vv >= H) continue;
          double zn = depth[(size_t)vv * W + uu];
          if (!in_range(zn, zmin, zmax)) continue;
          if (fabs(zn - z) <= dsup) support++;
        }
      if (support >= 2) {
        f->ok[i] = 1;
        f->z[i] = depth[i];
        f->P[3 * i] = z * ((u - cx) / fx);
        f->P[3 * i + 1] = z * ((v - cy) / fy);
        f->P[3 * i + 2] = z;
      }
    }
  for (int v = 1; v < H - 1; ++v)
    for (int u = 1; u < W - 1; ++u) {
      size_t i = (size_t)v * W + u;
      size_t il = i - 1, ir = i + 1, iu = i - W, idn = i + W;
      if (!f->ok[i] || !f->ok[il] || !f->ok[ir] || !f->ok[iu] || !f->ok[idn]) continue;
      double dx[3], dy[3], c[3];
      for (int a = 0; a < 3; ++a) {
        dx[a] = f->P[3 * ir + a] - f->P[3 * il + a];
        dy[a] = f->P[3 * idn + a] - f->P[3 * iu + a];
      }
      c[0] = dx[1] * dy[2] - dx[2] * dy[1];
      c[1] = dx[2] * dy[0] - dx[0] * dy[2];
      c[2] = dx[0] * dy[1] - dx[1] * dy[0];
      double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
      if (!(len > 0.0)) continue;
      for (int a = 0; a < 3; ++a) c[a] /= len;
      const double* P = f->P + 3 * i;
      const double s = c[0] * P[0] + c[1] * P[1] + c[2] * P[2];
      if (s > 0.0)
        for (int a = 0; a < 3; ++a) c[a] = -c[a];
      const double pl = sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
      f->tie[i] = fabs(s) < TIE_N * pl;
      for (int a = 0; a < 3; ++a) f->n[3 * i + a] = c[a];
      f->nok[i] = 1;
    }
  return 0;
}

/* Expose preprocessing: ok, nok, tie (u8 [n]); z (f32 [n]); P, n (f64 [3n]). */
int om_preprocess(const float* depth, int W, int H, float fx, float fy, float cx, float cy, float zmin, float zmax,
                  float dsup, uint8_t* ok, uint8_t* nok, uint8_t* tie, float* zf, double* P, double* nrm) {
  oframe f;
  memset(&f, 0, sizeof(f));
  if (frame_prepare(&f, depth, W, H, fx, fy, cx, cy, zmin, zmax, dsup) != 0) {
    frame_free(&f);
    return -1;
  }
  size_t n = (size_t)W * H;
  if (ok) memcpy(ok, f.ok, n);
  if (nok) memcpy(nok, f.nok, n);
  if (tie) memcpy(tie, f.tie, n);
  if (zf) memcpy(zf, f.z, n * sizeof(float));
  if (P) memcpy(P, f.P, 3 * n * sizeof(double));
  if (nrm) memcpy(nrm, f.n, 3 * n * sizeof(double));
  frame_free(&f);
  return 0;
}

/* ======================================================== allocation (A1) == */
/*
 * Blocks of 8^3 voxels (Sec. 7) are allocated for every (block, D) whose closed cube
 * the segment [p - tau r, p + tau r] meets, for each direction D the pixel's world
 * normal belongs to (Eq. angular_threshold: <n, v^D> > cos(theta)). The blocks are
 * found by testing every block of the segment's bounding box with the exact slab test
 * (the definition itself; an implementation may traverse them with a 3D DDA).
 * A block is a tie when the segment meets the cube grown by TIE_X on every side but
 * not the cube shrunk by TIE_X.
 */

/* Does the segment a + s d, s in [0, 1], meet the closed box [lo, hi]? */
static int seg_box(const double* a, const double* d, const double* lo, const double* hi) {
  double t0 = 0.0, t1 = 1.0;
  for (int k = 0; k < 3; ++k) {
    if (d[k] == 0.0) {
      if (a[k] < lo[k] || a[k] > hi[k]) return 0;
      continue;
    }
    double u0 = (lo[k] - a[k]) / d[k], u1 = (hi[k] - a[k]) / d[k];
    if (u0 > u1) {
      double x = u0;
      u0 = u1;
      u1 = x;
    }
    if (u0 > t0) t0 = u0;
    if (u1 < t1) t1 = u1;
    if (t0 > t1) return 0;
  }
  return 1;
}

/*
 * Blocks met by segment a-b: writes up to max_cells (x, y, z) triples and a flag per
 * cell (bit 0: the segment meets the block's closed cube; bit 1: the decision is a
 * tie). Returns the number of cells with either bit set.
 */
int om_segment_blocks(const double* a, const double* b, double block_size, const double* origin, int32_t* cells,
                      uint8_t* flags, int max_cells) {
  double A[3], d[3];
  int lo[3], hi[3];
  for (int k = 0; k < 3; ++k) {
    A[k] = a[k] - origin[k];
    d[k] = b[k] - a[k];
    const double mn = fmin(a[k], b[k]) - origin[k] - TIE_X, mx = fmax(a[k], b[k]) - origin[k] + TIE_X;
    lo[k] = (int)floor(mn / block_size);
    hi[k] = (int)floor(mx / block_size);
  }
  int n = 0;
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x) {
        const int c[3] = {x, y, z};
        double l0[3], h0[3], lg[3], hg[3], ls[3], hs[3];
        for (int k = 0; k < 3; ++k) {
          l0[k] = c[k] * block_size;
          h0[k] = (c[k] + 1) * block_size;
          lg[k] = l0[k] - TIE_X;
          hg[k] = h0[k] + TIE_X;
          ls[k] = l0[k] + TIE_X;
          hs[k] = h0[k] - TIE_X;
        }
        const int met = seg_box(A, d, l0, h0);
        const int tie = seg_box(A, d, lg, hg) && !seg_box(A, d, ls, hs);
        if (!met && !tie) continue;
        if (n < max_cells) {
          cells[3 * n] = x;
          cells[3 * n + 1] = y;
          cells[3 * n + 2] = z;
          flags[n] = (uint8_t)(met | (tie << 1));
        }
        ++n;
      }
  return n;
}

static void pose_d(const double* T, double R[9], double t[3]) {
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) R[3 * a + b] = T[4 * a + b];
    t[a] = T[4 * a + 3];
  }
}

static void rot_d(const double R[9], const double* x, double* y) {
  for (int a = 0; a < 3; ++a) y[a] = R[3 * a] * x[0] + R[3 * a + 1] * x[1] + R[3 * a + 2] * x[2];
}

#define MAX_SEG_CELLS 128

/*
 * Allocate the (block, D) of one frame. A pixel allocates (block, D) when its normal
 * belongs to D and the segment meets the block; the decision is a tie when the
 * membership cosine is within TIE_N of cos(theta), the block is a tie of the segment
 * test, or the normal's orientation is a tie (a flipped normal belongs to the opposite
 * directions). A key that some pixel allocates with no tie is firm; the other keys a
 * pixel decides with a tie are recorded as allocation ties of this frame.
 */
static int allocate_frame(omap* m, const oframe* f, const double* T, int frame) {
  double R[9], t[3];
  pose_d(T, R, t);
  const double bs = 8.0 * m->h;
  int32_t cells[3 * MAX_SEG_CELLS];
  uint8_t flags[MAX_SEG_CELLS];
  /* candidate tie keys of this frame: (x, y, z, D) */
  size_t ncand = 0, capc = 1024;
  int32_t* cand = (int32_t*)malloc(capc * 4 * sizeof(int32_t));
  /* bricks allocated firmly in this frame */
  size_t fcap = m->brick_cap ? m->brick_cap : 1024;
  uint8_t* firm = NULL;
  if (!cand) return -1;
  for (int v = 0; v < f->H; ++v)
    for (int u = 0; u < f->W; ++u) {
      size_t i = (size_t)v * f->W + u;
      if (!f->nok[i]) continue;
      double nw[3], rv[3], pw[3];
      rot_d(R, f->n + 3 * i, nw);
      int mem[ND], tD[ND], any = 0;
      for (int D = 0; D < ND; ++D) {
        const double c = (D & 1) ? -nw[D >> 1] : nw[D >> 1];
        mem[D] = c > m->costh;
        tD[D] = fabs(c - m->costh) < TIE_N;
      }
      for (int D = 0; D < ND; ++D) {
        if (f->tie[i]) tD[D] |= mem[D] != mem[D ^ 1];
        any |= mem[D] | tD[D];
      }
      if (!any) continue;
      rot_d(R, f->P + 3 * i, rv);
      for (int a = 0; a < 3; ++a) pw[a] = rv[a] + t[a];
      const double len = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
      double A[3], B[3];
      for (int a = 0; a < 3; ++a) {
        A[a] = pw[a] - m->tau * (rv[a] / len);
        B[a] = pw[a] + m->tau * (rv[a] / len);
      }
      int nc = om_segment_blocks(A, B, bs, m->origin, cells, flags, MAX_SEG_CELLS);
      if (nc > MAX_SEG_CELLS) nc = MAX_SEG_CELLS;
      for (int k = 0; k < nc; ++k) {
        const int met = flags[k] & 1, near = (flags[k] >> 1) & 1;
        for (int D = 0; D < ND; ++D) {
          const int* c = cells + 3 * k;
          if (mem[D] && met) {
            const int32_t b = brick_alloc(m, c[0], c[1], c[2], D, frame);
            if (b < 0) {
              free(cand);
              free(firm);
              return -1;
            }
            if (!near && !tD[D]) {
              if ((size_t)b >= fcap || !firm) {
                size_t nf = fcap;
                while ((size_t)b >= nf) nf *= 2;
                uint8_t* x = (uint8_t*)realloc(firm, nf);
                if (!x) {
                  free(cand);
                  free(firm);
                  return -1;
                }
                memset(x + (firm ? fcap : 0), 0, nf - (firm ? fcap : 0));
                firm = x;
                fcap = nf;
              }
              firm[b] = 1;
            }
          }
          if ((mem[D] || tD[D]) && (near || tD[D])) {
            if (ncand == capc) {
              capc *= 2;
              int32_t* x = (int32_t*)realloc(cand, capc * 4 * sizeof(int32_t));
              if (!x) {
                free(cand);
                free(firm);
                return -1;
              }
              cand = x;
            }
            cand[4 * ncand] = c[0];
            cand[4 * ncand + 1] = c[1];
            cand[4 * ncand + 2] = c[2];
            cand[4 * ncand + 3] = D;
            ++ncand;
          }
        }
      }
    }
  int rc = 0;
  for (size_t k = 0; k < ncand && rc == 0; ++k) {
    const int32_t* c = cand + 4 * k;
    const int32_t b = hash_find(m, c[0], c[1], c[2], c[3]);
    if (b >= 0 && firm && (size_t)b < fcap && firm[b]) continue;
    rc = tie_key_put(m, c[0], c[1], c[2], c[3], frame);
  }
  free(cand);
  free(firm);
  return rc;
}

/* ============================================================ fusion (A2) == */

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* Eq. direction_weight, as read: 1 in the exclusive zone, 0 beyond theta, linear in between. */
double om_w_dir(double cos_angle, double theta) {
  double alpha = acos(clampd(cos_angle, -1.0, 1.0));
  return clampd((theta - alpha) / (2.0 * theta - M_PI / 2.0), 0.0, 1.0);
}

/* distance of x + 1/2 to the nearest integer: the rounding floor(x + 1/2) is a tie below TIE_PX */
static int round_tie(double x) {
  const double s = x + 0.5;
  return fabs(s - floor(s + 0.5)) < TIE_PX;
}

/*
 * Voxel-projection fusion (Sec. 3). Every voxel of every allocated (block, D) is
 * projected into the frame; the nearest pixel supplies p and n; the point-to-plane
 * distance decides between carving (in front of the band, Sec. 3), the running-average
 * update with the combined weight of Eq. combined_fusion_weight (inside the band) and
 * nothing (behind it). A voxel is marked as a tie (bit 0; bit 1 for colour alone) when
 * one of the decisions about it in this frame lies within its margin: camera depth
 * near 0, a projection near a pixel boundary, a tie of the pixel's normal, the band
 * edges (TIE_X plus TIE_N times |x - p|), the direction membership or the colour radius.
 * The whole brick is marked when its allocation was a tie in a frame before or at the
 * one that allocated it here.
 */
static int fuse_frame(omap* m, const oframe* f, const uint8_t* rgb, const double* T) {
  double R[9], t[3];
  pose_d(T, R, t);
  const int W = f->W, H = f->H;
  const double tau = m->tau;
#pragma omp parallel for schedule(dynamic, 16)
  for (long b = 0; b < (long)m->nbricks; ++b) {
    const int32_t* bc = m->coord + 4 * b;
    const int D = bc[3];
    ovox* vb = m->vox + (size_t)b * BVOX;
    uint8_t* tb = m->tie + (size_t)b * BVOX;
    if (m->dense_dim <= 0) {
      const int32_t tf = tie_key_find(m, bc[0], bc[1], bc[2], D);
      if (tf >= 0 && tf <= m->first_frame[b]) memset(tb, 3, BVOX);
    }
    for (int k = 0; k < BLK; ++k)
      for (int j = 0; j < BLK; ++j)
        for (int i = 0; i < BLK; ++i) {
          const int vi = (k * BLK + j) * BLK + i;
          const int gi[3] = {BLK * bc[0] + i, BLK * bc[1] + j, BLK * bc[2] + k};
          double x[3], rel[3], xc[3];
          for (int a = 0; a < 3; ++a) {
            x[a] = gi[a] * m->h + m->origin[a];
            rel[a] = x[a] - t[a];
          }
          for (int a = 0; a < 3; ++a) xc[a] = R[a] * rel[0] + R[3 + a] * rel[1] + R[6 + a] * rel[2];
          if (!(xc[2] > 0.0)) {
            if (fabs(xc[2]) < TIE_X) tb[vi] |= 3;
            continue;
          }
          const double uf = (xc[0] / xc[2]) * f->fx + f->cx;
          const double vf = (xc[1] / xc[2]) * f->fy + f->cy;
          const int tie_proj = round_tie(uf) || round_tie(vf);
          const double ur = floor(uf + 0.5), vr = floor(vf + 0.5);
          if (!(ur >= 0.0 && vr >= 0.0 && ur < (double)W && vr < (double)H)) {
            if (tie_proj) tb[vi] |= 3;
            continue;
          }
          const int u = (int)ur, v = (int)vr;
          const size_t pi = (size_t)v * W + u;
          if (!f->nok[pi]) {
            if (tie_proj) tb[vi] |= 3;
            continue;
          }
          const double* P = f->P + 3 * pi;
          const double* n = f->n + 3 * pi;
          double e[3];
          for (int a = 0; a < 3; ++a) e[a] = xc[a] - P[a];
          const double draw = e[0] * n[0] + e[1] * n[1] + e[2] * n[2];
          const double dist = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
          const double band_eps = TIE_X + TIE_N * dist;
          int tie = tie_proj || f->tie[pi];
          ovox* vx = vb + vi;
          if (draw < -tau) {
            if (tie || fabs(draw + tau) < band_eps) tb[vi] |= 3;
            continue;
          }
          if (draw > tau) {
            if (tie || fabs(draw - tau) < band_eps) tb[vi] |= 3;
            /* free-space carving, unless a depth jump > tau lies within the carve radius */
            int jump = 0;
            const double zc = f->z[pi];
            for (int dv = -m->carve_r; dv <= m->carve_r && !jump; ++dv)
              for (int du = -m->carve_r; du <= m->carve_r; ++du) {
                int uu = u + du, vv = v + dv;
                if (uu < 0 || vv < 0 || uu >= W || vv >= H) continue;
                size_t qi = (size_t)vv * W + uu;
                if (!f->ok[qi]) continue;
                if (fabs((double)f->z[qi] - zc) > tau) {
                  jump = 1;
                  break;
                }
              }
            if (jump) continue;
            double wn = vx->w + m->wcarve;
            vx->sdf = (vx->w * vx->sdf + m->wcarve * 1.0) / wn;
            vx->w = wn < m->wmax ? wn : m->wmax;
            continue;
          }
          if (fabs(draw + tau) < band_eps || fabs(draw - tau) < band_eps) tie = 1;
          /* membership of the pixel normal in direction D (Eq. angular_threshold) */
          double nw[3];
          rot_d(R, n, nw);
          const double cd = (D & 1) ? -nw[D >> 1] : nw[D >> 1];
          if (fabs(cd - m->costh) < TIE_N) tie = 1;
          if (tie) tb[vi] |= 3;
          if (!(cd > m->costh)) continue;
          const double np = n[0] * P[0] + n[1] * P[1] + n[2] * P[2];
          if (!(np < 0.0)) continue;
          const double d = clampd(draw / tau, -1.0, 1.0);
          const double zp = P[2];
          const double w_depth = 1.0 / ((zp + 1.0 - m->zmin) * (zp + 1.0 - m->zmin));
          const double pl = sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
          const double w_angle = -np / pl;
          const double w_d = w_depth * w_angle * om_w_dir(cd, m->theta);
          const double wn = vx->w + w_d;
          vx->sdf = (vx->w * vx->sdf + w_d * d) / wn;
          vx->w = wn < m->wmax ? wn : m->wmax;
          if (m->color && rgb) {
            /* colour is fused only within tau of the observed point (Eq. color_weight) */
            if (fabs(dist - tau) < TIE_X) tb[vi] |= 2;
            if (dist < tau) {
              const double w_c = w_d * (1.0 - dist / tau);
              const uint8_t* c = rgb + 3 * pi;
              double wcn = vx->wc + w_c;
              vx->r = (vx->wc * vx->r + w_c * c[0]) / wcn;
              vx->g = (vx->wc * vx->g + w_c * c[1]) / wcn;
              vx->b = (vx->wc * vx->b + w_c * c[2]) / wcn;
              vx->wc = wcn < m->wmax ? wcn : m->wmax;
            }
          }
        }
  }
  return 0;
}

/* Fuse one frame: preprocess, allocate (hash mode only), voxel-projection fusion. */
int om_integrate(omap* m, const float* depth, const uint8_t* rgb, int W, int H, float fx, float fy, float cx,
                 float cy, const double* T_wc) {
  oframe f;
  memset(&f, 0, sizeof(f));
  int rc = frame_prepare(&f, depth, W, H, fx, fy, cx, cy, m->zmin, m->zmax, m->dsup);
  if (rc == 0 && m->dense_dim <= 0) rc = allocate_frame(m, &f, T_wc, m->frames);
  if (rc == 0) rc = fuse_frame(m, &f, rgb, T_wc);
  frame_free(&f);
  m->frames++;
  return rc;
}

/* ============================================================ render (A3-A5) */

typedef struct {
  int present;
  double phi, w, wc, col[3];
  int has_grad;
  double n[3];
} dsample;

/* Counting context of om_render_count (per thread; NULL in ordinary renders): the bricks whose
   voxels the march reads, the block cells whose hash entry it reads, and the colour voxels that
   enter the outputs. */
typedef struct {
  uint8_t* geom;   /* per brick */
  uint8_t* probe;  /* per brick: set on one brick of each probed block */
  uint8_t* colvox; /* per voxel (brick * 512 + voxel) */
} ocount;
static __thread const ocount* g_cnt = NULL;
static __thread int g_cnt_out = 0;

static void mark(uint8_t* p) { __atomic_store_n(p, (uint8_t)1, __ATOMIC_RELAXED); }

/* Trilinear sample of direction D at continuous voxel coordinate g (voxel units from the origin). */
static int trilinear(const omap* m, int D, const double* g, double* phi, double* w, double* wc, double* col) {
  double fl[3], fr[3];
  int b[3];
  for (int a = 0; a < 3; ++a) {
    fl[a] = floor(g[a]);
    fr[a] = g[a] - fl[a];
    b[a] = (int)fl[a];
  }
  double acc_s = 0, acc_w = 0, acc_wc = 0, acc_c[3] = {0, 0, 0};
  for (int c = 0; c < 8; ++c) {
    int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    int vi[3];
    double wt = 1.0;
    for (int a = 0; a < 3; ++a) {
      vi[a] = b[a] + o[a];
      wt *= o[a] ? fr[a] : 1.0 - fr[a];
    }
    int bx = (int)floor(vi[0] / 8.0), by = (int)floor(vi[1] / 8.0), bz = (int)floor(vi[2] / 8.0);
    int32_t br = hash_find(m, bx, by, bz, D);
    if (br < 0) return 0;
    if (g_cnt) mark(g_cnt->geom + br);
    const ovox* vx = m->vox + (size_t)br * BVOX + ((vi[2] - 8 * bz) * 8 + (vi[1] - 8 * by)) * 8 + (vi[0] - 8 * bx);
    if (!(vx->w > 0)) return 0;
    acc_s += wt * vx->sdf;
    acc_w += wt * vx->w;
    acc_wc += wt * vx->wc;
    acc_c[0] += wt * vx->r;
    acc_c[1] += wt * vx->g;
    acc_c[2] += wt * vx->b;
  }
  *phi = acc_s;
  if (w) *w = acc_w;
  if (wc) *wc = acc_wc;
  if (col) {
    col[0] = acc_c[0];
    col[1] = acc_c[1];
    col[2] = acc_c[2];
  }
  return 1;
}

static void sample_dir(const omap* m, int D, const double* x, dsample* s) {
  double g[3];
  for (int a = 0; a < 3; ++a) g[a] = (x[a] - m->origin[a]) / m->h;
  s->present = trilinear(m, D, g, &s->phi, &s->w, &s->wc, s->col);
  s->has_grad = 0;
  if (!s->present) return;
  double grad[3];
  for (int a = 0; a < 3; ++a) {
    double gp[3] = {g[0], g[1], g[2]}, gm[3] = {g[0], g[1], g[2]};
    gp[a] += 1.0;
    gm[a] -= 1.0;
    double fp, fm;
    if (!trilinear(m, D, gp, &fp, NULL, NULL, NULL)) return;
    if (!trilinear(m, D, gm, &fm, NULL, NULL, NULL)) return;
    grad[a] = (fp - fm) / (2.0 * m->h);
  }
  double nrm = sqrt(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]);
  if (!(nrm > 1e-12)) return;
  for (int a = 0; a < 3; ++a) s->n[a] = grad[a] / nrm;
  s->has_grad = 1;
}

/*
 * Combined SDF at world point x for unit view ray r (Eq. combine_weight, with the
 * Eq. combine_tsdf_weight fallback). Returns 1 if defined. wsum_comb receives the
 * sum of combination weights (0 when the fallback was used).
 */
typedef struct {
  double phi, wsum_comb;
  double n[3];
  int ncomb;
  double col[3];
  int col_ok;
} combo;

static int combine(const omap* m, const double* x, const double* r, combo* out) {
  dsample s[ND];
  double ws = 0, acc = 0, nacc[3] = {0, 0, 0}, cw = 0, cacc[3] = {0, 0, 0};
  int any = 0;
  for (int D = 0; D < ND; ++D) {
    sample_dir(m, D, x, &s[D]);
    if (!s[D].present) continue;
    any = 1;
    if (!s[D].has_grad) continue;
    double cosv = (D & 1) ? -s[D].n[D >> 1] : s[D].n[D >> 1];
    double facing = -(s[D].n[0] * r[0] + s[D].n[1] * r[1] + s[D].n[2] * r[2]);
    if (facing < 0) facing = 0;
    double wcomb = om_w_dir(cosv, m->theta) * facing * s[D].w;
    if (!(wcomb > 0)) continue;
    ws += wcomb;
    acc += wcomb * s[D].phi;
    for (int a = 0; a < 3; ++a) nacc[a] += wcomb * s[D].n[a];
    if (s[D].wc > 0) {
      cw += wcomb;
      for (int a = 0; a < 3; ++a) cacc[a] += wcomb * s[D].col[a];
      if (g_cnt && g_cnt_out) {
        /* the 8 colour voxels of direction D that enter the output */
        for (int q = 0; q < 8; ++q) {
          int vi[3];
          for (int a = 0; a < 3; ++a) vi[a] = (int)floor((x[a] - m->origin[a]) / m->h) + ((q >> a) & 1);
          const int bx = (int)floor(vi[0] / 8.0), by = (int)floor(vi[1] / 8.0), bz = (int)floor(vi[2] / 8.0);
          const int32_t br = hash_find(m, bx, by, bz, D);
          if (br >= 0)
            mark(g_cnt->colvox + (size_t)br * BVOX + ((vi[2] - 8 * bz) * 8 + (vi[1] - 8 * by)) * 8 + (vi[0] - 8 * bx));
        }
      }
    }
  }
  if (!any) return 0;
  out->col_ok = 0;
  if (ws > 0) {
    out->phi = acc / ws;
    out->wsum_comb = ws;
    double nl = sqrt(nacc[0] * nacc[0] + nacc[1] * nacc[1] + nacc[2] * nacc[2]);
    for (int a = 0; a < 3; ++a) out->n[a] = nl > 0 ? nacc[a] / nl : 0.0;
    out->ncomb = nl > 0;
    if (cw > 0) {
      for (int a = 0; a < 3; ++a) out->col[a] = cacc[a] / cw;
      out->col_ok = 1;
    }
    return 1;
  }
  double wf = 0, af = 0;
  for (int D = 0; D < ND; ++D) {
    if (!s[D].present) continue;
    double facing = -(VDIR[D][0] * r[0] + VDIR[D][1] * r[1] + VDIR[D][2] * r[2]);
    if (facing < 0) facing = 0;
    double w = s[D].w * facing;
    if (!(w > 0)) continue;
    wf += w;
    af += w * s[D].phi;
  }
  if (!(wf > 0)) return 0;
  out->phi = af / wf;
  out->wsum_comb = 0;
  out->ncomb = 0;
  return 1;
}

/* Exposed for tests: combined SDF at a world point. Returns 1 if defined; info = phi, wsum, n[3], col[3], col_ok. */
int om_eval(const omap* m, const double* x, const double* r, double* info) {
  combo c;
  memset(&c, 0, sizeof(c));
  int ok = combine(m, x, r, &c);
  info[0] = c.phi;
  info[1] = c.wsum_comb;
  for (int a = 0; a < 3; ++a) {
    info[2 + a] = c.n[a];
    info[5 + a] = c.col[a];
  }
  info[8] = c.col_ok;
  return ok;
}

static int cell_has_any(const omap* m, int cx, int cy, int cz) {
  for (int D = 0; D < ND; ++D) {
    const int32_t b = hash_find(m, cx, cy, cz, D);
    if (b >= 0) {
      if (g_cnt) mark(g_cnt->probe + b);
      return 1;
    }
  }
  return 0;
}

/*
 * Ray-cast one pixel (Sec. 4). Outputs depth (z, 0 = miss), camera-frame normal,
 * colour and colour validity. Returns 1 on a hit.
 */
static int render_pixel(const omap* m, const double* T, double fx, double fy, double cx, double cy, int u, int v,
                        double* depth, double* ncam, double* col, int* col_ok) {
  double rc[3] = {((double)u - cx) / fx, ((double)v - cy) / fy, 1.0};
  double rl = sqrt(rc[0] * rc[0] + rc[1] * rc[1] + rc[2] * rc[2]);
  double r[3], o[3] = {T[3], T[7], T[11]};
  for (int a = 0; a < 3; ++a) r[a] = (T[4 * a] * rc[0] + T[4 * a + 1] * rc[1] + T[4 * a + 2] * rc[2]) / rl;
  double step = 0.5 * m->h;
  double tn = m->zmin * rl, tf = m->zmax * rl;
  long k0 = (long)ceil(tn / step), k1 = (long)floor(tf / step);
  int prev_def = 0;
  double prev_phi = 0, prev_t = 0;
  int cell[3] = {0x7fffffff, 0, 0}, cell_any = 0;
  double bs = 8.0 * m->h;
  for (long k = k0; k <= k1; ++k) {
    double t = k * step;
    double x[3] = {o[0] + t * r[0], o[1] + t * r[1], o[2] + t * r[2]};
    int c[3];
    for (int a = 0; a < 3; ++a) c[a] = (int)floor((x[a] - m->origin[a]) / bs);
    if (c[0] != cell[0] || c[1] != cell[1] || c[2] != cell[2]) {
      cell[0] = c[0];
      cell[1] = c[1];
      cell[2] = c[2];
      cell_any = cell_has_any(m, c[0], c[1], c[2]);
    }
    combo cb;
    if (!cell_any || !combine(m, x, r, &cb)) {
      prev_def = 0;
      continue;
    }
    if (prev_def && prev_phi > 0 && cb.phi <= 0) {
      /* the hit: the root of the continuous Phi(t) in [prev_t, t] (Sec. 4: small steps
         after the regular probing), by bisection; an undefined midpoint counts as free
         space. Normal and colour at the root's non-positive side (hi, within 1e-10 m),
         where Phi is defined; a miss if no direction has a combination weight there. */
      double lo = prev_t, hi = t;
      while (hi - lo > ROOT_TOL) {
        const double tm = 0.5 * (lo + hi);
        const double xm[3] = {o[0] + tm * r[0], o[1] + tm * r[1], o[2] + tm * r[2]};
        combo cm;
        if (combine(m, xm, r, &cm) && cm.phi <= 0)
          hi = tm;
        else
          lo = tm;
      }
      const double ts = 0.5 * (lo + hi);
      const double xs[3] = {o[0] + hi * r[0], o[1] + hi * r[1], o[2] + hi * r[2]};
      combo ch;
      g_cnt_out = 1;
      const int have = combine(m, xs, r, &ch) && ch.wsum_comb > 0 && ch.ncomb;
      g_cnt_out = 0;
      if (!have) return 0;
      *depth = ts / rl;
      for (int a = 0; a < 3; ++a) ncam[a] = T[a] * ch.n[0] + T[4 + a] * ch.n[1] + T[8 + a] * ch.n[2];
      if (ch.col_ok)
        for (int a = 0; a < 3; ++a) col[a] = ch.col[a];
      *col_ok = ch.col_ok;
      return 1;
    }
    prev_def = 1;
    prev_phi = cb.phi;
    prev_t = t;
  }
  return 0;
}

/*
 * Render pixels. If pix is NULL all W*H pixels are rendered (row-major);
 * otherwise npix (u, v) pairs. Outputs per rendered pixel: depth (0 = miss),
 * normal (3, camera frame), colour (3, 0..255) and colour validity.
 */
int om_render(const omap* m, const double* T_wc, int W, int H, float fx, float fy, float cx, float cy,
              const int32_t* pix, long npix, double* depth, double* normal, double* color, uint8_t* color_ok) {
  long n = pix ? npix : (long)W * H;
#pragma omp parallel for schedule(dynamic, 64)
  for (long i = 0; i < n; ++i) {
    int u = pix ? pix[2 * i] : (int)(i % W);
    int v = pix ? pix[2 * i + 1] : (int)(i / W);
    double d = 0, nc[3] = {0, 0, 0}, col[3] = {0, 0, 0};
    int cok = 0;
    if (!render_pixel(m, T_wc, fx, fy, cx, cy, u, v, &d, nc, col, &cok)) {
      d = 0;
      nc[0] = nc[1] = nc[2] = 0;
      cok = 0;
    }
    depth[i] = d;
    if (normal)
      for (int a = 0; a < 3; ++a) normal[3 * i + a] = nc[a];
    if (color)
      for (int a = 0; a < 3; ++a) color[3 * i + a] = cok ? col[a] : 0.0;
    if (color_ok) color_ok[i] = (uint8_t)cok;
  }
  return 0;
}

/*
 * The algorithmic bytes of a render: render pixels as om_render does (pix NULL: all W*H) and
 * count the distinct bricks whose voxels the march reads (counts[0]), the distinct allocated
 * block cells whose hash entry it reads (counts[1]), the distinct colour voxels that enter the
 * outputs (counts[2]) and the hits (counts[3]).
 */
int om_render_count(const omap* m, const double* T_wc, int W, int H, float fx, float fy, float cx, float cy,
                    const int32_t* pix, long npix, int64_t* counts) {
  ocount c;
  c.geom = (uint8_t*)calloc(m->nbricks + 1, 1);
  c.probe = (uint8_t*)calloc(m->nbricks + 1, 1);
  c.colvox = (uint8_t*)calloc((m->nbricks + 1) * BVOX, 1);
  if (!c.geom || !c.probe || !c.colvox) {
    free(c.geom);
    free(c.probe);
    free(c.colvox);
    return -1;
  }
  long n = pix ? npix : (long)W * H;
  int64_t hits = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : hits)
  for (long i = 0; i < n; ++i) {
    g_cnt = &c;
    int u = pix ? pix[2 * i] : (int)(i % W);
    int v = pix ? pix[2 * i + 1] : (int)(i / W);
    double d = 0, nc[3], col[3];
    int cok = 0;
    hits += render_pixel(m, T_wc, fx, fy, cx, cy, u, v, &d, nc, col, &cok);
    g_cnt = NULL;
  }
  int64_t ng = 0, np = 0, nc = 0;
  for (size_t b = 0; b < m->nbricks; ++b) {
    ng += c.geom[b];
    np += c.probe[b];
  }
  for (size_t i = 0; i < m->nbricks * BVOX; ++i) nc += c.colvox[i];
  counts[0] = ng;
  counts[1] = np;
  counts[2] = nc;
  counts[3] = hits;
  free(c.geom);
  free(c.probe);
  free(c.colvox);
  return 0;
}

/* Threads of the oracle's parallel loops (OpenMP); 0 keeps the current setting. Returns the
   number that the next parallel loop will use. */
int om_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ====================================================== combined TSDF (Sec. 4, Sec. 7) */
/*
 * View-dependent combined TSDF. Sec. 4: the combined SDF can be pre-computed for every voxel of
 * the view frustum and then ray-cast like a regular TSDF from the pose of the combination.
 * Sec. 7: the lookups are at integer voxel positions, so no trilinear interpolation is needed
 * and a direction's gradient comes from its 6 neighbouring voxels. Readings:
 *   combined value at voxel v for the camera centre c: every direction D with W^D(v) > 0
 *   takes part; its gradient is the central difference of its 6 axis neighbours (all with
 *   weight > 0, norm > 1e-12); the view ray is r = (x_v - c) / |x_v - c|; the weights are
 *   those of Eq. combine_weight, with the fallback of Eq. combine_tsdf_weight when they all
 *   vanish; otherwise the voxel is undefined. The colour is the combination of the colours of
 *   the directions with a combination weight and a colour weight > 0 (none after the fallback).
 *   Here every allocated block is combined (the kernels combine the blocks of the padded view
 *   frustum, which hold every voxel a ray of that view reads).
 *   ray-cast: the rules of the direct render (samples at t = k h/2, the first pair of
 *   consecutive defined samples with Phi > 0 >= Phi, bisection to the root of Phi(t) in
 *   that bracket, outputs at its non-positive side) with Phi the trilinear interpolation of the combined values
 *   (defined if all 8 corners are), the normal the central difference of that field at +-h
 *   (defined if the 6 offset samples are, norm > 1e-12) and the colour the trilinear
 *   interpolation of the combined colours (where all 8 corners have one).
 */

static int floor8(int x) { return x >= 0 ? x / 8 : -((-x + 7) / 8); }

static const ovox* vox_at(const omap* m, int D, int x, int y, int z) {
  const int bx = floor8(x), by = floor8(y), bz = floor8(z);
  const int32_t br = hash_find(m, bx, by, bz, D);
  if (br < 0) return NULL;
  return m->vox + (size_t)br * BVOX + ((z - 8 * bz) * 8 + (y - 8 * by)) * 8 + (x - 8 * bx);
}

static uint64_t block_key(int bx, int by, int bz) { return pack_key(bx, by, bz, 0); }

static int32_t cblock_find(const omap* m, int bx, int by, int bz) {
  if (!m->ckeys) return -1;
  const uint64_t k = block_key(bx, by, bz);
  size_t i = mix64(k) & (m->ccap - 1);
  for (;;) {
    if (m->ckeys[i] == k) return m->cvals[i];
    if (m->ckeys[i] == EMPTY_KEY) return -1;
    i = (i + 1) & (m->ccap - 1);
  }
}

/* combined value of voxel (x, y, z) for the camera centre c; returns 1 if defined */
static int comb_voxel(const omap* m, int x, int y, int z, const double* c, double* phi, double* col, int* col_ok) {
  const double xw[3] = {m->origin[0] + x * m->h, m->origin[1] + y * m->h, m->origin[2] + z * m->h};
  double r[3] = {xw[0] - c[0], xw[1] - c[1], xw[2] - c[2]};
  const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  for (int a = 0; a < 3; ++a) r[a] /= rn;
  double ws = 0, acc = 0, wf = 0, af = 0, cw = 0, cacc[3] = {0, 0, 0};
  int any = 0;
  for (int D = 0; D < ND; ++D) {
    const ovox* v0 = vox_at(m, D, x, y, z);
    if (!v0 || !(v0->w > 0)) continue;
    any = 1;
    double ff = -(VDIR[D][0] * r[0] + VDIR[D][1] * r[1] + VDIR[D][2] * r[2]);
    if (ff < 0) ff = 0;
    const double w_f = v0->w * ff;
    if (w_f > 0) {
      wf += w_f;
      af += w_f * v0->sdf;
    }
    double g[3];
    int ok = 1;
    for (int a = 0; a < 3 && ok; ++a) {
      const int e[3] = {a == 0, a == 1, a == 2};
      const ovox* p = vox_at(m, D, x + e[0], y + e[1], z + e[2]);
      const ovox* q = vox_at(m, D, x - e[0], y - e[1], z - e[2]);
      if (!p || !q || !(p->w > 0) || !(q->w > 0)) {
        ok = 0;
        break;
      }
      g[a] = (p->sdf - q->sdf) / (2.0 * m->h);
    }
    if (!ok) continue;
    const double nrm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (!(nrm > 1e-12)) continue;
    const double n[3] = {g[0] / nrm, g[1] / nrm, g[2] / nrm};
    const double cosv = (D & 1) ? -n[D >> 1] : n[D >> 1];
    double facing = -(n[0] * r[0] + n[1] * r[1] + n[2] * r[2]);
    if (facing < 0) facing = 0;
    const double wc = om_w_dir(cosv, m->theta) * facing * v0->w;
    if (!(wc > 0)) continue;
    ws += wc;
    acc += wc * v0->sdf;
    if (v0->wc > 0) {
      cw += wc;
      cacc[0] += wc * v0->r;
      cacc[1] += wc * v0->g;
      cacc[2] += wc * v0->b;
    }
  }
  *col_ok = 0;
  if (!any) return 0;
  if (ws > 0) {
    *phi = acc / ws;
    if (cw > 0) {
      for (int a = 0; a < 3; ++a) col[a] = cacc[a] / cw;
      *col_ok = 1;
    }
    return 1;
  }
  if (wf > 0) {
    *phi = af / wf;
    return 1;
  }
  return 0;
}

/* Combine every allocated block for the camera centre c (replaces an earlier combination). */
int om_combine(omap* m, const double* c) {
  free(m->ckeys);
  free(m->cvals);
  free(m->comb);
  free(m->comb_col);
  m->ckeys = NULL;
  m->cvals = NULL;
  m->comb = NULL;
  m->comb_col = NULL;
  /* distinct blocks */
  size_t cap = 64;
  while (cap < 4 * m->nbricks + 64) cap <<= 1;
  m->ccap = cap;
  m->ckeys = (uint64_t*)malloc(cap * sizeof(uint64_t));
  m->cvals = (int32_t*)malloc(cap * sizeof(int32_t));
  int32_t* bl = (int32_t*)malloc(3 * (m->nbricks + 1) * sizeof(int32_t));
  if (!m->ckeys || !m->cvals || !bl) return -1;
  memset(m->ckeys, 0xFF, cap * sizeof(uint64_t));
  size_t nb = 0;
  for (size_t b = 0; b < m->nbricks; ++b) {
    const int bx = m->coord[4 * b], by = m->coord[4 * b + 1], bz = m->coord[4 * b + 2];
    const uint64_t k = block_key(bx, by, bz);
    size_t i = mix64(k) & (cap - 1);
    while (m->ckeys[i] != EMPTY_KEY && m->ckeys[i] != k) i = (i + 1) & (cap - 1);
    if (m->ckeys[i] == k) continue;
    m->ckeys[i] = k;
    m->cvals[i] = (int32_t)nb;
    bl[3 * nb] = bx;
    bl[3 * nb + 1] = by;
    bl[3 * nb + 2] = bz;
    ++nb;
  }
  m->nblocks = nb;
  m->comb = (double*)malloc(nb * BVOX * 5 * sizeof(double));
  m->comb_col = (uint8_t*)malloc(nb * BVOX);
  if (!m->comb || !m->comb_col) {
    free(bl);
    return -1;
  }
#pragma omp parallel for schedule(dynamic, 4)
  for (long b = 0; b < (long)nb; ++b) {
    for (int vi = 0; vi < BVOX; ++vi) {
      const int x = 8 * bl[3 * b] + (vi & 7), y = 8 * bl[3 * b + 1] + ((vi >> 3) & 7), z = 8 * bl[3 * b + 2] + (vi >> 6);
      double phi = 0, col[3] = {0, 0, 0};
      int cok = 0;
      const int def = comb_voxel(m, x, y, z, c, &phi, col, &cok);
      double* o = m->comb + ((size_t)b * BVOX + vi) * 5;
      o[0] = def ? phi : 0.0;
      o[1] = def;
      o[2] = col[0];
      o[3] = col[1];
      o[4] = col[2];
      m->comb_col[(size_t)b * BVOX + vi] = (uint8_t)(def && cok);
    }
  }
  free(bl);
  return 0;
}

/* combined voxel (x, y, z) of the last om_combine, NULL if undefined */
static const double* cvox(const omap* m, int x, int y, int z, int* col_ok) {
  const int bx = floor8(x), by = floor8(y), bz = floor8(z);
  const int32_t cb = cblock_find(m, bx, by, bz);
  if (cb < 0) return NULL;
  const size_t vi = (size_t)cb * BVOX + ((z - 8 * bz) * 8 + (y - 8 * by)) * 8 + (x - 8 * bx);
  const double* o = m->comb + vi * 5;
  if (!(o[1] > 0)) return NULL;
  *col_ok = m->comb_col[vi];
  return o;
}

/* trilinear combined field at voxel coordinate g; returns 1 if all 8 corners are defined */
static int comb_tri(const omap* m, const double* g, double* phi, double* col, int* col_ok) {
  double fl[3], fr[3];
  int b[3];
  for (int a = 0; a < 3; ++a) {
    fl[a] = floor(g[a]);
    fr[a] = g[a] - fl[a];
    b[a] = (int)fl[a];
  }
  double acc = 0, cacc[3] = {0, 0, 0};
  int all_col = 1;
  for (int q = 0; q < 8; ++q) {
    const int o[3] = {q & 1, (q >> 1) & 1, (q >> 2) & 1};
    double wt = 1.0;
    for (int a = 0; a < 3; ++a) wt *= o[a] ? fr[a] : 1.0 - fr[a];
    int cok = 0;
    const double* v = cvox(m, b[0] + o[0], b[1] + o[1], b[2] + o[2], &cok);
    if (!v) return 0;
    acc += wt * v[0];
    all_col &= cok;
    for (int a = 0; a < 3; ++a) cacc[a] += wt * v[2 + a];
  }
  *phi = acc;
  if (col) {
    *col_ok = all_col;
    for (int a = 0; a < 3; ++a) col[a] = cacc[a];
  }
  return 1;
}

/* combined field at world point x: value, normal (world, 1 if defined) and colour */
typedef struct {
  double phi, n[3], col[3];
  int has_n, col_ok;
} csample;

static int comb_eval(const omap* m, const double* x, csample* s) {
  double g[3];
  for (int a = 0; a < 3; ++a) g[a] = (x[a] - m->origin[a]) / m->h;
  if (!comb_tri(m, g, &s->phi, s->col, &s->col_ok)) return 0;
  s->has_n = 0;
  double gr[3];
  for (int a = 0; a < 3; ++a) {
    double gp[3] = {g[0], g[1], g[2]}, gm[3] = {g[0], g[1], g[2]};
    gp[a] += 1.0;
    gm[a] -= 1.0;
    double fp, fm;
    if (!comb_tri(m, gp, &fp, NULL, NULL) || !comb_tri(m, gm, &fm, NULL, NULL)) return 1;
    gr[a] = (fp - fm) / (2.0 * m->h);
  }
  const double nrm = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
  if (!(nrm > 1e-12)) return 1;
  for (int a = 0; a < 3; ++a) s->n[a] = gr[a] / nrm;
  s->has_n = 1;
  return 1;
}

static int render_pixel_comb(const omap* m, const double* T, double fx, double fy, double cx, double cy, int u, int v,
                             double* depth, double* ncam, double* col, int* col_ok) {
  double rc[3] = {((double)u - cx) / fx, ((double)v - cy) / fy, 1.0};
  double rl = sqrt(rc[0] * rc[0] + rc[1] * rc[1] + rc[2] * rc[2]);
  double r[3], o[3] = {T[3], T[7], T[11]};
  for (int a = 0; a < 3; ++a) r[a] = (T[4 * a] * rc[0] + T[4 * a + 1] * rc[1] + T[4 * a + 2] * rc[2]) / rl;
  const double step = 0.5 * m->h;
  const long k0 = (long)ceil(m->zmin * rl / step), k1 = (long)floor(m->zmax * rl / step);
  int prev_def = 0;
  double prev_phi = 0, prev_t = 0;
  for (long k = k0; k <= k1; ++k) {
    const double t = k * step;
    const double x[3] = {o[0] + t * r[0], o[1] + t * r[1], o[2] + t * r[2]};
    csample cs;
    if (!comb_eval(m, x, &cs)) {
      prev_def = 0;
      continue;
    }
    if (prev_def && prev_phi > 0 && cs.phi <= 0) {
      /* bisection to the root of the combined field, outputs at the root (as the direct render) */
      double lo = prev_t, hi = t;
      while (hi - lo > ROOT_TOL) {
        const double tm = 0.5 * (lo + hi);
        const double xm[3] = {o[0] + tm * r[0], o[1] + tm * r[1], o[2] + tm * r[2]};
        csample cm;
        if (comb_eval(m, xm, &cm) && cm.phi <= 0)
          hi = tm;
        else
          lo = tm;
      }
      const double ts = 0.5 * (lo + hi);
      const double xs[3] = {o[0] + hi * r[0], o[1] + hi * r[1], o[2] + hi * r[2]};
      csample ch;
      if (!(comb_eval(m, xs, &ch) && ch.has_n)) return 0;
      *depth = ts / rl;
      for (int a = 0; a < 3; ++a) ncam[a] = T[a] * ch.n[0] + T[4 + a] * ch.n[1] + T[8 + a] * ch.n[2];
      *col_ok = ch.col_ok;
      if (ch.col_ok)
        for (int a = 0; a < 3; ++a) col[a] = ch.col[a];
      return 1;
    }
    prev_def = 1;
    prev_phi = cs.phi;
    prev_t = t;
  }
  return 0;
}

/* Ray-cast the combined TSDF of the last om_combine (outputs as om_render). */
int om_render_combined(const omap* m, const double* T_wc, int W, int H, float fx, float fy, float cx, float cy,
                       const int32_t* pix, long npix, double* depth, double* normal, double* color,
                       uint8_t* color_ok) {
  if (!m->comb) return -1;
  long n = pix ? npix : (long)W * H;
#pragma omp parallel for schedule(dynamic, 64)
  for (long i = 0; i < n; ++i) {
    int u = pix ? pix[2 * i] : (int)(i % W);
    int v = pix ? pix[2 * i + 1] : (int)(i / W);
    double d = 0, nc[3] = {0, 0, 0}, col[3] = {0, 0, 0};
    int cok = 0;
    if (!render_pixel_comb(m, T_wc, fx, fy, cx, cy, u, v, &d, nc, col, &cok)) {
      d = 0;
      nc[0] = nc[1] = nc[2] = 0;
      cok = 0;
    }
    depth[i] = d;
    if (normal)
      for (int a = 0; a < 3; ++a) normal[3 * i + a] = nc[a];
    if (color)
      for (int a = 0; a < 3; ++a) color[3 * i + a] = cok ? col[a] : 0.0;
    if (color_ok) color_ok[i] = (uint8_t)cok;
  }
  return 0;
}

/* Exposed for tests: combined value of voxel (x, y, z) for camera centre c; info = phi, r, g, b, colour ok. */
int om_comb_voxel(const omap* m, int x, int y, int z, const double* c, double* info) {
  double phi = 0, col[3] = {0, 0, 0};
  int cok = 0;
  const int def = comb_voxel(m, x, y, z, c, &phi, col, &cok);
  info[0] = phi;
  info[1] = col[0];
  info[2] = col[1];
  info[3] = col[2];
  info[4] = cok;
  return def;
}

/* Test support: allocate brick (bx, by, bz, D) if needed and overwrite its 512 voxels with
 * vox (512 x 6: sdf, w, r, g, b, wc; voxel index i + 8 j + 64 k). Returns 0 on success. */
int om_set_brick(omap* m, int bx, int by, int bz, int D, const double* vox) {
  const int32_t b = brick_alloc(m, bx, by, bz, D, m->frames);
  if (b < 0) return -1;
  for (int vi = 0; vi < BVOX; ++vi) {
    ovox* o = m->vox + (size_t)b * BVOX + vi;
    o->sdf = vox[6 * vi];
    o->w = vox[6 * vi + 1];
    o->r = vox[6 * vi + 2];
    o->g = vox[6 * vi + 3];
    o->b = vox[6 * vi + 4];
    o->wc = vox[6 * vi + 5];
  }
  return 0;
}

/* ============================================ free-space combination (Sec. 4, Alg. 1) */
/*
 * Alg. 1 at a point p of the view ray (unit direction r from the camera centre c):
 *  - a direction takes part at a point where its trilinear field is present, unless its
 *    gradient exists and the gradient's normal lies outside the direction's angular range
 *    (w_dir = 0): the first implementation remark after Alg. 1 drops information whose gradient
 *    does not belong to the direction; a flat (truncated) field has no gradient and keeps its
 *    free-space or interior information;
 *  - F: taking-part directions with Phi^D(p) > 0, O: those with Phi^D(p) <= 0;
 *  - for D in F, q is the first zero transition of Phi^D met walking from p toward c over the
 *    march samples (consecutive present samples a (nearer the camera), b with
 *    Phi^D(a) <= 0 < Phi^D(b); q is the linear root between them); p is free space if some D in
 *    F has no q, or if at its q no taking-part direction D~ has Phi^D~(q) < 0 with
 *    <n^D~(q), -r> > 0;
 *  - the value is the fused-weight average of Phi^D over F (free space) or O (occupied);
 *    undefined when that set is empty.
 * The march and the root (bisection in the first Phi > 0 >= Phi bracket) are those of the
 * direct render (reading of Sec. 4); the normal, at the root's non-positive side, is the normalised fused-weight
 * sum of the chosen set's normals. No colour.
 */
typedef struct {
  int present, part;
  double phi, w, n[3];
} fsamp;

static void fs_all(const omap* m, const double* x, fsamp* S) {
  for (int D = 0; D < ND; ++D) {
    dsample d;
    sample_dir(m, D, x, &d);
    S[D].present = d.present;
    S[D].phi = d.present ? d.phi : 0.0;
    S[D].w = d.present ? d.w : 0.0;
    S[D].part = d.present;
    S[D].n[0] = S[D].n[1] = S[D].n[2] = 0.0;
    if (d.present && d.has_grad) {
      for (int a = 0; a < 3; ++a) S[D].n[a] = d.n[a];
      double cosv = (D & 1) ? -d.n[D >> 1] : d.n[D >> 1];
      S[D].part = om_w_dir(cosv, m->theta) > 0;
    }
  }
}

/* Is x inside the occupied space of a visible surface (some taking-part D~ with Phi < 0 and a
   gradient whose normal faces the camera)? */
static int fs_blocked(const omap* m, const double* x, const double* r) {
  fsamp S[ND];
  fs_all(m, x, S);
  for (int D = 0; D < ND; ++D) {
    if (!S[D].part || !(S[D].phi < 0)) continue;
    if (S[D].n[0] == 0 && S[D].n[1] == 0 && S[D].n[2] == 0) continue;
    double f = -(S[D].n[0] * r[0] + S[D].n[1] * r[1] + S[D].n[2] * r[2]);
    if (f > 0) return 1;
  }
  return 0;
}

/* Alg. 1 at the point with samples P at ray parameter tp; G[j*ND + D], gt[j] (j = 0..i0) are
   the march samples in front of it, gt[i0] the nearest. Returns 1 if defined (phi, nsum). */
static int fs_value(const omap* m, const double* o, const double* r, const fsamp* P, double tp, const fsamp* G,
                    const double* gt, long i0, double* phi, double* nsum) {
  int inF[ND], inO[ND], any_free = 0, nF = 0, nO = 0;
  for (int D = 0; D < ND; ++D) {
    inF[D] = P[D].part && P[D].phi > 0;
    inO[D] = P[D].part && !(P[D].phi > 0);
    nF += inF[D];
    nO += inO[D];
  }
  for (int D = 0; D < ND && !any_free; ++D) {
    if (!inF[D]) continue;
    /* walk from p toward the camera: pairs (a, b) with b the nearer-to-p sample */
    const fsamp* b = &P[D];
    double tb = tp;
    int found = 0;
    double tq = 0;
    for (long j = i0; j >= 0; --j) {
      const fsamp* a = &G[j * ND + D];
      if (a->present && b->present && a->phi <= 0 && b->phi > 0) {
        tq = gt[j] + (tb - gt[j]) * (-a->phi / (b->phi - a->phi));
        found = 1;
        break;
      }
      b = a;
      tb = gt[j];
    }
    if (!found) {
      any_free = 1;
    } else {
      double xq[3] = {o[0] + tq * r[0], o[1] + tq * r[1], o[2] + tq * r[2]};
      if (!fs_blocked(m, xq, r)) any_free = 1;
    }
  }
  const int* set = any_free ? inF : inO;
  if (!(any_free ? nF : nO)) return 0;
  double ws = 0, acc = 0, n[3] = {0, 0, 0};
  for (int D = 0; D < ND; ++D) {
    if (!set[D]) continue;
    ws += P[D].w;
    acc += P[D].w * P[D].phi;
    for (int a = 0; a < 3; ++a) n[a] += P[D].w * P[D].n[a];
  }
  if (!(ws > 0)) return 0;
  *phi = acc / ws;
  for (int a = 0; a < 3; ++a) nsum[a] = n[a];
  return 1;
}

static int render_pixel_fs(const omap* m, const double* T, double fx, double fy, double cx, double cy, int u, int v,
                           double* depth, double* ncam) {
  double rc[3] = {((double)u - cx) / fx, ((double)v - cy) / fy, 1.0};
  double rl = sqrt(rc[0] * rc[0] + rc[1] * rc[1] + rc[2] * rc[2]);
  double r[3], o[3] = {T[3], T[7], T[11]};
  for (int a = 0; a < 3; ++a) r[a] = (T[4 * a] * rc[0] + T[4 * a + 1] * rc[1] + T[4 * a + 2] * rc[2]) / rl;
  double step = 0.5 * m->h;
  double tn = m->zmin * rl, tf = m->zmax * rl;
  long k0 = (long)ceil(tn / step), k1 = (long)floor(tf / step);
  long nk = k1 >= k0 ? k1 - k0 + 1 : 0;
  fsamp* G = (fsamp*)calloc((size_t)(nk > 0 ? nk : 1) * ND, sizeof(fsamp));
  double* gt = (double*)calloc((size_t)(nk > 0 ? nk : 1), sizeof(double));
  double* gphi = (double*)calloc((size_t)(nk > 0 ? nk : 1), sizeof(double));
  double* gn = (double*)calloc((size_t)(nk > 0 ? nk : 1) * 3, sizeof(double));
  int* gdef = (int*)calloc((size_t)(nk > 0 ? nk : 1), sizeof(int));
  int hit = 0;
  double bs = 8.0 * m->h;
  for (long i = 0; i < nk && G && gt && gphi && gn && gdef; ++i) {
    double t = (k0 + i) * step;
    gt[i] = t;
    double x[3] = {o[0] + t * r[0], o[1] + t * r[1], o[2] + t * r[2]};
    int c[3];
    for (int a = 0; a < 3; ++a) c[a] = (int)floor((x[a] - m->origin[a]) / bs);
    if (cell_has_any(m, c[0], c[1], c[2])) fs_all(m, x, &G[i * ND]);
    gdef[i] = fs_value(m, o, r, &G[i * ND], t, G, gt, i - 1, &gphi[i], &gn[3 * i]);
    if (!(i > 0 && gdef[i - 1] && gdef[i] && gphi[i - 1] > 0 && gphi[i] <= 0)) continue;
    /* the root in [t_{i-1}, t_i] by bisection (an undefined midpoint counts as free space);
       the normal is the fused-weight normal sum at the root's non-positive side */
    double lo = gt[i - 1], hi = t;
    while (hi - lo > ROOT_TOL) {
      const double tm = 0.5 * (lo + hi);
      const double xm[3] = {o[0] + tm * r[0], o[1] + tm * r[1], o[2] + tm * r[2]};
      fsamp P[ND];
      fs_all(m, xm, P);
      double pm, nm[3];
      if (fs_value(m, o, r, P, tm, G, gt, i - 1, &pm, nm) && pm <= 0)
        hi = tm;
      else
        lo = tm;
    }
    const double ts = 0.5 * (lo + hi);
    {
      const double xs[3] = {o[0] + hi * r[0], o[1] + hi * r[1], o[2] + hi * r[2]};
      fsamp P[ND];
      fs_all(m, xs, P);
      double ps, nr[3];
      if (fs_value(m, o, r, P, hi, G, gt, i - 1, &ps, nr) && (nr[0] != 0 || nr[1] != 0 || nr[2] != 0)) {
        const double ln = sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
        *depth = ts / rl;
        for (int a = 0; a < 3; ++a) ncam[a] = (T[a] * nr[0] + T[4 + a] * nr[1] + T[8 + a] * nr[2]) / ln;
        hit = 1;
      }
    }
    break;
  }
  free(G);
  free(gt);
  free(gphi);
  free(gn);
  free(gdef);
  return hit;
}

/* Render pixels with Alg. 1 (pix NULL: all W*H, row-major). depth (0 = miss), normal (3, camera). */
int om_render_freespace(const omap* m, const double* T_wc, int W, int H, float fx, float fy, float cx, float cy,
                        const int32_t* pix, long npix, double* depth, double* normal) {
  long n = pix ? npix : (long)W * H;
#pragma omp parallel for schedule(dynamic, 16)
  for (long i = 0; i < n; ++i) {
    int u = pix ? pix[2 * i] : (int)(i % W);
    int v = pix ? pix[2 * i + 1] : (int)(i / W);
    double d = 0, nc[3] = {0, 0, 0};
    if (!render_pixel_fs(m, T_wc, fx, fy, cx, cy, u, v, &d, nc)) {
      d = 0;
      nc[0] = nc[1] = nc[2] = 0;
    }
    depth[i] = d;
    if (normal)
      for (int a = 0; a < 3; ++a) normal[3 * i + a] = nc[a];
  }
  return 0;
}

/* ====================================================== voxel recycling (Sec. 3) */
/*
 * Bricks that repeated carving turned into free space return to the pool: a brick is removed
 * when every voxel with weight > 0 has sdf >= free_sdf. The remaining bricks keep their order
 * and the hash is rebuilt; a later observation allocates a removed brick afresh (empty voxels).
 * Returns the number of bricks removed.
 */
int64_t om_recycle(omap* m, double free_sdf) {
  size_t w = 0;
  int64_t removed = 0;
  for (size_t b = 0; b < m->nbricks; ++b) {
    const ovox* v = m->vox + b * BVOX;
    int keep = 0;
    for (int i = 0; i < BVOX && !keep; ++i)
      if (v[i].w > 0 && !(v[i].sdf >= free_sdf)) keep = 1;
    if (!keep) {
      ++removed;
      continue;
    }
    if (w != b) {
      memmove(m->vox + w * BVOX, v, BVOX * sizeof(ovox));
      for (int a = 0; a < 4; ++a) m->coord[4 * w + a] = m->coord[4 * b + a];
      m->first_frame[w] = m->first_frame[b];
    }
    ++w;
  }
  m->nbricks = w;
  memset(m->keys, 0xFF, m->cap * sizeof(uint64_t));
  m->count = 0;
  for (size_t b = 0; b < w; ++b)
    hash_put(m, pack_key(m->coord[4 * b], m->coord[4 * b + 1], m->coord[4 * b + 2], m->coord[4 * b + 3]), (int32_t)b);
  return removed;
}
