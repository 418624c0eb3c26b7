/*
 * Seeded synthetic RGB-D input generator: ray-traces analytic scenes into
 * depth and RGB frames.
 *
 * This module is input generation only. It holds none of the DTSDF method's
 * arithmetic (no fusion, weighting, rendering of the map or ICP); the oracle
 * and the CUDA path both consume what it writes. It stands in for the indoor
 * RGB-D sequences the paper evaluates on (ICL-NUIM, TUM, Zhou), which are not
 * available here.
 *
 * Conventions: camera frame x right, y down, z forward; pixel (u, v) centres at
 * integer coordinates; poses T_wc are camera-to-world, row-major 4x4, double.
 * Depth is z-depth in metres, 0 marks an invalid pixel.
 *
 * Primitive kinds:
 *   0 room    : axis-aligned box seen from inside (camera inside), inward normals
 *   1 box     : solid oriented box (centre, half extents, rotation rows = axes);
 *               a thin sheet is a box with one small half extent
 *   2 cylinder: solid cylinder with vertical (z) axis and flat caps
 *   3 sphere  : solid sphere
 *
 * Texture: Perlin's improved gradient noise (Perlin 2002), written from the
 * published description (quintic fade, 12 edge gradients, permutation table),
 * with the permutation shuffled by a seeded splitmix64 stream.
 * Depth noise: z' = z + (s0 + s2 z^2) * N(0,1), with N(0,1) from Box-Muller over a
 * counter-based splitmix64 hash of (seed, frame, pixel).
 *
 * Build with -ffp-contract=off so x86 and Arm hosts produce the same frames.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define PRIM_ROOM 0
#define PRIM_BOX 1
#define PRIM_CYL 2
#define PRIM_SPHERE 3

/* One primitive, 24 doubles:
 *  [0] kind, [1] object id,
 *  [2..4] centre (room: lo corner), [5..7] half extents (room: hi corner;
 *  cylinder: r, z0, z1; sphere: r),
 *  [8..16] rotation rows (box only; local = R (x - c)),
 *  [17..19] colour A (0..255), [20..22] colour B, [23] texture frequency (1/m)
 */
#define PRIM_STRIDE 24

static uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

static double u01(uint64_t x) { /* (0, 1) */
  return ((double)(x >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* ---------------------------------------------------------------- noise -- */
typedef struct {
  int p[512];
} perlin_t;

static void perlin_init(perlin_t* P, uint64_t seed) {
  int i;
  uint64_t s = splitmix64(seed ^ 0x5EED5EEDull);
  for (i = 0; i < 256; ++i) P->p[i] = i;
  for (i = 255; i > 0; --i) {
    s = splitmix64(s);
    int j = (int)(s % (uint64_t)(i + 1));
    int t = P->p[i];
    P->p[i] = P->p[j];
    P->p[j] = t;
  }
  for (i = 0; i < 256; ++i) P->p[256 + i] = P->p[i];
}

static double fade(double t) { return t * t * t * (t * (t * 6.0 - 15.0) + 10.0); }
static double lerp(double t, double a, double b) { return a + t * (b - a); }
static double grad(int h, double x, double y, double z) {
  /* 12 edge directions of the cube (plus 4 repeats), selected by the low 4 bits */
  switch (h & 15) {
    case 0: return x + y;
    case 1: return -x + y;
    case 2: return x - y;
    case 3: return -x - y;
    case 4: return x + z;
    case 5: return -x + z;
    case 6: return x - z;
    case 7: return -x - z;
    case 8: return y + z;
    case 9: return -y + z;
    case 10: return y - z;
    case 11: return -y - z;
    case 12: return x + y;
    case 13: return -y + z;
    case 14: return -x + y;
    default: return -y - z;
  }
}

static double perlin(const perlin_t* P, double x, double y, double z) {
  double fx = floor(x), fy = floor(y), fz = floor(z);
  int X = ((int)fx) & 255, Y = ((int)fy) & 255, Z = ((int)fz) & 255;
  x -= fx;
  y -= fy;
  z -= fz;
  double u = fade(x), v = fade(y), w = fade(z);
  const int* p = P->p;
  int A = p[X] + Y, AA = p[A] + Z, AB = p[A + 1] + Z;
  int B = p[X + 1] + Y, BA = p[B] + Z, BB = p[B + 1] + Z;
  return lerp(w,
              lerp(v, lerp(u, grad(p[AA], x, y, z), grad(p[BA], x - 1, y, z)),
                   lerp(u, grad(p[AB], x, y - 1, z), grad(p[BB], x - 1, y - 1, z))),
              lerp(v, lerp(u, grad(p[AA + 1], x, y, z - 1), grad(p[BA + 1], x - 1, y, z - 1)),
                   lerp(u, grad(p[AB + 1], x, y - 1, z - 1), grad(p[BB + 1], x - 1, y - 1, z - 1))));
}

/* ------------------------------------------------------------ intersect -- */
typedef struct {
  double t;
  double n[3];
  int prim;
} hit_t;

static void consider(hit_t* h, double t, double nx, double ny, double nz, int prim) {
  if (t > 1e-9 && t < h->t) {
    h->t = t;
    h->n[0] = nx;
    h->n[1] = ny;
    h->n[2] = nz;
    h->prim = prim;
  }
}

static void isect_room(const double* P, const double* o, const double* d, int k, hit_t* h) {
  /* camera inside: the hit is the exit through the nearest far face */
  double best = 1e300;
  int axis = -1;
  double sgn = 0;
  for (int a = 0; a < 3; ++a) {
    if (d[a] > 0) {
      double t = (P[5 + a] - o[a]) / d[a];
      if (t < best) { best = t; axis = a; sgn = -1.0; }
    } else if (d[a] < 0) {
      double t = (P[2 + a] - o[a]) / d[a];
      if (t < best) { best = t; axis = a; sgn = 1.0; }
    }
  }
  if (axis >= 0) {
    double n[3] = {0, 0, 0};
    n[axis] = sgn;
    consider(h, best, n[0], n[1], n[2], k);
  }
}

static void isect_box(const double* P, const double* o, const double* d, int k, hit_t* h) {
  const double* c = P + 2;
  const double* e = P + 5;
  const double* R = P + 8;
  double ol[3], dl[3], rel[3] = {o[0] - c[0], o[1] - c[1], o[2] - c[2]};
  for (int a = 0; a < 3; ++a) {
    ol[a] = R[3 * a] * rel[0] + R[3 * a + 1] * rel[1] + R[3 * a + 2] * rel[2];
    dl[a] = R[3 * a] * d[0] + R[3 * a + 1] * d[1] + R[3 * a + 2] * d[2];
  }
  double tn = -1e300, tf = 1e300;
  int an = -1;
  double sn = 0;
  for (int a = 0; a < 3; ++a) {
    if (dl[a] == 0.0) {
      if (ol[a] < -e[a] || ol[a] > e[a]) return;
      continue;
    }
    double t1 = (-e[a] - ol[a]) / dl[a];
    double t2 = (e[a] - ol[a]) / dl[a];
    double s = -1.0;
    if (t1 > t2) { double tt = t1; t1 = t2; t2 = tt; s = 1.0; }
    if (t1 > tn) { tn = t1; an = a; sn = s; }
    if (t2 < tf) tf = t2;
  }
  if (tn > tf || an < 0 || tn <= 1e-9) return;
  /* outward normal of the entered face, back to world */
  double nl[3] = {0, 0, 0};
  nl[an] = sn;
  double nw[3];
  for (int b = 0; b < 3; ++b) nw[b] = R[b] * nl[0] + R[3 + b] * nl[1] + R[6 + b] * nl[2];
  consider(h, tn, nw[0], nw[1], nw[2], k);
}

static void isect_cyl(const double* P, const double* o, const double* d, int k, hit_t* h) {
  double cx = P[2], cy = P[3], r = P[5], z0 = P[6], z1 = P[7];
  double ox = o[0] - cx, oy = o[1] - cy;
  double a = d[0] * d[0] + d[1] * d[1];
  if (a > 0) {
    double b = ox * d[0] + oy * d[1];
    double c = ox * ox + oy * oy - r * r;
    double disc = b * b - a * c;
    if (disc >= 0) {
      double sq = sqrt(disc);
      double t = (-b - sq) / a;
      double z = o[2] + t * d[2];
      if (t > 1e-9 && z >= z0 && z <= z1) {
        double px = ox + t * d[0], py = oy + t * d[1];
        consider(h, t, px / r, py / r, 0.0, k);
      }
    }
  }
  if (d[2] != 0) {
    double zc[2] = {z0, z1};
    double ns[2] = {-1.0, 1.0};
    for (int i = 0; i < 2; ++i) {
      double t = (zc[i] - o[2]) / d[2];
      if (t <= 1e-9) continue;
      double px = ox + t * d[0], py = oy + t * d[1];
      /* a cap is entered only from its outer side */
      if (ns[i] * d[2] >= 0) continue;
      if (px * px + py * py <= r * r) consider(h, t, 0.0, 0.0, ns[i], k);
    }
  }
}

static void isect_sphere(const double* P, const double* o, const double* d, int k, hit_t* h) {
  double r = P[5];
  double oc[3] = {o[0] - P[2], o[1] - P[3], o[2] - P[4]};
  double a = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double b = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
  double c = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - r * r;
  double disc = b * b - a * c;
  if (disc < 0) return;
  double t = (-b - sqrt(disc)) / a;
  if (t <= 1e-9) return;
  double p[3] = {oc[0] + t * d[0], oc[1] + t * d[1], oc[2] + t * d[2]};
  consider(h, t, p[0] / r, p[1] / r, p[2] / r, k);
}

static void trace(const double* prims, int nprims, const double* o, const double* d, hit_t* h) {
  h->t = 1e300;
  h->prim = -1;
  for (int k = 0; k < nprims; ++k) {
    const double* P = prims + (size_t)k * PRIM_STRIDE;
    switch ((int)P[0]) {
      case PRIM_ROOM: isect_room(P, o, d, k, h); break;
      case PRIM_BOX: isect_box(P, o, d, k, h); break;
      case PRIM_CYL: isect_cyl(P, o, d, k, h); break;
      case PRIM_SPHERE: isect_sphere(P, o, d, k, h); break;
      default: break;
    }
  }
}

/*
 * Render one frame.
 *   prims/nprims : scene
 *   T_wc         : camera-to-world pose (row-major 4x4)
 *   W,H,fx,fy,cx,cy : pinhole intrinsics
 *   noise_s0, noise_s2 : depth noise sigma = s0 + s2 z^2 (0,0 = noise free)
 *   z_min, z_max : valid depth range (outside -> 0)
 *   seed, frame  : counter inputs of the noise stream
 *   tex_seed     : Perlin permutation seed
 * Outputs (any may be NULL):
 *   depth  f32 [H*W]    noisy z-depth (0 invalid)
 *   rgb    u8  [H*W*3]  texture colour at the hit
 *   pts    f64 [H*W*3]  exact camera-frame hit point (noise free; 0 if no hit)
 *   nrm    f64 [H*W*3]  exact camera-frame surface normal facing the camera
 *   ids    i32 [H*W]    primitive index hit (-1 none)
 */
int scene_render(const double* prims, int nprims, const double* T_wc, int W, int H, double fx,
                 double fy, double cx, double cy, double noise_s0, double noise_s2, double z_min,
                 double z_max, uint64_t seed, uint64_t frame, uint64_t tex_seed, float* depth,
                 uint8_t* rgb, double* pts, double* nrm, int32_t* ids) {
  perlin_t P;
  perlin_init(&P, tex_seed);
  const double* T = T_wc;
  double o[3] = {T[3], T[7], T[11]};
#pragma omp parallel for schedule(static)
  for (int v = 0; v < H; ++v) {
    for (int u = 0; u < W; ++u) {
      size_t i = (size_t)v * W + u;
      double dc[3] = {((double)u - cx) / fx, ((double)v - cy) / fy, 1.0};
      double d[3];
      for (int a = 0; a < 3; ++a) d[a] = T[4 * a] * dc[0] + T[4 * a + 1] * dc[1] + T[4 * a + 2] * dc[2];
      hit_t h;
      trace(prims, nprims, o, d, &h);
      float z_out = 0.0f;
      double pc[3] = {0, 0, 0}, nc[3] = {0, 0, 0};
      uint8_t col[3] = {0, 0, 0};
      if (h.prim >= 0) {
        double z = h.t; /* dc has unit z, so t is the z-depth */
        double pw[3] = {o[0] + h.t * d[0], o[1] + h.t * d[1], o[2] + h.t * d[2]};
        pc[0] = dc[0] * z;
        pc[1] = dc[1] * z;
        pc[2] = z;
        /* world normal -> camera frame (R^T n), oriented toward the camera */
        for (int a = 0; a < 3; ++a) nc[a] = T[a] * h.n[0] + T[4 + a] * h.n[1] + T[8 + a] * h.n[2];
        if (nc[0] * pc[0] + nc[1] * pc[1] + nc[2] * pc[2] > 0) {
          nc[0] = -nc[0];
          nc[1] = -nc[1];
          nc[2] = -nc[2];
        }
        const double* Pr = prims + (size_t)h.prim * PRIM_STRIDE;
        double f = Pr[23];
        double s = perlin(&P, pw[0] * f, pw[1] * f, pw[2] * f) +
                   0.5 * perlin(&P, pw[0] * 2.0 * f + 17.0, pw[1] * 2.0 * f + 31.0, pw[2] * 2.0 * f + 7.0);
        double m = 0.5 + 0.5 * s;
        if (m < 0) m = 0;
        if (m > 1) m = 1;
        for (int a = 0; a < 3; ++a) {
          double cval = Pr[17 + a] + m * (Pr[20 + a] - Pr[17 + a]);
          long q = lround(cval);
          col[a] = (uint8_t)(q < 0 ? 0 : (q > 255 ? 255 : q));
        }
        double zn = z;
        if (noise_s0 > 0 || noise_s2 > 0) {
          uint64_t key = splitmix64(seed * 0x9E3779B97F4A7C15ull ^ splitmix64(frame + 0x1234567ull) ^
                                    (uint64_t)i * 0xD1B54A32D192ED03ull);
          double u1 = u01(splitmix64(key)), u2 = u01(splitmix64(key ^ 0xA5A5A5A5A5A5A5A5ull));
          double g = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
          zn = z + (noise_s0 + noise_s2 * z * z) * g;
        }
        if (zn >= z_min && zn <= z_max) z_out = (float)zn;
      }
      if (depth) depth[i] = z_out;
      if (rgb) {
        rgb[3 * i] = col[0];
        rgb[3 * i + 1] = col[1];
        rgb[3 * i + 2] = col[2];
      }
      if (pts) {
        pts[3 * i] = pc[0];
        pts[3 * i + 1] = pc[1];
        pts[3 * i + 2] = pc[2];
      }
      if (nrm) {
        nrm[3 * i] = nc[0];
        nrm[3 * i + 1] = nc[1];
        nrm[3 * i + 2] = nc[2];
      }
      if (ids) ids[i] = h.prim;
    }
  }
  return 0;
}

/* Exact ray hit distance for one world-frame ray (for closed-form checks). */
double scene_ray_t(const double* prims, int nprims, const double* o, const double* d) {
  hit_t h;
  trace(prims, nprims, o, d, &h);
  return h.prim >= 0 ? h.t : -1.0;
}
