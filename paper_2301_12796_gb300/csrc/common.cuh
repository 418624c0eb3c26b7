// Shared device-side definitions of libdtsdf (sm_103a).
//
// Decision paths (which pixel a voxel projects to, which blocks a segment crosses,
// band and membership tests, projective association) use explicitly rounded
// single-precision operations (__fmul_rn & co.), which the compiler never fuses
// into FMAs, so that every such integer/boolean outcome is a fixed function of
// the float inputs. Value paths use ordinary FP32 arithmetic.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dtsdf.h"

namespace dtsdf {

constexpr int ND = 6;          // directions X+, X-, Y+, Y-, Z+, Z- (Sec. 3)
constexpr int BVOX = 512;      // voxels per 8^3 block (Sec. 7)
// Geometry bricks are stored padded: the 8^3 voxels of the block plus an apron that
// copies the neighbouring blocks' voxels at local coordinates -1 and 8, 9 on every axis,
// so every voxel that a sample with its base voxel in the block reads (8 trilinear
// corners, and the 24 further taps of the central differences at +-h) sits in one brick.
constexpr int PAD = 11;                 // padded edge: local coordinates -1 .. 9
constexpr int PVOX = PAD * PAD * PAD;   // 1331 voxels per padded geometry brick
__host__ __device__ __forceinline__ int pad_index(int x, int y, int z) {
  return ((z + 1) * PAD + (y + 1)) * PAD + (x + 1);
}
// Combined bricks hold local coordinates [0, 8]^3 (the trilinear corners of every sample whose
// base voxel lies in the block). STORE_COMBINED selects the ray-cast of the combined field.
constexpr int CEDGE = 9;
constexpr int CVOX = CEDGE * CEDGE * CEDGE;
constexpr int STORE_COMBINED = 2;
__host__ __device__ __forceinline__ int comb_index(int x, int y, int z) { return (z * CEDGE + y) * CEDGE + x; }
constexpr unsigned long long EMPTY_KEY = ~0ull;
constexpr int MAX_PROBE = 256;  // linear-probe bound; the table is kept at most half full
constexpr int SLOT_MASK = 6;    // dir_slots[d * 8 + 6]: bitmask of allocated directions
// Bisection steps that refine a crossing bracket of h/2 (Sec. 4: small steps after the regular
// probing) to h / 2^17 (38 nm at 5 mm voxels), about the single-precision spacing of ray
// parameters of a metre. The direct render takes the final bracket's midpoint as the root, the
// free-space render the linear root of the final bracket (its bisection keeps Phi's values).
constexpr int REFINE_HALVINGS = 16;

// error flags (MapView::counters[C_ERR])
constexpr uint32_t ERR_POOL_FULL = 1u;
constexpr uint32_t ERR_DIR_FULL = 2u;
constexpr uint32_t ERR_HASH_FULL = 4u;
constexpr uint32_t ERR_WORK_FULL = 8u;
constexpr uint32_t ERR_TIMEOUT = 16u;  // a bounded wait of a kernel ran out (the kernel stopped early)

// hash values pack the directory index (26 bits) with the allocated-direction mask (6 bits)
constexpr uint32_t VAL_EMPTY = 0xFFFFFFFFu;
constexpr uint32_t VAL_DIR_MASK = 0x3FFFFFFu;
__host__ __device__ __forceinline__ uint32_t pack_val(int d, uint32_t mask) { return (uint32_t)d | (mask << 26); }
__host__ __device__ __forceinline__ int val_dir(uint32_t v) { return v == VAL_EMPTY ? -1 : (int)(v & VAL_DIR_MASK); }
__host__ __device__ __forceinline__ uint32_t val_mask(uint32_t v) { return v == VAL_EMPTY ? 0u : v >> 26; }

// device counters
// C_FREE_N / C_FREE_TAKEN: bricks pushed to / taken from the ring of recycled bricks (both only
// grow; ring position = count mod pool_cap); C_FREE_BEFORE: C_FREE_TAKEN before this frame.
enum {
  C_DIR = 0,
  C_POOL = 1,
  C_WORK = 2,
  C_ERR = 3,
  C_DIR_BEFORE = 4,
  C_POOL_BEFORE = 5,
  C_FREE_N = 6,
  C_FREE_TAKEN = 7,
  C_FREE_BEFORE = 8,
  C_COUNT = 10
};

__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float rsqrt_exact(float a) { return __fsqrt_rn(a); }

// ((a0*b0 + a1*b1) + a2*b2), each step rounded
__device__ __forceinline__ float rdot3(float a0, float a1, float a2, float b0, float b1, float b2) {
  return radd(radd(rmul(a0, b0), rmul(a1, b1)), rmul(a2, b2));
}

struct Pose32 {
  float R[9];  // row-major rotation (or s R) of camera -> world
  float t[3];
};

// Pose given in device memory (row-major 4x4 double), rounded to single precision exactly
// as the host does for poses passed by value.
__device__ __forceinline__ Pose32 pose_from_device(const double* T) {
  Pose32 p;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) p.R[3 * a + b] = __double2float_rn(T[4 * a + b]);
    p.t[a] = __double2float_rn(T[4 * a + 3]);
  }
  return p;
}

struct Intr {
  int W, H;
  float fx, fy, cx, cy;
};

// Single-precision rounded rotation: y_a = (R[a0] x0 + R[a1] x1) + R[a2] x2
__device__ __forceinline__ void rrot(const float* R, float x0, float x1, float x2, float& y0, float& y1, float& y2) {
  y0 = rdot3(R[0], R[1], R[2], x0, x1, x2);
  y1 = rdot3(R[3], R[4], R[5], x0, x1, x2);
  y2 = rdot3(R[6], R[7], R[8], x0, x1, x2);
}

// Transposed rotation (world -> camera of a camera -> world R): y_a = (R[0a] x0 + R[1a] x1) + R[2a] x2
__device__ __forceinline__ void rrotT(const float* R, float x0, float x1, float x2, float& y0, float& y1,
                                      float& y2) {
  y0 = rdot3(R[0], R[3], R[6], x0, x1, x2);
  y1 = rdot3(R[1], R[4], R[7], x0, x1, x2);
  y2 = rdot3(R[2], R[5], R[8], x0, x1, x2);
}

__device__ __forceinline__ bool depth_in_range(float z, float zmin, float zmax) {
  return z > 0.0f && z >= zmin && z <= zmax;
}

// ---------------------------------------------------------------- hash ----
__host__ __device__ __forceinline__ unsigned long long pack_block(int bx, int by, int bz) {
  return ((unsigned long long)((uint32_t)(bx + (1 << 20)) & 0x1FFFFFu) << 42) |
         ((unsigned long long)((uint32_t)(by + (1 << 20)) & 0x1FFFFFu) << 21) |
         (unsigned long long)((uint32_t)(bz + (1 << 20)) & 0x1FFFFFu);
}

__host__ __device__ __forceinline__ void unpack_block(unsigned long long k, int& bx, int& by, int& bz) {
  bx = (int)((k >> 42) & 0x1FFFFFu) - (1 << 20);
  by = (int)((k >> 21) & 0x1FFFFFu) - (1 << 20);
  bz = (int)(k & 0x1FFFFFu) - (1 << 20);
}

__host__ __device__ __forceinline__ uint32_t hash_slot(unsigned long long k, uint32_t mask) {
  k ^= k >> 31;
  k *= 0x7fb5d329728ea185ull;
  k ^= k >> 27;
  k *= 0x81dadef4bc2dd44dull;
  k ^= k >> 33;
  return (uint32_t)k & mask;
}

// Device view of a map, passed by value to kernels.
struct MapView {
  float h, tau, theta, wmax, wcarve, zmin, zmax, dsup, costh, sinth;
  float ox, oy, oz;
  int carve_r, dense_dim, color, storage;
  // hash: block coordinate -> directory index
  unsigned long long* keys;
  uint32_t* vals;  // pack_val(directory index, allocated mask), VAL_EMPTY before assignment
  uint32_t* req;  // per hash slot: directions requested this frame
  uint32_t hmask;
  // directory: 8 ints per entry: slots of the 6 directions, allocated mask, unused
  int32_t* dir_slots;
  int32_t* dir_coord;  // 4 ints per entry: bx, by, bz, 0
  uint32_t dir_cap;
  // brick pool
  float2* geom;     // FP32: (sdf, weight) per voxel, PVOX per brick (padded, see pad_index)
  uint32_t* geom16; // FP16: half sdf | half weight (as u16) per voxel, PVOX per brick
  float4* col;      // FP32: (r, g, b, colour weight), BVOX per brick (unpadded)
  uint32_t* col8;   // FP16 storage: u8 r, g, b and the 8-bit log colour-weight code, BVOX per brick
  int32_t* brick_dir;  // per brick: dir index * 8 + D
  float* bound;        // per brick: minimum sdf over local voxels [0, 8]^3 with weight > 0 (+inf if none)
  uint32_t* stamp;     // per brick: last frame whose fusion or allocation changed its voxels
  uint32_t frame;      // id of the frame being fused
  // view-dependent combined TSDF (allocated on first use): per directory entry the combined
  // values of local voxels [0, 8]^3 (CVOX), x fastest, and the generation they belong to
  float2* comb;        // (phi, 1 if defined else 0)
  uint2* comb_col;     // r, g, b as 16-bit fixed point (c * 257, exact for 8-bit colours; the
                       // combination of colours rounds to 1/257) and 1 if defined else 0,
                       // colour maps only
  uint32_t* comb_gen;  // per directory entry
  uint8_t* comb_dirty; // per directory entry: a neighbouring block received bricks since its combination
  const uint32_t* comb_cur;  // device word: the current generation
  uint32_t* occ;       // occupancy filters: 2 x OCC_WORDS words (blocks, then 4^3-block super-cells)
  uint32_t pool_cap;
  int32_t* free_ring;  // recycled bricks (hash maps), pool_cap entries
  uint32_t* counters;
  int32_t* work;
  uint32_t work_cap;
};

// Packed hash value of block (bx, by, bz), VAL_EMPTY if absent.
__device__ __forceinline__ uint32_t hash_find_packed(const MapView& m, int bx, int by, int bz) {
  const unsigned long long k = pack_block(bx, by, bz);
  uint32_t i = hash_slot(k, m.hmask);
#pragma unroll 1
  for (int p = 0; p < MAX_PROBE; ++p) {
    const unsigned long long kk = __ldg(m.keys + i);
    if (kk == k) return __ldg(m.vals + i);
    if (kk == EMPTY_KEY) return VAL_EMPTY;
    i = (i + 1) & m.hmask;
  }
  return VAL_EMPTY;
}

__device__ __forceinline__ int hash_find(const MapView& m, int bx, int by, int bz) {
  return val_dir(hash_find_packed(m, bx, by, bz));
}

// float atomic minimum through the integer orderings of positive and negative floats
__device__ __forceinline__ void atomic_min_float(float* addr, float v) {
  if (v >= 0.0f)
    atomicMin((int*)addr, __float_as_int(v));
  else
    atomicMax((unsigned int*)addr, __float_as_uint(v));
}

// Occupancy filters: one bit per hashed block (and per hashed super-cell of 4^3 blocks),
// set when a block gets a directory entry. No false negatives; a false positive only costs
// the real hash probe.
constexpr uint32_t OCC_BITS_LOG2 = 23;
constexpr uint32_t OCC_WORDS = 1u << (OCC_BITS_LOG2 - 5);
__host__ __device__ __forceinline__ uint32_t occ_bit(int bx, int by, int bz, int level) {
  // 32-bit multiplicative hash of the coordinates (cheap enough to test at every cell a ray enters)
  uint32_t h = ((uint32_t)bx * 0x8da6b343u) ^ ((uint32_t)by * 0xd8163841u) ^ ((uint32_t)bz * 0xcb1ab31fu) ^
               (level ? 0x5bd1e995u : 0u);
  h ^= h >> 16;
  h *= 0x7feb352du;
  h ^= h >> 15;
  return h & ((1u << OCC_BITS_LOG2) - 1u);
}
__device__ __forceinline__ void occ_set(const MapView& m, int bx, int by, int bz) {
  const uint32_t a = occ_bit(bx, by, bz, 0), b = occ_bit(bx >> 2, by >> 2, bz >> 2, 1);
  atomicOr(m.occ + (a >> 5), 1u << (a & 31));
  atomicOr(m.occ + OCC_WORDS + (b >> 5), 1u << (b & 31));
}
__device__ __forceinline__ bool occ_test(const MapView& m, int bx, int by, int bz, int level) {
  const uint32_t a = level ? occ_bit(bx >> 2, by >> 2, bz >> 2, 1) : occ_bit(bx, by, bz, 0);
  return (__ldg(m.occ + (level ? OCC_WORDS : 0) + (a >> 5)) >> (a & 31)) & 1u;
}

// Storage accessors ---------------------------------------------------------
// FP16 form: sdf as IEEE half; the weight's u16 holds an IEEE half too (2^-11 relative
// resolution at every magnitude; a positive weight is kept at least at the smallest
// positive half, so "weight > 0" survives); colour as u8 r, g, b and an 8-bit logarithmic
// colour-weight code q: w = 2^((q - 128) / 16), q = 0 for w = 0.
__device__ __forceinline__ float2 unpack_geom16(uint32_t v) {
  __half_raw hs, hw;
  hs.x = (unsigned short)(v & 0xFFFFu);
  hw.x = (unsigned short)(v >> 16);
  return make_float2(__half2float(__half(hs)), __half2float(__half(hw)));
}

__device__ __forceinline__ uint32_t pack_geom16(float sdf, float w) {
  const __half_raw hs = __float2half_rn(sdf);
  __half_raw hw = __float2half_rn(fminf(w, 65504.0f));
  if (w > 0.0f && hw.x == 0) hw.x = 1;  // smallest positive subnormal half
  if (!(w > 0.0f)) hw.x = 0;
  return (uint32_t)hs.x | ((uint32_t)hw.x << 16);
}

__device__ __forceinline__ float col_weight_decode(uint32_t code) {
  return code ? exp2f(((float)code - 128.0f) * (1.0f / 16.0f)) : 0.0f;
}

__device__ __forceinline__ uint32_t col_weight_encode(float w) {
  if (!(w > 0.0f)) return 0u;
  const float q = rintf(16.0f * log2f(w) + 128.0f);
  return (uint32_t)fminf(fmaxf(q, 1.0f), 255.0f);
}

__device__ __forceinline__ uint32_t pack_col8(float r, float g, float b, float w) {
  const uint32_t R = (uint32_t)fminf(fmaxf(rintf(r), 0.f), 255.f);
  const uint32_t G = (uint32_t)fminf(fmaxf(rintf(g), 0.f), 255.f);
  const uint32_t B = (uint32_t)fminf(fmaxf(rintf(b), 0.f), 255.f);
  return R | (G << 8) | (B << 16) | (col_weight_encode(w) << 24);
}

// Combined colour: r, g, b in [0, 255] as round(c * 257) in 16 bits, and a defined flag.
__device__ __forceinline__ uint2 pack_comb_col(float r, float g, float b, bool defined) {
  const uint32_t qr = (uint32_t)__float2uint_rn(fminf(fmaxf(r, 0.f), 255.f) * 257.f);
  const uint32_t qg = (uint32_t)__float2uint_rn(fminf(fmaxf(g, 0.f), 255.f) * 257.f);
  const uint32_t qb = (uint32_t)__float2uint_rn(fminf(fmaxf(b, 0.f), 255.f) * 257.f);
  return make_uint2(qr | (qg << 16), qb | (defined ? 0x10000u : 0u));
}
__device__ __forceinline__ float4 unpack_comb_col(uint2 v) {
  const float s = 1.0f / 257.0f;
  return make_float4((float)(v.x & 0xFFFFu) * s, (float)(v.x >> 16) * s, (float)(v.y & 0xFFFFu) * s,
                     (v.y >> 16) ? 1.0f : 0.0f);
}

__device__ __forceinline__ float4 unpack_col8(uint32_t v) {
  return make_float4((float)(v & 0xFF), (float)((v >> 8) & 0xFF), (float)((v >> 16) & 0xFF),
                     col_weight_decode(v >> 24));
}

}  // namespace dtsdf
