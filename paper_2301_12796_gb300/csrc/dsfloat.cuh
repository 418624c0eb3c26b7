// Double-single arithmetic for the preprocessing kernels, whose normals and back-projected points
// need more than single precision while the GPU's FP64 pipe runs at a small fraction of its FP32
// rate. A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about 48
// significant bits. The building blocks are the published error-free transformations: Knuth's
// TwoSum (The Art of Computer Programming vol. 2, Sec. 4.2.2), the fused-multiply-add form of
// Dekker's TwoProduct (Dekker 1971), and the renormalisation after every operation of the
// double-double scheme of Hida, Li and Bailey (QD library, 2001), carried out here on floats.
// Square root and reciprocal take the single-precision result and one Newton correction
// computed in double-single (Karp and Markstein 1997). Relative error of every operation
// below 2^-44; the build must not reassociate floating point (no fast-math flags).
#pragma once

namespace dtsdf {

struct dsf {
  float hi, lo;
};

// s + e = a + b exactly, for |a| >= |b| (or a == 0)
__host__ __device__ __forceinline__ dsf ds_fast_two_sum(float a, float b) {
  const float s = a + b;
  return dsf{s, b - (s - a)};
}
// s + e = a + b exactly, any order of magnitude
__host__ __device__ __forceinline__ dsf ds_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dsf{s, (a - (s - bb)) + (b - bb)};
}
// p + e = a * b exactly (barring underflow)
__host__ __device__ __forceinline__ dsf ds_two_prod(float a, float b) {
  const float p = a * b;
  return dsf{p, fmaf(a, b, -p)};
}
__host__ __device__ __forceinline__ dsf ds_add(dsf x, dsf y) {
  const dsf s = ds_two_sum(x.hi, y.hi), t = ds_two_sum(x.lo, y.lo);
  const dsf u = ds_fast_two_sum(s.hi, s.lo + t.hi);
  return ds_fast_two_sum(u.hi, u.lo + t.lo);
}
__host__ __device__ __forceinline__ dsf ds_sub(dsf x, dsf y) { return ds_add(x, dsf{-y.hi, -y.lo}); }
__host__ __device__ __forceinline__ dsf ds_mul(dsf x, dsf y) {
  const dsf p = ds_two_prod(x.hi, y.hi);
  return ds_fast_two_sum(p.hi, p.lo + (x.hi * y.lo + x.lo * y.hi));
}
__host__ __device__ __forceinline__ dsf ds_mul_f(dsf x, float f) {
  const dsf p = ds_two_prod(x.hi, f);
  return ds_fast_two_sum(p.hi, p.lo + x.lo * f);
}
// square root: the float root y of hi, corrected by (x - y^2) / (2 y); 0 for x <= 0
__host__ __device__ __forceinline__ dsf ds_sqrt(dsf x) {
  if (!(x.hi > 0.0f)) return dsf{0.0f, 0.0f};
  const float y = sqrtf(x.hi);
  const dsf r = ds_sub(x, ds_two_prod(y, y));
  return ds_fast_two_sum(y, r.hi / (2.0f * y));
}
// reciprocal: the float reciprocal y of hi, corrected by y (1 - x y)
__host__ __device__ __forceinline__ dsf ds_recip(dsf x) {
  const float y = 1.0f / x.hi;
  const dsf r = ds_sub(dsf{1.0f, 0.0f}, ds_mul_f(x, y));
  return ds_fast_two_sum(y, y * r.hi);
}
// nearest float to hi + lo (hi is already the nearest float after renormalisation, save for
// the halfway case)
__host__ __device__ __forceinline__ float ds_to_float(dsf x) { return x.hi + x.lo; }
// a double split into the nearest float and the float nearest the remainder (host side)
inline dsf ds_from_double(double d) {
  const float hi = (float)d;
  return dsf{hi, (float)(d - (double)hi)};
}

}  // namespace dtsdf
