// Host driver for the double-single header: seeded operands, every result printed as hex floats
// so that the test can compare it with exact rational arithmetic.
#define __host__
#define __device__
#define __forceinline__ inline
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "dsfloat.cuh"

using dtsdf::dsf;

static uint64_t state = 0x9E3779B97F4A7C15ull;
static double uniform() {  // splitmix64, 53 random bits in [0, 1)
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53;
}
static double operand(bool positive) {  // magnitudes 2^-20 .. 2^20, random sign
  const double m = std::ldexp(1.0 + uniform(), (int)(uniform() * 41.0) - 20);
  return positive || uniform() < 0.5 ? m : -m;
}
static void put(dsf x) { std::printf(" %a %a", (double)x.hi, (double)x.lo); }

int main() {
  for (int i = 0; i < 4000; ++i) {
    const dsf a = dtsdf::ds_from_double(operand(false)), b = dtsdf::ds_from_double(operand(false));
    const float f = (float)operand(false);
    const dsf p = dtsdf::ds_from_double(operand(true));
    std::printf("add");
    put(a), put(b), put(dtsdf::ds_add(a, b));
    // near-cancelling sums: b close to -a
    const double d = operand(false);
    const dsf c = dtsdf::ds_from_double(d), e = dtsdf::ds_from_double(-d * (1.0 + std::ldexp(uniform(), -(int)(uniform() * 40.0))));
    std::printf("\nadd");
    put(c), put(e), put(dtsdf::ds_add(c, e));
    std::printf("\nmul");
    put(a), put(b), put(dtsdf::ds_mul(a, b));
    std::printf("\nmulf");
    put(a), std::printf(" %a", (double)f), put(dtsdf::ds_mul_f(a, f));
    std::printf("\nsqrt");
    put(p), put(dtsdf::ds_sqrt(p));
    std::printf("\nrecip");
    put(a), put(dtsdf::ds_recip(a));
    std::printf("\n");
  }
  return 0;
}
