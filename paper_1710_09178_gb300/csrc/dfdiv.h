// dfdiv.h - the quotient of two double-FP32 numbers (hi, lo) on the FP32 units.
//
// Dekker's division (T. J. Dekker, "A floating-point technique for extending the available precision",
// Numer. Math. 18 (1971) 224): q1 = fl(ah / bh); the remainder r = a - q1 b is formed with the exact
// product q1 bh = p + e (e from an FMA) and the lo parts; q2 = fl(r / bh) corrects q1, and (q1, q2) is
// renormalised.  The quotient carries about 2^-45 relative error (the FP32 rounding of q2 and of the
// remainder's lo terms), against ~2^-48 for the operands.  Every operation is an IEEE FP32 operation
// with one rounding (no contraction), so the host build, used by the tests, gives the device's bits.
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define LQCD_HD __host__ __device__ __forceinline__
#else
#define LQCD_HD inline
#endif

namespace lqcd {

struct DfPair {
  float hi, lo;
};

LQCD_HD float dfd_mul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
LQCD_HD float dfd_add(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
LQCD_HD float dfd_sub(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
LQCD_HD float dfd_div(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fdiv_rn(a, b);
#else
  return a / b;
#endif
}
LQCD_HD float dfd_fma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}

// (ah + al) / (bh + bl); bh != 0, both pairs normalised (|lo| <= ulp(hi) / 2)
LQCD_HD DfPair df_div_pair(float ah, float al, float bh, float bl) {
  const float q1 = dfd_div(ah, bh);
  const float p = dfd_mul(q1, bh);
  const float e = dfd_fma(q1, bh, -p);  // q1 bh = p + e exactly
  float r = dfd_sub(ah, p);             // exact: p is within a few ulps of ah
  r = dfd_sub(r, e);
  r = dfd_add(r, al);
  r = dfd_fma(-q1, bl, r);
  const float q2 = dfd_div(r, bh);
  const float h = dfd_add(q1, q2);
  DfPair o;
  o.hi = h;
  o.lo = dfd_sub(q2, dfd_sub(h, q1));
  return o;
}

}  // namespace lqcd
