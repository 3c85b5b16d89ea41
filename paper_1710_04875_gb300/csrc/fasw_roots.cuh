// FP64 powers of the per-cell auxiliaries by Newton's method from FP32 estimates (shared by the
// residual kernels and their forward-mode linearization).
#pragma once
#include "fasw_internal.cuh"

namespace fasw {

// rho^(-gamma) for gamma = 7/5: the root z of f(z) = rho^7 z^5 - 1.  The FP32 estimate
// (log2/exp2) has relative error d ~ 5e-7; the step z <- z (1 - f/5) is Newton's step to
// first order in f and leaves a relative error of about 3 d^2, so two steps reach FP64
// rounding (about one ulp of the exact 7/5 power; pow(rho, 1.4) raises to the double nearest
// 1.4, 8.9e-17 below 7/5, and differs from it by |ln rho| 8.9e-17 relative).
static_assert(GAM == 1.4, "rho^-gamma is formed as the root of rho^7 z^5 = 1");
__device__ __forceinline__ double pow_neg_gamma(double rho) {
  const float rf = (float)rho;
  double z = (double)exp2f(-1.4f * __log2f(rf));
  const double r2 = rho * rho, r7 = (r2 * r2) * (r2 * rho);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double z2 = z * z, z5 = (z2 * z2) * z;
    const double f = fma(r7, z5, -1.0);
    z = fma(-0.2 * f, z, z);
  }
  return z;
}

// (num/den)^(1/3) for positive num, den: the root c of den c^3 - num = 0, by Newton's method
// from the FP32 cube root with the derivative's reciprocal 1/(3 den c^2) taken in FP32 (the
// error contracts by ~1e-7 per step: two steps reach FP64 rounding).  No FP64 division.
__device__ __forceinline__ double cbrt_ratio(double num, double den) {
  const float nf = (float)num, df = (float)den;
  const float c0 = cbrtf(nf / df);
  const double d = (double)(1.0f / (3.0f * df * c0 * c0));
  double c = (double)c0;
#pragma unroll
  for (int it = 0; it < 2; ++it) c = fma(-fma(den, (c * c) * c, -num), d, c);
  return c;
}

}  // namespace fasw
