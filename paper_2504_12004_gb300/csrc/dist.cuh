// Bit-exact scaled squared distances and their float32 screening bound.
//
// Decisions (cluster membership, neighbour ranking) use
//   D(a, c) = sum_{t=0}^{d-1} (a_t - c_t)^2
// in FP64, dimensions added left to right, every difference, product and sum
// rounded separately (the __d*_rn intrinsics are never contracted into FMA),
// so every GB300 and the CPU oracle take the same decision.
//
// Screening: a float32 copy of the distance, D32, is cheap.  With M an upper
// bound of |coordinate| over all points and centres, each float32 difference
// is within eta = 4.0004 * 2^-24 * M of the exact one, so
//   |D32 - D| <= E(D32) = (d+2) 2^-24 D32 + 2 eta (sqrt(d D32 (1 + 2^-20)) + d eta) + d eta^2
// (float32 accumulation of d non-negative terms, plus the perturbation of
// each square).  Twice E is used as the margin: an entry whose lower bound
// D32 - 2E exceeds an exact FP64 threshold can never beat it.
#pragma once
#include <cuda_runtime.h>

namespace sbv {

template <int DM>
__device__ __forceinline__ double dist2_exact(const double* __restrict__ a,
                                              const double* __restrict__ c, int d) {
  double acc = 0.0;
#pragma unroll
  for (int t = 0; t < DM; ++t) {
    if (t < d) {
      double df = __dsub_rn(a[t], c[t]);
      acc = __dadd_rn(acc, __dmul_rn(df, df));
    }
  }
  return acc;
}

// Same sum with a runtime dimension and a stride between coordinates of a.
__device__ __forceinline__ double dist2_exact_strided(const double* __restrict__ a,
                                                      size_t stride,
                                                      const double* __restrict__ c, int d) {
  double acc = 0.0;
  for (int t = 0; t < d; ++t) {
    double df = __dsub_rn(a[(size_t)t * stride], c[t]);
    acc = __dadd_rn(acc, __dmul_rn(df, df));
  }
  return acc;
}

struct ScreenBound {
  float eta;      // per-coordinate error bound of a float32 difference
  float dd;       // d as float
};

__host__ __device__ inline ScreenBound make_screen(double M, int d) {
  ScreenBound s;
  s.eta = (float)(4.0004 * 5.9604644775390625e-08 * M * 1.0000001);
  s.dd = (float)d;
  return s;
}

// 2 * E(D32): margin separating a float32 distance from the exact one.
__device__ __forceinline__ float screen_margin(float D32, ScreenBound s) {
  const float u = 5.9604644775390625e-08f;  // 2^-24
  float D = fmaxf(D32, 0.0f);
  float e = (s.dd + 2.0f) * u * D + 2.0f * s.eta * (sqrtf(s.dd * D * 1.000001f) + s.dd * s.eta) +
            s.dd * s.eta * s.eta;
  return 2.0f * e * 1.0001f + 1e-30f;
}

}  // namespace sbv
