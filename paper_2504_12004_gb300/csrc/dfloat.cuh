// Double-float ("float-float") arithmetic: a value is the unevaluated sum
// h + l of two floats, |l| <= ulp(h)/2, about 48 significant bits.  Built
// from the error-free transformations of Knuth (TwoSum), Dekker
// (FastTwoSum) and the FMA-based TwoProduct, as in the double-double
// literature (Hida, Li & Bailey; Joldes, Muller & Popescu).  The __f*_rn
// intrinsics keep the compiler from fusing or reassociating the steps whose
// rounding errors are being captured.
//
// On GB300 FP32 issues about 58 times faster than FP64, so the
// FP64-accurate covariance entries of the mixed path are evaluated here:
// squared scaled distance, square root, exp(-r) and the Matern polynomial.
#pragma once
#include <cuda_runtime.h>

namespace sbv {

struct df {
  float h, l;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

// a + b where no catastrophic cancellation occurs (same signs, or |b| << |a|)
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.h, b.h);
  float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return fast_two_sum(s.h, e);
}

__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = two_sum(a.h, b);
  return fast_two_sum(s.h, __fadd_rn(s.l, a.l));
}

__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  float p = __fmul_rn(a.h, b);
  float e = __fmaf_rn(a.h, b, -p);
  e = __fmaf_rn(a.l, b, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_from_double(double v) {
  float h = (float)v;
  return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.h + (double)a.l; }

// sqrt of a non-negative double-float: correctly rounded float root plus one
// Newton correction computed from the exact residual s - rh^2.
__device__ __forceinline__ df df_sqrt(df s) {
  if (!(s.h > 0.0f)) return {0.0f, 0.0f};
  float rh = __fsqrt_rn(s.h);
  float p = __fmul_rn(rh, rh);
  float pe = __fmaf_rn(rh, rh, -p);
  float e = __fadd_rn(__fsub_rn(__fsub_rn(s.h, p), pe), s.l);
  float rl = __fmul_rn(e, __fdiv_rn(0.5f, rh));
  return fast_two_sum(rh, rl);
}

// Constants of df_exp_neg, filled from host FP64 values when the library loads:
// c_exp_tab[i] = 2^(-i/32) for i = 0..31; c_ln2, c_inv_ln2; c_inv_fact[k] = 1/k!.
struct DfConsts {
  float tab_h[32], tab_l[32];
  float ln2_h, ln2_l, ilog2_h, ilog2_l;
  float third_h, third_l, fifth2_h, fifth2_l, fifteenth_h, fifteenth_l;
  float fact_h[8], fact_l[8];  // 1/k! for k = 0..7
};
// One copy per translation unit that includes this header; each such unit
// uploads it (cudaMemcpyToSymbol) before its first launch.
static __constant__ DfConsts c_df;

// exp(-r) for r >= 0: exp(-r) = 2^(-q) * 2^(-i/32) * exp(-g), where
// r / ln2 = (32 q + i)/32 + f, 0 <= f < 1/32, g = f ln2 < 0.0217, and exp(-g)
// is its Taylor polynomial to degree 7 (truncation < 1e-16) evaluated by
// Horner's rule in double-float.
__device__ __forceinline__ df df_exp_neg(df r) {
  if (r.h > 85.0f) return {0.0f, 0.0f};
  df t = df_mul(r, df{c_df.ilog2_h, c_df.ilog2_l});
  float kf = floorf(t.h * 32.0f);
  int k = (int)kf;
  df f = fast_two_sum(__fsub_rn(t.h, kf * 0.03125f), t.l);
  df g = df_mul(f, df{c_df.ln2_h, c_df.ln2_l});
  // exp(-g) = sum_k (-g)^k / k!
  df ng = {-g.h, -g.l};
  df acc = {c_df.fact_h[7], c_df.fact_l[7]};
#pragma unroll
  for (int q = 6; q >= 0; --q) acc = df_add(df_mul(acc, ng), df{c_df.fact_h[q], c_df.fact_l[q]});
  df e = df_mul(acc, df{c_df.tab_h[k & 31], c_df.tab_l[k & 31]});
  int sh = -(k >> 5);
  return {ldexpf(e.h, sh), ldexpf(e.l, sh)};
}

// Matern correlation M_nu(r) for nu = nu2/2 (closed forms), r and s = r^2 in double-float.
__device__ __forceinline__ df df_matern(df r, df s, int nu2) {
  df e = df_exp_neg(r);
  const df one = {1.0f, 0.0f};
  switch (nu2) {
    case 1:
      return e;
    case 3:
      return df_mul(df_add(one, r), e);
    case 5: {
      df p = df_add(df_add(one, r), df_mul(s, df{c_df.third_h, c_df.third_l}));
      return df_mul(p, e);
    }
    default: {
      // 1 + r + 2 r^2 / 5 + r^3 / 15
      df p = df_add(df_add(one, r), df_mul(s, df{c_df.fifth2_h, c_df.fifth2_l}));
      p = df_add(p, df_mul(df_mul(s, r), df{c_df.fifteenth_h, c_df.fifteenth_l}));
      return df_mul(p, e);
    }
  }
}

}  // namespace sbv
