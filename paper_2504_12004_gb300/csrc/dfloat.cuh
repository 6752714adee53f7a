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

// a - b with full accuracy even under cancellation
__device__ __forceinline__ df df_sub_acc(df a, df b) {
  df s = two_sum(a.h, -b.h);
  df t = two_sum(a.l, -b.l);
  s.l = __fadd_rn(s.l, t.h);
  s = fast_two_sum(s.h, s.l);
  s.l = __fadd_rn(s.l, t.l);
  return fast_two_sum(s.h, s.l);
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
  float rl = __fmul_rn(e, __fdividef(0.5f, rh));
  return fast_two_sum(rh, rl);
}

// acc -= s * x for a double-float s (float pair) and a float x: the product
// s.h x is split exactly into p + e (FMA), s.l x is added to e; acc.l is left
// unnormalised (the caller renormalises once at the end of a dot product).
__device__ __forceinline__ void df_fnma_acc(df& acc, float2 s, float x) {
  const float p = __fmul_rn(s.x, x);
  float e = __fmaf_rn(s.x, x, -p);
  e = __fmaf_rn(s.y, x, e);
  const df t = two_sum(acc.h, -p);
  acc.h = t.h;
  acc.l = __fadd_rn(acc.l, __fsub_rn(t.l, e));
}

// 1 / x for a positive double-float: the float reciprocal plus one Newton
// correction from the exact residual 1 - x r (about 46 significant bits).
__device__ __forceinline__ df df_recip(df x) {
  const float r = __frcp_rn(x.h);
  const float p = __fmul_rn(x.h, r);
  const float pe = __fmaf_rn(x.h, r, -p);
  // 1 - x r = (1 - p) - pe - x.l r, with 1 - p exact (p is within an ulp of 1)
  const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), pe), __fmul_rn(x.l, r));
  return fast_two_sum(r, __fmul_rn(r, e));
}

// Constants of the double-float exponential, filled from host FP64 values:
// 1/ln2, ln2, 1/3, 2/5, 1/15 and the table 2^(-i/256), i = 0..255.
struct DfConsts {
  float ln2_h, ln2_l, ilog2_h, ilog2_l;
  float third_h, third_l, fifth2_h, fifth2_l, fifteenth_h, fifteenth_l;
  float tab_h[256], tab_l[256];
};

// exp(-r), r >= 0: r/ln2 = (256 q + i)/256 + f with 0 <= f < 1/256, so
// exp(-r) = 2^-q * 2^(-i/256) * exp(-g), g = f ln2 < 0.0028, and
// exp(-g) = 1 - g + g^2 (1/2 - g (1/6 - g/24)) (truncation < 2e-15 relative);
// the table is read from shared memory (tab_h, tab_l) because the index
// differs across a warp.
__device__ __forceinline__ df df_exp_neg(df r, const DfConsts& c, const float* tab_h,
                                         const float* tab_l) {
  if (r.h > 85.0f) return {0.0f, 0.0f};
  df t = df_mul(r, df{c.ilog2_h, c.ilog2_l});
  float kf = floorf(__fmul_rn(t.h, 256.0f));
  int k = (int)kf;
  df f = fast_two_sum(__fsub_rn(t.h, __fmul_rn(kf, 0.00390625f)), t.l);
  df g = df_mul(f, df{c.ln2_h, c.ln2_l});
  df g2 = df_mul(g, g);
  float inner = __fmul_rn(g.h, __fmaf_rn(-g.h, 0.041666668f, 0.16666667f));
  df w = two_sum(0.5f, -inner);
  df term = df_mul(g2, w);
  df one_m_g = two_sum(1.0f, -g.h);
  one_m_g = fast_two_sum(one_m_g.h, __fsub_rn(one_m_g.l, g.l));
  df e = df_add(one_m_g, term);
  e = df_mul(e, df{tab_h[k & 255], tab_l[k & 255]});
  // 2^-(k >> 8) is a normal float (k >> 8 <= 122 for r <= 85): an exact
  // power-of-two multiply, rounded once like ldexpf
  const float sc = __int_as_float((127 - (k >> 8)) << 23);
  return {__fmul_rn(e.h, sc), __fmul_rn(e.l, sc)};
}

// Matern correlation M_nu(r) for nu = nu2/2 (closed forms), r and s = r^2 in double-float.
__device__ __forceinline__ df df_matern(df r, df s, int nu2, const DfConsts& c, const float* tab_h,
                                        const float* tab_l) {
  df e = df_exp_neg(r, c, tab_h, tab_l);
  const df one = {1.0f, 0.0f};
  switch (nu2) {
    case 1:
      return e;
    case 3:
      return df_mul(df_add(one, r), e);
    case 5: {
      df p = df_add(df_add(one, r), df_mul(s, df{c.third_h, c.third_l}));
      return df_mul(p, e);
    }
    default: {
      // 1 + r + 2 r^2 / 5 + r^3 / 15
      df p = df_add(df_add(one, r), df_mul(s, df{c.fifth2_h, c.fifth2_l}));
      p = df_add(p, df_mul(df_mul(s, r), df{c.fifteenth_h, c.fifteenth_l}));
      return df_mul(p, e);
    }
  }
}

}  // namespace sbv
