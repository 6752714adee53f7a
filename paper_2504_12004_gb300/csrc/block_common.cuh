// Device building blocks shared by the block log-likelihood and prediction
// kernels: per-theta parameters, the gather of a block's points, the scaled
// Matern covariance (Eq. scale, Eq. maternkernel) and the work counter.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "sbv.h"
#include "sbv_internal.cuh"

namespace sbv {

// Derived parameters of one theta row.
struct ThetaDev {
  double sigma2;
  double tau2;
  double inv_beta[SBV_MAX_DIM];
  // the same values as float pairs (head, tail) for double-float arithmetic
  float s2_h, s2_l, diag_h, diag_l;   // sigma^2 and sigma^2 + tau^2
  float ib_h[SBV_MAX_DIM], ib_l[SBV_MAX_DIM];
};

// Closed-form Matern correlation 2^(1-nu)/Gamma(nu) r^nu K_nu(r), nu = nu2/2,
// at the scaled distance r (no sqrt(2 nu) factor).
__device__ __forceinline__ double matern64(double r, int nu2) {
  double e = exp(-r);
  switch (nu2) {
    case 1: return e;
    case 3: return (1.0 + r) * e;
    case 5: return fma(r, fma(r, 1.0 / 3.0, 1.0), 1.0) * e;
    default: return fma(r, fma(r, fma(r, 1.0 / 15.0, 0.4), 1.0), 1.0) * e;
  }
}

// Record the first failing item on the context's device status.
__device__ __forceinline__ void record_failure(DevStatus* st, int code, int item, int theta) {
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->item = item;
    st->theta = theta;
  }
  atomicAdd(&st->count, 1);
}

struct LoglikArgs {
  const void* X;
  int dtype;
  const double* y;
  int64_t n;
  int d;
  const int64_t* ptr;
  const int32_t* pts;
  const int32_t* nbr;
  const int32_t* cnt;
  int64_t bc;
  int m;
  const ThetaDev* theta;
  int B;
  int nu2;
  int ncap;                // largest N the launch can hold
  double* terms;           // B x bc
  int32_t* status;         // B x bc or NULL
  DevStatus* dstat;
  unsigned int* counter;   // work counter
  double* gmat;            // global scratch (one matrix per CTA) or NULL
  size_t gmat_stride;      // doubles per CTA slice
  // list mode (FP64 kernels only): when `list` is not NULL the items are
  // list[0 .. *list_n - 1] (filled by a previous kernel on the stream)
  const unsigned int* list;
  const unsigned int* list_n;
};

template <typename T>
__device__ __forceinline__ double ld_x(const void* X, int64_t i) {
  return (double)((const T*)X)[i];
}

// FP64 block-kernel launch plan (loglik.cu).
struct Fp64Plan {
  size_t smem;         // dynamic shared memory per CTA
  size_t gmat_stride;  // doubles per CTA of global matrix scratch, 0 when in shared memory
  int grid;
};
int fp64_plan(sbv_ctx* ctx, int nmax, int d, int64_t items, Fp64Plan* o);
int fp64_enqueue(sbv_ctx* ctx, const LoglikArgs& a, const Fp64Plan& o, cudaStream_t s);
int fp64_prepare(sbv_ctx* ctx);
// FP64 kernel over the items a mixed kernel handed over (list mode); the
// global matrices come from gmat_owned, or the context workspace when NULL
int fp64_fallback_enqueue(sbv_ctx* ctx, const LoglikArgs& a, int nmax, const unsigned int* list,
                          const unsigned int* list_n, unsigned int* counter, cudaStream_t s,
                          double* gmat_owned = nullptr);
int run_max_n(sbv_ctx* ctx, const int64_t* ptr, const int32_t* cnt, int64_t bc, int* out,
              cudaStream_t s);
int reduce_enqueue(sbv_ctx* ctx, const double* terms, int64_t bc, int B, double* ll,
                   cudaStream_t s);
std::vector<ThetaDev> derive_theta_rows(const double* h, int B, int d);

// Packed lower-triangular index of (i, j), j <= i.
__device__ __forceinline__ int tri(int i, int j) { return (i * (i + 1) >> 1) + j; }

}  // namespace sbv
