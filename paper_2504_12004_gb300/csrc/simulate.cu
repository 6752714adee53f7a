// Conditional simulation at the test points (Sec. 5.5): for every test point j,
// ndraws samples from N(mu_j, sigma_j), where mu_j and sigma_j are the
// predictive mean and variance (the diagonal of Sigma^new); then the sample
// mean, the sample variance (divisor ndraws - 1) and the 95 % interval
// sample mean -/+ z_{0.975} sample standard deviation.
//
// Random numbers: Philox4x64-10 (Salmon, Moraes, Dror & Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC 2011), a counter-based generator, so that
// every draw is a pure function of (seed, test point, draw index) and any
// subset can be recomputed independently.  Draw k of test point j uses the
// output block of counter (k / 4, base + j, 0, 0) under key (seed, 0): words
// 2p and 2p + 1 (p = (k mod 4) / 2) become two uniforms u = (w >> 12 + 1/2) 2^-52 in
// (0, 1), and the Box-Muller transform (Box & Muller, 1958) turns them into
// sqrt(-2 ln u1) cos(2 pi u2) (k even) and sqrt(-2 ln u1) sin(2 pi u2) (k odd).
//
// One warp per test point: lane l takes the output blocks l, l + 32, ...,
// keeps a running mean and sum of squared deviations (Welford), and the 32
// partial statistics are merged pairwise (Chan, Golub & LeVeque) through
// shuffles.  FP64 throughout; the paper fixes no precision here.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sbv_internal.cuh"

namespace sbv {

namespace {

constexpr uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t kPhiloxM1 = 0xCA5A826395121157ull;
constexpr uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ull;  // golden ratio
constexpr uint64_t kPhiloxW1 = 0xBB67AE8584CAA73Bull;  // sqrt(3) - 1
// z_{alpha/2} for alpha = 0.05: the 0.975 quantile of the standard normal
constexpr double kZ975 = 1.959963984540054;

struct U64x4 {
  uint64_t v[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(U64x4 c, uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t lo0 = kPhiloxM0 * c.v[0], hi0 = __umul64hi(kPhiloxM0, c.v[0]);
    const uint64_t lo1 = kPhiloxM1 * c.v[2], hi1 = __umul64hi(kPhiloxM1, c.v[2]);
    U64x4 o;
    o.v[0] = hi1 ^ c.v[1] ^ k0;
    o.v[1] = lo1;
    o.v[2] = hi0 ^ c.v[3] ^ k1;
    o.v[3] = lo0;
    c = o;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

__device__ __forceinline__ double unit_open(uint64_t w) {
  return ((double)(w >> 12) + 0.5) * 0x1.0p-52;   // exact: never 0 or 1
}

struct Moments {
  double n, mean, m2;
};

__device__ __forceinline__ void welford(Moments& a, double x) {
  a.n += 1.0;
  const double dx = x - a.mean;
  a.mean += dx / a.n;
  a.m2 = fma(dx, x - a.mean, a.m2);
}

__device__ __forceinline__ Moments merge(Moments a, Moments b) {
  if (b.n == 0.0) return a;
  if (a.n == 0.0) return b;
  const double n = a.n + b.n, dx = b.mean - a.mean;
  Moments o;
  o.n = n;
  o.mean = a.mean + dx * (b.n / n);
  o.m2 = a.m2 + b.m2 + dx * dx * (a.n * b.n / n);
  return o;
}

__global__ void __launch_bounds__(256)
simulate_kernel(const double* __restrict__ mean, const double* __restrict__ var, int64_t nt,
                int ndraws, uint64_t seed, uint64_t base, double* __restrict__ mu,
                double* __restrict__ var_s, double* __restrict__ lo, double* __restrict__ hi,
                double* __restrict__ draws) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int nblk = (ndraws + 3) >> 2;
  for (int64_t j = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); j < nt;
       j += warps) {
    const double m = mean[j], sd = sqrt(var[j]);
    Moments acc = {0.0, 0.0, 0.0};
    for (int b = lane; b < nblk; b += 32) {
      const U64x4 ctr = {{(uint64_t)b, base + (uint64_t)j, 0ull, 0ull}};
      const U64x4 w = philox4x64_10(ctr, seed, 0ull);
      double x[4];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const double u1 = unit_open(w.v[2 * p]), u2 = unit_open(w.v[2 * p + 1]);
        const double r = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        x[2 * p] = fma(sd, r * cs, m);
        x[2 * p + 1] = fma(sd, r * sn, m);
      }
      const int k0 = 4 * b;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (k0 + q < ndraws) {
          welford(acc, x[q]);
          if (draws) draws[j * (int64_t)ndraws + k0 + q] = x[q];
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      Moments b;
      b.n = __shfl_xor_sync(0xffffffffu, acc.n, o);
      b.mean = __shfl_xor_sync(0xffffffffu, acc.mean, o);
      b.m2 = __shfl_xor_sync(0xffffffffu, acc.m2, o);
      // merge in lane order so that every lane holds the same result
      acc = (lane & o) ? merge(b, acc) : merge(acc, b);
    }
    if (lane == 0) {
      const double v = acc.m2 / (double)(ndraws - 1);
      const double h = kZ975 * sqrt(v);
      mu[j] = acc.mean;
      var_s[j] = v;
      lo[j] = acc.mean - h;
      hi[j] = acc.mean + h;
    }
  }
}

}  // namespace

int run_simulate(sbv_ctx* ctx, const double* mean, const double* var, int64_t nt, int ndraws,
                 uint64_t seed, uint64_t base, double* mu, double* var_s, double* lo, double* hi,
                 double* draws, cudaStream_t s) {
  if (nt == 0) return SBV_OK;
  const int64_t want = (nt + 7) / 8;
  const int grid = (int)std::min<int64_t>(want, (int64_t)ctx->num_sms * 16);
  simulate_kernel<<<grid, 256, 0, s>>>(mean, var, nt, ndraws, seed, base, mu, var_s, lo, hi,
                                          draws);
  SBV_CUDA_TRY(ctx, cudaGetLastError());
  return SBV_OK;
}

}  // namespace sbv
