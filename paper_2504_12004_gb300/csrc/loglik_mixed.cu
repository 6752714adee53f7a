// Mixed-precision block log-likelihood (Alg. 5 per block).
//
// Per (theta, block) item, one CTA:
//  1. gather the N = m_i + bs_i points as double-float coordinates (split
//     once per call from FP64 X), scale by 1/beta in double-float, centre on
//     the first point and re-split on a common power-of-two grid so that every
//     difference of the float heads is exact;
//  2. evaluate the joint covariance in double-float (dfloat.cuh): the float
//     head of each entry feeds the FP32 factorisation; for the 16 x 16
//     diagonal tiles the head and tail are kept apart; the full double-float
//     matrix goes to a per-CTA scratch slice (L2-resident) for the
//     refinement residual;
//  3. blocked right-looking Cholesky: each diagonal tile is formed as
//     (double-float original) - (FP32-accumulated updates) with one exact
//     subtraction, rounded, and factored in FP32 registers by one warp; the
//     panel solve and the trailing update run in FP32; y is bordered as row
//     N so the factorisation also yields w0 = L^{-1} y;
//  4. x0 = L^-T w0 and x0_J = L_JJ^-T w0_J in FP32 (one two-column sweep);
//  5. one step of iterative refinement: r = y - Sigma x0 and r_J = y_J -
//     Sigma_JJ x0_J accumulated in double-float from the scratch matrix, the
//     corrections solved in FP32;
//  6. l_i = -1/2 [bs log 2pi + 2 sum_{t>=m} log L_tt + y^T x - y_J^T x_J],
//     log L_tt = e ln2 + log(mantissa) with the sums in FP64.
// y^T Sigma^{-1} y - y_J^T Sigma_JJ^{-1} y_J is the quadratic form of the
// Schur complement Sigma^lk - Sigma^cor of Alg. 5 (applied to y_B - mu^new),
// and the trailing log-determinant is its log-determinant.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "block_common.cuh"
#include "dfloat.cuh"
#include "sbv_internal.cuh"

namespace sbv {

static __constant__ DfConsts c_df;

constexpr int MX_THREADS = 256;
constexpr int MX_WARPS = MX_THREADS / 32;
constexpr int NB = 16;  // diagonal tile size

struct MixedLayout {
  int ncap;    // largest N held (rows 0..ncap-1 plus the bordered row)
  int ntile;   // tiles of NB columns
  int d;
  size_t off_A, off_K, off_vh, off_vl, off_y, off_v, off_part, bytes;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline MixedLayout mixed_layout(int ncap, int d) {
  MixedLayout L;
  L.ncap = ncap;
  L.ntile = (ncap + NB - 1) / NB;
  L.d = d;
  size_t o = 0;
  L.off_K = o;    o += (size_t)L.ntile * NB * NB * sizeof(float2);   // diagonal-tile originals
  L.off_y = o;    o += align_up((size_t)(ncap + 1) * sizeof(float2), 16);
  L.off_v = o;    o += align_up((size_t)6 * (ncap + 1) * sizeof(float), 16);  // x0 x0J r1 r2 ldiag idiag
  L.off_vh = o;   o += align_up((size_t)d * ncap * sizeof(float), 16);
  L.off_vl = o;   o += align_up((size_t)d * ncap * sizeof(float), 16);
  L.off_A = o;    o += align_up((size_t)(ncap + 1) * (ncap + 2) / 2 * sizeof(float), 16);
  L.off_part = L.off_vh;  // residual partial sums reuse the coordinate area
  L.bytes = o;
  return L;
}

// ---------------------------------------------------------------------------
// blocked FP32 triangular solves with the factor packed in A; idiag holds
// 1/L_tt.  Two right-hand sides, one per half-warp in the diagonal steps.
// ---------------------------------------------------------------------------
__device__ void fwd_solve2(const float* A, const float* idiag, int N, float* b1, float* b2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k0 = 0; k0 < N; k0 += NB) {
    const int k1 = min(k0 + NB, N), nbk = k1 - k0;
    if (warp == 0) {
      const int h = lane >> 4, r = lane & 15;
      float* b = h ? b2 : b1;
      const int row = k0 + r;
      const bool live = r < nbk;
      float v = live ? b[row] : 0.0f;
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        if (c < nbk) {
          float vc = __shfl_sync(0xffffffffu, v, (h << 4) + c) * idiag[k0 + c];
          if (r == c) v = vc;
          if (r > c && live) v = fmaf(-A[tri(row, k0 + c)], vc, v);
        }
      }
      if (live) b[row] = v;
    }
    __syncthreads();
    for (int i = k1 + threadIdx.x; i < N; i += blockDim.x) {
      float s1 = 0.0f, s2 = 0.0f;
      const float* Ai = A + tri(i, 0);
      for (int k = k0; k < k1; ++k) {
        const float a = Ai[k];
        s1 = fmaf(a, b1[k], s1);
        s2 = fmaf(a, b2[k], s2);
      }
      b1[i] -= s1;
      b2[i] -= s2;
    }
    __syncthreads();
  }
}

__device__ void bwd_solve2(const float* A, const float* idiag, int N, float* b1, float* b2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntile = (N + NB - 1) / NB;
  for (int kt = ntile - 1; kt >= 0; --kt) {
    const int k0 = kt * NB, k1 = min(k0 + NB, N), nbk = k1 - k0;
    if (warp == 0) {
      const int h = lane >> 4, r = lane & 15;
      float* b = h ? b2 : b1;
      const int row = k0 + r;
      const bool live = r < nbk;
      float v = live ? b[row] : 0.0f;
#pragma unroll
      for (int c = NB - 1; c >= 0; --c) {
        if (c < nbk) {
          float vc = __shfl_sync(0xffffffffu, v, (h << 4) + c) * idiag[k0 + c];
          if (r == c) v = vc;
          if (r < c) v = fmaf(-A[tri(k0 + c, row)], vc, v);
        }
      }
      if (live) b[row] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k0; i += blockDim.x) {
      float s1 = 0.0f, s2 = 0.0f;
      for (int k = k0; k < k1; ++k) {
        const float Lki = A[tri(k, i)];
        s1 = fmaf(Lki, b1[k], s1);
        s2 = fmaf(Lki, b2[k], s2);
      }
      b1[i] -= s1;
      b2[i] -= s2;
    }
    __syncthreads();
  }
}

// FP64 CTA sum, same value returned on every thread.
__device__ double cta_sum_mx(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < MX_WARPS; ++q) s += red[q];
  __syncthreads();
  return s;
}

// X split once per call into float pairs (hi, lo), hi + lo = x to ~2^-48 relative.
__global__ void split_points_kernel(const double* __restrict__ X, int64_t total,
                                    float2* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = X[i];
    const float h = (float)x;
    out[i] = make_float2(h, (float)(x - (double)h));
  }
}

struct MixedArgs {
  LoglikArgs a;
  const float2* Xs;      // split FP64 points, or NULL for FP32 points (a.X read directly)
  float2* scratch;
  size_t scratch_stride;
  MixedLayout lay;
};

__global__ void __launch_bounds__(MX_THREADS, 2)
loglik_mixed_kernel(MixedArgs P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const LoglikArgs& a = P.a;
  const MixedLayout& lay = P.lay;
  float2* Kd = (float2*)(smem + lay.off_K);
  float2* yv = (float2*)(smem + lay.off_y);
  float* vec = (float*)(smem + lay.off_v);
  float* vh = (float*)(smem + lay.off_vh);
  float* vl = (float*)(smem + lay.off_vl);
  float* A = (float*)(smem + lay.off_A);
  __shared__ float tab_h[256], tab_l[256];
  __shared__ unsigned int s_item;
  __shared__ int s_fail;
  __shared__ double red[MX_WARPS];
  __shared__ float s_org_h[SBV_MAX_DIM], s_org_l[SBV_MAX_DIM];
  __shared__ float s_grid;
  const DfConsts& C = c_df;
  float2* S = P.scratch + (size_t)blockIdx.x * P.scratch_stride;
  const int d = a.d, cap = lay.ncap;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned int total = (unsigned int)(a.bc * a.B);
  const double log2pi = 1.8378770664093454836;
  float* x0 = vec;
  float* x0J = vec + (cap + 1);
  float* r1 = vec + 2 * (cap + 1);
  float* r2 = vec + 3 * (cap + 1);
  float* ldiag = vec + 4 * (cap + 1);
  float* idiag = vec + 5 * (cap + 1);

  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    tab_h[i] = C.tab_h[i];
    tab_l[i] = C.tab_l[i];
  }

  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1u);
    __syncthreads();
    const unsigned int item = s_item;
    if (item >= total) break;
    const int th_i = (int)(item / a.bc);
    const int64_t blk = (int64_t)(item % a.bc);
    const ThetaDev& th = a.theta[th_i];
    const int bs = (int)(a.ptr[blk + 1] - a.ptr[blk]);
    const int mb = a.cnt[blk];
    const int N = mb + bs;
    if (N > cap) {
      if (threadIdx.x == 0) {
        a.terms[item] = __longlong_as_double(0x7ff8000000000000ll);
        if (a.status) a.status[item] = SBV_EUNSUPPORTED;
        record_failure(a.dstat, SBV_EUNSUPPORTED, (int)blk, th_i);
      }
      __syncthreads();
      continue;
    }
    const int64_t base = a.ptr[blk];
    // ---- 1. gather and scale in double-float; centre on point 0
    if (threadIdx.x == 0) s_fail = 0;
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      int64_t id = p < mb ? (int64_t)a.nbr[blk * a.m + p] : (int64_t)a.pts[base + (p - mb)];
      const double yy = a.y[id];
      const float yh = (float)yy;
      yv[p] = make_float2(yh, (float)(yy - (double)yh));
    }
    float mx = 0.0f;
    for (int e = threadIdx.x; e < N * d; e += blockDim.x) {
      const int p = e / d, t = e - p * d;
      int64_t id = p < mb ? (int64_t)a.nbr[blk * a.m + p] : (int64_t)a.pts[base + (p - mb)];
      df x;
      if (P.Xs) {
        const float2 xs = P.Xs[id * d + t];
        x = {xs.x, xs.y};
      } else {
        x = {((const float*)a.X)[id * d + t], 0.0f};
      }
      const df u = df_mul(x, df{th.ib_h[t], th.ib_l[t]});
      vh[t * N + p] = u.h;  // temporarily the uncentred coordinate
      vl[t * N + p] = u.l;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < d; t += blockDim.x) {
      s_org_h[t] = vh[t * N];
      s_org_l[t] = vl[t * N];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < N * d; e += blockDim.x) {
      const int t = e / N;
      const df v = df_sub_acc(df{vh[e], vl[e]}, df{s_org_h[t], s_org_l[t]});
      vh[e] = v.h;
      vl[e] = v.l;
      mx = fmaxf(mx, fabsf(v.h));
    }
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = (double)mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      float M = 0.0f;
      for (int q = 0; q < MX_WARPS; ++q) M = fmaxf(M, (float)red[q]);
      int ex;
      frexpf(M * 1.0001f + 1e-30f, &ex);  // M < 2^ex
      s_grid = ldexpf(1.0f, ex - 22);      // |head| / grid < 2^22: heads and their differences exact
    }
    __syncthreads();
    {
      const float g = s_grid, ig = 1.0f / g;  // powers of two: exact scaling
      for (int e = threadIdx.x; e < N * d; e += blockDim.x) {
        const float h = vh[e];
        const float hq = rintf(h * ig) * g;   // on the grid, exact
        vh[e] = hq;
        vl[e] = __fadd_rn(__fsub_rn(h, hq), vl[e]);  // h - hq is exact
      }
    }
    __syncthreads();
    // ---- 2. double-float covariance
    {
      const df s2 = {th.s2_h, th.s2_l};
      const df diag = {th.diag_h, th.diag_l};
      const int npair = N * (N + 1) / 2;
      int i = 0, j = threadIdx.x;
      while (j > i) { j -= i + 1; ++i; }
      for (int l = threadIdx.x; l < npair; l += blockDim.x) {
        df K;
        if (i == j) {
          K = diag;
        } else {
          float sh = 0.0f, sl = 0.0f;
          for (int t = 0; t < d; ++t) {
            const float dh = __fsub_rn(vh[t * N + i], vh[t * N + j]);  // exact
            const float dl = __fsub_rn(vl[t * N + i], vl[t * N + j]);
            const float p = __fmul_rn(dh, dh);
            float pe = __fmaf_rn(dh, dh, -p);
            pe = __fmaf_rn(2.0f * dh, dl, pe);
            pe = __fmaf_rn(dl, dl, pe);
            const df q = two_sum(sh, p);
            sh = q.h;
            sl = __fadd_rn(sl, __fadd_rn(q.l, pe));
          }
          const df s = fast_two_sum(sh, sl);
          const df r = df_sqrt(s);
          K = df_mul(s2, df_matern(r, s, a.nu2, C, tab_h, tab_l));
        }
        const int ti = i / NB, tj = j / NB;
        if (ti == tj) {
          Kd[(size_t)ti * NB * NB + (i % NB) * NB + (j % NB)] = make_float2(K.h, K.l);
          A[tri(i, j)] = 0.0f;
        } else {
          A[tri(i, j)] = K.h;
        }
        S[(size_t)j * N + i] = make_float2(K.h, K.l);
        S[(size_t)i * N + j] = make_float2(K.h, K.l);
        j += blockDim.x;
        while (j > i) { j -= i + 1; ++i; }
      }
      for (int p = threadIdx.x; p < N; p += blockDim.x) A[tri(N, p)] = yv[p].x;
    }
    __syncthreads();
    // ---- 3. blocked Cholesky
    for (int k0 = 0; k0 < N; k0 += NB) {
      const int k1 = min(k0 + NB, N), nbk = k1 - k0;
      if (warp == 0) {
        // lane r holds row r of the tile: original (double-float) plus the
        // accumulated FP32 updates (held negated in A), one exact subtraction
        const float2* Kt = Kd + (size_t)(k0 / NB) * NB * NB;
        const int r = lane;
        float row[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          float v = 0.0f;
          if (r < nbk && c <= r) {
            const float2 k = Kt[r * NB + c];
            const df s = two_sum(k.x, A[tri(k0 + r, k0 + c)]);
            v = __fadd_rn(s.h, __fadd_rn(s.l, k.y));
          }
          row[c] = v;
        }
        bool bad = false;
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if (c < nbk) {
            const float dcc = __shfl_sync(0xffffffffu, row[c], c);
            bad |= !(dcc > 0.0f);
            const float Lcc = sqrtf(fmaxf(dcc, 1e-30f));
            const float inv = 1.0f / Lcc;
            if (r == c) row[c] = Lcc;
            if (r > c) row[c] *= inv;
#pragma unroll
            for (int c2 = c + 1; c2 < NB; ++c2) {
              const float v = __shfl_sync(0xffffffffu, row[c], c2);  // L[c2][c]
              if (r >= c2 && c2 < nbk) row[c2] = fmaf(-row[c], v, row[c2]);
            }
          }
        }
        if (r < nbk) {
          float Lrr = 0.0f;
#pragma unroll
          for (int c = 0; c < NB; ++c) {
            if (c <= r) A[tri(k0 + r, k0 + c)] = row[c];
            if (c == r) Lrr = row[c];
          }
          ldiag[k0 + r] = Lrr;
          idiag[k0 + r] = 1.0f / Lrr;
        }
        if (bad && lane == 0) s_fail = 1;
      }
      __syncthreads();
      if (s_fail) break;
      // panel solve: rows k1..N, A(i, k0:k1) <- A(i, k0:k1) L_kk^{-T}
      for (int i = k1 + threadIdx.x; i <= N; i += blockDim.x) {
        float v[NB];
        float* Ai = A + tri(i, 0) + k0;
#pragma unroll
        for (int c = 0; c < NB; ++c) v[c] = c < nbk ? Ai[c] : 0.0f;
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if (c < nbk) {
            const float* Lc = A + tri(k0 + c, k0);
            float s = v[c];
#pragma unroll
            for (int c2 = 0; c2 < NB; ++c2)
              if (c2 < c) s = fmaf(-v[c2], Lc[c2], s);
            v[c] = s * idiag[k0 + c];
          }
        }
#pragma unroll
        for (int c = 0; c < NB; ++c)
          if (c < nbk) Ai[c] = v[c];
      }
      __syncthreads();
      // trailing update of rows k1..N, columns k1..min(i, N-1), 4x4 register blocks
      const int T = N + 1 - k1;
      if (T > 0) {
        const int RB = (T + 3) >> 2;
        const int nblk = RB * (RB + 1) / 2;
        int bi = 0, bj = threadIdx.x;
        while (bj > bi) { bj -= bi + 1; ++bi; }
        for (int l = threadIdx.x; l < nblk; l += blockDim.x) {
          const int i0 = k1 + 4 * bi, j0 = k1 + 4 * bj;
          float acc[4][4];
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] = 0.0f;
          const float* Ar[4];
          const float* Ac[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            Ar[p] = A + tri(min(i0 + p, N), 0) + k0;
            Ac[p] = A + tri(min(j0 + p, N), 0) + k0;
          }
          for (int k = 0; k < nbk; ++k) {
            float ar[4], ac[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              ar[p] = Ar[p][k];
              ac[p] = Ac[p][k];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
              for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(ar[p], ac[q], acc[p][q]);
          }
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const int ii = i0 + p;
            if (ii > N) continue;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int jj = j0 + q;
              if (jj <= ii && jj < N) A[tri(ii, jj)] -= acc[p][q];
            }
          }
          bj += blockDim.x;
          while (bj > bi) { bj -= bi + 1; ++bi; }
        }
      }
      __syncthreads();
    }
    if (s_fail) {
      if (threadIdx.x == 0) {
        a.terms[item] = __longlong_as_double(0x7ff8000000000000ll);
        if (a.status) a.status[item] = SBV_ENOTSPD;
        record_failure(a.dstat, SBV_ENOTSPD, (int)blk, th_i);
      }
      __syncthreads();
      continue;
    }
    // ---- 4. x0 = L^-T w0, x0J = L_JJ^-T w0_J  (w0 = row N of A)
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      const float w = A[tri(N, p)];
      x0[p] = w;
      x0J[p] = p < mb ? w : 0.0f;
    }
    __syncthreads();
    bwd_solve2(A, idiag, N, x0, x0J);
    // ---- 5. residuals in double-float; all warps: (32-row group, column chunk) tasks
    {
      const int G = (N + 31) / 32;
      const int CH = max(1, MX_WARPS / G);
      const int chunk = (N + CH - 1) / CH;
      float4* part = (float4*)(smem + lay.off_part);  // [CH][N] partial (h1, l1, h2, l2)
      for (int task = warp; task < G * CH; task += MX_WARPS) {
        const int g = task / CH, c = task % CH;
        const int i = g * 32 + lane;
        const int j0 = c * chunk, j1 = min(N, j0 + chunk);
        float h1 = 0.0f, l1 = 0.0f, h2 = 0.0f, l2 = 0.0f;
        if (i < N) {
          const bool inJ = i < mb;
#pragma unroll 4
          for (int j = j0; j < j1; ++j) {
            const float2 s = S[(size_t)j * N + i];
            const float xj = x0[j];
            const float p = __fmul_rn(s.x, xj);
            float pe = __fmaf_rn(s.x, xj, -p);
            pe = __fmaf_rn(s.y, xj, pe);
            const df q = two_sum(h1, p);
            h1 = q.h;
            l1 = __fadd_rn(l1, __fadd_rn(q.l, pe));
            if (inJ && j < mb) {
              const float zj = x0J[j];
              const float p2 = __fmul_rn(s.x, zj);
              float pe2 = __fmaf_rn(s.x, zj, -p2);
              pe2 = __fmaf_rn(s.y, zj, pe2);
              const df q2 = two_sum(h2, p2);
              h2 = q2.h;
              l2 = __fadd_rn(l2, __fadd_rn(q2.l, pe2));
            }
          }
          part[(size_t)c * N + i] = make_float4(h1, l1, h2, l2);
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        df s1 = {0.0f, 0.0f}, s2 = {0.0f, 0.0f};
        for (int c = 0; c < CH; ++c) {
          const float4 q = part[(size_t)c * N + i];
          s1 = df_add(s1, fast_two_sum(q.x, q.y));
          s2 = df_add(s2, fast_two_sum(q.z, q.w));
        }
        const df y = {yv[i].x, yv[i].y};
        r1[i] = df_sub_acc(y, s1).h;
        r2[i] = i < mb ? df_sub_acc(y, s2).h : 0.0f;
      }
      __syncthreads();
    }
    // corrections: (L L^T)^{-1} r and (L_JJ L_JJ^T)^{-1} r_J
    fwd_solve2(A, idiag, N, r1, r2);
    for (int p = mb + threadIdx.x; p < N; p += blockDim.x) r2[p] = 0.0f;
    __syncthreads();
    bwd_solve2(A, idiag, N, r1, r2);
    // ---- 6. log-determinant and quadratic forms, summed in FP64
    double v = 0.0;
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      const double yp = (double)yv[p].x + (double)yv[p].y;
      v += yp * ((double)x0[p] + (double)r1[p]);
      if (p < mb) v -= yp * ((double)x0J[p] + (double)r2[p]);
      if (p >= mb) {
        int ex;
        const float mant = frexpf(ldiag[p], &ex);  // L = mant 2^ex, mant in [0.5, 1)
        v += 2.0 * ((double)ex * 0.69314718055994530942 + (double)logf(mant));
      }
    }
    const double s = cta_sum_mx(v, red);
    if (threadIdx.x == 0) {
      const double term = -0.5 * ((double)bs * log2pi + s);
      a.terms[item] = term;
      const bool ok = isfinite(term);
      if (a.status) a.status[item] = ok ? 0 : SBV_ENOTSPD;
      if (!ok) record_failure(a.dstat, SBV_ENOTSPD, (int)blk, th_i);
    }
    __syncthreads();
  }
}

static bool g_consts_ready[64];

static int upload_df_consts(sbv_ctx* ctx) {
  if (ctx->device < 64 && g_consts_ready[ctx->device]) return SBV_OK;
  DfConsts c;
  auto split = [](double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
  };
  for (int i = 0; i < 256; ++i) split(exp2(-i / 256.0), c.tab_h[i], c.tab_l[i]);
  split(0.69314718055994530942, c.ln2_h, c.ln2_l);
  split(1.44269504088896340736, c.ilog2_h, c.ilog2_l);
  split(1.0 / 3.0, c.third_h, c.third_l);
  split(2.0 / 5.0, c.fifth2_h, c.fifth2_l);
  split(1.0 / 15.0, c.fifteenth_h, c.fifteenth_l);
  SBV_CUDA_TRY(ctx, cudaMemcpyToSymbol(c_df, &c, sizeof(c)));
  if (ctx->device < 64) g_consts_ready[ctx->device] = true;
  return SBV_OK;
}

int launch_loglik_mixed(sbv_ctx* ctx, const LoglikArgs& a0, int nmax, cudaStream_t s) {
  int st = 0;
  if ((st = upload_df_consts(ctx))) return st;
  MixedArgs P;
  P.a = a0;
  const int ncap = std::max(nmax, 1);
  P.lay = mixed_layout(ncap, a0.d);
  // residual partials (CH x N float4) reuse the coordinate area
  const int G = (ncap + 31) / 32;
  const int CH = std::max(1, MX_WARPS / G);
  const size_t need_part = (size_t)CH * ncap * sizeof(float4);
  const size_t have_part = P.lay.off_A - P.lay.off_vh;
  if (need_part > have_part) {
    const size_t extra = align_up(need_part - have_part, 16);
    P.lay.off_A += extra;
    P.lay.bytes += extra;
  }
  if (P.lay.bytes + 4096 > ctx->smem_optin)
    return fail(ctx, SBV_EUNSUPPORTED,
                "mixed path: a block with N=%d (d=%d) needs %zu bytes of shared memory", nmax,
                a0.d, P.lay.bytes);
  // split FP64 points once per call
  const int64_t total = a0.n * a0.d;
  if (a0.dtype == SBV_F64) {
    float2* xs = (float2*)ws_get(ctx, WS_XSPLIT, (size_t)total * sizeof(float2), &st);
    if (!xs) return st;
    int g = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 16);
    split_points_kernel<<<std::max(g, 1), 256, 0, s>>>((const double*)a0.X, total, xs);
    SBV_LAUNCH_CHECK(ctx, "split_points_kernel");
    P.Xs = xs;
  } else {
    P.Xs = nullptr;
  }
  const size_t static_smem = 2 * 256 * 4 + 1024;
  int per_sm = (int)std::max<size_t>(1, (228 * 1024) / (P.lay.bytes + static_smem + 1024));
  int grid = ctx->num_sms * std::min(per_sm, 2);
  int64_t items = a0.bc * (int64_t)a0.B;
  if (grid > items) grid = (int)items;
  P.scratch_stride = align_up((size_t)ncap * ncap, 64);
  P.scratch = (float2*)ws_get(ctx, WS_MATRIX, P.scratch_stride * grid * sizeof(float2), &st);
  if (!P.scratch) return st;
  SBV_CUDA_TRY(ctx, cudaFuncSetAttribute(loglik_mixed_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)P.lay.bytes));
  loglik_mixed_kernel<<<grid, MX_THREADS, P.lay.bytes, s>>>(P);
  SBV_LAUNCH_CHECK(ctx, "loglik_mixed_kernel");
  return SBV_OK;
}

}  // namespace sbv
