// Mixed-precision block log-likelihood (Alg. 5 per block).
//
// Per (theta, block) item, one CTA:
//  1. gather the N = m_i + bs_i points, scaled by 1/beta in FP64, centred on
//     the first point and split into float pairs on a common power-of-two
//     grid (hi exact on the grid, lo the float remainder), so that every
//     coordinate difference hi_a - hi_b is exact in FP32;
//  2. evaluate the joint covariance in double-float (dfloat.cuh): its float
//     head feeds the FP32 factorisation, the diagonal 16x16 tiles are kept in
//     FP64, and the full double-float matrix goes to a per-CTA scratch slice
//     (L2-resident) for the refinement residual;
//  3. blocked right-looking Cholesky: FP64 factorisation of each diagonal
//     tile (its FP32-accumulated updates subtracted from the FP64 original),
//     FP32 panel solve and FP32 trailing update, with y bordered as row N so
//     the factorisation also yields w0 = L^{-1} y;
//  4. x0 = L^-T w0 and x0_J = L_JJ^-T w0_J in FP32 (one two-column sweep);
//  5. one step of iterative refinement: r = y - Sigma x0, r_J = y_J -
//     Sigma_JJ x0_J accumulated in double-float from the scratch matrix, the
//     corrections solved in FP32;
//  6. l_i = -1/2 [bs log 2pi + 2 sum_{t>=m} log L_tt + y^T x - y_J^T x_J]
//     with the log-determinant and both quadratic forms in FP64.
// y^T Sigma^{-1} y - y_J^T Sigma_JJ^{-1} y_J is the quadratic form of the
// Schur complement Sigma^lk - Sigma^cor of Alg. 5 (y_B - mu^new, weighted),
// and the trailing log-determinant is its log-determinant.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "block_common.cuh"
#include "dfloat.cuh"
#include "sbv_internal.cuh"

namespace sbv {

constexpr int MX_THREADS = 512;
constexpr int MX_WARPS = MX_THREADS / 32;
constexpr int NB = 16;  // diagonal tile size

struct MixedLayout {
  int ncap;    // largest N held (rows 0..ncap-1 plus the bordered row)
  int ntile;   // tiles of NB columns
  int d;
  size_t off_A, off_D, off_uh, off_ul, off_y, off_v, bytes;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline MixedLayout mixed_layout(int ncap, int d) {
  MixedLayout L;
  L.ncap = ncap;
  L.ntile = (ncap + NB - 1) / NB;
  L.d = d;
  size_t o = 0;
  L.off_D = o;  o += (size_t)L.ntile * NB * NB * sizeof(double);
  L.off_y = o;  o += (size_t)(ncap + 1) * sizeof(double);
  L.off_v = o;  o += (size_t)8 * (ncap + 1) * sizeof(float);   // x0, x0J, r, rJ, c, cJ (+2 spare)
  L.off_uh = o; o += align_up((size_t)d * ncap * sizeof(float), 16);
  L.off_ul = o; o += align_up((size_t)d * ncap * sizeof(float), 16);
  L.off_A = o;  o += align_up((size_t)(ncap + 1) * (ncap + 2) / 2 * sizeof(float), 16);
  L.bytes = o;
  return L;
}

// ---------------------------------------------------------------------------
// blocked FP32 triangular solves with the factor stored packed in A (tiles
// on the diagonal hold the FP32 copy of the FP64 tile factor); two RHS.
// ---------------------------------------------------------------------------
// forward: L v = b for both columns (b overwritten by v)
__device__ void fwd_solve2(const float* A, int N, float* b1, float* b2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k0 = 0; k0 < N; k0 += NB) {
    const int k1 = min(k0 + NB, N);
    if (warp == 0) {
      // half-warp h solves column h; lane r = row k0 + r
      const int h = lane >> 4, r = lane & 15;
      float* b = h ? b2 : b1;
      const int row = k0 + r;
      float v = row < k1 ? b[row] : 0.0f;
      for (int c = 0; c < k1 - k0; ++c) {
        float piv = A[tri(k0 + c, k0 + c)];
        float vc = __shfl_sync(0xffffffffu, v, (h << 4) + c) / piv;
        if (r == c) v = vc;
        if (r > c && row < k1) v -= A[tri(row, k0 + c)] * vc;
      }
      if (row < k1) b[row] = v;
    }
    __syncthreads();
    // b_i -= sum_{k in tile} L_ik v_k for i >= k1
    for (int i = k1 + threadIdx.x; i < N; i += blockDim.x) {
      float s1 = 0.0f, s2 = 0.0f;
      const float* Ai = A + tri(i, 0);
      for (int k = k0; k < k1; ++k) {
        s1 = fmaf(Ai[k], b1[k], s1);
        s2 = fmaf(Ai[k], b2[k], s2);
      }
      b1[i] -= s1;
      b2[i] -= s2;
    }
    __syncthreads();
  }
}

// backward: L^T v = b for both columns
__device__ void bwd_solve2(const float* A, int N, float* b1, float* b2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntile = (N + NB - 1) / NB;
  for (int kt = ntile - 1; kt >= 0; --kt) {
    const int k0 = kt * NB, k1 = min(k0 + NB, N);
    if (warp == 0) {
      const int h = lane >> 4, r = lane & 15;
      float* b = h ? b2 : b1;
      const int row = k0 + r;
      float v = row < k1 ? b[row] : 0.0f;
      for (int c = k1 - k0 - 1; c >= 0; --c) {
        float piv = A[tri(k0 + c, k0 + c)];
        float vc = __shfl_sync(0xffffffffu, v, (h << 4) + c) / piv;
        if (r == c) v = vc;
        // (L^T)_{row, k0+c} = L_{k0+c, row} for row < k0 + c
        if (r < c) v -= A[tri(k0 + c, row)] * vc;
      }
      if (row < k1) b[row] = v;
    }
    __syncthreads();
    // b_i -= sum_{k in tile} L_ki v_k for i < k0
    for (int i = threadIdx.x; i < k0; i += blockDim.x) {
      float s1 = 0.0f, s2 = 0.0f;
      for (int k = k0; k < k1; ++k) {
        float Lki = A[tri(k, i)];
        s1 = fmaf(Lki, b1[k], s1);
        s2 = fmaf(Lki, b2[k], s2);
      }
      b1[i] -= s1;
      b2[i] -= s2;
    }
    __syncthreads();
  }
}

__device__ double cta_sum_mx(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < MX_WARPS; ++q) s += red[q];
  __syncthreads();
  return s;  // same value on every thread
}

__global__ void __launch_bounds__(MX_THREADS)
loglik_mixed_kernel(LoglikArgs a, MixedLayout lay, float2* __restrict__ scratch,
                    size_t scratch_stride) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* Dt = (double*)(smem + lay.off_D);
  double* yv = (double*)(smem + lay.off_y);
  float* vec = (float*)(smem + lay.off_v);
  float* uh = (float*)(smem + lay.off_uh);
  float* ul = (float*)(smem + lay.off_ul);
  float* A = (float*)(smem + lay.off_A);
  __shared__ unsigned int s_item;
  __shared__ int s_fail;
  __shared__ double red[MX_WARPS];
  __shared__ double s_org[SBV_MAX_DIM];
  __shared__ float s_grid;
  float2* S = scratch + (size_t)blockIdx.x * scratch_stride;
  const int d = a.d, cap = lay.ncap;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned int total = (unsigned int)(a.bc * a.B);
  const double log2pi = 1.8378770664093454836;
  float* x0 = vec;
  float* x0J = vec + (cap + 1);
  float* r1 = vec + 2 * (cap + 1);
  float* r2 = vec + 3 * (cap + 1);

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
    // ---- 1. gather: u = x / beta in FP64, centred, split on a common grid
    double* u64 = (double*)A;  // temporary, d x N doubles fit in the matrix area
    for (int e = threadIdx.x; e < N * d; e += blockDim.x) {
      int p = e / d, t = e - p * d;
      int64_t id = p < mb ? (int64_t)a.nbr[blk * a.m + p] : (int64_t)a.pts[base + (p - mb)];
      double x = a.dtype == SBV_F64 ? ld_x<double>(a.X, id * d + t) : ld_x<float>(a.X, id * d + t);
      u64[t * N + p] = x * th.inv_beta[t];
    }
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      int64_t id = p < mb ? (int64_t)a.nbr[blk * a.m + p] : (int64_t)a.pts[base + (p - mb)];
      yv[p] = a.y[id];
    }
    if (threadIdx.x == 0) s_fail = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < d; t += blockDim.x) s_org[t] = u64[t * N];
    __syncthreads();
    float mx = 0.0f;
    for (int e = threadIdx.x; e < N * d; e += blockDim.x) {
      int t = e / N;
      mx = fmaxf(mx, (float)fabs(u64[e] - s_org[t]));
    }
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = (double)mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      double M = 0.0;
      for (int q = 0; q < MX_WARPS; ++q) M = fmax(M, red[q]);
      int ex;
      frexp(M * 1.0000001 + 1e-30, &ex);  // M < 2^ex
      s_grid = ldexpf(1.0f, ex - 22);     // |hi| / grid < 2^22: hi and hi_a - hi_b exact in FP32
    }
    __syncthreads();
    {
      const double g = (double)s_grid, ig = 1.0 / g;
      for (int e = threadIdx.x; e < N * d; e += blockDim.x) {
        int t = e / N;
        double v = u64[e] - s_org[t];
        double hi = rint(v * ig) * g;
        uh[e] = (float)hi;
        ul[e] = (float)(v - hi);
      }
    }
    __syncthreads();
    // ---- 2. double-float covariance: A (float head), Dt (FP64 diagonal tiles), S (scratch)
    {
      const df s2 = df_from_double(th.sigma2);
      const double diag = th.sigma2 + th.tau2;
      const int npair = N * (N + 1) / 2;
      int i = 0, j = threadIdx.x;
      while (j > i) { j -= i + 1; ++i; }
      for (int l = threadIdx.x; l < npair; l += blockDim.x) {
        df K;
        if (i == j) {
          K = df_from_double(diag);
        } else {
          float sh = 0.0f, sl = 0.0f;
          for (int t = 0; t < d; ++t) {
            float dh = __fsub_rn(uh[t * N + i], uh[t * N + j]);  // exact
            float dl = __fsub_rn(ul[t * N + i], ul[t * N + j]);
            float p = __fmul_rn(dh, dh);
            float pe = __fmaf_rn(dh, dh, -p);
            pe = __fmaf_rn(2.0f * dh, dl, pe);
            pe = __fmaf_rn(dl, dl, pe);
            df q = two_sum(sh, p);
            sh = q.h;
            sl = __fadd_rn(sl, __fadd_rn(q.l, pe));
          }
          df s = fast_two_sum(sh, sl);
          df r = df_sqrt(s);
          K = df_mul(s2, df_matern(r, s, a.nu2));
        }
        const int ti = i / NB, tj = j / NB;
        if (ti == tj) {
          Dt[(size_t)ti * NB * NB + (i % NB) * NB + (j % NB)] = df_to_double(K);
          A[tri(i, j)] = 0.0f;
        } else {
          A[tri(i, j)] = K.h;
        }
        S[(size_t)j * N + i] = make_float2(K.h, K.l);
        S[(size_t)i * N + j] = make_float2(K.h, K.l);
        j += blockDim.x;
        while (j > i) { j -= i + 1; ++i; }
      }
      for (int p = threadIdx.x; p < N; p += blockDim.x) A[tri(N, p)] = (float)yv[p];
    }
    __syncthreads();
    // ---- 3. blocked Cholesky
    for (int k0 = 0; k0 < N; k0 += NB) {
      const int k1 = min(k0 + NB, N), nbk = k1 - k0;
      double* D = Dt + (size_t)(k0 / NB) * NB * NB;
      if (warp == 0) {
        // D += (double) A_tile  (A_tile holds minus the FP32-accumulated updates)
        for (int e = lane; e < nbk * nbk; e += 32) {
          int r = e / nbk, c = e % nbk;
          if (c <= r) D[r * NB + c] += (double)A[tri(k0 + r, k0 + c)];
        }
        __syncwarp();
        for (int c = 0; c < nbk; ++c) {
          if (lane == 0) {
            double piv = D[c * NB + c];
            if (!(piv > 0.0) || !isfinite(piv)) s_fail = 1;
            D[c * NB + c] = sqrt(fmax(piv, 1e-300));
          }
          __syncwarp();
          const double Lc = D[c * NB + c];
          if (lane > c && lane < nbk) D[lane * NB + c] /= Lc;
          __syncwarp();
          if (lane > c && lane < nbk) {
            const double Lrc = D[lane * NB + c];
            for (int c2 = c + 1; c2 <= lane; ++c2) D[lane * NB + c2] -= Lrc * D[c2 * NB + c];
          }
          __syncwarp();
        }
        for (int e = lane; e < nbk * nbk; e += 32) {
          int r = e / nbk, c = e % nbk;
          if (c <= r) A[tri(k0 + r, k0 + c)] = (float)D[r * NB + c];
        }
      }
      __syncthreads();
      if (s_fail) break;
      // panel solve: rows k1..N, A(i, k0:k1) <- A(i, k0:k1) L_kk^{-T}
      for (int i = k1 + threadIdx.x; i <= N; i += blockDim.x) {
        float v[NB];
        float* Ai = A + tri(i, 0);
#pragma unroll
        for (int c = 0; c < NB; ++c) v[c] = c < nbk ? Ai[k0 + c] : 0.0f;
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if (c < nbk) {
            const float* Lc = A + tri(k0 + c, k0);
            float s = v[c];
#pragma unroll
            for (int c2 = 0; c2 < NB; ++c2)
              if (c2 < c) s = fmaf(-v[c2], Lc[c2], s);
            v[c] = s / Lc[c];
          }
        }
#pragma unroll
        for (int c = 0; c < NB; ++c)
          if (c < nbk) Ai[k0 + c] = v[c];
      }
      __syncthreads();
      // trailing update of rows k1..N, columns k1..min(i, N-1), 4x4 register blocks
      const int T = N + 1 - k1;  // rows k1..N
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
            int ri = min(i0 + p, N), cj = min(j0 + p, N);
            Ar[p] = A + tri(ri, 0) + k0;
            Ac[p] = A + tri(cj, 0) + k0;
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
      float w = A[tri(N, p)];
      x0[p] = w;
      x0J[p] = p < mb ? w : 0.0f;
    }
    __syncthreads();
    bwd_solve2(A, N, x0, x0J);
    // ---- 5. residuals in double-float from the scratch matrix (warp per 32 rows)
    for (int i0 = warp * 32; i0 < N; i0 += MX_WARPS * 32) {
      const int i = i0 + lane;
      float h1 = 0.0f, l1 = 0.0f, h2 = 0.0f, l2 = 0.0f;
      if (i < N) {
        for (int j = 0; j < N; ++j) {
          const float2 s = S[(size_t)j * N + i];
          const float xj = x0[j];
          float p = __fmul_rn(s.x, xj);
          float pe = __fmaf_rn(s.x, xj, -p);
          pe = __fmaf_rn(s.y, xj, pe);
          df q = two_sum(h1, p);
          h1 = q.h;
          l1 = __fadd_rn(l1, __fadd_rn(q.l, pe));
          if (i < mb && j < mb) {
            const float zj = x0J[j];
            float p2 = __fmul_rn(s.x, zj);
            float pe2 = __fmaf_rn(s.x, zj, -p2);
            pe2 = __fmaf_rn(s.y, zj, pe2);
            df q2 = two_sum(h2, p2);
            h2 = q2.h;
            l2 = __fadd_rn(l2, __fadd_rn(q2.l, pe2));
          }
        }
        const double yi = yv[i];
        r1[i] = (float)(yi - ((double)h1 + (double)l1));
        r2[i] = i < mb ? (float)(yi - ((double)h2 + (double)l2)) : 0.0f;
      }
    }
    __syncthreads();
    // corrections: (L L^T)^{-1} r and (L_JJ L_JJ^T)^{-1} r_J
    fwd_solve2(A, N, r1, r2);
    for (int p = mb + threadIdx.x; p < N; p += blockDim.x) r2[p] = 0.0f;
    __syncthreads();
    bwd_solve2(A, N, r1, r2);
    // ---- 6. log-determinant and quadratic forms in FP64
    double v = 0.0;
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      const double yp = yv[p];
      v += yp * ((double)x0[p] + (double)r1[p]);
      if (p < mb) v -= yp * ((double)x0J[p] + (double)r2[p]);
      if (p >= mb) v += 2.0 * log(Dt[(size_t)(p / NB) * NB * NB + (p % NB) * (NB + 1)]);
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
  for (int i = 0; i < 32; ++i) split(exp2(-i / 32.0), c.tab_h[i], c.tab_l[i]);
  split(0.69314718055994530942, c.ln2_h, c.ln2_l);
  split(1.44269504088896340736, c.ilog2_h, c.ilog2_l);
  split(1.0 / 3.0, c.third_h, c.third_l);
  split(2.0 / 5.0, c.fifth2_h, c.fifth2_l);
  split(1.0 / 15.0, c.fifteenth_h, c.fifteenth_l);
  double f = 1.0;
  for (int k = 0; k < 8; ++k) {
    if (k > 0) f /= k;
    split(f, c.fact_h[k], c.fact_l[k]);
  }
  SBV_CUDA_TRY(ctx, cudaMemcpyToSymbol(c_df, &c, sizeof(c)));
  if (ctx->device < 64) g_consts_ready[ctx->device] = true;
  return SBV_OK;
}

int launch_loglik_mixed(sbv_ctx* ctx, const LoglikArgs& a0, int nmax, cudaStream_t s) {
  int st = 0;
  if ((st = upload_df_consts(ctx))) return st;
  LoglikArgs a = a0;
  const int ncap = std::max(nmax, 1);
  MixedLayout lay = mixed_layout(ncap, a.d);
  // the gather stage borrows the matrix area for d x N doubles
  size_t need_u64 = (size_t)a.d * ncap * sizeof(double);
  size_t matbytes = (size_t)(ncap + 1) * (ncap + 2) / 2 * sizeof(float);
  if (need_u64 > matbytes) {
    lay.bytes += align_up(need_u64 - matbytes, 16);
  }
  if (lay.bytes + 2048 > ctx->smem_optin)
    return fail(ctx, SBV_EUNSUPPORTED,
                "mixed path: a block with N=%d (d=%d) needs %zu bytes of shared memory", nmax, a.d,
                lay.bytes);
  int per_sm = (int)std::max<size_t>(1, (228 * 1024) / (lay.bytes + 3072));
  int grid = ctx->num_sms * std::min(per_sm, 4);
  int64_t items = a.bc * (int64_t)a.B;
  if (grid > items) grid = (int)items;
  size_t stride = align_up((size_t)ncap * ncap, 64);
  float2* scratch = (float2*)ws_get(ctx, WS_MATRIX, stride * grid * sizeof(float2), &st);
  if (!scratch) return st;
  SBV_CUDA_TRY(ctx, cudaFuncSetAttribute(loglik_mixed_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)lay.bytes));
  loglik_mixed_kernel<<<grid, MX_THREADS, lay.bytes, s>>>(a, lay, scratch, stride);
  SBV_LAUNCH_CHECK(ctx, "loglik_mixed_kernel");
  return SBV_OK;
}

}  // namespace sbv
