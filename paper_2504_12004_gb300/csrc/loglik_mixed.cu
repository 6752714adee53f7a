// Mixed-precision block log-likelihood (Alg. 5 per block).
//
// Per (theta, block) item, one CTA:
//  1. gather the N = m_i + bs_i points as double-float coordinates (split
//     once per call from FP64 X), scale by 1/beta in double-float, centre on
//     the first point and re-split on a common power-of-two grid so that every
//     difference of the float heads is exact;
//  2. evaluate the joint covariance in double-float (dfloat.cuh): the float
//     head of each off-diagonal-tile entry feeds the FP32 factorisation; the
//     full double-float matrix goes to a per-CTA scratch slice (L2-resident)
//     for the diagonal tiles and the refinement residual;
//  3. blocked right-looking Cholesky (16-column panels): each diagonal tile is
//     formed as (double-float original) - (FP32-accumulated updates) with one
//     exact subtraction, rounded, and factored in FP32 registers by one warp;
//     FP32 panel solve; trailing update either FP32 on the CUDA cores
//     (SBV_PREC_MIXED) or split-BF16 on the tensor cores with TMEM
//     accumulators (SBV_PREC_MIXED_BF16); y is bordered as row N so the
//     factorisation also yields w0 = L^{-1} y;
//  4. the diagonal tiles are replaced by their inverses, which turns the
//     diagonal steps of the triangular solves into small parallel products;
//     x0 = L^-T w0 and x0_J = L_JJ^-T w0_J in FP32 (one two-column sweep);
//  5. refinement of the two quadratic forms: each step forms r = y - Sigma x
//     and r_J = y_J - Sigma_JJ x_J in double-float from the scratch matrix,
//     w = L^{-1} r with the FP32 factor, and takes q = y^T x + x^T r + |w|^2
//     (third order in the error of x) for both systems; a block stops once
//     |w|^2 is below 1e-6 per point or stops halving, otherwise the backward
//     solve corrects x for another step (at most six; prediction takes
//     three);
//  6. l_i = -1/2 [bs log 2pi + 2 sum_{t>=m} log L_tt + q - q_J],
//     log L_tt = e ln2 + log(mantissa), sums in FP64.
// y^T Sigma^{-1} y - y_J^T Sigma_JJ^{-1} y_J is the quadratic form of the
// Schur complement Sigma^lk - Sigma^cor of Alg. 5 (applied to y_B - mu^new),
// and the trailing log-determinant is its log-determinant.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cuda_bf16.h>

#include "block_common.cuh"
#include "dfloat.cuh"
#include "mixed.cuh"
#include "sbv_internal.cuh"
#include "umma.cuh"

namespace sbv {

static __constant__ DfConsts c_df;

// ---------------------------------------------------------------------------
// Triangular solves with the factor packed in A, whose diagonal tiles hold
// the inverses of the diagonal blocks.  Two right-hand sides (lanes 0-15 and
// 16-31 of warp 0 in the diagonal steps).
// ---------------------------------------------------------------------------
__device__ void fwd_solve2(const float* A, int N, float* b1, float* b2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k0 = 0; k0 < N; k0 += NB) {
    const int k1 = min(k0 + NB, N), nbk = k1 - k0;
    if (warp == 0) {
      const int r = lane & 15;
      float* b = (lane >> 4) ? b2 : b1;
      float v = 0.0f;
      if (r < nbk) {
        const float* Li = A + trp(k0 + r, k0);  // row r of the tile inverse
        for (int c = 0; c <= r; ++c) v = fmaf(Li[c], b[k0 + c], v);
      }
      __syncwarp();
      if (r < nbk) b[k0 + r] = v;
    }
    __syncthreads();
    for (int i = k1 + threadIdx.x; i < N; i += blockDim.x) {
      float s1 = 0.0f, s2 = 0.0f;
      const float* Ai = A + trp(i, 0);
      if (nbk == NB) {
#pragma unroll
        for (int k = 0; k < NB; k += 4) {
          const float4 x = *(const float4*)(Ai + k0 + k);
          const float4 p = *(const float4*)(b1 + k0 + k);
          const float4 q = *(const float4*)(b2 + k0 + k);
          s1 = fmaf(x.x, p.x, s1); s1 = fmaf(x.y, p.y, s1); s1 = fmaf(x.z, p.z, s1); s1 = fmaf(x.w, p.w, s1);
          s2 = fmaf(x.x, q.x, s2); s2 = fmaf(x.y, q.y, s2); s2 = fmaf(x.z, q.z, s2); s2 = fmaf(x.w, q.w, s2);
        }
      } else {
        for (int k = k0; k < k1; ++k) {
          const float x = Ai[k];
          s1 = fmaf(x, b1[k], s1);
          s2 = fmaf(x, b2[k], s2);
        }
      }
      b1[i] -= s1;
      b2[i] -= s2;
    }
    __syncthreads();
  }
}

__device__ void bwd_solve2(const float* A, int N, float* b1, float* b2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntile = (N + NB - 1) / NB;
  for (int kt = ntile - 1; kt >= 0; --kt) {
    const int k0 = kt * NB, k1 = min(k0 + NB, N), nbk = k1 - k0;
    if (warp == 0) {
      const int r = lane & 15;
      float* b = (lane >> 4) ? b2 : b1;
      float v = 0.0f;
      if (r < nbk)
        for (int c = r; c < nbk; ++c) v = fmaf(A[trp(k0 + c, k0 + r)], b[k0 + c], v);
      __syncwarp();
      if (r < nbk) b[k0 + r] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k0; i += blockDim.x) {
      float s1 = 0.0f, s2 = 0.0f;
      for (int k = k0; k < k1; ++k) {
        const float x = A[trp(k, i)];
        s1 = fmaf(x, b1[k], s1);
        s2 = fmaf(x, b2[k], s2);
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
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
  __syncthreads();
  return s;
}

// Two sums over the CTA at once (red holds at least two doubles per warp).
__device__ double2 cta_sum2_mx(double a, double b, double* red) {
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[2 * (threadIdx.x >> 5)] = a;
    red[2 * (threadIdx.x >> 5) + 1] = b;
  }
  __syncthreads();
  double sa = 0.0, sb = 0.0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
    sa += red[2 * q];
    sb += red[2 * q + 1];
  }
  __syncthreads();
  return make_double2(sa, sb);
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

template <int THREADS, bool TC, bool PRED, bool GA>
__global__ void __launch_bounds__(THREADS, THREADS == 256 ? 2 : 1)
loglik_mixed_kernel(MixedArgs P) {
  constexpr int MX_WARPS = THREADS / 32;
  extern __shared__ __align__(128) unsigned char smem[];
  const LoglikArgs& a = P.a;
  const MixedLayout& lay = P.lay;
  float2* yv = (float2*)(smem + lay.off_y);
  float* vec = (float*)(smem + lay.off_v);
  float* vh = (float*)(smem + lay.off_u);
  float* vl = (float*)(smem + lay.off_vl);
  float* Pt = (float*)(smem + lay.off_u);                 // FP32 panel, column-major
  unsigned char* opnd = smem + lay.off_u;                 // BF16 panel pieces
  float4* part = (float4*)(smem + lay.off_u);             // residual partial sums
  float* A = GA ? P.gA + (size_t)blockIdx.x * lay.a_floats : (float*)(smem + lay.off_A);
  float* tab_h = (float*)(smem + lay.off_tab);   // covariance phase only
  float* tab_l = tab_h + 256;
  __shared__ unsigned int s_item;
  __shared__ int s_fail;
  __shared__ double red[2 * MX_WARPS];
  __shared__ float s_org_h[SBV_MAX_DIM], s_org_l[SBV_MAX_DIM];
  __shared__ float s_grid;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ int s_timeout;
  const DfConsts& C = c_df;
  float2* S = P.scratch + (size_t)blockIdx.x * P.scratch_stride;
  const int d = a.d, cap = lay.ncap, PS = lay.pstride;
  const uint32_t opnd_piece = lay.opnd_piece;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned int total = PRED ? (unsigned int)P.nt : (unsigned int)(a.bc * a.B);
  const double log2pi = 1.8378770664093454836;
  const int vs = (cap + 4) & ~3;   // vector stride, a multiple of four floats
  float* x0 = vec;
  float* x0J = vec + vs;
  float* r1 = vec + 2 * vs;
  float* r2 = vec + 3 * vs;
  float* ldiag = vec + 4 * vs;
  float* idiag = vec + 5 * vs;
  float* c1 = (float*)(smem + lay.off_c);   // live during refinement only
  float* c2 = c1 + (cap + 1);
  // refinement steps: one for the likelihood (its quadratic forms are second
  // order in the solve error); three for prediction, whose variance
  // sigma^2 + tau^2 - Sigma_*J z cancels and is first order in the error of z
  constexpr int NREF = PRED ? 3 : 6;   // at most
  // Likelihood: y^T Sigma^-1 y = y^T x + x^T r + r^T Sigma^-1 r exactly, for
  // any x and r = y - Sigma x.  Every step forms r at the current x (double
  // float) and w = L^-1 r (forward solve with the FP32 factor), and takes
  // q = y^T x + x^T r + |w|^2 for both systems: the error is rho |w|^2, rho
  // the FP32 factor's contraction, i.e. third order in the error of x.  The
  // block stops once |w|^2 (both systems) is below REF_TOL per point of the
  // block, or stops halving (the residual's rounding floor); only otherwise
  // does the backward solve complete the correction of x for another step.
  // Well-conditioned blocks finish after one residual and one forward solve.
  constexpr double REF_TOL = 1e-6;
  __shared__ double s_qvar;   // x^T r of the full system minus that of J
  __shared__ __align__(16) float s_col[2 * NB];   // column broadcast of the tile factorisation
  float2* s_tile = (float2*)(smem + lay.off_stile);  // a diagonal tile's originals (factorisation)

  if (threadIdx.x == 0) s_timeout = 0;
  uint32_t tmem_base = 0, mma_phase = 0;
  if (TC) {
    // 256 TMEM columns: two 128 x (<= 128) FP32 accumulators
    if (warp == 0) umma::tmem_alloc(&s_tmem, 256);
    if (threadIdx.x == 0) umma::mbar_init(&mma_bar, 1);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    tmem_base = s_tmem;
  }
  __syncthreads();

  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1u);
    __syncthreads();
    const unsigned int item = s_item;
    if (item >= total) break;
    // loglik: item = (theta row, block); prediction: item = test point with
    // J = its m nearest training points and the test point as the block
    const int th_i = PRED ? 0 : (int)(item / a.bc);
    const int64_t blk = PRED ? (int64_t)item : (int64_t)(item % a.bc);
    const ThetaDev& th = a.theta[th_i];
    const int bs = PRED ? 1 : (int)(a.ptr[blk + 1] - a.ptr[blk]);
    const int mb = PRED ? a.m : a.cnt[blk];
    const int N = mb + bs;
    if (N > cap) {
      if (threadIdx.x == 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        if (PRED) {
          P.mean[item] = nan;
          P.var[item] = nan;
          P.var_latent[item] = nan;
        } else {
          a.terms[item] = nan;
          if (a.status) a.status[item] = SBV_EUNSUPPORTED;
        }
        record_failure(a.dstat, SBV_EUNSUPPORTED, (int)blk, th_i);
      }
      __syncthreads();
      continue;
    }
    const int64_t base = PRED ? 0 : a.ptr[blk];
    // ---- 1. gather and scale in double-float; centre on point 0
    if (threadIdx.x == 0) s_fail = 0;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
      tab_h[i] = C.tab_h[i];
      tab_l[i] = C.tab_l[i];
    }
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      if (PRED && p == mb) {
        yv[p] = make_float2(0.0f, 0.0f);  // the test point's observation is unknown
        continue;
      }
      int64_t id = p < mb ? (int64_t)a.nbr[blk * a.m + p] : (int64_t)a.pts[base + (p - mb)];
      const double yy = a.y[id];
      const float yh = (float)yy;
      yv[p] = make_float2(yh, (float)(yy - (double)yh));
    }
    for (int e = threadIdx.x; e < N * d; e += blockDim.x) {
      const int p = e / d, t = e - p * d;
      df x;
      if (PRED && p == mb) {
        if (a.dtype == SBV_F64) {
          const double xv = ((const double*)P.Xt)[(int64_t)item * d + t];
          x = df_from_double(xv);
        } else {
          x = {((const float*)P.Xt)[(int64_t)item * d + t], 0.0f};
        }
      } else {
        int64_t id = p < mb ? (int64_t)a.nbr[blk * a.m + p] : (int64_t)a.pts[base + (p - mb)];
        if (P.Xs) {
          const float2 xs = P.Xs[id * d + t];
          x = {xs.x, xs.y};
        } else {
          x = {((const float*)a.X)[id * d + t], 0.0f};
        }
      }
      const df u = df_mul(x, df{th.ib_h[t], th.ib_l[t]});
      vh[t * N + p] = u.h;  // uncentred for now
      vl[t * N + p] = u.l;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < d; t += blockDim.x) {
      s_org_h[t] = vh[t * N];
      s_org_l[t] = vl[t * N];
    }
    __syncthreads();
    float mx = 0.0f;
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
        // diagonal-tile entries start at 0 in A: A accumulates minus the updates
        A[trp(i, j)] = (i / NB == j / NB) ? 0.0f : K.h;
        S[(size_t)j * N + i] = make_float2(K.h, K.l);
        S[(size_t)i * N + j] = make_float2(K.h, K.l);
        j += blockDim.x;
        while (j > i) { j -= i + 1; ++i; }
      }
      for (int p = threadIdx.x; p < N; p += blockDim.x) A[trp(N, p)] = yv[p].x;
    }
    __syncthreads();
    // ---- 3. blocked Cholesky.  CUDA-core variant with look-ahead: while the
    // other warps apply panel k to the trailing matrix, warp 0 first updates
    // the next diagonal tile (the first ten 4 x 4 blocks of the trailing
    // triangle) and factors it, so the tile factorisation overlaps the
    // trailing update instead of following it.  The tensor-core variant
    // factors each tile before its panel.
    //
    // factor_tile(k0), warp 0 only, lane r holding row r of the tile: the
    // double-float original (staged in s_tile) plus the accumulated FP32
    // updates (held negated in A), one exact subtraction, then an FP32
    // factorisation in registers; L, its diagonal and inverse diagonal are
    // stored.
    // stage_tile(kt), warp 0: asynchronous copies (cp.async, 8 bytes each) of
    // tile kt's double-float originals, lower triangle, column-major 16 x 16,
    // from the scratch matrix into s_tile.  Issued one panel ahead, right
    // after the previous tile was factored, so that the scratch matrix's DRAM
    // latency is off the critical path; factor_tile waits for them.
    auto stage_tile = [&](const int kt) {
      const int nt = min(kt + NB, N) - kt;
      __syncwarp();   // the previous tile's reads of s_tile are done
#pragma unroll
      for (int e = lane; e < NB * NB; e += 32) {
        const int c = e >> 4, r = e & 15;
        if (r < nt && c <= r) {
          const uint32_t dst = (uint32_t)__cvta_generic_to_shared(s_tile + e);
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst),
                       "l"(S + (size_t)(kt + c) * N + (kt + r)) : "memory");
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto factor_tile = [&](const int kt) {
      const int nt = min(kt + NB, N) - kt;
      const int r = lane;
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncwarp();
      float row[NB];
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        // rows past the tile are padded with the identity, so that no update
        // below needs a bound
        float v = c == r ? 1.0f : 0.0f;
        if (r < nt && c <= r) {
          const float2 k = s_tile[c * NB + r];
          const df s = two_sum(k.x, A[trp(kt + r, kt + c)]);
          v = __fadd_rn(s.h, __fadd_rn(s.l, k.y));
        }
        row[c] = v;
      }
      // right-looking elimination; column c is broadcast through shared memory
      // (double-buffered, four floats per load) instead of one shuffle per entry
      bool bad = false;
      float rinv = 0.0f;   // 1 / L[r][r]
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        float* cb = s_col + (c & 1) * NB;
        if (r < NB) cb[r] = row[c];
        __syncwarp();
        const float dcc = cb[c];
        bad |= !(dcc > 0.0f);
        // one reciprocal square root gives both the pivot and its inverse
        // (a few ulp: ~1e-8 per point of the log-determinant, random)
        const float inv = rsqrtf(fmaxf(dcc, 1e-30f));
        // a[r][c2] -= L[r][c] L[c2][c] = (a[r][c] / a[c][c]) a[c2][c]
        const float t = r > c ? row[c] * (inv * inv) : 0.0f;
        row[c] = r == c ? dcc * inv : row[c] * inv;
        if (r == c) rinv = inv;
#pragma unroll
        for (int j = (c + 1) & ~3; j < NB; j += 4) {
          const float4 q = *(const float4*)(cb + j);
          const float qq[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (j + u > c) row[j + u] = fmaf(-t, qq[u], row[j + u]);
        }
      }
      if (r < nt) {
        float Lrr = 0.0f;
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if (c <= r) A[trp(kt + r, kt + c)] = row[c];
          if (c == r) Lrr = row[c];
        }
        ldiag[kt + r] = Lrr;
        idiag[kt + r] = rinv;
      }
      if (bad && lane == 0) s_fail = 1;
    };
    // invert_tile(k0), one warp, lane r = row r: the tile's L is replaced in
    // place by L^{-1}, row by row (forward substitution).  Row c is final
    // once rows 0..c-1 are applied; lane c scales and stores it (16-byte
    // aligned rows, zeros past the diagonal land in the row's padding) and
    // the rows below read it back as broadcast float4 loads.  Only the
    // triangle q <= c is touched.
    auto invert_tile = [&](const int k0) {
      const int nbk = min(NB, N - k0);
      const int r = lane;
      float Lr[NB], Xr[NB];
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        Lr[c] = (r < nbk && c <= r) ? A[trp(k0 + r, k0 + c)] : 0.0f;
        Xr[c] = (c == r) ? 1.0f : 0.0f;
      }
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        if (c < nbk) {
          float* Xc = A + trp(k0 + c, k0);
          if (r == c) {
            const float ic = idiag[k0 + c];
#pragma unroll
            for (int q = 0; q <= c; ++q) Xr[q] *= ic;
#pragma unroll
            for (int q4 = 0; q4 <= c; q4 += 4)
              *(float4*)(Xc + q4) = make_float4(Xr[q4], Xr[q4 + 1], Xr[q4 + 2], Xr[q4 + 3]);
          }
          __syncwarp();
          if (r > c) {
#pragma unroll
            for (int q4 = 0; q4 <= c; q4 += 4) {
              const float4 x = *(const float4*)(Xc + q4);
              const float x4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (q4 + u <= c) Xr[q4 + u] = fmaf(-Lr[c], x4[u], Xr[q4 + u]);
            }
          }
        }
      }
      __syncwarp();
    };
    if (!TC) {
      if (warp == 0) {
        stage_tile(0);
        factor_tile(0);
        if (NB < N) stage_tile(NB);
      }
      __syncthreads();
    }
    for (int k0 = 0; k0 < N; k0 += NB) {
      const int k1 = min(k0 + NB, N), nbk = k1 - k0;
      if (TC) {
        if (warp == 0) {
          if (k0 == 0) stage_tile(0);
          factor_tile(k0);
          if (k1 < N) stage_tile(k1);
        }
        __syncthreads();
      }
      if (s_fail) break;
      // panel solve: rows k1..N, A(i, k0:k1) <- A(i, k0:k1) L_kk^{-T}; the panel
      // is also stored as the update operand (FP32 column-major, or BF16 pieces)
      const int T = N + 1 - k1;  // trailing rows k1..N (the last one is y)
      for (int i = k1 + threadIdx.x; i <= N; i += blockDim.x) {
        float v[NB];
        float* Ai = A + trp(i, 0) + k0;   // 16-byte aligned (padded rows)
        const bool full = nbk == NB;
        if (full) {
#pragma unroll
          for (int c = 0; c < NB; c += 4) {
            const float4 q = *(const float4*)(Ai + c);
            v[c] = q.x; v[c + 1] = q.y; v[c + 2] = q.z; v[c + 3] = q.w;
          }
        } else {
#pragma unroll
          for (int c = 0; c < NB; ++c) v[c] = c < nbk ? Ai[c] : 0.0f;
        }
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if (c < nbk) {
            // row c of the tile, four entries per (broadcast) load; the
            // entries at and past the diagonal are read but not used
            const float* Lc = A + trp(k0 + c, k0);
            float s = v[c];
#pragma unroll
            for (int c4 = 0; c4 < c; c4 += 4) {
              const float4 q = *(const float4*)(Lc + c4);
              const float l4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (c4 + u < c) s = fmaf(-v[c4 + u], l4[u], s);
            }
            v[c] = s * idiag[k0 + c];
          }
        }
        const int row = i - k1;
        if (full) {
#pragma unroll
          for (int c = 0; c < NB; c += 4) *(float4*)(Ai + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
        }
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if (!full && c < nbk) Ai[c] = v[c];
          if (TC) {
            const __nv_bfloat16 bh = __float2bfloat16_rn(v[c]);
            const float rr = v[c] - __bfloat162float(bh);           // exact
            const __nv_bfloat16 bm = __float2bfloat16_rn(rr);
            const __nv_bfloat16 bl = __float2bfloat16_rn(rr - __bfloat162float(bm));
            const uint32_t o = umma::op_offset(row, c);
            *(__nv_bfloat16*)(opnd + o) = bh;
            *(__nv_bfloat16*)(opnd + opnd_piece + o) = bm;
            *(__nv_bfloat16*)(opnd + 2 * opnd_piece + o) = bl;
          } else {
            Pt[c * PS + row] = v[c];
          }
        }
      }
      if (!TC) {
        // pad rows T .. round4(T) of the panel with zeros (read by the 4-row blocks)
        for (int e = threadIdx.x; e < NB * 4; e += blockDim.x) {
          const int c = e >> 2, row = T + (e & 3);
          if (row < PS) Pt[c * PS + row] = 0.0f;
        }
      }
      if (TC) umma::fence_proxy_async();
      __syncthreads();
      const int ncols_all = T - 1;  // matrix columns k1..N-1
      if (!TC) {
        // trailing update on the CUDA cores: 4 x 4 register blocks over the
        // lower triangle, both operands read as float4 from the panel copy
        if (ncols_all > 0) {
          const int RB = (T + 3) >> 2;
          const int nblk = RB * (RB + 1) / 2;
          // blocks 0..9 (rows and columns k1 .. k1+15: the next diagonal tile)
          // go to lanes 0..9 of warp 0, the rest to warps 1..
          const int first = warp == 0 ? lane : 10 + (int)threadIdx.x - 32;
          const int stride = warp == 0 ? 1 << 30 : (int)blockDim.x - 32;
          const int lend = warp == 0 ? min(10, nblk) : nblk;
          int bi = 0, bj = first;
          while (bj > bi) { bj -= bi + 1; ++bi; }
          for (int l = first; l < lend; l += stride) {
            float acc[4][4];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
              for (int q = 0; q < 4; ++q) acc[p][q] = 0.0f;
#pragma unroll 4
            for (int k = 0; k < nbk; ++k) {
              const float4 ar = *(const float4*)(Pt + k * PS + 4 * bi);
              const float4 ac = *(const float4*)(Pt + k * PS + 4 * bj);
              const float rr[4] = {ar.x, ar.y, ar.z, ar.w};
              const float cc[4] = {ac.x, ac.y, ac.z, ac.w};
#pragma unroll
              for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(rr[p], cc[q], acc[p][q]);
            }
            // one aligned float4 read-modify-write per block row; in a
            // diagonal block the entries past the diagonal land in the row's
            // padding, which nothing reads
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              const int ii = k1 + 4 * bi + p;
              if (ii > N) continue;
              float4* a4 = (float4*)(A + trp(ii, k1 + 4 * bj));
              float4 w = *a4;
              w.x -= acc[p][0];
              w.y -= acc[p][1];
              w.z -= acc[p][2];
              w.w -= acc[p][3];
              *a4 = w;
            }
            if (l + stride >= lend) break;   // before walking (bi, bj) that far
            bj += stride;
            while (bj > bi) { bj -= bi + 1; ++bi; }
          }
        }
        if (warp == 0 && k1 < N) {
          __syncwarp();
          factor_tile(k1);
          if (k1 + NB < N) stage_tile(k1 + NB);
        }
      } else {
        // trailing update on the tensor cores: for each 128-row tile of P and
        // each chunk of <= 128 columns, BF16 MMAs accumulate in TMEM (FP32):
        // hi.hi alone in one accumulator, the five smaller cross products
        // (lo.hi, hi.lo, mid.mid, mid.hi, hi.mid, small first) in a second
        // one, so that no small product is added to a large partial sum
        // inside the tensor core; the epilogue subtracts both from A.
        for (int r0 = 0; r0 < T && ncols_all > 0; r0 += 128) {
          const int ncols = min(r0 + 128, ncols_all);
          for (int c0 = 0; c0 < ncols; c0 += 128) {
            const int nc = min(128, ((ncols - c0 + 15) / 16) * 16);
            if (threadIdx.x == 0) {
              umma::fence_after_sync();
              const uint32_t sb = umma::smem_u32(opnd);
              const uint32_t idesc = umma::idesc_bf16_f32(128, nc);
              const uint32_t arow = (uint32_t)(r0 / 8) * 256, brow = (uint32_t)(c0 / 8) * 256;
              const int pa[6] = {0, 2, 0, 1, 1, 0}, pb[6] = {0, 0, 2, 1, 0, 1};
#pragma unroll
              for (int q = 0; q < 6; ++q) {
                const uint64_t ad = umma::smem_desc(sb + pa[q] * opnd_piece + arow, 128, 256);
                const uint64_t bd = umma::smem_desc(sb + pb[q] * opnd_piece + brow, 128, 256);
                umma::mma_bf16(tmem_base + (q == 0 ? 0u : 128u), ad, bd, idesc, q > 1);
              }
              umma::mma_commit(&mma_bar);
            }
            const bool done = umma::mbar_wait(&mma_bar, mma_phase, 1u << 24);
            mma_phase ^= 1u;
            if (!done && threadIdx.x == 0) s_timeout = 1;
            umma::fence_after_sync();
            if (done) {
              // warp w reads TMEM lanes 32 (w % 4) ..; the w / 4 groups split the columns
              const int q = warp & 3, grp = warp >> 2;
              const int ii = k1 + r0 + 32 * q + lane;  // matrix row of this lane
              for (int cc = grp * 16; cc < nc; cc += 16 * (MX_WARPS / 4)) {
                float dv[16], ds[16];
                const uint32_t ta = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)cc;
                umma::tmem_ld16(ta, dv);
                umma::tmem_ld16(ta + 128u, ds);
                umma::tmem_wait_ld();
                if (ii <= N) {
#pragma unroll
                  for (int e = 0; e < 16; ++e) {
                    const int jj = k1 + c0 + cc + e;
                    if (jj <= ii && jj < N) A[trp(ii, jj)] = (A[trp(ii, jj)] - ds[e]) - dv[e];
                  }
                }
              }
            }
            umma::fence_before_sync();
            __syncthreads();
            if (s_timeout) break;
          }
          if (s_timeout) break;
        }
        if (s_timeout) {
          if (threadIdx.x == 0) s_fail = 2;
          break;
        }
      }
      __syncthreads();
    }
    // a failed or cut-short factorisation can leave a staged tile in flight
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (s_fail) {
      if (threadIdx.x == 0) {
        const int code = s_fail == 2 ? SBV_ETIMEOUT : SBV_ENOTSPD;
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        if (PRED) {
          P.mean[item] = nan;
          P.var[item] = nan;
          P.var_latent[item] = nan;
        } else {
          a.terms[item] = nan;
          if (a.status) a.status[item] = code;
        }
        record_failure(a.dstat, code, (int)blk, th_i);
      }
      __syncthreads();
      if (s_timeout) break;  // leave the item loop; TMEM is released below
      continue;
    }
    // ---- right-hand sides, read before the diagonal tiles are overwritten:
    // x0 = w0 (row N of A, w0 = L^{-1} y) and x0J = w0_J, to become L^-T w0 and
    // L_JJ^-T w0_J.  Prediction: x0 = w0_J (-> Sigma_JJ^-1 y_J) and x0J = l_*,
    // the test point's row of L, which lies in the last diagonal tile
    // (-> Sigma_JJ^-1 Sigma_J*); both vanish beyond J.
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      const float w = A[trp(N, p)];
      if (PRED) {
        x0[p] = p < mb ? w : 0.0f;
        x0J[p] = p < mb ? A[trp(mb, p)] : 0.0f;
      } else {
        x0[p] = w;
        x0J[p] = p < mb ? w : 0.0f;
      }
    }
    __syncthreads();
    // ---- 4. diagonal tiles -> their inverses (one warp per tile)
    for (int k0 = warp * NB; k0 < N; k0 += MX_WARPS * NB) invert_tile(k0);
    __syncthreads();
    bwd_solve2(A, N, x0, x0J);
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      c1[p] = 0.0f;
      c2[p] = 0.0f;
    }
    __syncthreads();
    double dq_prev = INFINITY;   // per item
#pragma unroll 1
    for (int it = 0; it < NREF; ++it) {
    // ---- 5. residuals in double-float for x = x0 + c1 and x0J + c2; all
    // warps: (32-row group, column chunk) tasks
    {
      const int G = (N + 31) / 32;
      // column chunks: the count (within the partial-sum buffer) that
      // minimises the columns the busiest warp walks
      int CH = 1;
      {
        const int chmax = max(1, min(16, lay.part_cap / max(N, 1)));
        int best = G * N;
        for (int ch = 1; ch <= chmax; ++ch) {
          const int cols = ((G * ch + MX_WARPS - 1) / MX_WARPS) * ((N + ch - 1) / ch);
          if (cols < best) {
            best = cols;
            CH = ch;
          }
        }
      }
      const int chunk = (N + CH - 1) / CH;
      for (int task = warp; task < G * CH; task += MX_WARPS) {
        const int g = task / CH, c = task % CH;
        const int i = g * 32 + lane;
        const int j0 = c * chunk, j1 = min(N, j0 + chunk);
        float h1 = 0.0f, l1 = 0.0f, h2 = 0.0f, l2 = 0.0f;
        if (i < N) {
          const bool inJ = i < mb;
          // sixteen columns of the scratch matrix in flight per lane, then
          // their products in column order
          constexpr int RB = 16;
          for (int jb = j0; jb < j1; jb += RB) {
          float2 sv[RB];
#pragma unroll
          for (int u = 0; u < RB; ++u)
            sv[u] = jb + u < j1 ? S[(size_t)(jb + u) * N + i] : make_float2(0.0f, 0.0f);
#pragma unroll
          for (int u = 0; u < RB; ++u) {
            const int j = jb + u;
            if (j >= j1) break;
            const float2 s = sv[u];
            const float xj = x0[j];
            const float p = __fmul_rn(s.x, xj);
            float pe = __fmaf_rn(s.x, xj, -p);
            pe = __fmaf_rn(s.y, xj, pe);
            pe = __fmaf_rn(s.x, c1[j], pe);
            const df q = two_sum(h1, p);
            h1 = q.h;
            l1 = __fadd_rn(l1, __fadd_rn(q.l, pe));
            if (inJ && j < mb) {
              const float zj = x0J[j];
              const float p2 = __fmul_rn(s.x, zj);
              float pe2 = __fmaf_rn(s.x, zj, -p2);
              pe2 = __fmaf_rn(s.y, zj, pe2);
              pe2 = __fmaf_rn(s.x, c2[j], pe2);
              const df q2 = two_sum(h2, p2);
              h2 = q2.h;
              l2 = __fadd_rn(l2, __fadd_rn(q2.l, pe2));
            }
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
        if (PRED) {
          // both systems are J-only: r1 = y_J - Sigma_JJ x0, r2 = Sigma_J* - Sigma_JJ x0J
          const float2 kst = S[(size_t)mb * N + i];
          r1[i] = i < mb ? df_sub_acc(y, s1).h : 0.0f;
          r2[i] = i < mb ? df_sub_acc(df{kst.x, kst.y}, s2).h : 0.0f;
        } else {
          r1[i] = df_sub_acc(y, s1).h;
          r2[i] = i < mb ? df_sub_acc(y, s2).h : 0.0f;
        }
      }
      __syncthreads();
    }
    double t1 = 0.0, t2 = 0.0;
    if (!PRED) {
      for (int p = threadIdx.x; p < N; p += blockDim.x) {
        t1 += ((double)x0[p] + (double)c1[p]) * (double)r1[p];
        if (p < mb) t2 += ((double)x0J[p] + (double)c2[p]) * (double)r2[p];
      }
      const double2 t = cta_sum2_mx(t1, t2, red);   // the same in every thread
      t1 = t.x;
      t2 = t.y;
    }
    // corrections: (L L^T)^{-1} r and (L_JJ L_JJ^T)^{-1} r_J
    fwd_solve2(A, N, r1, r2);
    for (int p = mb + threadIdx.x; p < N; p += blockDim.x) {
      r2[p] = 0.0f;
      if (PRED) r1[p] = 0.0f;
    }
    __syncthreads();
    if (!PRED) {
      double u1 = 0.0, u2 = 0.0;
      for (int p = threadIdx.x; p < N; p += blockDim.x) {
        u1 += (double)r1[p] * (double)r1[p];
        u2 += (double)r2[p] * (double)r2[p];
      }
      const double2 uu = cta_sum2_mx(u1, u2, red);
      u1 = uu.x;
      u2 = uu.y;
      if (threadIdx.x == 0) s_qvar = (t1 + u1) - (t2 + u2);
      const double u = u1 + u2;
      if (u <= REF_TOL * (double)bs || u > 0.5 * dq_prev || it == NREF - 1) break;
      dq_prev = u;
    }
    bwd_solve2(A, N, r1, r2);
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      c1[p] += r1[p];
      c2[p] += r2[p];
    }
    __syncthreads();
    }  // refinement steps
    if (PRED) {
      // mean = Sigma_*J x, var = sigma^2 + tau^2 - Sigma_*J z, sums in FP64
      double vm = 0.0, vq = 0.0;
      for (int p = threadIdx.x; p < mb; p += blockDim.x) {
        const float2 k = S[(size_t)p * N + mb];
        const double kp = (double)k.x + (double)k.y;
        vm += kp * ((double)x0[p] + (double)c1[p]);
        vq += kp * ((double)x0J[p] + (double)c2[p]);
      }
      const double sm = cta_sum_mx(vm, red);
      const double sq = cta_sum_mx(vq, red);
      if (threadIdx.x == 0) {
        const double var = th.sigma2 + th.tau2 - sq;
        P.mean[item] = sm;
        P.var[item] = var;
        P.var_latent[item] = var - th.tau2;
        if (!isfinite(sm) || !isfinite(var)) record_failure(a.dstat, SBV_ENOTSPD, (int)blk, 0);
      }
      __syncthreads();
      continue;
    }
    // ---- 6. log-determinant and quadratic forms, summed in FP64
    double v = 0.0;
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      const double yp = (double)yv[p].x + (double)yv[p].y;
      v += yp * ((double)x0[p] + (double)c1[p]);
      if (p < mb) v -= yp * ((double)x0J[p] + (double)c2[p]);
      if (p >= mb) {
        int ex;
        const float mant = frexpf(ldiag[p], &ex);  // L = mant 2^ex, mant in [0.5, 1)
        v += 2.0 * ((double)ex * 0.69314718055994530942 + (double)logf(mant));
      }
    }
    const double s = cta_sum_mx(v, red) + s_qvar;
    if (threadIdx.x == 0) {
      const double term = -0.5 * ((double)bs * log2pi + s);
      a.terms[item] = term;
      const bool ok = isfinite(term);
      if (a.status) a.status[item] = ok ? 0 : SBV_ENOTSPD;
      if (!ok) record_failure(a.dstat, SBV_ENOTSPD, (int)blk, th_i);
    }
    __syncthreads();
  }
  if (TC) {
    // after a timed-out wait, give the outstanding MMAs one more bounded wait
    // before the accumulator columns are released
    if (s_timeout) umma::mbar_wait(&mma_bar, mma_phase ^ 1u, 1u << 24);
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem_base, 256);
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

template <int THREADS, bool TC, bool PRED, bool GA>
static int occ(sbv_ctx* ctx, size_t bytes, int* out) {
  SBV_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                        out, loglik_mixed_kernel<THREADS, TC, PRED, GA>, THREADS, bytes));
  return SBV_OK;
}

template <int THREADS>
static int occ_t(sbv_ctx* ctx, bool tc, bool pred, bool ga, size_t bytes, int* out) {
  if (ga) {
    if (tc) return pred ? occ<THREADS, true, true, true>(ctx, bytes, out) : occ<THREADS, true, false, true>(ctx, bytes, out);
    return pred ? occ<THREADS, false, true, true>(ctx, bytes, out) : occ<THREADS, false, false, true>(ctx, bytes, out);
  }
  if (tc) return pred ? occ<THREADS, true, true, false>(ctx, bytes, out) : occ<THREADS, true, false, false>(ctx, bytes, out);
  return pred ? occ<THREADS, false, true, false>(ctx, bytes, out) : occ<THREADS, false, false, false>(ctx, bytes, out);
}

static int mixed_occupancy(sbv_ctx* ctx, int threads, bool tc, bool pred, bool ga, size_t bytes,
                           int* out) {
  return threads == 512 ? occ_t<512>(ctx, tc, pred, ga, bytes, out)
                        : occ_t<256>(ctx, tc, pred, ga, bytes, out);
}

// ---------------------------------------------------------------------------
// Launch planning: layout, threads per CTA, grid, scratch size.  The shape
// (threads, CTAs per SM) comes from the context's autotuning record when one
// matches (precision, prediction mode, capacity, d), else 256 threads and as
// many CTAs per SM (<= 2) as shared memory allows.
// ---------------------------------------------------------------------------
static int mixed_static_smem(sbv_ctx* ctx, size_t* out);

int mixed_plan(sbv_ctx* ctx, int nmax, int d, int precision, bool pred, int64_t items,
               MixedPlan* o) {
  const bool tc = precision == SBV_PREC_MIXED_BF16;
  const int ncap = std::max(nmax, 1);
  o->tc = tc;
  o->pred = pred;
  o->lay = mixed_layout(ncap, d, tc);
  size_t static_smem = 0;
  if (int st0 = mixed_static_smem(ctx, &static_smem)) return st0;
  if (o->lay.bytes + static_smem > ctx->smem_optin) o->lay = mixed_layout(ncap, d, tc, true);
  if (o->lay.bytes + static_smem > ctx->smem_optin)
    return fail(ctx, SBV_EUNSUPPORTED,
                "mixed path: a block with N=%d (d=%d) needs %zu bytes of shared memory", nmax, d,
                o->lay.bytes);
  int st = mixed_prepare(ctx);   // occupancy queries need the shared-memory opt-in
  if (st) return st;
  int threads = 256, per_sm = 2;
  if (ctx->force.threads) {
    threads = ctx->force.threads;
    per_sm = ctx->force.per_sm;
  } else {
    for (const auto& t : ctx->tuned)
      if (t.precision == precision && t.pred == (int)pred && t.ncap == ncap && t.d == d) {
        threads = t.threads;
        per_sm = t.per_sm;
      }
  }
  // resident CTAs per SM for this variant and shared-memory size, from the
  // runtime's occupancy calculator (registers, shared memory, reservations)
  int fit = 0;
  if ((st = mixed_occupancy(ctx, threads, tc, pred, o->lay.ga, o->lay.bytes, &fit))) return st;
  if (fit < 1)
    return fail(ctx, SBV_EUNSUPPORTED, "mixed path: no CTA of %d threads fits an SM (N=%d, d=%d)",
                threads, nmax, d);
  per_sm = std::max(1, std::min(per_sm, fit));
  int grid = ctx->num_sms * per_sm;
  if (grid > items) grid = (int)std::max<int64_t>(items, 1);
  o->threads = threads;
  o->grid = grid;
  o->scratch_stride = align_up((size_t)ncap * ncap, 64);
  return SBV_OK;
}

int mixed_split(sbv_ctx* ctx, const void* X, int dtype, int64_t total, float2* xs,
                cudaStream_t s) {
  if (dtype != SBV_F64) return SBV_OK;
  int g = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 16);
  split_points_kernel<<<std::max(g, 1), 256, 0, s>>>((const double*)X, total, xs);
  SBV_LAUNCH_CHECK(ctx, "split_points_kernel");
  return SBV_OK;
}

template <int THREADS, bool TC, bool PRED>
static int launch_variant(sbv_ctx* ctx, const MixedArgs& P, int grid, cudaStream_t s) {
  if (P.lay.ga)
    loglik_mixed_kernel<THREADS, TC, PRED, true><<<grid, THREADS, P.lay.bytes, s>>>(P);
  else
    loglik_mixed_kernel<THREADS, TC, PRED, false><<<grid, THREADS, P.lay.bytes, s>>>(P);
  SBV_LAUNCH_CHECK(ctx, "loglik_mixed_kernel");
  return SBV_OK;
}

// Both variants may use the largest dynamic shared memory; the global-A
// variant prefers the smallest shared-memory carve-out so that the rest of
// the SM's 256 KB serves as L1 for its triangles.
template <int THREADS, bool TC, bool PRED>
static int allow_smem(sbv_ctx* ctx, int bytes) {
  SBV_CUDA_TRY(ctx, cudaFuncSetAttribute(loglik_mixed_kernel<THREADS, TC, PRED, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  SBV_CUDA_TRY(ctx, cudaFuncSetAttribute(loglik_mixed_kernel<THREADS, TC, PRED, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  SBV_CUDA_TRY(ctx, cudaFuncSetAttribute(loglik_mixed_kernel<THREADS, TC, PRED, true>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout, 0));
  return SBV_OK;
}

static bool g_mixed_ready[64];
static size_t g_mixed_static[64];

template <int THREADS, bool TC, bool PRED>
static size_t static_smem_of() {
  cudaFuncAttributes a{}, b{};
  if (cudaFuncGetAttributes(&a, loglik_mixed_kernel<THREADS, TC, PRED, false>) != cudaSuccess ||
      cudaFuncGetAttributes(&b, loglik_mixed_kernel<THREADS, TC, PRED, true>) != cudaSuccess)
    return 0;
  return std::max(a.sharedSizeBytes, b.sharedSizeBytes);
}

// The largest static shared memory of the variants (the tables, the staged
// diagonal tile, the reduction buffers), queried once per device.
static int mixed_static_smem(sbv_ctx* ctx, size_t* out) {
  const int dev = ctx->device;
  if (dev < 64 && g_mixed_static[dev]) {
    *out = g_mixed_static[dev];
    return SBV_OK;
  }
  const size_t v[8] = {static_smem_of<256, false, false>(), static_smem_of<256, true, false>(),
                       static_smem_of<256, false, true>(),  static_smem_of<256, true, true>(),
                       static_smem_of<512, false, false>(), static_smem_of<512, true, false>(),
                       static_smem_of<512, false, true>(),  static_smem_of<512, true, true>()};
  size_t m = 0;
  for (size_t x : v) {
    if (x == 0) return fail(ctx, SBV_ECUDA, "mixed path: cudaFuncGetAttributes failed");
    m = std::max(m, x);
  }
  if (dev < 64) g_mixed_static[dev] = m;
  *out = m;
  return SBV_OK;
}

// Once per device: upload the double-float constants and allow every variant
// the largest dynamic shared memory, so that later launches (and launches
// captured into a CUDA graph) make no other API call.
int mixed_prepare(sbv_ctx* ctx) {
  int st = 0;
  if (ctx->device < 64 && g_mixed_ready[ctx->device]) return SBV_OK;
  if ((st = upload_df_consts(ctx))) return st;
  size_t stat = 0;
  if ((st = mixed_static_smem(ctx, &stat))) return st;
  const int b = (int)(ctx->smem_optin - stat);
  if ((st = allow_smem<256, false, false>(ctx, b)) || (st = allow_smem<256, true, false>(ctx, b)) ||
      (st = allow_smem<256, false, true>(ctx, b)) || (st = allow_smem<256, true, true>(ctx, b)) ||
      (st = allow_smem<512, false, false>(ctx, b)) || (st = allow_smem<512, true, false>(ctx, b)) ||
      (st = allow_smem<512, false, true>(ctx, b)) || (st = allow_smem<512, true, true>(ctx, b)))
    return st;
  if (ctx->device < 64) g_mixed_ready[ctx->device] = true;
  return SBV_OK;
}

// Enqueue the kernel; P carries the arguments, Xs (or NULL) and the scratch.
int mixed_enqueue(sbv_ctx* ctx, MixedArgs& P, const MixedPlan& o, cudaStream_t s) {
  int st = 0;
  if ((st = mixed_prepare(ctx))) return st;
  P.lay = o.lay;
  P.scratch_stride = o.scratch_stride;
  const bool tc = o.tc, pred = o.pred;
  if (o.threads == 512) {
    if (pred) return tc ? launch_variant<512, true, true>(ctx, P, o.grid, s)
                        : launch_variant<512, false, true>(ctx, P, o.grid, s);
    return tc ? launch_variant<512, true, false>(ctx, P, o.grid, s)
              : launch_variant<512, false, false>(ctx, P, o.grid, s);
  }
  if (pred) return tc ? launch_variant<256, true, true>(ctx, P, o.grid, s)
                      : launch_variant<256, false, true>(ctx, P, o.grid, s);
  return tc ? launch_variant<256, true, false>(ctx, P, o.grid, s)
            : launch_variant<256, false, false>(ctx, P, o.grid, s);
}

// Plan, split the points and take the scratch from the context workspace.
static int launch_mixed(sbv_ctx* ctx, MixedArgs& P, int nmax, int precision, bool pred,
                        int64_t items, cudaStream_t s) {
  int st = 0;
  MixedPlan o;
  if ((st = mixed_plan(ctx, nmax, P.a.d, precision, pred, items, &o))) return st;
  const int64_t total = P.a.n * P.a.d;
  P.Xs = nullptr;
  if (P.a.dtype == SBV_F64) {
    float2* xs = (float2*)ws_get(ctx, WS_XSPLIT, (size_t)total * sizeof(float2), &st);
    if (!xs) return st;
    if ((st = mixed_split(ctx, P.a.X, P.a.dtype, total, xs, s))) return st;
    P.Xs = xs;
  }
  unsigned char* buf = (unsigned char*)ws_get(ctx, WS_MATRIX, o.scratch_bytes(), &st);
  if (!buf) return st;
  P.scratch = (float2*)buf;
  P.gA = o.lay.ga ? (float*)(buf + o.ga_offset()) : nullptr;
  return mixed_enqueue(ctx, P, o, s);
}

int launch_loglik_mixed(sbv_ctx* ctx, const LoglikArgs& a0, int nmax, int precision,
                        cudaStream_t s) {
  MixedArgs P;
  memset(&P, 0, sizeof(P));
  P.a = a0;
  return launch_mixed(ctx, P, nmax, precision, false, a0.bc * (int64_t)a0.B, s);
}

// Prediction: a0 carries X, y, d, nbr (ntest x m), m, theta, nu2, dstat, counter.
int launch_predict_mixed(sbv_ctx* ctx, const LoglikArgs& a0, const void* Xt, int64_t nt,
                         double* mean, double* var, double* var_latent, int precision,
                         cudaStream_t s) {
  MixedArgs P;
  memset(&P, 0, sizeof(P));
  P.a = a0;
  P.Xt = Xt;
  P.nt = nt;
  P.mean = mean;
  P.var = var;
  P.var_latent = var_latent;
  return launch_mixed(ctx, P, a0.m + 1, precision, true, nt, s);
}

}  // namespace sbv
