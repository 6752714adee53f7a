// Mixed-precision block log-likelihood and prediction: Alg. 5 per block with
// an FP32 factor of the neighbour covariance and a third-order corrected
// Schur complement.
//
// Per (theta, block) item, one CTA.  J = the block's mb neighbours, B = its
// bs points, B' = B plus the observations as a bordered right-hand side.
//  1. gather the N = mb + bs points as double-float coordinates (split once
//     per call from FP64 X), scale by 1/beta in double-float, centre on the
//     first point and re-split on a common power-of-two grid so that every
//     difference of the float heads is exact;
//  2. evaluate the joint covariance in double-float (dfloat.cuh): the full
//     matrix goes to a per-CTA global slice, the float heads of Sigma_JJ to
//     the packed triangle A and those of Sigma_{J,B'} = [Sigma_JB, y_J] to
//     the right-hand-side block X (one row per member of B');
//  3. POTRF of Sigma_JJ in FP32 (the first POTRF of Alg. 5), blocked right-looking with
//     16-column panels; each diagonal tile is formed as (double-float
//     original) - (FP32 updates) and factored by one warp, looked ahead
//     during the trailing update; the rows of X ride along as extra rows, so
//     they leave as L^{-1} Sigma_{J,B'} (the TRSM and TRSV of Alg. 5);
//  4. the diagonal tiles are replaced by their inverses;
//  5. backward substitution: X <- Sigma~_JJ^{-1} Sigma_{J,B'} (FP32), i.e.
//     the kriging weights of B and x_J = Sigma~^{-1} y_J;
//  6. residual R = Sigma_{J,B'} - Sigma_JJ X from the global copy of Sigma,
//     exact to about 2^-38 of the products: in SBV_PREC_MIXED_BF16 with
//     mb <= 128 on the tensor cores (X held on a 24-bit fixed-point grid per
//     column and split into three BF16 digits, Sigma_JJ into five, the digit
//     products of equal weight summed exactly in five FP32 TMEM
//     accumulators, all right-hand sides of a pass in one MMA), otherwise on
//     the CUDA cores with exact fixed-point product heads;
//  7. the conditional system of Alg. 5 (its GEMM, GEMV and Schur
//     subtraction) by the exact identity
//        S' = Sigma_{B'B'} - Sigma_{B'J} X - X^T R - R^T Sigma_JJ^{-1} R,
//     whose last term, taken with the FP32 factor as (L^{-1} R)^T (L^{-1} R),
//     is the only approximation: the error is third order in the error of
//     X.  S' holds Sigma^new (bs x bs) and, in its bordered row, y_B - mu^new;
//  8. LDL^T of Sigma^new in double-float (one column per step), bordered
//     by y_B - mu^new (the second POTRF and the TRSV of Alg. 5); the log-
//     determinant and the quadratic form are summed in FP64:
//        l_i = -1/2 [bs log 2pi + sum_t log d_t + sum_t z_t^2 / d_t].
// Prediction is the same pipeline with B = {test point} and no y_B: the
// mean is mu^new and the variance Sigma^new (Sec. 5.5).
// An item whose FP32 or double-float pivot is not positive, or whose
// conditional system does not fit the X region, is appended to a list that
// the FP64 kernel processes right after this one (same stream).
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
  constexpr int NW = THREADS / 32;
  extern __shared__ __align__(128) unsigned char smem[];
  const LoglikArgs& a = P.a;
  const MixedLayout& lay = P.lay;
  float2* yv = (float2*)(smem + lay.off_y);
  float* idiag = (float*)(smem + lay.off_v);
  float* vh = (float*)(smem + lay.off_u);       // covariance phase
  float* vl = (float*)(smem + lay.off_vl);
  float* tab_h = (float*)(smem + lay.off_tab);
  float* tab_l = tab_h + 256;
  float* Pt = (float*)(smem + lay.off_u);       // factorisation phase
  float2* s_tile = (float2*)(smem + lay.off_stile);
  float* G = P.gbase + (size_t)blockIdx.x * lay.g_stride;
  float2* S = (float2*)G;                       // double-float Sigma, N x N, column-major
  float* Rg = G + lay.g_R;                      // residual block, then L^{-1} R
  float2* Spg = (float2*)(G + lay.g_Sp);        // partial conditional system
  float* A = GA ? G + lay.g_A : (float*)(smem + lay.off_A);
  float* Xr = GA ? G + lay.g_X : (float*)(smem + lay.off_X);
  __shared__ unsigned int s_item;
  __shared__ int s_fail;
  __shared__ double red[2 * NW];
  __shared__ float s_org_h[SBV_MAX_DIM], s_org_l[SBV_MAX_DIM];
  __shared__ float s_grid;
  __shared__ __align__(16) float s_col[2 * NB];   // column broadcast of the tile factorisation
  const DfConsts& C = c_df;
  // tensor-core residual: right-hand sides per MMA pass and TMEM columns
  // (five accumulator groups of MX_NP columns; two CTAs of 256 threads or one
  // of 512 share an SM's 512 columns)
  constexpr int MX_NP = THREADS >= 512 ? 96 : 48;
  constexpr uint32_t MX_TMEM_COLS = THREADS >= 512 ? 512u : 256u;
  const int d = a.d, cap = lay.ncap, PS = lay.pstride;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned int total = PRED ? (unsigned int)P.nt : (unsigned int)(a.bc * a.B);
  const double log2pi = 1.8378770664093454836;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  // tensor-core residual: 5 accumulator groups x 16 columns of TMEM and one
  // mbarrier for MMA completion
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ int s_timeout;
  if (TC && warp == 0) umma::tmem_alloc(&s_tmem, MX_TMEM_COLS);
  if (tid == 0) {
    if (TC) umma::mbar_init(&mma_bar, 1);
    s_timeout = 0;
  }
  if (TC) umma::fence_before_sync();
  __syncthreads();
  if (TC) umma::fence_after_sync();
  const uint32_t tmem_base = TC ? s_tmem : 0u;
  uint32_t mma_phase = 0;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(a.counter, 1u);
    __syncthreads();
    const unsigned int item = s_item;
    if (item >= total) break;
    // loglik: item = (theta row, block); prediction: item = test point with
    // J = its m nearest training points and the test point as the block
    const int th_i = PRED ? 0 : (int)(item / a.bc);
    const int64_t blk = PRED ? (int64_t)item : (int64_t)(item % a.bc);
    const ThetaDev& th = a.theta[th_i];
    // prediction: the test points of the item are tpts[tb .. tb + bs)
    const int64_t tb = PRED ? (P.tptr ? P.tptr[blk] : (int64_t)item) : 0;
    const int bs = PRED ? (P.tptr ? (int)(P.tptr[blk + 1] - tb) : 1)
                        : (int)(a.ptr[blk + 1] - a.ptr[blk]);
    auto test_point = [&](int q) -> int64_t {
      return P.tptr ? (int64_t)P.tpts[tb + q] : (int64_t)item;
    };
    const int mb = PRED ? a.m : a.cnt[blk];
    const int N = mb + bs;
    const int nr = bs + 1;               // rows of the right-hand-side block: B, then y
    const int xs = rhs_stride(mb);
    const int mb4 = (mb + 3) & ~3;
    if (N > cap || mb > lay.mcap) {
      if (tid == 0) {
        if (PRED) {
          for (int q = 0; q < bs; ++q) {
            const int64_t pt = test_point(q);
            P.mean[pt] = nan;
            P.var[pt] = nan;
            P.var_latent[pt] = nan;
          }
        } else {
          a.terms[item] = nan;
          if (a.status) a.status[item] = SBV_EUNSUPPORTED;
        }
        record_failure(a.dstat, SBV_EUNSUPPORTED, (int)blk, th_i);
      }
      __syncthreads();
      continue;
    }
    // hand the item to the FP64 kernel (capacity, or a pivot that is not positive)
    auto hand_over = [&]() {
      if (tid == 0) {
        const unsigned int k = atomicAdd(P.fb_count, 1u);
        P.fb_list[k] = item;
        atomicAdd(&a.dstat->reruns, 1);
      }
      __syncthreads();
    };
    if ((size_t)nr * (nr + 1) > lay.x_floats) {
      hand_over();
      continue;
    }
    const int64_t base = PRED ? 0 : a.ptr[blk];
    // row i (0 <= i <= N) of the factorisation: J rows in A, B' rows in X
    auto rowp = [&](int i) -> float* {
      return i < mb ? A + trp(i, 0) : Xr + (size_t)(i - mb) * xs;
    };

    // ---- 1. gather and scale in double-float; centre on point 0
    if (tid == 0) s_fail = 0;
    for (int i = tid; i < 256; i += THREADS) {
      tab_h[i] = C.tab_h[i];
      tab_l[i] = C.tab_l[i];
    }
    for (int p = tid; p < N; p += THREADS) {
      if (PRED && p >= mb) {
        yv[p] = make_float2(0.0f, 0.0f);  // the test points' observations are unknown
        continue;
      }
      const int64_t id = p < mb ? (int64_t)a.nbr[blk * a.m + p] : (int64_t)a.pts[base + (p - mb)];
      const double yy = a.y[id];
      const float yh = (float)yy;
      yv[p] = make_float2(yh, (float)(yy - (double)yh));
    }
    for (int e = tid; e < N * d; e += THREADS) {
      const int p = e / d, t = e - p * d;
      df x;
      if (PRED && p >= mb) {
        const int64_t q = test_point(p - mb);
        if (a.dtype == SBV_F64) {
          x = df_from_double(((const double*)P.Xt)[q * d + t]);
        } else {
          x = {((const float*)P.Xt)[q * d + t], 0.0f};
        }
      } else {
        const int64_t id = p < mb ? (int64_t)a.nbr[blk * a.m + p] : (int64_t)a.pts[base + (p - mb)];
        if (P.Xs) {
          const float2 q = P.Xs[id * d + t];
          x = {q.x, q.y};
        } else {
          x = {((const float*)a.X)[id * d + t], 0.0f};
        }
      }
      const df u = df_mul(x, df{th.ib_h[t], th.ib_l[t]});
      vh[t * N + p] = u.h;  // uncentred for now
      vl[t * N + p] = u.l;
    }
    __syncthreads();
    for (int t = tid; t < d; t += THREADS) {
      s_org_h[t] = vh[t * N];
      s_org_l[t] = vl[t * N];
    }
    __syncthreads();
    float mx = 0.0f;
    for (int e = tid; e < N * d; e += THREADS) {
      const int t = e / N;
      const df v = df_sub_acc(df{vh[e], vl[e]}, df{s_org_h[t], s_org_l[t]});
      vh[e] = v.h;
      vl[e] = v.l;
      mx = fmaxf(mx, fabsf(v.h));
    }
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = (double)mx;
    __syncthreads();
    if (tid == 0) {
      float M = 0.0f;
      for (int q = 0; q < NW; ++q) M = fmaxf(M, (float)red[q]);
      int ex;
      frexpf(M * 1.0001f + 1e-30f, &ex);  // M < 2^ex
      s_grid = ldexpf(1.0f, ex - 22);      // |head| / grid < 2^22: heads and their differences exact
    }
    __syncthreads();
    {
      const float g = s_grid, ig = 1.0f / g;  // powers of two: exact scaling
      for (int e = tid; e < N * d; e += THREADS) {
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
      int i = 0, j = tid;
      while (j > i) { j -= i + 1; ++i; }
      for (int l = tid; l < npair; l += THREADS) {
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
        if (j < mb) {
          // the J columns: diagonal-tile entries of Sigma_JJ start at 0 in A
          // (A accumulates minus the updates); B' rows carry the float head
          if (i < mb)
            A[trp(i, j)] = (i / NB == j / NB) ? 0.0f : K.h;
          else
            Xr[(size_t)(i - mb) * xs + j] = K.h;
        }
        S[(size_t)j * N + i] = make_float2(K.h, K.l);
        S[(size_t)i * N + j] = make_float2(K.h, K.l);
        j += THREADS;
        while (j > i) { j -= i + 1; ++i; }
      }
      for (int p = tid; p < mb; p += THREADS) Xr[(size_t)bs * xs + p] = yv[p].x;
    }
    __syncthreads();
    // ---- 3. FP32 POTRF of Sigma_JJ; the B' rows ride along as extra rows.
    // While the other warps apply panel k to the trailing matrix, warp 0
    // first updates the next diagonal tile and factors it (look-ahead).
    //
    // factor_tile(kt), warp 0 only, lane r holding row r of the tile: the
    // double-float original (staged in s_tile) plus the accumulated FP32
    // updates (held negated in A), one exact subtraction, then an FP32
    // factorisation in registers; L and its inverse diagonal are stored.
    // stage_tile(kt), warp 0: asynchronous copies (cp.async, 8 bytes each) of
    // tile kt's double-float originals from the global copy of Sigma, one
    // panel ahead, so that their latency is off the critical path.
    auto stage_tile = [&](const int kt) {
      const int nt = min(kt + NB, mb) - kt;
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
      const int nt = min(kt + NB, mb) - kt;
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
      bool bad = false;
      float rinv = 0.0f;   // 1 / L[r][r]
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        float* cb = s_col + (c & 1) * NB;
        if (r < NB) cb[r] = row[c];
        __syncwarp();
        const float dcc = cb[c];
        bad |= !(dcc > 0.0f);
        const float inv = rsqrtf(fmaxf(dcc, 1e-30f));
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
#pragma unroll
        for (int c = 0; c < NB; ++c)
          if (c <= r) A[trp(kt + r, kt + c)] = row[c];
        idiag[kt + r] = rinv;
      }
      if (bad && lane == 0) s_fail = 1;
    };
    // invert_tile(k0), one warp, lane r = row r: the tile's L is replaced in
    // place by L^{-1}, row by row; only the triangle q <= c is touched (the
    // zeros past the diagonal land in the row's padding).
    auto invert_tile = [&](const int k0) {
      const int nbk = min(NB, mb - k0);
      const int r = lane;
      float Lr[NB], Xv[NB];
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        Lr[c] = (r < nbk && c <= r) ? A[trp(k0 + r, k0 + c)] : 0.0f;
        Xv[c] = (c == r) ? 1.0f : 0.0f;
      }
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        if (c < nbk) {
          float* Xc = A + trp(k0 + c, k0);
          if (r == c) {
            const float ic = idiag[k0 + c];
#pragma unroll
            for (int q = 0; q <= c; ++q) Xv[q] *= ic;
#pragma unroll
            for (int q4 = 0; q4 <= c; q4 += 4)
              *(float4*)(Xc + q4) = make_float4(Xv[q4], Xv[q4 + 1], Xv[q4 + 2], Xv[q4 + 3]);
          }
          __syncwarp();
          if (r > c) {
#pragma unroll
            for (int q4 = 0; q4 <= c; q4 += 4) {
              const float4 x = *(const float4*)(Xc + q4);
              const float x4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (q4 + u <= c) Xv[q4 + u] = fmaf(-Lr[c], x4[u], Xv[q4 + u]);
            }
          }
        }
      }
      __syncwarp();
    };
    if (mb > 0) {
      if (warp == 0) {
        stage_tile(0);
        factor_tile(0);
        if (NB < mb) stage_tile(NB);
      }
      __syncthreads();
    }
    for (int k0 = 0; k0 < mb; k0 += NB) {
      const int k1 = min(k0 + NB, mb), nbk = k1 - k0;
      if (s_fail) break;
      // panel solve: rows k1..N, A(i, k0:k1) <- A(i, k0:k1) L_kk^{-T}; the
      // panel is also stored column-major (Pt) as the update operand
      const int T = N + 1 - k1;  // trailing rows k1..N (J rows, then B')
      for (int i = k1 + tid; i <= N; i += THREADS) {
        float v[NB];
        float* Ai = rowp(i) + k0;   // 16-byte aligned
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
          Pt[c * PS + row] = c < nbk ? v[c] : 0.0f;
        }
      }
      // pad rows T .. round4(T) of the panel with zeros (read by the 4-row blocks)
      for (int e = tid; e < NB * 4; e += THREADS) {
        const int c = e >> 2, row = T + (e & 3);
        if (row < PS) Pt[c * PS + row] = 0.0f;
      }
      __syncthreads();
      // trailing update of the J columns k1..mb-1: 4 x 4 register blocks,
      // (bi, bj <= bi) over the J rows, then every B' row block against every
      // J column block; both operands read as float4 from the panel copy
      const int CJ = (mb - k1 + 3) >> 2;     // J column blocks
      if (CJ > 0) {
        const int RB = (T + 3) >> 2;
        const int ntri = CJ * (CJ + 1) / 2;
        const int nblk = ntri + (RB - CJ) * CJ;
        const int c4n = CJ < 4 ? CJ : 4;
        const int nfirst = c4n * (c4n + 1) / 2;   // blocks of the next diagonal tile
        const int first = warp == 0 ? lane : nfirst + tid - 32;
        const int stride = warp == 0 ? 1 << 30 : THREADS - 32;
        const int lend = warp == 0 ? nfirst : nblk;
        for (int l = first; l < lend; l += stride) {
          int bi, bj;
          if (l < ntri) {
            bi = (int)((sqrtf(8.0f * (float)l + 1.0f) - 1.0f) * 0.5f);
            while (bi * (bi + 1) / 2 > l) --bi;
            while ((bi + 1) * (bi + 2) / 2 <= l) ++bi;
            bj = l - bi * (bi + 1) / 2;
          } else {
            const int q = l - ntri;
            bi = CJ + q / CJ;
            bj = q - (q / CJ) * CJ;
          }
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
          // one aligned float4 read-modify-write per block row; entries past
          // the diagonal or past column mb - 1 land in padding that nothing
          // reads as data (the B' rows' padding is cleared after the loop)
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const int ii = k1 + 4 * bi + p;
            if (ii > N) continue;
            float4* a4 = (float4*)(rowp(ii) + k1 + 4 * bj);
            float4 w = *a4;
            w.x -= acc[p][0];
            w.y -= acc[p][1];
            w.z -= acc[p][2];
            w.w -= acc[p][3];
            *a4 = w;
          }
        }
        if (warp == 0) {
          __syncwarp();
          factor_tile(k1);
          if (k1 + NB < mb) stage_tile(k1 + NB);
        }
      }
      __syncthreads();
    }
    // a failed or cut-short factorisation can leave a staged tile in flight
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (s_fail) {
      hand_over();
      continue;
    }
    // clear the padding of the B' rows (columns mb .. xs-1)
    for (int e = tid; e < nr * (xs - mb); e += THREADS) {
      const int r = e / (xs - mb);
      Xr[(size_t)r * xs + mb + (e - r * (xs - mb))] = 0.0f;
    }
    // ---- 4. diagonal tiles -> their inverses (one warp per tile)
    for (int k0 = warp * NB; k0 < mb; k0 += NW * NB) invert_tile(k0);
    __syncthreads();
    const int ntile = (mb + NB - 1) / NB;
    // ---- 5. X <- L^{-T} X (backward substitution, tile by tile)
    for (int kt = ntile - 1; kt >= 0; --kt) {
      const int k0 = kt * NB, nbk = min(NB, mb - k0);
      // diagonal step, one thread per row: x = (L_kk^{-1})^T p
      for (int r = tid; r < nr; r += THREADS) {
        float* pr = Xr + (size_t)r * xs + k0;
        float p[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) p[c] = c < nbk ? pr[c] : 0.0f;
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if (c < nbk) {
            float s = 0.0f;
#pragma unroll
            for (int c2 = c; c2 < NB; ++c2)
              if (c2 < nbk) s = fmaf(A[trp(k0 + c2, k0 + c)], p[c2], s);
            pr[c] = s;
          }
        }
      }
      __syncthreads();
      // update of the columns before the tile: p[j] -= sum_c L[k0+c][j] x[k0+c]
      const int nj4 = k0 >> 2;
      for (int t = tid; t < nr * nj4; t += THREADS) {
        const int r = t / nj4, j = (t - r * nj4) * 4;
        float* pr = Xr + (size_t)r * xs;
        float4 acc = *(const float4*)(pr + j);
#pragma unroll 4
        for (int c = 0; c < nbk; ++c) {
          const float xc = pr[k0 + c];
          const float4 l = *(const float4*)(A + trp(k0 + c, j));
          acc.x = fmaf(-l.x, xc, acc.x);
          acc.y = fmaf(-l.y, xc, acc.y);
          acc.z = fmaf(-l.z, xc, acc.z);
          acc.w = fmaf(-l.w, xc, acc.w);
        }
        *(float4*)(pr + j) = acc;
      }
      __syncthreads();
    }
    // ---- 6. the residual and the conditional system, 16 right-hand sides
    // (columns r of X) at a time.  Products with Sigma are accumulated
    // exactly on a per-column fixed-point grid: with Pmax_r = (sigma^2 +
    // tau^2) max_k |X[r][k]| (every |Sigma_ij| <= sigma^2 + tau^2) and g_r =
    // 2^(ceil(log2(max(mb, 4) Pmax_r)) - 24), the head of each product
    // s.h x rounded to the grid (one FMA with C_r = 1.5 2^23 g_r) is exact and
    // so is its sum over k' (< 2^24 g_r); the remainder s.h x - head (an
    // FMA) plus s.l x is summed in FP32 over four terms and then folded into
    // a float pair.
    float* Rb = (float*)(smem + lay.off_u);      // residual block, then L^{-1} of it
    float* colC = (float*)(smem + lay.off_cc);   // C_r per right-hand side (CUDA-core residual)
    float* colX = colC + lay.ncap + 2;           // grid unit of X^ per right-hand side
    float* Qg = Rg;                              // L^{-1} R for every column, global
    const bool tc = TC && mb <= 128;
    // with tc, the products Sigma_BJ X^ of the conditional system also run on
    // the tensor cores (a second pass with the B rows of Sigma as A)
    const bool tcg = tc && bs <= 128 && mb > 0;   // (mb = 0: no products to take)
    // right-hand sides the tensor-core passes take: all, except a last pass
    // of at most 16 columns, which the CUDA cores take instead of a whole
    // round of digit splits
    int ntc = nr;
    if (nr > MX_NP && nr % MX_NP != 0 && nr % MX_NP <= 16) ntc = nr - nr % MX_NP;
    // X <- X^ on a 24-bit fixed-point grid per column (unit 2^(ex - 24),
    // |X| < 2^ex): every later use (residual, conditional system) sees the
    // same X^, whose digits the tensor cores take exactly
    for (int r = warp; r < nr; r += NW) {
      float mxv = 0.0f;
      for (int k = lane; k < mb; k += 32) mxv = fmaxf(mxv, fabsf(Xr[(size_t)r * xs + k]));
      for (int o = 16; o; o >>= 1) mxv = fmaxf(mxv, __shfl_xor_sync(0xffffffffu, mxv, o));
      int ex = -100;
      if (mxv > 0.0f) frexpf(mxv * 1.0001f, &ex);   // max |X_r| < 2^ex
      ex = max(ex, -100);
      const float up = ldexpf(1.0f, 24 - ex), unit = ldexpf(1.0f, ex - 24);
      for (int k = lane; k < mb; k += 32) {
        float* xp = Xr + (size_t)r * xs + k;
        *xp = rintf(*xp * up) * unit;
      }
      if (lane == 0) {
        colX[r] = unit;
        const float pm = (float)(th.sigma2 + th.tau2) * mxv * (float)max(mb, 4) * 1.0001f;
        int eg = -100;
        if (pm > 0.0f) frexpf(pm, &eg);   // pm < 2^eg
        colC[r] = 1.5f * ldexpf(1.0f, max(eg, -100) - 1);   // 1.5 * 2^23 * 2^(eg - 24)
      }
    }
    // Sigma_JJ digits: Sigma = 2^(eA - 8) (a1 + a2 2^-8 + ... + a5 2^-32),
    // |Sigma| <= sigma^2 + tau^2 < 2^eA
    int eA;
    frexpf((float)(th.sigma2 + th.tau2) * 1.0001f, &eA);
    __syncthreads();
    if (tc) {
      // ---- 6t. tensor-core residual of all right-hand sides, MX_NP columns
      // per pass: R[r][k] = Sigma_{J,B'}[k][r] - sum_k' Sigma_JJ[k][k'] X[r][k']
      // into the global slice (column r at Rg + r xs).  Every K-step of 16
      // writes the digit tiles of Sigma_JJ (128 x 16, rows past mb zero) and
      // of X^ (MX_NP x 16) into shared memory in the K-major core-matrix
      // layout, then one thread issues the 12 digit products (s, t) with
      // s + t <= 6 as 128 x N x 16 BF16 MMAs into TMEM group g = s + t - 2
      // (columns g MX_NP ..).  With |a_1|, |b_1| <= 256 and the other digits
      // <= 192 (Sigma) or 128 (X^), every group's sum over K <= 128 stays
      // below 2^24 (integers): exact in FP32.
      unsigned char* Ab = smem + lay.off_sch;      // five BF16 digit tiles of Sigma_JJ
      unsigned char* Bb = Ab + 5 * 4096;           // three BF16 digit tiles of X^
      constexpr uint32_t BT = MX_NP * 32;          // bytes of one X^ digit tile
      const int nks = (mb + 15) >> 4;
      const int am = tid >> 1, ak = (tid & 1) * 8;   // A digits: row am, k ak..ak+7
      const float sc8 = ldexpf(1.0f, 8 - eA);
      float2 sv[8];
      // target 0: A = Sigma_JJ (rows 0 .. mb-1 of Sigma), result R into Rg;
      // target 1: A = Sigma_BJ (rows mb .. mb+bs-1), result G = Sigma_BJ X^,
      // written as the partial conditional system Sigma_BB - G (lower triangle)
      for (int tgt = 0; tgt < (tcg ? 2 : 1); ++tgt) {
      const int ro = tgt ? mb : 0, arows = tgt ? bs : mb;
      auto load_sv = [&](int ks) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int kk = ks * 16 + ak + j;
          sv[j] = (tid < 256 && am < arows && kk < mb) ? S[(size_t)kk * N + ro + am]
                                                       : make_float2(0.0f, 0.0f);
        }
      };
      for (int pb = 0; pb < ntc; pb += MX_NP) {
        const int npc = min(MX_NP, ntc - pb);
        const int nn = (npc + 15) & ~15;   // MMA N
        load_sv(0);
        for (int ks = 0; ks < nks; ++ks) {
          if (ks > 0) {   // the previous step's MMAs have read the digit tiles
            const bool ok = umma::mbar_wait(&mma_bar, mma_phase, 1u << 24);
            mma_phase ^= 1u;
            if (!ok) s_timeout = 1;
          }
          if (tid < 256) {
            // five digits of 8 entries of Sigma_JJ, packed two BF16 per word:
            // the float head gives the first three digits exactly (|t| < 256,
            // every step an exact power-of-two scaling or subtraction); the
            // tail joins before the fourth
            uint32_t dg[5][4];
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
              float dv[2][5];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                float t = sv[j + h].x * sc8;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                  const float dq = rintf(t);
                  dv[h][q] = dq;
                  t = __fsub_rn(t, dq) * 256.0f;
                }
                t = __fmaf_rn(sv[j + h].y, sc8 * 16777216.0f, t);
                const float d4 = rintf(t);
                dv[h][3] = d4;
                dv[h][4] = rintf(__fsub_rn(t, d4) * 256.0f);
              }
#pragma unroll
              for (int q = 0; q < 5; ++q) {
                const __nv_bfloat162 p2 = __floats2bfloat162_rn(dv[0][q], dv[1][q]);
                dg[q][j >> 1] = *(const uint32_t*)&p2;
              }
            }
            const uint32_t off = umma::op_offset(am, ak);
#pragma unroll
            for (int q = 0; q < 5; ++q)
              *(uint4*)(Ab + q * 4096 + off) = make_uint4(dg[q][0], dg[q][1], dg[q][2], dg[q][3]);
          }
          if (tid < 2 * nn) {
            // three digits of 8 entries of X^ (row n = right-hand side pb + n)
            const int n = tid >> 1, bk = (tid & 1) * 8;
            const int r = pb + n;
            uint32_t bd[3][4];
            const float iu = n < npc ? 1.0f / colX[r] : 0.0f;   // a power of two
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
              float bv[2][3];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int kk = ks * 16 + bk + j + h;
                // integer T = X^ / unit, |T| < 2^24: exact in FP32
                const float T = (n < npc && kk < mb) ? Xr[(size_t)r * xs + kk] * iu : 0.0f;
                const float b1 = rintf(T * (1.0f / 65536.0f));
                const float r1 = __fsub_rn(T, b1 * 65536.0f);
                const float b2 = rintf(r1 * (1.0f / 256.0f));
                bv[h][0] = b1;
                bv[h][1] = b2;
                bv[h][2] = __fsub_rn(r1, b2 * 256.0f);
              }
#pragma unroll
              for (int q = 0; q < 3; ++q) {
                const __nv_bfloat162 p2 = __floats2bfloat162_rn(bv[0][q], bv[1][q]);
                bd[q][j >> 1] = *(const uint32_t*)&p2;
              }
            }
            const uint32_t boff = umma::op_offset(n, bk);
#pragma unroll
            for (int q = 0; q < 3; ++q)
              *(uint4*)(Bb + q * BT + boff) = make_uint4(bd[q][0], bd[q][1], bd[q][2], bd[q][3]);
          }
          if (ks + 1 < nks) load_sv(ks + 1);
          umma::fence_proxy_async();
          umma::fence_before_sync();
          __syncthreads();
          if (tid == 0 && !s_timeout) {
            umma::fence_after_sync();
            const uint32_t ab = umma::smem_u32(Ab), bb = umma::smem_u32(Bb);
            const uint32_t idesc = umma::idesc_bf16_f32(128, nn);
            // (s, t, group) with s + t <= 6; the first product of a group at
            // the first K-step overwrites the accumulator
            const int ps[12] = {1, 1, 2, 1, 2, 3, 2, 3, 4, 3, 4, 5};
            const int pt[12] = {1, 2, 1, 3, 2, 1, 3, 2, 1, 3, 2, 1};
            const int first[12] = {1, 1, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0};
#pragma unroll
            for (int q = 0; q < 12; ++q) {
              const uint64_t ad = umma::smem_desc(ab + (ps[q] - 1) * 4096, 128, 256);
              const uint64_t bdsc = umma::smem_desc(bb + (pt[q] - 1) * BT, 128, 256);
              const uint32_t g = (uint32_t)(ps[q] + pt[q] - 2);
              umma::mma_bf16(tmem_base + g * MX_NP, ad, bdsc, idesc,
                             (ks > 0 || !first[q]) ? 1u : 0u);
            }
            umma::mma_commit(&mma_bar);
          }
        }
        // the last step's products, then the five groups are read back (TMEM
        // lane quadrant = warp mod 4, rows k = 32 (warp mod 4) + lane; the
        // warps of a quadrant share its 16-column chunks) and combined in
        // double-float: D = 2^(eA + 8) unit_r sum_g G_g 2^(-8 g)
        if (nks > 0) {
          const bool ok = umma::mbar_wait(&mma_bar, mma_phase, 1u << 24);
          mma_phase ^= 1u;
          if (!ok) s_timeout = 1;
        }
        umma::fence_after_sync();
        if (nks > 0 && !s_timeout) {
          const int qd = warp & 3, k = 32 * qd + lane;
          const uint32_t ta = tmem_base + ((uint32_t)(32 * qd) << 16);
          for (int ch = warp >> 2; ch < (nn >> 4); ch += NW / 4) {
            df acc[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) acc[c] = {0.0f, 0.0f};
#pragma unroll
            for (int g = 4; g >= 0; --g) {   // smallest weight first
              float gv[16];
              umma::tmem_ld16(ta + (uint32_t)(g * MX_NP + 16 * ch), gv);
              umma::tmem_wait_ld();
              const float wg = ldexpf(1.0f, -8 * g);
#pragma unroll
              for (int c = 0; c < 16; ++c) acc[c] = df_add_f(acc[c], gv[c] * wg);
            }
            if (tgt == 0 && k < mb) {
#pragma unroll
              for (int c = 0; c < 16; ++c) {
                const int n = 16 * ch + c, r = pb + n;
                if (n < npc) {
                  const float scl = ldexpf(colX[r], eA + 8);   // exact power of two
                  const df dd = {acc[c].h * scl, acc[c].l * scl};
                  const float2 v = r < bs ? S[(size_t)(mb + r) * N + k] : yv[k];
                  const df rv = df_sub_acc(df{v.x, v.y}, dd);
                  Rg[(size_t)r * xs + k] = __fadd_rn(rv.h, rv.l);
                }
              }
            } else if (tgt == 1 && k < bs) {
              // row a = k of B: Sp[a][r] = Sigma_BB[a][r] - G[a][r] for r <= a
#pragma unroll
              for (int c = 0; c < 16; ++c) {
                const int n = 16 * ch + c, r = pb + n;
                if (n < npc && r <= k) {
                  const float scl = ldexpf(colX[r], eA + 8);
                  const df dd = {acc[c].h * scl, acc[c].l * scl};
                  const float2 v = S[(size_t)(mb + r) * N + (mb + k)];
                  const df sv2 = df_sub_acc(df{v.x, v.y}, dd);
                  Spg[tri0(k, r)] = make_float2(sv2.h, sv2.l);
                }
              }
            }
          }
        }
        umma::fence_before_sync();
        __syncthreads();   // TMEM and the digit tiles are free for the next pass
      }
      }   // targets
    }
    // right-hand sides per column block: as many as the residual block's
    // room holds (at most 64), split evenly
    const int Wroom = min(64, (int)((lay.off_cc - lay.off_u) / ((size_t)xs * sizeof(float))));
    const int Wcap = P.wcap > 0 ? min(P.wcap, Wroom) : Wroom;
    const int nwb = (nr + Wcap - 1) / Wcap;
    const int W = (nr + nwb - 1) / nwb;
    for (int cb = 0; cb < nr; cb += W) {
      const int nc = min(W, nr - cb);
      // 6a. Rb[c][k] = Sigma_{J,B'}[k][cb+c] - sum_k' Sigma_JJ[k][k'] X[cb+c][k']
      // columns [0, ctc) of the block come from the tensor-core pass, the
      // rest from the CUDA cores
      const int ctc = tc ? max(0, min(nc, ntc - cb)) : 0;
      for (int e = tid; e < ctc * (mb4 >> 2); e += THREADS) {
        const int c = e / (mb4 >> 2), k = (e - c * (mb4 >> 2)) * 4;
        *(float4*)(Rb + (size_t)c * xs + k) = *(const float4*)(Rg + (size_t)(cb + c) * xs + k);
      }
      if (ctc < nc) {
      // CUDA cores: thread (k, c0) streams row k of Sigma_JJ itself
      // (S[kp N + k], coalesced over the warp's rows k) with the next four
      // loads in flight, and keeps eight columns' accumulators in registers;
      // no CTA barrier inside.  Columns cofs + c of the block, c < ncx.
      {
        const int cofs = ctc, ncx = nc - ctc;
        const int ngrp = (ncx + 7) >> 3;   // groups of eight columns
        for (int t0 = 0; t0 < ngrp * mb; t0 += THREADS) {
          const int tk = t0 + tid;
          // tasks whose eight columns all lie past the block do nothing
          if (tk < ngrp * mb && (tk / mb) * 8 < ncx) {
            const int k = tk % mb, c0 = (tk / mb) * 8;
            float Cq[8], ahi[8];
            df atot[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              Cq[q] = c0 + q < ncx ? colC[cb + cofs + c0 + q] : 1.0f;
              ahi[q] = 0.0f;
              atot[q] = {0.0f, 0.0f};
            }
            const float* xc = Xr + (size_t)(cb + cofs + c0) * xs;
            const float2* sk = S + k;
            float2 nx[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) nx[u] = u < mb ? sk[(size_t)u * N] : make_float2(0.0f, 0.0f);
            float alo[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) alo[q] = 0.0f;
            for (int kp = 0; kp < mb4; kp += 4) {
              float2 sv[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                sv[u] = nx[u];
                const int kn = kp + 4 + u;
                nx[u] = kn < mb ? sk[(size_t)kn * N] : make_float2(0.0f, 0.0f);
              }
              // the eight columns' chains, four products each, X^ read as
              // float4 (xs and kp are multiples of four)
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                // columns past the block read column cb + c0 (c0 < nc: in
                // bounds) and are discarded
                const float4 x4 = *(const float4*)(xc + (size_t)(c0 + q < ncx ? q : 0) * xs + kp);
                const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  const float ph = __fsub_rn(__fmaf_rn(sv[u].x, xv[u], Cq[q]), Cq[q]);
                  float rr = __fmaf_rn(sv[u].x, xv[u], -ph);
                  rr = __fmaf_rn(sv[u].y, xv[u], rr);
                  ahi[q] = __fadd_rn(ahi[q], ph);
                  alo[q] = __fadd_rn(alo[q], rr);
                }
              }
              if ((kp & 4) || kp + 4 >= mb4) {   // fold every eight products
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                  const df u2 = two_sum(atot[q].h, alo[q]);
                  atot[q].h = u2.h;
                  atot[q].l = __fadd_rn(atot[q].l, u2.l);
                  alo[q] = 0.0f;
                }
              }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int r = cb + cofs + c0 + q;
              if (c0 + q < ncx) {
                const float2 v = r < bs ? S[(size_t)(mb + r) * N + k] : yv[k];
                df rv = df_sub_acc(df{v.x, v.y}, df{ahi[q], 0.0f});
                rv = df_sub_acc(rv, atot[q]);
                Rb[(size_t)(cofs + c0 + q) * xs + k] = __fadd_rn(rv.h, rv.l);
              }
            }
          }
        }
      }
      }   // tensor or CUDA-core residual
      for (int e = tid; e < nc * (mb4 - mb); e += THREADS) {
        const int c = e / (mb4 - mb);
        Rb[(size_t)c * xs + mb + (e - c * (mb4 - mb))] = 0.0f;
      }
      __syncthreads();
      // ---- 7. partial conditional system for the block's columns r < bs, rows a >= r:
      // Sp[a][r] = Sigma_{B'B'}[a][r] - Sigma_{B'J}[a] X[r] (double-float)
      //            - X[a] . R[r] (FP32)
      // (row a = bs is the bordered y row: Sigma_{B'J}[bs] = y_J and
      // Sigma_{B'B'}[bs][r] = y_{B,r})
      // Sigma_{B'J}[a] X[r] in double-float; the row of Sigma comes from the
      // global slice (L2), so each thread keeps three quads of it in flight
      {
        const int ncb = min(nc, bs - cb);   // columns of Sigma^new in this block
        const int na = nr - cb;
        for (int t = tid; t < max(ncb, 0) * na; t += THREADS) {
          const int c = t % ncb, ar = cb + t / ncb, r = cb + c;
          if (ar < r) continue;
          // prediction needs the diagonal and the bordered row only
          if (PRED && ar != r && ar != bs) continue;
          if (tcg && ar < bs && r < ntc) {
            // Sigma_BB - Sigma_BJ X^ came from the tensor cores: subtract X^[a] . R[r]
            const float* xa = Xr + (size_t)ar * xs;
            const float* rr = Rb + (size_t)c * xs;
            float d1 = 0.0f;
            for (int k = 0; k < mb4; k += 4) {
              const float4 a4 = *(const float4*)(xa + k);
              const float4 r4 = *(const float4*)(rr + k);
              d1 = fmaf(a4.x, r4.x, d1);
              d1 = fmaf(a4.y, r4.y, d1);
              d1 = fmaf(a4.z, r4.z, d1);
              d1 = fmaf(a4.w, r4.w, d1);
            }
            const float2 sp = Spg[tri0(ar, r)];
            const df sres = df_add_f(df{sp.x, sp.y}, -d1);
            Spg[tri0(ar, r)] = make_float2(sres.h, sres.l);
            continue;
          }
          const float2 v0 = ar < bs ? S[(size_t)(mb + r) * N + (mb + ar)] : yv[mb + r];
          df e = {v0.x, v0.y};
          float d1 = 0.0f;
          const float* xa = Xr + (size_t)ar * xs;
          const float* xr = Xr + (size_t)r * xs;
          const float* rr = Rb + (size_t)c * xs;
          const float2* sa = ar < bs ? S + (size_t)(mb + ar) * N : yv;
          float2 q0[4], q1[4], q2[4];
          auto ldq = [&](float2 (&q)[4], int k) {
#pragma unroll
            for (int u = 0; u < 4; ++u) q[u] = k + u < mb ? sa[k + u] : make_float2(0.0f, 0.0f);
          };
          ldq(q0, 0);
          ldq(q1, 4);
          ldq(q2, 8);
          for (int k = 0; k < mb4; k += 4) {
            float2 sv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              sv[u] = q0[u];
              q0[u] = q1[u];
              q1[u] = q2[u];
            }
            ldq(q2, k + 12);
            const float4 x4 = *(const float4*)(xr + k);
            const float4 a4 = *(const float4*)(xa + k);
            const float4 r4 = *(const float4*)(rr + k);
            const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) df_fnma_acc(e, sv[u], xv[u]);
            d1 = fmaf(a4.x, r4.x, d1);
            d1 = fmaf(a4.y, r4.y, d1);
            d1 = fmaf(a4.z, r4.z, d1);
            d1 = fmaf(a4.w, r4.w, d1);
          }
          e = fast_two_sum(e.h, e.l);
          const df sres = df_add_f(e, -d1);
          Spg[tri0(ar, r)] = make_float2(sres.h, sres.l);
        }
      }
      // ---- 8. Rb <- L^{-1} Rb (forward substitution, tile by tile), then to global
      for (int kt = 0; kt < ntile; ++kt) {
        const int k0 = kt * NB, k1 = min(k0 + NB, mb), nbk = k1 - k0;
        __syncthreads();   // the previous step's (or pass A's) reads of Rb are done
        // diagonal tile: thread (c, rr) for columns c = tid / 16 + j THREADS / 16
        constexpr int CPS = THREADS / 16;          // columns per sweep
        constexpr int NSW = (64 + CPS - 1) / CPS;  // sweeps for the widest block
        const int rr = tid & 15;
        float xo[NSW];
#pragma unroll
        for (int j = 0; j < NSW; ++j) {
          const int c = (tid >> 4) + j * CPS;
          xo[j] = 0.0f;
          if (c < nc && rr < nbk) {
            const float* Lr = A + trp(k0 + rr, k0);
            const float* pc = Rb + (size_t)c * xs + k0;
            for (int r2 = 0; r2 <= rr; ++r2) xo[j] = fmaf(Lr[r2], pc[r2], xo[j]);
          }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NSW; ++j) {
          const int c = (tid >> 4) + j * CPS;
          if (c < nc && rr < nbk) Rb[(size_t)c * xs + k0 + rr] = xo[j];
        }
        __syncthreads();
        // trailing rows: thread (i, c), the columns fastest so that a warp
        // shares the row of L (a broadcast) and reads its columns' solved
        // tile entries; a full tile (nbk = 16) whenever rows remain below it
        const int ni = mb - k1;
        for (int t = tid; t < nc * ni; t += THREADS) {
          const int ir = t / nc, c = t - ir * nc, i = k1 + ir;
          float* pr = Rb + (size_t)c * xs;
          const float* Lr = A + trp(i, k0);
          float acc = pr[i];
#pragma unroll
          for (int q4 = 0; q4 < NB; q4 += 4) {
            const float4 l = *(const float4*)(Lr + q4);
            const float4 x = *(const float4*)(pr + k0 + q4);
            acc = fmaf(-l.x, x.x, acc);
            acc = fmaf(-l.y, x.y, acc);
            acc = fmaf(-l.z, x.z, acc);
            acc = fmaf(-l.w, x.w, acc);
          }
          pr[i] = acc;
        }
      }
      __syncthreads();
      for (int e = tid; e < nc * (mb4 >> 2); e += THREADS) {
        const int c = e / (mb4 >> 2), k = (e - c * (mb4 >> 2)) * 4;
        *(float4*)(Qg + (size_t)(cb + c) * xs + k) = *(const float4*)(Rb + (size_t)c * xs + k);
      }
      __syncthreads();
    }
    // ---- 9. conditional system S' = Sp - Q[a] . Q[b] (Q = L^{-1} R), as
    // double-float into the X region (X is no longer needed)
    float2* Sf = (float2*)Xr;
    for (int t = tid; t < nr * bs; t += THREADS) {
      const int ar = t / bs, b = t - ar * bs;
      if (b > ar) continue;
      if (PRED && ar != b && ar != bs) continue;
      float d2 = 0.0f;
      const float* qa = Qg + (size_t)ar * xs;
      const float* qb = Qg + (size_t)b * xs;
      // global (L2) reads: three quads of each row in flight
      const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      float4 a0 = *(const float4*)qa, b0 = *(const float4*)qb;
      float4 a1 = 4 < mb4 ? *(const float4*)(qa + 4) : z4, b1 = 4 < mb4 ? *(const float4*)(qb + 4) : z4;
      float4 a2 = 8 < mb4 ? *(const float4*)(qa + 8) : z4, b2 = 8 < mb4 ? *(const float4*)(qb + 8) : z4;
      for (int k = 0; k < mb4; k += 4) {
        const float4 a4 = a0, b4 = b0;
        a0 = a1;
        b0 = b1;
        a1 = a2;
        b1 = b2;
        a2 = k + 12 < mb4 ? *(const float4*)(qa + k + 12) : z4;
        b2 = k + 12 < mb4 ? *(const float4*)(qb + k + 12) : z4;
        d2 = fmaf(a4.x, b4.x, d2);
        d2 = fmaf(a4.y, b4.y, d2);
        d2 = fmaf(a4.z, b4.z, d2);
        d2 = fmaf(a4.w, b4.w, d2);
      }
      const float2 sp = Spg[tri0(ar, b)];
      const df sres = df_add_f(df{sp.x, sp.y}, -d2);
      Sf[tri0(ar, b)] = make_float2(sres.h, sres.l);
    }
    __syncthreads();
    if (PRED) {
      // per test point q: mean = mu^new_q, var = Sigma^new_qq; the bordered
      // row holds 0 - mu
      for (int q = tid; q < bs; q += THREADS) {
        const float2 v = Sf[tri0(q, q)], mu = Sf[tri0(bs, q)];
        const double var = (double)v.x + (double)v.y;
        const double mean = -((double)mu.x + (double)mu.y);
        const int64_t pt = test_point(q);
        P.mean[pt] = mean;
        P.var[pt] = var;
        P.var_latent[pt] = var - th.tau2;
        if (!isfinite(mean) || !isfinite(var)) record_failure(a.dstat, SBV_ENOTSPD, (int)blk, 0);
      }
      __syncthreads();
      continue;
    }
    // ---- 10. LDL^T of Sigma^new (bs x bs) bordered by z = y_B - mu^new, in
    // double-float, right-looking in panels of eight columns: inside a panel
    // one column per step, the CTA updating the panel's later columns
    // (S_ij -= (S_ik / d_k) S_jk, rows down to the bordered row bs); then the
    // trailing matrix takes the panel's eight columns in one pass,
    // S_ij -= sum_k S_ik W_jk with W_jk = S_jk / d_k.  Afterwards log det =
    // sum log d_k and the quadratic form = sum z_k^2 / d_k (z in the
    // bordered row).
    {
      constexpr int PW = 8;
      float2* Wp = (float2*)(smem + lay.off_u);   // W_jk of the panel, PW per row j
      __shared__ float2 s_inv[PW];
      bool bad = false;
      for (int k0 = 0; k0 < bs && !bad; k0 += PW) {
        const int k1 = min(k0 + PW, bs);
        for (int k = k0; k < k1; ++k) {
          const float2 dk2 = Sf[tri0(k, k)];
          if (!(dk2.x > 0.0f)) {   // the same value in every thread
            bad = true;
            break;
          }
          const df inv = df_recip(df{dk2.x, dk2.y});
          if (tid == 0) s_inv[k - k0] = make_float2(inv.h, inv.l);
          // panel columns j = k+1 .. k1-1, rows i = j .. bs
          const int pc = k1 - 1 - k, prow = bs - k;
          for (int e = tid; e < pc * prow; e += THREADS) {
            const int jj = e / prow, i = k + 1 + (e - jj * prow), jc = k + 1 + jj;
            if (jc > i) continue;
            const float2 a = Sf[tri0(i, k)], b = Sf[tri0(jc, k)], c = Sf[tri0(i, jc)];
            const df r = df_sub_acc(df{c.x, c.y},
                                    df_mul(df_mul(df{a.x, a.y}, inv), df{b.x, b.y}));
            Sf[tri0(i, jc)] = make_float2(r.h, r.l);
          }
          __syncthreads();
        }
        if (bad || k1 >= bs) break;
        const int np = k1 - k0;
        // W_jk = S_jk / d_k for the trailing columns j = k1 .. bs-1
        for (int e = tid; e < (bs - k1) * PW; e += THREADS) {
          const int jr = e / PW, q = e - jr * PW;
          float2 w = make_float2(0.0f, 0.0f);
          if (q < np) {
            const float2 sjk = Sf[tri0(k1 + jr, k0 + q)], iv = s_inv[q];
            const df t = df_mul(df{sjk.x, sjk.y}, df{iv.x, iv.y});
            w = make_float2(t.h, t.l);
          }
          Wp[e] = w;
        }
        __syncthreads();
        const int Tn = bs - k1;                  // trailing rows/columns k1 .. bs-1
        const int ntri = Tn * (Tn + 1) / 2;
        const int ntr = ntri + Tn;               // plus the bordered row's Tn entries
        for (int l = tid; l < ntr; l += THREADS) {
          int i, jr;
          if (l < ntri) {
            int ii = (int)((sqrtf(8.0f * (float)l + 1.0f) - 1.0f) * 0.5f);
            while (ii * (ii + 1) / 2 > l) --ii;
            while ((ii + 1) * (ii + 2) / 2 <= l) ++ii;
            i = k1 + ii;
            jr = l - ii * (ii + 1) / 2;
          } else {
            i = bs;
            jr = l - ntri;
          }
          const float2* si = Sf + tri0(i, k0);
          const float4* wj = (const float4*)(Wp + jr * PW);
          const float2 sij = Sf[tri0(i, k1 + jr)];
          df r = {sij.x, sij.y};
#pragma unroll
          for (int q2 = 0; q2 < PW / 2; ++q2) {
            const float4 w2 = wj[q2];
            if (2 * q2 < np) {
              const float2 a0 = si[2 * q2];
              r = df_sub_acc(r, df_mul(df{a0.x, a0.y}, df{w2.x, w2.y}));
            }
            if (2 * q2 + 1 < np) {
              const float2 a1 = si[2 * q2 + 1];
              r = df_sub_acc(r, df_mul(df{a1.x, a1.y}, df{w2.z, w2.w}));
            }
          }
          Sf[tri0(i, k1 + jr)] = make_float2(r.h, r.l);
        }
        __syncthreads();
      }
      if (tid == 0) s_fail = bad ? 1 : 0;
    }
    __syncthreads();
    if (s_fail) {
      hand_over();
      continue;
    }
    double v = 0.0;
    for (int t = tid; t < bs; t += THREADS) {
      const float2 dk = Sf[tri0(t, t)], z = Sf[tri0(bs, t)];
      const double dd = (double)dk.x + (double)dk.y, zz = (double)z.x + (double)z.y;
      v += log(dd) + zz * zz / dd;
    }
    const double s = cta_sum_mx(v, red);
    if (tid == 0) {
      double term = -0.5 * ((double)bs * log2pi + s);
      if (s_timeout) term = nan;
      a.terms[item] = term;
      const bool ok = isfinite(term);
      const int code = s_timeout ? SBV_ETIMEOUT : SBV_ENOTSPD;
      if (a.status) a.status[item] = ok ? 0 : code;
      if (!ok) record_failure(a.dstat, code, (int)blk, th_i);
    }
    __syncthreads();
    // the item's global slice is dead: drop its L2 lines without writing
    // them back to HBM (a discarded line reads as indeterminate until it is
    // written again, and every item writes each slice entry it reads).  The
    // slice starts on a 256-byte boundary and spans whole 256-byte units.
    {
      const char* g0 = (const char*)G;
      const int lines = (int)(lay.g_stride * sizeof(float) / 128);
      for (int q = tid; q < lines; q += THREADS)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(g0 + (size_t)q * 128) : "memory");
    }
    if (s_timeout) break;   // leave the item loop; TMEM is released below
  }
  // after a timed-out wait, give the outstanding MMAs one more bounded wait
  // before the accumulator columns are released
  if (TC) {
    if (s_timeout) umma::mbar_wait(&mma_bar, mma_phase, 1u << 24);
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem_base, MX_TMEM_COLS);
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

// Matern correlation at squared scaled distances d2 through the covariance
// arithmetic of the mixed kernel (stage 2): double-float square root,
// exponential and closed-form polynomial, the input split into a float pair.
__global__ void __launch_bounds__(256) matern_df_kernel(const double* d2, int64_t n, int nu2,
                                                        double* out) {
  __shared__ float tab_h[256], tab_l[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    tab_h[i] = c_df.tab_h[i];
    tab_l[i] = c_df.tab_l[i];
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const df s = df_from_double(d2[i]);
    const df r = df_sqrt(s);
    out[i] = df_to_double(df_matern(r, s, nu2, c_df, tab_h, tab_l));
  }
}

int run_matern_df(sbv_ctx* ctx, int nu2, const double* d2, int64_t n, double* out,
                  cudaStream_t s) {
  int st = upload_df_consts(ctx);
  if (st) return st;
  if (n == 0) return SBV_OK;
  const int64_t want = (n + 255) / 256;
  const int grid = (int)std::min<int64_t>(want, (int64_t)ctx->num_sms * 8);
  matern_df_kernel<<<grid, 256, 0, s>>>(d2, n, nu2, out);
  SBV_CUDA_TRY(ctx, cudaGetLastError());
  return SBV_OK;
}

template <int THREADS, bool TC, bool PRED, bool GA>
static int occ(sbv_ctx* ctx, size_t bytes, int* out) {
  SBV_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                        out, loglik_mixed_kernel<THREADS, TC, PRED, GA>, THREADS, bytes));
  return SBV_OK;
}

template <int THREADS, bool TC>
static int occ_t(sbv_ctx* ctx, bool pred, bool ga, size_t bytes, int* out) {
  if (ga) return pred ? occ<THREADS, TC, true, true>(ctx, bytes, out)
                      : occ<THREADS, TC, false, true>(ctx, bytes, out);
  return pred ? occ<THREADS, TC, true, false>(ctx, bytes, out)
              : occ<THREADS, TC, false, false>(ctx, bytes, out);
}

static int mixed_occupancy(sbv_ctx* ctx, int threads, bool tc, bool pred, bool ga, size_t bytes,
                           int* out) {
  if (tc) return threads == 512 ? occ_t<512, true>(ctx, pred, ga, bytes, out)
                                : occ_t<256, true>(ctx, pred, ga, bytes, out);
  return threads == 512 ? occ_t<512, false>(ctx, pred, ga, bytes, out)
                        : occ_t<256, false>(ctx, pred, ga, bytes, out);
}

// ---------------------------------------------------------------------------
// Launch planning: layout, threads per CTA, grid, scratch size.  The shape
// (threads, CTAs per SM) comes from the context's autotuning record when one
// matches (precision, prediction mode, capacity, d), else 256 threads and as
// many CTAs per SM (<= 2) as shared memory allows.
// ---------------------------------------------------------------------------
static int mixed_static_smem(sbv_ctx* ctx, size_t* out);

int mixed_plan(sbv_ctx* ctx, int nmax, int mcap, int bcap, int d, int precision, bool pred,
               int64_t items, MixedPlan* o) {
  const int ncap = std::max(nmax, 1);
  // the tensor-core residual is the SBV_PREC_MIXED_BF16 variant (likelihood only)
  const bool tc = precision == SBV_PREC_MIXED_BF16 && !pred;
  o->pred = pred;
  o->tc = tc;
  int threads = 256, per_sm = 2, tile = 0;
  if (ctx->force.threads) {
    threads = ctx->force.threads;
    per_sm = ctx->force.per_sm;
    tile = ctx->force.tile;
  } else {
    for (const auto& t : ctx->tuned)
      if (t.precision == precision && t.pred == (int)pred && t.ncap == ncap && t.d == d) {
        threads = t.threads;
        per_sm = t.per_sm;
        tile = t.tile;
      }
  }
  o->wcap = tile;
  const int tc_np = threads >= 512 ? 96 : 48;   // MX_NP of the kernel variant
  o->lay = mixed_layout(ncap, mcap, bcap, d, tc, false, tc_np);
  size_t static_smem = 0;
  if (int st0 = mixed_static_smem(ctx, &static_smem)) return st0;
  if (o->lay.bytes + static_smem > ctx->smem_optin)
    o->lay = mixed_layout(ncap, mcap, bcap, d, tc, true, tc_np);
  if (o->lay.bytes + static_smem > ctx->smem_optin)
    return fail(ctx, SBV_EUNSUPPORTED,
                "mixed path: a block with N=%d (d=%d) needs %zu bytes of shared memory", nmax, d,
                o->lay.bytes);
  int st = mixed_prepare(ctx);   // occupancy queries need the shared-memory opt-in
  if (st) return st;
  int fit = 0;
  // The occupancy calculator admits one CTA per SM for any variant with
  // tcgen05 instructions, whatever its shared memory; the SM runs two when
  // shared memory and registers allow (measured: 25.4 ms at two CTAs of 256
  // threads per SM against 40.3 ms at one on the 1M-point workload).  So the
  // tensor-core variant takes the cap of its twin without tcgen05 (same
  // threads, registers and shared memory) and of TMEM: MX_TMEM_COLS columns
  // per CTA (256 at 256 threads, 512 at 512) out of an SM's 512.
  if ((st = mixed_occupancy(ctx, threads, false, pred, o->lay.ga, o->lay.bytes, &fit))) return st;
  if (tc) fit = std::min(fit, threads >= 512 ? 1 : 2);
  if (fit < 1)
    return fail(ctx, SBV_EUNSUPPORTED, "mixed path: no CTA of %d threads fits an SM (N=%d, d=%d)",
                threads, nmax, d);
  per_sm = std::max(1, std::min(per_sm, fit));
  int grid = ctx->num_sms * per_sm;
  if (grid > items) grid = (int)std::max<int64_t>(items, 1);
  o->threads = threads;
  o->grid = grid;
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
// the SM's 256 KB serves as L1 for its slices.
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

// The largest static shared memory of the variants, queried once per device.
static int mixed_static_smem(sbv_ctx* ctx, size_t* out) {
  const int dev = ctx->device;
  if (dev < 64 && g_mixed_static[dev]) {
    *out = g_mixed_static[dev];
    return SBV_OK;
  }
  // prediction never takes the tensor-core residual: no <TC, PRED> variant
  const size_t v[6] = {static_smem_of<256, false, false>(), static_smem_of<256, false, true>(),
                       static_smem_of<512, false, false>(), static_smem_of<512, false, true>(),
                       static_smem_of<256, true, false>(),  static_smem_of<512, true, false>()};
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
  if ((st = allow_smem<256, false, false>(ctx, b)) || (st = allow_smem<256, false, true>(ctx, b)) ||
      (st = allow_smem<512, false, false>(ctx, b)) || (st = allow_smem<512, false, true>(ctx, b)) ||
      (st = allow_smem<256, true, false>(ctx, b)) || (st = allow_smem<512, true, false>(ctx, b)))
    return st;
  if (ctx->device < 64) g_mixed_ready[ctx->device] = true;
  return SBV_OK;
}

// Enqueue the kernel; P carries the arguments, Xs (or NULL), the scratch and
// the hand-over list.
int mixed_enqueue(sbv_ctx* ctx, MixedArgs& P, const MixedPlan& o, cudaStream_t s) {
  int st = 0;
  if ((st = mixed_prepare(ctx))) return st;
  P.lay = o.lay;
  P.wcap = o.wcap;
  if (o.pred)
    return o.threads == 512 ? launch_variant<512, false, true>(ctx, P, o.grid, s)
                            : launch_variant<256, false, true>(ctx, P, o.grid, s);
  if (o.tc)
    return o.threads == 512 ? launch_variant<512, true, false>(ctx, P, o.grid, s)
                            : launch_variant<256, true, false>(ctx, P, o.grid, s);
  return o.threads == 512 ? launch_variant<512, false, false>(ctx, P, o.grid, s)
                          : launch_variant<256, false, false>(ctx, P, o.grid, s);
}

// Plan, split the points and take the scratch from the context workspace.
static int launch_mixed(sbv_ctx* ctx, MixedArgs& P, int nmax, int mcap, int bcap, int precision,
                        bool pred, int64_t items, cudaStream_t s) {
  int st = 0;
  MixedPlan o;
  if ((st = mixed_plan(ctx, nmax, mcap, bcap, P.a.d, precision, pred, items, &o))) return st;
  const int64_t total = P.a.n * P.a.d;
  P.Xs = nullptr;
  if (P.a.dtype == SBV_F64) {
    float2* xs = (float2*)ws_get(ctx, WS_XSPLIT, (size_t)total * sizeof(float2), &st);
    if (!xs) return st;
    if ((st = mixed_split(ctx, P.a.X, P.a.dtype, total, xs, s))) return st;
    P.Xs = xs;
  }
  float* buf = (float*)ws_get(ctx, WS_MATRIX, o.scratch_bytes(), &st);
  if (!buf) return st;
  P.gbase = buf;
  return mixed_enqueue(ctx, P, o, s);
}

int launch_loglik_mixed(sbv_ctx* ctx, const LoglikArgs& a0, int nmax, int bsmax, int precision,
                        unsigned int* fb_list, unsigned int* fb_count, cudaStream_t s) {
  MixedArgs P;
  memset(&P, 0, sizeof(P));
  P.a = a0;
  P.fb_list = fb_list;
  P.fb_count = fb_count;
  return launch_mixed(ctx, P, nmax, a0.m, bsmax, precision, false, a0.bc * (int64_t)a0.B, s);
}

// Prediction: a0 carries X, y, d, nbr (ntest x m), m, theta, nu2, dstat, counter.
int launch_predict_mixed(sbv_ctx* ctx, const LoglikArgs& a0, const void* Xt, int64_t nt,
                         double* mean, double* var, double* var_latent, int precision,
                         unsigned int* fb_list, unsigned int* fb_count, cudaStream_t s,
                         const int64_t* tptr, const int32_t* tpts, int bsmax) {
  MixedArgs P;
  memset(&P, 0, sizeof(P));
  P.a = a0;
  P.Xt = Xt;
  P.nt = nt;
  P.mean = mean;
  P.var = var;
  P.var_latent = var_latent;
  P.fb_list = fb_list;
  P.fb_count = fb_count;
  P.tptr = tptr;
  P.tpts = tpts;
  if (!tptr) bsmax = 1;
  return launch_mixed(ctx, P, a0.m + bsmax, a0.m, bsmax, precision, true, nt, s);
}

}  // namespace sbv
