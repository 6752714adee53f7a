// Types and launch helpers of the mixed-precision block kernel, shared by the
// per-call path (loglik_mixed.cu) and the captured-graph path (graph.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "block_common.cuh"
#include "sbv_internal.cuh"

namespace sbv {

// threads per CTA: 256 (two CTAs per SM when shared memory allows) or 512
// (one CTA per SM); the autotuner picks per structure
constexpr int MX_MAX_WARPS = 16;
constexpr int NB = 16;  // panel width = diagonal tile size of the FP32 factor of Sigma_JJ

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Packed lower triangle with every row padded to a multiple of four floats:
// row i = 4a + b starts at 4 (a + 1)(2a + b), so a four-column segment that
// starts at a multiple of four is 16-byte aligned (float4 access).  trp_size
// is the number of floats of rows 0 .. rows-1.
__host__ __device__ __forceinline__ int trp(int i, int j) {
  const int a = i >> 2, b = i & 3;
  return 4 * (a + 1) * (2 * a + b) + j;
}
__host__ __device__ inline size_t trp_size(int rows) {
  const size_t a = (size_t)rows >> 2, b = (size_t)rows & 3;
  return 4 * (a + 1) * (2 * a + b);
}

// Row stride (floats) of the right-hand-side block of an item with mb
// neighbours: at least mb rounded up to four, and 4 (mod 32), so that lanes
// reading float4 segments of consecutive rows hit distinct banks.
__host__ __device__ __forceinline__ int rhs_stride(int mb) { return ((mb + 27) / 32) * 32 + 4; }

// Packed lower triangle without padding (the bs x bs conditional system).
__host__ __device__ __forceinline__ int tri0(int i, int j) { return (i * (i + 1) >> 1) + j; }

// Shared memory of one CTA (one item at a time):
//   y       observations of the item's points as float pairs
//   idiag   1 / L_tt of the FP32 factor of Sigma_JJ
//   union   covariance phase: scaled coordinates (hi, lo) and the exp2 table;
//           factorisation: the FP32 panel copy and a staged diagonal tile
//   A       packed lower triangle of Sigma_JJ -> its FP32 factor L (diagonal
//           tiles later replaced by their inverses)
//   X       right-hand-side block: row r < bs holds Sigma_{J, b_r}, row bs
//           holds y_J; they become L^{-1} (.), then Sigma_JJ^{-1} (.); after
//           the Schur-complement passes the region holds the bs x bs
//           conditional system (bordered by y_B - mu) in double-float
// With ga, A and X live in a per-CTA slice of global memory instead.
//   union   residual phase: two constants per right-hand side, and a block
//           of 16 residual columns (then L^{-1} of them) or, before it, the
//           BF16 digit tiles of one K-step of the tensor-core residual
// Per-CTA global memory: the double-float joint covariance (N x N, both
// triangles), L^{-1} R for every right-hand side and the partial
// Schur-complement system.
struct MixedLayout {
  int ncap;             // largest N = mb + bs held
  int mcap;             // largest mb (neighbour count)
  int d;
  int pstride;          // column stride of the FP32 panel copy (floats)
  bool ga;              // A and X in global memory
  size_t a_floats;      // floats of A (rounded to 64)
  size_t x_floats;      // floats of the X region (rounded to 64)
  size_t off_y, off_v, off_u, off_vl, off_tab, off_stile, off_cc, off_sch, off_A, off_X, bytes;
  // per-CTA global slice, in floats
  size_t g_R, g_Sp, g_A, g_X, g_stride;
};

// bcap: the largest bs of the structure when known (0: any bs up to ncap).
// tc_np: right-hand sides per tensor-core pass (48 for 256 threads, 96 for 512).
__host__ __device__ inline MixedLayout mixed_layout(int ncap, int mcap, int bcap, int d,
                                                    bool tc, bool ga = false, int tc_np = 96) {
  MixedLayout L;
  L.ncap = ncap;
  L.mcap = mcap < ncap ? mcap : ncap;
  L.d = d;
  L.ga = ga;
  L.a_floats = align_up(trp_size(L.mcap), 64);
  // the largest right-hand-side block: nr = N + 1 - mb rows (at most bcap + 1)
  // of rhs_stride(mb); with bcap known, also room for the largest bordered
  // conditional system, (bcap + 1) (bcap + 2) floats
  const int nrcap = bcap > 0 && bcap < ncap ? bcap + 1 : ncap + 1;
  size_t xf = 8;
  for (int mb = 0; mb <= L.mcap; ++mb) {
    const int nr = ncap + 1 - mb < nrcap ? ncap + 1 - mb : nrcap;
    const size_t v = (size_t)nr * rhs_stride(mb);
    if (v > xf) xf = v;
  }
  if (bcap > 0 && (size_t)nrcap * (nrcap + 1) > xf) xf = (size_t)nrcap * (nrcap + 1);
  L.x_floats = align_up(xf, 64);
  L.pstride = (int)align_up((size_t)ncap + 1, 4);
  size_t o = 0;
  L.off_y = o;  o += align_up((size_t)(ncap + 1) * sizeof(float2), 16);
  L.off_v = o;  o += align_up((size_t)(L.mcap + 4) * sizeof(float), 16);
  o = align_up(o, 128);
  const size_t coord = align_up((size_t)d * ncap * sizeof(float), 16);
  const size_t tab = 2 * 256 * sizeof(float);             // exp2 table, hi and lo
  const size_t stile = (size_t)NB * NB * sizeof(float2);   // a diagonal tile's originals
  const size_t panel = align_up((size_t)NB * L.pstride * sizeof(float), 16);
  // residual phase: a block of 16 right-hand sides of the residual, then one
  // grid constant per right-hand side
  const size_t rblk = align_up((size_t)16 * rhs_stride(L.mcap) * sizeof(float), 16);
  const size_t cc = align_up((size_t)2 * (ncap + 2) * sizeof(float), 128);
  // tensor-core residual (before the residual block is used): five 128 x 16
  // BF16 digit tiles of Sigma_JJ and three tc_np x 16 digit tiles of X^
  // (K-major core-matrix layout)
  const size_t sch = tc ? 5 * 4096 + 3 * (size_t)tc_np * 32 : 0;
  const size_t rpart = align_up(rblk > sch ? rblk : sch, 128);
  size_t uni = 2 * coord + tab;
  if (panel + stile > uni) uni = panel + stile;
  if (rpart + cc > uni) uni = rpart + cc;
  uni = align_up(uni, 128);
  L.off_u = o;
  L.off_vl = o + coord;
  L.off_tab = o + 2 * coord;
  L.off_stile = o + panel;
  L.off_sch = o;               // 128-byte aligned (the digit tiles need 16)
  // the constants at the end of the union, so the residual block can take
  // everything before them (more than 16 right-hand sides when room allows)
  L.off_cc = o + uni - cc;
  o += align_up(uni, 128);
  L.off_A = o;
  if (!ga) o += L.a_floats * sizeof(float);
  L.off_X = o;
  if (!ga) o += L.x_floats * sizeof(float);
  L.bytes = o;
  // global slice: S (ncap^2 float pairs), R, Sp, then A and X when ga
  size_t g = align_up((size_t)2 * ncap * ncap, 64);
  L.g_R = g;  g += L.x_floats;
  L.g_Sp = g; g += L.x_floats;
  L.g_A = g;  if (ga) g += L.a_floats;
  L.g_X = g;  if (ga) g += L.x_floats;
  L.g_stride = align_up(g, 64);
  return L;
}

struct MixedArgs {
  LoglikArgs a;
  const float2* Xs;      // split FP64 points, or NULL for FP32 points (a.X read directly)
  float* gbase;          // per-CTA global slices (lay.g_stride floats each)
  MixedLayout lay;
  // items the mixed kernel hands to the FP64 kernel: a pivot that is not
  // positive in FP32 or double-float, or a conditional system larger than the
  // X region; fb_count and the list are read by the FP64 kernel in list mode
  unsigned int* fb_list;
  unsigned int* fb_count;
  // right-hand sides per column block of the residual and the conditional
  // system (0: as many as the residual block's room holds, at most 64)
  int wcap;
  // prediction mode: one item per test point, J = its m nearest training
  // points, or (tptr set) one item per block of test points b, the points
  // tpts[tptr[b] .. tptr[b+1]) sharing the block's J
  const void* Xt;        // test points (dtype of a.X)
  int64_t nt;            // items
  const int64_t* tptr;
  const int32_t* tpts;
  double* mean;
  double* var;
  double* var_latent;
};

struct MixedPlan {
  MixedLayout lay;
  bool pred, tc;
  int threads, grid, wcap;
  size_t scratch_bytes() const { return lay.g_stride * sizeof(float) * (size_t)grid; }
};

int mixed_plan(sbv_ctx* ctx, int nmax, int mcap, int bcap, int d, int precision, bool pred,
               int64_t items, MixedPlan* o);
int mixed_split(sbv_ctx* ctx, const void* X, int dtype, int64_t total, float2* xs,
                cudaStream_t s);
int mixed_enqueue(sbv_ctx* ctx, MixedArgs& P, const MixedPlan& o, cudaStream_t s);
int mixed_prepare(sbv_ctx* ctx);

}  // namespace sbv
