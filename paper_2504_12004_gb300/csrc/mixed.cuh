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
constexpr int NB = 16;  // panel width = diagonal tile size

struct MixedLayout {
  int ncap;             // largest N held (rows 0..ncap-1 plus the bordered row)
  int d;
  int pstride;          // row stride of the FP32 column-major panel (CUDA-core update)
  uint32_t opnd_piece;  // bytes of one BF16 operand piece (tensor-core update)
  bool ga;              // the packed triangle A lives in global memory (per-CTA slice)
  size_t a_floats;      // floats of one padded packed triangle (rounded to 64)
  int part_cap;         // float4 partial sums the residual phase may hold
  size_t off_y, off_v, off_u, off_vl, off_c, off_tab, off_stile, off_A, bytes;
};

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

// One shared-memory region (off_u) serves three phases in turn: the scaled
// coordinates and the exp2 tables (covariance), the panel operand and the
// staged diagonal tile (factorisation) and, during refinement, the residual
// partial sums followed (off_c) by the two accumulated corrections.
// With ga, the packed triangle (the largest piece, 4 (N+1)(N+2)/2 bytes) is
// left out of shared memory; the kernel then addresses a per-CTA slice of a
// global buffer, which stays in L1/L2 for the CTA's lifetime.
__host__ __device__ inline MixedLayout mixed_layout(int ncap, int d, bool tc, bool ga = false) {
  MixedLayout L;
  L.ncap = ncap;
  L.d = d;
  L.ga = ga;
  L.a_floats = align_up(trp_size(ncap + 1), 64);
  L.pstride = (int)align_up((size_t)ncap + 1, 4);
  L.opnd_piece = (uint32_t)(((ncap + 1 + 127) / 128) * 128 * 32);
  size_t o = 0;
  L.off_y = o;  o += align_up((size_t)(ncap + 1) * sizeof(float2), 16);
  // x0 x0J r1 r2 ldiag idiag, each 16-byte aligned
  L.off_v = o;  o += (size_t)6 * align_up((size_t)ncap + 1, 4) * sizeof(float);
  o = align_up(o, 128);
  const size_t coord = align_up((size_t)d * ncap * sizeof(float), 16);
  const size_t tab = 2 * 256 * sizeof(float);          // exp2 table, hi and lo
  const size_t stile = (size_t)NB * NB * sizeof(float2);  // a diagonal tile's originals
  size_t uni = 2 * coord + tab;
  const size_t panel =
      align_up(tc ? 3 * (size_t)L.opnd_piece : (size_t)NB * L.pstride * sizeof(float), 16) + stile;
  size_t part = (size_t)(32 * MX_MAX_WARPS > ncap ? 32 * MX_MAX_WARPS : ncap) * sizeof(float4);
  const size_t corr = align_up((size_t)2 * (ncap + 1) * sizeof(float), 16);
  if (panel > uni) uni = panel;
  if (part + corr > uni) uni = part + corr;
  // the partial sums take whatever the region holds anyway (more column
  // chunks for the residual), up to 16 chunks
  const size_t part_max = (size_t)16 * (ncap + 1) * sizeof(float4);
  part = (uni - corr) / sizeof(float4) * sizeof(float4);
  if (part > part_max) part = part_max;
  L.part_cap = (int)(part / sizeof(float4));
  L.off_u = o;
  L.off_vl = o + coord;
  L.off_tab = o + 2 * coord;
  L.off_stile = o + panel - stile;
  L.off_c = o + part;
  o += align_up(uni, 16);
  L.off_A = o;
  if (!ga) o += align_up(trp_size(ncap + 1) * sizeof(float), 16);
  L.bytes = o;
  return L;
}

struct MixedArgs {
  LoglikArgs a;
  const float2* Xs;      // split FP64 points, or NULL for FP32 points (a.X read directly)
  float2* scratch;
  size_t scratch_stride;
  float* gA;             // packed triangles, lay.a_floats per CTA (lay.ga only)
  MixedLayout lay;
  // prediction mode: one item per test point, J = its m nearest training points
  const void* Xt;        // test points (dtype of a.X)
  int64_t nt;
  double* mean;
  double* var;
  double* var_latent;
};

struct MixedPlan {
  MixedLayout lay;
  bool tc, pred;
  int threads, grid;
  size_t scratch_stride;  // float2 elements per CTA slice
  // bytes of the per-CTA scratch buffer: the FP32-pair copy of Sigma, then
  // (lay.ga) the packed triangles from byte offset ga_offset
  size_t scratch_bytes() const {
    return ga_offset() + (lay.ga ? lay.a_floats * sizeof(float) * (size_t)grid : 0);
  }
  size_t ga_offset() const { return align_up(scratch_stride * sizeof(float2) * (size_t)grid, 256); }
};

int mixed_plan(sbv_ctx* ctx, int nmax, int d, int precision, bool pred, int64_t items,
               MixedPlan* o);
int mixed_split(sbv_ctx* ctx, const void* X, int dtype, int64_t total, float2* xs,
                cudaStream_t s);
int mixed_enqueue(sbv_ctx* ctx, MixedArgs& P, const MixedPlan& o, cudaStream_t s);
int mixed_prepare(sbv_ctx* ctx);

}  // namespace sbv
