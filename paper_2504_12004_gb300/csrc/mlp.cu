// Likelihood surrogate network on the tensor cores: in -> 256 -> 256 -> 256 -> 1
// with GELU, trained by MSE and Adam.  The paper has no learned part; the
// network proposes parameter vectors to the likelihood maximisation (Alg. 1
// Step 5 evaluated repeatedly), and the exact likelihood judges them.
//
// Precision: the two 256 x 256 layers run as tcgen05 BF16 MMAs with FP32
// accumulation in TMEM, in the forward pass (H W^T), the backward pass
// (dZ W) and the weight gradients (dZ^T H).  The input layer (in <= 16), the
// output layer, biases, GELU and its derivative, bias and input-weight
// gradients and Adam run in FP32 on the CUDA cores.
//
// Kernels per training step (all persistent state lives in sbv_mlp):
//   mlp_fused_kernel   one CTA per 128 rows (one TMEM lane per row): forward,
//                      loss, backward down to dZ1; writes the transposed BF16
//                      operands of the weight-gradient GEMMs and per-tile
//                      partial sums of the CUDA-core gradients
//   mlp_wgrad_kernel   dW2, dW3 = dZ^T H, split over the batch (split-K),
//                      one 128 x 256 TMEM accumulator per CTA
//   mlp_adam_kernel    sums the partials in a fixed order (deterministic),
//                      applies Adam to the FP32 masters and refreshes the
//                      tiled BF16 operand copies of W2, W3 and their transposes
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sbv_internal.cuh"
#include "umma.cuh"

using namespace sbv;

namespace {

constexpr int WID = 256;            // hidden width
constexpr int TILE = 128;           // rows per CTA = TMEM lanes
constexpr int MAXIN = SBV_MLP_MAX_IN;
constexpr int A_BYTES = TILE * WID * 2;   // 128 x 256 BF16 operand
constexpr int B_BYTES = WID * WID * 2;    // 256 x 256 BF16 operand
constexpr uint32_t kWait = 1u << 24;      // bounded mbarrier polls
constexpr int KCH = 64;                   // batch rows per weight-gradient chunk

// Byte offset of element (row, k) of a K-major operand with `rows` rows, no
// swizzle, stored as consecutive K-slices of 16: slice k/16 holds rows x 16
// elements in 8 x 8 core matrices (core matrix (row/8, (k%16)/8) at
// (row/8)*256 + ((k%16)/8)*128, row r of it at 16 (r%8)).
__host__ __device__ __forceinline__ uint32_t tiled_off(int row, int k, int rows) {
  return (uint32_t)((k >> 4) * rows * 32 + (row >> 3) * 256 + ((k >> 3) & 1) * 128 +
                    (row & 7) * 16 + (k & 7) * 2);
}

// packed FP32 parameter offsets: W1 b1 W2 b2 W3 b3 w4 b4
struct Off {
  int64_t W1, b1, W2, b2, W3, b3, w4, b4, total;
};
__host__ __device__ inline Off offsets(int in) {
  Off o;
  o.W1 = 0;
  o.b1 = (int64_t)WID * in;
  o.W2 = o.b1 + WID;
  o.b2 = o.W2 + (int64_t)WID * WID;
  o.W3 = o.b2 + WID;
  o.b3 = o.W3 + (int64_t)WID * WID;
  o.w4 = o.b3 + WID;
  o.b4 = o.w4 + WID;
  o.total = o.b4 + 1;
  return o;
}

// per-tile partial sums written by the fused kernel
struct PartOff {
  int dw4, db3, db2, db1, dW1, db4, loss, stride;
};
__host__ __device__ inline PartOff part_offsets(int in) {
  PartOff p;
  p.dw4 = 0;
  p.db3 = WID;
  p.db2 = 2 * WID;
  p.db1 = 3 * WID;
  p.dW1 = 4 * WID;
  p.db4 = 4 * WID + WID * in;
  p.loss = p.db4 + 1;
  p.stride = (p.loss + 1 + 3) & ~3;
  return p;
}

struct FusedArgs {
  const float* X;        // rows x in (row-major)
  const float* t;        // targets (training) or NULL
  const int32_t* idx;    // row indices of the batch into X / t, or NULL
  int64_t K;             // rows in the batch
  int64_t kpad;          // row stride of the transposed operands (multiple of 128)
  float inv_K;           // 1 / K
  int in;
  int train;
  const float* p;        // FP32 master parameters
  const uint4* w2;       // tiled BF16 W2   (B operand of H1 W2^T)
  const uint4* w3;       // tiled BF16 W3
  const uint4* w2t;      // tiled BF16 W2^T (B operand of dZ2 W2)
  const uint4* w3t;      // tiled BF16 W3^T
  __nv_bfloat16* h1t;    // [256][kpad] transposed BF16 H1, H2, dZ2, dZ3
  __nv_bfloat16* h2t;
  __nv_bfloat16* dz2t;
  __nv_bfloat16* dz3t;
  float* part;           // [tiles][PartOff::stride]
  float* s;              // predictions (predict mode)
  float* dsdx;           // K x in input gradients (predict mode) or NULL
  int* timeout;
};

__device__ __forceinline__ float gelu_f(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_prime_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

// 16 consecutive features of one row as two 16-byte core-matrix rows
__device__ __forceinline__ void store_row16(unsigned char* op, int row, int c, const float (&v)[16]) {
  uint4 lo = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                        pack_bf16(v[6], v[7]));
  uint4 hi = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]),
                        pack_bf16(v[14], v[15]));
  *reinterpret_cast<uint4*>(op + tiled_off(row, c, TILE)) = lo;
  *reinterpret_cast<uint4*>(op + tiled_off(row, c + 8, TILE)) = hi;
}

// Sum 16 values over the 32 lanes of a warp with 16 shuffles (recursive
// halving); afterwards lane l holds the total of value index
// 8 b4 + 4 b3 + 2 b2 + b1 (b_k = bit k of l), lanes l and l^1 alike.
__device__ __forceinline__ float warp_colsum16(float (&v)[16], int lane) {
  {
    const bool up = lane & 16;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float send = up ? v[i] : v[i + 8];
      const float keep = up ? v[i + 8] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
  {
    const bool up = lane & 8;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float send = up ? v[i] : v[i + 4];
      const float keep = up ? v[i + 4] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
  }
  {
    const bool up = lane & 4;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float send = up ? v[i] : v[i + 2];
      const float keep = up ? v[i + 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
  }
  {
    const bool up = lane & 2;
    const float send = up ? v[0] : v[1];
    const float keep = up ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}
__device__ __forceinline__ int colsum_index(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

// Start copying a 128 KB tiled operand into shared memory with the bulk-copy
// engine (four 32 KB copies on one mbarrier); stage_wait blocks every thread
// until it has landed.  Thread 0 issues; the caller guarantees that nothing
// still reads the destination (its previous MMA has completed).
__device__ __forceinline__ void stage_issue(unsigned char* sB, const uint4* g, uint64_t* bar) {
  if (threadIdx.x == 0) {
    umma::mbar_arrive_expect_tx(bar, B_BYTES);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      umma::bulk_g2s(sB + q * (B_BYTES / 4), reinterpret_cast<const unsigned char*>(g) + q * (B_BYTES / 4),
                     B_BYTES / 4, bar);
  }
}
__device__ __forceinline__ bool stage_wait(uint64_t* bar, uint32_t& phase, int* s_timeout) {
  if (!umma::mbar_wait(bar, phase, kWait)) *s_timeout = 1;
  phase ^= 1u;
  __syncthreads();   // the outcome is the same for every thread
  return *s_timeout == 0;
}

// D[tmem] = A (128 x 256) * B (256 x 256)^T from the tiled operands in shared
// memory; every thread calls, thread 0 issues the 16 MMAs of K = 16.
__device__ bool gemm_128x256(uint32_t d_tmem, const unsigned char* sA, const unsigned char* sB,
                             uint64_t* bar, uint32_t& phase, int* s_timeout) {
  umma::fence_proxy_async();
  umma::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0) {
    umma::fence_after_sync();
    const uint32_t idesc = umma::idesc_bf16_f32(128, 256);
    const uint32_t a0 = umma::smem_u32(sA), b0 = umma::smem_u32(sB);
#pragma unroll 1
    for (int kk = 0; kk < WID / 16; ++kk) {
      const uint64_t ad = umma::smem_desc(a0 + kk * (TILE * 32), 128, 256);
      const uint64_t bd = umma::smem_desc(b0 + kk * (WID * 32), 128, 256);
      umma::mma_bf16(d_tmem, ad, bd, idesc, kk > 0 ? 1u : 0u);
    }
    umma::mma_commit(bar);
  }
  const bool done = umma::mbar_wait(bar, phase, kWait);
  phase ^= 1u;
  if (!done) *s_timeout = 1;
  umma::fence_after_sync();
  __syncthreads();   // the outcome is the same for every thread
  return *s_timeout == 0;
}

__device__ __forceinline__ void tmem_row16(uint32_t taddr, float (&v)[16]) {
  umma::tmem_ld16(taddr, v);
  umma::tmem_wait_ld();
}

// Two threads per row: warps 0-3 take columns 0..127 of rows 32 (w % 4) ..,
// warps 4-7 columns 128..255 of the same rows (a warp reads TMEM lanes
// 32 (w % 4) .. 32 (w % 4) + 31).
constexpr int MT = 2 * TILE;

__global__ void __launch_bounds__(MT, 1) mlp_fused_kernel(FusedArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;
  unsigned char* sB = smem + A_BYTES;
  float* sX = reinterpret_cast<float*>(sB + B_BYTES);   // TILE x MAXIN
  float* sred = sX + TILE * MAXIN;                       // 3 x 4 row groups x 256
  __shared__ uint64_t bar;    // MMA completion
  __shared__ uint64_t tbar;   // bulk copies of the weight operands
  __shared__ uint32_t s_tmem;
  __shared__ int s_timeout;
  __shared__ float s_loss[8];
  __shared__ float s_part[2][TILE];   // per-half partial outputs

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int rg = warp & 3, hf = warp >> 2;
  const int r = rg * 32 + lane;                       // row in the tile
  const int cb = hf * (WID / 2), ce = cb + WID / 2;   // this thread's columns
  const int64_t row = (int64_t)blockIdx.x * TILE + r;
  const bool valid = row < a.K;
  const int in = a.in;
  const Off o = offsets(in);
  const PartOff po = part_offsets(in);
  const float* __restrict__ P = a.p;

  if (warp == 0) umma::tmem_alloc(&s_tmem, 512);
  if (t == 0) {
    umma::mbar_init(&bar, 1);
    umma::mbar_init(&tbar, 1);
    s_timeout = 0;
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tm = s_tmem;
  const uint32_t lane_base = tm + ((uint32_t)(32 * rg) << 16);
  uint32_t phase = 0, tphase = 0;
  bool ok = true;
  stage_issue(sB, a.w2, &tbar);   // lands while layer 1 runs

  // ---- input row and layer 1 (CUDA cores, FP32) ----
  float x[MAXIN];
  const int64_t src = valid ? (a.idx ? (int64_t)a.idx[row] : row) : 0;
#pragma unroll
  for (int j = 0; j < MAXIN; ++j) {
    x[j] = (valid && j < in) ? a.X[src * in + j] : 0.0f;
    if (hf == 0) sX[r * MAXIN + j] = x[j];
  }
  const float tgt = (valid && a.train) ? a.t[src] : 0.0f;
  for (int c = cb; c < ce; c += 16) {
    float h[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int f = c + e;
      float z = __ldg(P + o.b1 + f);
#pragma unroll
      for (int j = 0; j < MAXIN; ++j)
        if (j < in) z = fmaf(__ldg(P + o.W1 + (int64_t)f * in + j), x[j], z);
      h[e] = gelu_f(z);
      if (a.train) a.h1t[(int64_t)f * a.kpad + row] = __float2bfloat16_rn(h[e]);
    }
    store_row16(sA, r, c, h);
  }
  // ---- layer 2: Z2 = H1 W2^T + b2 -> TMEM columns 0..255 ----
  ok = stage_wait(&tbar, tphase, &s_timeout);
  if (ok) ok = gemm_128x256(tm, sA, sB, &bar, phase, &s_timeout);
  bool pending = false;
  if (ok) {
    stage_issue(sB, a.w3, &tbar);   // sB is free: lands during the epilogue
    pending = true;
  }
  if (ok) {
    for (int c = cb; c < ce; c += 16) {
      float v[16];
      tmem_row16(lane_base + c, v);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        v[e] = gelu_f(v[e] + __ldg(P + o.b2 + c + e));
        if (a.train) a.h2t[(int64_t)(c + e) * a.kpad + row] = __float2bfloat16_rn(v[e]);
      }
      store_row16(sA, r, c, v);
    }
  }
  __syncthreads();
  // ---- layer 3: Z3 = H2 W3^T + b3 -> TMEM columns 256..511 ----
  if (pending) {
    ok = stage_wait(&tbar, tphase, &s_timeout) && ok;
    pending = false;
  }
  if (ok) ok = gemm_128x256(tm + 256, sA, sB, &bar, phase, &s_timeout);
  if (ok) {
    stage_issue(sB, a.w3t, &tbar);
    pending = true;
  }
  // ---- output and loss ----
  float sp = 0.0f;
  if (ok) {
    for (int c = cb; c < ce; c += 16) {
      float v[16];
      tmem_row16(lane_base + 256 + c, v);
#pragma unroll
      for (int e = 0; e < 16; ++e)
        sp = fmaf(gelu_f(v[e] + __ldg(P + o.b3 + c + e)), __ldg(P + o.w4 + c + e), sp);
    }
  }
  s_part[hf][r] = sp;
  __syncthreads();
  const float sv = (__ldg(P + o.b4) + s_part[0][r]) + s_part[1][r];
  float ds;
  if (a.train) {
    const float res = sv - tgt;
    ds = valid ? 2.0f * res * a.inv_K : 0.0f;
    float l2 = (valid && hf == 0) ? res * res : 0.0f;
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, sh);
    if (lane == 0) s_loss[warp] = l2;
  } else {
    ds = valid ? 1.0f : 0.0f;
    if (valid && hf == 0) a.s[row] = sv;
  }
  // ---- dZ3 = ds w4 * GELU'(Z3); partial sums of dw4 and db3 ----
  float* red_w4 = sred;
  float* red_b3 = sred + 4 * WID;
  float* red_b2 = sred + 8 * WID;
  if (ok) {
    for (int c = cb; c < ce; c += 16) {
      float v[16], g[16], hw[16];
      tmem_row16(lane_base + 256 + c, v);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const float z = v[e] + __ldg(P + o.b3 + c + e);
        hw[e] = ds * gelu_f(z);
        g[e] = ds * __ldg(P + o.w4 + c + e) * gelu_prime_f(z);
        if (a.train) a.dz3t[(int64_t)(c + e) * a.kpad + row] = __float2bfloat16_rn(g[e]);
      }
      store_row16(sA, r, c, g);
      if (a.train) {
        const int ci = colsum_index(lane);
        const float sw = warp_colsum16(hw, lane);
        const float sb = warp_colsum16(g, lane);
        if ((lane & 1) == 0) {
          red_w4[rg * WID + c + ci] = sw;
          red_b3[rg * WID + c + ci] = sb;
        }
      }
    }
  }
  // ---- dH2 = dZ3 W3 -> TMEM columns 256..511; dZ2 = dH2 * GELU'(Z2) ----
  if (pending) {
    ok = stage_wait(&tbar, tphase, &s_timeout) && ok;
    pending = false;
  }
  if (ok) ok = gemm_128x256(tm + 256, sA, sB, &bar, phase, &s_timeout);
  if (ok) {
    stage_issue(sB, a.w2t, &tbar);
    pending = true;
  }
  if (ok) {
    for (int c = cb; c < ce; c += 16) {
      float dh[16], z[16];
      tmem_row16(lane_base + 256 + c, dh);
      tmem_row16(lane_base + c, z);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        dh[e] *= gelu_prime_f(z[e] + __ldg(P + o.b2 + c + e));
        if (a.train) a.dz2t[(int64_t)(c + e) * a.kpad + row] = __float2bfloat16_rn(dh[e]);
      }
      store_row16(sA, r, c, dh);
      if (a.train) {
        const int ci = colsum_index(lane);
        const float sb = warp_colsum16(dh, lane);
        if ((lane & 1) == 0) red_b2[rg * WID + c + ci] = sb;
      }
    }
  }
  __syncthreads();
  // ---- dH1 = dZ2 W2 -> TMEM columns 0..255; dZ1 = dH1 * GELU'(Z1) ----
  if (pending) {
    ok = stage_wait(&tbar, tphase, &s_timeout) && ok;
    pending = false;
  }
  if (ok) ok = gemm_128x256(tm, sA, sB, &bar, phase, &s_timeout);
  __syncthreads();   // every thread past the MMA wait: sB may now hold dZ1
  float* sdz = reinterpret_cast<float*>(sB);  // 128 x 256 FP32, 16-byte groups XOR-swizzled by row
  float gx[MAXIN];
#pragma unroll
  for (int j = 0; j < MAXIN; ++j) gx[j] = 0.0f;
  if (ok) {
    for (int c = cb; c < ce; c += 16) {
      float dh[16];
      tmem_row16(lane_base + c, dh);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int f = c + e;
        float z = __ldg(P + o.b1 + f);
        float w1[MAXIN];
#pragma unroll
        for (int j = 0; j < MAXIN; ++j) {
          w1[j] = j < in ? __ldg(P + o.W1 + (int64_t)f * in + j) : 0.0f;
          z = fmaf(w1[j], x[j], z);
        }
        dh[e] *= gelu_prime_f(z);
        if (!a.train)
#pragma unroll
          for (int j = 0; j < MAXIN; ++j) gx[j] = fmaf(dh[e], w1[j], gx[j]);
      }
      if (a.train) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int grp = ((c >> 2) + q) ^ (r & 7);
          *reinterpret_cast<float4*>(sdz + r * WID + grp * 4) =
              make_float4(dh[4 * q], dh[4 * q + 1], dh[4 * q + 2], dh[4 * q + 3]);
        }
      }
    }
  }
  if (!a.train) {
    // ds/dx = dZ1 W1: the two halves' partial sums meet in shared memory
    float* sgx = reinterpret_cast<float*>(sB);
    if (hf == 1)
#pragma unroll
      for (int j = 0; j < MAXIN; ++j) sgx[r * MAXIN + j] = gx[j];
    __syncthreads();
    if (hf == 0 && valid && a.dsdx)
#pragma unroll
      for (int j = 0; j < MAXIN; ++j)
        if (j < in) a.dsdx[row * in + j] = gx[j] + sgx[r * MAXIN + j];
  }
  __syncthreads();
  // ---- per-tile partial sums (fixed order) ----
  if (a.train && ok) {
    float* part = a.part + (int64_t)blockIdx.x * po.stride;
    for (int f = t; f < WID; f += MT) {
      part[po.dw4 + f] = ((red_w4[f] + red_w4[WID + f]) + red_w4[2 * WID + f]) + red_w4[3 * WID + f];
      part[po.db3 + f] = ((red_b3[f] + red_b3[WID + f]) + red_b3[2 * WID + f]) + red_b3[3 * WID + f];
      part[po.db2 + f] = ((red_b2[f] + red_b2[WID + f]) + red_b2[2 * WID + f]) + red_b2[3 * WID + f];
      float gw[MAXIN], gb = 0.0f;
#pragma unroll
      for (int j = 0; j < MAXIN; ++j) gw[j] = 0.0f;
      for (int q = 0; q < TILE; ++q) {
        const float dz = sdz[q * WID + (((f >> 2) ^ (q & 7)) << 2) + (f & 3)];
        gb += dz;
#pragma unroll
        for (int j = 0; j < MAXIN; ++j) gw[j] = fmaf(dz, sX[q * MAXIN + j], gw[j]);
      }
      part[po.db1 + f] = gb;
#pragma unroll
      for (int j = 0; j < MAXIN; ++j)
        if (j < in) part[po.dW1 + f * in + j] = gw[j];
    }
    if (t == 0) part[po.loss] = ((s_loss[0] + s_loss[1]) + s_loss[2]) + s_loss[3];
    // db4 = sum of ds over the tile (each row counted once, by warps 0-3)
    float d4 = hf == 0 ? ds : 0.0f;
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) d4 += __shfl_xor_sync(0xffffffffu, d4, sh);
    __syncthreads();
    if (lane == 0) s_loss[warp] = d4;
    __syncthreads();
    if (t == 0) part[po.db4] = ((s_loss[0] + s_loss[1]) + s_loss[2]) + s_loss[3];
  }
  if (s_timeout && t == 0) atomicExch(a.timeout, 1);
  // a timed-out wait: one more bounded wait for the MMAs and copies in flight
  if (s_timeout) umma::mbar_wait(&bar, phase ^ 1u, kWait);
  if (pending) stage_wait(&tbar, tphase, &s_timeout);
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tm, 512);
}

// dW (256 x 256) = dZ^T H over the batch rows [k0, k1) of this split, for
// the output-feature rows [128 m, 128 m + 128): A = dZ^T rows, B = H^T rows,
// both K-major in global memory (feature-major, batch contiguous).
struct WgradArgs {
  const __nv_bfloat16* dzt[2];   // layer 2, layer 3
  const __nv_bfloat16* ht[2];
  int64_t kpad;
  int chunks_per_split;
  int nchunks;
  float* gpart;                  // [2][splits][256][256]
  int splits;
  int* timeout;
};

__global__ void __launch_bounds__(TILE, 1) mlp_wgrad_kernel(WgradArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                    // 128 x 64 BF16 (4 slices)
  unsigned char* sB = smem + TILE * KCH * 2;   // 256 x 64 BF16
  __shared__ uint64_t bar;
  __shared__ uint32_t s_tmem;
  __shared__ int s_timeout;
  const int t = threadIdx.x, warp = t >> 5;
  const int split = blockIdx.x, mt = blockIdx.y, layer = blockIdx.z;
  if (warp == 0) umma::tmem_alloc(&s_tmem, 256);
  if (t == 0) {
    umma::mbar_init(&bar, 1);
    s_timeout = 0;
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tm = s_tmem;
  uint32_t phase = 0;
  const __nv_bfloat16* dzt = a.dzt[layer] + (int64_t)(mt * TILE) * a.kpad;
  const __nv_bfloat16* ht = a.ht[layer];
  const int c0 = split * a.chunks_per_split;
  const int c1 = min(a.nchunks, c0 + a.chunks_per_split);
  bool ok = true;
  int issued = 0;
  for (int ch = c0; ch < c1 && ok; ++ch) {
    const int64_t k0 = (int64_t)ch * KCH;
    // 16-byte pieces: 8 per operand row (64 batch rows)
    for (int i = t; i < TILE * 8; i += TILE) {
      const int r = i >> 3, kq = (i & 7) * 8;
      *reinterpret_cast<uint4*>(sA + tiled_off(r, kq, TILE)) =
          *reinterpret_cast<const uint4*>(dzt + (int64_t)r * a.kpad + k0 + kq);
    }
    for (int i = t; i < WID * 8; i += TILE) {
      const int r = i >> 3, kq = (i & 7) * 8;
      *reinterpret_cast<uint4*>(sB + tiled_off(r, kq, WID)) =
          *reinterpret_cast<const uint4*>(ht + (int64_t)r * a.kpad + k0 + kq);
    }
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();
    if (t == 0) {
      umma::fence_after_sync();
      const uint32_t idesc = umma::idesc_bf16_f32(128, 256);
      const uint32_t a0 = umma::smem_u32(sA), b0 = umma::smem_u32(sB);
#pragma unroll
      for (int kk = 0; kk < KCH / 16; ++kk) {
        const uint64_t ad = umma::smem_desc(a0 + kk * (TILE * 32), 128, 256);
        const uint64_t bd = umma::smem_desc(b0 + kk * (WID * 32), 128, 256);
        umma::mma_bf16(tm, ad, bd, idesc, (issued > 0 || kk > 0) ? 1u : 0u);
      }
      umma::mma_commit(&bar);
    }
    ++issued;
    if (!umma::mbar_wait(&bar, phase, kWait)) s_timeout = 1;
    phase ^= 1u;
    umma::fence_after_sync();
    __syncthreads();   // operands consumed before the next chunk overwrites them
    ok = s_timeout == 0;
  }
  float* out = a.gpart + (((int64_t)layer * a.splits + split) * WID + mt * TILE + t) * WID;
  if (ok) {
    const uint32_t lane_base = tm + ((uint32_t)(32 * warp) << 16);
    for (int c = 0; c < WID; c += 16) {
      float v[16];
      if (issued > 0) {
        tmem_row16(lane_base + c, v);
      } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(out + c + 4 * q) =
            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
  }
  if (s_timeout && t == 0) atomicExch(a.timeout, 1);
  if (s_timeout) umma::mbar_wait(&bar, phase ^ 1u, kWait);
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tm, 256);
}

struct AdamArgs {
  float* p;
  float* m;
  float* v;
  float* g;               // reduced gradient (output)
  const float* part;      // [tiles][stride]
  int tiles;
  const float* gpart;     // [2][splits][256][256]
  int splits;
  int in;
  int apply;              // 0: reduce only; 1: reduce and update
  float lr, beta1, beta2, eps, c1, c2;   // c1 = 1/(1-beta1^t), c2 = 1/(1-beta2^t)
  float inv_K;
  float* loss;            // mean squared error of the batch (device scalar) or NULL
  uint32_t* w2;           // tiled BF16 copies (as 16-bit halves of uint32 words)
  uint32_t* w3;
  uint32_t* w2t;
  uint32_t* w3t;
};

__device__ __forceinline__ void put_bf16(uint32_t* base, uint32_t off, float x) {
  reinterpret_cast<__nv_bfloat16*>(base)[off >> 1] = __float2bfloat16_rn(x);
}

__global__ void mlp_adam_kernel(AdamArgs a) {
  const Off o = offsets(a.in);
  const PartOff po = part_offsets(a.in);
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0 && a.loss) {
    float l = 0.0f;
    for (int i = 0; i < a.tiles; ++i) l += a.part[(int64_t)i * po.stride + po.loss];
    *a.loss = l * a.inv_K;
  }
  if (q >= o.total) return;
  float g = 0.0f;
  int layer = -1, pidx = -1;
  if (q < o.b1) pidx = po.dW1 + (int)q;
  else if (q < o.W2) pidx = po.db1 + (int)(q - o.b1);
  else if (q < o.b2) layer = 0;
  else if (q < o.W3) pidx = po.db2 + (int)(q - o.b2);
  else if (q < o.b3) layer = 1;
  else if (q < o.w4) pidx = po.db3 + (int)(q - o.b3);
  else if (q < o.b4) pidx = po.dw4 + (int)(q - o.w4);
  else pidx = po.db4;
  if (layer >= 0) {
    const int64_t e = q - (layer == 0 ? o.W2 : o.W3);
    for (int s = 0; s < a.splits; ++s) g += a.gpart[((int64_t)layer * a.splits + s) * WID * WID + e];
  } else {
    for (int i = 0; i < a.tiles; ++i) g += a.part[(int64_t)i * po.stride + pidx];
  }
  a.g[q] = g;
  float w = a.p[q];
  if (a.apply) {
    const float m = a.beta1 * a.m[q] + (1.0f - a.beta1) * g;
    const float v = a.beta2 * a.v[q] + (1.0f - a.beta2) * g * g;
    a.m[q] = m;
    a.v[q] = v;
    w -= a.lr * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
    a.p[q] = w;
  }
  if (layer >= 0) {
    const int e = (int)(q - (layer == 0 ? o.W2 : o.W3));
    const int r = e / WID, c = e % WID;   // W[r][c]: output feature r, input feature c
    put_bf16(layer == 0 ? a.w2 : a.w3, tiled_off(r, c, WID), w);
    put_bf16(layer == 0 ? a.w2t : a.w3t, tiled_off(c, r, WID), w);
  }
}

// host-side SplitMix64 (same published definition as the blocking stage)
struct Mix64 {
  uint64_t s;
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  uint64_t below(uint64_t n) {   // Lemire's multiply-and-reject
    unsigned __int128 prod = (unsigned __int128)next() * n;
    uint64_t low = (uint64_t)prod;
    if (low < n) {
      const uint64_t thr = (0 - n) % n;
      while (low < thr) {
        prod = (unsigned __int128)next() * n;
        low = (uint64_t)prod;
      }
    }
    return (uint64_t)(prod >> 64);
  }
};

constexpr size_t fused_smem() { return (size_t)A_BYTES + B_BYTES + (TILE * MAXIN + 12 * WID) * 4; }
// the operands take 48 KB; asking for 80 KB keeps at most two CTAs (2 x 256
// TMEM columns) on an SM, so tcgen05.alloc never waits
constexpr size_t wgrad_smem() { return std::max<size_t>((size_t)(TILE + WID) * KCH * 2, 80 * 1024); }

}  // namespace

struct sbv_mlp {
  sbv_ctx* ctx = nullptr;
  int in = 0;
  int64_t P = 0;
  float* p = nullptr;        // FP32 masters
  float* m = nullptr;        // Adam moments
  float* v = nullptr;
  float* g = nullptr;        // last reduced gradient
  float* loss = nullptr;     // last batch loss (device scalar)
  uint4* wb = nullptr;       // 4 tiled BF16 operands: W2, W3, W2^T, W3^T
  int* timeout = nullptr;
  int adam_t = 0;
  // grow-only scratch
  unsigned char* ops = nullptr;   size_t ops_bytes = 0;    // transposed activations
  float* part = nullptr;          size_t part_bytes = 0;
  float* gpart = nullptr;         size_t gpart_bytes = 0;
  int32_t* idx = nullptr;         size_t idx_bytes = 0;
  // geometry of the last gradient (for the Adam step)
  int last_tiles = 0, last_splits = 0;
  float last_inv_K = 0.0f;
};

namespace {

int grow(sbv_mlp* h, void** p, size_t* have, size_t need) {
  if (*have >= need) return SBV_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc(p, need) != cudaSuccess) {
    cudaGetLastError();
    return fail(h->ctx, SBV_ENOMEM, "surrogate scratch of %zu bytes", need);
  }
  *have = need;
  return SBV_OK;
}

bool g_mlp_ready[64];

int mlp_prepare(sbv_ctx* ctx) {
  if (ctx->device < 64 && g_mlp_ready[ctx->device]) return SBV_OK;
  SBV_CUDA_TRY(ctx, cudaFuncSetAttribute(mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fused_smem()));
  SBV_CUDA_TRY(ctx, cudaFuncSetAttribute(mlp_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)wgrad_smem()));
  if (ctx->device < 64) g_mlp_ready[ctx->device] = true;
  return SBV_OK;
}

// reduce (apply = 0) or reduce + Adam (apply = 1); refreshes the BF16 copies
int enqueue_adam(sbv_mlp* h, int apply, float lr, float b1, float b2, float eps, cudaStream_t s) {
  AdamArgs a;
  memset(&a, 0, sizeof(a));
  a.p = h->p;
  a.m = h->m;
  a.v = h->v;
  a.g = h->g;
  a.part = h->part;
  a.tiles = h->last_tiles;
  a.gpart = h->gpart;
  a.splits = h->last_splits;
  a.in = h->in;
  a.apply = apply;
  a.lr = lr;
  a.beta1 = b1;
  a.beta2 = b2;
  a.eps = eps;
  if (apply) {
    const int t = h->adam_t;
    a.c1 = (float)(1.0 / (1.0 - pow((double)b1, t)));
    a.c2 = (float)(1.0 / (1.0 - pow((double)b2, t)));
  }
  a.inv_K = h->last_inv_K;
  a.loss = h->last_tiles > 0 ? h->loss : nullptr;
  uint32_t* wb = reinterpret_cast<uint32_t*>(h->wb);
  const size_t words = (size_t)B_BYTES / 4;
  a.w2 = wb;
  a.w3 = wb + words;
  a.w2t = wb + 2 * words;
  a.w3t = wb + 3 * words;
  const int threads = 256;
  const int blocks = (int)((h->P + threads - 1) / threads);
  mlp_adam_kernel<<<blocks, threads, 0, s>>>(a);
  SBV_LAUNCH_CHECK(h->ctx, "mlp_adam_kernel");
  return SBV_OK;
}

// fused forward/backward over K rows (train or predict), plus the weight
// gradients when training
int enqueue_pass(sbv_mlp* h, const float* X, const float* tv, const int32_t* idx, int64_t K,
                 int train, float* s_out, float* dsdx, cudaStream_t s) {
  sbv_ctx* ctx = h->ctx;
  int st = mlp_prepare(ctx);
  if (st) return st;
  const int64_t tiles = (K + TILE - 1) / TILE;
  const int64_t kpad = tiles * TILE;
  FusedArgs a;
  memset(&a, 0, sizeof(a));
  a.X = X;
  a.t = tv;
  a.idx = idx;
  a.K = K;
  a.kpad = kpad;
  a.inv_K = 1.0f / (float)K;
  a.in = h->in;
  a.train = train;
  a.p = h->p;
  a.w2 = h->wb;
  a.w3 = h->wb + B_BYTES / 16;
  a.w2t = h->wb + 2 * (B_BYTES / 16);
  a.w3t = h->wb + 3 * (B_BYTES / 16);
  a.s = s_out;
  a.dsdx = dsdx;
  a.timeout = h->timeout;
  const PartOff po = part_offsets(h->in);
  int splits = 0, cps = 0, nchunks = 0;
  if (train) {
    if ((st = grow(h, (void**)&h->ops, &h->ops_bytes, (size_t)4 * WID * kpad * 2))) return st;
    if ((st = grow(h, (void**)&h->part, &h->part_bytes, (size_t)tiles * po.stride * 4))) return st;
    nchunks = (int)(kpad / KCH);
    const int max_splits = std::max(1, ctx->num_sms / 4);
    cps = std::max(1, (nchunks + max_splits - 1) / max_splits);
    splits = (nchunks + cps - 1) / cps;
    if ((st = grow(h, (void**)&h->gpart, &h->gpart_bytes, (size_t)2 * splits * WID * WID * 4)))
      return st;
    __nv_bfloat16* base = reinterpret_cast<__nv_bfloat16*>(h->ops);
    a.h1t = base;
    a.h2t = base + (size_t)WID * kpad;
    a.dz2t = base + (size_t)2 * WID * kpad;
    a.dz3t = base + (size_t)3 * WID * kpad;
    a.part = h->part;
  }
  mlp_fused_kernel<<<(unsigned)tiles, MT, fused_smem(), s>>>(a);
  SBV_LAUNCH_CHECK(ctx, "mlp_fused_kernel");
  if (train) {
    WgradArgs w;
    memset(&w, 0, sizeof(w));
    w.dzt[0] = a.dz2t;
    w.dzt[1] = a.dz3t;
    w.ht[0] = a.h1t;
    w.ht[1] = a.h2t;
    w.kpad = kpad;
    w.chunks_per_split = cps;
    w.nchunks = nchunks;
    w.gpart = h->gpart;
    w.splits = splits;
    w.timeout = h->timeout;
    mlp_wgrad_kernel<<<dim3(splits, 2, 2), TILE, wgrad_smem(), s>>>(w);
    SBV_LAUNCH_CHECK(ctx, "mlp_wgrad_kernel");
    h->last_tiles = (int)tiles;
    h->last_splits = splits;
    h->last_inv_K = a.inv_K;
  }
  return SBV_OK;
}

int check_timeout(sbv_mlp* h, cudaStream_t s) {
  int flag = 0;
  SBV_CUDA_TRY(h->ctx, cudaMemcpyAsync(&flag, h->timeout, sizeof(int), cudaMemcpyDeviceToHost, s));
  SBV_CUDA_TRY(h->ctx, cudaStreamSynchronize(s));
  if (flag) {
    cudaMemsetAsync(h->timeout, 0, sizeof(int), s);
    return fail(h->ctx, SBV_ETIMEOUT, "surrogate kernel: a tensor-core wait gave up");
  }
  return SBV_OK;
}

}  // namespace

extern "C" int64_t sbv_mlp_num_params(int32_t in_dim) {
  if (in_dim < 1 || in_dim > MAXIN) return -1;
  return offsets(in_dim).total;
}

extern "C" void sbv_mlp_destroy(sbv_mlp* h) {
  if (!h) return;
  cudaSetDevice(h->ctx->device);
  cudaDeviceSynchronize();
  void* bufs[] = {h->p, h->m, h->v, h->g, h->loss, h->wb, h->timeout, h->ops, h->part, h->gpart,
                  h->idx};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete h;
}

extern "C" int sbv_mlp_set_params(sbv_mlp* h, const float* params, int64_t n) {
  if (!h) return SBV_EINVAL;
  if (!params || n != h->P) return fail(h->ctx, SBV_EINVAL, "expected %lld parameters", (long long)h->P);
  SBV_CUDA_TRY(h->ctx, cudaSetDevice(h->ctx->device));
  SBV_CUDA_TRY(h->ctx, cudaMemcpy(h->p, params, n * sizeof(float), cudaMemcpyHostToDevice));
  SBV_CUDA_TRY(h->ctx, cudaMemset(h->m, 0, n * sizeof(float)));
  SBV_CUDA_TRY(h->ctx, cudaMemset(h->v, 0, n * sizeof(float)));
  h->adam_t = 0;
  h->last_tiles = 0;
  h->last_splits = 0;
  int st = enqueue_adam(h, 0, 0.f, 0.f, 0.f, 0.f, 0);   // refresh the BF16 copies
  if (st) return st;
  SBV_CUDA_TRY(h->ctx, cudaDeviceSynchronize());
  return SBV_OK;
}

extern "C" int sbv_mlp_get_params(sbv_mlp* h, float* params, int64_t n) {
  if (!h) return SBV_EINVAL;
  if (!params || n != h->P) return fail(h->ctx, SBV_EINVAL, "expected %lld parameters", (long long)h->P);
  SBV_CUDA_TRY(h->ctx, cudaSetDevice(h->ctx->device));
  SBV_CUDA_TRY(h->ctx, cudaDeviceSynchronize());
  SBV_CUDA_TRY(h->ctx, cudaMemcpy(params, h->p, n * sizeof(float), cudaMemcpyDeviceToHost));
  return SBV_OK;
}

extern "C" int sbv_mlp_create(sbv_ctx* ctx, int32_t in_dim, uint64_t seed, sbv_mlp** out) {
  if (!ctx) return SBV_EINVAL;
  if (!out) return fail(ctx, SBV_EINVAL, "out is null");
  *out = nullptr;
  if (in_dim < 1 || in_dim > MAXIN) return fail(ctx, SBV_EINVAL, "in_dim=%d not in [1, %d]", in_dim, MAXIN);
  SBV_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  sbv_mlp* h = new sbv_mlp();
  h->ctx = ctx;
  h->in = in_dim;
  h->P = offsets(in_dim).total;
  const size_t pb = (size_t)h->P * sizeof(float);
  bool okm = cudaMalloc((void**)&h->p, pb) == cudaSuccess && cudaMalloc((void**)&h->m, pb) == cudaSuccess &&
             cudaMalloc((void**)&h->v, pb) == cudaSuccess && cudaMalloc((void**)&h->g, pb) == cudaSuccess &&
             cudaMalloc((void**)&h->loss, sizeof(float)) == cudaSuccess &&
             cudaMalloc((void**)&h->wb, 4 * (size_t)B_BYTES) == cudaSuccess &&
             cudaMalloc((void**)&h->timeout, sizeof(int)) == cudaSuccess;
  if (!okm) {
    cudaGetLastError();
    sbv_mlp_destroy(h);
    return fail(ctx, SBV_ENOMEM, "surrogate parameters");
  }
  cudaMemset(h->timeout, 0, sizeof(int));
  cudaMemset(h->g, 0, pb);
  // Uniform(-a, a), a = 1/sqrt(fan_in), tensors in packed order, one
  // SplitMix64 stream; u = (next >> 11) 2^-53, value (2u - 1) a rounded to FP32
  const Off o = offsets(in_dim);
  std::vector<float> w((size_t)h->P);
  Mix64 rng{seed};
  for (int64_t q = 0; q < h->P; ++q) {
    const int fan = (q < o.b1 || q < o.W2) ? in_dim : WID;
    const double a = 1.0 / sqrt((double)fan);
    const double u = (double)(rng.next() >> 11) * (1.0 / 9007199254740992.0);
    w[q] = (float)((2.0 * u - 1.0) * a);
  }
  int st = sbv_mlp_set_params(h, w.data(), h->P);
  if (st) {
    sbv_mlp_destroy(h);
    return st;
  }
  *out = h;
  return SBV_OK;
}

extern "C" int sbv_mlp_grad(sbv_mlp* h, const float* X, const float* t, int64_t K, float* grads,
                            float* loss, void* stream) {
  if (!h) return SBV_EINVAL;
  if (!X || !t || K < 1) return fail(h->ctx, SBV_EINVAL, "null input or K < 1");
  cudaStream_t s = (cudaStream_t)stream;
  SBV_CUDA_TRY(h->ctx, cudaSetDevice(h->ctx->device));
  int st = enqueue_pass(h, X, t, nullptr, K, 1, nullptr, nullptr, s);
  if (!st) st = enqueue_adam(h, 0, 0.f, 0.f, 0.f, 0.f, s);
  if (st) return st;
  if (grads)
    SBV_CUDA_TRY(h->ctx, cudaMemcpyAsync(grads, h->g, h->P * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (loss) SBV_CUDA_TRY(h->ctx, cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
  return check_timeout(h, s);
}

extern "C" int sbv_mlp_adam(sbv_mlp* h, float lr, float beta1, float beta2, float eps, void* stream) {
  if (!h) return SBV_EINVAL;
  if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return fail(h->ctx, SBV_EINVAL, "bad Adam hyper-parameters");
  if (h->last_tiles == 0) return fail(h->ctx, SBV_EINVAL, "no gradient computed yet");
  SBV_CUDA_TRY(h->ctx, cudaSetDevice(h->ctx->device));
  h->adam_t += 1;
  return enqueue_adam(h, 1, lr, beta1, beta2, eps, (cudaStream_t)stream);
}

extern "C" int sbv_mlp_train(sbv_mlp* h, const float* X, const float* t, int64_t K, int32_t steps,
                             int32_t batch, float lr, uint64_t seed, float* loss_out, void* stream) {
  if (!h) return SBV_EINVAL;
  if (!X || !t || K < 1 || steps < 0 || batch < 1 || !(lr > 0.f))
    return fail(h->ctx, SBV_EINVAL, "bad training arguments");
  cudaStream_t s = (cudaStream_t)stream;
  SBV_CUDA_TRY(h->ctx, cudaSetDevice(h->ctx->device));
  if (steps == 0) return SBV_OK;
  const int64_t bsz = std::min<int64_t>(batch, K);
  // mini-batches: consecutive slices of Fisher-Yates permutations of [0, K),
  // one permutation per pass over the rows, a shorter last slice per pass
  std::vector<int32_t> order;
  std::vector<int64_t> start, len;
  Mix64 rng{seed};
  std::vector<int32_t> perm((size_t)K);
  int64_t pos = K;
  for (int i = 0; i < steps; ++i) {
    if (pos >= K) {
      for (int64_t j = 0; j < K; ++j) perm[j] = (int32_t)j;
      for (int64_t j = 0; j + 1 < K; ++j) std::swap(perm[j], perm[j + (int64_t)rng.below(K - j)]);
      pos = 0;
    }
    const int64_t l = std::min(bsz, K - pos);
    start.push_back((int64_t)order.size());
    len.push_back(l);
    order.insert(order.end(), perm.begin() + pos, perm.begin() + pos + l);
    pos += l;
  }
  int st = grow(h, (void**)&h->idx, &h->idx_bytes, order.size() * sizeof(int32_t));
  if (st) return st;
  SBV_CUDA_TRY(h->ctx, cudaMemcpyAsync(h->idx, order.data(), order.size() * sizeof(int32_t),
                                       cudaMemcpyHostToDevice, s));
  // scratch sized for the largest batch before the first launch
  if ((st = enqueue_pass(h, X, t, h->idx + start[0], len[0], 1, nullptr, nullptr, s))) return st;
  for (int i = 0; i < steps; ++i) {
    if (i > 0 && (st = enqueue_pass(h, X, t, h->idx + start[i], len[i], 1, nullptr, nullptr, s)))
      return st;
    h->adam_t += 1;
    if ((st = enqueue_adam(h, 1, lr, 0.9f, 0.999f, 1e-8f, s))) return st;
  }
  if (loss_out)
    SBV_CUDA_TRY(h->ctx, cudaMemcpyAsync(loss_out, h->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
  return check_timeout(h, s);   // also keeps `order` alive until the copy has run
}

extern "C" int sbv_mlp_predict(sbv_mlp* h, const float* X, int64_t K, float* s_out, float* dsdx,
                               void* stream) {
  if (!h) return SBV_EINVAL;
  if (!X || !s_out || K < 1) return fail(h->ctx, SBV_EINVAL, "null input or K < 1");
  cudaStream_t s = (cudaStream_t)stream;
  SBV_CUDA_TRY(h->ctx, cudaSetDevice(h->ctx->device));
  int st = enqueue_pass(h, X, nullptr, nullptr, K, 0, s_out, dsdx, s);
  if (st) return st;
  return check_timeout(h, s);
}
