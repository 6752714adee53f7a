// Internal declarations shared by the translation units of libsbv.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string>
#include <vector>

#include "sbv.h"

namespace sbv {

// Device-side error record written by kernels (first failure wins).
struct DevStatus {
  int32_t code;      // 0 or SBV_ENOTSPD / SBV_ETIMEOUT
  int32_t item;      // block or test-point index of the first failure
  int32_t theta;     // parameter row of the first failure
  int32_t count;     // number of failures
  int32_t reruns;    // items the mixed kernels handed to the FP64 kernels
  int32_t pad[3];
};

// Grow-only device buffer owned by the context.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Launch shape of the block kernels: threads per CTA and resident CTAs per SM.
struct LaunchShape {
  int threads = 0;  // 0: no forced shape
  int per_sm = 0;
  int tile = 0;     // mixed kernels: right-hand sides per column block (0: as many as fit)
};

// Autotuning record: the fastest shape measured for one kind of launch.
struct TunedShape {
  int precision, pred, ncap, d;
  int threads, per_sm, tile;
};

// Named device workspace slots of a context (grow-only buffers).
enum WsSlot {
  WS_Z = 0,       // scaled coordinates
  WS_SORT_A,      // sort keys / values
  WS_SORT_B,
  WS_SORT_C,
  WS_SORT_D,
  WS_CUB,         // cub temporary storage
  WS_SMALL,       // counters, flags
  WS_PARAMS,      // per-theta derived parameters
  WS_TERMS,       // block terms when the caller passes NULL
  WS_ORDER,       // rank-ordered point list
  WS_MATRIX,      // global-memory matrices for blocks too large for shared memory
  WS_CENTRES,
  WS_EXTRA,
  WS_XSPLIT,      // points split into float pairs for the mixed path
  WS_TUNE,        // results of the autotuner's timing runs
  WS_PRED,        // prediction neighbour lists when the caller passes NULL
  WS_GRAD,        // per-block gradients when the caller passes NULL
  WS_GRADZ,       // per-CTA right-hand sides of the gradient kernel
  WS_RERUN,       // items the mixed kernels hand to the FP64 kernels
  WS_GMAT64,      // global matrices of the FP64 kernel after a mixed launch
  WS_TBLK,        // blocking of the test points (block prediction)
  WS_BOUNDS,      // distance bounds and point list of the bounded K-means assignment
  WS_COUNT
};

}  // namespace sbv

struct sbv_ctx {
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  std::string err;
  sbv::DevStatus* d_status = nullptr;  // device record
  sbv::DevBuf ws[sbv::WS_COUNT];       // named workspace slots
  sbv::LaunchShape force;              // set while the autotuner times a shape
  std::vector<sbv::TunedShape> tuned;  // autotuning records
  int knn_mode = 0;                    // 0 automatic, 1 brute force, 2 pruned search
  // largest block sizes last read for a structure (ptr, cnt, bc): calls with a
  // size hint reuse bsmax for the same arrays (a stale value only makes the
  // mixed kernel hand the oversized items to the FP64 kernel)
  const void* sz_ptr = nullptr;
  const void* sz_cnt = nullptr;
  int64_t sz_bc = 0;
  int sz_nmax = 0, sz_bsmax = 0;
  // pinned host ring for parameter rows: slot k is reused only after the
  // event recorded behind its previous copy has completed
  static const int kRing = 8;
  unsigned char* h_ring = nullptr;
  size_t ring_slot = 0;
  cudaEvent_t ring_ev[kRing] = {};
  int ring_next = 0;
};

namespace sbv {

int fail(sbv_ctx* ctx, int code, const char* fmt, ...);
int cuda_fail(sbv_ctx* ctx, cudaError_t e, const char* where);
void* ws_get(sbv_ctx* ctx, int slot, size_t bytes, int* status);

#define SBV_CUDA_TRY(ctx, call)                                     \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return ::sbv::cuda_fail(ctx, e_, #call); \
  } while (0)

#define SBV_LAUNCH_CHECK(ctx, what)                                 \
  do {                                                              \
    cudaError_t e_ = cudaGetLastError();                            \
    if (e_ != cudaSuccess) return ::sbv::cuda_fail(ctx, e_, what);  \
  } while (0)

// ---- launchers implemented in the .cu files ----
// scaling / blocking
int scale_points(sbv_ctx* ctx, const void* X, int dtype, int64_t n, int d,
                 const double* d_inv_unused, const double* h_beta, double* Z,
                 cudaStream_t s);
int run_blocking(sbv_ctx* ctx, const double* Z, const void* X, int dtype, const double* h_beta,
                 int64_t n, int d, int64_t bc, int kmeans_iters, uint64_t seed, int partitions,
                 int32_t* blk, int64_t* ptr, int32_t* pts, int32_t* rank, double* centres,
                 int64_t* bc_eff, cudaStream_t s, const int64_t* h_anchors = nullptr);
// kNN
int run_slabs(sbv_ctx* ctx, const void* X, int dtype, int64_t n, int d, const double* h_beta,
              int P, int32_t* slab, cudaStream_t s);
int rac_plan(uint64_t seed, int P, const int64_t* counts, int64_t bc, int64_t* quota,
             int64_t* pos, int64_t k_eff, int32_t* rank);
int run_knn(sbv_ctx* ctx, const double* Z, int64_t n, int d, const int64_t* ptr,
            const int32_t* pts, const int32_t* rank, const double* centres,
            int64_t bc, int m, int32_t* nbr, int32_t* cnt, cudaStream_t s);
int run_knn_all(sbv_ctx* ctx, const double* Z, int64_t n, int d,
                const double* Q, int64_t nq, int m, int32_t* nbr, cudaStream_t s);
int run_knn_blocks_all(sbv_ctx* ctx, const double* Z, int64_t n, int d, const int64_t* ptr,
                       const int32_t* pts, const int32_t* rank, const double* centres,
                       int64_t bc, const double* Q, int64_t nq, int m, int32_t* nbr,
                       cudaStream_t s);
// likelihood and prediction
int run_max_sizes(sbv_ctx* ctx, const int64_t* ptr, const int32_t* cnt, int64_t bc, int* nmax,
                  int* bsmax, cudaStream_t s);
int run_loglik(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n,
               int d, const int64_t* ptr, const int32_t* pts, const int32_t* nbr,
               const int32_t* cnt, int64_t bc, int m, int nmax, const double* h_theta,
               int B, int nu2, int precision, double* ll, double* terms, int32_t* status,
               cudaStream_t s);
int run_loglik_grad(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n, int d,
                    const int64_t* ptr, const int32_t* pts, const int32_t* nbr,
                    const int32_t* cnt, int64_t bc, int m, int nmax_hint, const double* h_theta,
                    int B, int nu2, double* ll, double* grad, double* terms, double* gterms,
                    int32_t* status, cudaStream_t s);
// covariance function alone (FP64 or double-float arithmetic of the likelihood)
int run_matern(sbv_ctx* ctx, int precision, int nu2, const double* d2, int64_t n, double* out,
               cudaStream_t s);
int run_matern_df(sbv_ctx* ctx, int nu2, const double* d2, int64_t n, double* out,
                  cudaStream_t s);
// conditional simulation from predictive means and variances
int run_simulate(sbv_ctx* ctx, const double* mean, const double* var, int64_t nt, int ndraws,
                 uint64_t seed, uint64_t base, double* mu, double* var_s, double* lo, double* hi,
                 double* draws, cudaStream_t s);
int run_predict(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n,
                int d, const void* Xt, int64_t nt, const int32_t* nbr, int m,
                const double* h_theta, int nu2, int precision, double* mean,
                double* var, double* var_latent, cudaStream_t s,
                const int64_t* tptr = nullptr, const int32_t* tpts = nullptr, int bsmax = 1);

}  // namespace sbv
