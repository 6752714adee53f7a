// C ABI of libsbv.so: contexts, argument checks, workspace, and the entry
// points declared in include/sbv.h.  Every computation is delegated to the
// CUDA kernels of the other translation units.
#include <stdarg.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sbv_internal.cuh"

namespace sbv {

int fail(sbv_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

int cuda_fail(sbv_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, SBV_ECUDA, "%s: %s (%s)", where, cudaGetErrorName(e),
              cudaGetErrorString(e));
}

void* ws_get(sbv_ctx* ctx, int slot, size_t bytes, int* status) {
  DevBuf& b = ctx->ws[slot];
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return b.p;
  if (b.p) {
    cudaDeviceSynchronize();
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  size_t want = bytes + bytes / 8;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *status = fail(ctx, SBV_ENOMEM, "workspace allocation of %zu bytes failed: %s", want,
                   cudaGetErrorString(e));
    return nullptr;
  }
  b.bytes = want;
  return b.p;
}

}  // namespace sbv

using namespace sbv;

extern "C" int sbv_version(void) { return 100; }

extern "C" int sbv_create(sbv_ctx** out, int device) {
  if (!out) return SBV_EINVAL;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return SBV_ECUDA;
  if (device < 0 || device >= ndev) return SBV_EINVAL;
  sbv_ctx* ctx = new sbv_ctx();
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete ctx;
    return SBV_ECUDA;
  }
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  ctx->smem_optin = (size_t)optin;
  if (cudaMalloc(&ctx->d_status, sizeof(DevStatus)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(DevStatus)) != cudaSuccess) {
    delete ctx;
    return SBV_ENOMEM;
  }
  *out = ctx;
  return SBV_OK;
}

extern "C" void sbv_destroy(sbv_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto& b : ctx->ws)
    if (b.p) cudaFree(b.p);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->h_ring) cudaFreeHost(ctx->h_ring);
  for (auto& e : ctx->ring_ev)
    if (e) cudaEventDestroy(e);
  delete ctx;
}

extern "C" const char* sbv_last_error(const sbv_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

static int check_common(sbv_ctx* ctx, const void* X, int dtype, int64_t n, int32_t d) {
  if (!ctx) return SBV_EINVAL;
  if (!X) return fail(ctx, SBV_EINVAL, "X is null");
  if (dtype != SBV_F64 && dtype != SBV_F32) return fail(ctx, SBV_EINVAL, "bad dtype %d", dtype);
  if (n < 1 || n > (int64_t)INT32_MAX - 1) return fail(ctx, SBV_EINVAL, "n=%lld out of range", (long long)n);
  if (d < 1 || d > SBV_MAX_DIM) return fail(ctx, SBV_EINVAL, "d=%d outside [1,%d]", d, SBV_MAX_DIM);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, SBV_ECUDA, "cudaSetDevice failed");
  return SBV_OK;
}

static int check_beta(sbv_ctx* ctx, const double* beta, int d, const char* name) {
  if (!beta) return fail(ctx, SBV_EINVAL, "%s is null", name);
  for (int t = 0; t < d; ++t)
    if (!(beta[t] > 0.0) || !isfinite(beta[t]))
      return fail(ctx, SBV_EINVAL, "%s[%d]=%g must be positive and finite", name, t, beta[t]);
  return SBV_OK;
}

static int check_theta(sbv_ctx* ctx, const double* theta, int B, int d) {
  if (!theta) return fail(ctx, SBV_EINVAL, "theta is null");
  if (B < 1) return fail(ctx, SBV_EINVAL, "B=%d must be >= 1", B);
  for (int b = 0; b < B; ++b) {
    const double* r = theta + (size_t)b * (2 + d);
    if (!(r[0] > 0.0) || !isfinite(r[0]))
      return fail(ctx, SBV_EINVAL, "theta[%d]: sigma^2=%g must be positive", b, r[0]);
    if (!(r[1] >= 0.0) || !isfinite(r[1]))
      return fail(ctx, SBV_EINVAL, "theta[%d]: tau^2=%g must be >= 0", b, r[1]);
    for (int t = 0; t < d; ++t)
      if (!(r[2 + t] > 0.0) || !isfinite(r[2 + t]))
        return fail(ctx, SBV_EINVAL, "theta[%d]: beta_%d=%g must be positive", b, t + 1, r[2 + t]);
  }
  return SBV_OK;
}

// 2 nu: the mixed precisions evaluate the four closed forms in double-float;
// the FP64 paths also take any other nu = nu2 / 2 <= 20 through K_nu
static bool nu_ok(int nu2) { return nu2 == 1 || nu2 == 3 || nu2 == 5 || nu2 == 7; }
static bool nu_ok_prec(int nu2, int precision) {
  return precision == SBV_PREC_FP64 ? (nu2 >= 1 && nu2 <= SBV_MAX_NU2) : nu_ok(nu2);
}

extern "C" int sbv_blocking_partitioned(sbv_ctx* ctx, const void* X, int dtype, int64_t n,
                                        int32_t d, const double* beta_scale, int64_t bc,
                                        int32_t kmeans_iters, uint64_t seed, int32_t partitions,
                                        int32_t* blk, int64_t* ptr, int32_t* pts, int32_t* rank,
                                        double* centres, int64_t* bc_eff, void* stream) {
  int st = check_common(ctx, X, dtype, n, d);
  if (st) return st;
  if ((st = check_beta(ctx, beta_scale, d, "beta_scale"))) return st;
  if (bc < 1 || bc > n) return fail(ctx, SBV_EINVAL, "bc=%lld outside [1, n]", (long long)bc);
  if (kmeans_iters < 0) return fail(ctx, SBV_EINVAL, "kmeans_iters must be >= 0");
  if (partitions < 1 || (int64_t)partitions > bc)
    return fail(ctx, SBV_EINVAL, "partitions=%d outside [1, bc]", partitions);
  if (!blk || !ptr || !pts || !rank || !centres || !bc_eff)
    return fail(ctx, SBV_EINVAL, "null output pointer");
  cudaStream_t s = (cudaStream_t)stream;
  double* Z = (double*)ws_get(ctx, WS_Z, (size_t)n * d * sizeof(double), &st);
  if (!Z) return st;
  if ((st = scale_points(ctx, X, dtype, n, d, nullptr, beta_scale, Z, s))) return st;
  return run_blocking(ctx, Z, X, dtype, beta_scale, n, d, bc, kmeans_iters, seed, partitions, blk,
                      ptr, pts, rank, centres, bc_eff, s);
}

extern "C" int sbv_blocking(sbv_ctx* ctx, const void* X, int dtype, int64_t n, int32_t d,
                            const double* beta_scale, int64_t bc, int32_t kmeans_iters,
                            uint64_t seed, int32_t* blk, int64_t* ptr, int32_t* pts,
                            int32_t* rank, double* centres, int64_t* bc_eff, void* stream) {
  return sbv_blocking_partitioned(ctx, X, dtype, n, d, beta_scale, bc, kmeans_iters, seed, 1,
                                  blk, ptr, pts, rank, centres, bc_eff, stream);
}

extern "C" int sbv_slabs(sbv_ctx* ctx, const void* X, int dtype, int64_t n, int32_t d,
                         const double* beta_scale, int32_t partitions, int32_t* slab,
                         void* stream) {
  if (ctx && n == 0) return SBV_OK;
  int st = check_common(ctx, X, dtype, n, d);
  if (st) return st;
  if ((st = check_beta(ctx, beta_scale, d, "beta_scale"))) return st;
  if (partitions < 1) return fail(ctx, SBV_EINVAL, "partitions=%d must be >= 1", partitions);
  if (!slab) return fail(ctx, SBV_EINVAL, "null output pointer");
  return run_slabs(ctx, X, dtype, n, d, beta_scale, partitions, slab, (cudaStream_t)stream);
}

extern "C" int sbv_rac_plan(uint64_t seed, int32_t partitions, const int64_t* slab_counts,
                            int64_t bc, int64_t* quota, int64_t* anchor_pos, int64_t bc_eff,
                            int32_t* rank) {
  if (partitions < 1 || !slab_counts) return SBV_EINVAL;
  int64_t n = 0;
  for (int q = 0; q < partitions; ++q) {
    if (slab_counts[q] < 0) return SBV_EINVAL;
    n += slab_counts[q];
  }
  if (n < 1 || bc < 1 || bc > n || (int64_t)partitions > bc) return SBV_EINVAL;
  if (rank && (bc_eff < 1 || bc_eff > bc)) return SBV_EINVAL;
  return rac_plan(seed, partitions, slab_counts, bc, quota, anchor_pos, rank ? bc_eff : 0, rank);
}

extern "C" int sbv_blocking_anchored(sbv_ctx* ctx, const void* X, int dtype, int64_t n, int32_t d,
                                     const double* beta_scale, const int64_t* anchors, int64_t k,
                                     int32_t kmeans_iters, int32_t* blk, int64_t* ptr,
                                     int32_t* pts, double* centres, int64_t* bc_eff,
                                     void* stream) {
  int st = check_common(ctx, X, dtype, n, d);
  if (st) return st;
  if ((st = check_beta(ctx, beta_scale, d, "beta_scale"))) return st;
  if (k < 1 || k > n) return fail(ctx, SBV_EINVAL, "k=%lld outside [1, n]", (long long)k);
  if (kmeans_iters < 0) return fail(ctx, SBV_EINVAL, "kmeans_iters must be >= 0");
  if (!anchors || !blk || !ptr || !pts || !centres || !bc_eff)
    return fail(ctx, SBV_EINVAL, "null pointer argument");
  {
    std::vector<int64_t> a(anchors, anchors + k);
    std::sort(a.begin(), a.end());
    for (int64_t j = 0; j < k; ++j) {
      if (a[j] < 0 || a[j] >= n)
        return fail(ctx, SBV_EINVAL, "anchor %lld outside [0, n)", (long long)a[j]);
      if (j > 0 && a[j] == a[j - 1])
        return fail(ctx, SBV_EINVAL, "anchor %lld repeated", (long long)a[j]);
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* Z = (double*)ws_get(ctx, WS_Z, (size_t)n * d * sizeof(double), &st);
  if (!Z) return st;
  if ((st = scale_points(ctx, X, dtype, n, d, nullptr, beta_scale, Z, s))) return st;
  return run_blocking(ctx, Z, X, dtype, beta_scale, n, d, k, kmeans_iters, 0, 1, blk, ptr, pts,
                      nullptr, centres, bc_eff, s, anchors);
}

extern "C" int sbv_set_knn_mode(sbv_ctx* ctx, int32_t mode) {
  if (!ctx) return SBV_EINVAL;
  if (mode < 0 || mode > 2) return fail(ctx, SBV_EINVAL, "knn mode %d not in {0, 1, 2}", mode);
  ctx->knn_mode = mode;
  return SBV_OK;
}

extern "C" int sbv_knn(sbv_ctx* ctx, const void* X, int dtype, int64_t n, int32_t d,
                       const double* beta_scale, const int64_t* ptr, const int32_t* pts,
                       const int32_t* rank, const double* centres, int64_t bc, int32_t m,
                       int32_t* nbr, int32_t* cnt, void* stream) {
  int st = check_common(ctx, X, dtype, n, d);
  if (st) return st;
  if ((st = check_beta(ctx, beta_scale, d, "beta_scale"))) return st;
  if (bc < 1 || bc > n) return fail(ctx, SBV_EINVAL, "bc=%lld outside [1, n]", (long long)bc);
  if (m < 0) return fail(ctx, SBV_EINVAL, "m=%d must be >= 0", m);
  if (m > SBV_MAX_BLOCK_N - 1) return fail(ctx, SBV_EUNSUPPORTED, "m=%d above %d", m, SBV_MAX_BLOCK_N - 1);
  if (!ptr || !pts || !rank || !centres || !cnt || (m > 0 && !nbr))
    return fail(ctx, SBV_EINVAL, "null pointer argument");
  cudaStream_t s = (cudaStream_t)stream;
  double* Z = (double*)ws_get(ctx, WS_Z, (size_t)n * d * sizeof(double), &st);
  if (!Z) return st;
  if ((st = scale_points(ctx, X, dtype, n, d, nullptr, beta_scale, Z, s))) return st;
  return run_knn(ctx, Z, n, d, ptr, pts, rank, centres, bc, m, nbr, cnt, s);
}

extern "C" int sbv_loglik(sbv_ctx* ctx, const void* X, int dtype, const double* y,
                          int64_t n, int32_t d, const int64_t* ptr, const int32_t* pts,
                          const int32_t* nbr, const int32_t* cnt, int64_t bc, int32_t m,
                          int32_t nmax, const double* theta, int32_t B, int32_t nu2,
                          int32_t precision, double* ll, double* block_terms,
                          int32_t* status, void* stream) {
  int st = check_common(ctx, X, dtype, n, d);
  if (st) return st;
  if (!y || !ptr || !pts || !cnt || !ll || (m > 0 && !nbr))
    return fail(ctx, SBV_EINVAL, "null pointer argument");
  if (bc < 1 || bc > n) return fail(ctx, SBV_EINVAL, "bc=%lld outside [1, n]", (long long)bc);
  if (m < 0) return fail(ctx, SBV_EINVAL, "m=%d must be >= 0", m);
  if ((st = check_theta(ctx, theta, B, d))) return st;
  if (precision != SBV_PREC_FP64 && precision != SBV_PREC_MIXED &&
      precision != SBV_PREC_MIXED_BF16)
    return fail(ctx, SBV_EINVAL, "precision=%d unknown", precision);
  if (!nu_ok_prec(nu2, precision))
    return fail(ctx, SBV_EINVAL, "nu2=%d: FP64 takes 1..%d, the mixed precisions {1,3,5,7}", nu2,
                SBV_MAX_NU2);
  if (nmax < 0) return fail(ctx, SBV_EINVAL, "nmax=%d must be >= 0", nmax);
  return run_loglik(ctx, X, dtype, y, n, d, ptr, pts, nbr, cnt, bc, m, nmax, theta, B, nu2,
                    precision, ll, block_terms, status, (cudaStream_t)stream);
}

extern "C" int sbv_loglik_grad(sbv_ctx* ctx, const void* X, int dtype, const double* y,
                               int64_t n, int32_t d, const int64_t* ptr, const int32_t* pts,
                               const int32_t* nbr, const int32_t* cnt, int64_t bc, int32_t m,
                               int32_t nmax, const double* theta, int32_t B, int32_t nu2,
                               double* ll, double* grad, double* block_terms,
                               double* block_grads, int32_t* status, void* stream) {
  int st = check_common(ctx, X, dtype, n, d);
  if (st) return st;
  if (!y || !ptr || !pts || !cnt || !ll || !grad || (m > 0 && !nbr))
    return fail(ctx, SBV_EINVAL, "null pointer argument");
  if (bc < 1 || bc > n) return fail(ctx, SBV_EINVAL, "bc=%lld outside [1, n]", (long long)bc);
  if (m < 0) return fail(ctx, SBV_EINVAL, "m=%d must be >= 0", m);
  if ((st = check_theta(ctx, theta, B, d))) return st;
  if (!nu_ok_prec(nu2, SBV_PREC_FP64))
    return fail(ctx, SBV_EINVAL, "nu2=%d outside 1..%d", nu2, SBV_MAX_NU2);
  if (nmax < 0) return fail(ctx, SBV_EINVAL, "nmax=%d must be >= 0", nmax);
  return run_loglik_grad(ctx, X, dtype, y, n, d, ptr, pts, nbr, cnt, bc, m, nmax, theta, B, nu2,
                         ll, grad, block_terms, block_grads, status, (cudaStream_t)stream);
}

extern "C" int sbv_sync_status(sbv_ctx* ctx, void* stream) {
  if (!ctx) return SBV_EINVAL;
  cudaSetDevice(ctx->device);
  DevStatus h;
  cudaStream_t s = (cudaStream_t)stream;
  SBV_CUDA_TRY(ctx, cudaMemcpyAsync(&h, ctx->d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  SBV_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(DevStatus), s));
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (h.code == SBV_ENOTSPD)
    return fail(ctx, SBV_ENOTSPD,
                "%d matrices not positive definite; first: item %d of parameter row %d",
                h.count, h.item, h.theta);
  if (h.code != 0)
    return fail(ctx, h.code, "device reported code %d at item %d", h.code, h.item);
  return SBV_OK;
}

extern "C" int sbv_fp64_reruns(sbv_ctx* ctx, void* stream, int64_t* count) {
  if (!ctx || !count) return SBV_EINVAL;
  cudaSetDevice(ctx->device);
  DevStatus h;
  cudaStream_t s = (cudaStream_t)stream;
  SBV_CUDA_TRY(ctx, cudaMemcpyAsync(&h, ctx->d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  *count = h.reruns;
  return SBV_OK;
}

static int predict_common(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n,
                          int32_t d, const void* Xtest, int64_t ntest, const double* beta_scale,
                          int32_t m_pred, const double* theta, int32_t nu2, int32_t precision,
                          const int64_t* ptr, const int32_t* pts, const int32_t* rank,
                          const double* centres, int64_t bc, double* mean, double* var,
                          double* var_latent, int32_t* nbr, void* stream) {
  int st = check_common(ctx, X, dtype, n, d);
  if (st) return st;
  if (!y || !Xtest || !mean || !var || !var_latent)
    return fail(ctx, SBV_EINVAL, "null pointer argument");
  if (ntest < 1 || ntest > (int64_t)INT32_MAX - 1) return fail(ctx, SBV_EINVAL, "ntest out of range");
  if ((st = check_beta(ctx, beta_scale, d, "beta_scale"))) return st;
  if (m_pred < 1 || m_pred > n) return fail(ctx, SBV_EINVAL, "m_pred=%d outside [1, n]", m_pred);
  if (m_pred > SBV_MAX_BLOCK_N - 1)
    return fail(ctx, SBV_EUNSUPPORTED, "m_pred=%d above %d", m_pred, SBV_MAX_BLOCK_N - 1);
  if ((st = check_theta(ctx, theta, 1, d))) return st;
  if (precision != SBV_PREC_FP64 && precision != SBV_PREC_MIXED &&
      precision != SBV_PREC_MIXED_BF16)
    return fail(ctx, SBV_EINVAL, "precision=%d unknown", precision);
  if (!nu_ok_prec(nu2, precision))
    return fail(ctx, SBV_EINVAL, "nu2=%d: FP64 takes 1..%d, the mixed precisions {1,3,5,7}", nu2,
                SBV_MAX_NU2);
  if (ptr && (!pts || !rank || !centres || bc < 1 || bc > n))
    return fail(ctx, SBV_EINVAL, "incomplete block structure");
  cudaStream_t s = (cudaStream_t)stream;
  size_t zbytes = (size_t)(n + ntest) * d * sizeof(double);
  double* Z = (double*)ws_get(ctx, WS_Z, zbytes, &st);
  if (!Z) return st;
  double* Zt = Z + (size_t)n * d;
  if ((st = scale_points(ctx, X, dtype, n, d, nullptr, beta_scale, Z, s))) return st;
  if ((st = scale_points(ctx, Xtest, dtype, ntest, d, nullptr, beta_scale, Zt, s))) return st;
  int32_t* knbr = nbr;
  if (!knbr) {
    knbr = (int32_t*)ws_get(ctx, WS_PRED, (size_t)ntest * m_pred * sizeof(int32_t), &st);
    if (!knbr) return st;
  }
  if (ptr)
    st = run_knn_blocks_all(ctx, Z, n, d, ptr, pts, rank, centres, bc, Zt, ntest, m_pred, knbr, s);
  else
    st = run_knn_all(ctx, Z, n, d, Zt, ntest, m_pred, knbr, s);
  if (st) return st;
  if ((st = run_predict(ctx, X, dtype, y, n, d, Xtest, ntest, knbr, m_pred, theta, nu2,
                        precision, mean, var, var_latent, s)))
    return st;
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  return sbv_sync_status(ctx, stream);
}

extern "C" int sbv_predict_blocks(sbv_ctx* ctx, const void* X, int dtype, const double* y,
                                  int64_t n, int32_t d, const void* Xtest, int64_t ntest,
                                  const double* beta_scale, int32_t m_pred, const double* theta,
                                  int32_t nu2, int32_t precision, const int64_t* ptr,
                                  const int32_t* pts, const int32_t* rank, const double* centres,
                                  int64_t bc, double* mean, double* var, double* var_latent,
                                  int32_t* nbr, void* stream) {
  if (ctx && !ptr) return fail(ctx, SBV_EINVAL, "ptr is null");
  return predict_common(ctx, X, dtype, y, n, d, Xtest, ntest, beta_scale, m_pred, theta, nu2,
                        precision, ptr, pts, rank, centres, bc, mean, var, var_latent, nbr, stream);
}

extern "C" int sbv_predict(sbv_ctx* ctx, const void* X, int dtype, const double* y,
                           int64_t n, int32_t d, const void* Xtest, int64_t ntest,
                           const double* beta_scale, int32_t m_pred, const double* theta,
                           int32_t nu2, int32_t precision, double* mean, double* var,
                           double* var_latent, int32_t* nbr, void* stream) {
  return predict_common(ctx, X, dtype, y, n, d, Xtest, ntest, beta_scale, m_pred, theta, nu2,
                        precision, nullptr, nullptr, nullptr, nullptr, 0, mean, var, var_latent,
                        nbr, stream);
}

extern "C" int sbv_predict_blocked(sbv_ctx* ctx, const void* X, int dtype, const double* y,
                                   int64_t n, int32_t d, const void* Xtest, int64_t ntest,
                                   const double* beta_scale, int32_t m_pred, int64_t bc_test,
                                   int32_t kmeans_iters, uint64_t seed, const double* theta,
                                   int32_t nu2, int32_t precision, const int64_t* ptr,
                                   const int32_t* pts, const int32_t* rank,
                                   const double* centres, int64_t bc, double* mean, double* var,
                                   double* var_latent, int32_t* test_block, int32_t* nbr,
                                   int64_t* bc_test_eff, void* stream) {
  int st = check_common(ctx, X, dtype, n, d);
  if (st) return st;
  if (!y || !Xtest || !mean || !var || !var_latent)
    return fail(ctx, SBV_EINVAL, "null pointer argument");
  if (ntest < 1 || ntest > (int64_t)INT32_MAX - 1) return fail(ctx, SBV_EINVAL, "ntest out of range");
  if ((st = check_beta(ctx, beta_scale, d, "beta_scale"))) return st;
  if (m_pred < 1 || m_pred > n) return fail(ctx, SBV_EINVAL, "m_pred=%d outside [1, n]", m_pred);
  if (bc_test < 1 || bc_test > ntest)
    return fail(ctx, SBV_EINVAL, "bc_test=%lld outside [1, ntest]", (long long)bc_test);
  if (kmeans_iters < 0) return fail(ctx, SBV_EINVAL, "kmeans_iters must be >= 0");
  if ((st = check_theta(ctx, theta, 1, d))) return st;
  if (precision != SBV_PREC_FP64 && precision != SBV_PREC_MIXED &&
      precision != SBV_PREC_MIXED_BF16)
    return fail(ctx, SBV_EINVAL, "precision=%d unknown", precision);
  if (!nu_ok_prec(nu2, precision))
    return fail(ctx, SBV_EINVAL, "nu2=%d: FP64 takes 1..%d, the mixed precisions {1,3,5,7}", nu2,
                SBV_MAX_NU2);
  if (ptr && (!pts || !rank || !centres || bc < 1 || bc > n))
    return fail(ctx, SBV_EINVAL, "incomplete block structure");
  cudaStream_t s = (cudaStream_t)stream;
  SBV_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  size_t zbytes = (size_t)(n + ntest) * d * sizeof(double);
  double* Z = (double*)ws_get(ctx, WS_Z, zbytes, &st);
  if (!Z) return st;
  double* Zt = Z + (size_t)n * d;
  if ((st = scale_points(ctx, X, dtype, n, d, nullptr, beta_scale, Z, s))) return st;
  if ((st = scale_points(ctx, Xtest, dtype, ntest, d, nullptr, beta_scale, Zt, s))) return st;
  // blocks of test points (RAC + Lloyd in the same scaled space)
  const size_t tb_bytes = (size_t)ntest * 2 * sizeof(int32_t) + (size_t)(bc_test + 1) * 8 +
                          (size_t)bc_test * d * sizeof(double) + 256;
  char* tw = (char*)ws_get(ctx, WS_TBLK, tb_bytes, &st);
  if (!tw) return st;
  double* tcent = (double*)tw;
  int64_t* tptr = (int64_t*)(tcent + (size_t)bc_test * d);
  int32_t* tpts = (int32_t*)(tptr + bc_test + 1);
  int32_t* tblk = tpts + ntest;
  int64_t kt = 0;
  if ((st = run_blocking(ctx, Zt, Xtest, dtype, beta_scale, ntest, d, bc_test, kmeans_iters, seed,
                         1, tblk, tptr, tpts, nullptr, tcent, &kt, s)))
    return st;
  // m_pred nearest training points of every test block's centre
  int32_t* knbr = nbr;
  if (!knbr) {
    knbr = (int32_t*)ws_get(ctx, WS_PRED, (size_t)kt * m_pred * sizeof(int32_t), &st);
    if (!knbr) return st;
  }
  if (ptr)
    st = run_knn_blocks_all(ctx, Z, n, d, ptr, pts, rank, centres, bc, tcent, kt, m_pred, knbr, s);
  else
    st = run_knn_all(ctx, Z, n, d, tcent, kt, m_pred, knbr, s);
  if (st) return st;
  std::vector<int64_t> hptr((size_t)kt + 1);
  SBV_CUDA_TRY(ctx, cudaMemcpyAsync(hptr.data(), tptr, (kt + 1) * sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, s));
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  int bsmax = 1;
  for (int64_t b = 0; b < kt; ++b) bsmax = std::max<int>(bsmax, (int)(hptr[b + 1] - hptr[b]));
  if (m_pred + bsmax > SBV_MAX_BLOCK_N)
    return fail(ctx, SBV_EUNSUPPORTED, "m_pred + largest test block = %d above %d",
                m_pred + bsmax, SBV_MAX_BLOCK_N);
  if ((st = run_predict(ctx, X, dtype, y, n, d, Xtest, kt, knbr, m_pred, theta, nu2, precision,
                        mean, var, var_latent, s, tptr, tpts, bsmax)))
    return st;
  if (test_block)
    SBV_CUDA_TRY(ctx, cudaMemcpyAsync(test_block, tblk, (size_t)ntest * sizeof(int32_t),
                                      cudaMemcpyDeviceToDevice, s));
  if (bc_test_eff) *bc_test_eff = kt;
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  return sbv_sync_status(ctx, stream);
}

extern "C" int sbv_matern(sbv_ctx* ctx, int32_t precision, int32_t nu2, const double* d2,
                          int64_t n, double* out, void* stream) {
  if (!ctx) return SBV_EINVAL;
  if (n < 0) return fail(ctx, SBV_EINVAL, "n=%lld is negative", (long long)n);
  if (n > 0 && (!d2 || !out)) return fail(ctx, SBV_EINVAL, "null pointer argument");
  if (precision != SBV_PREC_FP64 && precision != SBV_PREC_MIXED &&
      precision != SBV_PREC_MIXED_BF16)
    return fail(ctx, SBV_EINVAL, "precision=%d unknown", precision);
  if (!nu_ok_prec(nu2, precision))
    return fail(ctx, SBV_EINVAL, "nu2=%d: FP64 takes 1..%d, the mixed precisions {1,3,5,7}", nu2,
                SBV_MAX_NU2);
  SBV_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return run_matern(ctx, precision, nu2, d2, n, out, (cudaStream_t)stream);
}

extern "C" int sbv_simulate(sbv_ctx* ctx, const double* mean, const double* var, int64_t ntest,
                            int32_t ndraws, uint64_t seed, uint64_t index_base,
                            double* sample_mean,
                            double* sample_var, double* ci_lo, double* ci_hi, double* draws,
                            void* stream) {
  if (!ctx) return SBV_EINVAL;
  if (ntest < 0) return fail(ctx, SBV_EINVAL, "ntest=%lld is negative", (long long)ntest);
  if (ndraws < 2 || ndraws > SBV_MAX_DRAWS)
    return fail(ctx, SBV_EINVAL, "ndraws=%d outside [2, %d]", ndraws, SBV_MAX_DRAWS);
  if (ntest > 0 && (!mean || !var || !sample_mean || !sample_var || !ci_lo || !ci_hi))
    return fail(ctx, SBV_EINVAL, "null pointer argument");
  SBV_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  return run_simulate(ctx, mean, var, ntest, ndraws, seed, index_base, sample_mean, sample_var, ci_lo, ci_hi,
                      draws, (cudaStream_t)stream);
}
