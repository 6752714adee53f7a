// Batched Block Vecchia log-likelihood (Alg. 5 per block, Alg. 1 Step 5 for
// the sum) and block-Vecchia prediction (Sec. 4.2, 5.5): FP64 path.
//
// One CTA factors one (theta, block) work item at a time; a persistent grid
// takes items from an atomic counter.  The item's N = m_i + bs_i points are
// gathered, the packed lower triangle of the joint covariance of [J; B] is
// built in shared memory (global scratch when it does not fit) with the
// observations bordered as row N, and a right-looking Cholesky of the first N
// columns leaves L on the diagonal/below and w = L^{-1} y in row N.  Then
//   l_i = -1/2 [ bs log 2pi + 2 sum_{t>=m_i} log L_tt + sum_{t>=m_i} w_t^2 ],
// which is the Schur-complement chain of Alg. 5 (POTRF of Sigma^con, TRSM,
// GEMM, Schur with Sigma^lk, POTRF, TRSV, dot, log-det) done in one pass.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bessel.cuh"
#include "block_common.cuh"
#include "sbv_internal.cuh"

namespace sbv {

constexpr int LL_THREADS = 256;

// Matern correlation of the FP64 paths: the closed forms for nu2 in
// {1, 3, 5, 7}, the Bessel-function form (bessel.cuh) for any other nu2.
__device__ __forceinline__ double matern_fp64(double r, int nu2) {
  if (nu2 == 1 || nu2 == 3 || nu2 == 5 || nu2 == 7) return matern64(r, nu2);
  return matern_general(r, 0.5 * nu2);
}

// Gather the N points of an item into u[t][p] = x_p,t / beta_t and yv[p].
// Point p < mb is neighbour p of the block, p >= mb is member p - mb.
__device__ void gather_item(const LoglikArgs& a, int64_t blk, int mb, int N,
                            const ThetaDev& th, double* u, int ustride, double* yv) {
  const int d = a.d;
  const int64_t base = a.ptr[blk];
  for (int e = threadIdx.x; e < N * d; e += blockDim.x) {
    int p = e / d, t = e - p * d;
    int64_t id = p < mb ? (int64_t)a.nbr[blk * a.m + p] : (int64_t)a.pts[base + (p - mb)];
    double x = a.dtype == SBV_F64 ? ld_x<double>(a.X, id * d + t) : ld_x<float>(a.X, id * d + t);
    u[t * ustride + p] = x * th.inv_beta[t];
  }
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    int64_t id = p < mb ? (int64_t)a.nbr[blk * a.m + p] : (int64_t)a.pts[base + (p - mb)];
    yv[p] = a.y[id];
  }
}

// Packed lower triangle of the joint covariance, rows 0..N-1, plus row N = yv.
__device__ void build_cov(const double* u, int ustride, int d, int N, const ThetaDev& th,
                          int nu2, const double* yv, double* A) {
  const int total = N * (N + 1) / 2;
  int i = 0, j = threadIdx.x;
  while (j > i) { j -= i + 1; ++i; }
  for (int l = threadIdx.x; l < total; l += blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < d; ++t) {
      double df = u[t * ustride + i] - u[t * ustride + j];
      s = fma(df, df, s);
    }
    double K = th.sigma2 * matern_fp64(sqrt(s), nu2);
    if (i == j) K += th.tau2;
    A[l] = K;
    j += blockDim.x;
    while (j > i) { j -= i + 1; ++i; }
  }
  const int rowN = N * (N + 1) / 2;
  for (int p = threadIdx.x; p < N; p += blockDim.x) A[rowN + p] = yv[p];
}

// Right-looking Cholesky of columns 0..kend-1 of the (N+1)-row packed matrix
// (row N is the bordered right-hand side).  Returns false if a pivot is not
// positive; all threads return the same value.
__device__ bool chol_columns(double* A, int N, int kend, double* s_scalar, int* s_flag) {
  for (int k = 0; k < kend; ++k) {
    if (threadIdx.x == 0) {
      double piv = A[tri(k, k)];
      if (!(piv > 0.0) || !isfinite(piv)) {
        *s_flag = 1;
      } else {
        double L = sqrt(piv);
        A[tri(k, k)] = L;
        *s_scalar = 1.0 / L;
      }
    }
    __syncthreads();
    if (*s_flag) return false;
    const double inv = *s_scalar;
    for (int i = k + 1 + threadIdx.x; i <= N; i += blockDim.x) A[tri(i, k)] *= inv;
    __syncthreads();
    // trailing update of rows k+1..N, columns k+1..min(i, N-1)
    const int T = N - 1 - k;
    const int tri_n = T * (T + 1) / 2;
    const int total = tri_n + T;
    int ii = 0, jj = threadIdx.x;
    while (jj > ii) { jj -= ii + 1; ++ii; }
    for (int l = threadIdx.x; l < total; l += blockDim.x) {
      int i, j;
      if (l < tri_n) {
        i = k + 1 + ii;
        j = k + 1 + jj;
      } else {
        i = N;
        j = k + 1 + (l - tri_n);
      }
      A[tri(i, j)] -= A[tri(i, k)] * A[tri(j, k)];
      jj += blockDim.x;
      while (jj > ii) { jj -= ii + 1; ++ii; }
    }
    __syncthreads();
  }
  return true;
}

// Deterministic CTA sum of v over threads (fixed tree).
__device__ double cta_sum(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < nw; ++q) s += red[q];
  return s;  // valid on thread 0
}

__global__ void __launch_bounds__(LL_THREADS)
loglik_fp64_kernel(LoglikArgs a) {
  extern __shared__ __align__(16) double sm[];
  __shared__ double s_scalar;
  __shared__ int s_flag;
  __shared__ unsigned int s_item;
  __shared__ double red[LL_THREADS / 32];
  const int d = a.d;
  const int ustride = a.ncap + 1;
  double* u = sm;                               // d x (ncap+1)
  double* yv = u + (size_t)d * ustride;         // ncap+1
  double* A = a.gmat ? a.gmat + (size_t)blockIdx.x * a.gmat_stride : yv + ustride;
  // all items, or (list mode) the items a previous kernel handed over
  const unsigned int total = a.list ? *a.list_n : (unsigned int)(a.bc * a.B);
  const double log2pi = 1.8378770664093454836;

  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned int k = atomicAdd(a.counter, 1u);
      s_item = k < total ? (a.list ? a.list[k] : k) : 0xffffffffu;
    }
    __syncthreads();
    const unsigned int item = s_item;
    if (item == 0xffffffffu) break;
    const int th_i = (int)(item / a.bc);
    const int64_t blk = (int64_t)(item % a.bc);
    const ThetaDev& th = a.theta[th_i];
    const int bs = (int)(a.ptr[blk + 1] - a.ptr[blk]);
    const int mb = a.cnt[blk];
    const int N = mb + bs;
    if (N > a.ncap) {
      if (threadIdx.x == 0) {
        a.terms[item] = __longlong_as_double(0x7ff8000000000000ll);
        if (a.status) a.status[item] = SBV_EUNSUPPORTED;
        record_failure(a.dstat, SBV_EUNSUPPORTED, (int)blk, th_i);
      }
      __syncthreads();
      continue;
    }
    gather_item(a, blk, mb, N, th, u, ustride, yv);
    __syncthreads();
    build_cov(u, ustride, d, N, th, a.nu2, yv, A);
    if (threadIdx.x == 0) s_flag = 0;
    __syncthreads();
    bool ok = chol_columns(A, N, N, &s_scalar, &s_flag);
    double v = 0.0;
    if (ok) {
      for (int t = mb + threadIdx.x; t < N; t += blockDim.x) {
        double w = A[tri(N, t)];
        v += 2.0 * log(A[tri(t, t)]) + w * w;
      }
    }
    double s = cta_sum(v, red);
    if (threadIdx.x == 0) {
      if (ok) {
        a.terms[item] = -0.5 * ((double)bs * log2pi + s);
        if (a.status) a.status[item] = 0;
      } else {
        a.terms[item] = __longlong_as_double(0x7ff8000000000000ll);
        if (a.status) a.status[item] = SBV_ENOTSPD;
        record_failure(a.dstat, SBV_ENOTSPD, (int)blk, th_i);
      }
    }
    __syncthreads();
  }
}

// ll[b] = sum_i terms[b, i]: each thread adds a fixed strided subset in order,
// then a fixed tree; identical results on every call.
__global__ void reduce_terms_kernel(const double* __restrict__ terms, int64_t bc,
                                    double* __restrict__ ll) {
  __shared__ double red[32];
  const double* t = terms + (int64_t)blockIdx.x * bc;
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < bc; i += blockDim.x) v += t[i];
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) ll[blockIdx.x] = w;
  }
}

// Largest m_i + bs_i over blocks.
__global__ void max_n_kernel(const int64_t* __restrict__ ptr, const int32_t* __restrict__ cnt,
                             int64_t bc, int* __restrict__ out) {
  int v = 0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < bc;
       j += (int64_t)gridDim.x * blockDim.x)
    v = max(v, (int)(ptr[j + 1] - ptr[j]) + cnt[j]);
  for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}

// Largest m_i + bs_i (out[0]) and largest bs_i (out[1]) over blocks.
__global__ void max_sizes_kernel(const int64_t* __restrict__ ptr, const int32_t* __restrict__ cnt,
                                 int64_t bc, int* __restrict__ out) {
  int v = 0, w = 0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < bc;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int bs = (int)(ptr[j + 1] - ptr[j]);
    v = max(v, bs + cnt[j]);
    w = max(w, bs);
  }
  for (int o = 16; o; o >>= 1) {
    v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, v);
    atomicMax(out + 1, w);
  }
}

static std::vector<ThetaDev> derive_theta(const double* h, int B, int d) {
  std::vector<ThetaDev> out(B);
  for (int b = 0; b < B; ++b) {
    const double* r = h + (size_t)b * (2 + d);
    memset(&out[b], 0, sizeof(ThetaDev));
    out[b].sigma2 = r[0];
    out[b].tau2 = r[1];
    for (int t = 0; t < d; ++t) out[b].inv_beta[t] = 1.0 / r[2 + t];
    auto split = [](double v, float& h, float& l) {
      h = (float)v;
      l = (float)(v - (double)h);
    };
    split(r[0], out[b].s2_h, out[b].s2_l);
    split(r[0] + r[1], out[b].diag_h, out[b].diag_l);
    for (int t = 0; t < d; ++t) split(out[b].inv_beta[t], out[b].ib_h[t], out[b].ib_l[t]);
  }
  return out;
}

// Copy derived theta rows to the device.  A pageable-to-device cudaMemcpyAsync
// stages the bytes before returning, so the host vector may die right away
// and no host synchronisation is needed.
static int upload_theta(sbv_ctx* ctx, const double* h, int B, int d, ThetaDev** out,
                        cudaStream_t s) {
  int st = 0;
  std::vector<ThetaDev> v = derive_theta(h, B, d);
  size_t bytes = v.size() * sizeof(ThetaDev);
  ThetaDev* dth = (ThetaDev*)ws_get(ctx, WS_PARAMS, bytes, &st);
  if (!dth) return st;
  // stage through a pinned ring slot so that the copy is truly asynchronous
  if (ctx->ring_slot < bytes) {
    SBV_CUDA_TRY(ctx, cudaDeviceSynchronize());
    if (ctx->h_ring) cudaFreeHost(ctx->h_ring);
    ctx->h_ring = nullptr;
    ctx->ring_slot = 0;
    const size_t slot = ((bytes + 4095) / 4096) * 4096;
    SBV_CUDA_TRY(ctx, cudaMallocHost((void**)&ctx->h_ring, slot * sbv_ctx::kRing));
    ctx->ring_slot = slot;
    for (auto& e : ctx->ring_ev)
      if (!e) SBV_CUDA_TRY(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  const int k = ctx->ring_next;
  ctx->ring_next = (k + 1) % sbv_ctx::kRing;
  SBV_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ring_ev[k]));  // previous copy from this slot done
  unsigned char* slot = ctx->h_ring + (size_t)k * ctx->ring_slot;
  memcpy(slot, v.data(), bytes);
  SBV_CUDA_TRY(ctx, cudaMemcpyAsync(dth, slot, bytes, cudaMemcpyHostToDevice, s));
  SBV_CUDA_TRY(ctx, cudaEventRecord(ctx->ring_ev[k], s));
  *out = dth;
  return SBV_OK;
}

// Largest N over blocks (one small reduction and a host read per call; the
// kernels still check every item against the capacity they were launched with).
static int structure_max_n(sbv_ctx* ctx, const int64_t* ptr, const int32_t* cnt, int64_t bc,
                           int* out, cudaStream_t s) {
  int st = 0;
  int* d = (int*)ws_get(ctx, WS_SMALL, 64, &st);
  if (!d) return st;
  SBV_CUDA_TRY(ctx, cudaMemsetAsync(d, 0, 4, s));
  int g = (int)std::min<int64_t>((bc + 255) / 256, (int64_t)ctx->num_sms * 8);
  max_n_kernel<<<std::max(g, 1), 256, 0, s>>>(ptr, cnt, bc, d);
  SBV_LAUNCH_CHECK(ctx, "max_n_kernel");
  SBV_CUDA_TRY(ctx, cudaMemcpyAsync(out, d, 4, cudaMemcpyDeviceToHost, s));
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  return SBV_OK;
}

int launch_loglik_mixed(sbv_ctx* ctx, const LoglikArgs& a, int nmax, int bsmax, int precision,
                        unsigned int* fb_list, unsigned int* fb_count, cudaStream_t s);
int launch_predict_mixed(sbv_ctx* ctx, const LoglikArgs& a0, const void* Xt, int64_t nt,
                         double* mean, double* var, double* var_latent, int precision,
                         unsigned int* fb_list, unsigned int* fb_count, cudaStream_t s,
                         const int64_t* tptr, const int32_t* tpts, int bsmax);

int run_max_n(sbv_ctx* ctx, const int64_t* ptr, const int32_t* cnt, int64_t bc, int* out,
              cudaStream_t s) {
  return structure_max_n(ctx, ptr, cnt, bc, out, s);
}

// Largest m_i + bs_i and largest bs_i (one small kernel and a host read).
int run_max_sizes(sbv_ctx* ctx, const int64_t* ptr, const int32_t* cnt, int64_t bc, int* nmax,
                  int* bsmax, cudaStream_t s) {
  int st = 0;
  int* d = (int*)ws_get(ctx, WS_SMALL, 64, &st);
  if (!d) return st;
  SBV_CUDA_TRY(ctx, cudaMemsetAsync(d, 0, 8, s));
  int g = (int)std::min<int64_t>((bc + 255) / 256, (int64_t)ctx->num_sms * 8);
  max_sizes_kernel<<<std::max(g, 1), 256, 0, s>>>(ptr, cnt, bc, d);
  SBV_LAUNCH_CHECK(ctx, "max_sizes_kernel");
  int h[2] = {0, 0};
  SBV_CUDA_TRY(ctx, cudaMemcpyAsync(h, d, 8, cudaMemcpyDeviceToHost, s));
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  *nmax = h[0];
  *bsmax = h[1];
  ctx->sz_ptr = ptr;
  ctx->sz_cnt = cnt;
  ctx->sz_bc = bc;
  ctx->sz_nmax = h[0];
  ctx->sz_bsmax = h[1];
  return SBV_OK;
}

std::vector<ThetaDev> derive_theta_rows(const double* h, int B, int d) {
  return derive_theta(h, B, d);
}

// FP64 kernel launch plan: shared-memory matrices when they fit (global
// scratch slices otherwise) and resident CTAs per SM from the autotuning
// record or the shared-memory limit (<= 4).
int fp64_plan(sbv_ctx* ctx, int nmax, int d, int64_t items, Fp64Plan* o) {
  const size_t ub = (size_t)(d + 1) * (nmax + 1) * sizeof(double);
  const size_t mat = (size_t)(nmax + 1) * (nmax + 2) / 2 * sizeof(double);
  o->gmat_stride = 0;
  int fit, per_sm;
  if (ub + mat + 1024 <= ctx->smem_optin) {
    o->smem = ub + mat;
    fit = (int)std::max<size_t>(1, (228 * 1024) / (o->smem + 2048));
    per_sm = std::min(fit, 4);
  } else {
    o->smem = ub;
    if (ub + 1024 > ctx->smem_optin)
      return fail(ctx, SBV_EUNSUPPORTED, "d=%d with N=%d exceeds shared memory", d, nmax);
    fit = 4;
    per_sm = 2;
    o->gmat_stride = (mat / sizeof(double) + 31) & ~(size_t)31;
  }
  if (ctx->force.threads) {
    per_sm = ctx->force.per_sm;
  } else {
    for (const auto& t : ctx->tuned)
      if (t.precision == SBV_PREC_FP64 && t.pred == 0 && t.ncap == nmax && t.d == d) per_sm = t.per_sm;
  }
  per_sm = std::max(1, std::min(per_sm, fit));
  int64_t grid = (int64_t)ctx->num_sms * per_sm;
  if (grid > items) grid = std::max<int64_t>(items, 1);
  o->grid = (int)grid;
  return SBV_OK;
}

static bool g_fp64_ready[64];

// Once per device: allow the FP64 kernel the largest dynamic shared memory,
// so that later launches (and captured ones) make no other API call.
int fp64_prepare(sbv_ctx* ctx) {
  if (ctx->device < 64 && g_fp64_ready[ctx->device]) return SBV_OK;
  SBV_CUDA_TRY(ctx, cudaFuncSetAttribute(loglik_fp64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ctx->smem_optin - 1024));
  if (ctx->device < 64) g_fp64_ready[ctx->device] = true;
  return SBV_OK;
}

int fp64_enqueue(sbv_ctx* ctx, const LoglikArgs& a, const Fp64Plan& o, cudaStream_t s) {
  int st = fp64_prepare(ctx);
  if (st) return st;
  loglik_fp64_kernel<<<o.grid, LL_THREADS, o.smem, s>>>(a);
  SBV_LAUNCH_CHECK(ctx, "loglik_fp64_kernel");
  return SBV_OK;
}

int reduce_enqueue(sbv_ctx* ctx, const double* terms, int64_t bc, int B, double* ll,
                   cudaStream_t s) {
  reduce_terms_kernel<<<B, 1024, 0, s>>>(terms, bc, ll);
  SBV_LAUNCH_CHECK(ctx, "reduce_terms_kernel");
  return SBV_OK;
}

// FP64 kernel in list mode over the items the mixed kernel handed over
// (list[0 .. *list_n - 1]); a persistent grid whose CTAs leave at once when
// the list is empty.
int fp64_fallback_enqueue(sbv_ctx* ctx, const LoglikArgs& a0, int nmax, const unsigned int* list,
                          const unsigned int* list_n, unsigned int* counter, cudaStream_t s,
                          double* gmat_owned) {
  int st = 0;
  LoglikArgs a = a0;
  a.list = list;
  a.list_n = list_n;
  a.counter = counter;
  Fp64Plan o;
  if ((st = fp64_plan(ctx, nmax, a.d, a.bc * (int64_t)a.B, &o))) return st;
  if (o.gmat_stride) {
    double* g = gmat_owned;
    if (!g) {
      g = (double*)ws_get(ctx, WS_GMAT64, o.gmat_stride * o.grid * sizeof(double), &st);
      if (!g) return st;
    }
    a.gmat = g;
    a.gmat_stride = o.gmat_stride;
  }
  return fp64_enqueue(ctx, a, o, s);
}

int run_loglik(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n, int d,
               const int64_t* ptr, const int32_t* pts, const int32_t* nbr, const int32_t* cnt,
               int64_t bc, int m, int nmax_hint, const double* h_theta, int B, int nu2,
               int precision, double* ll, double* terms, int32_t* status, cudaStream_t s) {
  int st = 0;
  if ((uint64_t)bc * (uint64_t)B >= 0xffffffffull)
    return fail(ctx, SBV_EUNSUPPORTED, "bc*B too large");
  // with a size hint the largest block size is not read back, and the mixed
  // kernel's layout assumes the largest bs the hint allows
  int nmax = nmax_hint, bsmax = 0;
  if (nmax <= 0 && (st = run_max_sizes(ctx, ptr, cnt, bc, &nmax, &bsmax, s))) return st;
  if (nmax_hint > 0 && ctx->sz_ptr == (const void*)ptr && ctx->sz_cnt == (const void*)cnt &&
      ctx->sz_bc == bc && ctx->sz_nmax == nmax_hint)
    bsmax = ctx->sz_bsmax;
  if (nmax > SBV_MAX_BLOCK_N)
    return fail(ctx, SBV_EUNSUPPORTED, "a block has m_i + bs_i = %d > %d", nmax, SBV_MAX_BLOCK_N);
  ThetaDev* dth = nullptr;
  if ((st = upload_theta(ctx, h_theta, B, d, &dth, s))) return st;
  if (!terms) {
    terms = (double*)ws_get(ctx, WS_TERMS, (size_t)B * bc * sizeof(double), &st);
    if (!terms) return st;
  }
  unsigned int* counter = (unsigned int*)ws_get(ctx, WS_SMALL, 64, &st);
  if (!counter) return st;
  counter += 4;  // first words hold the max-N scratch; then the work counter,
                 // the hand-over count and the FP64 kernel's work counter
  SBV_CUDA_TRY(ctx, cudaMemsetAsync(counter, 0, 3 * sizeof(unsigned int), s));

  LoglikArgs a;
  memset(&a, 0, sizeof(a));
  a.X = X;
  a.dtype = dtype;
  a.y = y;
  a.n = n;
  a.d = d;
  a.ptr = ptr;
  a.pts = pts;
  a.nbr = nbr;
  a.cnt = cnt;
  a.bc = bc;
  a.m = m;
  a.theta = dth;
  a.B = B;
  a.nu2 = nu2;
  a.ncap = nmax;
  a.terms = terms;
  a.status = status;
  a.dstat = ctx->d_status;
  a.counter = counter;
  a.gmat = nullptr;
  a.gmat_stride = 0;

  if (precision == SBV_PREC_MIXED || precision == SBV_PREC_MIXED_BF16) {
    unsigned int* list =
        (unsigned int*)ws_get(ctx, WS_RERUN, (size_t)B * bc * sizeof(unsigned int), &st);
    if (!list) return st;
    if ((st = launch_loglik_mixed(ctx, a, nmax, bsmax, precision, list, counter + 1, s))) return st;
    // the items handed over (pivots, capacity) go through the FP64 kernel
    if ((st = fp64_fallback_enqueue(ctx, a, nmax, list, counter + 1, counter + 2, s))) return st;
  } else {
    Fp64Plan o;
    if ((st = fp64_plan(ctx, nmax, d, bc * (int64_t)B, &o))) return st;
    if (o.gmat_stride) {
      double* g = (double*)ws_get(ctx, WS_MATRIX, o.gmat_stride * o.grid * sizeof(double), &st);
      if (!g) return st;
      a.gmat = g;
      a.gmat_stride = o.gmat_stride;
    }
    if ((st = fp64_enqueue(ctx, a, o, s))) return st;
  }
  reduce_terms_kernel<<<B, 1024, 0, s>>>(terms, bc, ll);
  SBV_LAUNCH_CHECK(ctx, "reduce_terms_kernel");
  return SBV_OK;
}

// ---------------------------------------------------------------------------
// Gradient of the block terms with respect to theta = (sigma^2, tau^2,
// beta_1..beta_d), FP64 (the gradient information of Sec. 6).  For either
// Gaussian system (joint S = J u B, and J), with x = Sigma^{-1} y,
//   d log N(y; 0, Sigma) / d theta_k = 1/2 x^T dSigma_k x - 1/2 tr(Sigma^{-1} dSigma_k),
// and l_i is the joint log-density minus the J one.  From the item's factor L:
//   * x = L^{-T} w and x_J = L_JJ^{-T} w_J (= L^{-T} (w_J, 0) restricted to J),
//   * Sigma^{-1} - [Sigma_JJ^{-1}, 0; 0, 0] = Z_B^T Z_B, Z_B the B rows of L^{-1},
// all from one backward substitution with L^T over bs + 2 right-hand sides
// (unit vectors e_t for t in B, w, (w_J, 0)).  Then one pass over the pairs
// (i >= j) adds  c_ij dSigma_ij,k  with
//   c_ij = (2 - [i = j]) (1/2 (x_i x_j - xJ_i xJ_j) - 1/2 (Z_B^T Z_B)_ij),
//   dSigma/dsigma^2 = M(r), dSigma/dtau^2 = [i = j],
//   dSigma/dbeta_t = sigma^2 h(r) u_t^2 / beta_t,  h = -M'(r) / r,
// u_t the scaled coordinate difference, r = |u|.
// ---------------------------------------------------------------------------
constexpr int GR_CHUNK = 16;   // gradient components accumulated per pass over the pairs

struct GradArgs {
  double* gterms;      // B x bc x (2 + d): d l_{b,i} / d theta_k
  double* zt;          // per CTA: N x (bs + 2) right-hand sides, row-major
  size_t zt_stride;    // doubles per CTA slice (ncap x (ncap + 2))
};

// -M'(r) / r: closed forms for nu2 in {1, 3, 5, 7} (0 at r = 0 for nu = 1/2,
// where every u_t is 0 as well), the Bessel-function form for any other nu2.
__device__ __forceinline__ double h_nu64(double r, int nu2) {
  const double e = exp(-r);
  switch (nu2) {
    case 1: return r > 0.0 ? e / r : 0.0;
    case 3: return e;
    case 5: return (1.0 + r) * e * (1.0 / 3.0);
    case 7: return fma(r, r + 3.0, 3.0) * e * (1.0 / 15.0);
    default: return matern_general_h(r, 0.5 * nu2);
  }
}

__global__ void __launch_bounds__(LL_THREADS)
loglik_grad_fp64_kernel(LoglikArgs a, GradArgs g) {
  extern __shared__ __align__(16) double sm[];
  __shared__ double s_scalar;
  __shared__ int s_flag;
  __shared__ unsigned int s_item;
  __shared__ double red[LL_THREADS / 32];
  __shared__ double gred[LL_THREADS / 32][GR_CHUNK];
  const int d = a.d, p = d + 2;
  const int ustride = a.ncap + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double* u = sm;                               // d x (ncap+1)
  double* yv = u + (size_t)d * ustride;         // ncap+1
  double* A = a.gmat ? a.gmat + (size_t)blockIdx.x * a.gmat_stride : yv + ustride;
  double* Zt = g.zt + (size_t)blockIdx.x * g.zt_stride;
  const unsigned int total = (unsigned int)(a.bc * a.B);
  const double log2pi = 1.8378770664093454836;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);

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
    double* gout = g.gterms + (size_t)item * p;
    if (N > a.ncap) {
      if (threadIdx.x == 0) {
        a.terms[item] = nan;
        if (a.status) a.status[item] = SBV_EUNSUPPORTED;
        record_failure(a.dstat, SBV_EUNSUPPORTED, (int)blk, th_i);
      }
      for (int k = threadIdx.x; k < p; k += blockDim.x) gout[k] = nan;
      __syncthreads();
      continue;
    }
    gather_item(a, blk, mb, N, th, u, ustride, yv);
    __syncthreads();
    build_cov(u, ustride, d, N, th, a.nu2, yv, A);
    if (threadIdx.x == 0) s_flag = 0;
    __syncthreads();
    const bool ok = chol_columns(A, N, N, &s_scalar, &s_flag);
    double v = 0.0;
    if (ok) {
      for (int t = mb + threadIdx.x; t < N; t += blockDim.x) {
        const double w = A[tri(N, t)];
        v += 2.0 * log(A[tri(t, t)]) + w * w;
      }
    }
    const double s = cta_sum(v, red);
    if (threadIdx.x == 0) {
      if (ok) {
        a.terms[item] = -0.5 * ((double)bs * log2pi + s);
        if (a.status) a.status[item] = 0;
      } else {
        a.terms[item] = nan;
        if (a.status) a.status[item] = SBV_ENOTSPD;
        record_failure(a.dstat, SBV_ENOTSPD, (int)blk, th_i);
      }
    }
    if (!ok) {
      for (int k = threadIdx.x; k < p; k += blockDim.x) gout[k] = nan;
      __syncthreads();
      continue;
    }
    // right-hand sides: columns q < bs the unit vectors e_{mb+q}, column bs
    // w = L^{-1} y (row N of A), column bs+1 (w_J, 0)
    const int nq = bs + 2;
    for (int e = threadIdx.x; e < N * nq; e += blockDim.x) {
      const int k = e / nq, q = e - k * nq;
      double r0;
      if (q < bs) r0 = (k == mb + q) ? 1.0 : 0.0;
      else if (q == bs || k < mb) r0 = A[tri(N, k)];
      else r0 = 0.0;
      Zt[e] = r0;
    }
    __syncthreads();
    // backward substitution with L^T for all right-hand sides: row c is final
    // once rows c+1..N-1 are subtracted; then it is removed from rows 0..c-1
    for (int c = N - 1; c >= 0; --c) {
      const double inv = 1.0 / A[tri(c, c)];
      for (int q = threadIdx.x; q < nq; q += blockDim.x) Zt[(size_t)c * nq + q] *= inv;
      __syncthreads();
      for (int e = threadIdx.x; e < c * nq; e += blockDim.x) {
        const int k = e / nq, q = e - k * nq;
        Zt[e] = fma(-A[tri(c, k)], Zt[(size_t)c * nq + q], Zt[e]);
      }
      __syncthreads();
    }
    // pass over the pairs, GR_CHUNK gradient components at a time
    const int npair = N * (N + 1) / 2;
    for (int k0 = 0; k0 < p; k0 += GR_CHUNK) {
      double acc[GR_CHUNK];
#pragma unroll
      for (int c = 0; c < GR_CHUNK; ++c) acc[c] = 0.0;
      int i = 0, j = threadIdx.x;
      while (j > i) { j -= i + 1; ++i; }
      for (int l = threadIdx.x; l < npair; l += blockDim.x) {
        double r2 = 0.0;
        for (int t = 0; t < d; ++t) {
          const double df = u[t * ustride + i] - u[t * ustride + j];
          r2 = fma(df, df, r2);
        }
        const double r = sqrt(r2);
        const double* zi = Zt + (size_t)i * nq;
        const double* zj = Zt + (size_t)j * nq;
        double D = 0.0;
        for (int q = 0; q < bs; ++q) D = fma(zi[q], zj[q], D);
        double wgt = 0.5 * (zi[bs] * zj[bs] - zi[bs + 1] * zj[bs + 1]) - 0.5 * D;
        if (i != j) wgt *= 2.0;
        const double Mv = matern_fp64(r, a.nu2);
        const double hv = th.sigma2 * h_nu64(r, a.nu2);
#pragma unroll
        for (int c = 0; c < GR_CHUNK; ++c) {
          const int k = k0 + c;
          double dk = 0.0;
          if (k == 0) {
            dk = Mv;
          } else if (k == 1) {
            dk = (i == j) ? 1.0 : 0.0;
          } else if (k < p) {
            const int t = k - 2;
            const double df = u[t * ustride + i] - u[t * ustride + j];
            dk = hv * df * df * th.inv_beta[t];
          }
          acc[c] = fma(wgt, dk, acc[c]);
        }
        j += blockDim.x;
        while (j > i) { j -= i + 1; ++i; }
      }
      // fixed-order CTA reduction of the chunk
#pragma unroll
      for (int c = 0; c < GR_CHUNK; ++c) {
        double x = acc[c];
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) gred[warp][c] = x;
      }
      __syncthreads();
      if (threadIdx.x < GR_CHUNK && k0 + (int)threadIdx.x < p) {
        double x = 0.0;
        for (int w = 0; w < nw; ++w) x += gred[w][threadIdx.x];
        gout[k0 + threadIdx.x] = x;
      }
      __syncthreads();
    }
  }
}

// grad[b, k] = sum_i gterms[b, i, k] in a fixed order (as reduce_terms_kernel).
__global__ void reduce_grad_kernel(const double* __restrict__ gterms, int64_t bc, int p,
                                   double* __restrict__ grad) {
  __shared__ double red[32];
  const int b = blockIdx.x / p, k = blockIdx.x - b * p;
  const double* t = gterms + (size_t)b * bc * p + k;
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < bc; i += blockDim.x) v += t[(size_t)i * p];
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) grad[blockIdx.x] = w;
  }
}

static bool g_grad_ready[64];

int run_loglik_grad(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n, int d,
                    const int64_t* ptr, const int32_t* pts, const int32_t* nbr,
                    const int32_t* cnt, int64_t bc, int m, int nmax_hint, const double* h_theta,
                    int B, int nu2, double* ll, double* grad, double* terms, double* gterms,
                    int32_t* status, cudaStream_t s) {
  int st = 0;
  const int p = d + 2;
  if ((uint64_t)bc * (uint64_t)B >= 0xffffffffull)
    return fail(ctx, SBV_EUNSUPPORTED, "bc*B too large");
  // with a size hint the largest block size is not read back, and the mixed
  // kernel's layout assumes the largest bs the hint allows
  int nmax = nmax_hint, bsmax = 0;
  if (nmax <= 0 && (st = run_max_sizes(ctx, ptr, cnt, bc, &nmax, &bsmax, s))) return st;
  if (nmax_hint > 0 && ctx->sz_ptr == (const void*)ptr && ctx->sz_cnt == (const void*)cnt &&
      ctx->sz_bc == bc && ctx->sz_nmax == nmax_hint)
    bsmax = ctx->sz_bsmax;
  if (nmax > SBV_MAX_BLOCK_N)
    return fail(ctx, SBV_EUNSUPPORTED, "a block has m_i + bs_i = %d > %d", nmax, SBV_MAX_BLOCK_N);
  ThetaDev* dth = nullptr;
  if ((st = upload_theta(ctx, h_theta, B, d, &dth, s))) return st;
  if (!terms) {
    terms = (double*)ws_get(ctx, WS_TERMS, (size_t)B * bc * sizeof(double), &st);
    if (!terms) return st;
  }
  if (!gterms) {
    gterms = (double*)ws_get(ctx, WS_GRAD, (size_t)B * bc * p * sizeof(double), &st);
    if (!gterms) return st;
  }
  unsigned int* counter = (unsigned int*)ws_get(ctx, WS_SMALL, 64, &st);
  if (!counter) return st;
  counter += 4;
  SBV_CUDA_TRY(ctx, cudaMemsetAsync(counter, 0, sizeof(unsigned int), s));
  if (!(ctx->device < 64 && g_grad_ready[ctx->device])) {
    SBV_CUDA_TRY(ctx, cudaFuncSetAttribute(loglik_grad_fp64_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)ctx->smem_optin - 4096));
    if (ctx->device < 64) g_grad_ready[ctx->device] = true;
  }
  // the FP64 plan, with room for this kernel's larger static shared memory
  const size_t ub = (size_t)(d + 1) * (nmax + 1) * sizeof(double);
  const size_t mat = (size_t)(nmax + 1) * (nmax + 2) / 2 * sizeof(double);
  size_t smem = ub + mat, gstride = 0;
  if (smem + 4096 > ctx->smem_optin) {
    smem = ub;
    if (ub + 4096 > ctx->smem_optin)
      return fail(ctx, SBV_EUNSUPPORTED, "d=%d with N=%d exceeds shared memory", d, nmax);
    gstride = (mat / sizeof(double) + 31) & ~(size_t)31;
  }
  int64_t grid = (int64_t)ctx->num_sms * std::max(1, std::min(2, (int)((228 * 1024) / (smem + 4096))));
  if (grid > bc * (int64_t)B) grid = std::max<int64_t>(bc * (int64_t)B, 1);
  LoglikArgs a;
  memset(&a, 0, sizeof(a));
  a.X = X;
  a.dtype = dtype;
  a.y = y;
  a.n = n;
  a.d = d;
  a.ptr = ptr;
  a.pts = pts;
  a.nbr = nbr;
  a.cnt = cnt;
  a.bc = bc;
  a.m = m;
  a.theta = dth;
  a.B = B;
  a.nu2 = nu2;
  a.ncap = nmax;
  a.terms = terms;
  a.status = status;
  a.dstat = ctx->d_status;
  a.counter = counter;
  a.gmat = nullptr;
  a.gmat_stride = 0;
  if (gstride) {
    double* gm = (double*)ws_get(ctx, WS_MATRIX, gstride * grid * sizeof(double), &st);
    if (!gm) return st;
    a.gmat = gm;
    a.gmat_stride = gstride;
  }
  GradArgs ga;
  ga.gterms = gterms;
  ga.zt_stride = ((size_t)nmax * (nmax + 2) + 31) & ~(size_t)31;
  ga.zt = (double*)ws_get(ctx, WS_GRADZ, ga.zt_stride * grid * sizeof(double), &st);
  if (!ga.zt) return st;
  loglik_grad_fp64_kernel<<<(int)grid, LL_THREADS, smem, s>>>(a, ga);
  SBV_LAUNCH_CHECK(ctx, "loglik_grad_fp64_kernel");
  reduce_terms_kernel<<<B, 1024, 0, s>>>(terms, bc, ll);
  SBV_LAUNCH_CHECK(ctx, "reduce_terms_kernel");
  reduce_grad_kernel<<<B * p, 1024, 0, s>>>(gterms, bc, p, grad);
  SBV_LAUNCH_CHECK(ctx, "reduce_grad_kernel");
  return SBV_OK;
}

// ---------------------------------------------------------------------------
// Prediction: one test point per item, conditioned on its m nearest training
// points; the joint matrix is [J; *] with the bordered row (y_J, 0).
// ---------------------------------------------------------------------------
struct PredictArgs {
  const void* X;
  const void* Xt;
  int dtype;
  const double* y;
  int d;
  const int32_t* nbr;   // nt x m
  int64_t nt;
  int m;
  const ThetaDev* theta;
  int nu2;
  double* mean;
  double* var;
  double* var_latent;
  DevStatus* dstat;
  unsigned int* counter;
  double* gmat;
  size_t gmat_stride;
  const unsigned int* list;     // list mode: the items handed over, or NULL
  const unsigned int* list_n;
  // blocks of test points (Sec. 5.5): item b predicts test points
  // tpts[tptr[b] .. tptr[b+1]) from the m training neighbours nbr[b]; NULL:
  // one item per test point
  const int64_t* tptr;
  const int32_t* tpts;
  int nmax;                     // m + the largest test block
};

__global__ void __launch_bounds__(LL_THREADS)
predict_fp64_kernel(PredictArgs a) {
  extern __shared__ __align__(16) double sm[];
  __shared__ double s_scalar;
  __shared__ int s_flag;
  __shared__ unsigned int s_item;
  const int d = a.d, m = a.m;
  const int ustride = a.nmax + 1;
  double* u = sm;
  double* yv = u + (size_t)d * ustride;
  double* A = a.gmat ? a.gmat + (size_t)blockIdx.x * a.gmat_stride : yv + ustride;
  const ThetaDev& th = a.theta[0];
  const unsigned int total = a.list ? *a.list_n : (unsigned int)a.nt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned int k = atomicAdd(a.counter, 1u);
      s_item = k < total ? (a.list ? a.list[k] : k) : 0xffffffffu;
    }
    __syncthreads();
    const unsigned int item = s_item;
    if (item == 0xffffffffu) break;
    const int64_t t0 = a.tptr ? a.tptr[item] : (int64_t)item;
    const int bs = a.tptr ? (int)(a.tptr[item + 1] - t0) : 1;
    const int N = m + bs;
    // the test point of member q
    auto tp = [&](int q) -> int64_t { return a.tptr ? (int64_t)a.tpts[t0 + q] : (int64_t)item; };
    for (int e = threadIdx.x; e < N * d; e += blockDim.x) {
      int p = e / d, t = e - p * d;
      double x;
      if (p < m) {
        int64_t id = a.nbr[(int64_t)item * m + p];
        x = a.dtype == SBV_F64 ? ld_x<double>(a.X, id * d + t) : ld_x<float>(a.X, id * d + t);
      } else {
        const int64_t q = tp(p - m);
        x = a.dtype == SBV_F64 ? ld_x<double>(a.Xt, q * d + t) : ld_x<float>(a.Xt, q * d + t);
      }
      u[t * ustride + p] = x * th.inv_beta[t];
    }
    for (int p = threadIdx.x; p < N; p += blockDim.x)
      yv[p] = p < m ? a.y[a.nbr[(int64_t)item * m + p]] : 0.0;
    __syncthreads();
    build_cov(u, ustride, d, N, th, a.nu2, yv, A);
    if (threadIdx.x == 0) s_flag = 0;
    __syncthreads();
    // factor the m columns of Sigma_JJ: row m + q then holds
    // w_q = L^{-1} Sigma_{J,q}, the bordered row z = L^{-1} y_J, and the
    // diagonal entry Sigma_qq - |w_q|^2 (the marginal conditional variance)
    const bool ok = chol_columns(A, N, m, &s_scalar, &s_flag);
    for (int q = warp; q < bs; q += nw) {
      double v = 0.0;
      if (ok)
        for (int t = lane; t < m; t += 32) v += A[tri(m + q, t)] * A[tri(N, t)];
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) {
        const int64_t pt = tp(q);
        if (ok) {
          const double var = A[tri(m + q, m + q)];
          a.mean[pt] = v;
          a.var[pt] = var;
          a.var_latent[pt] = var - th.tau2;
        } else {
          const double nan = __longlong_as_double(0x7ff8000000000000ll);
          a.mean[pt] = nan;
          a.var[pt] = nan;
          a.var_latent[pt] = nan;
        }
      }
    }
    if (!ok && threadIdx.x == 0) record_failure(a.dstat, SBV_ENOTSPD, (int)item, 0);
    __syncthreads();
  }
}

int run_predict(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n, int d,
                const void* Xt, int64_t nt, const int32_t* nbr, int m, const double* h_theta,
                int nu2, int precision, double* mean, double* var, double* var_latent,
                cudaStream_t s, const int64_t* tptr, const int32_t* tpts, int bsmax) {
  if (!tptr) bsmax = 1;
  int st = 0;
  ThetaDev* dth = nullptr;
  if ((st = upload_theta(ctx, h_theta, 1, d, &dth, s))) return st;
  unsigned int* counter = (unsigned int*)ws_get(ctx, WS_SMALL, 64, &st);
  if (!counter) return st;
  counter += 4;
  SBV_CUDA_TRY(ctx, cudaMemsetAsync(counter, 0, 3 * sizeof(unsigned int), s));
  unsigned int* list = nullptr;
  if (precision != SBV_PREC_FP64) {
    list = (unsigned int*)ws_get(ctx, WS_RERUN, (size_t)nt * sizeof(unsigned int), &st);
    if (!list) return st;
    LoglikArgs la;
    memset(&la, 0, sizeof(la));
    la.X = X;
    la.dtype = dtype;
    la.y = y;
    la.n = n;
    la.d = d;
    la.nbr = nbr;
    la.bc = nt;
    la.m = m;
    la.theta = dth;
    la.B = 1;
    la.nu2 = nu2;
    la.ncap = m + 1;
    la.dstat = ctx->d_status;
    la.counter = counter;
    if ((st = launch_predict_mixed(ctx, la, Xt, nt, mean, var, var_latent, precision, list,
                                   counter + 1, s, tptr, tpts, bsmax)))
      return st;
  }
  PredictArgs a;
  memset(&a, 0, sizeof(a));
  a.X = X;
  a.Xt = Xt;
  a.dtype = dtype;
  a.y = y;
  a.d = d;
  a.nbr = nbr;
  a.nt = nt;
  a.m = m;
  a.theta = dth;
  a.nu2 = nu2;
  a.mean = mean;
  a.var = var;
  a.var_latent = var_latent;
  a.dstat = ctx->d_status;
  a.counter = counter;
  a.gmat = nullptr;
  a.gmat_stride = 0;
  a.tptr = tptr;
  a.tpts = tpts;
  a.nmax = m + bsmax;
  if (list) {  // FP64 pass over the items the mixed kernel handed over
    a.list = list;
    a.list_n = counter + 1;
    a.counter = counter + 2;
  }
  const int N = m + bsmax;
  const size_t ub = (size_t)(d + 1) * (N + 1) * sizeof(double);
  const size_t mat = (size_t)(N + 1) * (N + 2) / 2 * sizeof(double);
  size_t smem = ub + mat;
  int grid;
  if (smem + 1024 <= ctx->smem_optin) {
    int per_sm = (int)std::max<size_t>(1, (228 * 1024) / (smem + 2048));
    grid = ctx->num_sms * std::min(per_sm, 4);
  } else {
    smem = ub;
    if (smem + 1024 > ctx->smem_optin)
      return fail(ctx, SBV_EUNSUPPORTED, "d=%d with m_pred=%d exceeds shared memory", d, m);
    grid = ctx->num_sms * 2;
    size_t stride = (mat / sizeof(double) + 31) & ~(size_t)31;
    double* g = (double*)ws_get(ctx, WS_GMAT64, stride * grid * sizeof(double), &st);
    if (!g) return st;
    a.gmat = g;
    a.gmat_stride = stride;
  }
  if (grid > nt) grid = (int)nt;
  SBV_CUDA_TRY(ctx, cudaFuncSetAttribute(predict_fp64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  predict_fp64_kernel<<<grid, LL_THREADS, smem, s>>>(a);
  SBV_LAUNCH_CHECK(ctx, "predict_fp64_kernel");
  return SBV_OK;
}

// Matern correlation at squared scaled distances d2 through the FP64 paths'
// arithmetic: r = sqrt(d2), then the closed form or the K_nu quadrature.
__global__ void __launch_bounds__(256) matern_fp64_eval_kernel(const double* d2, int64_t n,
                                                               int nu2, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = matern_fp64(sqrt(d2[i]), nu2);
}

int run_matern(sbv_ctx* ctx, int precision, int nu2, const double* d2, int64_t n, double* out,
               cudaStream_t s) {
  if (precision != SBV_PREC_FP64) return run_matern_df(ctx, nu2, d2, n, out, s);
  if (n == 0) return SBV_OK;
  const int64_t want = (n + 255) / 256;
  const int grid = (int)std::min<int64_t>(want, (int64_t)ctx->num_sms * 8);
  matern_fp64_eval_kernel<<<grid, 256, 0, s>>>(d2, n, nu2, out);
  SBV_CUDA_TRY(ctx, cudaGetLastError());
  return SBV_OK;
}

}  // namespace sbv
