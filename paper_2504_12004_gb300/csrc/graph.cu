// One likelihood evaluation captured as a CUDA graph, and the launch-shape
// autotuner (Sec. 5.4 batches all blocks of an evaluation into one batched
// launch; here one persistent kernel covers every (theta, block) item and the
// whole evaluation replays as one graph).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "block_common.cuh"
#include "mixed.cuh"
#include "sbv_internal.cuh"

using namespace sbv;

struct sbv_graph {
  sbv_ctx* ctx = nullptr;
  int B = 0, d = 0;
  int64_t bc = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ThetaDev* d_theta = nullptr;      // parameter rows read by the captured kernel
  ThetaDev* h_theta = nullptr;      // pinned staging of the rows
  cudaEvent_t staged = nullptr;     // recorded after the copy out of h_theta
  void* owned[8] = {};              // device buffers owned by the graph
};

namespace {

int check_loglik_args(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n,
                      int32_t d, const int64_t* ptr, const int32_t* pts, const int32_t* nbr,
                      const int32_t* cnt, int64_t bc, int32_t m, int32_t B, int32_t nu2,
                      int32_t precision) {
  if (!ctx) return SBV_EINVAL;
  if (!X || !y || !ptr || !pts || !cnt || (m > 0 && !nbr))
    return fail(ctx, SBV_EINVAL, "null pointer argument");
  if (dtype != SBV_F64 && dtype != SBV_F32) return fail(ctx, SBV_EINVAL, "bad dtype %d", dtype);
  if (n < 1 || d < 1 || d > SBV_MAX_DIM || bc < 1 || bc > n || m < 0)
    return fail(ctx, SBV_EINVAL, "bad sizes");
  if (B < 1) return fail(ctx, SBV_EINVAL, "B=%d must be >= 1", B);
  // as sbv_loglik: the captured FP64 kernel takes any nu2 in 1..SBV_MAX_NU2,
  // the mixed kernels the closed forms
  const bool closed = nu2 == 1 || nu2 == 3 || nu2 == 5 || nu2 == 7;
  if (precision == SBV_PREC_FP64 ? (nu2 < 1 || nu2 > SBV_MAX_NU2) : !closed)
    return fail(ctx, SBV_EINVAL, "nu2=%d: FP64 takes 1..%d, the mixed precisions {1,3,5,7}", nu2,
                SBV_MAX_NU2);
  if (precision != SBV_PREC_FP64 && precision != SBV_PREC_MIXED &&
      precision != SBV_PREC_MIXED_BF16)
    return fail(ctx, SBV_EINVAL, "precision=%d unknown", precision);
  if ((uint64_t)bc * (uint64_t)B >= 0xffffffffull)
    return fail(ctx, SBV_EUNSUPPORTED, "bc*B too large");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, SBV_ECUDA, "cudaSetDevice");
  return SBV_OK;
}

int check_theta_rows(sbv_ctx* ctx, const double* theta, int B, int d) {
  if (!theta) return fail(ctx, SBV_EINVAL, "theta is null");
  for (int b = 0; b < B; ++b) {
    const double* r = theta + (size_t)b * (2 + d);
    bool ok = r[0] > 0.0 && isfinite(r[0]) && r[1] >= 0.0 && isfinite(r[1]);
    for (int t = 0; t < d; ++t) ok = ok && r[2 + t] > 0.0 && isfinite(r[2 + t]);
    if (!ok) return fail(ctx, SBV_EINVAL, "theta row %d invalid", b);
  }
  return SBV_OK;
}

int own(sbv_graph* g, int slot, size_t bytes, void** out) {
  if (cudaMalloc(&g->owned[slot], bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(g->ctx, SBV_ENOMEM, "graph buffer of %zu bytes", bytes);
  }
  *out = g->owned[slot];
  return SBV_OK;
}

}  // namespace

extern "C" void sbv_loglik_graph_destroy(sbv_graph* g) {
  if (!g) return;
  cudaSetDevice(g->ctx->device);
  cudaDeviceSynchronize();
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->staged) cudaEventDestroy(g->staged);
  if (g->h_theta) cudaFreeHost(g->h_theta);
  for (void* p : g->owned)
    if (p) cudaFree(p);
  delete g;
}

extern "C" int sbv_loglik_graph_create(sbv_ctx* ctx, const void* X, int dtype, const double* y,
                                       int64_t n, int32_t d, const int64_t* ptr,
                                       const int32_t* pts, const int32_t* nbr, const int32_t* cnt,
                                       int64_t bc, int32_t m, int32_t nmax, int32_t B,
                                       int32_t nu2, int32_t precision, double* ll,
                                       double* block_terms, int32_t* status, sbv_graph** out) {
  int st = check_loglik_args(ctx, X, dtype, y, n, d, ptr, pts, nbr, cnt, bc, m, B, nu2, precision);
  if (st) return st;
  if (!ll || !out) return fail(ctx, SBV_EINVAL, "null pointer argument");
  *out = nullptr;
  cudaStream_t cap = nullptr;
  SBV_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  // the largest block sizes fix the mixed kernel's layout (one read at creation)
  int nmax_s = 0, bsmax = 0;
  if ((st = run_max_sizes(ctx, ptr, cnt, bc, &nmax_s, &bsmax, cap))) {
    cudaStreamDestroy(cap);
    return st;
  }
  if (nmax <= 0) nmax = nmax_s;
  if (nmax < nmax_s) bsmax = 0;   // a smaller hint: the blocks above it are reported, not held
  if (nmax > SBV_MAX_BLOCK_N) {
    cudaStreamDestroy(cap);
    return fail(ctx, SBV_EUNSUPPORTED, "a block has m_i + bs_i = %d > %d", nmax, SBV_MAX_BLOCK_N);
  }
  sbv_graph* g = new sbv_graph();
  g->ctx = ctx;
  g->B = B;
  g->d = d;
  g->bc = bc;
  auto bail = [&](int code) {
    cudaStreamDestroy(cap);
    sbv_loglik_graph_destroy(g);
    return code;
  };
  void* p = nullptr;
  if ((st = own(g, 0, (size_t)B * sizeof(ThetaDev), &p))) return bail(st);
  g->d_theta = (ThetaDev*)p;
  if (cudaMallocHost((void**)&g->h_theta, (size_t)B * sizeof(ThetaDev)) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->staged, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(ctx, SBV_ENOMEM, "pinned staging"));
  if ((st = own(g, 1, 64, &p))) return bail(st);
  unsigned int* counter = (unsigned int*)p;
  double* terms = block_terms;
  if (!terms) {
    if ((st = own(g, 2, (size_t)B * bc * sizeof(double), &p))) return bail(st);
    terms = (double*)p;
  }
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
  a.theta = g->d_theta;
  a.B = B;
  a.nu2 = nu2;
  a.ncap = nmax;
  a.terms = terms;
  a.status = status;
  a.dstat = ctx->d_status;
  a.counter = counter;
  const int64_t items = bc * (int64_t)B;
  const bool mixed = precision != SBV_PREC_FP64;
  MixedArgs P;
  MixedPlan mp;
  Fp64Plan fp;
  double* fb_gmat = nullptr;
  if (mixed) {
    memset(&P, 0, sizeof(P));
    P.a = a;
    if ((st = mixed_plan(ctx, nmax, m, bsmax, d, precision, false, items, &mp))) return bail(st);
    if (dtype == SBV_F64) {  // X is fixed: split it once, outside the graph
      if ((st = own(g, 3, (size_t)n * d * sizeof(float2), &p))) return bail(st);
      if ((st = mixed_split(ctx, X, dtype, n * d, (float2*)p, cap))) return bail(st);
      P.Xs = (const float2*)p;
    }
    if ((st = own(g, 4, mp.scratch_bytes(), &p))) return bail(st);
    P.gbase = (float*)p;
    // hand-over list and the FP64 kernel's global matrices (when its blocks
    // do not fit shared memory)
    if ((st = own(g, 6, (size_t)items * sizeof(unsigned int), &p))) return bail(st);
    P.fb_list = (unsigned int*)p;
    P.fb_count = counter + 1;
    if ((st = fp64_plan(ctx, nmax, d, items, &fp))) return bail(st);
    if (fp.gmat_stride) {
      if ((st = own(g, 7, fp.gmat_stride * fp.grid * sizeof(double), &p))) return bail(st);
      fb_gmat = (double*)p;
    }
    if ((st = mixed_prepare(ctx)) || (st = fp64_prepare(ctx))) return bail(st);
  } else {
    if ((st = fp64_plan(ctx, nmax, d, items, &fp))) return bail(st);
    if (fp.gmat_stride) {
      if ((st = own(g, 5, fp.gmat_stride * fp.grid * sizeof(double), &p))) return bail(st);
      a.gmat = (double*)p;
      a.gmat_stride = fp.gmat_stride;
    }
    if ((st = fp64_prepare(ctx))) return bail(st);
  }
  if (cudaStreamSynchronize(cap) != cudaSuccess) return bail(fail(ctx, SBV_ECUDA, "prepare"));
  // capture: reset the work counter, the block kernel, the deterministic sum
  SBV_CUDA_TRY(ctx, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  int cst = SBV_OK;
  // work counter, hand-over count, FP64 work counter
  if (cudaMemsetAsync(counter, 0, 3 * sizeof(unsigned int), cap) != cudaSuccess) cst = SBV_ECUDA;
  if (!cst) cst = mixed ? mixed_enqueue(ctx, P, mp, cap) : fp64_enqueue(ctx, a, fp, cap);
  if (!cst && mixed)
    cst = fp64_fallback_enqueue(ctx, a, nmax, P.fb_list, counter + 1, counter + 2, cap, fb_gmat);
  if (!cst) cst = reduce_enqueue(ctx, terms, bc, B, ll, cap);
  cudaError_t e = cudaStreamEndCapture(cap, &g->graph);
  if (cst) return bail(cst);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaStreamEndCapture"));
  e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "cudaGraphInstantiate"));
  cudaStreamDestroy(cap);
  *out = g;
  return SBV_OK;
}

extern "C" int sbv_loglik_graph_launch(sbv_graph* g, const double* theta, void* stream) {
  if (!g) return SBV_EINVAL;
  sbv_ctx* ctx = g->ctx;
  int st = check_theta_rows(ctx, theta, g->B, g->d);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  SBV_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  std::vector<ThetaDev> v = derive_theta_rows(theta, g->B, g->d);
  SBV_CUDA_TRY(ctx, cudaEventSynchronize(g->staged));  // previous copy out of the staging done
  memcpy(g->h_theta, v.data(), v.size() * sizeof(ThetaDev));
  SBV_CUDA_TRY(ctx, cudaMemcpyAsync(g->d_theta, g->h_theta, v.size() * sizeof(ThetaDev),
                                    cudaMemcpyHostToDevice, s));
  SBV_CUDA_TRY(ctx, cudaEventRecord(g->staged, s));
  SBV_CUDA_TRY(ctx, cudaGraphLaunch(g->exec, s));
  return SBV_OK;
}

// ---------------------------------------------------------------------------
// autotuner: time every launch shape once (after one warm-up) on the caller's
// structure and keep the fastest for later calls with the same key
// ---------------------------------------------------------------------------
extern "C" int sbv_autotune(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n,
                            int32_t d, const int64_t* ptr, const int32_t* pts,
                            const int32_t* nbr, const int32_t* cnt, int64_t bc, int32_t m,
                            int32_t nmax, const double* theta, int32_t B, int32_t nu2,
                            int32_t precision, int32_t* threads, int32_t* ctas_per_sm,
                            void* stream) {
  int st = check_loglik_args(ctx, X, dtype, y, n, d, ptr, pts, nbr, cnt, bc, m, B, nu2, precision);
  if (st) return st;
  if ((st = check_theta_rows(ctx, theta, B, d))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int nmax_s = 0, bsmax = 0;
  if ((st = run_max_sizes(ctx, ptr, cnt, bc, &nmax_s, &bsmax, s))) return st;
  if (nmax <= 0) nmax = nmax_s;
  std::vector<LaunchShape> shapes;
  if (precision == SBV_PREC_FP64) {
    for (int k = 1; k <= 4; ++k) shapes.push_back({256, k});
  } else {
    // launch shape x right-hand sides per column block of the residual and
    // the conditional system (the tile size the mixed kernel leaves open)
    for (int tile : {16, 32, 64}) {
      shapes.push_back({256, 2, tile});
      shapes.push_back({256, 1, tile});
      shapes.push_back({512, 1, tile});
    }
  }
  double* ll = (double*)ws_get(ctx, WS_TUNE, (size_t)B * sizeof(double), &st);
  if (!ll) return st;
  cudaEvent_t e0, e1;
  SBV_CUDA_TRY(ctx, cudaEventCreate(&e0));
  SBV_CUDA_TRY(ctx, cudaEventCreate(&e1));
  float best = INFINITY;
  LaunchShape pick = shapes[0];
  for (const LaunchShape& sh : shapes) {
    ctx->force = sh;
    float t = INFINITY;
    for (int rep = 0; rep < 3 && !st; ++rep) {
      cudaEventRecord(e0, s);
      // size hint 0: the call reads both sizes, as a graph created later does
      st = run_loglik(ctx, X, dtype, y, n, d, ptr, pts, nbr, cnt, bc, m, nmax == nmax_s ? 0 : nmax,
                      theta, B, nu2,
                      precision, ll, nullptr, nullptr, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = cuda_fail(ctx, cudaGetLastError(), "autotune");
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) t = std::min(t, ms);  // the first run of a shape is the warm-up
    }
    if (st == SBV_EUNSUPPORTED) {  // a shape the structure cannot use
      st = SBV_OK;
      continue;
    }
    if (st) break;
    if (t < best) {
      best = t;
      pick = sh;
    }
  }
  ctx->force = LaunchShape();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  TunedShape rec = {precision, 0, nmax, d, pick.threads, pick.per_sm, pick.tile};
  bool replaced = false;
  for (auto& t : ctx->tuned)
    if (t.precision == rec.precision && t.pred == rec.pred && t.ncap == rec.ncap && t.d == rec.d) {
      t = rec;
      replaced = true;
    }
  if (!replaced) ctx->tuned.push_back(rec);
  if (threads) *threads = pick.threads;
  if (ctas_per_sm) *ctas_per_sm = pick.per_sm;
  return sbv_sync_status(ctx, stream);
}

extern "C" int sbv_tuned_shape(sbv_ctx* ctx, int32_t precision, int32_t nmax, int32_t d,
                               int32_t* threads, int32_t* ctas_per_sm, int32_t* tile) {
  if (!ctx) return SBV_EINVAL;
  for (const auto& t : ctx->tuned)
    if (t.precision == precision && t.pred == 0 && t.ncap == nmax && t.d == d) {
      if (threads) *threads = t.threads;
      if (ctas_per_sm) *ctas_per_sm = t.per_sm;
      if (tile) *tile = t.tile;
      return SBV_OK;
    }
  return fail(ctx, SBV_EINVAL, "no autotuning record for precision %d, nmax %d, d %d", precision,
              nmax, d);
}
