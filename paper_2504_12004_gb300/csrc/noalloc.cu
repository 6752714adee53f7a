// sbv_loglik_fp64_noalloc: the FP64 block log-likelihood with every piece of
// scratch in one fixed device array of this file, so the call allocates
// nothing (no cudaMalloc, no cudaFree, no host allocation, no allocating
// library routine).
//
// Who needs it: code that may not allocate device memory while it runs --
// for example a serving loop whose device memory is owned by another
// allocator (a framework's caching allocator, or a fixed memory budget where
// a library-side cudaMalloc could fail or fragment it), or a real-time loop
// where the latency and implicit synchronisation of cudaMalloc/cudaFree are
// not acceptable.  They pass inputs and outputs; the library keeps its
// scratch in `g_noalloc_scratch` below, which every GPU that loads libsbv.so
// holds (about 8.1 MB) until the process exits.
//
// The kernels are those of sbv_loglik's FP64 path (loglik.cu), launched with
// pointers into the fixed array instead of the context workspace.
#include <math.h>
#include <string.h>

#include "block_common.cuh"
#include "sbv_internal.cuh"

namespace sbv {

// kernels of the FP64 path (defined in loglik.cu)
__global__ void loglik_fp64_kernel(LoglikArgs a);
__global__ void reduce_terms_kernel(const double* __restrict__ terms, int64_t bc,
                                    double* __restrict__ ll);
__global__ void max_n_kernel(const int64_t* __restrict__ ptr, const int32_t* __restrict__ cnt,
                             int64_t bc, int* __restrict__ out);

constexpr int NA_THREADS = 256;  // block size of loglik_fp64_kernel

// Layout of the fixed scratch array.
struct NoallocScratch {
  DevStatus status;                              // failure record (cleared per call)
  unsigned int counter;                          // work counter (cleared per call)
  int nmax;                                      // largest block size when computed here
  unsigned char pad[256 - sizeof(DevStatus) - 2 * sizeof(int)];
  ThetaDev theta[SBV_NOALLOC_MAX_THETA];         // derived parameter rows
  double terms[SBV_NOALLOC_MAX_TERMS];           // block terms when the caller passes none
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// Device address of the array, looked up once per device (with that device
// current) by cudaGetSymbolAddress; in host code the symbol itself is only a
// host-side stand-in and must never be passed to a kernel.
static NoallocScratch* g_scratch_addr[64];

static int scratch_for_current_device(NoallocScratch** out, int* device) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SBV_ECUDA;
  if (dev < 0 || dev >= 64) return SBV_EUNSUPPORTED;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SBV_ECUDA;
    g_scratch_addr[dev] = (NoallocScratch*)p;
  }
  *out = g_scratch_addr[dev];
  *device = dev;
  return SBV_OK;
}

}  // namespace sbv

using namespace sbv;

extern "C" int sbv_loglik_fp64_noalloc(const void* X, int dtype, const double* y, int64_t n,
                                       int32_t d, const int64_t* ptr, const int32_t* pts,
                                       const int32_t* nbr, const int32_t* cnt, int64_t bc,
                                       int32_t m, int32_t nmax, const double* theta, int32_t B,
                                       int32_t nu2, double* ll, double* block_terms,
                                       int32_t* status, void* stream) {
  // argument checks (same rules as sbv_loglik) and the limits of the fixed array
  if (!X || !y || !ptr || !pts || !cnt || !ll || !theta || (m > 0 && !nbr)) return SBV_EINVAL;
  if (dtype != SBV_F64 && dtype != SBV_F32) return SBV_EINVAL;
  if (n < 1 || d < 1 || d > SBV_MAX_DIM || bc < 1 || bc > n || m < 0 || nmax < 0) return SBV_EINVAL;
  // the FP64 kernel evaluates the closed forms and, for any other nu2, K_nu
  if (nu2 < 1 || nu2 > SBV_MAX_NU2) return SBV_EINVAL;
  if (B < 1 || B > SBV_NOALLOC_MAX_THETA) return SBV_EUNSUPPORTED;
  if (!block_terms && (uint64_t)bc * (uint64_t)B > (uint64_t)SBV_NOALLOC_MAX_TERMS)
    return SBV_EUNSUPPORTED;
  if ((uint64_t)bc * (uint64_t)B >= 0xffffffffull) return SBV_EUNSUPPORTED;
  for (int b = 0; b < B; ++b) {
    const double* r = theta + (size_t)b * (2 + d);
    if (!(r[0] > 0.0) || !isfinite(r[0]) || !(r[1] >= 0.0) || !isfinite(r[1])) return SBV_EINVAL;
    for (int t = 0; t < d; ++t)
      if (!(r[2 + t] > 0.0) || !isfinite(r[2 + t])) return SBV_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  NoallocScratch* S = nullptr;
  int dev = 0;
  int st = scratch_for_current_device(&S, &dev);
  if (st) return st;
  int sms = 0, optin = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return SBV_ECUDA;

  // largest block size (one small kernel and a read into a host stack variable)
  if (nmax == 0) {
    if (cudaMemsetAsync(&S->nmax, 0, sizeof(int), s) != cudaSuccess) return SBV_ECUDA;
    int g = (int)((bc + 255) / 256);
    if (g > sms * 8) g = sms * 8;
    max_n_kernel<<<g < 1 ? 1 : g, 256, 0, s>>>(ptr, cnt, bc, &S->nmax);
    if (cudaGetLastError() != cudaSuccess) return SBV_ECUDA;
    int h = 0;
    if (cudaMemcpyAsync(&h, &S->nmax, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return SBV_ECUDA;
    nmax = h;
  }
  if (nmax < 1 || nmax > SBV_MAX_BLOCK_N) return SBV_EUNSUPPORTED;
  // the matrix of every block must fit in shared memory (no global matrix scratch here)
  const size_t smem = (size_t)(d + 1) * (nmax + 1) * sizeof(double) +
                      (size_t)(nmax + 1) * (nmax + 2) / 2 * sizeof(double);
  if (smem + 1024 > (size_t)optin) return SBV_EUNSUPPORTED;

  // parameter rows: derived one at a time on the stack and copied into the
  // fixed array (a pageable copy is staged before cudaMemcpyAsync returns)
  for (int b = 0; b < B; ++b) {
    const double* r = theta + (size_t)b * (2 + d);
    ThetaDev t;
    memset(&t, 0, sizeof(t));
    t.sigma2 = r[0];
    t.tau2 = r[1];
    for (int q = 0; q < d; ++q) t.inv_beta[q] = 1.0 / r[2 + q];
    if (cudaMemcpyAsync(&S->theta[b], &t, sizeof(t), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return SBV_ECUDA;
  }
  // what must start at zero: the work counter and the failure record
  if (cudaMemsetAsync(&S->status, 0, sizeof(DevStatus) + sizeof(unsigned int), s) != cudaSuccess)
    return SBV_ECUDA;

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
  a.theta = S->theta;
  a.B = B;
  a.nu2 = nu2;
  a.ncap = nmax;
  a.terms = block_terms ? block_terms : S->terms;
  a.status = status;
  a.dstat = &S->status;
  a.counter = &S->counter;
  a.gmat = nullptr;
  a.gmat_stride = 0;
  int per_sm = (int)((228 * 1024) / (smem + 2048));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  int64_t grid = (int64_t)sms * per_sm;
  if (grid > bc * (int64_t)B) grid = bc * (int64_t)B;
  // the same limit sbv_loglik's FP64 path sets (the largest opt-in minus the
  // static shared memory), never this call's smaller size: the attribute is
  // per kernel and per process, and later sbv_loglik launches with larger
  // blocks rely on it
  if (cudaFuncSetAttribute(loglik_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - 1024) != cudaSuccess)
    return SBV_ECUDA;
  loglik_fp64_kernel<<<(int)grid, NA_THREADS, smem, s>>>(a);
  if (cudaGetLastError() != cudaSuccess) return SBV_ECUDA;
  reduce_terms_kernel<<<B, 1024, 0, s>>>(a.terms, bc, ll);
  if (cudaGetLastError() != cudaSuccess) return SBV_ECUDA;
  return SBV_OK;
}
