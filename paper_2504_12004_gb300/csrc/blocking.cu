// Scaling (Alg. 2), Random Anchor Clustering and Lloyd iterations (Alg. 3,
// K-means of Sec. 5.2), compaction and the random block order (Alg. 1 Step 2).
#include <cub/cub.cuh>
#include <algorithm>
#include <unordered_map>
#include <vector>

#include "dist.cuh"
#include "sbv_internal.cuh"

namespace sbv {

// ---------------------------------------------------------------------------
// Host-side random choices: SplitMix64 stream, Lemire's bounded draw and
// Fisher-Yates shuffles (the generator reading adopted for Alg. 1 and 3).
// ---------------------------------------------------------------------------
struct SplitMix64 {
  uint64_t state;
  explicit SplitMix64(uint64_t seed) : state(seed) {}
  uint64_t next() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  // uniform in [0, s): high word of x*s; reject while the low word < (2^64 - s) mod s
  uint64_t below(uint64_t s) {
    unsigned __int128 p = (unsigned __int128)next() * s;
    uint64_t low = (uint64_t)p;
    if (low < s) {
      uint64_t t = (0ull - s) % s;
      while (low < t) {
        p = (unsigned __int128)next() * s;
        low = (uint64_t)p;
      }
    }
    return (uint64_t)(p >> 64);
  }
};

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
struct BetaArg {
  double b[SBV_MAX_DIM];
};

template <typename T>
__global__ void scale_kernel(const T* __restrict__ X, int64_t n, int d, BetaArg beta,
                             double* __restrict__ Z) {
  int64_t total = n * d;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int t = (int)(i % d);
    Z[i] = __ddiv_rn((double)X[i], beta.b[t]);
  }
}

__global__ void absmax_kernel(const double* __restrict__ Z, int64_t total,
                              unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(Z[i]));
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void gather_rows_kernel(const double* __restrict__ Z, const int32_t* __restrict__ idx,
                                   int64_t k, int d, double* __restrict__ C) {
  int64_t total = k * d;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i / d;
    int t = (int)(i % d);
    C[i] = Z[(int64_t)idx[r] * d + t];
  }
}

// One thread per point: argmin over all centres of the exact FP64 distance,
// screened by float32 distances (two passes over centre tiles in shared memory).
constexpr int ASSIGN_THREADS = 256;
constexpr int ASSIGN_TILE = 128;

// Bounds for skipping points in later Lloyd iterations (Hamerly, "Making
// k-means even faster", SDM 2010): ub >= the distance to the assigned centre,
// lb <= the distance to every other centre, both for true distances with a
// relative slack that covers the rounding of the FP64 squared distances the
// argmin compares.  When ub < lb after the centres moved (ub grown by the
// assigned centre's move, lb shrunk by the largest move), the assigned centre
// is still the unique nearest one and the point keeps its block.
constexpr double kBoundSlack = 1e-12;

// list: when not NULL, the thread's point is list[g] for g < *list_n (the
// points whose bounds did not decide); ub/lb: when not NULL, the bounds of
// each assigned point are written.
template <int DM>
__global__ void __launch_bounds__(ASSIGN_THREADS)
assign_kernel(const double* __restrict__ Z, int64_t n, int d, const double* __restrict__ C,
              int64_t k, ScreenBound sb, const int32_t* __restrict__ old_blk,
              int32_t* __restrict__ blk, unsigned long long* __restrict__ changed,
              const int32_t* __restrict__ list, const unsigned int* __restrict__ list_n,
              double* __restrict__ ub, double* __restrict__ lb) {
  __shared__ float cf[ASSIGN_TILE * DM];
  const int64_t g = blockIdx.x * (int64_t)ASSIGN_THREADS + threadIdx.x;
  const int64_t nl = list ? (int64_t)*list_n : n;
  if (list && (int64_t)blockIdx.x * ASSIGN_THREADS >= nl) return;   // the whole CTA is idle
  int64_t i = g;
  bool live = g < nl;
  if (list) i = live ? (int64_t)list[g] : 0;
  float zf[DM];
#pragma unroll
  for (int t = 0; t < DM; ++t) zf[t] = (live && t < d) ? (float)Z[i * d + t] : 0.0f;

  // pass 1: smallest upper bound D32 + margin
  float best_ub = INFINITY;
  for (int64_t j0 = 0; j0 < k; j0 += ASSIGN_TILE) {
    int nt = (int)min((int64_t)ASSIGN_TILE, k - j0);
    __syncthreads();
    for (int e = threadIdx.x; e < nt * d; e += ASSIGN_THREADS) {
      int jj = e / d, t = e % d;
      cf[jj * DM + t] = (float)C[(j0 + jj) * d + t];
    }
    __syncthreads();
    if (live) {
      for (int jj = 0; jj < nt; ++jj) {
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < DM; ++t) {
          if (t < d) {
            float df = zf[t] - cf[jj * DM + t];
            acc = fmaf(df, df, acc);
          }
        }
        float ub = acc + screen_margin(acc, sb);
        best_ub = fminf(best_ub, ub);
      }
    }
  }
  // pass 2: exact FP64 distance for every centre whose lower bound can reach
  // best_ub; `second` bounds every other centre from below (exact values
  // where computed, the screen's lower bound elsewhere)
  double best = INFINITY, second = INFINITY;
  int64_t arg = 0;
  double zi[DM];
#pragma unroll
  for (int t = 0; t < DM; ++t) zi[t] = (live && t < d) ? Z[i * d + t] : 0.0;
  for (int64_t j0 = 0; j0 < k; j0 += ASSIGN_TILE) {
    int nt = (int)min((int64_t)ASSIGN_TILE, k - j0);
    __syncthreads();
    for (int e = threadIdx.x; e < nt * d; e += ASSIGN_THREADS) {
      int jj = e / d, t = e % d;
      cf[jj * DM + t] = (float)C[(j0 + jj) * d + t];
    }
    __syncthreads();
    if (live) {
      for (int jj = 0; jj < nt; ++jj) {
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < DM; ++t) {
          if (t < d) {
            float df = zf[t] - cf[jj * DM + t];
            acc = fmaf(df, df, acc);
          }
        }
        float lb32 = acc - screen_margin(acc, sb);
        if (lb32 <= best_ub) {
          double D = dist2_exact<DM>(zi, C + (j0 + jj) * d, d);
          if (D < best) {  // strict: ties keep the smaller index
            // the old best joins the others (a pruned centre's bound may
            // already be below it)
            second = fmin(second, best);
            best = D;
            arg = j0 + jj;
          } else {
            second = fmin(second, D);
          }
        } else {
          // the screen's lower bound, widened against its own float rounding
          second = fmin(second, (double)fmaxf(lb32, 0.0f) * (1.0 - 1e-6));
        }
      }
    }
  }
  if (live) {
    int32_t a = (int32_t)arg;
    if (old_blk && old_blk[i] != a) atomicAdd(changed, 1ull);
    blk[i] = a;
    if (ub) {
      ub[i] = sqrt(best) * (1.0 + kBoundSlack);
      lb[i] = sqrt(second) * (1.0 - kBoundSlack);
    }
  }
}

// How far each centre moved (rounded up), and the largest move.
__global__ void centre_move_kernel(const double* __restrict__ Cold, const double* __restrict__ Cnew,
                                   int64_t k, int d, double* __restrict__ delta,
                                   unsigned long long* __restrict__ dmax) {
  double m = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < k;
       j += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < d; ++t) {
      const double q = Cnew[j * d + t] - Cold[j * d + t];
      s = fma(q, q, s);
    }
    const double v = sqrt(s) * (1.0 + kBoundSlack) + 1e-300;
    delta[j] = v;
    m = fmax(m, v);
  }
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(dmax, (unsigned long long)__double_as_longlong(m));
}

// Move the bounds with the centres; list the points they no longer decide.
__global__ void bound_filter_kernel(int64_t n, const int32_t* __restrict__ blk,
                                    const double* __restrict__ delta,
                                    const unsigned long long* __restrict__ dmax,
                                    double* __restrict__ ub, double* __restrict__ lb,
                                    int32_t* __restrict__ list, unsigned int* __restrict__ list_n) {
  const double dm = __longlong_as_double((long long)*dmax);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double u = ub[i] + delta[blk[i]];
    const double l = lb[i] - dm;
    ub[i] = u;
    lb[i] = l;
    if (!(u < l)) list[atomicAdd(list_n, 1u)] = (int32_t)i;
  }
}

// Alg. 2: slab of each point, int(x_dmax * P) on the unscaled coordinate
// (FP64 product, floor), clamped to [0, P-1].
template <typename T>
__global__ void slab_kernel(const T* __restrict__ X, int64_t n, int d, int dmax, int P,
                            int32_t* __restrict__ slab) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double q = floor(__dmul_rn((double)X[i * d + dmax], (double)P));
    slab[i] = q >= (double)(P - 1) ? P - 1 : (q > 0.0 ? (int32_t)q : 0);
  }
}

// Assignment inside slabs (Alg. 3 per partition): the thread of sorted
// position i handles point order[i]; its candidates are the centres
// [cstart[s], cstart[s+1]) of its slab s.  Points are sorted by slab, so a
// CTA usually meets one slab; centre tiles cover the union of its slabs'
// ranges and every thread skips the centres of other slabs.  Same two-pass
// screen and exact FP64 decision (ties to the smaller index) as assign_kernel.
template <int DM>
__global__ void __launch_bounds__(ASSIGN_THREADS)
assign_slab_kernel(const double* __restrict__ Z, int64_t n, int d, const double* __restrict__ C,
                   const int32_t* __restrict__ order, const int32_t* __restrict__ pslab,
                   const int64_t* __restrict__ cstart, ScreenBound sb,
                   const int32_t* __restrict__ old_blk, int32_t* __restrict__ blk,
                   unsigned long long* __restrict__ changed) {
  __shared__ float cf[ASSIGN_TILE * DM];
  __shared__ unsigned long long s_lo, s_hi;
  const int64_t i = blockIdx.x * (int64_t)ASSIGN_THREADS + threadIdx.x;
  const bool live = i < n;
  const int64_t p = live ? (int64_t)order[i] : 0;
  int64_t c0 = 0, c1 = 0;
  if (live) {
    const int sl = pslab[p];
    c0 = cstart[sl];
    c1 = cstart[sl + 1];
  }
  if (threadIdx.x == 0) {
    s_lo = ~0ull;
    s_hi = 0ull;
  }
  __syncthreads();
  if (live && c1 > c0) {
    atomicMin(&s_lo, (unsigned long long)c0);
    atomicMax(&s_hi, (unsigned long long)c1);
  }
  __syncthreads();
  const int64_t lo = (int64_t)s_lo, hi = (int64_t)s_hi;
  float zf[DM];
#pragma unroll
  for (int t = 0; t < DM; ++t) zf[t] = (live && t < d) ? (float)Z[p * d + t] : 0.0f;
  float best_ub = INFINITY;
  for (int64_t j0 = lo; j0 < hi; j0 += ASSIGN_TILE) {
    const int nt = (int)min((int64_t)ASSIGN_TILE, hi - j0);
    __syncthreads();
    for (int e = threadIdx.x; e < nt * d; e += ASSIGN_THREADS) {
      const int jj = e / d, t = e % d;
      cf[jj * DM + t] = (float)C[(j0 + jj) * d + t];
    }
    __syncthreads();
    if (live) {
      for (int jj = 0; jj < nt; ++jj) {
        const int64_t j = j0 + jj;
        if (j < c0 || j >= c1) continue;
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < DM; ++t) {
          if (t < d) {
            const float df = zf[t] - cf[jj * DM + t];
            acc = fmaf(df, df, acc);
          }
        }
        best_ub = fminf(best_ub, acc + screen_margin(acc, sb));
      }
    }
  }
  double best = INFINITY;
  int64_t arg = c0;
  double zi[DM];
#pragma unroll
  for (int t = 0; t < DM; ++t) zi[t] = (live && t < d) ? Z[p * d + t] : 0.0;
  for (int64_t j0 = lo; j0 < hi; j0 += ASSIGN_TILE) {
    const int nt = (int)min((int64_t)ASSIGN_TILE, hi - j0);
    __syncthreads();
    for (int e = threadIdx.x; e < nt * d; e += ASSIGN_THREADS) {
      const int jj = e / d, t = e % d;
      cf[jj * DM + t] = (float)C[(j0 + jj) * d + t];
    }
    __syncthreads();
    if (live) {
      for (int jj = 0; jj < nt; ++jj) {
        const int64_t j = j0 + jj;
        if (j < c0 || j >= c1) continue;
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < DM; ++t) {
          if (t < d) {
            const float df = zf[t] - cf[jj * DM + t];
            acc = fmaf(df, df, acc);
          }
        }
        if (acc - screen_margin(acc, sb) <= best_ub) {
          const double D = dist2_exact<DM>(zi, C + j * d, d);
          if (D < best) {  // strict: ties keep the smaller index
            best = D;
            arg = j;
          }
        }
      }
    }
  }
  if (live) {
    const int32_t a = (int32_t)arg;
    if (old_blk && old_blk[p] != a) atomicAdd(changed, 1ull);
    blk[p] = a;
  }
}

__global__ void take_kernel(const int32_t* __restrict__ src, const int64_t* __restrict__ pos,
                            int64_t k, int32_t* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < k;
       j += (int64_t)gridDim.x * blockDim.x)
    out[j] = src[pos[j]];
}

__global__ void iota_kernel(int32_t* __restrict__ v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (int32_t)i;
}

__global__ void count_kernel(const int32_t* __restrict__ keys, int64_t n,
                             int64_t* __restrict__ counts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd((unsigned long long*)&counts[keys[i]], 1ull);
}

// Mean of each block's members, summed one by one in increasing point index.
// One thread per (block, dimension).  Empty blocks keep `prev` (if given).
__global__ void centroid_kernel(const double* __restrict__ Z, int d,
                                const int64_t* __restrict__ ptr,
                                const int32_t* __restrict__ pts, int64_t k,
                                const double* __restrict__ prev, double* __restrict__ C) {
  int64_t total = k * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = e / d;
    int t = (int)(e % d);
    int64_t a = ptr[j], b = ptr[j + 1];
    if (b == a) {
      C[e] = prev ? prev[e] : __longlong_as_double(0x7ff8000000000000ll);
      continue;
    }
    double s = 0.0;
    for (int64_t q = a; q < b; ++q) s = __dadd_rn(s, Z[(int64_t)pts[q] * d + t]);
    C[e] = __ddiv_rn(s, (double)(b - a));
  }
}

__global__ void used_kernel(const int64_t* __restrict__ counts, int64_t k,
                            int32_t* __restrict__ used) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < k;
       j += (int64_t)gridDim.x * blockDim.x)
    used[j] = counts[j] > 0 ? 1 : 0;
}

// remap: new id of used block j = exclusive prefix of used flags
__global__ void compact_kernel(const int64_t* __restrict__ ptr_old, const int32_t* __restrict__ used,
                               const int32_t* __restrict__ newid, int64_t k, int64_t n,
                               int64_t* __restrict__ ptr_new, int64_t bc_eff) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < k;
       j += (int64_t)gridDim.x * blockDim.x)
    if (used[j]) ptr_new[newid[j]] = ptr_old[j];
  if (blockIdx.x == 0 && threadIdx.x == 0) ptr_new[bc_eff] = n;
}

__global__ void relabel_kernel(int32_t* __restrict__ blk, int64_t n,
                               const int32_t* __restrict__ newid) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    blk[i] = newid[blk[i]];
}

static int grid_for(int64_t work, int threads, int sms) {
  int64_t g = (work + threads - 1) / threads;
  int64_t cap = (int64_t)sms * 32;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

int scale_points(sbv_ctx* ctx, const void* X, int dtype, int64_t n, int d, const double*,
                 const double* h_beta, double* Z, cudaStream_t s) {
  BetaArg ba;
  for (int t = 0; t < d; ++t) ba.b[t] = h_beta[t];
  int g = grid_for(n * d, 256, ctx->num_sms);
  if (dtype == SBV_F64)
    scale_kernel<double><<<g, 256, 0, s>>>((const double*)X, n, d, ba, Z);
  else
    scale_kernel<float><<<g, 256, 0, s>>>((const float*)X, n, d, ba, Z);
  SBV_LAUNCH_CHECK(ctx, "scale_kernel");
  return SBV_OK;
}

// Upper bound of |coordinate| over Z (n x d), for the float32 screening margin.
int absmax(sbv_ctx* ctx, const double* Z, int64_t total, double* out, cudaStream_t s) {
  int st = 0;
  unsigned long long* d = (unsigned long long*)ws_get(ctx, WS_SMALL, 64, &st);
  if (!d) return st;
  SBV_CUDA_TRY(ctx, cudaMemsetAsync(d, 0, 8, s));
  absmax_kernel<<<grid_for(total, 256, ctx->num_sms), 256, 0, s>>>(Z, total, d);
  SBV_LAUNCH_CHECK(ctx, "absmax_kernel");
  unsigned long long h = 0;
  SBV_CUDA_TRY(ctx, cudaMemcpyAsync(&h, d, 8, cudaMemcpyDeviceToHost, s));
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  double v;
  memcpy(&v, &h, 8);
  *out = v;
  return SBV_OK;
}

static int launch_assign(sbv_ctx* ctx, const double* Z, int64_t n, int d, const double* C,
                         int64_t k, ScreenBound sb, const int32_t* old_blk, int32_t* blk,
                         unsigned long long* changed, cudaStream_t s,
                         const int32_t* list = nullptr, const unsigned int* list_n = nullptr,
                         double* ub = nullptr, double* lb = nullptr) {
  int g = (int)((n + ASSIGN_THREADS - 1) / ASSIGN_THREADS);
#define SBV_ASSIGN(DM)                                                                     \
  assign_kernel<DM><<<g, ASSIGN_THREADS, 0, s>>>(Z, n, d, C, k, sb, old_blk, blk, changed, \
                                                 list, list_n, ub, lb)
  if (d <= 4) SBV_ASSIGN(4);
  else if (d <= 8) SBV_ASSIGN(8);
  else if (d <= 12) SBV_ASSIGN(12);
  else if (d <= 16) SBV_ASSIGN(16);
  else if (d <= 24) SBV_ASSIGN(24);
  else if (d <= 32) SBV_ASSIGN(32);
  else SBV_ASSIGN(64);
#undef SBV_ASSIGN
  SBV_LAUNCH_CHECK(ctx, "assign_kernel");
  return SBV_OK;
}

static int launch_assign_slab(sbv_ctx* ctx, const double* Z, int64_t n, int d, const double* C,
                              const int32_t* order, const int32_t* pslab, const int64_t* cstart,
                              ScreenBound sb, const int32_t* old_blk, int32_t* blk,
                              unsigned long long* changed, cudaStream_t s) {
  int g = (int)((n + ASSIGN_THREADS - 1) / ASSIGN_THREADS);
#define SBV_ASSIGN(DM)                                                                   \
  assign_slab_kernel<DM><<<g, ASSIGN_THREADS, 0, s>>>(Z, n, d, C, order, pslab, cstart, sb, \
                                                      old_blk, blk, changed)
  if (d <= 4) SBV_ASSIGN(4);
  else if (d <= 8) SBV_ASSIGN(8);
  else if (d <= 12) SBV_ASSIGN(12);
  else if (d <= 16) SBV_ASSIGN(16);
  else if (d <= 24) SBV_ASSIGN(24);
  else if (d <= 32) SBV_ASSIGN(32);
  else SBV_ASSIGN(64);
#undef SBV_ASSIGN
  SBV_LAUNCH_CHECK(ctx, "assign_slab_kernel");
  return SBV_OK;
}

// Anchors per slab (the reading for Alg. 3's k_p): one for every non-empty
// slab, the remaining bc - #non-empty in proportion to the slab sizes by the
// largest remainder (exact integers, ties to the lower slab), capped at the
// slab's size.
static std::vector<int64_t> slab_quota(const std::vector<int64_t>& cnt, int64_t bc) {
  const size_t P = cnt.size();
  int64_t n = 0, nonempty = 0;
  for (int64_t c : cnt) {
    n += c;
    nonempty += c > 0;
  }
  std::vector<int64_t> k(P, 0), rem(P, 0);
  const int64_t R = std::max<int64_t>(bc - nonempty, 0);
  int64_t given = 0;
  for (size_t q = 0; q < P; ++q) {
    const unsigned __int128 prod = (unsigned __int128)R * (uint64_t)cnt[q];
    const int64_t base = (int64_t)(prod / (uint64_t)n);
    rem[q] = (int64_t)(prod % (uint64_t)n);
    k[q] = (cnt[q] > 0 ? 1 : 0) + base;
    given += base;
  }
  std::vector<size_t> ord(P);
  for (size_t q = 0; q < P; ++q) ord[q] = q;
  std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return rem[a] > rem[b]; });
  for (int64_t e = 0; e < R - given && e < (int64_t)P; ++e) k[ord[e]] += 1;
  for (size_t q = 0; q < P; ++q) k[q] = std::min(k[q], cnt[q]);
  return k;
}

// First k entries of a Fisher-Yates shuffle of [0, n) (step j swaps a[j] and
// a[j + U(n - j)]), from the caller's stream.
static void partial_shuffle(int64_t n, int64_t k, SplitMix64& rng, int64_t* out) {
  std::unordered_map<int64_t, int64_t> sw;
  sw.reserve((size_t)k * 2);
  auto get = [&](int64_t i) {
    auto it = sw.find(i);
    return it == sw.end() ? i : it->second;
  };
  for (int64_t j = 0; j < k; ++j) {
    const int64_t r = j + (int64_t)rng.below((uint64_t)(n - j));
    const int64_t aj = get(j), ar = get(r);
    sw[j] = ar;
    sw[r] = aj;
    out[j] = ar;
  }
}

// Sort point ids by block (stable: increasing index inside a block) and build
// counts and CSR offsets for k blocks.
static int group_by_block(sbv_ctx* ctx, const int32_t* blk, int64_t n, int64_t k,
                          int32_t* ids_tmp, int32_t* keys_out, int32_t* pts,
                          int64_t* counts, int64_t* ptr, cudaStream_t s) {
  int st = 0;
  iota_kernel<<<grid_for(n, 256, ctx->num_sms), 256, 0, s>>>(ids_tmp, n);
  int end_bit = 1;
  while ((1ll << end_bit) < k) ++end_bit;
  size_t tb = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tb, blk, keys_out, ids_tmp, pts, (int)n, 0, end_bit, s);
  size_t tb2 = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tb2, counts, ptr, (int)(k + 1), s);
  void* tmp = ws_get(ctx, WS_CUB, std::max(tb, tb2), &st);
  if (!tmp) return st;
  SBV_CUDA_TRY(ctx, cub::DeviceRadixSort::SortPairs(tmp, tb, blk, keys_out, ids_tmp, pts, (int)n,
                                                    0, end_bit, s));
  SBV_CUDA_TRY(ctx, cudaMemsetAsync(counts, 0, (k + 1) * sizeof(int64_t), s));
  count_kernel<<<grid_for(n, 256, ctx->num_sms), 256, 0, s>>>(blk, n, counts);
  SBV_LAUNCH_CHECK(ctx, "count_kernel");
  SBV_CUDA_TRY(ctx, cub::DeviceScan::ExclusiveSum(tmp, tb2, counts, ptr, (int)(k + 1), s));
  return SBV_OK;
}

int run_blocking(sbv_ctx* ctx, const double* Z, const void* X, int dtype, const double* h_beta,
                 int64_t n, int d, int64_t bc, int kmeans_iters, uint64_t seed, int partitions,
                 int32_t* blk, int64_t* ptr, int32_t* pts, int32_t* rank, double* centres,
                 int64_t* bc_eff, cudaStream_t s, const int64_t* h_anchors) {
  int st = 0;
  // workspace: two centre buffers, old assignment, sort scratch, counts, ptr
  size_t cbytes = (size_t)bc * d * sizeof(double);
  char* wsA = (char*)ws_get(ctx, WS_CENTRES, 2 * cbytes + 256, &st);
  if (!wsA) return st;
  double* Ca = (double*)wsA;
  double* Cb = (double*)(wsA + ((cbytes + 255) / 256) * 256);
  char* wsB = (char*)ws_get(ctx, WS_SORT_A, (size_t)n * 3 * sizeof(int32_t) + 1024, &st);
  if (!wsB) return st;
  int32_t* old_blk = (int32_t*)wsB;
  int32_t* ids_tmp = old_blk + n;
  int32_t* keys_out = ids_tmp + n;
  char* wsC = (char*)ws_get(ctx, WS_SORT_B, (size_t)(bc + 1) * (2 * sizeof(int64_t) + 2 * sizeof(int32_t)) + 1024, &st);
  if (!wsC) return st;
  int64_t* counts = (int64_t*)wsC;
  int64_t* ptr_tmp = counts + (bc + 1);
  int32_t* used = (int32_t*)(ptr_tmp + (bc + 1));
  int32_t* newid = used + (bc + 1);
  unsigned long long* changed = (unsigned long long*)ws_get(ctx, WS_SMALL, 64, &st);
  if (!changed) return st;

  double M = 0.0;
  if ((st = absmax(ctx, Z, n * d, &M, s))) return st;
  ScreenBound sb = make_screen(M, d);

  SplitMix64 rng(seed);
  int32_t* d_anchor = newid;  // reuse (bc entries) before compaction needs it
  // partitioned blocking (Alg. 2 then Alg. 3 per slab): slab of every point,
  // points sorted by slab, anchors drawn slab by slab
  int32_t* pslab = nullptr;
  int32_t* sorder = nullptr;
  int64_t* cstart = nullptr;
  if (partitions > 1) {
    const int P = partitions;
    char* wsD = (char*)ws_get(ctx, WS_SORT_C, (size_t)n * 3 * sizeof(int32_t) + (size_t)(P + 1) * 16 + 1024, &st);
    if (!wsD) return st;
    pslab = (int32_t*)wsD;
    sorder = pslab + n;
    int32_t* skeys = sorder + n;
    int64_t* scount = (int64_t*)(((uintptr_t)(skeys + n) + 15) & ~(uintptr_t)15);
    cstart = scount + (P + 1);
    int dmax = 0;
    for (int t = 1; t < d; ++t)
      if (1.0 / h_beta[t] > 1.0 / h_beta[dmax]) dmax = t;
    const int g = grid_for(n, 256, ctx->num_sms);
    if (dtype == SBV_F64)
      slab_kernel<double><<<g, 256, 0, s>>>((const double*)X, n, d, dmax, P, pslab);
    else
      slab_kernel<float><<<g, 256, 0, s>>>((const float*)X, n, d, dmax, P, pslab);
    SBV_LAUNCH_CHECK(ctx, "slab_kernel");
    // stable sort of point ids by slab and slab sizes
    if ((st = group_by_block(ctx, pslab, n, P, ids_tmp, skeys, sorder, scount, ptr_tmp, s)))
      return st;
    std::vector<int64_t> cnt(P), off(P + 1);
    SBV_CUDA_TRY(ctx, cudaMemcpyAsync(cnt.data(), scount, P * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    off[0] = 0;
    for (int q = 0; q < P; ++q) off[q + 1] = off[q] + cnt[q];
    const std::vector<int64_t> kq = slab_quota(cnt, bc);
    std::vector<int64_t> cs(P + 1, 0), pos;
    for (int q = 0; q < P; ++q) cs[q + 1] = cs[q] + kq[q];
    const int64_t K = cs[P];
    pos.resize((size_t)K);
    for (int q = 0; q < P; ++q) {
      if (kq[q] == 0) continue;
      partial_shuffle(cnt[q], kq[q], rng, pos.data() + cs[q]);
      for (int64_t j = cs[q]; j < cs[q + 1]; ++j) pos[j] += off[q];
    }
    int64_t* d_pos = (int64_t*)ws_get(ctx, WS_EXTRA, (size_t)K * sizeof(int64_t) + 64, &st);
    if (!d_pos) return st;
    SBV_CUDA_TRY(ctx, cudaMemcpyAsync(d_pos, pos.data(), K * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    SBV_CUDA_TRY(ctx, cudaMemcpyAsync(cstart, cs.data(), (P + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    take_kernel<<<grid_for(K, 256, ctx->num_sms), 256, 0, s>>>(sorder, d_pos, K, d_anchor);
    SBV_LAUNCH_CHECK(ctx, "take_kernel");
    SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));  // host vectors copied before they go
    bc = K;
  } else {
    // RAC anchors: first bc entries of a Fisher-Yates shuffle of [0, n), or
    // the caller's (one partition of a distributed blocking)
    std::vector<int64_t> a64(bc);
    if (h_anchors)
      std::copy(h_anchors, h_anchors + bc, a64.begin());
    else
      partial_shuffle(n, bc, rng, a64.data());
    std::vector<int32_t> anchors(a64.begin(), a64.end());
    SBV_CUDA_TRY(ctx, cudaMemcpyAsync(d_anchor, anchors.data(), bc * sizeof(int32_t),
                                      cudaMemcpyHostToDevice, s));
    SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  }
  gather_rows_kernel<<<grid_for(bc * d, 256, ctx->num_sms), 256, 0, s>>>(Z, d_anchor, bc, d, Ca);
  SBV_LAUNCH_CHECK(ctx, "gather_rows_kernel");
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));  // anchors buffer reused below

  // flat blocking with Lloyd iterations: bounds let later assignments skip
  // the points whose block cannot change (Hamerly); the slab-partitioned
  // assignment scans every centre of the point's slab
  double* bnd_u = nullptr;
  double* bnd_l = nullptr;
  double* delta = nullptr;
  int32_t* blist = nullptr;
  unsigned int* blist_n = nullptr;
  unsigned long long* dmax = nullptr;
  if (!pslab && kmeans_iters > 0) {
    char* wb = (char*)ws_get(ctx, WS_BOUNDS,
                             (size_t)n * (2 * sizeof(double) + sizeof(int32_t)) +
                                 (size_t)bc * sizeof(double) + 256, &st);
    if (!wb) return st;
    bnd_u = (double*)wb;
    bnd_l = bnd_u + n;
    delta = bnd_l + n;
    blist = (int32_t*)(delta + bc);
    blist_n = (unsigned int*)(changed + 1);
    dmax = changed + 2;
  }
  auto assign = [&](const double* Cc, const int32_t* old, int32_t* out, bool listed) {
    return pslab ? launch_assign_slab(ctx, Z, n, d, Cc, sorder, pslab, cstart, sb, old, out, changed, s)
                 : launch_assign(ctx, Z, n, d, Cc, bc, sb, old, out, changed, s,
                                 listed ? blist : nullptr, listed ? blist_n : nullptr, bnd_u,
                                 bnd_l);
  };
  if ((st = assign(Ca, nullptr, blk, false))) return st;
  double* C = Ca;
  double* Cn = Cb;
  for (int it = 0; it < kmeans_iters; ++it) {
    if ((st = group_by_block(ctx, blk, n, bc, ids_tmp, keys_out, pts, counts, ptr_tmp, s)))
      return st;
    centroid_kernel<<<grid_for(bc * d, 128, ctx->num_sms), 128, 0, s>>>(Z, d, ptr_tmp, pts, bc,
                                                                         C, Cn);
    SBV_LAUNCH_CHECK(ctx, "centroid_kernel");
    if (bnd_u) {
      SBV_CUDA_TRY(ctx, cudaMemsetAsync(blist_n, 0, 16, s));   // list count and largest move
      centre_move_kernel<<<grid_for(bc, 256, ctx->num_sms), 256, 0, s>>>(C, Cn, bc, d, delta,
                                                                         dmax);
      SBV_LAUNCH_CHECK(ctx, "centre_move_kernel");
      bound_filter_kernel<<<grid_for(n, 256, ctx->num_sms), 256, 0, s>>>(
          n, blk, delta, dmax, bnd_u, bnd_l, blist, blist_n);
      SBV_LAUNCH_CHECK(ctx, "bound_filter_kernel");
    }
    std::swap(C, Cn);
    SBV_CUDA_TRY(ctx, cudaMemcpyAsync(old_blk, blk, n * sizeof(int32_t),
                                      cudaMemcpyDeviceToDevice, s));
    SBV_CUDA_TRY(ctx, cudaMemsetAsync(changed, 0, 8, s));
    if ((st = assign(C, old_blk, blk, bnd_u != nullptr))) return st;
    unsigned long long h_changed = 0;
    SBV_CUDA_TRY(ctx, cudaMemcpyAsync(&h_changed, changed, 8, cudaMemcpyDeviceToHost, s));
    SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (h_changed == 0) break;
  }
  // final grouping, compaction of empty blocks
  if ((st = group_by_block(ctx, blk, n, bc, ids_tmp, keys_out, pts, counts, ptr_tmp, s)))
    return st;
  used_kernel<<<grid_for(bc, 256, ctx->num_sms), 256, 0, s>>>(counts, bc, used);
  SBV_LAUNCH_CHECK(ctx, "used_kernel");
  {
    size_t tb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, used, newid, (int)bc, s);
    void* tmp = ws_get(ctx, WS_CUB, tb, &st);
    if (!tmp) return st;
    SBV_CUDA_TRY(ctx, cub::DeviceScan::ExclusiveSum(tmp, tb, used, newid, (int)bc, s));
  }
  int32_t last_new = 0, last_used = 0;
  SBV_CUDA_TRY(ctx, cudaMemcpyAsync(&last_new, newid + bc - 1, 4, cudaMemcpyDeviceToHost, s));
  SBV_CUDA_TRY(ctx, cudaMemcpyAsync(&last_used, used + bc - 1, 4, cudaMemcpyDeviceToHost, s));
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  int64_t k_eff = (int64_t)last_new + last_used;
  compact_kernel<<<grid_for(bc, 256, ctx->num_sms), 256, 0, s>>>(ptr_tmp, used, newid, bc, n, ptr,
                                                                 k_eff);
  SBV_LAUNCH_CHECK(ctx, "compact_kernel");
  relabel_kernel<<<grid_for(n, 256, ctx->num_sms), 256, 0, s>>>(blk, n, newid);
  SBV_LAUNCH_CHECK(ctx, "relabel_kernel");
  centroid_kernel<<<grid_for(k_eff * d, 128, ctx->num_sms), 128, 0, s>>>(Z, d, ptr, pts, k_eff,
                                                                         nullptr, centres);
  SBV_LAUNCH_CHECK(ctx, "centroid_kernel");
  *bc_eff = k_eff;
  if (!rank) {   // anchored blocking: the caller orders the blocks
    SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return SBV_OK;
  }
  // random block order: full Fisher-Yates shuffle from the same stream
  std::vector<int32_t> perm(k_eff), rk(k_eff);
  for (int64_t j = 0; j < k_eff; ++j) perm[j] = (int32_t)j;
  for (int64_t j = 0; j + 1 < k_eff; ++j) {
    int64_t r = j + (int64_t)rng.below((uint64_t)(k_eff - j));
    std::swap(perm[j], perm[r]);
  }
  for (int64_t r = 0; r < k_eff; ++r) rk[perm[r]] = (int32_t)r;
  SBV_CUDA_TRY(ctx, cudaMemcpyAsync(rank, rk.data(), k_eff * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s));
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  *bc_eff = k_eff;
  return SBV_OK;
}

// Slab of every point (Alg. 2) on its own: the routing step of a distributed
// blocking.
int run_slabs(sbv_ctx* ctx, const void* X, int dtype, int64_t n, int d, const double* h_beta,
              int P, int32_t* slab, cudaStream_t s) {
  int dmax = 0;
  for (int t = 1; t < d; ++t)
    if (1.0 / h_beta[t] > 1.0 / h_beta[dmax]) dmax = t;
  if (n == 0) return SBV_OK;
  const int g = grid_for(n, 256, ctx->num_sms);
  if (dtype == SBV_F64)
    slab_kernel<double><<<g, 256, 0, s>>>((const double*)X, n, d, dmax, P, slab);
  else
    slab_kernel<float><<<g, 256, 0, s>>>((const float*)X, n, d, dmax, P, slab);
  SBV_LAUNCH_CHECK(ctx, "slab_kernel");
  return SBV_OK;
}

// Replay of the random choices of a partitioned blocking from the slab sizes
// alone (the draws depend on nothing else): anchors per slab and their
// positions, then, given the number of non-empty blocks, the block order.
int rac_plan(uint64_t seed, int P, const int64_t* counts, int64_t bc, int64_t* quota,
             int64_t* pos, int64_t k_eff, int32_t* rank) {
  std::vector<int64_t> cnt(counts, counts + P);
  const std::vector<int64_t> kq = slab_quota(cnt, bc);
  SplitMix64 rng(seed);
  int64_t o = 0;
  for (int q = 0; q < P; ++q) {
    if (quota) quota[q] = kq[q];
    if (kq[q] == 0) continue;
    std::vector<int64_t> tmp((size_t)kq[q]);
    partial_shuffle(cnt[q], kq[q], rng, tmp.data());
    if (pos) std::copy(tmp.begin(), tmp.end(), pos + o);
    o += kq[q];
  }
  if (rank) {
    std::vector<int32_t> perm((size_t)k_eff);
    for (int64_t j = 0; j < k_eff; ++j) perm[j] = (int32_t)j;
    for (int64_t j = 0; j + 1 < k_eff; ++j) {
      const int64_t r = j + (int64_t)rng.below((uint64_t)(k_eff - j));
      std::swap(perm[j], perm[r]);
    }
    for (int64_t r = 0; r < k_eff; ++r) rank[perm[r]] = (int32_t)r;
  }
  return SBV_OK;
}

}  // namespace sbv
