// Earlier-ordered m nearest neighbours of every block (Alg. 4; Eq.
// mmsearchingBV) and the all-points neighbour search of prediction (Sec. 4.2).
//
// Design: points are laid out in block-rank order, so the candidates of the
// block with rank r are exactly the prefix [0, rptr[r]) of that layout.  One
// CTA serves KNN_Q queries of consecutive rank and streams their common
// prefix through shared memory once (float32 structure-of-arrays tiles);
// every warp owns KNN_QW queries and keeps, per query, a buffer of exact keys
// (FP64 squared distance, point index).  A candidate enters a buffer only if
// its float32 distance can still beat the query's current m-th key (rigorous
// bound from dist.cuh) and its exact key does; a full buffer is sorted by the
// owning warp and cut back to m keys, which tightens the threshold.  The m
// smallest keys are unique, so the result is independent of thread timing.
#include <cub/cub.cuh>

#include "dist.cuh"
#include "sbv_internal.cuh"

namespace sbv {

constexpr int KNN_WARPS = 8;
constexpr int KNN_QW = 2;                       // queries per warp
constexpr int KNN_Q = KNN_WARPS * KNN_QW;       // queries per CTA
constexpr int KNN_TILE = 256;                   // candidates per shared-memory tile

struct Key {
  unsigned long long dbits;  // bits of a non-negative double: ordered like the value
  int32_t id;
};

__device__ __forceinline__ bool key_less(unsigned long long da, int32_t ia, unsigned long long db,
                                         int32_t ib) {
  return da < db || (da == db && ia < ib);
}

// Smallest L such that every D32 > L has D32 - 2E(D32) > thr (D32 - 2E is increasing).
__device__ __forceinline__ float screen_limit(double thr, ScreenBound sb) {
  if (!(thr < 1e300)) return INFINITY;
  float t = (float)thr;
  t = t * 1.0000005f + 1e-30f;  // round up
  float L = t;
#pragma unroll
  for (int it = 0; it < 4; ++it) L = t + screen_margin(L, sb);
  return t + 1.5f * screen_margin(L * 1.01f + screen_margin(0.0f, sb), sb);
}

// Warp-cooperative bitonic sort of cap (power of two) keys in shared memory,
// ascending; entries beyond `count` must already hold the +inf key.
__device__ void warp_sort(unsigned long long* kd, int32_t* ki, int cap) {
  const int lane = threadIdx.x & 31;
  for (int size = 2; size <= cap; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int e = lane; e < cap / 2; e += 32) {
        int lo = 2 * e - (e & (stride - 1));
        int hi = lo + stride;
        bool up = ((lo & size) == 0);
        unsigned long long a = kd[lo], b = kd[hi];
        int32_t ia = ki[lo], ib = ki[hi];
        bool swap = up ? key_less(b, ib, a, ia) : key_less(a, ia, b, ib);
        if (swap) {
          kd[lo] = b; kd[hi] = a;
          ki[lo] = ib; ki[hi] = ia;
        }
      }
      __syncwarp();
    }
  }
}

struct KnnArgs {
  const float* Z32;       // d x n structure-of-arrays, candidate layout order
  const double* Z64;      // d x n structure-of-arrays, candidate layout order
  const int32_t* cid;     // candidate position -> point index (NULL: identity)
  int64_t n;
  int d;
  const double* Q;        // query coordinates, row-major nq x d
  int64_t nq;
  const int32_t* qlimit_rank;  // per query: rank r (candidates = [0, rptr[r])) or NULL
  const int64_t* rptr;         // prefix offsets by rank (NULL: all n candidates)
  const int32_t* qorder;       // query slot -> query index (NULL: identity)
  int m;
  int cap;                 // buffer capacity per query (power of two >= m + KNN_TILE)
  ScreenBound sb;
  int32_t* nbr;            // nq x m
  int32_t* cnt;            // nq (or NULL)
};

template <int DM>
__global__ void __launch_bounds__(KNN_WARPS * 32)
knn_kernel(KnnArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int cap = a.cap;
  float* tile = (float*)smem;                                          // DM x KNN_TILE
  unsigned long long* kd = (unsigned long long*)(tile + DM * KNN_TILE); // KNN_Q x cap
  int32_t* ki = (int32_t*)(kd + (size_t)KNN_Q * cap);                  // KNN_Q x cap
  __shared__ int fill[KNN_Q];
  __shared__ double thr[KNN_Q];
  __shared__ int32_t thr_id[KNN_Q];
  __shared__ float lim[KNN_Q];
  __shared__ int64_t qend[KNN_Q];
  __shared__ int64_t qidx[KNN_Q];
  __shared__ double qc[KNN_Q * DM];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t slot0 = (int64_t)blockIdx.x * KNN_Q;

  for (int q = threadIdx.x; q < KNN_Q; q += blockDim.x) {
    int64_t slot = slot0 + q;
    int64_t qi = -1, end = 0;
    if (slot < a.nq) {
      qi = a.qorder ? a.qorder[slot] : slot;
      end = a.rptr ? a.rptr[a.qlimit_rank[qi]] : a.n;
    }
    qidx[q] = qi;
    qend[q] = end;
    fill[q] = 0;
    thr[q] = INFINITY;
    thr_id[q] = 0x7fffffff;
    lim[q] = INFINITY;
    for (int t = 0; t < DM; ++t) qc[q * DM + t] = (qi >= 0 && t < a.d) ? a.Q[qi * a.d + t] : 0.0;
  }
  for (int e = threadIdx.x; e < KNN_Q * cap; e += blockDim.x) {
    kd[e] = ~0ull;
    ki[e] = 0x7fffffff;
  }
  __syncthreads();
  int64_t cmax = 0;
  for (int q = 0; q < KNN_Q; ++q) cmax = max(cmax, qend[q]);

  float qf[KNN_QW][DM];
#pragma unroll
  for (int w = 0; w < KNN_QW; ++w)
#pragma unroll
    for (int t = 0; t < DM; ++t) qf[w][t] = (float)qc[(warp * KNN_QW + w) * DM + t];

  for (int64_t base = 0; base < cmax; base += KNN_TILE) {
    const int nt = (int)min((int64_t)KNN_TILE, cmax - base);
    __syncthreads();
    for (int e = threadIdx.x; e < DM * KNN_TILE; e += blockDim.x) {
      int t = e / KNN_TILE, c = e % KNN_TILE;
      tile[e] = (t < a.d && c < nt) ? a.Z32[(size_t)t * a.n + base + c] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < KNN_QW; ++w) {
      const int q = warp * KNN_QW + w;
      if (qidx[q] < 0 || base >= qend[q]) continue;
      // make room: a tile adds at most KNN_TILE keys
      if (fill[q] > cap - KNN_TILE) {
        warp_sort(kd + (size_t)q * cap, ki + (size_t)q * cap, cap);
        if (lane == 0) {
          int keep = min(fill[q], a.m);
          fill[q] = keep;
          if (keep == a.m && keep > 0) {
            thr[q] = __longlong_as_double((long long)kd[(size_t)q * cap + keep - 1]);
            thr_id[q] = ki[(size_t)q * cap + keep - 1];
            lim[q] = screen_limit(thr[q], a.sb);
          }
        }
        __syncwarp();
        for (int e = a.m + lane; e < cap; e += 32) {
          kd[(size_t)q * cap + e] = ~0ull;
          ki[(size_t)q * cap + e] = 0x7fffffff;
        }
        __syncwarp();
      }
      const int64_t qe = qend[q];
      const float L = lim[q];
      const double T = thr[q];
      const int32_t Tid = thr_id[q];
      for (int c = lane; c < nt; c += 32) {
        int64_t p = base + c;
        if (p >= qe) break;
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < DM; ++t) {
          if (t < a.d) {
            float df = tile[t * KNN_TILE + c] - qf[w][t];
            acc = fmaf(df, df, acc);
          }
        }
        if (acc <= L) {
          double D = dist2_exact_strided(a.Z64 + p, (size_t)a.n, qc + q * DM, a.d);
          int32_t id = a.cid ? a.cid[p] : (int32_t)p;
          unsigned long long db = (unsigned long long)__double_as_longlong(D);
          if (key_less(db, id, (unsigned long long)__double_as_longlong(T), Tid)) {
            int pos = atomicAdd(&fill[q], 1);
            kd[(size_t)q * cap + pos] = db;
            ki[(size_t)q * cap + pos] = id;
          }
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // final: sort and emit the m smallest keys of every query
#pragma unroll
  for (int w = 0; w < KNN_QW; ++w) {
    const int q = warp * KNN_QW + w;
    if (qidx[q] < 0) continue;
    warp_sort(kd + (size_t)q * cap, ki + (size_t)q * cap, cap);
    const int keep = min(fill[q], a.m);
    const int64_t qi = qidx[q];
    for (int e = lane; e < a.m; e += 32)
      a.nbr[qi * a.m + e] = e < keep ? ki[(size_t)q * cap + e] : -1;
    if (lane == 0 && a.cnt) a.cnt[qi] = keep;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// layout helpers
// ---------------------------------------------------------------------------
__global__ void rank_counts_kernel(const int64_t* __restrict__ ptr, const int32_t* __restrict__ rank,
                                   int64_t bc, int64_t* __restrict__ rcount) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < bc;
       j += (int64_t)gridDim.x * blockDim.x)
    rcount[rank[j]] = ptr[j + 1] - ptr[j];
}

// One warp per block: copy its members to their rank-ordered positions.
__global__ void rank_scatter_kernel(const int64_t* __restrict__ ptr, const int32_t* __restrict__ pts,
                                    const int32_t* __restrict__ rank, const int64_t* __restrict__ rptr,
                                    int64_t bc, int32_t* __restrict__ rorder) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  for (; w < bc; w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    int64_t a = ptr[w], b = ptr[w + 1], o = rptr[rank[w]];
    for (int64_t q = a + lane; q < b; q += 32) rorder[o + (q - a)] = pts[q];
  }
}

// Structure-of-arrays copies (d x n) of the scaled coordinates in layout order.
__global__ void soa_kernel(const double* __restrict__ Z, const int32_t* __restrict__ order,
                           int64_t n, int d, double* __restrict__ Z64, float* __restrict__ Z32) {
  int64_t total = n * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int t = (int)(e / n);
    int64_t p = e % n;
    int64_t src = order ? (int64_t)order[p] : p;
    double v = Z[src * d + t];
    Z64[e] = v;
    Z32[e] = (float)v;
  }
}

__global__ void rank_sorted_blocks_kernel(const int32_t* __restrict__ rank, int64_t bc,
                                          int32_t* __restrict__ by_rank) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < bc;
       j += (int64_t)gridDim.x * blockDim.x)
    by_rank[bc - 1 - rank[j]] = (int32_t)j;  // longest prefixes first
}

static int grid_for(int64_t work, int threads, int sms) {
  int64_t g = (work + threads - 1) / threads;
  int64_t cap = (int64_t)sms * 32;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

int absmax(sbv_ctx* ctx, const double* Z, int64_t total, double* out, cudaStream_t s);

static int launch_knn(sbv_ctx* ctx, KnnArgs& a, cudaStream_t s) {
  int cap = 1;
  while (cap < a.m + KNN_TILE + 32) cap <<= 1;
  a.cap = cap;
  int dm = a.d <= 4 ? 4 : a.d <= 8 ? 8 : a.d <= 12 ? 12 : a.d <= 16 ? 16 : a.d <= 24 ? 24 : a.d <= 32 ? 32 : 64;
  size_t smem = (size_t)dm * KNN_TILE * sizeof(float) + (size_t)KNN_Q * cap * (8 + 4);
  size_t stat = (size_t)KNN_Q * (4 + 8 + 4 + 4 + 8 + 8) + (size_t)KNN_Q * dm * 8;
  if (smem + stat > ctx->smem_optin)
    return fail(ctx, SBV_EUNSUPPORTED, "kNN needs %zu bytes of shared memory (m=%d, d=%d)",
                smem + stat, a.m, a.d);
  int grid = (int)((a.nq + KNN_Q - 1) / KNN_Q);
#define SBV_KNN(DM)                                                                         \
  do {                                                                                      \
    SBV_CUDA_TRY(ctx, cudaFuncSetAttribute(knn_kernel<DM>,                                  \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                           (int)smem));                                     \
    knn_kernel<DM><<<grid, KNN_WARPS * 32, smem, s>>>(a);                                   \
  } while (0)
  switch (dm) {
    case 4: SBV_KNN(4); break;
    case 8: SBV_KNN(8); break;
    case 12: SBV_KNN(12); break;
    case 16: SBV_KNN(16); break;
    case 24: SBV_KNN(24); break;
    case 32: SBV_KNN(32); break;
    default: SBV_KNN(64); break;
  }
#undef SBV_KNN
  SBV_LAUNCH_CHECK(ctx, "knn_kernel");
  return SBV_OK;
}

int run_knn(sbv_ctx* ctx, const double* Z, int64_t n, int d, const int64_t* ptr,
            const int32_t* pts, const int32_t* rank, const double* centres, int64_t bc, int m,
            int32_t* nbr, int32_t* cnt, cudaStream_t s) {
  int st = 0;
  if (m == 0) {
    SBV_CUDA_TRY(ctx, cudaMemsetAsync(cnt, 0, bc * sizeof(int32_t), s));
    SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return SBV_OK;
  }
  char* w = (char*)ws_get(ctx, WS_ORDER,
                          (size_t)n * d * (8 + 4) + (size_t)n * 4 + (size_t)(bc + 1) * 16 +
                              (size_t)bc * 4 + 4096,
                          &st);
  if (!w) return st;
  double* Z64 = (double*)w;
  float* Z32 = (float*)(Z64 + (size_t)n * d);
  int32_t* rorder = (int32_t*)(Z32 + (size_t)n * d);
  int64_t* rcount = (int64_t*)(((uintptr_t)(rorder + n) + 15) & ~(uintptr_t)15);
  int64_t* rptr = rcount + (bc + 1);
  int32_t* by_rank = (int32_t*)(rptr + (bc + 1));

  SBV_CUDA_TRY(ctx, cudaMemsetAsync(rcount, 0, (bc + 1) * sizeof(int64_t), s));
  rank_counts_kernel<<<grid_for(bc, 256, ctx->num_sms), 256, 0, s>>>(ptr, rank, bc, rcount);
  SBV_LAUNCH_CHECK(ctx, "rank_counts_kernel");
  size_t tb = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tb, rcount, rptr, (int)(bc + 1), s);
  void* tmp = ws_get(ctx, WS_CUB, tb, &st);
  if (!tmp) return st;
  SBV_CUDA_TRY(ctx, cub::DeviceScan::ExclusiveSum(tmp, tb, rcount, rptr, (int)(bc + 1), s));
  rank_scatter_kernel<<<grid_for(bc * 32, 256, ctx->num_sms), 256, 0, s>>>(ptr, pts, rank, rptr, bc,
                                                                           rorder);
  SBV_LAUNCH_CHECK(ctx, "rank_scatter_kernel");
  soa_kernel<<<grid_for(n * d, 256, ctx->num_sms), 256, 0, s>>>(Z, rorder, n, d, Z64, Z32);
  SBV_LAUNCH_CHECK(ctx, "soa_kernel");
  rank_sorted_blocks_kernel<<<grid_for(bc, 256, ctx->num_sms), 256, 0, s>>>(rank, bc, by_rank);
  SBV_LAUNCH_CHECK(ctx, "rank_sorted_blocks_kernel");

  double M = 0.0;
  if ((st = absmax(ctx, Z, n * d, &M, s))) return st;
  double Mc = 0.0;
  if ((st = absmax(ctx, centres, bc * d, &Mc, s))) return st;
  KnnArgs a;
  a.Z32 = Z32;
  a.Z64 = Z64;
  a.cid = rorder;
  a.n = n;
  a.d = d;
  a.Q = centres;
  a.nq = bc;
  a.qlimit_rank = rank;
  a.rptr = rptr;
  a.qorder = by_rank;  // consecutive ranks share a CTA (their prefixes nearly coincide)
  a.m = m;
  a.sb = make_screen(M > Mc ? M : Mc, d);
  a.nbr = nbr;
  a.cnt = cnt;
  if ((st = launch_knn(ctx, a, s))) return st;
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  return SBV_OK;
}

int run_knn_all(sbv_ctx* ctx, const double* Z, int64_t n, int d, const double* Q, int64_t nq,
                int m, int32_t* nbr, cudaStream_t s) {
  int st = 0;
  char* w = (char*)ws_get(ctx, WS_ORDER, (size_t)n * d * (8 + 4) + 4096, &st);
  if (!w) return st;
  double* Z64 = (double*)w;
  float* Z32 = (float*)(Z64 + (size_t)n * d);
  soa_kernel<<<grid_for(n * d, 256, ctx->num_sms), 256, 0, s>>>(Z, nullptr, n, d, Z64, Z32);
  SBV_LAUNCH_CHECK(ctx, "soa_kernel");
  double M = 0.0, Mq = 0.0;
  if ((st = absmax(ctx, Z, n * d, &M, s))) return st;
  if ((st = absmax(ctx, Q, nq * d, &Mq, s))) return st;
  KnnArgs a;
  a.Z32 = Z32;
  a.Z64 = Z64;
  a.cid = nullptr;
  a.n = n;
  a.d = d;
  a.Q = Q;
  a.nq = nq;
  a.qlimit_rank = nullptr;
  a.rptr = nullptr;
  a.qorder = nullptr;
  a.m = m;
  a.sb = make_screen(M > Mq ? M : Mq, d);
  a.nbr = nbr;
  a.cnt = nullptr;
  return launch_knn(ctx, a, s);
}

}  // namespace sbv
