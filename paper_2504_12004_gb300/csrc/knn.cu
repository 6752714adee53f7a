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

// ---------------------------------------------------------------------------
// Pruned exact search for large inputs.  The candidates are grouped in
// blocks (the Vecchia blocks, listed by rank) with a centre and a bounding
// box; a 2-D grid over the two longest scaled dimensions indexes the block
// centres.  A query with search radius R scans only the blocks whose box lies
// within R of it (the grid window has half-width R plus the largest box
// half-extent); every other candidate lies farther than R.  If
// the m-th smallest key found has D < R^2 (1 - 1e-9), no skipped candidate
// can enter the m nearest, and the result equals the brute-force one key for
// key.  Queries that fail this test are retried with a larger R and finally
// sent to the brute-force kernel.  The radius plays the part of the
// paper's lambda (Eq. distancethreshold), made exact by the check.
// ---------------------------------------------------------------------------
constexpr int PK_WARPS = 8;

struct PrunedArgs {
  const float* Z32;        // d x n, candidate (rank) order
  const double* Z64;
  const int32_t* cid;      // candidate position -> point index
  int64_t n;
  int d;
  const int64_t* rptr;     // block of rank r: candidates [rptr[r], rptr[r+1])
  const float* bcen;       // block centres by rank, nb x d
  const float* blo;        // block bounding boxes by rank, nb x d (rounded outwards)
  const float* bhi;
  float rad_max;           // largest half-extent of a box in grid dimension g0 ...
  float rad_max1;          // ... and in g1
  float slack;             // absolute slack of the float32 centre tests
  int g0, g1;              // grid dimensions
  double gmin0, gmin1, cell;
  int nc0, nc1;
  const int64_t* cell_ptr; // nc0 * nc1 + 1
  const int32_t* cell_blk; // block ranks per cell, ascending
  const double* Q;         // nq x d query coordinates
  const int32_t* qlimit_rank;  // NULL: every block is a candidate
  const int64_t* qlist;    // queries to process
  int64_t nlist;
  const float* qR;         // search radius per list entry
  int m;
  int cap;
  ScreenBound sb;
  int32_t* nbr;            // nq x m
  int32_t* cnt;            // nq (or NULL)
  int64_t* failed;         // queries whose check failed
  unsigned long long* nfailed;
};

// sort the warp's buffer, keep the m smallest, update threshold and limit
__device__ __forceinline__ void pk_compact(unsigned long long* kd, int32_t* ki, int cap, int m,
                                           int& fill, double& thr, int32_t& thr_id, float& lim,
                                           ScreenBound sb) {
  const int lane = threadIdx.x & 31;
  warp_sort(kd, ki, cap);
  const int keep = min(fill, m);
  fill = keep;
  if (keep == m && keep > 0) {
    thr = __longlong_as_double((long long)kd[keep - 1]);
    thr_id = ki[keep - 1];
    lim = screen_limit(thr, sb);
  }
  for (int e = keep + lane; e < cap; e += 32) {
    kd[e] = ~0ull;
    ki[e] = 0x7fffffff;
  }
  __syncwarp();
}

template <int DM>
__global__ void __launch_bounds__(PK_WARPS * 32) knn_pruned_kernel(PrunedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cap = a.cap;
  unsigned long long* kd = (unsigned long long*)smem + (size_t)warp * cap;
  int32_t* ki = (int32_t*)((unsigned long long*)smem + (size_t)PK_WARPS * cap) + (size_t)warp * cap;
  const int64_t li = (int64_t)blockIdx.x * PK_WARPS + warp;
  if (li >= a.nlist) return;   // warp-uniform; the kernel uses no CTA barrier
  const int64_t qi = a.qlist[li];
  double qc[DM];
  float qf[DM];
#pragma unroll
  for (int t = 0; t < DM; ++t) {
    qc[t] = t < a.d ? a.Q[qi * a.d + t] : 0.0;
    qf[t] = (float)qc[t];
  }
  const int64_t nb_lim = a.qlimit_rank ? (int64_t)a.qlimit_rank[qi] : INT64_MAX;
  const float R = a.qR[li];
  for (int e = lane; e < cap; e += 32) {
    kd[e] = ~0ull;
    ki[e] = 0x7fffffff;
  }
  __syncwarp();
  int fill = 0;
  double thr = INFINITY;
  int32_t thr_id = 0x7fffffff;
  float lim = INFINITY;
  const double W = (double)R + (double)a.rad_max + (double)a.slack;
  const double W1 = (double)R + (double)a.rad_max1 + (double)a.slack;
  auto cell_of = [&](double v, double gmin, int nc) {
    double c = floor((v - gmin) / a.cell);
    return c < 0.0 ? 0 : (c > (double)(nc - 1) ? nc - 1 : (int)c);
  };
  // one extra cell on each side absorbs rounding of the cell indices
  const int i0 = max(cell_of(qc[a.g0] - W, a.gmin0, a.nc0) - 1, 0);
  const int i1 = min(cell_of(qc[a.g0] + W, a.gmin0, a.nc0) + 1, a.nc0 - 1);
  const int j0 = max(cell_of(qc[a.g1] - W1, a.gmin1, a.nc1) - 1, 0);
  const int j1 = min(cell_of(qc[a.g1] + W1, a.gmin1, a.nc1) + 1, a.nc1 - 1);
  for (int ci = i0; ci <= i1; ++ci) {
    for (int cj = j0; cj <= j1; ++cj) {
      const int64_t cs = a.cell_ptr[(int64_t)ci * a.nc1 + cj], ce = a.cell_ptr[(int64_t)ci * a.nc1 + cj + 1];
      for (int64_t base = cs; base < ce; base += 32) {
        const int64_t idx = base + lane;
        const int32_t b = idx < ce ? a.cell_blk[idx] : 0x7fffffff;
        bool ok = idx < ce && (int64_t)b < nb_lim;
        const bool past = __any_sync(0xffffffffu, idx < ce && (int64_t)b >= nb_lim);
        if (ok) {
          // distance from the query to the block's bounding box
          float acc = 0.0f;
#pragma unroll
          for (int t = 0; t < DM; ++t) {
            if (t < a.d) {
              const float l = a.blo[(int64_t)b * a.d + t], h = a.bhi[(int64_t)b * a.d + t];
              const float df = fmaxf(fmaxf(l - qf[t], qf[t] - h), 0.0f);
              acc = fmaf(df, df, acc);
            }
          }
          ok = sqrtf(acc) <= R + a.slack;
        }
        unsigned mask = __ballot_sync(0xffffffffu, ok);
        while (mask) {
          const int src = __ffs(mask) - 1;
          mask &= mask - 1;
          const int32_t bb = __shfl_sync(0xffffffffu, b, src);
          const int64_t p0 = a.rptr[bb], p1 = a.rptr[bb + 1];
          for (int64_t pb = p0; pb < p1; pb += 32) {
            if (fill > cap - 32) pk_compact(kd, ki, cap, a.m, fill, thr, thr_id, lim, a.sb);
            const int64_t p = pb + lane;
            bool take = false;
            unsigned long long db = 0;
            int32_t id = 0;
            if (p < p1) {
              float acc = 0.0f;
#pragma unroll
              for (int t = 0; t < DM; ++t) {
                if (t < a.d) {
                  const float df = a.Z32[(size_t)t * a.n + p] - qf[t];
                  acc = fmaf(df, df, acc);
                }
              }
              if (acc <= lim) {
                const double D = dist2_exact_strided(a.Z64 + p, (size_t)a.n, qc, a.d);
                id = a.cid[p];
                db = (unsigned long long)__double_as_longlong(D);
                take = key_less(db, id, (unsigned long long)__double_as_longlong(thr), thr_id);
              }
            }
            const unsigned tm = __ballot_sync(0xffffffffu, take);
            if (take) {
              const int pos = fill + __popc(tm & ((1u << lane) - 1u));
              kd[pos] = db;
              ki[pos] = id;
            }
            fill += __popc(tm);
            __syncwarp();
          }
        }
        if (past) break;   // ranks ascend inside a cell
      }
    }
  }
  pk_compact(kd, ki, cap, a.m, fill, thr, thr_id, lim, a.sb);
  const double R2 = (double)R * (double)R * (1.0 - 1e-9);
  const bool exact = fill == a.m && thr < R2;
  if (exact) {
    for (int e = lane; e < a.m; e += 32) a.nbr[qi * a.m + e] = ki[e];
    if (lane == 0 && a.cnt) a.cnt[qi] = a.m;
  } else if (lane == 0) {
    a.failed[atomicAdd(a.nfailed, 1ull)] = qi;
  }
}

// Centre and bounding box (float32, rounded outwards) of the block of every
// rank, and the largest box half-extent over the grid candidates; one warp
// per block.
__global__ void block_bounds_kernel(const double* __restrict__ Z64, int64_t n, int d,
                                    const int64_t* __restrict__ rptr,
                                    const double* __restrict__ centres,
                                    const int32_t* __restrict__ blk_of_rank, int64_t nb,
                                    float* __restrict__ bcen, float* __restrict__ blo,
                                    float* __restrict__ bhi, float* __restrict__ bhalf) {
  // bhalf: nb x d, half-extent of the box around the centre per dimension
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (; w < nb; w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const double* c = centres + (int64_t)blk_of_rank[w] * d;
    for (int t = 0; t < d; ++t) {
      double lo = INFINITY, hi = -INFINITY;
      for (int64_t p = rptr[w] + lane; p < rptr[w + 1]; p += 32) {
        const double v = Z64[(size_t)t * n + p];
        lo = fmin(lo, v);
        hi = fmax(hi, v);
      }
      for (int o = 16; o; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      if (lane == 0) {
        blo[w * d + t] = __double2float_rd(lo);
        bhi[w * d + t] = __double2float_ru(hi);
        bcen[w * d + t] = (float)c[t];
        bhalf[w * d + t] = __double2float_ru(fmax(c[t] - lo, hi - c[t]));
      }
    }
  }
}

__global__ void iota_i32_kernel(int32_t* __restrict__ v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (int32_t)i;
}

__global__ void cell_count_kernel(const int32_t* __restrict__ keys, int64_t n,
                                  int64_t* __restrict__ counts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd((unsigned long long*)&counts[keys[i]], 1ull);
}

__global__ void block_of_rank_kernel(const int32_t* __restrict__ rank, int64_t nb,
                                     int32_t* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nb;
       j += (int64_t)gridDim.x * blockDim.x)
    out[rank[j]] = (int32_t)j;
}

__global__ void cell_key_kernel(const float* __restrict__ bcen, int64_t nb, int d, int g0, int g1,
                                double gmin0, double gmin1, double cell, int nc0, int nc1,
                                int32_t* __restrict__ key) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nb;
       j += (int64_t)gridDim.x * blockDim.x) {
    double c0 = floor(((double)bcen[j * d + g0] - gmin0) / cell);
    double c1 = floor(((double)bcen[j * d + g1] - gmin1) / cell);
    int i = c0 < 0.0 ? 0 : (c0 > nc0 - 1 ? nc0 - 1 : (int)c0);
    int k = c1 < 0.0 ? 0 : (c1 > nc1 - 1 ? nc1 - 1 : (int)c1);
    key[j] = i * nc1 + k;
  }
}

// search radius per listed query: the ball expected to hold alpha * m of its
// candidates at the average density, times `grow`
__global__ void radius_kernel(const int64_t* __restrict__ qlist, int64_t nlist,
                              const int32_t* __restrict__ qlimit_rank,
                              const int64_t* __restrict__ rptr, int64_t n, double vol_over_vd,
                              int m, int d, double grow, float* __restrict__ qR) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlist;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ne = qlimit_rank ? rptr[qlimit_rank[qlist[i]]] : n;
    const double r = pow(3.0 * m * vol_over_vd / (double)(ne > 0 ? ne : 1), 1.0 / d);
    qR[i] = (float)(r * grow);
  }
}

__global__ void minmax_kernel(const float* __restrict__ v, int64_t nb, int d,
                              unsigned int* __restrict__ mn, unsigned int* __restrict__ mx) {
  // order-preserving map of float bits to unsigned
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nb * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    unsigned int u = __float_as_uint(v[e]);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    atomicMin(&mn[e % d], u);
    atomicMax(&mx[e % d], u);
  }
}

static float unmap_float(unsigned int u) {
  u = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
  float f;
  memcpy(&f, &u, 4);
  return f;
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

__global__ void split_queries_kernel(const int32_t* __restrict__ qlimit_rank,
                                     const int64_t* __restrict__ rptr, int64_t n, int64_t nq,
                                     int64_t small, int64_t* __restrict__ big_list,
                                     unsigned long long* __restrict__ nbig,
                                     int64_t* __restrict__ small_list,
                                     unsigned long long* __restrict__ nsmall) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ne = qlimit_rank ? rptr[qlimit_rank[q]] : n;
    if (ne > small) big_list[atomicAdd(nbig, 1ull)] = q;
    else small_list[atomicAdd(nsmall, 1ull)] = q;
  }
}

__global__ void i64_to_i32_kernel(const int64_t* __restrict__ a, int64_t k, int32_t* __restrict__ b) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < k;
       j += (int64_t)gridDim.x * blockDim.x)
    b[j] = (int32_t)a[j];
}

// The pruned search over the blocks of `base` (candidates in rank order):
// queries whose candidate prefix is short, or whose check fails three times
// with growing radius, go to the brute-force kernel.  Results are those of
// the brute-force search for every query.
static int knn_pruned(sbv_ctx* ctx, KnnArgs base, const int32_t* rank_of_block, int64_t nb,
                      const double* centres, cudaStream_t s) {
  int st = 0;
  const int64_t n = base.n, nq = base.nq;
  const int d = base.d, m = base.m;
  const int sms = ctx->num_sms;
  size_t bytes = (size_t)nb * 4 + (size_t)nb * d * 4 * 4 + (size_t)nb * 4 * 3 +
                 (size_t)(nq + 8) * 8 * 4 + (size_t)nq * 4 * 2 + 4096 + (size_t)64 * 8;
  char* wp = (char*)ws_get(ctx, WS_SORT_D, bytes, &st);
  if (!wp) return st;
  auto take = [&](size_t b) {
    char* r = wp;
    wp += (b + 255) / 256 * 256;
    return r;
  };
  int32_t* blk_of_rank = (int32_t*)take((size_t)nb * 4);
  float* bcen = (float*)take((size_t)nb * d * 4);
  float* blo = (float*)take((size_t)nb * d * 4);
  float* bhi = (float*)take((size_t)nb * d * 4);
  float* brad = (float*)take((size_t)nb * d * 4);   // box half-extents per dimension
  int32_t* keys = (int32_t*)take((size_t)nb * 4);
  int32_t* keys_sorted = (int32_t*)take((size_t)nb * 4);
  int32_t* iota = (int32_t*)take((size_t)nb * 4);
  int64_t* listA = (int64_t*)take((size_t)(nq + 8) * 8);
  int64_t* listB = (int64_t*)take((size_t)(nq + 8) * 8);
  int64_t* small_list = (int64_t*)take((size_t)(nq + 8) * 8);
  int64_t* spare = (int64_t*)take((size_t)(nq + 8) * 8);
  float* qR = (float*)take((size_t)nq * 4);
  int32_t* brute = (int32_t*)take((size_t)nq * 4);
  unsigned long long* counters = (unsigned long long*)take(2048);
  unsigned int* mm = (unsigned int*)(counters + 8);  // 64 mins, 64 maxima, radius min and max
  (void)spare;
  block_of_rank_kernel<<<grid_for(nb, 256, sms), 256, 0, s>>>(rank_of_block, nb, blk_of_rank);
  block_bounds_kernel<<<grid_for(nb * 32, 256, sms), 256, 0, s>>>(base.Z64, n, d, base.rptr, centres,
                                                                 blk_of_rank, nb, bcen, blo, bhi, brad);
  SBV_LAUNCH_CHECK(ctx, "block_bounds_kernel");
  // extents of the block centres and the largest radius
  // mm: 64 minima and 64 maxima of the centres, then 64 minima and 64 maxima
  // of the box half-extents, per dimension
  std::vector<unsigned int> init(256);
  for (int t = 0; t < 256; ++t) init[t] = (t < 64 || (t >= 128 && t < 192)) ? 0xffffffffu : 0u;
  SBV_CUDA_TRY(ctx, cudaMemcpyAsync(mm, init.data(), 256 * 4, cudaMemcpyHostToDevice, s));
  minmax_kernel<<<grid_for(nb * d, 256, sms), 256, 0, s>>>(bcen, nb, d, mm, mm + 64);
  minmax_kernel<<<grid_for(nb * d, 256, sms), 256, 0, s>>>(brad, nb, d, mm + 128, mm + 192);
  SBV_LAUNCH_CHECK(ctx, "minmax_kernel");
  std::vector<unsigned int> hm(256);
  SBV_CUDA_TRY(ctx, cudaMemcpyAsync(hm.data(), mm, 256 * 4, cudaMemcpyDeviceToHost, s));
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  std::vector<double> lo(d), ext(d);
  for (int t = 0; t < d; ++t) {
    lo[t] = unmap_float(hm[t]);
    ext[t] = std::max((double)unmap_float(hm[64 + t]) - lo[t], 1e-30);
  }
  std::vector<double> half(d);
  double rad_max = 0.0;
  for (int t = 0; t < d; ++t) {
    half[t] = unmap_float(hm[192 + t]);
    rad_max = std::max(rad_max, half[t]);
  }
  int g0 = 0, g1 = d > 1 ? 1 : 0;
  for (int t = 0; t < d; ++t)
    if (ext[t] > ext[g0]) g0 = t;
  if (d > 1) {
    g1 = g0 == 0 ? 1 : 0;
    for (int t = 0; t < d; ++t)
      if (t != g0 && ext[t] > ext[g1]) g1 = t;
  }
  // density: points spread over the centres' box grown by the largest radius
  double vol = 1.0;
  for (int t = 0; t < d; ++t) vol *= ext[t] + 2.0 * rad_max;
  const double vd = pow(M_PI, 0.5 * d) / tgamma(0.5 * d + 1.0);
  const double vol_over_vd = vol / vd;
  const double r_typ = pow(3.0 * m * vol_over_vd / std::max<double>(n / 2, 1), 1.0 / d);
  double cell = r_typ + std::max(half[g0], half[g1]);
  int nc0 = std::max(1, (int)ceil(ext[g0] / cell)), nc1 = std::max(1, (int)ceil(ext[g1] / cell));
  while ((int64_t)nc0 * nc1 > (1 << 22)) {
    cell *= 2.0;
    nc0 = std::max(1, (int)ceil(ext[g0] / cell));
    nc1 = std::max(1, (int)ceil(ext[g1] / cell));
  }
  const int ncell = nc0 * nc1;
  cell_key_kernel<<<grid_for(nb, 256, sms), 256, 0, s>>>(bcen, nb, d, g0, g1, lo[g0], lo[g1], cell, nc0,
                                                        nc1, keys);
  iota_i32_kernel<<<grid_for(nb, 256, sms), 256, 0, s>>>(iota, nb);
  SBV_LAUNCH_CHECK(ctx, "cell_key_kernel");
  int32_t* cell_blk = (int32_t*)ws_get(ctx, WS_EXTRA, (size_t)nb * 4 + (size_t)(ncell + 1) * 8 * 2 + 1024, &st);
  if (!cell_blk) return st;
  int64_t* ccount = (int64_t*)(((uintptr_t)(cell_blk + nb) + 15) & ~(uintptr_t)15);
  int64_t* cell_ptr = ccount + (ncell + 1);
  {
    int end_bit = 1;
    while ((1ll << end_bit) < ncell) ++end_bit;
    size_t tb = 0, tb2 = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tb, keys, keys_sorted, iota, cell_blk, (int)nb, 0, end_bit, s);
    cub::DeviceScan::ExclusiveSum(nullptr, tb2, ccount, cell_ptr, ncell + 1, s);
    void* tmp = ws_get(ctx, WS_CUB, std::max(tb, tb2), &st);
    if (!tmp) return st;
    SBV_CUDA_TRY(ctx, cub::DeviceRadixSort::SortPairs(tmp, tb, keys, keys_sorted, iota, cell_blk, (int)nb,
                                                      0, end_bit, s));
    SBV_CUDA_TRY(ctx, cudaMemsetAsync(ccount, 0, (ncell + 1) * 8, s));
    cell_count_kernel<<<grid_for(nb, 256, sms), 256, 0, s>>>(keys, nb, ccount);
    SBV_LAUNCH_CHECK(ctx, "cell_count_kernel");
    SBV_CUDA_TRY(ctx, cub::DeviceScan::ExclusiveSum(tmp, tb2, ccount, cell_ptr, ncell + 1, s));
  }
  // queries: short candidate prefixes go straight to the brute-force kernel
  SBV_CUDA_TRY(ctx, cudaMemsetAsync(counters, 0, 8 * 8, s));
  const int64_t small = (int64_t)64 * m;
  split_queries_kernel<<<grid_for(nq, 256, sms), 256, 0, s>>>(base.qlimit_rank, base.rptr, n, nq, small,
                                                              listA, counters, small_list, counters + 1);
  SBV_LAUNCH_CHECK(ctx, "split_queries_kernel");
  unsigned long long hc[2];
  SBV_CUDA_TRY(ctx, cudaMemcpyAsync(hc, counters, 16, cudaMemcpyDeviceToHost, s));
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  int64_t nlist = (int64_t)hc[0], nsmall = (int64_t)hc[1];
  int cap = 1;
  while (cap < m + 96) cap <<= 1;
  const size_t smem = (size_t)PK_WARPS * cap * 12;
  if (smem > ctx->smem_optin) return fail(ctx, SBV_EUNSUPPORTED, "pruned kNN: m=%d too large", m);
  PrunedArgs a;
  a.Z32 = base.Z32;
  a.Z64 = base.Z64;
  a.cid = base.cid;
  a.n = n;
  a.d = d;
  a.rptr = base.rptr;
  a.bcen = bcen;
  a.blo = blo;
  a.bhi = bhi;
  a.rad_max = (float)half[g0];
  a.rad_max1 = (float)half[g1];
  double zmax = 0.0;
  for (int t = 0; t < d; ++t) zmax = std::max(zmax, std::max(fabs(lo[t]), fabs(lo[t] + ext[t])));
  a.slack = (float)(1e-5 * (zmax + rad_max + 1.0) * d);
  a.g0 = g0;
  a.g1 = g1;
  a.gmin0 = lo[g0];
  a.gmin1 = lo[g1];
  a.cell = cell;
  a.nc0 = nc0;
  a.nc1 = nc1;
  a.cell_ptr = cell_ptr;
  a.cell_blk = cell_blk;
  a.Q = base.Q;
  a.qlimit_rank = base.qlimit_rank;
  a.qR = qR;
  a.m = m;
  a.cap = cap;
  a.sb = base.sb;
  a.nbr = base.nbr;
  a.cnt = base.cnt;
  int64_t* cur = listA;
  int64_t* nxt = listB;
  for (int attempt = 0; attempt < 3 && nlist > 0; ++attempt) {
    radius_kernel<<<grid_for(nlist, 256, sms), 256, 0, s>>>(cur, nlist, base.qlimit_rank, base.rptr, n,
                                                           vol_over_vd, m, d, (double)(1 << attempt), qR);
    SBV_CUDA_TRY(ctx, cudaMemsetAsync(counters + 2, 0, 8, s));
    a.qlist = cur;
    a.nlist = nlist;
    a.failed = nxt;
    a.nfailed = counters + 2;
    const unsigned grid = (unsigned)((nlist + PK_WARPS - 1) / PK_WARPS);
#define SBV_PK(DM)                                                                                   \
  do {                                                                                               \
    SBV_CUDA_TRY(ctx, cudaFuncSetAttribute(knn_pruned_kernel<DM>,                                    \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    knn_pruned_kernel<DM><<<grid, PK_WARPS * 32, smem, s>>>(a);                                      \
  } while (0)
    if (d <= 4) SBV_PK(4);
    else if (d <= 8) SBV_PK(8);
    else if (d <= 12) SBV_PK(12);
    else if (d <= 16) SBV_PK(16);
    else if (d <= 24) SBV_PK(24);
    else if (d <= 32) SBV_PK(32);
    else SBV_PK(64);
#undef SBV_PK
    SBV_LAUNCH_CHECK(ctx, "knn_pruned_kernel");
    unsigned long long hf = 0;
    SBV_CUDA_TRY(ctx, cudaMemcpyAsync(&hf, counters + 2, 8, cudaMemcpyDeviceToHost, s));
    SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    nlist = (int64_t)hf;
    std::swap(cur, nxt);
  }
  // brute force: short prefixes and queries that failed every attempt
  const int64_t nbrute = nsmall + nlist;
  if (nbrute > 0) {
    if (nsmall > 0)
      i64_to_i32_kernel<<<grid_for(nsmall, 256, sms), 256, 0, s>>>(small_list, nsmall, brute);
    if (nlist > 0)
      i64_to_i32_kernel<<<grid_for(nlist, 256, sms), 256, 0, s>>>(cur, nlist, brute + nsmall);
    SBV_LAUNCH_CHECK(ctx, "i64_to_i32_kernel");
    KnnArgs b = base;
    b.qorder = brute;
    b.nq = nbrute;
    if (!base.qlimit_rank) b.rptr = nullptr;   // all-points mode: every candidate
    if ((st = launch_knn(ctx, b, s))) return st;
  }
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
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
  // brute force scans sum_r rptr[r] ~ n bc / 2 candidates; above ~1e11 the
  // pruned search is used (or as the context's mode says)
  const bool pruned = ctx->knn_mode == 2 || (ctx->knn_mode == 0 && (double)n * (double)bc > 2e11);
  if (pruned) return knn_pruned(ctx, a, rank, bc, centres, s);
  if ((st = launch_knn(ctx, a, s))) return st;
  SBV_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  return SBV_OK;
}

// m nearest training points of every query over all n points, using the
// training blocks (ptr, pts, rank, centres) as the clusters of the pruned
// search; the result equals run_knn_all key for key.
int run_knn_blocks_all(sbv_ctx* ctx, const double* Z, int64_t n, int d, const int64_t* ptr,
                       const int32_t* pts, const int32_t* rank, const double* centres,
                       int64_t bc, const double* Q, int64_t nq, int m, int32_t* nbr,
                       cudaStream_t s) {
  int st = 0;
  char* w = (char*)ws_get(ctx, WS_ORDER,
                          (size_t)n * d * (8 + 4) + (size_t)n * 4 + (size_t)(bc + 1) * 16 + 4096, &st);
  if (!w) return st;
  double* Z64 = (double*)w;
  float* Z32 = (float*)(Z64 + (size_t)n * d);
  int32_t* rorder = (int32_t*)(Z32 + (size_t)n * d);
  int64_t* rcount = (int64_t*)(((uintptr_t)(rorder + n) + 15) & ~(uintptr_t)15);
  int64_t* rptr = rcount + (bc + 1);
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
  double M = 0.0, Mq = 0.0;
  if ((st = absmax(ctx, Z, n * d, &M, s))) return st;
  if ((st = absmax(ctx, Q, nq * d, &Mq, s))) return st;
  KnnArgs a;
  a.Z32 = Z32;
  a.Z64 = Z64;
  a.cid = rorder;
  a.n = n;
  a.d = d;
  a.Q = Q;
  a.nq = nq;
  a.qlimit_rank = nullptr;
  a.rptr = rptr;
  a.qorder = nullptr;
  a.m = m;
  a.sb = make_screen(M > Mq ? M : Mq, d);
  a.nbr = nbr;
  a.cnt = nullptr;
  return knn_pruned(ctx, a, rank, bc, centres, s);
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
