// Maximum-likelihood estimation around the batched likelihood (host code).
//
// The paper keeps the data resident on the GPU and maximises the SBV
// log-likelihood with an optimiser that calls Alg. 5 (summed as in Alg. 1
// Step 5) once per iteration, for hundreds of iterations (Sec. 5.4, Sec. 7);
// it does not name the algorithm.  Here the optimiser is BFGS on
// u = log theta inside box bounds, shaped around the batched launch: every
// central-difference gradient (2p parameter rows, p = 2 + d) is one call,
// and every line search (a ladder of step lengths) is one call.
//
// sbv_mle_multistart runs the same loop from several starts.  With a
// surrogate network, every start after the first `exact_starts` begins
// where the network -- trained on all (log theta, l) pairs that the exact
// likelihood produced so far -- predicts high likelihood: gradient ascent on
// the network from points around the given start proposes candidates, one
// exact call judges them together with the start itself, and the exact BFGS
// loop continues from the best.  Inside that loop the network proposes too:
// every line-search call also carries its maximisers within a trust radius
// of the iterate, refitted to the growing history every few accepted
// iterations.  The exact likelihood decides every step.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "block_common.cuh"
#include "sbv_internal.cuh"

using namespace sbv;

namespace {

struct Mix64 {
  uint64_t s;
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

struct Problem {
  sbv_ctx* ctx;
  const void* X;
  int dtype;
  const double* y;
  int64_t n;
  int d;
  const int64_t* ptr;
  const int32_t* pts;
  const int32_t* nbr;
  const int32_t* cnt;
  int64_t bc;
  int m;
  int nmax;
  int nu2;
  int precision;
  cudaStream_t s;
};

using Vec = std::vector<double>;

// Exact evaluations of parameter rows given in log space, with the history
// of every evaluated row.
struct Evaluator {
  Problem pb;
  int p = 0;
  Vec lo, hi;                 // log bounds
  double* d_ll = nullptr;
  int cap = 0;
  int64_t evals = 0;
  int64_t grad_evals = 0;
  int calls = 0;
  double* d_g = nullptr;      // analytic gradient of one row
  std::vector<Vec> hist_u;    // every evaluated row (log theta) ...
  Vec hist_l;                 // ... and its log-likelihood (-inf if it failed)

  ~Evaluator() {
    if (d_ll) cudaFree(d_ll);
    if (d_g) cudaFree(d_g);
  }
  Vec clamp(const Vec& u) const {
    Vec v(u);
    for (int j = 0; j < p; ++j) v[j] = std::min(std::max(v[j], lo[j]), hi[j]);
    return v;
  }
  int eval(std::vector<Vec>& U, Vec& F) {
    sbv_ctx* ctx = pb.ctx;
    const int B = (int)U.size();
    if (B > cap) {
      if (d_ll) cudaFree(d_ll);
      d_ll = nullptr;
      cap = 0;
      if (cudaMalloc(&d_ll, (size_t)B * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, SBV_ENOMEM, "likelihood buffer");
      }
      cap = B;
    }
    Vec th((size_t)B * p);
    for (int b = 0; b < B; ++b) {
      U[b] = clamp(U[b]);
      for (int j = 0; j < p; ++j) th[(size_t)b * p + j] = exp(U[b][j]);
    }
    int st = run_loglik(ctx, pb.X, pb.dtype, pb.y, pb.n, pb.d, pb.ptr, pb.pts, pb.nbr, pb.cnt,
                        pb.bc, pb.m, pb.nmax, th.data(), B, pb.nu2, pb.precision, d_ll, nullptr,
                        nullptr, pb.s);
    if (st) return st;
    F.assign(B, 0.0);
    DevStatus ds;
    SBV_CUDA_TRY(ctx, cudaMemcpyAsync(F.data(), d_ll, (size_t)B * sizeof(double),
                                      cudaMemcpyDeviceToHost, pb.s));
    SBV_CUDA_TRY(ctx, cudaMemcpyAsync(&ds, ctx->d_status, sizeof(ds), cudaMemcpyDeviceToHost, pb.s));
    SBV_CUDA_TRY(ctx, cudaStreamSynchronize(pb.s));
    if (ds.code != 0) {
      // a parameter row that makes some block matrix indefinite is simply a
      // bad candidate (its total is NaN); anything else ends the estimation
      SBV_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(DevStatus), pb.s));
      if (ds.code != SBV_ENOTSPD)
        return fail(ctx, ds.code, "likelihood kernel reported code %d", ds.code);
    }
    for (int b = 0; b < B; ++b) {
      if (!isfinite(F[b])) F[b] = -INFINITY;
      hist_u.push_back(U[b]);
      hist_l.push_back(F[b]);
    }
    evals += B;
    calls += 1;
    return SBV_OK;
  }
  // FP64 value and analytic gradient in log theta (d l / d log theta_k =
  // theta_k d l / d theta_k) of one row; the row joins the history
  int eval_grad(Vec& u, double& f, Vec& g) {
    sbv_ctx* ctx = pb.ctx;
    if (cap < 1) {
      if (d_ll) cudaFree(d_ll);
      d_ll = nullptr;
      if (cudaMalloc(&d_ll, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, SBV_ENOMEM, "likelihood buffer");
      }
      cap = 1;
    }
    if (!d_g) {
      if (cudaMalloc(&d_g, (size_t)p * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        d_g = nullptr;
        return fail(ctx, SBV_ENOMEM, "gradient buffer");
      }
    }
    u = clamp(u);
    Vec th(p), gt(p);
    for (int j = 0; j < p; ++j) th[j] = exp(u[j]);
    int st = run_loglik_grad(ctx, pb.X, pb.dtype, pb.y, pb.n, pb.d, pb.ptr, pb.pts, pb.nbr,
                             pb.cnt, pb.bc, pb.m, pb.nmax, th.data(), 1, pb.nu2, d_ll, d_g,
                             nullptr, nullptr, nullptr, pb.s);
    if (st) return st;
    DevStatus ds;
    SBV_CUDA_TRY(ctx, cudaMemcpyAsync(&f, d_ll, sizeof(double), cudaMemcpyDeviceToHost, pb.s));
    SBV_CUDA_TRY(ctx, cudaMemcpyAsync(gt.data(), d_g, (size_t)p * sizeof(double),
                                      cudaMemcpyDeviceToHost, pb.s));
    SBV_CUDA_TRY(ctx, cudaMemcpyAsync(&ds, ctx->d_status, sizeof(ds), cudaMemcpyDeviceToHost, pb.s));
    SBV_CUDA_TRY(ctx, cudaStreamSynchronize(pb.s));
    if (ds.code != 0) {
      SBV_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(DevStatus), pb.s));
      if (ds.code != SBV_ENOTSPD)
        return fail(ctx, ds.code, "gradient kernel reported code %d", ds.code);
    }
    g.assign(p, 0.0);
    if (!isfinite(f)) {
      f = -INFINITY;
    } else {
      for (int j = 0; j < p; ++j) g[j] = isfinite(gt[j]) ? th[j] * gt[j] : 0.0;
    }
    hist_u.push_back(u);
    hist_l.push_back(f);
    evals += 1;
    grad_evals += 1;
    calls += 1;
    return SBV_OK;
  }
};

sbv_mle_opts default_opts() {
  sbv_mle_opts o;
  memset(&o, 0, sizeof(o));
  o.max_evals = 4000;
  o.fd_step = 1e-3;
  o.ftol = 1e-10;
  o.max_step = 1.0;
  o.line_points = 8;
  o.precision = SBV_PREC_MIXED;
  o.nu2 = 5;
  o.gradient = 0;
  return o;
}

int check_opts(sbv_ctx* ctx, const sbv_mle_opts& o) {
  if (o.max_evals < 1 || !(o.fd_step > 0.0 && o.fd_step < 1.0) || !(o.ftol >= 0.0) ||
      !(o.max_step > 0.0) || o.line_points < 1 || o.line_points > 64)
    return fail(ctx, SBV_EINVAL, "bad MLE options");
  const bool closed = o.nu2 == 1 || o.nu2 == 3 || o.nu2 == 5 || o.nu2 == 7;
  if (!(closed || (o.precision == SBV_PREC_FP64 && o.nu2 >= 1 && o.nu2 <= SBV_MAX_NU2)))
    return fail(ctx, SBV_EINVAL, "nu2=%d: FP64 takes 1..%d, the mixed precisions {1,3,5,7}",
                o.nu2, SBV_MAX_NU2);
  if (o.gradient != 0 && o.gradient != 1)
    return fail(ctx, SBV_EINVAL, "gradient=%d not 0 or 1", o.gradient);
  if (o.precision != SBV_PREC_FP64 && o.precision != SBV_PREC_MIXED &&
      o.precision != SBV_PREC_MIXED_BF16)
    return fail(ctx, SBV_EINVAL, "precision=%d unknown", o.precision);
  return SBV_OK;
}

// central differences at u: rows u + h e_j, then u - h e_j
int fd_gradient(Evaluator& E, const Vec& u, double h, Vec& g) {
  const int p = E.p;
  std::vector<Vec> U;
  for (int sgn = 0; sgn < 2; ++sgn)
    for (int j = 0; j < p; ++j) {
      Vec v(u);
      v[j] += sgn == 0 ? h : -h;
      U.push_back(v);
    }
  Vec F;
  int st = E.eval(U, F);
  if (st) return st;
  g.assign(p, 0.0);
  for (int j = 0; j < p; ++j) {
    // a one-sided difference where a bound clipped the stencil
    const double up = U[j][j], dn = U[p + j][j];
    g[j] = (up > dn && isfinite(F[j]) && isfinite(F[p + j])) ? (F[j] - F[p + j]) / (up - dn) : 0.0;
  }
  return SBV_OK;
}

// ---- surrogate ------------------------------------------------------------
struct Surrogate {
  sbv_mlp* net;
  std::vector<float> init;     // parameters at creation: every fit starts there
  float* d_x = nullptr;        // training rows (K x p) and targets (K)
  float* d_t = nullptr;
  float* d_q = nullptr;        // ascent points (Q x p), values (Q), gradients (Q x p)
  float* d_s = nullptr;
  float* d_g = nullptr;
  size_t cap_rows = 0, cap_q = 0;
  // standardisation of the last fit and the box its rows span
  bool fitted = false;
  Vec mu, sd, bmin, bmax;
  double fm = 0.0, fs = 1.0;
  ~Surrogate() {
    for (float* q : {d_x, d_t, d_q, d_s, d_g})
      if (q) cudaFree(q);
  }
};

// Fit the network, from its initial parameters, to every finite (log theta,
// l) pair of the history, standardised per coordinate.  With fewer than 4p
// pairs nothing is fitted and S.fitted is false.
int fit(Evaluator& E, Surrogate& S, const sbv_surrogate_opts& so) {
  sbv_ctx* ctx = E.pb.ctx;
  const int p = E.p;
  std::vector<const Vec*> rows;
  Vec ls;
  for (size_t i = 0; i < E.hist_l.size(); ++i)
    if (isfinite(E.hist_l[i])) {
      rows.push_back(&E.hist_u[i]);
      ls.push_back(E.hist_l[i]);
    }
  const int64_t K = (int64_t)rows.size();
  S.fitted = false;
  if (K < 4 * p) return SBV_OK;
  Vec mu(p, 0.0), sd(p, 0.0), bmin(p, INFINITY), bmax(p, -INFINITY);
  double fm = 0.0, fs = 0.0;
  for (int64_t i = 0; i < K; ++i) {
    for (int j = 0; j < p; ++j) {
      mu[j] += (*rows[i])[j];
      bmin[j] = std::min(bmin[j], (*rows[i])[j]);
      bmax[j] = std::max(bmax[j], (*rows[i])[j]);
    }
    fm += ls[i];
  }
  for (int j = 0; j < p; ++j) mu[j] /= K;
  fm /= K;
  for (int64_t i = 0; i < K; ++i) {
    for (int j = 0; j < p; ++j) sd[j] += ((*rows[i])[j] - mu[j]) * ((*rows[i])[j] - mu[j]);
    fs += (ls[i] - fm) * (ls[i] - fm);
  }
  for (int j = 0; j < p; ++j) sd[j] = sqrt(sd[j] / K) + 1e-6;
  fs = sqrt(fs / K) + 1e-12;
  std::vector<float> hx((size_t)K * p), ht((size_t)K);
  for (int64_t i = 0; i < K; ++i) {
    for (int j = 0; j < p; ++j) hx[(size_t)i * p + j] = (float)(((*rows[i])[j] - mu[j]) / sd[j]);
    ht[i] = (float)((ls[i] - fm) / fs);
  }
  if ((size_t)K > S.cap_rows) {
    if (S.d_x) cudaFree(S.d_x);
    if (S.d_t) cudaFree(S.d_t);
    S.d_x = S.d_t = nullptr;
    S.cap_rows = 0;
    if (cudaMalloc(&S.d_x, (size_t)K * p * 4) != cudaSuccess || cudaMalloc(&S.d_t, (size_t)K * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, SBV_ENOMEM, "surrogate training rows");
    }
    S.cap_rows = (size_t)K;
  }
  SBV_CUDA_TRY(ctx, cudaMemcpy(S.d_x, hx.data(), hx.size() * 4, cudaMemcpyHostToDevice));
  SBV_CUDA_TRY(ctx, cudaMemcpy(S.d_t, ht.data(), ht.size() * 4, cudaMemcpyHostToDevice));
  int st = sbv_mlp_set_params(S.net, S.init.data(), (int64_t)S.init.size());
  if (!st) st = sbv_mlp_train(S.net, S.d_x, S.d_t, K, so.train_steps, so.batch, so.lr, so.seed,
                              nullptr, E.pb.s);
  if (st) return st;
  S.mu = mu;
  S.sd = sd;
  S.bmin = bmin;
  S.bmax = bmax;
  S.fm = fm;
  S.fs = fs;
  S.fitted = true;
  return SBV_OK;
}

// Gradient ascent on the fitted network from `ascent_starts` points: the
// centre and points drawn uniformly within max-norm `radius` of it, kept in
// the box that the training rows span (and the bounds), narrowed to the
// radius around the centre when `local` is set; sign steps of 1/200 of the
// box per iteration.  The `k` best maximisers that lie at least `sep` apart
// (max-norm) are returned, best first.
int ascend(Evaluator& E, Surrogate& S, const sbv_surrogate_opts& so, const Vec& centre,
           double radius, bool local, int k, double sep, Mix64& rng, std::vector<Vec>& cand) {
  sbv_ctx* ctx = E.pb.ctx;
  const int p = E.p;
  cudaStream_t s = E.pb.s;
  cand.clear();
  if (!S.fitted) return SBV_OK;
  const int Q = so.ascent_starts;
  if ((size_t)Q > S.cap_q) {
    for (float** q : {&S.d_q, &S.d_s, &S.d_g}) {
      if (*q) cudaFree(*q);
      *q = nullptr;
    }
    S.cap_q = 0;
    if (cudaMalloc(&S.d_q, (size_t)Q * p * 4) != cudaSuccess || cudaMalloc(&S.d_s, (size_t)Q * 4) != cudaSuccess ||
        cudaMalloc(&S.d_g, (size_t)Q * p * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, SBV_ENOMEM, "surrogate ascent rows");
    }
    S.cap_q = (size_t)Q;
  }
  Vec lo(p), hi(p);
  for (int j = 0; j < p; ++j) {
    lo[j] = std::max(S.bmin[j], E.lo[j]);
    hi[j] = std::min(S.bmax[j], E.hi[j]);
    if (local) {
      lo[j] = std::max(lo[j], centre[j] - radius);
      hi[j] = std::min(hi[j], centre[j] + radius);
    }
    if (hi[j] < lo[j]) hi[j] = lo[j];
  }
  std::vector<Vec> P(Q, Vec(p));
  for (int q = 0; q < Q; ++q)
    for (int j = 0; j < p; ++j) {
      const double v = q == 0 ? centre[j] : centre[j] + radius * (2.0 * rng.uniform() - 1.0);
      P[q][j] = std::min(std::max(v, lo[j]), hi[j]);
    }
  std::vector<float> hq((size_t)Q * p), hs(Q), hg((size_t)Q * p);
  auto upload = [&]() -> int {
    for (int q = 0; q < Q; ++q)
      for (int j = 0; j < p; ++j) hq[(size_t)q * p + j] = (float)((P[q][j] - S.mu[j]) / S.sd[j]);
    SBV_CUDA_TRY(ctx, cudaMemcpy(S.d_q, hq.data(), hq.size() * 4, cudaMemcpyHostToDevice));
    return SBV_OK;
  };
  int st = 0;
  for (int it = 0; it < so.ascent_iters; ++it) {
    if ((st = upload())) return st;
    if ((st = sbv_mlp_predict(S.net, S.d_q, Q, S.d_s, S.d_g, s))) return st;
    SBV_CUDA_TRY(ctx, cudaMemcpy(hg.data(), S.d_g, hg.size() * 4, cudaMemcpyDeviceToHost));
    for (int q = 0; q < Q; ++q)
      for (int j = 0; j < p; ++j) {
        const float gj = hg[(size_t)q * p + j];
        const double step = 0.005 * (hi[j] - lo[j]) * (gj > 0.f ? 1.0 : (gj < 0.f ? -1.0 : 0.0));
        P[q][j] = std::min(std::max(P[q][j] + step, lo[j]), hi[j]);
      }
  }
  if ((st = upload())) return st;
  if ((st = sbv_mlp_predict(S.net, S.d_q, Q, S.d_s, nullptr, s))) return st;
  SBV_CUDA_TRY(ctx, cudaMemcpy(hs.data(), S.d_s, hs.size() * 4, cudaMemcpyDeviceToHost));
  std::vector<int> order(Q);
  for (int q = 0; q < Q; ++q) order[q] = q;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hs[a] > hs[b]; });
  for (int q : order) {
    if ((int)cand.size() >= k) break;
    bool far = true;
    for (const Vec& c : cand) {
      double dist = 0.0;
      for (int j = 0; j < p; ++j) dist = std::max(dist, fabs(c[j] - P[q][j]));
      far = far && dist > sep;
    }
    if (far) cand.push_back(P[q]);
  }
  return SBV_OK;
}

// Restart proposal: fit to the whole history, climb from points around the
// start over the box the history spans.
int propose(Evaluator& E, Surrogate& S, const sbv_surrogate_opts& so, const Vec& u_start,
            Mix64& rng, std::vector<Vec>& cand) {
  int st = fit(E, S, so);
  if (st) return st;
  return ascend(E, S, so, u_start, so.ascent_radius, false, so.candidates, 0.05, rng, cand);
}

// Proposals inside the BFGS loop: every iteration the network's maximisers
// within the trust radius of the iterate join the line search's call, and
// the exact values decide.  The radius doubles (up to ascent_radius) when a
// proposal wins the call and halves (down to step_radius / 64) when it does
// not; the network is refitted to the grown history every refit_every
// accepted iterations.
struct InLoop {
  Surrogate* S = nullptr;
  const sbv_surrogate_opts* so = nullptr;
  Mix64* rng = nullptr;
  int since_fit = 0;   // accepted iterations since the last fit
};

// BFGS on -l with the inverse-Hessian update; H0 = 0.1 I
int bfgs(Evaluator& E, const Vec& u0, const sbv_mle_opts& o, Vec& u_out, sbv_mle_result& r,
         InLoop* IL = nullptr) {
  const int p = E.p;
  const int64_t ev0 = E.evals;
  const size_t h0 = E.hist_l.size();
  const int c0 = E.calls;
  const int64_t gv0 = E.grad_evals;
  const double h = o.fd_step;
  const bool analytic = o.gradient == 1;
  Vec u = E.clamp(u0), g, gn;
  Vec F;
  double f = 0.0;
  int st = 0;
  if (analytic) {
    if ((st = E.eval_grad(u, f, g))) return st;
  } else {
    std::vector<Vec> U{u};
    if ((st = E.eval(U, F))) return st;
    f = F[0];
    if ((st = fd_gradient(E, u, h, g))) return st;
  }
  std::vector<double> H((size_t)p * p, 0.0);
  auto reset = [&]() {
    std::fill(H.begin(), H.end(), 0.0);
    for (int j = 0; j < p; ++j) H[(size_t)j * p + j] = 0.1;
  };
  reset();
  bool fresh = true;
  int iters = 0, conv = 0;
  const int L = o.line_points;
  const int kp = IL ? IL->so->step_candidates : 0;
  const int per_iter = L + (analytic ? 1 : 2 * p) + kp;
  double radius = IL ? IL->so->step_radius : 0.0;
  const double rmin = radius / 64.0;
  int won = 0;
  while (E.evals - ev0 + per_iter <= o.max_evals) {
    Vec dir(p, 0.0);
    double mx = 0.0;
    for (int i = 0; i < p; ++i) {
      for (int j = 0; j < p; ++j) dir[i] += H[(size_t)i * p + j] * g[j];
      mx = std::max(mx, fabs(dir[i]));
    }
    if (!(mx > 0.0)) {
      conv = 2;
      break;
    }
    if (mx > o.max_step)
      for (double& v : dir) v *= o.max_step / mx;
    std::vector<Vec> C;
    double a = 1.0;
    for (int k = 0; k < L; ++k, a *= 0.5) {
      Vec v(u);
      for (int j = 0; j < p; ++j) v[j] += a * dir[j];
      C.push_back(v);
    }
    if (kp > 0) {
      if (IL->since_fit >= IL->so->refit_every) {
        if ((st = fit(E, *IL->S, *IL->so))) return st;
        IL->since_fit = 0;
      }
      std::vector<Vec> props;
      if ((st = ascend(E, *IL->S, *IL->so, u, radius, true, kp, 0.05 * radius, *IL->rng, props)))
        return st;
      for (Vec& v : props) C.push_back(v);
    }
    if ((st = E.eval(C, F))) return st;
    int kb = 0;
    for (int k = 1; k < (int)C.size(); ++k)
      if (F[k] > F[kb]) kb = k;
    if ((int)C.size() > L) {
      if (kb >= L) {
        ++won;
        radius = std::min(2.0 * radius, IL->so->ascent_radius);
      } else {
        radius = std::max(0.5 * radius, rmin);
      }
    }
    if (!(F[kb] > f + 1e-12 * fabs(f))) {
      if (fresh) {
        conv = 2;   // no ascent along the gradient direction: stationary
        break;
      }
      reset();
      fresh = true;
      continue;
    }
    ++iters;
    if (IL) ++IL->since_fit;
    Vec un = C[kb];   // clamped by the evaluator
    double fn = F[kb];
    if (analytic) {
      // the FP64 value at the accepted point replaces the line search's one
      if ((st = E.eval_grad(un, fn, gn))) return st;
    } else if ((st = fd_gradient(E, un, h, gn))) {
      return st;
    }
    Vec s(p), yv(p);
    double ys = 0.0;
    for (int j = 0; j < p; ++j) {
      s[j] = un[j] - u[j];
      yv[j] = -(gn[j] - g[j]);
      ys += yv[j] * s[j];
    }
    if (ys > 1e-12) {
      // H <- (I - r s y^T) H (I - r y s^T) + r s s^T
      const double rr = 1.0 / ys;
      Vec Hy(p, 0.0), yH(p, 0.0);
      for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) {
          Hy[i] += H[(size_t)i * p + j] * yv[j];
          yH[j] += yv[i] * H[(size_t)i * p + j];
        }
      double yHy = 0.0;
      for (int j = 0; j < p; ++j) yHy += yv[j] * Hy[j];
      for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j)
          H[(size_t)i * p + j] += -rr * (s[i] * yH[j] + Hy[i] * s[j]) + (rr * rr * yHy + rr) * s[i] * s[j];
      fresh = false;
    }
    const double gain = fn - f;
    u = un;
    f = fn;
    g = gn;
    if (gain < o.ftol * fabs(f)) {
      conv = 1;
      break;
    }
  }
  // the result is the best row the exact likelihood saw in this run (a
  // stencil point can beat the last iterate by rounding-level amounts)
  size_t kb = h0;
  for (size_t i = h0; i < E.hist_l.size(); ++i)
    if (E.hist_l[i] > E.hist_l[kb]) kb = i;
  u_out = E.hist_l[kb] > f ? E.hist_u[kb] : u;
  r.ll = std::max(E.hist_l[kb], f);
  r.evals = (int32_t)(E.evals - ev0);
  r.calls = E.calls - c0;
  r.iterations = iters;
  r.converged = conv;
  r.grad_evals = (int32_t)(E.grad_evals - gv0);
  r.proposals_won = won;
  return SBV_OK;
}

int make_problem(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n, int32_t d,
                 const int64_t* ptr, const int32_t* pts, const int32_t* nbr, const int32_t* cnt,
                 int64_t bc, int32_t m, int32_t nmax, const sbv_mle_opts& o, void* stream,
                 Problem* pb) {
  if (!ctx) return SBV_EINVAL;
  if (!X || !y || !ptr || !pts || !cnt || (m > 0 && !nbr))
    return fail(ctx, SBV_EINVAL, "null pointer argument");
  if ((dtype != SBV_F64 && dtype != SBV_F32) || n < 1 || d < 1 || d > SBV_MAX_DIM || bc < 1 ||
      bc > n || m < 0 || nmax < 0)
    return fail(ctx, SBV_EINVAL, "bad sizes");
  int st = check_opts(ctx, o);
  if (st) return st;
  SBV_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (nmax == 0 && (st = run_max_n(ctx, ptr, cnt, bc, &nmax, s))) return st;
  *pb = Problem{ctx, X, dtype, y, n, d, ptr, pts, nbr, cnt, bc, m, nmax, o.nu2, o.precision, s};
  return SBV_OK;
}

int set_bounds(Evaluator& E, const double* lower, const double* upper) {
  const int p = E.p, d = p - 2;
  E.lo.assign(p, 0.0);
  E.hi.assign(p, 0.0);
  for (int j = 0; j < p; ++j) {
    const double dl = j == 0 ? 1e-6 : (j == 1 ? 1e-10 : 1e-4);
    const double du = j == 0 ? 1e6 : (j == 1 ? 1e3 : 1e3);
    const double l = lower ? lower[j] : dl, u = upper ? upper[j] : du;
    if (!(l > 0.0) || !(u >= l) || !isfinite(u))
      return fail(E.pb.ctx, SBV_EINVAL, "bound %d invalid (0 < lower <= upper < inf)", j);
    E.lo[j] = log(l);
    E.hi[j] = log(u);
  }
  (void)d;
  return SBV_OK;
}

Vec log_start(const Evaluator& E, const double* theta) {
  Vec u(E.p);
  for (int j = 0; j < E.p; ++j) u[j] = theta[j] > 0.0 ? log(theta[j]) : E.lo[j];
  return E.clamp(u);
}

void write_history(const Evaluator& E, int64_t from, double* hist_u, double* hist_l, int64_t cap,
                   int64_t* len) {
  if (!len) return;
  int64_t k = 0;
  for (int64_t i = from; i < (int64_t)E.hist_l.size() && k < cap; ++i, ++k) {
    if (hist_u)
      for (int j = 0; j < E.p; ++j) hist_u[k * E.p + j] = E.hist_u[i][j];
    if (hist_l) hist_l[k] = E.hist_l[i];
  }
  *len = k;
}

sbv_surrogate_opts default_surrogate_opts() {
  sbv_surrogate_opts o;
  memset(&o, 0, sizeof(o));
  o.exact_starts = 4;
  o.train_steps = 4000;
  o.batch = 512;
  o.lr = 1e-3f;
  o.ascent_starts = 256;
  o.ascent_iters = 300;
  o.candidates = 8;
  o.ascent_radius = 1.0;
  o.seed = 1;
  o.step_candidates = 2;
  o.step_radius = 0.5;
  o.refit_every = 10;
  return o;
}

}  // namespace

extern "C" int sbv_mle(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n,
                       int32_t d, const int64_t* ptr, const int32_t* pts, const int32_t* nbr,
                       const int32_t* cnt, int64_t bc, int32_t m, int32_t nmax,
                       const double* theta0, const double* lower, const double* upper,
                       const sbv_mle_opts* opts, double* theta_out, sbv_mle_result* result,
                       double* hist_u, double* hist_l, int64_t hist_cap, int64_t* hist_len,
                       void* stream) {
  const sbv_mle_opts o = opts ? *opts : default_opts();
  Problem pb;
  int st = make_problem(ctx, X, dtype, y, n, d, ptr, pts, nbr, cnt, bc, m, nmax, o, stream, &pb);
  if (st) return st;
  if (!theta0 || !theta_out) return fail(ctx, SBV_EINVAL, "theta0 and theta_out are required");
  Evaluator E;
  E.pb = pb;
  E.p = d + 2;
  if ((st = set_bounds(E, lower, upper))) return st;
  Vec u;
  sbv_mle_result r;
  memset(&r, 0, sizeof(r));
  if ((st = bfgs(E, log_start(E, theta0), o, u, r))) return st;
  for (int j = 0; j < E.p; ++j) theta_out[j] = exp(u[j]);
  if (result) *result = r;
  write_history(E, 0, hist_u, hist_l, hist_cap, hist_len);
  return SBV_OK;
}

extern "C" int sbv_mle_multistart(sbv_ctx* ctx, const void* X, int dtype, const double* y,
                                  int64_t n, int32_t d, const int64_t* ptr, const int32_t* pts,
                                  const int32_t* nbr, const int32_t* cnt, int64_t bc, int32_t m,
                                  int32_t nmax, const double* starts, int32_t S,
                                  const double* lower, const double* upper,
                                  const sbv_mle_opts* opts, sbv_mlp* mlp,
                                  const sbv_surrogate_opts* sopts, const double* prior_u,
                                  const double* prior_l, int64_t prior_n, double* theta_out,
                                  sbv_mle_result* results, void* stream) {
  const sbv_mle_opts o = opts ? *opts : default_opts();
  const sbv_surrogate_opts so = sopts ? *sopts : default_surrogate_opts();
  Problem pb;
  int st = make_problem(ctx, X, dtype, y, n, d, ptr, pts, nbr, cnt, bc, m, nmax, o, stream, &pb);
  if (st) return st;
  if (!starts || S < 1 || !theta_out || !results)
    return fail(ctx, SBV_EINVAL, "starts, S >= 1, theta_out and results are required");
  if (mlp && (so.exact_starts < 0 || so.train_steps < 1 || so.batch < 1 || !(so.lr > 0.f) ||
              so.ascent_starts < 1 || so.ascent_iters < 0 || so.candidates < 0 ||
              !(so.ascent_radius >= 0.0) || so.step_candidates < 0 || so.step_candidates > 64 ||
              !(so.step_radius > 0.0) || !(so.step_radius <= so.ascent_radius) ||
              so.refit_every < 1))
    return fail(ctx, SBV_EINVAL, "bad surrogate options");
  if (prior_n < 0 || (prior_n > 0 && (!prior_u || !prior_l)))
    return fail(ctx, SBV_EINVAL, "prior_n >= 0 rows of prior_u and prior_l required");
  Evaluator E;
  E.pb = pb;
  E.p = d + 2;
  if ((st = set_bounds(E, lower, upper))) return st;
  // pairs of earlier runs join the history (they count as no evaluation here)
  for (int64_t i = 0; i < prior_n; ++i) {
    E.hist_u.emplace_back(prior_u + i * E.p, prior_u + (i + 1) * E.p);
    E.hist_l.push_back(isfinite(prior_l[i]) ? prior_l[i] : -INFINITY);
  }
  Surrogate Sg;
  Sg.net = mlp;
  if (mlp) {
    const int64_t np = sbv_mlp_num_params(E.p);
    if (np < 0) return fail(ctx, SBV_EINVAL, "the network takes at most %d inputs", SBV_MLP_MAX_IN);
    Sg.init.resize((size_t)np);
    if ((st = sbv_mlp_get_params(mlp, Sg.init.data(), np))) return st;
  }
  Mix64 rng{so.seed};
  for (int i = 0; i < S; ++i) {
    Vec u0 = log_start(E, starts + (size_t)i * E.p);
    sbv_mle_result r;
    memset(&r, 0, sizeof(r));
    const int64_t ev0 = E.evals;
    const int c0 = E.calls;
    InLoop il;
    il.S = &Sg;
    il.so = &so;
    il.rng = &rng;
    il.since_fit = so.refit_every;   // fit before the first in-loop proposal ...
    if (mlp && i >= so.exact_starts && so.candidates > 0) {
      std::vector<Vec> cand;
      if ((st = propose(E, Sg, so, u0, rng, cand))) return st;
      il.since_fit = 0;              // ... unless the restart proposal just did
      if (!cand.empty()) {
        cand.push_back(u0);   // the start itself competes: the exact values decide
        Vec F;
        if ((st = E.eval(cand, F))) return st;
        int kb = (int)cand.size() - 1;
        for (int k = 0; k < (int)cand.size(); ++k)
          if (F[k] > F[kb]) kb = k;
        u0 = cand[kb];
      }
    }
    Vec u;
    const bool inloop = mlp && i >= so.exact_starts && so.step_candidates > 0;
    if ((st = bfgs(E, u0, o, u, r, inloop ? &il : nullptr))) return st;
    r.evals = (int32_t)(E.evals - ev0);   // proposal calls included
    r.calls = E.calls - c0;
    for (int j = 0; j < E.p; ++j) theta_out[(size_t)i * E.p + j] = exp(u[j]);
    results[i] = r;
  }
  return SBV_OK;   // the network keeps its last fit
}
