"""Maximum-likelihood estimation on the GPU against the oracle, and what the
surrogate network gains for restarts.

- Scale family (tau^2 -> 0, ranges fixed by equal bounds): sbv_mle must find
  sigma^2 = Q/n, with Q from two oracle evaluations at tau^2 = 0.
- All parameters free on a small problem: the GPU optimum, scored by the
  oracle, equals the oracle optimiser's optimum.
- Restarts (sine-sum data, 12 parameters, several local maxima; FP64
  likelihood so that the paths do not hinge on rounding): after
  `exact_starts` exact runs, restarts that begin from the network's proposals
  need fewer exact likelihood rows (bar: 80%) and end, on average, at better
  maxima than restarts from the given points.  They exploit the basins the
  history has seen; a random restart can still land in an unseen, better
  basin, so neither the best single maximum nor a per-start comparison is
  asserted.
- Proposals inside the loop (the same data): the pairs of exact runs from 8
  starts train the network (passed as prior history); from 8 further starts
  BFGS runs exact-only and with the network's maximisers in every
  line-search call, alone and together with the restart proposal.  Both
  need fewer exact rows, proposals win line searches, and most starts end at
  the same or a better maximum.
"""
import numpy as np
import pytest
import torch

from oracle import mle as omle
from oracle import sbv
from synth.inputs import uniform_points, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2504_12004_gb300 import build, Context
    build.build()
    return Context(0)


def small_problem(ctx, n, d, bc, m, theta_true, nu2, seed):
    X = uniform_points(n, d, seed)
    beta = np.full(d, 0.3)
    idx = np.arange(n)
    S = sbv.cov_points(X, idx, idx, theta_true, nu2)
    y = np.linalg.cholesky(S) @ np.random.default_rng(seed + 1).standard_normal(n)
    b = sbv.blocking(X, beta, bc, 3, seed)
    nbr, cnt = sbv.knn(b["Z"], b["blk"], b["rank"], b["centres"], m)
    def i32(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()
    dev = dict(X=torch.from_numpy(X).cuda(), y=torch.from_numpy(y).cuda(),
               ptr=torch.from_numpy(np.asarray(b["ptr"], dtype=np.int64)).cuda(), pts=i32(b["pts"]),
               nbr=i32(nbr), cnt=i32(cnt))
    f = omle.make_loglik(X, y, b["ptr"], b["pts"], nbr, cnt, b["rank"], nu2)
    return dev, f


def test_scale_family_closed_form(ctx):
    from paper_2504_12004_gb300._lib import mle_opts
    theta = np.array([1.3, 0.0, 0.2, 0.5])
    dev, f = small_problem(ctx, 400, 2, 40, 12, theta, 1, 5)
    want = omle.sigma2_closed_form(f, theta, 400)
    tiny = 1e-13   # tau^2 held at a value whose effect is far below the tolerance
    lower = np.array([1e-3, tiny, 0.2, 0.5])
    upper = np.array([1e3, tiny, 0.2, 0.5])
    th, res = ctx.sbv_mle(dev["X"], dev["y"], dev["ptr"], dev["pts"], dev["nbr"], dev["cnt"],
                          [1.0, tiny, 0.2, 0.5], lower, upper, mle_opts(precision="fp64", nu2=1))
    assert abs(th[0] - want) <= 1e-5 * want, (th[0], want, res.as_dict())
    assert res.converged in (1, 2)


def test_optimum_matches_oracle_optimiser(ctx):
    from paper_2504_12004_gb300._lib import mle_opts
    theta_true = np.array([1.2, 0.02, 0.15, 0.4])
    dev, f = small_problem(ctx, 600, 2, 60, 15, theta_true, 5, 7)
    theta0 = np.array([0.7, 0.05, 0.5, 0.5])
    lower = np.array([1e-3, 1e-6, 1e-3, 1e-3])
    upper = np.array([1e2, 1e1, 1e1, 1e1])
    th_o, l_o, _ = omle.mle(f, theta0, lower=lower, upper=upper)
    th_g, res = ctx.sbv_mle(dev["X"], dev["y"], dev["ptr"], dev["pts"], dev["nbr"], dev["cnt"],
                            theta0, lower, upper, mle_opts(precision="fp64"))
    l_g = f(th_g)                     # the GPU optimum scored by the oracle
    assert abs(res.ll - l_g) <= 1e-9 * 600
    assert l_g >= f(theta0)
    assert abs(l_g - l_o) <= 1e-7 * abs(l_o) + 1e-5, (l_g, l_o, th_g, th_o)


def test_history_records_every_row(ctx):
    from paper_2504_12004_gb300._lib import mle_opts
    dev, f = small_problem(ctx, 300, 2, 30, 10, np.array([1.0, 0.01, 0.2, 0.3]), 5, 9)
    th, res, (hu, hl) = ctx.sbv_mle(dev["X"], dev["y"], dev["ptr"], dev["pts"], dev["nbr"], dev["cnt"],
                                    [1.0, 0.01, 0.3, 0.3], opts=mle_opts(precision="fp64", max_evals=300),
                                    history=10000)
    assert len(hl) == res.evals and res.evals <= 300
    k = int(np.argmax(hl))
    assert abs(hl[k] - f(np.exp(hu[k]))) <= 1e-9 * 300
    assert hl.max() == pytest.approx(res.ll, abs=0)


def lhs(rs, n, lo, hi):
    P = np.stack([rs.permutation(n) for _ in range(len(lo))], 1)
    return lo + (P + rs.uniform(size=(n, len(lo)))) / n * (hi - lo)


def test_surrogate_restarts_need_fewer_exact_rows(ctx):
    from paper_2504_12004_gb300 import Mlp
    from paper_2504_12004_gb300._lib import mle_opts, surrogate_opts
    w = workload("sine10d", n=20000, bc=400, m=60)
    X = torch.from_numpy(w["X"]).cuda()
    y = torch.from_numpy(w["y"]).cuda()
    b = ctx.sbv_blocking(X, w["beta_scale"], w["bc"], 3, 11)
    nbr, cnt = ctx.sbv_knn(X, w["beta_scale"], b["ptr"], b["pts"], b["rank"], b["centres"], w["m"])
    nbr = nbr.contiguous()
    d = X.shape[1]
    p = d + 2
    lower = np.r_[1e-2, 1e-6, np.full(d, 1e-2)]
    upper = np.r_[1e2, 1e1, np.full(d, 1e1)]
    vy = float(np.var(w["y"]))
    centre = np.log(np.r_[vy, 0.01 * vy, np.full(d, 0.5)])
    lo = np.maximum(centre - 1.5, np.log(lower))
    hi = np.minimum(centre + 1.5, np.log(upper))
    starts = np.exp(lhs(np.random.default_rng(123), 12, lo, hi))
    S0 = 8
    # FP64 likelihood: the optimisation paths must not hinge on rounding-level
    # changes of the mixed kernel
    opts = mle_opts(precision="fp64", max_evals=4000)
    args = (X, y, b["ptr"], b["pts"], nbr, cnt, starts, lower, upper, opts)
    th_e, res_e = ctx.sbv_mle_multistart(*args)
    net = Mlp(ctx, p, seed=1)
    th_s, res_s = ctx.sbv_mle_multistart(*args, mlp=net,
                                         sopts=surrogate_opts(exact_starts=S0, step_candidates=0))
    # the first S0 starts do not involve the network: identical runs
    for i in range(S0):
        assert res_e[i].ll == res_s[i].ll and res_e[i].evals == res_s[i].evals
    ev_e = sum(r.evals for r in res_e[S0:])
    ev_s = sum(r.evals for r in res_s[S0:])
    ll_e = [r.ll for r in res_e[S0:]]
    ll_s = [r.ll for r in res_s[S0:]]
    print("exact restarts:", ev_e, np.round(ll_e, 3), "surrogate restarts:", ev_s, np.round(ll_s, 3))
    assert ev_s <= 0.8 * ev_e
    # better on average; a single proposal-started run can still end in a
    # worse basin than the run from its own start (measured once: one of four)
    assert np.mean(ll_s) >= np.mean(ll_e)


def test_analytic_gradient_reaches_the_optimum_with_fewer_rows(ctx):
    """BFGS with sbv_loglik_grad at each accepted point instead of central
    differences: same optimum as the oracle's optimiser, far fewer exact rows."""
    import time
    from paper_2504_12004_gb300._lib import mle_opts
    theta_true = np.array([1.2, 0.02, 0.15, 0.4])
    dev, f = small_problem(ctx, 600, 2, 60, 15, theta_true, 5, 7)
    theta0 = np.array([0.7, 0.05, 0.5, 0.5])
    lower = np.array([1e-3, 1e-6, 1e-3, 1e-3])
    upper = np.array([1e2, 1e1, 1e1, 1e1])
    th_o, l_o, _ = omle.mle(f, theta0, lower=lower, upper=upper)
    args = (dev["X"], dev["y"], dev["ptr"], dev["pts"], dev["nbr"], dev["cnt"], theta0, lower, upper)
    t0 = time.perf_counter()
    th_a, res_a = ctx.sbv_mle(*args, mle_opts(precision="fp64", gradient="analytic"))
    t1 = time.perf_counter()
    th_d, res_d = ctx.sbv_mle(*args, mle_opts(precision="fp64"))
    t2 = time.perf_counter()
    print("analytic:", res_a.as_dict(), f"{t1 - t0:.3f} s", " differences:", res_d.as_dict(),
          f"{t2 - t1:.3f} s")
    l_a = f(th_a)
    assert abs(res_a.ll - l_a) <= 1e-9 * 600
    assert abs(l_a - l_o) <= 1e-7 * abs(l_o) + 1e-5, (l_a, l_o, th_a, th_o)
    assert res_a.grad_evals >= 1 and res_d.grad_evals == 0
    # each gradient is 1 row instead of 2 (2 + d) = 8; the 8-point line search
    # per iteration is common to both (measured: 91 against 169 rows)
    assert res_a.evals < 0.6 * res_d.evals


def test_surrogate_proposals_inside_the_loop(ctx):
    from paper_2504_12004_gb300 import Mlp
    from paper_2504_12004_gb300._lib import mle_opts, surrogate_opts
    w = workload("sine10d", n=20000, bc=400, m=60)
    X = torch.from_numpy(w["X"]).cuda()
    y = torch.from_numpy(w["y"]).cuda()
    b = ctx.sbv_blocking(X, w["beta_scale"], w["bc"], 3, 11)
    nbr, cnt = ctx.sbv_knn(X, w["beta_scale"], b["ptr"], b["pts"], b["rank"], b["centres"], w["m"])
    S = (X, y, b["ptr"], b["pts"], nbr.contiguous(), cnt)
    d = X.shape[1]
    lower = np.r_[1e-2, 1e-6, np.full(d, 1e-2)]
    upper = np.r_[1e2, 1e1, np.full(d, 1e1)]
    vy = float(np.var(w["y"]))
    centre = np.log(np.r_[vy, 0.01 * vy, np.full(d, 0.5)])
    lo = np.maximum(centre - 1.5, np.log(lower))
    hi = np.minimum(centre + 1.5, np.log(upper))
    starts = np.exp(lhs(np.random.default_rng(123), 16, lo, hi))
    opts = mle_opts(precision="fp64", max_evals=4000)
    hu, hl = [], []
    for st in starts[:8]:
        _, _, (u_, l_) = ctx.sbv_mle(*S, st, lower, upper, opts, history=4000)
        hu.append(u_)
        hl.append(l_)
    prior = (np.concatenate(hu), np.concatenate(hl))
    later = starts[8:]
    ex = [ctx.sbv_mle(*S, st, lower, upper, opts)[1] for st in later]
    rows_e = sum(r.evals for r in ex)
    # measured: in-loop only 19,125 rows against 24,008 (7 of 8 starts at the
    # same or a better maximum, 35 line searches won); with the restart
    # proposal 12,830 (6 of 8)
    for name, so, bar in (("in-loop", surrogate_opts(exact_starts=0, candidates=0), 0.9),
                          ("restart + in-loop", surrogate_opts(exact_starts=0), 0.7)):
        _, rs = ctx.sbv_mle_multistart(*S, later, lower, upper, opts, mlp=Mlp(ctx, d + 2, seed=1),
                                       sopts=so, prior=prior)
        rows_s = sum(r.evals for r in rs)
        same_or_better = sum(s_.ll >= e.ll - 1e-4 * abs(e.ll) for s_, e in zip(rs, ex))
        won = sum(r.proposals_won for r in rs)
        print(name, rows_s, "vs", rows_e, [round(s_.ll - e.ll, 3) for s_, e in zip(rs, ex)], won)
        assert rows_s <= bar * rows_e
        assert same_or_better >= 6
        if name == "in-loop":
            assert won >= 8


def test_surrogate_option_and_prior_errors(ctx):
    from paper_2504_12004_gb300 import Mlp, SBVError
    from paper_2504_12004_gb300._lib import mle_opts, surrogate_opts
    dev, f = small_problem(ctx, 300, 2, 30, 10, np.array([1.0, 0.01, 0.2, 0.3]), 5, 9)
    S = (dev["X"], dev["y"], dev["ptr"], dev["pts"], dev["nbr"], dev["cnt"])
    start = np.array([[1.0, 0.01, 0.3, 0.3]])
    opts = mle_opts(precision="fp64", max_evals=200)
    net = Mlp(ctx, 4, seed=1)
    for bad in (surrogate_opts(step_candidates=-1), surrogate_opts(step_candidates=65),
                surrogate_opts(step_radius=0.0), surrogate_opts(step_radius=2.0, ascent_radius=1.0),
                surrogate_opts(refit_every=0), surrogate_opts(candidates=-1)):
        with pytest.raises(SBVError):
            ctx.sbv_mle_multistart(*S, start, opts=opts, mlp=net, sopts=bad)
    with pytest.raises(ValueError):
        ctx.sbv_mle_multistart(*S, start, opts=opts, prior=(np.zeros((3, 4)), np.zeros(2)))
    # prior pairs join the history but are not counted as evaluations
    _, r0 = ctx.sbv_mle_multistart(*S, start, opts=opts)
    prior = (np.log(np.tile(start, (50, 1))) + 0.01 * np.arange(50)[:, None], -np.arange(50.0))
    _, r1 = ctx.sbv_mle_multistart(*S, start, opts=opts, prior=prior)
    assert r1[0].evals == r0[0].evals and r1[0].ll == r0[0].ll
