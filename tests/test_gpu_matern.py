"""The covariance arithmetic of both precisions on its own (sbv_matern): the
double-float square root, exponential and Matern polynomial of the mixed
kernel against the closed forms in FP64 (relative error bounds of ~48-bit
arithmetic), the FP64 closed forms, and the FP64 path's K_nu quadrature
against scipy's K_nu (an independent implementation).
"""
import numpy as np
import pytest
import torch
from scipy.special import gamma, kv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2504_12004_gb300 import build, Context
    build.build()
    return Context(0)


def closed_form(r, nu2):
    r = np.asarray(r, dtype=np.float64)
    e = np.exp(-r)
    return {1: e, 3: (1 + r) * e, 5: (1 + r + r * r / 3) * e,
            7: (1 + r + 2 * r * r / 5 + r ** 3 / 15) * e}[nu2]


def distances():
    # squared scaled distances from 0 (the diagonal) through the range where
    # exp(-r) is still a normal float pair (r <= 60), plus a far tail
    r = np.concatenate([[0.0], np.logspace(-7, -1, 200), np.linspace(0.1, 60.0, 6000),
                        np.linspace(60.0, 84.0, 50)])
    return r * r


@pytest.mark.parametrize("nu2", [1, 3, 5, 7])
def test_double_float_matern_against_fp64(ctx, nu2):
    d2 = distances()
    d = torch.from_numpy(d2).cuda()
    got = ctx.sbv_matern(d, nu2, "mixed").cpu().numpy()
    ref = closed_form(np.sqrt(d2), nu2)
    r = np.sqrt(d2)
    # up to r = 60 the tail of the float pair is a normal float
    near = r <= 60.0
    # ~48-bit arithmetic: the split of d2 into a float pair, the
    # Newton-corrected square root, r / ln 2 and the table and Taylor steps of
    # the exponential each round at a few units of 2^-48 = 3.6e-15 relative;
    # exp(-r) has condition number r with respect to r, so the relative error
    # of the result grows like (a few) 2^-48 (1 + r)
    rel = np.abs(got[near] - ref[near]) / ref[near]
    bound = 1.5e-14 * (1.0 + r[near])
    assert np.all(rel <= bound), (rel.max(), r[near][np.argmax(rel / bound)])
    # further out the tail float loses bits to underflow (entries below
    # 1e-26 of the diagonal, irrelevant to any factorisation)
    assert np.all(np.abs(got[~near] - ref[~near]) <= 1e-8 * ref[~near] + 1e-44)
    assert got[0] == 1.0
    # the mixed and bf16 precisions share the covariance arithmetic
    assert torch.equal(ctx.sbv_matern(d, nu2, "mixed_bf16"), ctx.sbv_matern(d, nu2, "mixed"))


def test_double_float_exp_is_monotone_and_exact_at_zero(ctx):
    d2 = np.linspace(0.0, 4.0, 100001) ** 2
    got = ctx.sbv_matern(torch.from_numpy(d2).cuda(), 1, "mixed").cpu().numpy()
    assert got[0] == 1.0
    assert np.all(np.diff(got) <= 0.0)
    # exp(-r) against FP64 over a dense grid (table boundaries included)
    r = np.sqrt(d2)
    rel = np.abs(got - np.exp(-r)) / np.exp(-r)
    assert np.all(rel <= 1.5e-14 * (1.0 + r))


@pytest.mark.parametrize("nu2", [1, 3, 5, 7])
def test_fp64_closed_forms(ctx, nu2):
    d2 = distances()
    got = ctx.sbv_matern(torch.from_numpy(d2).cuda(), nu2, "fp64").cpu().numpy()
    ref = closed_form(np.sqrt(d2), nu2)
    np.testing.assert_allclose(got, ref, rtol=4e-15, atol=1e-300)


@pytest.mark.parametrize("nu2", [2, 4, 6, 9, 13, 20, 40])
def test_fp64_general_nu_against_scipy(ctx, nu2):
    nu = nu2 / 2
    r = np.concatenate([np.logspace(-6, -1, 50), np.linspace(0.1, 60.0, 600)])
    got = ctx.sbv_matern(torch.from_numpy(r * r).cuda(), nu2, "fp64").cpu().numpy()
    ref = 2.0 ** (1 - nu) / gamma(nu) * r ** nu * kv(nu, r)
    rel = np.abs(got - ref) / ref
    assert rel.max() < 1e-11, (rel.max(), r[rel.argmax()])


def test_matern_rejects_bad_arguments(ctx):
    from paper_2504_12004_gb300 import SBVError
    d = torch.ones(3, dtype=torch.float64, device="cuda")
    with pytest.raises(SBVError):
        ctx.sbv_matern(d, 4, "mixed")     # general nu is FP64 only
    with pytest.raises(SBVError):
        ctx.sbv_matern(d, 0, "fp64")
    assert ctx.sbv_matern(torch.empty(0, dtype=torch.float64, device="cuda"), 5).numel() == 0
