"""Pins of the conditional-simulation oracle (Sec. 5.5) against facts that do
not come from the oracle itself: numpy's own Philox implementation and the
published known-answer vector of Philox4x64-10, the normal law (KS test),
the sampling distribution of the sample mean and variance, the coverage of
the 95 % interval, and scipy's normal quantile.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import simulate as osim

MASK = (1 << 64) - 1


def numpy_block(counter, key):
    """Four raw words of numpy's Philox (4 x 64, 10 rounds) for one counter
    value: numpy advances its 256-bit counter before it produces a block, so
    it starts one below."""
    c = sum(int(v) << (64 * i) for i, v in enumerate(counter))
    c = (c - 1) % (1 << 256)
    words = np.array([(c >> (64 * i)) & MASK for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(counter=words, key=np.array(key, dtype=np.uint64))
    return [int(v) for v in bg.random_raw(4)]


def test_philox_matches_numpy_implementation():
    rng = np.random.default_rng(17)
    cases = [((0, 0, 0, 0), (0, 0)), ((1, 2, 3, 4), (5, 6)), ((MASK, MASK, MASK, MASK), (MASK, MASK))]
    for _ in range(40):
        cases.append((tuple(int(v) for v in rng.integers(0, 2**63, 4)),
                      tuple(int(v) for v in rng.integers(0, 2**63, 2))))
    for ctr, key in cases:
        assert osim.philox4x64(ctr, key) == numpy_block(ctr, key), (ctr, key)


def test_philox_known_answer_zero():
    # the known-answer vector of Philox4x64-10 for zero counter and key
    # published with the generator's reference implementation (Random123)
    assert osim.philox4x64((0, 0, 0, 0), (0, 0)) == [
        0x16554D9ECA36314C, 0xDB20FE9D672D0FDC, 0xD7E772CEE186176B, 0x7E68B68AEC7BA23B]


def test_rounds_matter():
    # fewer rounds give a different block (the round count is not ignored)
    assert osim.philox4x64((3, 1, 4, 1), (5, 9), rounds=7) != osim.philox4x64((3, 1, 4, 1), (5, 9))


def test_normals_follow_the_normal_law():
    z = np.concatenate([osim.std_normals(j, 4000, 20240601) for j in range(5)])
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the two members of a Box-Muller pair are uncorrelated
    c = np.corrcoef(z[0::2], z[1::2])[0, 1]
    assert abs(c) < 4 / np.sqrt(z.size / 2)
    # draws of distinct test points are distinct streams
    assert not np.allclose(osim.std_normals(0, 64, 1), osim.std_normals(1, 64, 1))
    assert not np.allclose(osim.std_normals(0, 64, 1), osim.std_normals(0, 64, 2))


def test_uniform_map_is_open_and_centred():
    assert osim.unit_open(0) == 2.0**-53
    assert osim.unit_open(MASK) == 1.0 - 2.0**-53
    assert 0.0 < osim.unit_open(0) and osim.unit_open(MASK) < 1.0


def test_z975_is_the_normal_quantile():
    assert osim.Z975 == pytest.approx(stats.norm.ppf(0.975), rel=1e-15)


def test_sample_statistics_have_their_sampling_laws():
    rng = np.random.default_rng(4)
    nt, nd = 400, 100
    mean = rng.normal(0.0, 3.0, nt)
    var = rng.uniform(0.1, 4.0, nt)
    draws, mu, s2, lo, hi = osim.simulate(mean, var, nd, seed=99)
    assert draws.shape == (nt, nd)
    # (mu~ - mu) / (sigma / sqrt(n)) ~ N(0, 1) over the test points
    t = (mu - mean) / np.sqrt(var / nd)
    assert abs(t.mean()) < 4 / np.sqrt(nt)
    assert 0.75 < t.var() < 1.3
    # (n - 1) s^2 / sigma^2 ~ chi^2_{n-1}: mean n - 1
    q = (nd - 1) * s2 / var
    assert abs(q.mean() - (nd - 1)) < 4 * np.sqrt(2 * (nd - 1) / nt)
    # the statistics are those of the returned draws
    np.testing.assert_allclose(mu, draws.mean(axis=1), rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(s2, draws.var(axis=1, ddof=1), rtol=1e-12)
    np.testing.assert_allclose(hi - lo, 2 * stats.norm.ppf(0.975) * np.sqrt(s2), rtol=1e-12)


def test_interval_covers_fresh_draws_at_95_percent():
    rng = np.random.default_rng(8)
    nt = 200
    mean = rng.normal(0.0, 1.0, nt)
    var = rng.uniform(0.5, 2.0, nt)
    _, _, _, lo, hi = osim.simulate(mean, var, 1000, seed=5)
    fresh = mean[:, None] + np.sqrt(var)[:, None] * rng.standard_normal((nt, 50))
    cover = np.mean((fresh >= lo[:, None]) & (fresh <= hi[:, None]))
    assert 0.935 < cover < 0.965


def test_zero_variance_and_index_base():
    draws, mu, s2, lo, hi = osim.simulate(np.array([2.5, -1.0]), np.array([0.0, 0.0]), 7, seed=1)
    assert np.all(draws == np.array([[2.5], [-1.0]]))
    assert np.all(s2 == 0.0) and np.all(lo == mu) and np.all(hi == mu)
    # a chunk that starts at index_base draws as those points of the whole set
    mean, var = np.arange(6.0), np.full(6, 2.0)
    whole = osim.simulate(mean, var, 9, seed=3)[0]
    part = osim.simulate(mean[4:], var[4:], 9, seed=3, index_base=4)[0]
    np.testing.assert_array_equal(part, whole[4:])
