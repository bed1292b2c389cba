"""Pins for the oracle's coin: Philox4x32-10 (Salmon et al., SC'11) and the
Bernoulli keep rule of MACH (Algorithm 1/2; Theorem 1's sampling law).

No known-answer vectors for Philox are available offline, so the generator is
pinned by what its published definition fixes: the Weyl constants are the
32-bit fractional parts of the golden ratio and of sqrt(3); the multipliers
are odd (the round is then a bijection); ten rounds give full avalanche while
a truncated generator does not; the words are uniform.  The coin is pinned
statistically (count ~ Binomial, per-index uniformity, unbiasedness of X^).
"""
import math

import numpy as np
import pytest

from oracle import mach_oracle as O


def test_weyl_constants_from_closed_forms():
    m0, m1, w0, w1 = O.philox_constants()
    assert w0 == int(math.floor((math.sqrt(5.0) - 1.0) / 2.0 * 2 ** 32))
    assert w1 == int(math.floor((math.sqrt(3.0) - 1.0) * 2 ** 32))


def test_multipliers_are_odd_32bit():
    m0, m1, _, _ = O.philox_constants()
    assert m0 % 2 == 1 and m1 % 2 == 1
    assert 2 ** 31 < m0 < 2 ** 32 and 2 ** 31 < m1 < 2 ** 32


def _avalanche(rounds, trials=64, seed=12345):
    rng = np.random.default_rng(seed)
    fracs = []
    for _ in range(trials):
        ctr = [int(v) for v in rng.integers(0, 2 ** 32, size=4, dtype=np.uint64)]
        key = [int(v) for v in rng.integers(0, 2 ** 32, size=2, dtype=np.uint64)]
        base = O.philox4x32(ctr, key, rounds)
        for bit in range(0, 128, 5):
            c2 = list(ctr)
            c2[bit // 32] ^= 1 << (bit % 32)
            out = O.philox4x32(c2, key, rounds)
            flipped = sum(bin(a ^ b).count("1") for a, b in zip(base, out))
            fracs.append(flipped / 128.0)
    return float(np.mean(fracs)), float(np.min(fracs))


def test_avalanche_ten_rounds_and_truncated_fails():
    mean10, min10 = _avalanche(10)
    assert abs(mean10 - 0.5) < 0.01
    assert min10 > 0.25
    mean2, min2 = _avalanche(2)
    assert min2 < 0.2 or abs(mean2 - 0.5) > 0.02


def test_round_count_matters():
    a = O.philox4x32([1, 2, 3, 4], [5, 6], 10)
    b = O.philox4x32([1, 2, 3, 4], [5, 6], 9)
    assert a != b


def test_words_uniform_chi_square():
    q = np.arange(200_000, dtype=np.uint64) + np.uint64(7)
    w = O.philox_batch(q, seed=0xDEADBEEF12345)
    from scipy.stats import chisquare
    for col in range(4):
        for shift in (0, 24):
            bins = np.bincount(((w[:, col] >> np.uint32(shift)) & np.uint32(255)).astype(np.int64), minlength=256)
            assert chisquare(bins).pvalue > 1e-6


def test_batch_matches_single_and_key_layout():
    seed = (0x01234567 << 32) | 0x89ABCDEF
    q = np.array([0, 1, 2 ** 32 + 5], dtype=np.uint64)
    w = O.philox_batch(q, seed)
    for i, qi in enumerate(q):
        single = O.philox4x32([int(qi) & 0xFFFFFFFF, int(qi) >> 32, 0, 0], [0x89ABCDEF, 0x01234567])
        assert list(w[i]) == single
    # the high seed word matters
    w2 = O.philox_batch(q, seed & 0xFFFFFFFF)
    assert not np.array_equal(w, w2)


def test_threshold():
    assert O.keep_threshold(1.0) == 2 ** 32
    assert O.keep_threshold(0.5) == 2 ** 31
    assert O.keep_threshold(0.1) == int(math.floor(0.1 * 2 ** 32))
    with pytest.raises(ValueError):
        O.keep_threshold(0.0)
    with pytest.raises(ValueError):
        O.keep_threshold(1.5)


def test_keep_is_word_l_mod_4_of_counter_l_div_4():
    seed = 987654321
    T = O.keep_threshold(0.3)
    q = np.arange(0, 50, dtype=np.uint64)
    w = O.philox_batch(q, seed)
    for l in range(200):
        assert O.keep(l, 0.3, seed) == (int(w[l // 4, l % 4]) < T)


def test_p_one_keeps_everything():
    idx = O.kept_indices(0, 10_000, 1.0, 42)
    assert np.array_equal(idx, np.arange(10_000))


@pytest.mark.parametrize("p", [0.01, 0.1, 0.5, 0.9])
def test_count_binomial(p):
    N = 400_000
    idx = O.kept_indices(0, N, p, 2024)
    q = O.keep_threshold(p) / 2 ** 32
    mu, sd = N * q, math.sqrt(N * q * (1 - q))
    assert abs(idx.size - mu) < 5 * sd
    assert np.all(np.diff(idx) > 0)


def test_windows_concatenate():
    p, seed = 0.2, 77
    whole = O.kept_indices(0, 5001, p, seed)
    parts = np.concatenate([O.kept_indices(a, min(5001, a + 777), p, seed) for a in range(0, 5001, 777)])
    assert np.array_equal(whole, parts)


def test_per_mode_index_uniform():
    from scipy.stats import chisquare
    dims = (40, 30, 50)
    X = np.ones(dims)
    idx, _ = O.sample(X, 0.1, 5)
    coords = np.unravel_index(idx, dims)
    for k in range(3):
        counts = np.bincount(coords[k], minlength=dims[k])
        assert chisquare(counts).pvalue > 1e-6


def test_kept_set_independent_of_values():
    rng = np.random.default_rng(0)
    X1 = rng.standard_normal((7, 8, 9))
    X2 = rng.standard_normal((7, 8, 9)) * 100.0
    X2[0, 0, :] = 0.0
    i1, v1 = O.sample(X1, 0.3, 11)
    i2, v2 = O.sample(X2, 0.3, 11)
    assert np.array_equal(i1, i2)
    assert np.array_equal(v1, X1.reshape(-1)[i1])


def test_unbiased_sampled_tensor():
    """E[X^] = X: X^ = x/p with probability p, else 0 (Theorem 1)."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((4, 3, 5))
    p = 0.2
    q = O.keep_threshold(p) / 2 ** 32
    nseed = 2000
    acc = np.zeros_like(X)
    for s in range(nseed):
        acc += O.sampled_dense(X, p, 1000 + s)
    mean = acc / nseed
    # X^ uses 1/p; its mean is X * q / p, within 2^-32 relative of X
    expect = X * q / p
    sd = np.abs(X) / p * math.sqrt(q * (1 - q) / nseed)
    z = np.abs(mean - expect) / sd
    assert np.max(z) < 5.0
    from scipy.stats import chi2
    stat = float(np.sum(z ** 2))
    assert chi2.sf(stat, X.size) > 1e-6
