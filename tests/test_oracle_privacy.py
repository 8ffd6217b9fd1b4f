"""Pins of the oracle's privacy-preserving SRP (§4.5: the sign of the projection plus noise),
each against something other than the oracle's own noise arithmetic: Python integers and
fractions, closed forms, and the exact binomial law (scipy)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def _g(seed, t):
    """(ones(draw t) - 32) / 4 with Python's own bit count."""
    return Fraction(bin(oracle.splitmix64_draw(seed, t)).count("1") - 32, 4)


def _pack(bits, K, L):
    n = bits.shape[0]
    ids = np.zeros((n, L), dtype=np.uint32)
    for j in range(L):
        for k in range(K):
            ids[:, j] |= bits[:, j * K + k].astype(np.uint32) << k
    return ids


def test_large_sigma_gives_the_noise_sign():
    """sigma = 2^40 dwarfs every projection: a bit is [g > 0], or the SRP bit where g = 0.
    The index of the draw is (nbase + i) K L + c."""
    d, K, L, seed, nseed, nbase = 20, 5, 7, 3, 99, 1234
    rng = np.random.default_rng(0)
    X = rng.standard_normal((40, d)).astype(np.float32)
    W = oracle.projection_from_seed(d, K, L, seed)
    s = oracle.project(X, W)
    assert np.abs(s).max() < 2 ** 10
    KL = K * L
    bits = np.zeros((40, KL), dtype=bool)
    zeros = 0
    for i in range(40):
        for c in range(KL):
            g = _g(nseed, (nbase + i) * KL + c)
            zeros += g == 0
            bits[i, c] = g > 0 if g != 0 else s[i, c] > 0
    assert zeros > 0  # P(g = 0) = C(64, 32) / 2^64, about 0.099
    got = oracle.hash_ids_noisy(X, W, K, L, 2.0 ** 40, nseed, nbase)
    assert np.array_equal(got, _pack(bits, K, L))


def test_tiny_sigma_is_plain_srp():
    """sigma = 2^-60 moves no projection of Gaussian data across zero (|eta| <= 8 * 2^-60)."""
    d, K, L = 33, 6, 9
    rng = np.random.default_rng(1)
    X = rng.standard_normal((300, d)).astype(np.float32)
    W = oracle.projection_from_seed(d, K, L, 5)
    assert np.abs(oracle.project(X, W)).min() > 2.0 ** -50
    assert np.array_equal(oracle.hash_ids_noisy(X, W, K, L, 2.0 ** -60, 7, 0), oracle.hash_ids(X, W, K, L))


def test_exact_ties_in_rational_arithmetic():
    """Integer points, W with entries k/4 (the integer-only generator) and sigma = 1: every
    projection and every eta is a multiple of 1/16, many sums are exactly 0 (bit 0).  Each bit
    equals [s + eta > 0] computed in exact rationals."""
    d, K, L, nseed, nbase = 6, 4, 5, 11, 3
    rng = np.random.default_rng(2)
    X = rng.integers(-2, 3, size=(60, d)).astype(np.float32)
    W = oracle.projection_from_seed(d, K, L, 8, counter=True)
    KL = K * L
    bits = np.zeros((60, KL), dtype=bool)
    ties = 0
    for i in range(60):
        for c in range(KL):
            s = sum(Fraction(int(X[i, t])) * Fraction(float(W[t, c])) for t in range(d))
            v = s + _g(nseed, (nbase + i) * KL + c)
            ties += v == 0
            bits[i, c] = v > 0
    assert ties >= 10
    assert np.array_equal(oracle.hash_ids_noisy(X, W, K, L, 1.0, nseed, nbase), _pack(bits, K, L))


def test_flip_frequency_follows_the_binomial_law():
    """One point hashed 6000 times with fresh noise: bit c is 1 with probability
    P(s_c + sigma (B - 32) / 4 > 0), B ~ Binomial(64, 1/2) (mean 0, variance sigma^2)."""
    stats = pytest.importorskip("scipy.stats")
    d, K, L, n, sigma = 16, 4, 4, 6000, 0.5
    rng = np.random.default_rng(3)
    x = rng.standard_normal(d).astype(np.float32)
    W = oracle.projection_from_seed(d, K, L, 6)
    s = oracle.project(x[None, :], W)[0]
    X = np.repeat(x[None, :], n, axis=0)
    ids = oracle.hash_ids_noisy(X, W, K, L, sigma, 21, 0)
    freq = np.array([((ids[:, c // K] >> (c % K)) & 1).mean() for c in range(K * L)])
    # bit = 1 iff B > 32 - 4 s / sigma
    p = stats.binom.sf(np.floor(32 - 4 * s / sigma), 64, 0.5)
    se = np.sqrt(np.maximum(p * (1 - p), 1e-4) / n)
    assert np.all(np.abs(freq - p) < 5 * se), np.abs(freq - p) / se
    assert np.any((p > 0.05) & (p < 0.95))  # some columns are really noisy


def test_noise_index_runs_across_calls():
    """The detector's noise index advances by each hashed batch: two calls give the same ids
    as one call over both batches; an insert_score hashes once."""
    d, K, L = 12, 5, 6
    rng = np.random.default_rng(4)
    X = rng.standard_normal((90, d)).astype(np.float32)
    W = oracle.projection_from_seed(d, K, L, 2)
    whole = oracle.hash_ids_noisy(X, W, K, L, 0.75, 5, 0)
    det = oracle.Detector(d, K, L, W=W)
    det.set_privacy(0.75, 5)
    a = det.hash(X[:35])
    b = det.hash(X[35:])
    assert np.array_equal(np.concatenate([a, b]), whole) and det.nbase == 90
    det2 = oracle.Detector(d, K, L, W=W)
    det2.set_privacy(0.75, 5)
    det2.insert_score(X[:50])
    assert det2.nbase == 50
    _, sums, _ = det2.score(X[50:])
    ids = oracle.hash_ids_noisy(X[50:], W, K, L, 0.75, 5, 50)
    assert np.array_equal(sums, oracle.gather(ids, det2.counts, K))
    with pytest.raises(ValueError):
        det2.delete(X[:1])
