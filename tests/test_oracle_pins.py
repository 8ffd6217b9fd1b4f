"""Pins for the CPU oracle: each test checks it against something the paper or the
mathematics fixes, not against a second copy of its own formulas.

* hand example (Eq. 1, Eq. 2, Algorithm 1, Eq. 11, §5.3), values worked out by hand;
* SplitMix64 published reference outputs;
* Eq. 1 / Eq. 2 collision probabilities 1 - theta/pi and (1 - theta/pi)^K, by brute force;
* Theorem 1 (§3.3): the count estimator is unbiased for S(q, D) = sum_i p_i^K (Eq. 3);
* invariants: every array sums to the number of inserts; the Q identity of Eq. 11;
  H(2^k x) = H(x); negation flips every bit whose projection is non-zero;
* library routines: numpy's float64 matmul signs, bincount, mean and population std.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1706_06664_gb300 import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ------------------------------------------------------------------------------------------
# Hand example
# ------------------------------------------------------------------------------------------
def _hand():
    g = _load("hand_example.json")
    W = np.array(g["W_columns"], dtype=np.float32).T.copy()  # d x KL, column c = W[:, c]
    X = np.array(g["X"], dtype=np.float32)
    return g, W, X


def test_hand_example_projections_and_ids():
    g, W, X = _hand()
    s = oracle.project(X, W)
    assert s.tolist() == g["projections"]
    ids = oracle.hash_ids(X, W, g["K"], g["L"])
    assert ids.tolist() == g["ids"]


def test_hand_example_insert_score_flag():
    g, W, X = _hand()
    det = oracle.Detector(g["d"], g["K"], g["L"], W=W)
    scores, sums, flags = det.insert_score(X, g["alpha"])
    assert det.counts.tolist() == g["counts"]
    assert sums.tolist() == g["sums"]
    assert scores.tolist() == g["scores"]
    assert flags.tolist() == g["flags"]
    st = det.stats(g["alpha"])
    assert st["Q"] == g["Q"]
    assert st["mu_ins"] == g["mu_ins"]
    assert st["mu"] == g["mu"]
    # sqrt, a division and a subtraction: each within half an ulp of its exact result
    assert st["sigma"] == pytest.approx(g["sigma"], rel=4 * 2.0**-53, abs=0)
    assert st["threshold"] == pytest.approx(g["threshold"], rel=4 * 2.0**-53, abs=0)


def test_hand_example_incremental_mean_eq11():
    g, W, X = _hand()
    ids = oracle.hash_ids(X, W, g["K"], g["L"])
    counts = np.zeros((g["L"], 1 << g["K"]), dtype=np.uint32)
    mu, trace = oracle.mu_incremental(ids, counts, g["K"])
    assert np.allclose(trace, g["mu_incremental_trace"], rtol=1e-15, atol=0)
    assert counts.tolist() == g["counts"]
    # the literal post-increment reading of Algorithm 1 would give 3.0 after x1
    assert trace[0] != g["mu_after_first_point_literal_post_increment_reading"]


# ------------------------------------------------------------------------------------------
# Generator
# ------------------------------------------------------------------------------------------
def test_splitmix64_reference_vectors():
    for v in _load("splitmix64.json")["vectors"]:
        assert oracle.splitmix64_draw(v["seed"], v["t"]) == v["out"]


def test_projection_from_seed_hand_derived_values():
    """Two Box-Muller pairs derived by hand from the generator's definition and the published
    SplitMix64 outputs (tests/golden/projection_pins.json): the cos half at even flat indices,
    the sin half at odd ones, and u1 in (0,1] (the first pair has draw 0 = 0, which gives
    u1 = 2^-53 and r = sqrt(106 ln 2) instead of an infinite value)."""
    g = _load("projection_pins.json")
    for pr in g["pairs"]:
        assert oracle.splitmix64_draw(pr["seed"], 0) == pr["draw0"]
        assert oracle.splitmix64_draw(pr["seed"], 1) == pr["draw1"]
        W = oracle.projection_from_seed(1, 2, 1, seed=pr["seed"])
        bits = W.ravel().view(np.uint32)
        assert int(bits[0]) == pr["flat0_f32_bits"] and int(bits[1]) == pr["flat1_f32_bits"], (W, pr)
        assert abs(float(W.ravel()[0]) - float(pr["flat0"])) < 1e-6 * abs(float(pr["flat0"]))
    assert math.isclose(float(g["pairs"][0]["r"]), math.sqrt(106 * math.log(2)), rel_tol=1e-15)
    for pr in g["pairs"]:  # the bfloat16-valued variant (ACE_W_BF16) of the same draws
        bits = oracle.projection_from_seed(1, 2, 1, seed=pr["seed"], w_bf16=True).ravel().view(np.uint32)
        assert int(bits[0]) == pr["flat0_bf16_bits"] and int(bits[1]) == pr["flat1_bf16_bits"]


def test_projection_bf16_variant_rounds_to_nearest_even():
    """ACE_W_BF16 draws are the binary32 draws rounded to bfloat16, ties to even: over a million
    entries (a dozen exact ties expected) they equal an independent rounding of the binary32
    matrix, and each lies within half a bfloat16 unit of it."""
    W = oracle.projection_from_seed(64, 16, 1024, seed=99)
    Wb = oracle.projection_from_seed(64, 16, 1024, seed=99, w_bf16=True)
    assert np.array_equal(workloads.bf16_bits_to_f32(workloads.to_bf16_bits(W)), Wb)
    assert not (Wb.view(np.uint32) & 0xFFFF).any()
    low = W.view(np.uint32) & 0xFFFF
    ties = low == 0x8000
    assert ties.sum() >= 1 and not ((Wb.view(np.uint32)[ties] >> 16) & 1).any()
    assert (np.abs(W.astype(np.float64) - Wb) <= np.abs(W.astype(np.float64)) * 2.0**-8).all()


def test_projection_from_seed_is_standard_normal():
    W = oracle.projection_from_seed(64, 16, 256, seed=12345).astype(np.float64).ravel()
    assert W.size == 64 * 16 * 256
    m, v = W.mean(), W.var()
    se = 1.0 / math.sqrt(W.size)
    assert abs(m) < 5 * se
    assert abs(v - 1.0) < 5 * math.sqrt(2.0) * se
    kurt = np.mean((W - m) ** 4) / v**2
    assert abs(kurt - 3.0) < 5 * math.sqrt(24.0) * se
    scipy_stats = pytest.importorskip("scipy.stats")
    ks = scipy_stats.kstest(W, "norm")
    assert ks.pvalue > 1e-4
    # even and odd flat indices (cos and sin halves) are each N(0,1) and uncorrelated
    e, o = W[0::2], W[1::2]
    assert abs(np.corrcoef(e, o)[0, 1]) < 5 * math.sqrt(2.0) * se
    assert scipy_stats.kstest(e, "norm").pvalue > 1e-4
    assert scipy_stats.kstest(o, "norm").pvalue > 1e-4


def test_projection_from_seed_deterministic_and_seed_dependent():
    a = oracle.projection_from_seed(5, 3, 4, seed=7)
    b = oracle.projection_from_seed(5, 3, 4, seed=7)
    c = oracle.projection_from_seed(5, 3, 4, seed=8)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    # the matrix is a prefix-stable function of the flat index: a larger L extends it
    big = oracle.projection_from_seed(5, 3, 8, seed=7)
    assert np.array_equal(big.ravel()[:4], a.ravel()[:4])


# ------------------------------------------------------------------------------------------
# Eq. 1 / Eq. 2 collision probabilities
# ------------------------------------------------------------------------------------------
def _pair_at_angle(theta, d):
    x = np.zeros(d, dtype=np.float32)
    y = np.zeros(d, dtype=np.float32)
    x[0] = 1.0
    y[0] = np.float32(math.cos(theta))
    y[1] = np.float32(math.sin(theta))
    return np.stack([x, y])


@pytest.mark.parametrize("theta", [math.pi / 6, math.pi / 3, math.pi / 2, 2 * math.pi / 3])
@pytest.mark.parametrize("source", ["seed", "numpy"])
def test_srp_collision_probability_eq1(theta, source):
    d, M = 4, 1 << 17
    W = oracle.projection_from_seed(d, 1, M, seed=99) if source == "seed" else workloads.gaussian_w(d, 1, M, 99)
    X = _pair_at_angle(theta, d)
    ids = oracle.hash_ids(X, W, 1, M)
    # recompute theta from the binary32 inputs actually hashed
    xd, yd = X.astype(np.float64)
    th = math.acos(float(xd @ yd) / (np.linalg.norm(xd) * np.linalg.norm(yd)))
    p = 1.0 - th / math.pi
    frac = float(np.mean(ids[0] == ids[1]))
    assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / M)


@pytest.mark.parametrize("K", [2, 4])
def test_srp_collision_probability_eq2(K):
    d, L = 4, 1 << 15
    theta = math.pi / 4
    W = oracle.projection_from_seed(d, K, L, seed=2024 + K)
    X = _pair_at_angle(theta, d)
    ids = oracle.hash_ids(X, W, K, L)
    xd, yd = X.astype(np.float64)
    th = math.acos(float(xd @ yd) / (np.linalg.norm(xd) * np.linalg.norm(yd)))
    p = (1.0 - th / math.pi) ** K
    frac = float(np.mean(ids[0] == ids[1]))
    assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / L)


# ------------------------------------------------------------------------------------------
# Theorem 1: E[S^(q)] = sum_i p_i^K
# ------------------------------------------------------------------------------------------
def test_theorem1_unbiased():
    rng = np.random.default_rng(5)
    d, K, L = 3, 2, 100_000
    D = rng.standard_normal((6, d)).astype(np.float32)
    q = rng.standard_normal((1, d)).astype(np.float32)
    det = oracle.Detector(d, K, L, seed=77)
    det.insert(D)
    scores, sums, _ = det.score(q, 1.0)
    Dd, qd = D.astype(np.float64), q[0].astype(np.float64)
    cos = Dd @ qd / (np.linalg.norm(Dd, axis=1) * np.linalg.norm(qd))
    p = 1.0 - np.arccos(np.clip(cos, -1, 1)) / math.pi
    S = float(np.sum(p**K))
    # Var of one array's count <= E[A^2] <= n * S; the estimator averages L independent arrays
    se = math.sqrt(len(D) * S / L)
    assert abs(scores[0] - S) < 5 * se


# ------------------------------------------------------------------------------------------
# Invariants and library-routine cross-checks
# ------------------------------------------------------------------------------------------
def test_hash_matches_float64_matmul_signs():
    rng = np.random.default_rng(11)
    n, d, K, L = 300, 37, 7, 9
    X = rng.standard_normal((n, d)).astype(np.float32)
    W = workloads.gaussian_w(d, K, L, 3)
    ids = oracle.hash_ids(X, W, K, L)
    S = X.astype(np.float64) @ W.astype(np.float64)
    margin = np.abs(S) > 1e-9 * (np.abs(X.astype(np.float64)) @ np.abs(W.astype(np.float64)))
    bits = (S > 0).astype(np.uint32).reshape(n, L, K)
    ref = (bits << np.arange(K, dtype=np.uint32)).sum(axis=2)
    got_bits = (ids[:, :, None] >> np.arange(K, dtype=np.uint32)) & 1
    ok = margin.reshape(n, L, K)
    assert np.all(got_bits[ok] == bits[ok])
    assert ok.mean() > 0.999
    assert np.array_equal(ids[ok.all(axis=2)], ref[ok.all(axis=2)])


def test_counts_match_bincount_and_sum_to_n():
    w = workloads.small(seed=3, n=3000)
    det = oracle.Detector(w["d"], w["K"], w["L"], seed=5)
    ids = det.insert(w["X"])
    for j in range(w["L"]):
        assert np.array_equal(det.counts[j], np.bincount(ids[:, j], minlength=1 << w["K"]))
        assert int(det.counts[j].sum()) == 3000
    ids2 = det.insert(w["X"][:777])
    for j in range(w["L"]):
        assert int(det.counts[j].sum()) == 3777


def test_hand_example_delete_eq12():
    """Deletion (§3.4.1) on the worked example: counts, Q, mu_ins, and Eq. 12 point by point,
    all against the values worked out by hand."""
    g, W, X = _hand()
    gd = _load("hand_example_delete.json")
    det = oracle.Detector(g["d"], g["K"], g["L"], W=W)
    det.insert(X)
    counts = det.counts.copy()
    ids = oracle.hash_ids(X[gd["delete_order"]], W, g["K"], g["L"])
    mu, trace = oracle.mu_decremental(ids, counts, g["K"], n_before=4, mu_before=g["mu"])
    assert trace.tolist() == gd["mu_decremental_trace"]
    for step, i in enumerate(gd["delete_order"]):
        det.delete(X[i:i + 1])
        assert det.counts.tolist() == gd["counts_after"][step]
        st = det.stats()
        assert st["Q"] == gd["Q_after"][step]
        assert st["mu_ins"] == gd["mu_ins_after"][step]
        assert st["n_ins"] == 3 - step
    assert counts.tolist() == gd["counts_after"][-1]


def test_delete_rejects_points_not_inserted():
    g, W, X = _hand()
    gd = _load("hand_example_delete.json")
    det = oracle.Detector(g["d"], g["K"], g["L"], W=W)
    det.insert(X)
    before = det.counts.copy()
    x = np.array([gd["not_inserted_point"]], dtype=np.float32)
    assert oracle.hash_ids(x, W, g["K"], g["L"]).tolist() == [gd["not_inserted_ids"]]
    with pytest.raises(ValueError):
        det.delete(np.concatenate([X[:1], x]))  # a valid point first: nothing may change
    assert np.array_equal(det.counts, before) and det.n_ins == 4


def test_delete_inverts_insert_and_eq12_matches_closed_form():
    """Inserting A then B and deleting B leaves exactly the arrays of A alone; Eq. 12 point
    by point agrees with Q/(nL) at every stage of the deletion."""
    w = workloads.small(seed=11, n=3000)
    A, Bset = w["X"][:1800], w["X"][1800:]
    det = oracle.Detector(w["d"], w["K"], w["L"], seed=3)
    only_a = oracle.Detector(w["d"], w["K"], w["L"], seed=3)
    det.insert(A)
    only_a.insert(A)
    det.insert(Bset)
    mu_full = det.stats()["mu_ins"]
    counts = det.counts.copy()
    ids_b = det.hash(Bset)
    mu_dec, trace = oracle.mu_decremental(ids_b, counts, w["K"], n_before=3000, mu_before=mu_full)
    det.delete(Bset)
    assert np.array_equal(det.counts, only_a.counts) and np.array_equal(counts, det.counts)
    assert det.stats()["Q"] == only_a.stats()["Q"]
    assert mu_dec == pytest.approx(only_a.stats()["mu_ins"], rel=1e-12)
    # a midpoint of the deletion: the first 600 of B removed
    mid = oracle.Detector(w["d"], w["K"], w["L"], seed=3)
    mid.insert(A)
    mid.insert(Bset[600:])
    assert trace[599] == pytest.approx(mid.stats()["mu_ins"], rel=1e-12)


def test_mu_identity_three_ways():
    """Eq. 11 point by point == Q/(nL) == mean score of the inserted set at final counts."""
    w = workloads.small(seed=4, n=2000)
    det = oracle.Detector(w["d"], w["K"], w["L"], seed=6)
    ids = det.insert(w["X"])
    counts = np.zeros_like(det.counts)
    mu_inc, _ = oracle.mu_incremental(ids, counts, w["K"])
    assert np.array_equal(counts, det.counts)
    Q = det.q()
    assert Q == int(np.sum(det.counts.astype(np.int64) ** 2))
    mu_q = det.stats()["mu_ins"]
    sums = oracle.gather(ids, det.counts, w["K"])
    mu_scores = float(np.mean(sums.astype(np.float64) / w["L"]))
    assert mu_q == pytest.approx(mu_scores, rel=1e-14)
    assert mu_inc == pytest.approx(mu_q, rel=1e-12)
    assert int(sums.sum()) == Q  # sum over points of their counts = sum over buckets of count^2


def test_power_of_two_scaling_invariance():
    rng = np.random.default_rng(12)
    X = rng.standard_normal((50, 20)).astype(np.float32)
    W = workloads.gaussian_w(20, 6, 5, 1)
    base = oracle.hash_ids(X, W, 6, 5)
    for k in (-7, -1, 3, 20):
        assert np.array_equal(oracle.hash_ids(X * np.float32(2.0**k), W, 6, 5), base)


def test_negation_flips_nonzero_bits():
    rng = np.random.default_rng(13)
    X = rng.standard_normal((40, 8)).astype(np.float32)
    X[0] = 0.0
    X[1, :] = [1, 1, 1, 0, 0, 0, 0, 0]
    W = workloads.gaussian_w(8, 5, 6, 2)
    W[:, 0] = [1, -1, 0, 0, 0, 0, 0, 0]  # x[1] projects to exactly 0 on column 0
    K, L = 5, 6
    s = oracle.project(X, W)
    a = oracle.hash_ids(X, W, K, L)
    b = oracle.hash_ids(-X, W, K, L)
    ba = ((a[:, :, None] >> np.arange(K, dtype=np.uint32)) & 1).reshape(40, K * L)
    bb = ((b[:, :, None] >> np.arange(K, dtype=np.uint32)) & 1).reshape(40, K * L)
    nz = s != 0
    assert np.all(ba[nz] + bb[nz] == 1)
    assert np.all(ba[~nz] == 0) and np.all(bb[~nz] == 0)
    assert np.all(a[0] == 0)  # the zero vector goes to bucket 0 of every array
    assert ba[1, 0] == 0 and bb[1, 0] == 0


def test_stats_match_numpy_mean_and_population_std():
    w = workloads.small(seed=8, n=5000)
    det = oracle.Detector(w["d"], w["K"], w["L"], seed=9)
    scores, sums, flags = det.insert_score(w["X"], 1.0)
    st = det.stats(1.0)
    assert st["mu"] == pytest.approx(float(np.mean(scores)), rel=1e-13)
    assert st["sigma"] == pytest.approx(float(np.std(scores)), rel=1e-12)
    assert st["threshold"] == pytest.approx(st["mu"] - st["sigma"], rel=1e-15)
    assert np.array_equal(flags.astype(bool), scores < st["threshold"])
    # with "insert everything, then score everything", mu equals the inserted-set mean
    assert st["mu"] == pytest.approx(st["mu_ins"], rel=1e-14)


def test_running_stats_span_batches():
    w = workloads.small(seed=10, n=3000)
    det = oracle.Detector(w["d"], w["K"], w["L"], seed=11)
    det.insert(w["X"])
    s1, _, _ = det.score(w["X"][:1000], 2.0)
    s2, _, f2 = det.score(w["X"][1000:], 2.0)
    allsc = np.concatenate([s1, s2])
    st = det.stats(2.0)
    assert st["n_scored"] == 3000
    assert st["mu"] == pytest.approx(float(allsc.mean()), rel=1e-13)
    assert st["sigma"] == pytest.approx(float(allsc.std()), rel=1e-12)
    assert np.array_equal(f2.astype(bool), s2 < st["threshold"])


def test_score_does_not_insert_and_insert_score_order():
    w = workloads.small(seed=12, n=1000)
    a = oracle.Detector(w["d"], w["K"], w["L"], seed=13)
    a.score(w["X"], 1.0)
    assert int(a.counts.sum()) == 0 and a.n_ins == 0
    b = oracle.Detector(w["d"], w["K"], w["L"], seed=13)
    c = oracle.Detector(w["d"], w["K"], w["L"], seed=13)
    sb, ub, fb = b.insert_score(w["X"], 1.0)
    c.insert(w["X"])
    sc, uc, fc = c.score(w["X"], 1.0)
    assert np.array_equal(ub, uc) and np.array_equal(fb, fc)


def test_insert_order_independent():
    w = workloads.small(seed=14, n=1500)
    a = oracle.Detector(w["d"], w["K"], w["L"], seed=15)
    b = oracle.Detector(w["d"], w["K"], w["L"], seed=15)
    a.insert(w["X"])
    b.insert(w["X"][::-1].copy())
    assert np.array_equal(a.counts, b.counts)


def test_empty_batch_and_overflow():
    det = oracle.Detector(4, 3, 2, seed=1)
    ids = det.insert(np.zeros((0, 4), dtype=np.float32))
    assert ids.shape == (0, 2) and int(det.counts.sum()) == 0
    det.counts[0, 0] = np.uint32(2**32 - 1)
    before = det.counts.copy()
    with pytest.raises(OverflowError):
        det.insert(np.zeros((1, 4), dtype=np.float32))  # the zero vector hits bucket 0
    assert np.array_equal(det.counts, before)


def test_bf16_inputs_hash_like_their_float32_values():
    rng = np.random.default_rng(21)
    Xf = rng.standard_normal((64, 48)).astype(np.float32)
    Xb = workloads.to_bf16_bits(Xf)
    W = workloads.gaussian_w(48, 8, 4, 5)
    a = oracle.hash_ids(Xb, W, 8, 4)
    b = oracle.hash_ids(workloads.bf16_bits_to_f32(Xb), W, 8, 4)
    assert np.array_equal(a, b)


def test_nonfinite_inputs_follow_binary64_semantics():
    # NaN anywhere makes every projection NaN, and NaN > 0 is false: bucket 0 everywhere.
    W = workloads.gaussian_w(5, 4, 3, 8)
    X = np.zeros((2, 5), dtype=np.float32)
    X[0, 2] = np.nan
    X[1, 0] = np.inf
    ids = oracle.hash_ids(X, W, 4, 3)
    assert np.all(ids[0] == 0)
    bits = ((ids[1][:, None] >> np.arange(4, dtype=np.uint32)) & 1).ravel()
    expect = (W[0] > 0).astype(np.uint32)  # inf * w has the sign of w (w != 0)
    assert np.array_equal(bits, expect)


def test_window_hand_example():
    """Sliding window of two points over the hand example, one point at a time: counts, Q and
    mu_ins after each insert equal the hand-counted values (tests/golden/hand_example_window.json)."""
    g = _load("hand_example.json")
    gw = _load("hand_example_window.json")
    W = np.array(g["W_columns"], dtype=np.float32).T.copy()
    X = np.array(g["X"], dtype=np.float32)
    det = oracle.WindowDetector(3, 2, 2, window=gw["window"], W=W)
    for i in range(4):
        det.insert(X[i:i + 1])
        st = det.stats()
        assert det.counts.tolist() == gw["counts_after"][i]
        assert st["n_ins"] == gw["held_after"][i] and st["Q"] == gw["Q_after"][i]
        assert st["mu_ins"] == gw["mu_ins_after"][i]


def test_window_equals_plain_detector_on_the_last_points():
    """After any sequence of batches, a window detector's arrays equal those of a plain
    detector fed only the last `window` points (a path through insertion alone)."""
    rng = np.random.default_rng(8)
    d, K, L, win = 12, 5, 6, 1000
    W = rng.standard_normal((d, K * L)).astype(np.float32)
    det = oracle.WindowDetector(d, K, L, window=win, W=W)
    seen = []
    for n in (300, 700, 1, 999, 1000, 250, 5):
        X = rng.standard_normal((n, d)).astype(np.float32)
        det.insert(X)
        seen.append(X)
        last = np.concatenate(seen)[-win:]
        plain = oracle.Detector(d, K, L, W=W)
        plain.insert(last)
        assert np.array_equal(det.counts, plain.counts) and det.n_ins == last.shape[0]
    with pytest.raises(ValueError):
        det.insert(rng.standard_normal((win + 1, d)).astype(np.float32))


# ------------------------------------------------------------------------------------------
# Integer-only projection (ACE_W_COUNTER)
# ------------------------------------------------------------------------------------------
def test_counter_projection_from_published_draws():
    """Entries (popcount(draw_f) - 32) / 4 for the published SplitMix64 outputs
    (tests/golden/splitmix64.json: seed 0 draw 0, seed 1234567 draws 0 to 2), the ones counted
    by Python's own integer routine."""
    vec = {(v["seed"], v["t"]): v["out"] for v in _load("splitmix64.json")["vectors"]}
    W = oracle.projection_from_seed(1, 3, 1, seed=1234567, counter=True).ravel()
    for t in range(3):
        assert W[t] == (bin(vec[(1234567, t)]).count("1") - 32) / 4, t
    assert oracle.projection_from_seed(1, 1, 1, seed=0, counter=True).ravel()[0] == (bin(vec[(0, 0)]).count("1") - 32) / 4
    # flat index f = i K L + c: entry (i, c) is draw i K L + c
    W2 = oracle.projection_from_seed(3, 2, 2, seed=1234567, counter=True)
    assert W2[0, 1] == W.ravel()[1] and W2[0, 2] == W.ravel()[2]


def test_counter_projection_is_binomial():
    """4 w + 32 follows Binomial(64, 1/2) over a million entries (chi-square over the 65 values,
    sparse tails merged), so w has mean 0 and variance 1; every entry is a bfloat16 value."""
    W = oracle.projection_from_seed(64, 16, 1024, seed=777, counter=True).astype(np.float64).ravel()
    k = W * 4 + 32
    assert np.array_equal(k, np.rint(k)) and k.min() >= 0 and k.max() <= 64
    assert np.array_equal(workloads.bf16_bits_to_f32(workloads.to_bf16_bits(W.astype(np.float32))), W.astype(np.float32))
    obs = np.bincount(k.astype(int), minlength=65).astype(np.float64)
    pmf = np.array([math.comb(64, i) for i in range(65)], dtype=np.float64) / 2.0**64
    exp = pmf * k.size
    lo, hi = 20, 44  # merge the tails (expected counts below ~100 outside)
    o = np.concatenate([[obs[:lo].sum()], obs[lo:hi + 1], [obs[hi + 1:].sum()]])
    e = np.concatenate([[exp[:lo].sum()], exp[lo:hi + 1], [exp[hi + 1:].sum()]])
    chi2 = float(((o - e) ** 2 / e).sum())
    scipy_stats = pytest.importorskip("scipy.stats")
    assert scipy_stats.chi2.sf(chi2, len(o) - 1) > 1e-4, chi2
    se = 1.0 / math.sqrt(W.size)
    assert abs(W.mean()) < 5 * se and abs(W.var() - 1.0) < 5 * math.sqrt(2.0) * se


@pytest.mark.parametrize("theta", [math.pi / 6, math.pi / 2, 5 * math.pi / 6])
def test_counter_projection_collision_probability(theta):
    """SRP with the integer-only W: two points at angle theta in d = 16 (random directions)
    get the same bit on a fraction 1 - theta/pi of 2^17 columns, within sampling error and a
    0.005 allowance (Binomial(64, 1/2) entries are nearly, not exactly, rotation-invariant)."""
    d, M = 16, 1 << 17
    rng = np.random.default_rng(int(theta * 1000))
    x = rng.standard_normal(d)
    x /= np.linalg.norm(x)
    z = rng.standard_normal(d)
    z -= (z @ x) * x
    z /= np.linalg.norm(z)
    X = np.stack([x, math.cos(theta) * x + math.sin(theta) * z]).astype(np.float32)
    W = oracle.projection_from_seed(d, 1, M, seed=4242, counter=True)
    ids = oracle.hash_ids(X, W, 1, M)
    xd, yd = X.astype(np.float64)
    th = math.acos(float(xd @ yd) / (np.linalg.norm(xd) * np.linalg.norm(yd)))
    p = 1.0 - th / math.pi
    frac = float(np.mean(ids[0] == ids[1]))
    assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / M) + 0.005, (frac, p)



# ------------------------------------------------------------------------------------------
# Eq. 3 computed exactly (the estimator-accuracy workload)
# ------------------------------------------------------------------------------------------
def test_exact_score_closed_forms():
    """S(q, D) = sum_i p_i^K with p = 1 - theta/pi: a copy of q gives 1 (any scale), its
    negation 0, an orthogonal point 2^-K, a point at angle theta (1 - theta/pi)^K, a zero point
    2^-K (p = 1/2), and two zero vectors 1; the sum over a set is the sum of those."""
    K = 7
    q = np.array([[1.0, 2.0, -2.0]], dtype=np.float32)  # ||q|| = 3
    u = q[0] / 3.0
    v = np.array([2.0, 1.0, 2.0], dtype=np.float32) / 3.0  # u . v = 0
    th = 0.7
    at = (math.cos(th) * u + math.sin(th) * v).astype(np.float32)
    Dset = np.stack([5 * q[0], -q[0], v, at, np.zeros(3, np.float32)]).astype(np.float32)
    per = [1.0, 0.0, 2.0**-K, None, 2.0**-K]
    xd = at.astype(np.float64)
    thd = math.acos(float(xd @ u.astype(np.float64)) / (np.linalg.norm(xd) * np.linalg.norm(u.astype(np.float64))))
    per[3] = (1 - thd / math.pi) ** K
    for i, want in enumerate(per):
        got = float(oracle.exact_score(q, Dset[i:i + 1], K)[0])
        assert math.isclose(got, want, rel_tol=1e-12, abs_tol=1e-15), (i, got, want)
    assert math.isclose(float(oracle.exact_score(q, Dset, K)[0]), sum(per), rel_tol=1e-12)
    z = np.zeros((1, 3), dtype=np.float32)
    assert float(oracle.exact_score(z, z, K)[0]) == 1.0
    # RSE over the whole set is S itself
    assert math.isclose(float(oracle.rse(q, Dset, K, np.arange(5))[0]), sum(per), rel_tol=1e-12)


def test_theorem1_with_exact_score():
    """The oracle detector's score averages, over L arrays, to S(q, D) of Eq. 3 (Theorem 1):
    within five standard errors at L = 60,000 for three queries on a small clustered set."""
    rng = np.random.default_rng(9)
    d, K, L = 4, 3, 60_000
    D = (rng.standard_normal((12, d)) + np.array([2.0, 0, 0, 0])).astype(np.float32)
    Q = rng.standard_normal((3, d)).astype(np.float32)
    det = oracle.Detector(d, K, L, seed=5)
    det.insert(D)
    scores, _, _ = det.score(Q, 1.0)
    S = oracle.exact_score(Q, D, K)
    for j in range(3):
        se = math.sqrt(len(D) * S[j] / L)
        assert abs(scores[j] - S[j]) < 5 * se + 1e-12, (j, scores[j], S[j])


# ------------------------------------------------------------------------------------------
# Structured projection (ACE_W_HADAMARD)
# ------------------------------------------------------------------------------------------
def test_hadamard_projection_definition():
    """W[i][c] = D_b[i] H[j][i] (c = b dp + j): scipy's Sylvester-Hadamard matrix and the sign
    of each SplitMix64 draw (whose values the published vectors pin) give the same matrix, for
    a d that needs padding (41 -> 64) and several blocks (K L = 750)."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    d, K, L, seed = 41, 15, 50, 99
    W = oracle.projection_from_seed(d, K, L, seed, hadamard=True)
    dp, KL = 64, K * L
    H = scipy_linalg.hadamard(dp)
    ref = np.zeros((d, KL), dtype=np.float32)
    for c in range(KL):
        b, j = divmod(c, dp)
        for i in range(d):
            ref[i, c] = (-1.0 if oracle.splitmix64_draw(seed, b * dp + i) & 1 else 1.0) * H[j, i]
    assert np.array_equal(W, ref)


def test_hadamard_blocks_are_orthogonal():
    """With d = dp (no padding) the dp columns of one block are orthogonal: W_b^T W_b = dp I."""
    d = 64
    W = oracle.projection_from_seed(d, 16, 12, 7, hadamard=True).astype(np.int64)
    for b in range(W.shape[1] // d):
        Wb = W[:, b * d:(b + 1) * d]
        assert np.array_equal(Wb.T @ Wb, d * np.eye(d, dtype=np.int64)), b


@pytest.mark.parametrize("theta", [math.pi / 6, math.pi / 2, 5 * math.pi / 6])
def test_hadamard_collision_probability(theta):
    """Each column is a random +-1 vector (a Hadamard row times random signs), so one SRP bit
    of two points at angle theta agrees with probability close to 1 - theta/pi: within 0.01
    over 2^17 columns (4,096 blocks with independent signs) in d = 16."""
    d, M = 16, 1 << 17
    rng = np.random.default_rng(int(theta * 1000))
    x = rng.standard_normal(d)
    x /= np.linalg.norm(x)
    z = rng.standard_normal(d)
    z -= (z @ x) * x
    z /= np.linalg.norm(z)
    X = np.stack([x, math.cos(theta) * x + math.sin(theta) * z]).astype(np.float32)
    W = oracle.projection_from_seed(d, 1, M, seed=4242, hadamard=True)
    ids = oracle.hash_ids(X, W, 1, M)
    xd, yd = X.astype(np.float64)
    th = math.acos(float(xd @ yd) / (np.linalg.norm(xd) * np.linalg.norm(yd)))
    assert abs(float(np.mean(ids[0] == ids[1])) - (1.0 - th / math.pi)) < 0.01
