"""The seeded input recipes (paper_1706_06664_gb300/workloads.py) have the shapes and
distributions their descriptions state: the anomaly fractions and shifts, the min-max
normalisation of the KDD-shaped table, unit-norm bfloat16 rows for the high-dimensional
config, log-uniform batched shapes and request sizes, a stream whose means drift, and
bfloat16 rounding to nearest even (checked against torch's own conversion).  The same seed
gives the same batch."""
import math

import numpy as np
import pytest

from paper_1706_06664_gb300 import workloads


def test_bf16_rounding_is_round_to_nearest_even():
    one = np.float32(1.0)
    half_ulp = np.float32(2.0 ** -8)  # half of bfloat16's 2^-7 spacing at 1
    x = np.array([one, one + half_ulp, one + 3 * half_ulp, one + half_ulp * np.float32(1.5), -3.0], np.float32)
    got = workloads.bf16_bits_to_f32(workloads.to_bf16_bits(x))
    # ties go to the even neighbour: 1 + 2^-8 -> 1, 1 + 3 2^-8 -> 1 + 2^-6; above a tie, up
    assert got.tolist() == [1.0, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -3.0]
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(0).standard_normal(100000).astype(np.float32) * np.float32(1e3)
    ref = torch.from_numpy(r).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(workloads.to_bf16_bits(r), ref)


def test_small_recipe():
    w = workloads.small(seed=1, n=20000)
    X, lab = w["X"], w["labels"]
    assert X.shape == (20000, 32) and X.dtype == np.float32 and (w["K"], w["L"]) == (10, 20)
    assert lab.sum() == 200
    shift = X[lab].mean(axis=0) - X[~lab].mean(axis=0)
    assert (shift > 3.5).sum() == 3 and (np.abs(shift) < 0.5).sum() == 29  # +4 in 3 dimensions
    assert np.array_equal(workloads.small(seed=1, n=20000)["X"], X)


def test_kdd_recipe():
    w = workloads.kdd(seed=2, n=20000)
    X, lab = w["X"], w["labels"]
    assert X.shape == (20000, 41) and X.dtype == np.float32 and (w["K"], w["L"]) == (15, 50)
    assert lab.sum() == 200
    assert X.min() >= 0.0 and X.max() <= 1.0
    inl = X[~lab]  # min-max normalised over the inliers: each feature spans exactly [0, 1]
    assert np.all(inl.min(axis=0) == 0.0) and np.all(inl.max(axis=0) == 1.0)
    # anomalies are uniform in the unit box; inliers sit in tight clusters
    assert abs(X[lab].mean() - 0.5) < 0.02 and X[lab].std() > 0.25
    assert np.array_equal(workloads.kdd(seed=2, n=20000)["X"], X)


def test_highdim_recipe():
    w = workloads.highdim(seed=3, n=4000, d=1024)
    B, lab = w["X"], w["labels"]
    assert B.shape == (4000, 1024) and B.dtype == np.uint16 and (w["K"], w["L"]) == (16, 64)
    assert lab.sum() == 20  # 0.5 %
    X = workloads.bf16_bits_to_f32(B).astype(np.float64)
    assert np.all(np.abs(np.linalg.norm(X, axis=1) - 1.0) < 4e-3)  # unit rows, bfloat16-rounded
    # inliers are close to one of 64 centres: pairs of inliers are either near-parallel (same
    # centre, cosine about 1/(1 + 0.01) = 0.99) or nearly orthogonal (different centres)
    G = X[~lab][:300] @ X[~lab][:300].T
    off = G[~np.eye(300, dtype=bool)]
    assert np.all((off > 0.97) | (np.abs(off) < 0.2))
    assert 0.005 < (off > 0.97).mean() < 0.05  # about 1/64 of the pairs share a centre
    A = X[lab] @ X[~lab][:300].T
    assert np.abs(A).max() < 0.2  # anomalies are uniform on the sphere


def test_batched_shapes_are_log_uniform():
    specs = workloads.batched_specs(seed=4, n_det=2048)
    d = np.array([s[0] for s in specs])
    n = np.array([s[1] for s in specs])
    assert d.min() >= 16 and d.max() <= 512 and n.min() >= 100 and n.max() <= 100000
    assert abs(math.log(np.median(d)) - 0.5 * math.log(16 * 512)) < 0.15
    assert abs(math.log(np.median(n)) - 0.5 * math.log(100 * 100000)) < 0.25
    assert len({s[2] for s in specs}) == 2048  # a seed of its own per detector
    assert specs == workloads.batched_specs(seed=4, n_det=2048)
    X = workloads.batched_points(37, 500, specs[0][2])
    assert X.shape == (500, 37) and X.dtype == np.float32


def test_stream_drifts_and_request_sizes():
    total = 1_000_000
    a = workloads.stream_chunk(31, 0, 20000, total=total)
    b = workloads.stream_chunk(31, 20000, 20000, total=total)
    z = workloads.stream_chunk(31, total - 20000, 20000, total=total)
    assert a.shape == (20000, 128) and a.dtype == np.float32
    assert np.array_equal(a, workloads.stream_chunk(31, 0, 20000, total=total))
    near = np.linalg.norm(a.mean(axis=0) - b.mean(axis=0))
    far = np.linalg.norm(a.mean(axis=0) - z.mean(axis=0))
    assert far > 10 * near  # the means move across the stream, not within a few windows
    s = workloads.request_sizes(5, 20000)
    assert s.min() >= 1 and s.max() <= 8192
    assert abs(math.log(np.median(s)) - 0.5 * math.log(8192)) < 0.1  # log-uniform in [1, 8192]
