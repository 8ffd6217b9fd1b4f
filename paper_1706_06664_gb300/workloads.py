"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no step of the ACE method: it only draws input batches (points X and,
for tests, explicit projection matrices) from numpy's PCG64 generator.  Both the CUDA
library's tests/benchmark and the CPU oracle are fed from here; neither side's arithmetic
lives here.

Recipes (sizes are the defaults; tests pass smaller n):

* ``small``    — n=10,000 binary32 points, d=32: 99% iid N(0,1); 1% anomalies N(4,1) in
                 3 seed-chosen dimensions (the same 3 for all) and N(0,1) elsewhere.
                 K=10, L=20, alpha=1.  A smoke-sized Algorithm 1 run.
* ``kdd``      — stand-in for the KDD-Cup99 HTTP table (§5.1, Table 1: 596,853 x 36; the
                 dataset itself is not available): n=500,000 binary32 rows, d=41, a mixture
                 of 23 Gaussian clusters (weights proportional to log-uniform[1,1000] draws;
                 per-feature scale log-uniform[1e-3,1e3]; means U[0,1]*scale; within-cluster
                 sd 0.05*scale), min-max normalised to [0,1] in binary64, then 1% anomalies
                 uniform in the unit box; rows shuffled; rounded to binary32.  K=15, L=50
                 (Table 2).
* ``highdim``  — n=1,000,000 bfloat16 points, d=1024: 64 centres uniform on the unit
                 sphere, x = normalize(c + (0.1/sqrt(d)) g) with g ~ N(0,I), plus 0.5%
                 anomalies normalize(g); rounded to bfloat16 (round to nearest even).
                 K=16, L=64.
* ``batched``  — many independent detectors: d log-uniform in [16,512], n log-uniform in
                 [100,100000], 8 clusters N(m_c, I) with m_c ~ N(0,4I), 1% anomalies shifted
                 by +4 in 3 dimensions; K=12, L=32.
* ``stream_chunk`` — a drifting stream for serving: d=128 binary32, 16 means that move
                 linearly from m0_c to m1_c (both ~ N(0,4I)) over the stream's length, points
                 N(m_c(t), I); 0.1% anomalies in bursts of 100 consecutive points, shifted by
                 +6 in 3 seed-chosen dimensions.  Chunks are drawn from (seed, start), so any
                 window of the stream can be generated on its own.  K=15, L=50, 64 detectors;
                 request sizes log-uniform in [1, 8192] (``request_sizes``).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["small", "kdd", "highdim", "highdim_device", "batched_specs", "batched_points", "stream_chunk", "request_sizes",
           "to_bf16_bits", "bf16_bits_to_f32", "gaussian_w"]


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed) & (2**63 - 1), int(stream)]))


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """binary32 -> bfloat16 bit patterns (uint16), round to nearest even (finite inputs)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (b.astype(np.uint32) << 16).view(np.float32)


def gaussian_w(d: int, K: int, L: int, seed: int) -> np.ndarray:
    """An explicit d x KL binary32 N(0,1) projection matrix (for create-with-projection)."""
    return _rng(seed, 7).standard_normal((d, K * L), dtype=np.float32)


def small(seed: int = 1, n: int = 10_000, d: int = 32):
    rng = _rng(seed, 1)
    X = rng.standard_normal((n, d), dtype=np.float32)
    n_anom = max(1, n // 100)
    dims = rng.choice(d, size=min(3, d), replace=False)
    idx = rng.choice(n, size=n_anom, replace=False)
    X[np.ix_(idx, dims)] += np.float32(4.0)
    labels = np.zeros(n, dtype=bool)
    labels[idx] = True
    return {"name": "small", "X": X, "d": d, "K": 10, "L": 20, "alpha": 1.0, "labels": labels,
            "dtype": "f32"}


def kdd(seed: int = 2, n: int = 500_000, d: int = 41, clusters: int = 23):
    rng = _rng(seed, 2)
    n_anom = n // 100
    n_in = n - n_anom
    w = np.exp(rng.uniform(0.0, math.log(1000.0), size=clusters))
    w /= w.sum()
    sizes = rng.multinomial(n_in, w)
    scale = np.exp(rng.uniform(math.log(1e-3), math.log(1e3), size=d))
    means = rng.uniform(0.0, 1.0, size=(clusters, d)) * scale
    parts = []
    for c in range(clusters):
        if sizes[c]:
            parts.append(means[c] + 0.05 * scale * rng.standard_normal((sizes[c], d)))
    Xin = np.concatenate(parts, axis=0)
    lo, hi = Xin.min(axis=0), Xin.max(axis=0)
    span = np.where(hi > lo, hi - lo, 1.0)
    Xin = (Xin - lo) / span
    Xan = rng.uniform(0.0, 1.0, size=(n_anom, d))
    X = np.concatenate([Xin, Xan], axis=0)
    labels = np.zeros(n, dtype=bool)
    labels[n_in:] = True
    perm = rng.permutation(n)
    return {"name": "kdd", "X": np.ascontiguousarray(X[perm], dtype=np.float32), "d": d, "K": 15,
            "L": 50, "alpha": 1.0, "labels": labels[perm], "dtype": "f32"}


def highdim(seed: int = 3, n: int = 1_000_000, d: int = 1024, clusters: int = 64,
            chunk: int = 65536):
    rng = _rng(seed, 3)
    C = rng.standard_normal((clusters, d))
    C /= np.linalg.norm(C, axis=1, keepdims=True)
    n_anom = max(1, n * 5 // 1000)
    is_anom = np.zeros(n, dtype=bool)
    is_anom[rng.choice(n, size=n_anom, replace=False)] = True
    which = rng.integers(0, clusters, size=n)
    out = np.empty((n, d), dtype=np.uint16)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        g = rng.standard_normal((e - s, d))
        x = np.where(is_anom[s:e, None], g, C[which[s:e]] + (0.1 / math.sqrt(d)) * g)
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        out[s:e] = to_bf16_bits(x.astype(np.float32))
    return {"name": "highdim", "X": out, "d": d, "K": 16, "L": 64, "alpha": 1.0,
            "labels": is_anom, "dtype": "bf16"}


def highdim_device(seed: int = 3, n: int = 1_000_000, d: int = 1024, clusters: int = 64):
    """The ``highdim`` recipe drawn on the current CUDA device with torch's generator (for the
    full-size batch, whose host draw takes minutes): 64 centres uniform on the unit sphere,
    x = normalize(c + (0.1/sqrt(d)) g), 0.5% anomalies normalize(g), rounded to bfloat16 (round
    to nearest even).  Returns (X as an int16 tensor of bfloat16 bits on the device, anomaly
    mask as a numpy array).  Same recipe as ``highdim``; a different random stream."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(int(seed) & (2**63 - 1))
    C = torch.randn(clusters, d, device="cuda", generator=g, dtype=torch.float64)
    C /= C.norm(dim=1, keepdim=True)
    n_anom = max(1, n * 5 // 1000)
    perm = torch.randperm(n, device="cuda", generator=g)
    is_anom = torch.zeros(n, dtype=torch.bool, device="cuda")
    is_anom[perm[:n_anom]] = True
    which = torch.randint(0, clusters, (n,), device="cuda", generator=g)
    out = torch.empty((n, d), dtype=torch.bfloat16, device="cuda")
    chunk = 1 << 16
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        gg = torch.randn(e - s, d, device="cuda", generator=g, dtype=torch.float64)
        x = torch.where(is_anom[s:e, None], gg, C[which[s:e]] + (0.1 / math.sqrt(d)) * gg)
        x /= x.norm(dim=1, keepdim=True)
        out[s:e] = x.to(torch.float32).to(torch.bfloat16)
    return out.view(torch.int16), is_anom.cpu().numpy()


def batched_specs(seed: int = 4, n_det: int = 2048, d_range=(16, 512), n_range=(100, 100_000)):
    """(d_i, n_i, seed_i) for each independent detector."""
    rng = _rng(seed, 4)
    d = np.rint(np.exp(rng.uniform(math.log(d_range[0]), math.log(d_range[1]), size=n_det))).astype(int)
    n = np.rint(np.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]), size=n_det))).astype(int)
    seeds = rng.integers(1, 2**62, size=n_det)
    return [(int(d[i]), int(n[i]), int(seeds[i])) for i in range(n_det)]


def batched_points(d: int, n: int, seed: int, clusters: int = 8):
    rng = _rng(seed, 5)
    means = 2.0 * rng.standard_normal((clusters, d))
    which = rng.integers(0, clusters, size=n)
    X = means[which] + rng.standard_normal((n, d))
    n_anom = max(1, n // 100)
    idx = rng.choice(n, size=n_anom, replace=False)
    dims = rng.choice(d, size=min(3, d), replace=False)
    X[np.ix_(idx, dims)] += 4.0
    return np.ascontiguousarray(X, dtype=np.float32)


def stream_chunk(seed: int, start: int, n: int, total: int = 100_000_000, d: int = 128, means: int = 16):
    """Points [start, start + n) of the drifting stream (see the module notes)."""
    base = _rng(seed, 0)
    m0 = base.normal(0.0, 2.0, size=(means, d))
    m1 = base.normal(0.0, 2.0, size=(means, d))
    dims = base.choice(d, size=3, replace=False)
    r = _rng(seed, 1 + int(start))
    pos = np.arange(start, start + n, dtype=np.float64)
    t = (pos / float(total))[:, None]
    c = r.integers(0, means, size=n)
    X = (1.0 - t) * m0[c] + t * m1[c] + r.normal(size=(n, d))
    # one burst of 100 anomalous points in every 100,000 (0.1%), at a seed-chosen offset
    off = int(base.integers(0, 100_000 - 100))
    burst = ((pos.astype(np.int64) % 100_000) >= off) & ((pos.astype(np.int64) % 100_000) < off + 100)
    X[np.ix_(burst, dims)] += 6.0
    return np.ascontiguousarray(X, dtype=np.float32)


def request_sizes(seed: int, count: int, lo: int = 1, hi: int = 8192) -> np.ndarray:
    """Request sizes log-uniform in [lo, hi]."""
    r = _rng(seed, 7)
    return np.exp(r.uniform(math.log(lo), math.log(hi), size=count)).round().astype(np.int64).clip(lo, hi)
