"""Estimator-accuracy workload (§4.2): how well ACE's score estimates the score family it is
built on, against random sampling.

For a dataset D and queries Q, the exact S(q, D) = sum_i p(q, x_i)^K (Eq. 3, SRP's p) comes
from ``ace.exact_score`` (binary64 on the GPU).  ACE's estimate is the mean count (1/L)
sum_j A_j[H_j(q)] of a detector holding D (Theorem 1: unbiased); the random sampling
estimator RSE (Eq. 10) is n/L times the sum of p^K over L points of D drawn uniformly without
replacement (Theorem 2: unbiased).  Both are compared at the same L by their mean square error
over the queries, for several L.  Everything runs through the library; nothing here computes a
step of the method itself.
"""
from __future__ import annotations

import numpy as np

from . import ace


def estimator_mse(D, Q, K: int, Ls, seed: int = 0, rse_draws: int = 20, precision: str = "auto") -> dict:
    """D (n x d) and Q (m x d): device tensors of one dtype (binary32, or bfloat16 as bf16 or
    int16 bit patterns).  Returns {"S": exact scores, "L": {L: {"ace_mse", "rse_mse",
    "ace_bias", "rse_bias"}}}; RSE's MSE averages rse_draws samples per L."""
    import torch
    n = D.shape[0]
    S = ace.exact_score(Q, D, K).cpu().numpy()
    rng = np.random.default_rng(seed)
    out = {"S": S, "L": {}}
    for L in Ls:
        det = ace.Detector(D.shape[1], K, int(L), seed=seed * 7919 + int(L), precision=precision)
        det.insert(D)
        sc, _, _ = det.score(Q, 1.0)
        est = sc.cpu().numpy()
        det.close()
        rse_err = []
        rse_mean = np.zeros_like(S)
        for _ in range(rse_draws):
            idx = torch.from_numpy(rng.choice(n, size=min(int(L), n), replace=False)).to(D.device)
            r = ace.exact_score(Q, D[idx], K).cpu().numpy() * (n / len(idx))
            rse_err.append((r - S) ** 2)
            rse_mean += r / rse_draws
        out["L"][int(L)] = {"ace_mse": float(np.mean((est - S) ** 2)), "rse_mse": float(np.mean(rse_err)),
                            "ace_bias": float(np.mean(est - S)), "rse_bias": float(np.mean(rse_mean - S))}
    return out
