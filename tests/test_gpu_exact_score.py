"""The exact score family on the GPU (ace_exact_score, Eq. 3 with SRP's p) against the oracle's
binary64 definition, and the estimator-accuracy workload built on it.

Tolerance: both sides compute cos in binary64, in different summation orders; near cos = 1 a
difference of a few units in the last place moves the angle by up to sqrt(2 * 4 * 2^-53),
about 3e-8, so p^K by up to K * 1e-8 per pair: 1e-6 relative covers K <= 15 with margin."""
import math

import numpy as np
import pytest

import oracle
from paper_1706_06664_gb300 import ace, accuracy, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _close(got, want):
    got = got.cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-6 * np.abs(want) + 1e-12), np.max(np.abs(got - want) / (np.abs(want) + 1e-300))


@pytest.mark.parametrize("K", [1, 7, 15])
def test_exact_score_matches_oracle(K):
    w = workloads.kdd(seed=4, n=5000)
    X = w["X"]
    Q = np.concatenate([X[:40], np.zeros((1, X.shape[1]), np.float32), -X[:3]])  # copies, a zero row, negations
    D = X.copy()
    D[17] = 0.0
    _close(ace.exact_score(torch.from_numpy(Q).cuda(), torch.from_numpy(D).cuda(), K), oracle.exact_score(Q, D, K))


def test_exact_score_bf16_high_d_and_edges():
    h = workloads.highdim(seed=2, n=3000)
    X = h["X"]
    Q, D = X[:25], X[25:]
    Qd, Dd = torch.from_numpy(Q.view(np.int16)).cuda(), torch.from_numpy(D.view(np.int16)).cuda()
    _close(ace.exact_score(Qd, Dd, 16), oracle.exact_score(Q, D, 16))
    # an empty dataset scores 0; ragged sizes (not a multiple of the 256-point block)
    assert not ace.exact_score(Qd, Dd[:0], 16).cpu().numpy().any()
    _close(ace.exact_score(Qd, Dd[:257], 16), oracle.exact_score(Q, D[:257], 16))
    with pytest.raises(ace.AceError) as e:
        ace.exact_score(Qd, Dd, 0)
    assert e.value.code == ace.ACE_ERR_ARG


def test_estimator_accuracy_workload():
    """Theorem 1 and Theorem 2 on the GPU: ACE's score and RSE are unbiased for S(q, D) (their
    mean error over 30 queries is within a few standard errors of 0), and ACE's scores are the
    oracle's for the same detector."""
    w = workloads.kdd(seed=6, n=4000)
    D = torch.from_numpy(w["X"]).cuda()
    Q = torch.from_numpy(w["X"][:30]).cuda()
    K = 6
    res = accuracy.estimator_mse(D, Q, K, Ls=[50, 200], seed=3, rse_draws=10)
    S = res["S"]
    assert np.all(S > 0)
    for L, r in res["L"].items():
        assert math.isfinite(r["ace_mse"]) and math.isfinite(r["rse_mse"])
        assert abs(r["ace_bias"]) <= 5 * math.sqrt(r["ace_mse"] / len(S)) + 1e-9, (L, r)
        assert abs(r["rse_bias"]) <= 5 * math.sqrt(r["rse_mse"] / len(S) / 10) + 1e-9, (L, r)
    # ACE's estimate is the detector's score: the same as the oracle's detector with that W
    det = ace.Detector(w["d"], K, 50, seed=3 * 7919 + 50)
    det.insert(D)
    sc, _, _ = det.score(Q, 1.0)
    ref = oracle.Detector(w["d"], K, 50, W=det.projection())
    ref.insert(w["X"])
    rs, _, _ = ref.score(w["X"][:30], 1.0)
    assert np.array_equal(sc.cpu().numpy(), rs)
