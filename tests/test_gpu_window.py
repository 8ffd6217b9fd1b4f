"""Sliding-window detector on the device (ace_window_enable; §3.4.1 deletion of the oldest
points, Eq. 12) against the oracle's window detector: counts, scores, flags and statistics
bit for bit over a stream of batches that wrap the ring, on every engine."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1706_06664_gb300 import ace, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(X):
    if X.dtype == np.uint16:
        return torch.from_numpy(X.view(np.int16)).cuda()
    return torch.from_numpy(X).cuda()


@pytest.mark.parametrize("engine", ["fp32", "bf16", "streaming", "host"])
def test_window_stream_matches_oracle(engine):
    if engine == "streaming":
        d, K, L, win = 128, 16, 8, 5000
        stream = [workloads.to_bf16_bits(workloads.stream_chunk(7, s, n, d=d)) for s, n in
                  ((0, 3000), (3000, 2500), (5500, 1), (5501, 5000), (10501, 1234), (11735, 4000))]
        precision = "bf16"
    else:
        d, K, L, win = 41, 15, 50, 20000
        stream = [workloads.kdd(seed=40 + i, n=n)["X"] for i, n in enumerate((12000, 9000, 1, 20000, 777, 15000))]
        precision = "fp32" if engine == "fp32" else ("bf16" if engine == "bf16" else "auto")
    det = ace.Detector(d, K, L, seed=3, precision=precision)
    det.window(win)
    ref = oracle.WindowDetector(d, K, L, window=win, W=det.projection())
    for i, X in enumerate(stream):
        rs, ru, rf = ref.insert_score(X, 1.0)
        if engine == "host":
            n = X.shape[0]
            sc, su, fl = np.empty(n), np.empty(n, dtype=np.uint32), np.empty(n, dtype=np.uint8)
            det.insert_score_host(X, 1.0, sc, su, fl)
        else:
            sc, su, fl = det.insert_score(_dev(X), 1.0)
            torch.cuda.synchronize()
            sc, su, fl = sc.cpu().numpy(), ace.u32(su), fl.cpu().numpy()
        assert np.array_equal(su, ru) and np.array_equal(sc, rs) and np.array_equal(fl, rf), i
        assert np.array_equal(det.counts(), ref.counts), i
        s, r = det.stats(), ref.stats()
        for k in ("n_ins", "Q", "mu_ins", "n_scored", "S1", "S2", "mu", "sigma"):
            assert s[k] == r[k], (i, k)
    if engine == "streaming":
        assert det.stats()["tc_products"] == 2
    # plain inserts follow the window too
    X = stream[0][:700]
    det.insert(_dev(X))
    ref.insert(X)
    assert np.array_equal(det.counts(), ref.counts) and det.stats()["n_ins"] == ref.n_ins


def test_window_hand_example_and_refusals():
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_example.json")))
    gw = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_example_window.json")))
    W = np.array(g["W_columns"], dtype=np.float32).T.copy()
    X = np.array(g["X"], dtype=np.float32)
    det = ace.Detector(3, 2, 2, W=W)
    det.window(gw["window"])
    for i in range(4):
        det.insert(_dev(X[i:i + 1]))
        st = det.stats()
        assert det.counts().tolist() == gw["counts_after"][i]
        assert st["n_ins"] == gw["held_after"][i] and st["Q"] == gw["Q_after"][i] and st["mu_ins"] == gw["mu_ins_after"][i]
    for call in (lambda: det.insert(_dev(X[:3])), lambda: det.delete(_dev(X[:1])), lambda: det.save(),
                 lambda: det.window(5)):
        with pytest.raises(ace.AceError) as e:
            call()
        assert e.value.code == ace.ACE_ERR_ARG
    det.reset()
    det.window(3)  # allowed again once empty
    det.insert(_dev(X[:3]))
    assert det.stats()["n_ins"] == 3
