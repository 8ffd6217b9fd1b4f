"""Graph replay (ace_set_graph) of repeated score / insert_score calls: with the same buffers and
new contents each call, every output equals a direct call's and the oracle's, on every engine;
the launch counters count the replayed kernels."""
import numpy as np
import pytest

import oracle
from paper_1706_06664_gb300 import ace, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("engine", ["fp32", "bf16", "streaming"])
def test_graph_replay_matches_direct_calls(engine):
    if engine == "streaming":
        d, K, L, n = 128, 16, 8, 3000
        batches = [workloads.to_bf16_bits(workloads.stream_chunk(5, i * n, n, d=d)) for i in range(6)]
        precision = "bf16"
    else:
        d, K, L, n = 32, 10, 20, 10_000
        batches = [workloads.small(seed=10 + i)["X"] for i in range(6)]
        precision = engine
    g = ace.Detector(d, K, L, seed=4, precision=precision)
    g.set_graph(True)
    plain = ace.Detector(d, K, L, seed=4, precision=precision)
    ref = oracle.Detector(d, K, L, W=g.projection())
    stream = torch.cuda.Stream()  # the legacy default stream cannot be captured
    torch.cuda.set_stream(stream)
    tx = torch.empty((n, d), dtype=torch.int16 if engine == "streaming" else torch.float32, device="cuda")
    sc = torch.empty(n, dtype=torch.float64, device="cuda")
    su = torch.empty(n, dtype=torch.int32, device="cuda")
    fl = torch.empty(n, dtype=torch.uint8, device="cuda")
    g.profile_read()
    for i, X in enumerate(batches):
        tx.copy_(torch.from_numpy(X.view(np.int16) if X.dtype == np.uint16 else X))
        if i % 3 == 2:  # a score call in between (its own graph key)
            g.score(tx, 1.0, scores=sc, sums=su, flags=fl)
            ps, pu, pf = plain.score(tx, 1.0)
            rs, ru, rf = ref.score(X, 1.0)
        else:
            g.insert_score(tx, 1.0, scores=sc, sums=su, flags=fl)
            ps, pu, pf = plain.insert_score(tx, 1.0)
            rs, ru, rf = ref.insert_score(X, 1.0)
        torch.cuda.synchronize()
        assert torch.equal(sc, ps) and torch.equal(su, pu) and torch.equal(fl, pf), i
        assert np.array_equal(ace.u32(su), ru) and np.array_equal(sc.cpu().numpy(), rs), i
    assert np.array_equal(g.counts(), ref.counts)
    a, b = g.stats(), ref.stats()
    for k in ("n_ins", "n_scored", "Q", "S1", "S2", "mu", "sigma", "mu_ins"):
        assert a[k] == b[k], k
    p = g.profile_read()
    assert p["hash"]["launches"] == 6 and p["score"]["launches"] == 6 and p["flags"]["launches"] == 6
    torch.cuda.set_stream(torch.cuda.default_stream())


def test_graph_replay_is_faster_for_small_batches():
    """The small config (n = 10,000): replayed calls take less time than direct ones."""
    w = workloads.small(seed=1)
    X = torch.from_numpy(w["X"]).cuda()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {}
    for mode in (False, True):
        det = ace.Detector(w["d"], w["K"], w["L"], seed=4, precision="fp32")
        det.set_graph(mode)
        sc = torch.empty(X.shape[0], dtype=torch.float64, device="cuda")
        su = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
        fl = torch.empty(X.shape[0], dtype=torch.uint8, device="cuda")
        for _ in range(5):
            det.insert_score(X, 1.0, scores=sc, sums=su, flags=fl)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(200):
            det.insert_score(X, 1.0, scores=sc, sums=su, flags=fl)
        e1.record()
        torch.cuda.synchronize()
        out[mode] = e0.elapsed_time(e1) / 200
    torch.cuda.set_stream(torch.cuda.default_stream())
    assert out[True] < out[False], out
