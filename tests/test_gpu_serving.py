"""Request server (continuous batching over several detectors): every request's outputs
equal the oracle's, which replays each detector's requests in submission order; and a
detector's results are the same when its requests run alone as when they run mixed with
other detectors' requests."""
import numpy as np
import pytest

import oracle
from paper_1706_06664_gb300 import ace, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pinned(n, dtype):
    t = {np.float64: torch.float64, np.uint32: torch.int32, np.uint8: torch.uint8}[dtype]
    a = torch.empty(max(n, 1), dtype=t).pin_memory().numpy()[:n]
    return a.view(np.uint32) if dtype == np.uint32 else a


def _requests(seed, shapes, per_det):
    """Interleaved (det, op, X) requests: ops cycle insert / insert_score / score at random,
    sizes log-uniform in [1, 2000]; the first request of each detector inserts."""
    rng = np.random.default_rng(seed)
    reqs = []
    for det, (d, K, L) in enumerate(shapes):
        sizes = workloads.request_sizes(seed + det, per_det, 1, 2000)
        start = 0
        for k, n in enumerate(sizes):
            op = ace.OP_INSERT if k == 0 else int(rng.integers(0, 3))
            if d == 41:
                X = workloads.kdd(seed=100 * det + k, n=int(n))["X"]
            else:
                X = workloads.stream_chunk(seed + det, start, int(n), total=10_000_000, d=d)
            start += int(n)
            X = torch.from_numpy(X).pin_memory().numpy()
            reqs.append((det, op, X))
    # mix detectors at random, each detector's requests staying in their order
    mixed, queues = [], {d: [r for r in reqs if r[0] == d] for d in range(len(shapes))}
    while any(queues.values()):
        det = int(rng.choice([d for d, q in queues.items() if q]))
        mixed.append(queues[det].pop(0))
    return mixed


def _run(shapes, reqs, seeds):
    dets = [ace.Detector(d, K, L, seed=sd) for (d, K, L), sd in zip(shapes, seeds)]
    srv = ace.Server(dets, mem_budget_bytes=64 << 20)
    tickets, outs = [], []
    for det, op, X in reqs:
        n = X.shape[0]
        o = (_pinned(n, np.float64), _pinned(n, np.uint32), _pinned(n, np.uint8)) if op != ace.OP_INSERT else (None,) * 3
        tickets.append(srv.submit(det, op, X, 1.0, *o))
        outs.append(o)
    lat = [srv.wait(t) for t in tickets]
    srv.close()
    return dets, outs, lat


SHAPES = [(41, 15, 50), (41, 15, 50), (128, 15, 50), (128, 15, 50), (41, 15, 50)]


def test_server_matches_oracle_and_alone():
    reqs = _requests(21, SHAPES, per_det=14)
    dets, outs, lat = _run(SHAPES, reqs, seeds=[50 + i for i in range(len(SHAPES))])
    assert all(v > 0 for v in lat)
    refs = [oracle.Detector(d, K, L, W=dets[i].projection()) for i, (d, K, L) in enumerate(SHAPES)]
    for (det, op, X), o in zip(reqs, outs):
        ref = refs[det]
        if op == ace.OP_INSERT:
            ref.insert(X)
            continue
        rs, ru, rf = ref.insert_score(X, 1.0) if op == ace.OP_INSERT_SCORE else ref.score(X, 1.0)
        assert np.array_equal(o[1], ru) and np.array_equal(o[0], rs) and np.array_equal(o[2], rf)
    for dd, ref in zip(dets, refs):
        assert np.array_equal(dd.counts(), ref.counts)
        s, r = dd.stats(), ref.stats()
        for k in ("n_ins", "n_scored", "Q", "S1", "S2", "mu_ins", "mu", "sigma"):
            assert s[k] == r[k], k
    # detector 2's requests alone, through a fresh server: identical outputs
    alone = [r for r in reqs if r[0] == 2]
    alone_reqs = [(0, op, X) for (_, op, X) in alone]
    _, outs_alone, _ = _run([SHAPES[2]], alone_reqs, seeds=[52])
    mixed_outs = [o for (det, _, _), o in zip(reqs, outs) if det == 2]
    for a, m in zip(outs_alone, mixed_outs):
        if a[0] is not None:
            assert np.array_equal(a[0], m[0]) and np.array_equal(a[1], m[1]) and np.array_equal(a[2], m[2])


@pytest.mark.parametrize("threads", ["1", "4"])
def test_consecutive_inserts_are_coalesced_exactly(threads, monkeypatch):
    """A burst of small inserts to one detector, with scores between some of them, from a
    server with one and with four scheduler threads: the inserts that queue up behind the two
    in flight are admitted as one launch set (the server reports them), and every score, the
    counts and the statistics equal the oracle's replay of the requests one by one."""
    monkeypatch.setenv("ACE_SERVER_THREADS", threads)
    d, K, L = 128, 15, 50
    dets = [ace.Detector(d, K, L, seed=70 + i) for i in range(6)]
    srv = ace.Server(dets, mem_budget_bytes=64 << 20)
    assert srv.info()["threads"] == int(threads)
    refs = [oracle.Detector(d, K, L, W=dd.projection()) for dd in dets]
    rng = np.random.default_rng(5)
    reqs, start = [], 0
    for k in range(120):
        det = 0 if k % 3 else int(rng.integers(0, 6))
        n = int(rng.integers(1, 400))
        X = torch.from_numpy(workloads.stream_chunk(9, start, n, total=10_000_000, d=d)).pin_memory().numpy()
        start += n
        op = ace.OP_SCORE if k % 17 == 16 else ace.OP_INSERT
        reqs.append((det, op, X))
    tickets, outs = [], []
    for det, op, X in reqs:
        n = X.shape[0]
        o = (_pinned(n, np.float64), _pinned(n, np.uint32), _pinned(n, np.uint8)) if op == ace.OP_SCORE else (None,) * 3
        tickets.append(srv.submit(det, op, X, 1.0, *o))
        outs.append(o)
    for t in tickets:
        srv.wait(t)
    info = srv.info()
    srv.close()
    assert info["coalesced"] > 0, info
    for (det, op, X), o in zip(reqs, outs):
        if op == ace.OP_INSERT:
            refs[det].insert(X)
        else:
            rs, ru, rf = refs[det].score(X, 1.0)
            assert np.array_equal(o[1], ru) and np.array_equal(o[0], rs) and np.array_equal(o[2], rf)
    for dd, ref in zip(dets, refs):
        assert np.array_equal(dd.counts(), ref.counts)
        s, r = dd.stats(), ref.stats()
        for k in ("n_ins", "n_scored", "Q", "S1", "S2", "mu_ins", "mu", "sigma"):
            assert s[k] == r[k], k


def test_server_refuses_a_detector_twice():
    a = ace.Detector(20, 10, 4, seed=1)
    with pytest.raises(ace.AceError) as e:
        ace.Server([a, a])
    assert e.value.code == ace.ACE_ERR_ARG
