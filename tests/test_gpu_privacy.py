"""Privacy-preserving hashing (§4.5, ace_set_privacy): every engine and entry point that
hashes with noise gives the oracle's ids (the sign of the binary64 projection plus the exact
noise term), counts, scores, flags and statistics bit for bit; the noise index runs the same
way on both sides; what the noise cannot support is refused."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1706_06664_gb300 import ace, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(X):
    return torch.from_numpy(X.view(np.int16) if X.dtype == np.uint16 else X).cuda()


def _pair(d, K, L, seed, sigma, nseed, precision="auto", **kw):
    det = ace.Detector(d, K, L, seed=seed, precision=precision, **kw)
    det.set_privacy(sigma, nseed)
    ref = oracle.Detector(d, K, L, W=det.projection())
    ref.set_privacy(sigma, nseed)
    return det, ref


def _same_state(det, ref):
    assert np.array_equal(det.counts(), ref.counts)
    s, r = det.stats(), ref.stats()
    for k in ("n_ins", "n_scored", "Q", "S1", "S2", "mu_ins", "mu", "sigma"):
        assert s[k] == r[k], k
    assert det.privacy()["next_index"] == ref.nbase


def _step(det, ref, X, op="insert_score"):
    Xd = _dev(X)
    if op == "hash":
        assert np.array_equal(ace.u32(det.hash(Xd)), ref.hash(X))
        return
    if op == "insert":
        det.insert(Xd)
        ref.insert(X)
        torch.cuda.synchronize()
        return
    sc, su, fl = getattr(det, op)(Xd, 1.0)
    rs, ru, rf = getattr(ref, op)(X, 1.0)
    torch.cuda.synchronize()
    assert np.array_equal(ace.u32(su), ru)
    assert np.array_equal(sc.cpu().numpy(), rs) and np.array_equal(fl.cpu().numpy(), rf)


@pytest.mark.parametrize("shape,sigma", [((32, 10, 20), 0.5), ((41, 15, 50), 2.0), ((200, 12, 7), 0.05),
                                         ((1024, 16, 8), 3.0), ((77, 24, 3), 1.0)])
def test_simt_engine_parity(shape, sigma):
    """Binary32 engine: several tiles and a ragged tail, 16- and 32-bit ids, every entry point
    in turn (hash, insert, score, insert_score), binary32 and bfloat16 input."""
    d, K, L = shape
    det, ref = _pair(d, K, L, seed=d + K, sigma=sigma, nseed=1000 + d)
    rng = np.random.default_rng(d)
    for n, op in ((1, "insert"), (257, "insert_score"), (3000, "score"), (700, "hash"), (2100, "insert_score")):
        _step(det, ref, rng.standard_normal((n, d)).astype(np.float32), op)
    Xb = workloads.to_bf16_bits(rng.standard_normal((1500, d)).astype(np.float32))
    _step(det, ref, Xb, "insert_score")
    _same_state(det, ref)
    assert det.stats()["precision"] == ace.ACE_PROJ_FP32


def test_exact_ties_reach_the_binary64_tier():
    """Integer points, W entries k/4 (ACE_W_COUNTER) and sigma = 1: many noisy projections are
    exactly 0 (bit 0), so the Dot2 filter cannot decide them and the binary64 tier does."""
    d, K, L = 24, 12, 10
    det, ref = _pair(d, K, L, seed=5, sigma=1.0, nseed=77, precision="fp32", w_counter=True)
    assert np.array_equal(det.projection(), oracle.projection_from_seed(d, K, L, 5, counter=True))
    rng = np.random.default_rng(8)
    for n in (300, 4000):
        _step(det, ref, rng.integers(-2, 3, size=(n, d)).astype(np.float32))
    _same_state(det, ref)
    assert det.stats()["rechecks"] > 0


@pytest.mark.parametrize("shape", [(100, 12, 7), (256, 20, 8), (1024, 16, 64)])
def test_structured_engine_parity(shape):
    """ACE_W_HADAMARD detectors keep the transform engine under noise; integer rows with
    sigma = 4 put many noisy outputs exactly at 0."""
    d, K, L = shape
    det, ref = _pair(d, K, L, seed=d, sigma=0.7, nseed=5, w_hadamard=True)
    rng = np.random.default_rng(d + 1)
    _step(det, ref, rng.standard_normal((2000, d)).astype(np.float32))
    _step(det, ref, rng.standard_normal((333, d)).astype(np.float32), "hash")
    _same_state(det, ref)
    assert det.stats()["precision"] == ace.ACE_PROJ_FWHT
    det.set_privacy(4.0, 6)
    ref.set_privacy(4.0, 6)
    _step(det, ref, rng.integers(-1, 2, size=(1500, d)).astype(np.float32))
    _same_state(det, ref)
    assert det.stats()["rechecks"] > 0


def test_kdd_auto_engine_and_host_path():
    """At d = 41 the automatic choice would be the tensor-core engine; with noise it is the
    binary32 one.  The host-buffer entry point hashes in chunks: the chunks take consecutive
    noise indices."""
    w = workloads.kdd(seed=3, n=150000)
    det, ref = _pair(w["d"], w["K"], w["L"], seed=9, sigma=0.3, nseed=10)
    _step(det, ref, w["X"][:20000])
    assert det.stats()["precision"] == ace.ACE_PROJ_FP32
    X = np.ascontiguousarray(w["X"][20000:])
    n = X.shape[0]
    sc, su, fl = np.empty(n), np.empty(n, dtype=np.uint32), np.empty(n, dtype=np.uint8)
    det.insert_score_host(X, 1.0, sc, su, fl)
    rs, ru, rf = ref.insert_score(X, 1.0)
    assert np.array_equal(su, ru) and np.array_equal(sc, rs) and np.array_equal(fl, rf)
    _same_state(det, ref)


def test_batch_noalloc_graph_window_checkpoint():
    """The batched launch (noisy and noise-free detectors mixed), the allocation-free entry
    point, graph replay (not used under noise: repeated identical calls draw fresh noise), a
    sliding window (removal by stored ids), and a checkpoint that carries the noise index."""
    K, L = 12, 32
    specs = workloads.batched_specs(seed=15, n_det=8, d_range=(16, 300), n_range=(1, 4000))
    dets, refs = [], []
    for g, (d, n, sd) in enumerate(specs):
        dt = ace.Detector(d, K, L, seed=sd, precision="fp32")
        rf = oracle.Detector(d, K, L, W=dt.projection())
        if g % 2:
            dt.set_privacy(0.1 * (g + 1), 500 + g)
            rf.set_privacy(0.1 * (g + 1), 500 + g)
        dets.append(dt)
        refs.append(rf)
    Xs = [workloads.batched_points(d, n, sd) for (d, n, sd) in specs]
    sc, su, fl = ace.batch_insert_score(dets, [_dev(X) for X in Xs])
    torch.cuda.synchronize()
    for g, (det, ref, X) in enumerate(zip(dets, refs, Xs)):
        rs, ru, rf = ref.insert_score(X, 1.0)
        assert np.array_equal(ace.u32(su[g]), ru), g
        assert np.array_equal(sc[g].cpu().numpy(), rs) and np.array_equal(fl[g].cpu().numpy(), rf), g
        _same_state(det, ref)

    d, K, L = 64, 14, 20
    det, ref = _pair(d, K, L, seed=1, sigma=0.25, nseed=2)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((900, d)).astype(np.float32)
    Xd = _dev(X)
    sc, su, fl = det.insert_score_noalloc(Xd, 1.0)
    rs, ru, rf = ref.insert_score(X, 1.0)
    assert np.array_equal(ace.u32(su), ru) and np.array_equal(fl.cpu().numpy(), rf)
    det.set_graph(True)
    for _ in range(4):  # same arguments every time
        _step(det, ref, X, "score")
    _same_state(det, ref)

    blob = det.save()
    det2 = ace.Detector.load(blob)
    assert det2.privacy() == det.privacy()
    ref2 = oracle.Detector(d, K, L, W=ref.W)
    ref2.counts[...] = ref.counts
    ref2.n_ins, ref2.st[:] = ref.n_ins, ref.st
    ref2.sigma, ref2.noise_seed, ref2.nbase = ref.sigma, ref.noise_seed, ref.nbase
    _step(det2, ref2, rng.standard_normal((500, d)).astype(np.float32))
    _same_state(det2, ref2)

    wd = ace.Detector(d, K, L, seed=3)
    wd.window(1000)
    wd.set_privacy(0.5, 4)
    wr = oracle.WindowDetector(d, K, L, 1000, W=wd.projection())
    wr.set_privacy(0.5, 4)
    for n in (600, 700, 900):
        _step(wd, wr, rng.standard_normal((n, d)).astype(np.float32))
    _same_state(wd, wr)


def test_server_requests_take_noise_in_order():
    """The request server (coalescing consecutive inserts) hashes a detector's requests in
    submission order: the noise indices are the oracle's."""
    d, K, L = 41, 15, 50
    det = ace.Detector(d, K, L, seed=21)
    det.set_privacy(0.4, 8)
    ref = oracle.Detector(d, K, L, W=det.projection())
    ref.set_privacy(0.4, 8)
    srv = ace.Server([det], mem_budget_bytes=64 << 20)
    reqs, tickets = [], []
    for k, n in enumerate((500, 40, 41, 1200, 7, 300)):
        X = torch.from_numpy(workloads.kdd(seed=40 + k, n=n)["X"]).pin_memory().numpy()
        op = ace.OP_INSERT if k < 3 or k == 4 else ace.OP_INSERT_SCORE
        outs = (np.empty(n), np.empty(n, dtype=np.uint32), np.empty(n, dtype=np.uint8)) if op != ace.OP_INSERT else (None,) * 3
        tickets.append(srv.submit(0, op, X, 1.0, *outs))
        reqs.append((op, X, outs))
    for t in tickets:
        srv.wait(t)
    srv.close()
    for op, X, outs in reqs:
        if op == ace.OP_INSERT:
            ref.insert(X)
        else:
            rs, ru, rf = ref.insert_score(X, 1.0)
            assert np.array_equal(outs[1], ru) and np.array_equal(outs[0], rs) and np.array_equal(outs[2], rf)
    _same_state(det, ref)


def test_refusals():
    d, K, L = 41, 15, 50
    det = ace.Detector(d, K, L, seed=3)
    for bad in (-1.0, float("nan"), float("inf"), 1e-30):
        with pytest.raises(ace.AceError) as e:
            det.set_privacy(bad, 1)
        assert e.value.code == ace.ACE_ERR_ARG
    with pytest.raises(ace.AceError) as e:
        det.set_privacy(1.0, 3)  # the projection's own seed
    assert e.value.code == ace.ACE_ERR_ARG
    det.set_precision("bf16")
    with pytest.raises(ace.AceError) as e:
        det.set_privacy(1.0, 4)
    assert e.value.code == ace.ACE_ERR_UNSUPPORTED
    det.set_precision("auto")
    det.set_privacy(1.0, 4)
    with pytest.raises(ace.AceError) as e:
        det.set_precision("bf16")
    assert e.value.code == ace.ACE_ERR_UNSUPPORTED
    X = torch.from_numpy(workloads.kdd(seed=1, n=100)["X"]).cuda()
    det.insert(X)
    with pytest.raises(ace.AceError) as e:
        det.delete(X[:10])
    assert e.value.code == ace.ACE_ERR_UNSUPPORTED
    # projections stay noise-free; turning the noise off restores plain SRP
    ref = oracle.Detector(d, K, L, W=det.projection())
    assert np.array_equal(det.project(X).cpu().numpy(), det.project(X).cpu().numpy())
    det.set_privacy(0.0, 0)
    assert det.privacy() == {"sigma": 0.0, "noise_seed": 0, "next_index": 0}
    assert np.array_equal(ace.u32(det.hash(X)), ref.hash(X.cpu().numpy()))
    lib = ace.load_library()
    assert lib.ace_set_privacy(None, ctypes.c_float(1.0), ctypes.c_uint64(1)) == ace.ACE_ERR_ARG
