"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element,
on the same seeded inputs.  Ids, counts, sums, flags and scores are compared bit-exactly;
mu and sigma are compared bit-exactly too (tighter than the 1e-12 relative bar), because both
sides take the same correctly rounded binary64 steps on the same exact integers."""
import numpy as np
import pytest

import oracle
from paper_1706_06664_gb300 import ace, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = ["fp32", "bf16"]


def _dev(X):
    if X.dtype == np.uint16:
        return torch.from_numpy(X.view(np.int16)).cuda()
    return torch.from_numpy(X).cuda()


def _detector(d, K, L, seed=0, W=None, precision="fp32"):
    try:
        return ace.Detector(d, K, L, seed=seed, W=W, precision=precision)
    except ace.AceError as e:
        if e.code == ace.ACE_ERR_UNSUPPORTED:
            pytest.skip(f"{precision} engine not available for d={d} K={K} L={L}")
        raise


def _pair(d, K, L, seed=None, W=None, precision="fp32"):
    det = _detector(d, K, L, seed=seed or 0, W=W, precision=precision)
    ref = oracle.Detector(d, K, L, seed=seed, W=W if W is not None else det.projection())
    return det, ref


def _engine_used(det, precision):
    want = {"fp32": ace.ACE_PROJ_FP32, "bf16": ace.ACE_PROJ_BF16}[precision]
    assert det.stats()["precision"] == want


def _compare_score(out, ref_out):
    sc, su, fl = out
    rs, ru, rf = ref_out
    torch.cuda.synchronize()
    assert np.array_equal(ace.u32(su), ru)
    assert np.array_equal(sc.cpu().numpy(), rs)
    assert np.array_equal(fl.cpu().numpy(), rf)


def _compare_stats(det, ref, alpha=1.0):
    s, r = det.stats(), ref.stats(alpha)
    for k in ("n_ins", "n_scored", "Q", "S1", "S2"):
        assert s[k] == r[k], k
    for k in ("mu_ins", "mu", "sigma"):
        assert s[k] == r[k], (k, s[k], r[k])
    assert s["status"] == 0


def test_projection_generator_matches_oracle():
    for (d, K, L, seed) in [(32, 10, 20, 1), (41, 15, 50, 2), (7, 3, 5, 2**63 + 12345), (1024, 16, 64, 9)]:
        for w_bf16 in (False, True):
            det = ace.Detector(d, K, L, seed=seed, w_bf16=w_bf16)
            assert np.array_equal(det.projection(), oracle.projection_from_seed(d, K, L, seed, w_bf16=w_bf16))
            det.close()


@pytest.mark.parametrize("precision", PRECS)
def test_hand_example(precision):
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_example.json")))
    W = np.array(g["W_columns"], dtype=np.float32).T.copy()
    X = np.array(g["X"], dtype=np.float32)
    det = _detector(3, 2, 2, W=W, precision=precision)
    ids = ace.u32(det.hash(_dev(X)))
    assert ids.tolist() == g["ids"]
    sc, su, fl = det.insert_score(_dev(X), 1.0)
    torch.cuda.synchronize()
    assert det.counts().tolist() == g["counts"]
    assert ace.u32(su).tolist() == g["sums"]
    assert sc.cpu().numpy().tolist() == g["scores"]
    assert fl.cpu().numpy().tolist() == g["flags"]
    st = det.stats()
    assert st["Q"] == g["Q"] and st["mu_ins"] == g["mu_ins"] and st["mu"] == g["mu"]
    ref = oracle.Detector(3, 2, 2, W=W)
    ref.insert_score(X, 1.0)
    assert st["sigma"] == ref.stats()["sigma"]
    assert st["rechecks"] >= 1  # x1 projects to exactly 0 on column 3


def _deferral_bounded(det, pairs, precision, frac=0.02):
    """The tensor-core engine defers only the (point, table) pairs with a column inside its
    error bound: a small fraction on these recipes.  A broken classification that defers most
    pairs still gives exact results (the deferred pairs are resolved exactly), so the count is
    checked on its own.  The SIMT engine defers nothing."""
    st = det.stats()
    if precision == "fp32":
        assert st["deferred"] == 0
    else:
        assert 0 < st["deferred"] <= frac * pairs, (st["deferred"], pairs)


@pytest.mark.parametrize("precision", PRECS)
def test_small_config_full_size(precision):
    """Config 'small' at its full size: n=10,000, d=32, K=10, L=20; insert all, score all."""
    w = workloads.small(seed=1)
    det, ref = _pair(w["d"], w["K"], w["L"], seed=17, precision=precision)
    Xd = _dev(w["X"])
    assert np.array_equal(ace.u32(det.hash(Xd)), ref.hash(w["X"]))
    det.insert(Xd)
    ref.insert(w["X"])
    assert np.array_equal(det.counts(), ref.counts)
    _compare_score(det.score(Xd, w["alpha"]), ref.score(w["X"], w["alpha"]))
    _compare_stats(det, ref)
    _engine_used(det, precision)
    _deferral_bounded(det, 3 * w["X"].shape[0] * w["L"], precision)


@pytest.mark.parametrize("precision", PRECS)
def test_kdd_shaped_reduced(precision):
    """KDD-shaped recipe (d=41, K=15, L=50) at n=20,011: many tiles and a ragged tail."""
    w = workloads.kdd(seed=2, n=20_011)
    det, ref = _pair(w["d"], w["K"], w["L"], seed=5, precision=precision)
    Xd = _dev(w["X"])
    _compare_score(det.insert_score(Xd, 1.0), ref.insert_score(w["X"], 1.0))
    assert np.array_equal(det.counts(), ref.counts)
    _compare_stats(det, ref)
    # a second batch: scores use the running statistics over both batches
    w2 = workloads.kdd(seed=3, n=3001)
    _compare_score(det.score(_dev(w2["X"]), 2.0), ref.score(w2["X"], 2.0))
    _compare_stats(det, ref, 2.0)
    _engine_used(det, precision)
    _deferral_bounded(det, (w["X"].shape[0] + w2["X"].shape[0]) * w["L"], precision)


@pytest.mark.parametrize("precision", ["fp32"])
def test_highdim_bf16_reduced(precision):
    """High-dimensional recipe (bfloat16 inputs, d=1024, K=16, L=64) at n=1,500."""
    w = workloads.highdim(seed=3, n=1500)
    det, ref = _pair(w["d"], w["K"], w["L"], seed=9, precision=precision)
    Xd = _dev(w["X"])
    assert np.array_equal(ace.u32(det.hash(Xd)), ref.hash(w["X"]))
    _compare_score(det.insert_score(Xd, 1.0), ref.insert_score(w["X"], 1.0))
    assert np.array_equal(det.counts(), ref.counts)
    _compare_stats(det, ref)


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 24, 2), (5, 17, 3), (64, 2, 100), (33, 7, 40), (130, 13, 11)])
def test_shapes_and_ragged_batches(shape, precision):
    d, K, L = shape
    rng = np.random.default_rng(sum(shape))
    det, ref = _pair(d, K, L, seed=d * 1000 + K, precision=precision)
    for n in (1, 127, 129, 300):
        X = rng.standard_normal((n, d)).astype(np.float32)
        _compare_score(det.insert_score(_dev(X), 1.0), ref.insert_score(X, 1.0))
    assert np.array_equal(det.counts(), ref.counts)
    _compare_stats(det, ref)


@pytest.mark.parametrize("precision", PRECS)
def test_edge_values_exact_zeros_nonfinite_subnormal_huge(precision):
    d, K, L = 6, 4, 5
    W = workloads.gaussian_w(d, K, L, 3)
    W[:, 0] = [1, -1, 0, 0, 0, 0]
    X = np.zeros((12, d), dtype=np.float32)
    X[1] = [1, 1, 0, 0, 0, 0]             # exact zero on column 0
    X[2, 3] = np.nan                        # NaN -> every projection NaN -> bucket 0
    X[3, 0] = np.inf                        # +inf
    X[4, 1] = -np.inf
    X[5] = 1e-40                            # subnormal coordinates
    X[6] = [3e38, -3e38, 1e38, 0, 0, 0]     # squared norm overflows binary32
    X[7] = [2.0**-140, 0, 0, 0, 0, 0]
    X[8] = 1.0
    X[9] = -1.0
    X[10, 5] = 1.0
    X[11] = [1, 1, 1e-7, -1e-7, 0, 0]
    det, ref = _pair(d, K, L, W=W, precision=precision)
    Xd = _dev(X)
    assert np.array_equal(ace.u32(det.hash(Xd)), ref.hash(X))
    _compare_score(det.insert_score(Xd, 1.0), ref.insert_score(X, 1.0))
    st = det.stats()
    assert st["nonfinite_points"] >= 4
    assert st["rechecks"] > 0


@pytest.mark.parametrize("precision", PRECS)
def test_zero_column_and_zero_batch(precision):
    d, K, L = 4, 3, 2
    W = workloads.gaussian_w(d, K, L, 4)
    W[:, 2] = 0.0
    rng = np.random.default_rng(1)
    X = rng.standard_normal((50, d)).astype(np.float32)
    det, ref = _pair(d, K, L, W=W, precision=precision)
    det.insert(_dev(np.zeros((0, d), dtype=np.float32)))
    _compare_score(det.insert_score(_dev(X), 0.5), ref.insert_score(X, 0.5))
    _compare_stats(det, ref, 0.5)


def test_score_does_not_insert_and_reset():
    w = workloads.small(seed=5, n=2000)
    det, ref = _pair(w["d"], w["K"], w["L"], seed=3)
    Xd = _dev(w["X"])
    det.score(Xd, 1.0)
    torch.cuda.synchronize()
    assert int(det.counts().sum()) == 0
    det.insert(Xd)
    det.reset()
    st = det.stats()
    assert st["n_ins"] == 0 and st["n_scored"] == 0 and int(det.counts().sum()) == 0


@pytest.mark.parametrize("precision", PRECS)
def test_near_orthogonal_points_are_exact(precision):
    """Points whose projection on chosen columns is tiny relative to ||x|| (|x.w| / (||x|| ||w||)
    from 1e-3 down to 1e-9 and exactly 0): every such bit is decided inside the guard band and
    must still equal the binary64 definition."""
    w = workloads.kdd(seed=11, n=4096)
    d, K, L = w["d"], w["K"], w["L"]
    det, ref = _pair(d, K, L, seed=21, precision=precision)
    W = det.projection().astype(np.float64)
    rng = np.random.default_rng(3)
    X = w["X"].astype(np.float64).copy()
    eps = [1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9, 0.0]
    for i in range(X.shape[0]):
        c = rng.integers(0, K * L)
        wc = W[:, c]
        x = X[i] - (X[i] @ wc) / (wc @ wc) * wc
        e = eps[i % len(eps)] * np.linalg.norm(x) / np.linalg.norm(wc) * rng.choice([-1, 1])
        X[i] = x + e * wc
    X = X.astype(np.float32)
    _compare_score(det.insert_score(_dev(X), 1.0), ref.insert_score(X, 1.0))
    assert np.array_equal(det.counts(), ref.counts)
    _compare_stats(det, ref)
    assert det.stats()["rechecks"] > X.shape[0] // 4
    _engine_used(det, precision)


def test_cancelling_instructions_next_to_the_band():
    """The tensor-core engine's accumulation model under stress, next to the edge of its band
    (B = tau ||x||_up; at d = 41, tau = 5.1019e-5: the bfloat16 split's 3 2^-16, the
    accumulation term over three plus six instructions, 1 % margin).  Each point is x = a (t_i w_i) along its chosen unit
    column w = w_c / ||w_c||, with t_i = +1 on the first 16 coordinates (one MMA instruction),
    -1 on the next 16 and balancing signs on the rest: every instruction's addends then add up
    to about ||x|| (the Cauchy-Schwarz worst case the bound is built on), the accumulator swings
    out and back, and the small products are truncated against it.  One coordinate then places
    x.w at r tau ||x|| for r from 0.5 to 10, either sign, so many bits are decided just outside
    the band, on the model alone.  Every id, count and score must equal the oracle's; the
    points with r < 1 are deferred, the far ones (r >= 1.5) are not."""
    d, K, L = 41, 15, 50
    det, ref = _pair(d, K, L, seed=33, precision="bf16")
    W = det.projection().astype(np.float64)
    rng = np.random.default_rng(41)
    tau = 5.10191e-5
    ratios = [0.5, 0.9, 0.99, 1.01, 1.02, 1.05, 1.1, 1.2, 1.5, 2.0, 3.0, 10.0]
    n = 24 * len(ratios) * 10
    X = np.zeros((n, d))
    for i in range(n):
        c = int(rng.integers(0, K * L))
        w = W[:, c] / np.linalg.norm(W[:, c])
        t = np.where(np.arange(d) < 16, 1.0, -1.0)
        acc = float((t[:32] * w[:32] ** 2).sum())
        for k in range(32, d):  # the last coordinates bring the sum back towards 0
            t[k] = -1.0 if acc > 0 else 1.0
            acc += t[k] * w[k] ** 2
        x = t * w * 2.0 ** rng.uniform(-4, 8)
        k = 32 + int(np.argmax(np.abs(w[32:])))
        sign = 1.0 if (i // len(ratios)) % 2 == 0 else -1.0
        for _ in range(6):  # the norm moves with x[k]: a few rounds settle the ratio
            x[k] += (sign * ratios[i % len(ratios)] * tau * np.linalg.norm(x) - x @ w) / w[k]
        X[i] = x
    X = X.astype(np.float32)
    _compare_score(det.insert_score(_dev(X), 1.0), ref.insert_score(X, 1.0))
    assert np.array_equal(det.counts(), ref.counts)
    _compare_stats(det, ref)
    _engine_used(det, "bf16")
    inside = sum(1 for i in range(n) if ratios[i % len(ratios)] < 1.0)
    far = sum(1 for i in range(n) if ratios[i % len(ratios)] >= 1.5)
    deferred = det.stats()["deferred"]
    assert inside <= deferred <= n - far + n // 3, (inside, deferred, far)


def test_near_orthogonal_points_high_d_are_exact():
    """d = 1024 on the binary32 engine, where the warp recheck, Dot2 and the binary64
    definition each decide some bits: points whose projection on a chosen column is 1e-3 down
    to 1e-9 of ||x|| ||w_c||, and exact ties (two equal rows of W, x = a (e_r1 - e_r2): every
    projection is exactly 0, so every bit is 0)."""
    d, K, L, n = 1024, 16, 8, 1024
    rng = np.random.default_rng(29)
    W = rng.standard_normal((d, K * L)).astype(np.float32)
    W[7] = W[500]
    X = rng.standard_normal((n, d))
    Wd = W.astype(np.float64)
    eps = [1e-3, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9]
    for i in range(n):
        if i % 8 == 7:
            X[i] = 0.0
            X[i, 7], X[i, 500] = 1.5 + i, -(1.5 + i)
            continue
        wc = Wd[:, rng.integers(0, K * L)]
        x = X[i] - (X[i] @ wc) / (wc @ wc) * wc
        X[i] = x + eps[i % len(eps)] * np.linalg.norm(x) / np.linalg.norm(wc) * rng.choice([-1, 1]) * wc
    X = X.astype(np.float32)
    det, ref = _pair(d, K, L, W=W, precision="fp32")
    Xd = _dev(X)
    ids = ace.u32(det.hash(Xd))
    assert np.array_equal(ids, ref.hash(X))
    assert not ids[7::8].any()  # the exact ties
    _compare_score(det.insert_score(Xd, 1.0), ref.insert_score(X, 1.0))
    assert np.array_equal(det.counts(), ref.counts)
    _compare_stats(det, ref)
    assert det.stats()["rechecks"] > 0  # some bits reached Dot2 / binary64


@pytest.mark.parametrize("precision", PRECS)
def test_output_buffers_at_any_alignment(precision):
    """Scores, sums and flags written to caller buffers that start 8, 4 and 1 bytes past an
    aligned address, and to aligned ones, for a ragged batch: all equal the oracle's."""
    w = workloads.small(seed=1, n=1001)
    X = w["X"]
    Xd = _dev(X)
    for shift in (0, 1):
        det, ref = _pair(w["d"], w["K"], w["L"], seed=17, precision=precision)
        n = X.shape[0]
        sc = torch.empty(n + 1, dtype=torch.float64, device="cuda")[shift:shift + n]
        su = torch.empty(n + 1, dtype=torch.int32, device="cuda")[shift:shift + n]
        fl = torch.empty(n + 1, dtype=torch.uint8, device="cuda")[shift:shift + n]
        _compare_score(det.insert_score(Xd, 1.0, scores=sc, sums=su, flags=fl), ref.insert_score(X, 1.0))
        # sums left to the library (aligned scratch), scores and flags as above
        s2, _, f2 = det.score(Xd, 2.0, scores=sc, sums=None, flags=fl)
        torch.cuda.synchronize()
        r2 = ref.score(X, 2.0)
        assert np.array_equal(s2.cpu().numpy(), r2[0]) and np.array_equal(f2.cpu().numpy(), r2[2])
        det.close()


def test_tensor_core_engine_refuses_unfit_shapes():
    """No tensor-core design covers d > 64 with d not a multiple of 8; AUTO then runs the SIMT
    engine."""
    with pytest.raises(ace.AceError) as e:
        ace.Detector(1028, 16, 64, seed=1, precision="bf16")
    assert e.value.code == ace.ACE_ERR_UNSUPPORTED
    det = ace.Detector(1028, 16, 64, seed=1, precision="auto")
    X = torch.zeros((4, 1028), dtype=torch.bfloat16, device="cuda")
    det.insert(X)
    assert det.stats()["precision"] == ace.ACE_PROJ_FP32


def test_host_entry_point_matches_device_path():
    w = workloads.kdd(seed=6, n=7777)
    a, ref = _pair(w["d"], w["K"], w["L"], seed=8)
    n = w["X"].shape[0]
    sc = np.empty(n, dtype=np.float64)
    su = np.empty(n, dtype=np.uint32)
    fl = np.empty(n, dtype=np.uint8)
    a.insert_score_host(w["X"], 1.0, sc, su, fl)
    rs, ru, rf = ref.insert_score(w["X"], 1.0)
    assert np.array_equal(su, ru) and np.array_equal(sc, rs) and np.array_equal(fl, rf)
    _compare_stats(a, ref)


@pytest.mark.parametrize("precision", PRECS)
def test_host_entry_point_chunked(precision):
    """A batch large enough for the host entry point to copy and hash it in eight chunks
    (ragged last chunk), twice in a row: every output equals the oracle's."""
    w = workloads.kdd(seed=9, n=262147)
    a, ref = _pair(w["d"], w["K"], w["L"], seed=4, precision=precision)
    n = w["X"].shape[0]
    for rep in range(2):
        X = w["X"] if rep == 0 else np.ascontiguousarray(w["X"][::-1])
        sc = np.empty(n, dtype=np.float64)
        su = np.empty(n, dtype=np.uint32)
        fl = np.empty(n, dtype=np.uint8)
        a.insert_score_host(X, 1.0, sc, su, fl)
        rs, ru, rf = ref.insert_score(X, 1.0)
        assert np.array_equal(su, ru) and np.array_equal(sc, rs) and np.array_equal(fl, rf)
    _engine_used(a, precision)
    _compare_stats(a, ref)
    assert np.array_equal(a.counts(), ref.counts)


@pytest.mark.parametrize("precision", PRECS)
def test_host_async_batches_in_order(precision):
    """Three batches enqueued back to back (two staging slots alternate, buffers grow between
    batches of different sizes), then one wait: each batch's outputs equal the oracle's run
    of the same batches in the same order."""
    w = workloads.kdd(seed=10, n=200000)
    a, ref = _pair(w["d"], w["K"], w["L"], seed=6, precision=precision)
    parts = [w["X"][:70000], w["X"][70000:190001], w["X"][190001:]]
    outs = []
    for X in parts:
        n = X.shape[0]
        o = (torch.empty(n, dtype=torch.float64).pin_memory().numpy(),
             torch.empty(n, dtype=torch.int32).pin_memory().numpy().view(np.uint32),
             torch.empty(n, dtype=torch.uint8).pin_memory().numpy())
        a.insert_score_host_async(X, 1.0, *o)
        outs.append(o)
    a.host_wait()
    for X, (sc, su, fl) in zip(parts, outs):
        rs, ru, rf = ref.insert_score(X, 1.0)
        assert np.array_equal(su, ru) and np.array_equal(sc, rs) and np.array_equal(fl, rf)
    _engine_used(a, precision)
    _compare_stats(a, ref)


@pytest.mark.parametrize("precision", PRECS)
def test_host_async_small_and_chunked_batches_mixed(precision):
    """Small single-chunk batches (their copy runs on the caller's stream) and chunked ones
    (copy stream, two chunks or more) alternate over the two staging slots with no wait in
    between: each batch's outputs equal the oracle's run of the same batches in order."""
    w = workloads.kdd(seed=11, n=200000)
    a, ref = _pair(w["d"], w["K"], w["L"], seed=7, precision=precision)
    sizes = [1, 5000, 40000, 300, 70000, 2, 9000, 33000, 128, 17]
    cuts = np.concatenate([[0], np.cumsum(sizes)])
    parts = [w["X"][cuts[i]:cuts[i + 1]] for i in range(len(sizes))]
    outs = []
    for X in parts:
        n = X.shape[0]
        o = (torch.empty(n, dtype=torch.float64).pin_memory().numpy(),
             torch.empty(n, dtype=torch.int32).pin_memory().numpy().view(np.uint32),
             torch.empty(n, dtype=torch.uint8).pin_memory().numpy())
        a.insert_score_host_async(X, 1.0, *o)
        outs.append(o)
    a.host_wait()
    for X, (sc, su, fl) in zip(parts, outs):
        rs, ru, rf = ref.insert_score(X, 1.0)
        assert np.array_equal(su, ru) and np.array_equal(sc, rs) and np.array_equal(fl, rf)
    _engine_used(a, precision)
    _compare_stats(a, ref)


def test_kdd_full_size_against_oracle():
    """KDD-shaped recipe at its full size (n=500,000, d=41, K=15, L=50) in the bench's launch
    configuration (one insert_score call on the whole batch), on both engines: every id,
    count, sum, score and flag, and the statistics, against the oracle's run of the same batch
    (computed once)."""
    w = workloads.kdd(seed=2)
    X = w["X"]
    Xd = _dev(X)
    ref = oracle.Detector(w["d"], w["K"], w["L"], seed=5)
    ref_ids = ref.hash(X)
    rs, ru, rf = ref.insert_score(X, 1.0)
    for precision in PRECS:
        det = _detector(w["d"], w["K"], w["L"], seed=5, precision=precision)
        assert np.array_equal(det.projection(), ref.W)
        assert np.array_equal(ace.u32(det.hash(Xd)), ref_ids)
        _compare_score(det.insert_score(Xd, 1.0), (rs, ru, rf))
        assert np.array_equal(det.counts(), ref.counts)
        _compare_stats(det, ref)
        _engine_used(det, precision)
        det.close()


@pytest.mark.parametrize("precision", PRECS)
def test_delete_matches_oracle(precision):
    """§3.4.1 deletion on the device: insert A and B, delete B, then score C — counts,
    statistics and scores equal the oracle's, and the arrays equal those of A alone."""
    w = workloads.kdd(seed=12, n=60000)
    A, Bset, C = w["X"][:30000], w["X"][30000:52000], w["X"][52000:]
    a, ref = _pair(w["d"], w["K"], w["L"], seed=7, precision=precision)
    a.insert(_dev(A))
    ref.insert(A)
    a.insert(_dev(Bset))
    ref.insert(Bset)
    a.delete(_dev(Bset))
    ref.delete(Bset)
    assert np.array_equal(a.counts(), ref.counts)
    only_a = oracle.Detector(w["d"], w["K"], w["L"], W=a.projection())
    only_a.insert(A)
    assert np.array_equal(a.counts(), only_a.counts)
    sc, su, fl = a.score(_dev(C), 1.0)
    rs, ru, rf = ref.score(C, 1.0)
    torch.cuda.synchronize()
    assert np.array_equal(ace.u32(su), ru) and np.array_equal(sc.cpu().numpy(), rs)
    assert np.array_equal(fl.cpu().numpy(), rf)
    _engine_used(a, precision)
    _compare_stats(a, ref)


@pytest.mark.parametrize("precision", PRECS)
def test_delete_hand_example_and_rejection(precision):
    import json, os
    gd_path = os.path.join(os.path.dirname(__file__), "golden")
    g = json.load(open(os.path.join(gd_path, "hand_example.json")))
    gd = json.load(open(os.path.join(gd_path, "hand_example_delete.json")))
    W = np.array(g["W_columns"], dtype=np.float32).T.copy()
    X = np.array(g["X"], dtype=np.float32)
    det = _detector(3, 2, 2, W=W, precision=precision)
    det.insert(_dev(X))
    bad = np.array([X[0], gd["not_inserted_point"]], dtype=np.float32)
    with pytest.raises(ace.AceError) as e:
        det.delete(_dev(bad))
    assert e.value.code == ace.ACE_ERR_ARG
    assert det.counts().tolist() == g["counts"] and det.stats()["n_ins"] == 4
    for step, i in enumerate(gd["delete_order"]):
        det.delete(_dev(X[i:i + 1]))
        st = det.stats()
        assert det.counts().tolist() == gd["counts_after"][step]
        assert st["Q"] == gd["Q_after"][step] and st["mu_ins"] == gd["mu_ins_after"][step]
    with pytest.raises(ace.AceError):
        det.delete(_dev(X))  # four points from a detector that holds two


@pytest.mark.parametrize("precision", PRECS)
def test_projection_error_within_guard_bound(precision):
    """ace_project: each engine's binary32 estimate of x.w_c lies within the bound its guard
    relies on (binary32 chain: (gamma_d + gamma64_d) ||x|| ||w_c||; tensor cores: the band tau
    of the BF16 split, the probed accumulation model and the binary64 sum), against the
    oracle's binary64 projection; and the call changes no state."""
    for w in (workloads.small(seed=3, n=3000), workloads.kdd(seed=4, n=4000)):
        det = _detector(w["d"], w["K"], w["L"], seed=9, precision=precision)
        X = w["X"]
        est = det.project(_dev(X)).cpu().numpy().astype(np.float64)
        torch.cuda.synchronize()
        W = det.projection()
        s64 = oracle.project(X, W)
        xn = np.linalg.norm(X.astype(np.float64), axis=1)[:, None]
        wn = np.linalg.norm(W.astype(np.float64), axis=0)[None, :]
        rel = np.abs(est - s64) / (xn * wn)
        d = w["d"]
        u32, u64 = 2.0**-24, 2.0**-53
        if precision == "fp32":
            bound = (d * u32 / (1 - d * u32) + d * u64 / (1 - d * u64)) * 1.02
        else:
            d_pad = (d + 15) // 16 * 16
            tau_acc = 5.25 * 1.5 * ((d_pad // 16 + 1) + 2 * d_pad // 16 * 2.0**-6) * 2.0**-23 * (1 + 2.0**-6)
            bound = (3 * 2.0**-16 * (1 + 2.0**-6) + tau_acc * (1 + 2.0**-6) + 2.0**-23 + d * u64) * 1.01 + 2.0**-23
        assert rel.max() <= bound, (precision, rel.max(), bound)
        assert det.stats()["n_ins"] == 0 and det.stats()["rechecks"] == 0 and not det.counts().any()
