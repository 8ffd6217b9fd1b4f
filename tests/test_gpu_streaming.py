"""GPU parity of the streaming tensor-core engine (large d, bfloat16 input; hash_gemm.cu)
against the CPU oracle, through the C ABI.  Ids, counts, sums, scores and flags are compared
bit-exactly, mu and sigma too.

Inputs include rows built to sit inside the engine's guard band, just outside it, and on
exact ties, so that a wrong error model (a band too narrow) or a wrong recheck shows up as an
id mismatch."""
import math

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


def _bf16(x):
    return workloads.bf16_bits_to_f32(workloads.to_bf16_bits(np.asarray(x, dtype=np.float32))).astype(np.float64)


def _row_band(W, Xf):
    """The streaming engine's guard band for each row, relative to ||x|| (the bound of
    hash_gemm.cu with the constants of plan_gemm, evaluated in binary64): B / ||x|| with
    B = ca E + cx ||x|| + tau_abs, E = sum_t ||x_<16t|| WP_t + ||x_Bt|| WB_t over the MMA
    instructions t of one pass."""
    d, KL = W.shape
    dp = (d + 63) // 64 * 64
    S = dp // 16
    Wd = W.astype(np.float64)
    hi = np.zeros((dp, KL))
    one = np.array_equal(_bf16(W), Wd)  # bfloat16-valued W: one product; the bound of column c
    if one:                              # is B ||w_c||, B from the normalised columns' profile
        hi[:d] = Wd / np.linalg.norm(Wd, axis=0)[None, :]
        rmax, tnorm = 0.0, 0.0
    else:
        wu = (Wd / np.linalg.norm(Wd, axis=0)[None, :]).astype(np.float32)
        hi[:d] = _bf16(wu)
        lo = _bf16(wu.astype(np.float64) - hi[:d])
        rmax, tnorm = np.sqrt(((wu.astype(np.float64) - hi[:d] - lo) ** 2).sum(axis=0).max()), 2.0**-23
    blk = (hi.reshape(S, 16, KL) ** 2).sum(axis=1)            # S x KL
    pre = np.vstack([np.zeros((1, KL)), np.cumsum(blk, axis=0)[:-1]])
    WP, WB = np.sqrt(pre.max(axis=1)), np.sqrt(blk.max(axis=1))
    # per k-block of four instructions: the prefix at the k-block's end for all four, and
    # Cauchy-Schwarz over the four block terms
    WPk = WP.reshape(-1, 4).sum(axis=1)
    WBk = np.sqrt((WB.reshape(-1, 4) ** 2).sum(axis=1))
    Xp = np.zeros((Xf.shape[0], dp))
    Xp[:, :d] = Xf
    xk = (Xp.reshape(-1, dp // 64, 64) ** 2).sum(axis=2)       # n x nkb
    E = np.sqrt(np.cumsum(xk, axis=1)) @ WPk + np.sqrt(xk) @ WBk
    xn = np.linalg.norm(Xf, axis=1)
    ca = 5.25 * 2.0**-23 * 1.25
    cx = ca * (2.0**-6 * S + 1) + rmax + tnorm + d * 2.0**-53 / (1 - d * 2.0**-53)
    return (ca * E + cx * xn) * 1.01 / xn


def _compare(out, ref_out):
    sc, su, fl = out
    rs, ru, rf = ref_out
    torch.cuda.synchronize()
    assert np.array_equal(ace.u32(su), ru)
    assert np.array_equal(sc.cpu().numpy(), rs)
    assert np.array_equal(fl.cpu().numpy(), rf)


def _stats_equal(det, ref, alpha=1.0):
    s, r = det.stats(), ref.stats(alpha)
    for k in ("n_ins", "n_scored", "Q", "S1", "S2", "mu_ins", "mu", "sigma"):
        assert s[k] == r[k], (k, s[k], r[k])
    assert s["status"] == 0


def _pair(d, K, L, seed=0, W=None, w_bf16=False):
    det = ace.Detector(d, K, L, seed=seed, W=W, precision="bf16", w_bf16=w_bf16)
    ref = oracle.Detector(d, K, L, W=det.projection())
    return det, ref


@pytest.mark.parametrize("w_bf16", [False, True])
def test_highdim_recipe_parity(w_bf16):
    """High-dimensional recipe (d=1024, K=16, L=64, bfloat16) at n=3,000 (23 full tiles and a
    ragged one), with binary32 W (two products) and bfloat16-valued W (one product): ids,
    counts, scores, flags and statistics equal the oracle's, the streaming engine did the
    hashing, and it deferred a small fraction of the columns."""
    w = workloads.highdim(seed=3, n=3000)
    det, ref = _pair(w["d"], w["K"], w["L"], seed=9, w_bf16=w_bf16)
    assert np.array_equal(det.projection(), oracle.projection_from_seed(w["d"], w["K"], w["L"], 9, w_bf16=w_bf16))
    Xd = _dev(w["X"])
    assert np.array_equal(ace.u32(det.hash(Xd)), ref.hash(w["X"]))
    _compare(det.insert_score(Xd, 1.0), ref.insert_score(w["X"], 1.0))
    assert np.array_equal(det.counts(), ref.counts)
    _stats_equal(det, ref)
    st = det.stats()
    assert st["precision"] == ace.ACE_PROJ_BF16 and st["tc_products"] == (1 if w_bf16 else 2)
    n, KL = w["X"].shape[0], w["K"] * w["L"]
    # the columns within the band of their row: about one per point on this recipe
    assert 0 < st["deferred"] <= 3 * n, st["deferred"]


@pytest.mark.parametrize("w_bf16", [False, True])
@pytest.mark.parametrize("shape", [(72, 16, 4), (128, 12, 7), (200, 20, 5), (256, 16, 17), (1024, 7, 3)])
def test_shapes_and_ragged_batches(shape, w_bf16):
    """Padded d (72 -> 128), K that does not divide 256 (12, 7: zero image rows in every unit),
    32-bit ids (K=20), several units per tile (L=17 at K=16), and batches of 1, 127, 129 and 300
    points in a row: every output equals the oracle's."""
    d, K, L = shape
    rng = np.random.default_rng(sum(shape))
    det, ref = _pair(d, K, L, seed=d * 7 + K, w_bf16=w_bf16)
    for n in (1, 127, 129, 300):
        X = workloads.to_bf16_bits(rng.standard_normal((n, d)).astype(np.float32))
        _compare(det.insert_score(_dev(X), 1.0), ref.insert_score(X, 1.0))
    assert np.array_equal(det.counts(), ref.counts)
    _stats_equal(det, ref)
    assert det.stats()["precision"] == ace.ACE_PROJ_BF16


def _near_orthogonal(W, n, rels, rng, ties_every=8, tie_rows=(7, 500)):
    """bfloat16 rows x whose projection on a chosen column c is rel * ||x|| ||w_c|| for rel in
    `rels` (cycling; both signs; a callable rel(x) is evaluated on the row), and exact ties.
    Four coordinates with large |w_c| are freed and set one after another to cancel the
    remaining projection (each step shrinks it by the bfloat16 rounding, 2^-8), so the target
    is met to about 2^-32 of the starting value.  Every `ties_every`-th row is a (e_r1 - e_r2)
    with two equal rows of W: every projection is exactly 0, every bit 0."""
    d, KL = W.shape
    Wd = W.astype(np.float64)
    X = np.zeros((n, d), dtype=np.float64)
    for i in range(n):
        if i % ties_every == ties_every - 1:
            a = 2.0**-3 * (1 + (i % 16) / 16)
            X[i, tie_rows[0]], X[i, tie_rows[1]] = a, -a
            continue
        c = int(rng.integers(0, KL))
        w = Wd[:, c]
        x = _bf16(rng.standard_normal(d) / math.sqrt(d))
        order = np.argsort(-np.abs(w))
        free = [int(t) for t in order[:12] if t not in tie_rows][:4]
        x[free] = 0.0
        rel = rels[i % len(rels)]
        rel = rel(x) if callable(rel) else rel
        want = rel * rng.choice([-1.0, 1.0]) * np.linalg.norm(x) * np.linalg.norm(w)
        for f in free:
            r = x @ w - want
            x[f] = _bf16([-r / w[f]])[0]
        X[i] = x
    return workloads.to_bf16_bits(X.astype(np.float32))


@pytest.mark.parametrize("w_bf16", [False, True])
def test_near_orthogonal_ties_and_band_edge(w_bf16):
    """d = 1024: rows whose projection on a chosen column is 3, 1.5 and 1.1 times the row's
    band (decided by the tensor cores: a band that is too narrow would give wrong bits here),
    0.9, 0.5, 1e-1, 1e-2 ... 1e-6 times it and 1e-14 of ||x|| ||w|| (resolved by the recheck
    tiers: binary32 running bound, Dot2, binary64), and exact ties.  Every id equals the
    oracle's."""
    d, K, L, n = 1024, 16, 8, 2048
    rng = np.random.default_rng(41)
    W = rng.standard_normal((d, K * L)).astype(np.float32)
    if w_bf16:
        W = _bf16(W).astype(np.float32)
    W[7] = W[500]

    def band(f):
        return lambda x: f * _row_band(W, x[None, :])[0]

    rels = [band(3), band(1.5), band(1.1), band(0.9), band(0.5), band(1e-1), band(1e-2), band(1e-3), band(1e-4),
            band(1e-6), 1e-14]
    X = _near_orthogonal(W, n, rels, rng)
    det, ref = _pair(d, K, L, W=W)
    Xd = _dev(X)
    ids = ace.u32(det.hash(Xd))
    assert np.array_equal(ids, ref.hash(X))
    assert not ids[7::8].any()  # the exact ties
    _compare(det.insert_score(Xd, 1.0), ref.insert_score(X, 1.0))
    assert np.array_equal(det.counts(), ref.counts)
    _stats_equal(det, ref)
    st = det.stats()
    assert st["precision"] == ace.ACE_PROJ_BF16 and st["rechecks"] > n // 4
    assert st["tc_products"] == (1 if w_bf16 else 2)


def _wide_cancelling_rows(n, d, rng):
    """bfloat16 rows in which each block of 16 coordinates (one MMA instruction's products)
    mixes magnitudes from 2^0 down to 2^-24 with alternating signs, so that the large products
    of a block cancel and the small ones fall below the accumulator's alignment."""
    X = np.zeros((n, d), dtype=np.float64)
    for i in range(n):
        e = rng.integers(0, 25, size=d)
        s = np.where(np.arange(d) % 2 == 0, 1.0, -1.0) * rng.choice([-1.0, 1.0], size=d // 16).repeat(16)
        X[i] = s * np.ldexp(1.0 + rng.integers(0, 128, size=d) / 128.0, -e)
        X[i, ::16] = s[::16] * 1.0
    return workloads.to_bf16_bits(X.astype(np.float32))


def test_projection_error_within_band_adversarial():
    """ace_project on the streaming engine: the binary32 estimate of x.w_c against the oracle's
    binary64 projection stays within the band tau ||x|| ||w_c|| (plus the final scaling's
    rounding) on the high-dimensional recipe and on rows built to stress the accumulation
    (wide exponent spread and cancellation inside every MMA instruction); the call changes
    no state."""
    d, K, L = 1024, 16, 8
    rng = np.random.default_rng(5)
    cases = [(workloads.highdim(seed=4, n=600)["X"], False), (_wide_cancelling_rows(400, d, rng), False),
             (workloads.highdim(seed=4, n=600)["X"], True), (_wide_cancelling_rows(400, d, rng), True)]
    for X, w_bf16 in cases:
        det = ace.Detector(d, K, L, seed=13, precision="bf16", w_bf16=w_bf16)
        est = det.project(_dev(X)).cpu().numpy().astype(np.float64)
        W = det.projection()
        s64 = oracle.project(X, W)
        Xf = workloads.bf16_bits_to_f32(X).astype(np.float64)
        rel = np.abs(est - s64) / (np.linalg.norm(Xf, axis=1)[:, None] * np.linalg.norm(W.astype(np.float64), axis=0)[None, :])
        band = _row_band(W, Xf)
        worst = (rel.max(axis=1) / band).max()
        assert (rel <= band[:, None] + 2.0**-23).all(), worst
        st = det.stats()
        assert st["n_ins"] == 0 and st["rechecks"] == 0 and not det.counts().any()
        # the same rows hash exactly
        ref = oracle.Detector(d, K, L, W=W)
        assert np.array_equal(ace.u32(det.hash(_dev(X))), ref.hash(X))
        det.close()


def test_host_entry_point_chunked_streaming():
    """The host-buffer entry copies and hashes a 70,001-point bfloat16 batch in chunks on the
    streaming engine (ids of each chunk into its slice of the batch's scratch), then inserts and
    scores the whole batch: every output equals the oracle's."""
    w = workloads.highdim(seed=8, n=70_001)
    d, K, L = w["d"], 16, 4
    det, ref = _pair(d, K, L, seed=3)
    n = w["X"].shape[0]
    sc = np.empty(n, dtype=np.float64)
    su = np.empty(n, dtype=np.uint32)
    fl = np.empty(n, dtype=np.uint8)
    det.insert_score_host(w["X"], 1.0, sc, su, fl)
    rs, ru, rf = ref.insert_score(w["X"], 1.0)
    assert np.array_equal(su, ru) and np.array_equal(sc, rs) and np.array_equal(fl, rf)
    assert det.stats()["precision"] == ace.ACE_PROJ_BF16
    _stats_equal(det, ref)


def test_delete_on_streaming_engine():
    """§3.4.1 deletion with the streaming engine: insert A and B, delete B: the arrays equal A's."""
    w = workloads.highdim(seed=12, n=4000)
    d, K, L = w["d"], 16, 8
    det, ref = _pair(d, K, L, seed=4)
    A, B = w["X"][:2500], w["X"][2500:]
    det.insert(_dev(A))
    det.insert(_dev(B))
    det.delete(_dev(B))
    ref.insert(A)
    assert np.array_equal(det.counts(), ref.counts)


def test_engine_selection_and_refusals():
    """d = 1024 runs the streaming engine for bfloat16 input; binary32 input falls back to the
    SIMT engine under AUTO and is refused when the tensor cores are forced; d not a multiple of
    8 (above 64) has no tensor-core engine."""
    det = ace.Detector(1024, 16, 4, seed=1, precision="auto")
    Xb = torch.zeros((4, 1024), dtype=torch.bfloat16, device="cuda")
    Xb[:, 0] = 1.0
    det.insert(Xb)
    assert det.stats()["precision"] == ace.ACE_PROJ_BF16
    det.insert(torch.zeros((4, 1024), dtype=torch.float32, device="cuda"))
    assert det.stats()["precision"] == ace.ACE_PROJ_FP32
    det.set_precision("bf16")
    with pytest.raises(ace.AceError) as e:
        det.insert(torch.zeros((4, 1024), dtype=torch.float32, device="cuda"))
    assert e.value.code == ace.ACE_ERR_UNSUPPORTED
    assert det.stats()["n_ins"] == 8
    with pytest.raises(ace.AceError) as e:
        ace.Detector(1030, 16, 4, seed=1, precision="bf16")
    assert e.value.code == ace.ACE_ERR_UNSUPPORTED


def test_edge_values_streaming():
    """d = 72 on the streaming engine: an all-zero row (every bit 0 without recheck), NaN and
    infinite coordinates, subnormal and huge values, a row whose squared norm overflows binary32
    and a row of one tiny value: every id equals the oracle's binary64 definition."""
    d, K, L = 72, 16, 4
    W = workloads.gaussian_w(d, K, L, 3)
    X = np.zeros((12, d), dtype=np.float32)
    X[1, :2] = [1, 1]
    X[2, 3] = np.nan
    X[3, 0] = np.inf
    X[4, 1] = -np.inf
    X[5] = 1e-39
    X[6, :3] = [3e38, -3e38, 1e38]
    X[7, 0] = 2.0**-130
    X[8] = 1.0
    X[9] = -1.0
    X[10, 5] = 1.0
    X[11, :4] = [1, 1, 2.0**-20, -(2.0**-20)]
    Xb = workloads.to_bf16_bits(np.nan_to_num(X, nan=0.0, posinf=0.0, neginf=0.0))
    Xb[2, 3], Xb[3, 0], Xb[4, 1] = 0x7FC0, 0x7F80, 0xFF80  # NaN, +inf, -inf
    det, ref = _pair(d, K, L, W=W)
    Xd = _dev(Xb)
    assert np.array_equal(ace.u32(det.hash(Xd)), ref.hash(Xb))
    _compare(det.insert_score(Xd, 1.0), ref.insert_score(Xb, 1.0))
    st = det.stats()
    assert st["nonfinite_points"] >= 4 and st["rechecks"] > 0
    assert st["precision"] == ace.ACE_PROJ_BF16


def test_highdim_full_size_sampled():
    """The high-dimensional recipe at its full size (n=1,000,000, d=1024, K=16, L=64), drawn on
    the device, in the bench's launch configuration (one insert_score call): the ids of a
    sample of 2,000 points (first and last included) against the oracle, and at full size the
    properties that tie every output to the ids (counts = per-table histograms of the ids, sums
    = gathers of the counts, Q = sum of the sums, scores = sums / L)."""
    d, K, L = 1024, 16, 64
    Xd, _ = workloads.highdim_device(seed=3, n=1_000_000)
    n = Xd.shape[0]
    det = ace.Detector(d, K, L, seed=9, precision="bf16")
    ids = ace.u32(det.hash(Xd))
    rng = np.random.default_rng(0)
    sample = np.unique(np.concatenate([rng.choice(n, size=2000, replace=False), [0, n - 1]]))
    Xs = Xd[torch.from_numpy(sample).cuda()].cpu().numpy().view(np.uint16)
    ref = oracle.Detector(d, K, L, W=det.projection())
    assert np.array_equal(ids[sample], ref.hash(Xs))
    sc, su, fl = det.insert_score(Xd, 1.0)
    torch.cuda.synchronize()
    counts = det.counts()
    assert np.all(counts.sum(axis=1, dtype=np.uint64) == n)
    for j in range(L):
        assert np.array_equal(counts[j], np.bincount(ids[:, j], minlength=1 << K)), j
    sums = ace.u32(su).astype(np.int64)
    expect = np.zeros(n, dtype=np.int64)
    for j in range(L):
        expect += counts[j][ids[:, j]]
    assert np.array_equal(sums, expect)
    assert np.array_equal(sc.cpu().numpy(), expect / L)
    st = det.stats()
    assert st["Q"] == int(sums.sum()) and st["precision"] == ace.ACE_PROJ_BF16 and st["status"] == 0
    ref.counts[:] = counts
    ref.n_ins = n
    _, _, ref_fl = ref._score_ids(ids, 1.0)
    assert np.array_equal(fl.cpu().numpy(), ref_fl)


def test_nonfinite_rows_at_high_d():
    """d = 1024: a batch mixing ordinary rows with rows holding NaN or infinities, and rows of
    one tiny coordinate (squared norm below the engine's floor): every column of such a row is
    resolved by the exact tiers; ids equal the binary64 definition."""
    d, K, L, n = 1024, 16, 8, 1500
    rng = np.random.default_rng(17)
    X = rng.standard_normal((n, d)).astype(np.float32) / 32
    X[::50, 3] = np.nan
    X[7::50, 11] = np.inf
    X[9::50, 12] = -np.inf
    X[11::50, 40], X[11::50, 41] = np.inf, -np.inf
    X[13::50] = 0.0
    X[13::50, 5] = 2.0**-40
    Xb = workloads.to_bf16_bits(np.nan_to_num(X, nan=0.0, posinf=0.0, neginf=0.0))
    Xb[::50, 3] = 0x7FC0
    Xb[7::50, 11], Xb[9::50, 12] = 0x7F80, 0xFF80
    Xb[11::50, 40], Xb[11::50, 41] = 0x7F80, 0xFF80
    det, ref = _pair(d, K, L, seed=8)
    Xd = _dev(Xb)
    assert np.array_equal(ace.u32(det.hash(Xd)), ref.hash(Xb))
    _compare(det.insert_score(Xd, 1.0), ref.insert_score(Xb, 1.0))
    assert np.array_equal(det.counts(), ref.counts)
    # every hash counts the points whose squared norm is not finite (hash, then insert_score)
    assert det.stats()["nonfinite_points"] == 2 * (4 * n // 50) and det.stats()["status"] == 0
