"""GPU parity of the E4M3 projection (ACE_PROJ_FP8; the streaming engine's kind::f8f6f4
variant) against the CPU oracle, through the C ABI.

The E4M3 path splits each bfloat16 row, scaled by a power of two 2^s chosen from its first
k-block, as X1 + X2 (+ a remainder X3 where X2 falls into E4M3's subnormal range) and each
bfloat16-valued W column as W1 + W2 (+ W3), and
accumulates the four products in binary32 on the tensor cores.  Ids, counts, sums, scores and
flags are compared bit-exactly with the oracle's binary64 definition, on the high-dimensional
recipe, on ragged shapes, on rows placed just inside and just outside the E4M3 guard band, on
rows that defeat the row scale (saturation, underflow, a zero first k-block) and on
non-finite rows."""
import math

import numpy as np
import pytest

import oracle
from paper_1706_06664_gb300 import ace, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(X):
    return torch.from_numpy(X.view(np.int16)).cuda()


def _bf16(x):
    return workloads.bf16_bits_to_f32(workloads.to_bf16_bits(np.asarray(x, dtype=np.float32))).astype(np.float64)


def e4m3(v):
    """Round to the nearest E4M3 value (ties to even), saturating at +-448 (binary64 in/out)."""
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    _, ex = np.frexp(a)
    E = np.maximum(ex - 1, -6)        # the subnormal range shares exponent -6 (quantum 2^-9)
    q = np.ldexp(1.0, E - 3)
    r = np.minimum(np.round(a / q) * q, 448.0)
    return np.where(a == 0, 0.0, np.sign(v) * r)


def split4(y):
    """The kernel's leading part of y: Veltkamp's split to four significant bits in binary32,
    c = RN((2^20 + 1) y), h = RN(c - RN(c - y))."""
    y = np.asarray(y, dtype=np.float32)
    c = (y * np.float32(1048577.0)).astype(np.float32)
    return (c - (c - y).astype(np.float32)).astype(np.float32).astype(np.float64)


def _row_scale(Xf):
    """2^s per row: the largest |x| of the first 64 coordinates to [32, 64) (s = 0 if zero)."""
    mx = np.abs(Xf[:, :64]).max(axis=1)
    _, ex = np.frexp(np.where(mx > 0, mx, 1.0))
    s = np.clip(5 - (ex - 1), -100, 100)
    return np.where(mx > 0, np.ldexp(1.0, s), 1.0)


def _row_band_fp8(W, Xf):
    """The E4M3 engine's band per row, relative to ||x|| ||w_c|| (the bound of hash_gemm.cu with
    the constants of plan_gemm_fp8, in binary64)."""
    d, KL = W.shape
    dp = (d + 63) // 64 * 64
    S8, nkb = dp // 32, dp // 64
    Wd = np.zeros((dp, KL))
    Wd[:d] = W.astype(np.float64)
    _, e = np.frexp(np.linalg.norm(Wd, axis=0))
    v = Wd * np.ldexp(1.0, -e)[None, :]
    _, fx = np.frexp(np.abs(v).max(axis=0))
    vs = v * np.ldexp(1.0, 8 - fx)[None, :]
    W1 = e4m3(vs)
    W2 = e4m3(vs - W1)
    W3 = vs - W1 - W2
    nrm = np.linalg.norm(vs, axis=0)
    w1m = (np.linalg.norm(W1, axis=0) / nrm).max()
    w2m = (np.linalg.norm(W2, axis=0) / nrm).max()
    rres = (np.linalg.norm(W3, axis=0) / nrm).max()
    blk = ((W1 / nrm[None, :]).reshape(S8, 32, KL) ** 2).sum(axis=1)
    pre = np.vstack([np.zeros((1, KL)), np.cumsum(blk, axis=0)[:-1]])
    wp, wb = pre.max(axis=1), blk.max(axis=1)
    WPk = np.sqrt(wp).reshape(nkb, 2).sum(axis=1)
    WBk = np.sqrt(wb.reshape(nkb, 2).sum(axis=1))
    sumw = (np.sqrt(wp) + np.sqrt(wb)).sum()
    Y = np.zeros((Xf.shape[0], dp))
    Y[:, :d] = Xf * _row_scale(Xf)[:, None]
    H = split4(Y)
    X1 = e4m3(H)
    X2 = e4m3(Y - H)
    X3 = Y - X1 - X2
    yk = (Y.reshape(-1, nkb, 64) ** 2).sum(axis=2)
    E = np.sqrt(np.cumsum(yk, axis=1)) @ WPk + np.sqrt(yk) @ WBk
    yu = np.linalg.norm(Y, axis=1)
    x2u, x3u = np.linalg.norm(X2, axis=1), np.linalg.norm(X3, axis=1)
    T0 = x2u * (w1m + w2m) + (yu + x2u + x3u) * w2m
    ca = 9.25 * 2.0**-23 * 1.25
    g64 = d * 2.0**-53 / (1 - d * 2.0**-53)
    B = ca * E + (rres + g64) * yu + ca * sumw * (x2u + x3u) + ca * (4 * S8 + 1) * T0 + (1 + rres) * x3u
    return B * 1.01 / yu


def _pair(d, K, L, seed=0, W=None):
    det = ace.Detector(d, K, L, seed=seed, W=W, precision="fp8", w_bf16=W is None)
    ref = oracle.Detector(d, K, L, W=det.projection())
    return det, ref


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


def test_fp8_highdim_recipe_parity():
    """High-dimensional recipe (d=1024, K=16, L=64) at n=3,000 (23 full tiles and a ragged one),
    bfloat16-valued W: ids, counts, scores, flags and statistics equal the oracle's, the E4M3
    engine (four products) did the hashing, and it deferred a small fraction of the columns."""
    w = workloads.highdim(seed=3, n=3000)
    det, ref = _pair(w["d"], w["K"], w["L"], seed=9)
    Xd = _dev(w["X"])
    assert np.array_equal(ace.u32(det.hash(Xd)), ref.hash(w["X"]))
    _compare(det.insert_score(Xd, 1.0), ref.insert_score(w["X"], 1.0))
    assert np.array_equal(det.counts(), ref.counts)
    _stats_equal(det, ref)
    st = det.stats()
    assert st["precision"] == ace.ACE_PROJ_FP8 and st["tc_products"] == 4
    assert 0 < st["deferred"] <= 3 * w["X"].shape[0], st["deferred"]


@pytest.mark.parametrize("shape", [(72, 16, 4), (128, 12, 7), (200, 20, 5), (256, 16, 17), (1024, 7, 3)])
def test_fp8_shapes_and_ragged_batches(shape):
    """Padded d (72 -> 128), K that does not divide 256, 32-bit ids (K=20), several units per
    tile (L=17 at K=16), and batches of 1, 127, 129 and 300 points in a row."""
    d, K, L = shape
    rng = np.random.default_rng(sum(shape) + 1)
    det, ref = _pair(d, K, L, seed=d * 7 + K)
    for n in (1, 127, 129, 300):
        X = workloads.to_bf16_bits(rng.standard_normal((n, d)).astype(np.float32))
        _compare(det.insert_score(_dev(X), 1.0), ref.insert_score(X, 1.0))
    assert np.array_equal(det.counts(), ref.counts)
    _stats_equal(det, ref)
    assert det.stats()["precision"] == ace.ACE_PROJ_FP8


def _near_orthogonal(W, n, rels, rng, ties_every=8, tie_rows=(7, 500)):
    """bfloat16 rows whose projection on a chosen column is rel * ||x|| ||w_c|| (cycling over
    `rels`; a callable is evaluated on the row), met by setting four coordinates with large
    |w_c| one after another; every `ties_every`-th row an exact tie (two equal rows of W)."""
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
        free = [int(t) for t in order[:12] if t not in tie_rows and t >= 64][:4]  # keep the scale
        x[free] = 0.0
        rel = rels[i % len(rels)]
        rel = rel(x) if callable(rel) else rel
        want = rel * rng.choice([-1.0, 1.0]) * np.linalg.norm(x) * np.linalg.norm(w)
        for f in free:
            r = x @ w - want
            x[f] = _bf16([-r / w[f]])[0]
        X[i] = x
    return workloads.to_bf16_bits(X.astype(np.float32))


def test_fp8_near_orthogonal_ties_and_band_edge():
    """d = 1024: rows whose projection on a chosen column is 3, 1.5 and 1.1 times the row's E4M3
    band (decided by the tensor cores: a band that is too narrow gives wrong bits here), 0.9,
    0.5, 1e-2, 1e-4 and 1e-6 times it and 1e-14 of ||x|| ||w|| (resolved exactly), and exact
    ties.  Every id equals the oracle's."""
    d, K, L, n = 1024, 16, 8, 2048
    rng = np.random.default_rng(43)
    W = _bf16(rng.standard_normal((d, K * L))).astype(np.float32)
    W[7] = W[500]

    def band(f):
        return lambda x: f * _row_band_fp8(W, x[None, :])[0]

    rels = [band(3), band(1.5), band(1.1), band(0.9), band(0.5), band(1e-2), band(1e-4), band(1e-6), 1e-14]
    X = _near_orthogonal(W, n, rels, rng)
    det, ref = _pair(d, K, L, W=W)
    Xd = _dev(X)
    ids = ace.u32(det.hash(Xd))
    assert np.array_equal(ids, ref.hash(X))
    assert not ids[7::8].any()
    _compare(det.insert_score(Xd, 1.0), ref.insert_score(X, 1.0))
    _stats_equal(det, ref)
    st = det.stats()
    assert st["precision"] == ace.ACE_PROJ_FP8 and st["rechecks"] > n // 4


def _scale_breaking_rows(n, d, rng):
    """Rows the first-k-block scale handles badly: later coordinates 2^10 .. 2^20 times the first
    block's largest (saturated to 448, the excess in X3), coordinates 2^-30 below it (E4M3
    underflow), a zero first k-block, a single coordinate, and ordinary rows between them."""
    X = rng.standard_normal((n, d)) / math.sqrt(d)
    for i in range(n):
        kind = i % 6
        if kind == 0:
            X[i, 64 + (i % (d - 64))] *= 2.0 ** (10 + i % 11)
        elif kind == 1:
            X[i, 64:] *= 2.0**-30
        elif kind == 2:
            X[i, :64] = 0.0
        elif kind == 3:
            X[i] = 0.0
            X[i, (7 * i) % d] = 2.0 ** ((i % 40) - 20)
        elif kind == 4:
            X[i, :32] *= 2.0**-12
    return workloads.to_bf16_bits(X.astype(np.float32))


def test_fp8_rows_that_defeat_the_row_scale():
    """Saturation, underflow, a zero first k-block and single-coordinate rows: wider bands or
    whole-row deferral, never a wrong bit."""
    d, K, L, n = 256, 16, 8, 600
    rng = np.random.default_rng(3)
    X = _scale_breaking_rows(n, d, rng)
    det, ref = _pair(d, K, L, seed=21)
    Xd = _dev(X)
    assert np.array_equal(ace.u32(det.hash(Xd)), ref.hash(X))
    _compare(det.insert_score(Xd, 1.0), ref.insert_score(X, 1.0))
    _stats_equal(det, ref)


def test_fp8_nonfinite_and_edge_rows():
    """d = 72: zero rows, NaN and infinite coordinates, subnormal and huge values: ids equal the
    binary64 definition and non-finite rows are counted."""
    d, K, L = 72, 16, 4
    X = np.zeros((12, d), dtype=np.float32)
    X[1, :2] = [1, 1]
    X[5] = 1e-39
    X[6, :3] = [3e38, -3e38, 1e38]
    X[7, 0] = 2.0**-130
    X[8] = 1.0
    X[9] = -1.0
    X[10, 5] = 1.0
    X[11, :4] = [1, 1, 2.0**-20, -(2.0**-20)]
    Xb = workloads.to_bf16_bits(X)
    Xb[2, 3], Xb[3, 0], Xb[4, 1] = 0x7FC0, 0x7F80, 0xFF80
    det, ref = _pair(d, K, L, seed=5)
    Xd = _dev(Xb)
    assert np.array_equal(ace.u32(det.hash(Xd)), ref.hash(Xb))
    _compare(det.insert_score(Xd, 1.0), ref.insert_score(Xb, 1.0))
    st = det.stats()
    assert st["nonfinite_points"] >= 4 and st["precision"] == ace.ACE_PROJ_FP8


def test_fp8_projection_error_within_band():
    """ace_project on the E4M3 engine: the binary32 estimate of x.w_c stays within the row's
    band (times ||w_c||) on the high-dimensional recipe and on rows with a wide exponent spread
    and cancellation inside every instruction's 32 products; the call changes no state."""
    d, K, L = 1024, 16, 8
    rng = np.random.default_rng(6)
    rows = [workloads.highdim(seed=4, n=600)["X"]]
    Xw = np.zeros((400, d))
    for i in range(400):
        e = rng.integers(0, 25, size=d)
        s = np.where(np.arange(d) % 2 == 0, 1.0, -1.0) * rng.choice([-1.0, 1.0], size=d // 32).repeat(32)
        Xw[i] = s * np.ldexp(1.0 + rng.integers(0, 128, size=d) / 128.0, -e)
        Xw[i, ::32] = s[::32]
    rows.append(workloads.to_bf16_bits(Xw.astype(np.float32)))
    for X in rows:
        det = ace.Detector(d, K, L, seed=13, precision="fp8", w_bf16=True)
        est = det.project(_dev(X)).cpu().numpy().astype(np.float64)
        W = det.projection()
        s64 = oracle.project(X, W)
        Xf = workloads.bf16_bits_to_f32(X).astype(np.float64)
        rel = np.abs(est - s64) / (np.linalg.norm(Xf, axis=1)[:, None] * np.linalg.norm(W.astype(np.float64), axis=0)[None, :])
        band = _row_band_fp8(W, Xf)
        assert (rel <= band[:, None] + 2.0**-23).all(), (rel.max(axis=1) / band).max()
        st = det.stats()
        assert st["n_ins"] == 0 and st["rechecks"] == 0 and not det.counts().any()
        ref = oracle.Detector(d, K, L, W=W)
        assert np.array_equal(ace.u32(det.hash(_dev(X))), ref.hash(X))
        det.close()


def test_fp8_refusals():
    """ACE_PROJ_FP8 needs the streaming engine and a bfloat16-valued W: a binary32 W, d <= 64 and
    binary32 input are refused with ACE_ERR_UNSUPPORTED, and nothing is counted."""
    with pytest.raises(ace.AceError) as e:
        ace.Detector(1024, 16, 4, seed=1, precision="fp8")
    assert e.value.code == ace.ACE_ERR_UNSUPPORTED
    with pytest.raises(ace.AceError) as e:
        ace.Detector(41, 15, 4, seed=1, precision="fp8", w_bf16=True)
    assert e.value.code == ace.ACE_ERR_UNSUPPORTED
    det = ace.Detector(1024, 16, 4, seed=1, precision="fp8", w_bf16=True)
    with pytest.raises(ace.AceError) as e:
        det.insert(torch.zeros((4, 1024), dtype=torch.float32, device="cuda"))
    assert e.value.code == ace.ACE_ERR_UNSUPPORTED
    assert det.stats()["n_ins"] == 0


def test_fp8_full_size_sampled():
    """The high-dimensional recipe at its full size (n=1,000,000) on the E4M3 engine, in the
    bench's launch configuration: the ids of 2,000 sampled points (first and last included)
    against the oracle, and at full size the properties that tie every output to the ids."""
    d, K, L = 1024, 16, 64
    Xd, _ = workloads.highdim_device(seed=3, n=1_000_000)
    n = Xd.shape[0]
    det = ace.Detector(d, K, L, seed=9, precision="fp8", w_bf16=True)
    ids = ace.u32(det.hash(Xd))
    rng = np.random.default_rng(1)
    sample = np.unique(np.concatenate([rng.choice(n, size=2000, replace=False), [0, n - 1]]))
    Xs = Xd[torch.from_numpy(sample).cuda()].cpu().numpy().view(np.uint16)
    ref = oracle.Detector(d, K, L, W=det.projection())
    assert np.array_equal(ids[sample], ref.hash(Xs))
    sc, su, fl = det.insert_score(Xd, 1.0)
    torch.cuda.synchronize()
    counts = det.counts()
    for j in range(L):
        assert np.array_equal(counts[j], np.bincount(ids[:, j], minlength=1 << K)), j
    sums = ace.u32(su).astype(np.int64)
    expect = np.zeros(n, dtype=np.int64)
    for j in range(L):
        expect += counts[j][ids[:, j]]
    assert np.array_equal(sums, expect)
    st = det.stats()
    assert st["precision"] == ace.ACE_PROJ_FP8 and st["status"] == 0
