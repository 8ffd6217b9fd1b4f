"""The structured engine (ACE_W_HADAMARD, ACE_PROJ_FWHT: fast Walsh-Hadamard transforms)
against the oracle run with the explicit +-1 W of its own generator: ids, counts, scores,
flags and statistics bit for bit, on ragged shapes (padding, several blocks, 32-bit ids), on
exact ties and near-ties of the transform, and on non-finite rows."""
import math

import numpy as np
import pytest

import oracle
from paper_1706_06664_gb300 import ace, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pair(d, K, L, seed, precision="auto"):
    det = ace.Detector(d, K, L, seed=seed, precision=precision, w_hadamard=True)
    W = oracle.projection_from_seed(d, K, L, seed, hadamard=True)
    assert np.array_equal(det.projection(), W)
    return det, oracle.Detector(d, K, L, W=W)


def _dev(X):
    return torch.from_numpy(X.view(np.int16) if X.dtype == np.uint16 else X).cuda()


def _check(det, ref, X):
    Xd = _dev(X)
    assert np.array_equal(ace.u32(det.hash(Xd)), ref.hash(X))
    sc, su, fl = det.insert_score(Xd, 1.0)
    rs, ru, rf = ref.insert_score(X, 1.0)
    torch.cuda.synchronize()
    assert np.array_equal(ace.u32(su), ru)
    assert np.array_equal(sc.cpu().numpy(), rs) and np.array_equal(fl.cpu().numpy(), rf)
    assert np.array_equal(det.counts(), ref.counts)
    s, r = det.stats(), ref.stats()
    for k in ("n_ins", "n_scored", "Q", "S1", "S2", "mu_ins", "mu", "sigma"):
        assert s[k] == r[k], k


@pytest.mark.parametrize("shape", [(32, 10, 20), (41, 15, 50), (100, 12, 7), (256, 20, 8), (520, 16, 8), (1001, 12, 10),
                                   (1024, 16, 64)])
def test_structured_engine_parity(shape):
    d, K, L = shape
    det, ref = _pair(d, K, L, seed=d * 3 + K)
    rng = np.random.default_rng(d)
    for n in (1, 255, 2000):
        X = rng.standard_normal((n, d)).astype(np.float32)
        _check(det, ref, X)
    assert det.stats()["precision"] == ace.ACE_PROJ_FWHT


def test_structured_engine_kdd_and_bf16():
    w = workloads.kdd(seed=9, n=20000)
    det, ref = _pair(w["d"], w["K"], w["L"], seed=5)
    _check(det, ref, w["X"])
    h = workloads.highdim(seed=4, n=3000)
    det, ref = _pair(h["d"], h["K"], h["L"], seed=6)
    _check(det, ref, h["X"])
    assert det.stats()["precision"] == ace.ACE_PROJ_FWHT


def test_structured_engine_ties_and_edges():
    """Rows that put transform outputs exactly at 0 (x_a = x_b with H rows that cancel them),
    outputs near 0 relative to the rounding bound, zero rows, and NaN / infinite coordinates:
    every bit is the binary64 definition's."""
    d, K, L = 64, 16, 8
    det, ref = _pair(d, K, L, seed=11)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((400, d)).astype(np.float32)
    X[::5] = 0.0
    X[::5, 3] = 1.0
    X[::5, 5] = 1.0                   # two equal coordinates: half of the outputs are exactly 0
    X[1::7] = np.float32(2.0**-10)    # constant rows: only the outputs of the first Hadamard row differ from 0
    X[2::11] *= np.float32(1e-30)     # tiny values
    X[3::13, 7] = np.nan
    X[4::17, 9] = np.inf
    # two equal large coordinates over tiny ones (an exponent range of 40 binades): the outputs
    # where the large ones cancel lie inside the bound, and the range is too wide for the warp's
    # split binary64 sum, so each is evaluated in index order
    X[6::19] = np.float32(2.0**-40) * np.sign(rng.standard_normal((len(X[6::19]), d))).astype(np.float32)
    X[6::19, 2] = 1.0
    X[6::19, 10] = 1.0
    _check(det, ref, X)
    assert det.stats()["rechecks"] > 0


def test_structured_engine_refusals_and_other_engines():
    """ACE_PROJ_FWHT needs ACE_W_HADAMARD; the stored W of a structured detector gives the same
    ids on the SIMT and tensor-core engines."""
    with pytest.raises(ace.AceError) as e:
        ace.Detector(64, 16, 4, seed=1, precision="fwht")
    assert e.value.code == ace.ACE_ERR_UNSUPPORTED
    d, K, L = 64, 16, 8
    X = np.random.default_rng(1).standard_normal((500, d)).astype(np.float32)
    ids = {}
    for prec in ("fwht", "fp32", "bf16"):
        det = ace.Detector(d, K, L, seed=2, precision=prec, w_hadamard=True)
        ids[prec] = ace.u32(det.hash(_dev(X)))
    assert np.array_equal(ids["fwht"], ids["fp32"]) and np.array_equal(ids["fwht"], ids["bf16"])


def test_structured_engine_full_size_sampled():
    """The high-dimensional shape at its full size (n = 1,000,000 bfloat16 points drawn on the
    device, d = 1024, K = 16, L = 64) in the bench's launch configuration (one insert_score call
    on the structured engine): the ids of 2,000 sampled points (first and last included) against the
    oracle, and at full size the properties that tie every output to the ids."""
    d, K, L = 1024, 16, 64
    Xd, _ = workloads.highdim_device(seed=3, n=1_000_000)
    n = Xd.shape[0]
    det = ace.Detector(d, K, L, seed=9, w_hadamard=True)
    ids = ace.u32(det.hash(Xd))
    rng = np.random.default_rng(1)
    sample = np.unique(np.concatenate([rng.choice(n, size=2000, replace=False), [0, n - 1]]))
    Xs = Xd[torch.from_numpy(sample).cuda()].cpu().numpy().view(np.uint16)
    ref = oracle.Detector(d, K, L, W=oracle.projection_from_seed(d, K, L, 9, hadamard=True))
    assert np.array_equal(ids[sample], ref.hash(Xs))
    sc, su, fl = det.insert_score(Xd, 1.0)
    torch.cuda.synchronize()
    counts = det.counts()
    for j in range(L):
        assert np.array_equal(counts[j], np.bincount(ids[:, j], minlength=1 << K)), j
    expect = np.zeros(n, dtype=np.int64)
    for j in range(L):
        expect += counts[j][ids[:, j]]
    assert np.array_equal(ace.u32(su).astype(np.int64), expect)
    assert np.array_equal(sc.cpu().numpy(), expect / L)
    st = det.stats()
    assert st["precision"] == ace.ACE_PROJ_FWHT and st["status"] == 0 and st["rechecks"] > 0
    ref.counts[:] = counts
    ref.n_ins = n
    _, _, ref_fl = ref._score_ids(ids, 1.0)
    assert np.array_equal(fl.cpu().numpy(), ref_fl)
