"""Checkpoint round trip (ace_save / ace_load) through the C ABI: a detector saved after some
batches and restored into a new handle gives exactly the results of the uninterrupted one, and
both equal the oracle's run of the same batches."""
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


def _outs(t):
    sc, su, fl = t
    torch.cuda.synchronize()
    return sc.cpu().numpy(), ace.u32(su), fl.cpu().numpy()


@pytest.mark.parametrize("case", ["kdd", "highdim", "highdim_wbf16"])
def test_save_load_continues_exactly(case):
    if case == "kdd":
        w = workloads.kdd(seed=21, n=30_000)
        kw = {}
    else:
        w = workloads.highdim(seed=22, n=6_000)
        kw = {"w_bf16": case == "highdim_wbf16"}
    X = w["X"]
    A, B, C = X[: len(X) // 2], X[len(X) // 2: 5 * len(X) // 6], X[5 * len(X) // 6:]
    d, K, L = w["d"], w["K"], w["L"] if case == "kdd" else 16
    det = ace.Detector(d, K, L, seed=5, **kw)
    ref = oracle.Detector(d, K, L, W=det.projection())
    det.insert_score(_dev(A), 1.0)
    ref.insert_score(A, 1.0)
    blob = det.save()
    det2 = ace.Detector.load(blob)
    assert np.array_equal(det2.projection(), det.projection())
    assert np.array_equal(det2.counts(), det.counts())
    for k in ("n_ins", "n_scored", "Q", "S1", "S2", "mu", "sigma", "mu_ins"):
        assert det2.stats()[k] == det.stats()[k], k
    for D in (det, det2):
        o1 = _outs(D.insert_score(_dev(B), 1.0))
        o2 = _outs(D.score(_dev(C), 2.0))
        r1 = ref.insert_score(B, 1.0) if D is det else r1
        r2 = ref.score(C, 2.0) if D is det else r2
        for a, b in zip(o1 + o2, r1 + r2):
            assert np.array_equal(a, b)
    assert np.array_equal(det.counts(), det2.counts()) and np.array_equal(det.counts(), ref.counts)
    s1, s2, sr = det.stats(), det2.stats(), ref.stats(2.0)
    for k in ("n_ins", "n_scored", "Q", "S1", "S2", "mu", "sigma", "mu_ins"):
        assert s1[k] == s2[k] == sr[k], k


def test_load_rejects_damaged_blobs():
    det = ace.Detector(16, 8, 4, seed=1)
    det.insert(torch.randn(100, 16, device="cuda"))
    blob = bytearray(det.save())
    for bad in (bytes(blob[:-1]), b"NOTACE01" + bytes(blob[8:])):
        with pytest.raises(ace.AceError) as e:
            ace.Detector.load(bad)
        assert e.value.code == ace.ACE_ERR_ARG
    blob[200] ^= 0x40  # one bit of W
    with pytest.raises(ace.AceError) as e:
        ace.Detector.load(bytes(blob))
    assert e.value.code == ace.ACE_ERR_ARG and "checksum" in str(e.value)
