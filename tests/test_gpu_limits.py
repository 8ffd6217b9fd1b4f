"""Shapes at the library's limits, against the oracle: the widest projection the ABI accepts
(K L = 65,536 columns: 4,096 tables of 2^16 counts, 1 GiB of count arrays), the widest ids
(K = 24), a long row (d = 4,096) on every engine that takes it, and one-point and one-column
degenerate shapes."""
import numpy as np
import pytest

import oracle
from paper_1706_06664_gb300 import ace, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(X):
    return torch.from_numpy(X.view(np.int16) if X.dtype == np.uint16 else X).cuda()


def _run(det, ref, X):
    sc, su, fl = det.insert_score(_dev(X), 1.0)
    rs, ru, rf = ref.insert_score(X, 1.0)
    torch.cuda.synchronize()
    assert np.array_equal(ace.u32(su), ru)
    assert np.array_equal(sc.cpu().numpy(), rs) and np.array_equal(fl.cpu().numpy(), rf)
    s, r = det.stats(), ref.stats()
    for k in ("n_ins", "n_scored", "Q", "S1", "S2", "mu_ins", "mu", "sigma"):
        assert s[k] == r[k], k


def test_widest_projection():
    """K L = 65,536 (the ABI's limit): every id, count and score equals the oracle's; a wider
    shape is refused."""
    d, K, L = 8, 16, 4096
    det = ace.Detector(d, K, L, seed=3)
    ref = oracle.Detector(d, K, L, W=det.projection())
    rng = np.random.default_rng(1)
    for n in (1, 300):
        _run(det, ref, rng.standard_normal((n, d)).astype(np.float32))
    assert np.array_equal(det.counts(), ref.counts)
    det.close()
    with pytest.raises(ace.AceError):
        ace.Detector(d, 16, 4097, seed=3)


@pytest.mark.parametrize("precision", ["fp32", "auto"])
def test_long_rows(precision):
    """d = 4,096 bfloat16 rows (the streaming tensor-core engine under auto, the binary32 one
    under fp32), several tiles and a ragged tail."""
    d, K, L = 4096, 12, 10
    det = ace.Detector(d, K, L, seed=5, precision=precision)
    ref = oracle.Detector(d, K, L, W=det.projection())
    rng = np.random.default_rng(2)
    for n in (1, 129, 300):
        _run(det, ref, workloads.to_bf16_bits(rng.standard_normal((n, d)).astype(np.float32)))
    assert np.array_equal(det.counts(), ref.counts)


@pytest.mark.parametrize("shape", [(1, 24, 3), (2, 1, 1), (97, 24, 1)])
def test_degenerate_and_widest_ids(shape):
    """One coordinate, one column, one table, and 24-bit ids (32-bit id storage)."""
    d, K, L = shape
    for precision in ("fp32", "auto"):
        det = ace.Detector(d, K, L, seed=d + K, precision=precision)
        ref = oracle.Detector(d, K, L, W=det.projection())
        rng = np.random.default_rng(d)
        for n in (1, 2, 1000):
            _run(det, ref, rng.standard_normal((n, d)).astype(np.float32))
        assert np.array_equal(det.counts(), ref.counts)
