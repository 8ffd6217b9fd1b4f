"""Many detectors in one set of launches (ace_batch_insert_score): every detector's scores,
sums, flags, counts and statistics equal the oracle's run of that detector alone."""
import numpy as np
import pytest

import oracle
from paper_1706_06664_gb300 import ace, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _batch_points(specs, salt):
    out = []
    for (d, n, sd) in specs:
        X = workloads.batched_points(d, n, sd + salt) if n > 0 else np.zeros((0, d), dtype=np.float32)
        out.append(X)
    return out


def _check(dets, refs, Xs, res):
    sc, su, fl = res
    torch.cuda.synchronize()
    for g, (det, ref, X) in enumerate(zip(dets, refs, Xs)):
        rs, ru, rf = ref.insert_score(X, 1.0)
        assert np.array_equal(ace.u32(su[g]), ru), g
        assert np.array_equal(sc[g].cpu().numpy(), rs) and np.array_equal(fl[g].cpu().numpy(), rf), g
        assert np.array_equal(det.counts(), ref.counts), g
        s, r = det.stats(), ref.stats()
        for k in ("n_ins", "n_scored", "Q", "S1", "S2", "mu_ins", "mu", "sigma"):
            assert s[k] == r[k], (g, k)


@pytest.mark.parametrize("K,L", [(12, 32), (18, 6)])
def test_batch_matches_each_detector_alone(K, L):
    specs = workloads.batched_specs(seed=5, n_det=24, d_range=(16, 160), n_range=(1, 3000))
    specs[3] = (specs[3][0], 0, specs[3][2])   # an empty detector
    specs[7] = (specs[7][0], 1, specs[7][2])   # a single point
    dets = [ace.Detector(d, K, L, seed=sd) for (d, n, sd) in specs]
    refs = [oracle.Detector(d, K, L, W=det.projection()) for (d, n, sd), det in zip(specs, dets)]
    for salt in (0, 1):  # two batches: the statistics carry over
        Xs = _batch_points(specs, salt)
        res = ace.batch_insert_score(dets, [torch.from_numpy(X).cuda() for X in Xs])
        _check(dets, refs, Xs, res)


def test_batch_at_bench_shapes():
    """The bench's shape range: 34 detectors with K=12, L=32, d log-uniform in [16, 512] and n
    log-uniform in [100, 100,000], plus both extremes (d=512 with n=100,000; d=16 with n=100):
    each detector's outputs, counts and statistics equal the oracle's run of it alone."""
    K, L = 12, 32
    specs = workloads.batched_specs(seed=9, n_det=32, d_range=(16, 512), n_range=(100, 100_000))
    specs += [(512, 100_000, 77), (16, 100, 78)]
    dets = [ace.Detector(d, K, L, seed=sd) for (d, n, sd) in specs]
    refs = [oracle.Detector(d, K, L, W=det.projection()) for (d, n, sd), det in zip(specs, dets)]
    Xs = _batch_points(specs, 0)
    res = ace.batch_insert_score(dets, [torch.from_numpy(X).cuda() for X in Xs])
    _check(dets, refs, Xs, res)


def test_batch_tiles_are_autotuned_and_every_tile_is_exact():
    """The autotuner records a tile per shape class met by a batch (points and columns per block
    in {64, 128}); and each of the four tiles, forced through single-shape batches of ragged
    sizes, gives the oracle's results (the tuner may pick any of them)."""
    K, L = 12, 32
    specs = [(200, 5000, 11), (40, 3000, 12), (512, 2500, 13)]
    dets = [ace.Detector(d, K, L, seed=sd) for (d, n, sd) in specs]
    refs = [oracle.Detector(d, K, L, W=det.projection()) for (d, n, sd), det in zip(specs, dets)]
    Xs = _batch_points(specs, 3)
    _check(dets, refs, Xs, ace.batch_insert_score(dets, [torch.from_numpy(X).cuda() for X in Xs]))
    for (d, n, sd) in specs:
        p, c = ace.batch_tile(d, K, L)
        assert p in (64, 128) and c in (64, 128), (d, p, c)
    assert ace.batch_tile(7777, K, L) == (0, 0)


def test_batch_rejects_duplicates_and_mixed_k():
    a = ace.Detector(20, 12, 8, seed=1)
    b = ace.Detector(20, 18, 4, seed=2)
    X = torch.zeros((5, 20), dtype=torch.float32, device="cuda")
    with pytest.raises(ace.AceError) as e:
        ace.batch_insert_score([a, a], [X, X])
    assert e.value.code == ace.ACE_ERR_ARG
    with pytest.raises(ace.AceError) as e:
        ace.batch_insert_score([a, b], [X, X])
    assert e.value.code == ace.ACE_ERR_ARG
    assert a.stats()["n_ins"] == 0 and b.stats()["n_ins"] == 0
