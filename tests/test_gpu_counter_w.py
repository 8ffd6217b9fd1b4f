"""Detectors whose W is regenerated from the seed (ACE_W_COUNTER): the library's W equals the
oracle's integer-only generator, and every engine's outputs equal the oracle's run with the
oracle's own W (so the kernels' regeneration of W tiles is checked bit for bit, not only the
stored copy)."""
import numpy as np
import pytest

import oracle
from paper_1706_06664_gb300 import ace, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pair(d, K, L, seed, precision):
    det = ace.Detector(d, K, L, seed=seed, precision=precision, w_counter=True)
    W = oracle.projection_from_seed(d, K, L, seed, counter=True)
    assert np.array_equal(det.projection(), W)
    return det, oracle.Detector(d, K, L, W=W)


def _check(det, ref, X, Xd):
    sc, su, fl = det.insert_score(Xd, 1.0)
    rs, ru, rf = ref.insert_score(X, 1.0)
    torch.cuda.synchronize()
    assert np.array_equal(ace.u32(su), ru)
    assert np.array_equal(sc.cpu().numpy(), rs) and np.array_equal(fl.cpu().numpy(), rf)
    assert np.array_equal(det.counts(), ref.counts)
    s, r = det.stats(), ref.stats()
    for k in ("n_ins", "n_scored", "Q", "S1", "S2", "mu_ins", "mu", "sigma"):
        assert s[k] == r[k], k


@pytest.mark.parametrize("shape", [(32, 10, 20), (41, 15, 50), (200, 12, 7), (1024, 16, 8)])
def test_simt_engine_regenerates_w(shape):
    """The binary32 engine reads no W: its tiles are regenerated from the seed in the kernel."""
    d, K, L = shape
    det, ref = _pair(d, K, L, seed=d + K, precision="fp32")
    rng = np.random.default_rng(d)
    for n in (1, 257, 3000):
        X = rng.standard_normal((n, d)).astype(np.float32)
        _check(det, ref, X, torch.from_numpy(X).cuda())
    assert det.stats()["precision"] == ace.ACE_PROJ_FP32


def test_tensor_core_engines_with_counter_w():
    """The resident engine (d = 41) and the streaming engine (d = 1024, one bfloat16 product:
    the entries are bfloat16 values; and E4M3) use the materialised copy: same results."""
    w = workloads.kdd(seed=5, n=20000)
    det, ref = _pair(w["d"], w["K"], w["L"], seed=3, precision="bf16")
    _check(det, ref, w["X"], torch.from_numpy(w["X"]).cuda())
    assert det.stats()["tc_products"] == 3
    h = workloads.highdim(seed=6, n=2000)
    for prec, products in (("bf16", 1), ("fp8", 4)):
        det, ref = _pair(h["d"], h["K"], h["L"], seed=4, precision=prec)
        _check(det, ref, h["X"], torch.from_numpy(h["X"].view(np.int16)).cuda())
        assert det.stats()["tc_products"] == products


def test_batch_with_counter_w():
    """A batch mixing regenerated and stored W: each detector equals the oracle's run of it."""
    K, L = 12, 32
    specs = workloads.batched_specs(seed=15, n_det=12, d_range=(16, 300), n_range=(1, 4000))
    dets, refs = [], []
    for g, (d, n, sd) in enumerate(specs):
        if g % 2:
            dt, rf = _pair(d, K, L, seed=sd, precision="fp32")
        else:
            dt = ace.Detector(d, K, L, seed=sd, precision="fp32")
            rf = oracle.Detector(d, K, L, W=dt.projection())
        dets.append(dt)
        refs.append(rf)
    Xs = [workloads.batched_points(d, n, sd) for (d, n, sd) in specs]
    sc, su, fl = ace.batch_insert_score(dets, [torch.from_numpy(X).cuda() for X in Xs])
    torch.cuda.synchronize()
    for g, (det, ref, X) in enumerate(zip(dets, refs, Xs)):
        rs, ru, rf = ref.insert_score(X, 1.0)
        assert np.array_equal(ace.u32(su[g]), ru), g
        assert np.array_equal(sc[g].cpu().numpy(), rs) and np.array_equal(fl[g].cpu().numpy(), rf), g
        assert np.array_equal(det.counts(), ref.counts), g


def test_counter_w_checkpoint_and_unknown_flags():
    """A saved detector with regenerated W loads with the same W stored and continues
    identically; an unknown creation flag is refused."""
    d, K, L = 64, 12, 10
    det, ref = _pair(d, K, L, seed=8, precision="fp32")
    rng = np.random.default_rng(2)
    X1 = rng.standard_normal((500, d)).astype(np.float32)
    X2 = rng.standard_normal((300, d)).astype(np.float32)
    _check(det, ref, X1, torch.from_numpy(X1).cuda())
    det2 = ace.Detector.load(det.save())
    det2.set_precision("fp32")
    assert np.array_equal(det2.projection(), det.projection())
    _check(det2, ref, X2, torch.from_numpy(X2).cuda())
    import ctypes
    h = ctypes.c_void_p()
    rc = ace.load_library().ace_create_ex(d, K, L, ctypes.c_uint64(1), 0x8, ctypes.byref(h))
    assert rc == ace.ACE_ERR_ARG and not h.value
