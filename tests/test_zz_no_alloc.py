"""The allocation-free entry point, ace_insert_score_noalloc, against ace_insert_score.

Some callers cannot call cudaMalloc (their device memory is held by another allocator, or
they must never block on the device-wide synchronisation a cudaFree implies); for them the
library keeps its scratch in one static device array.  This file is named so pytest
collects it last; it passes alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_1706_06664_gb300 import ace, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _call_noalloc(lib, det, X, alpha, sc, su, fl):
    dt = ace.ACE_F32 if X.dtype == torch.float32 else ace.ACE_BF16
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.ace_insert_score_noalloc(det._h, ctypes.c_void_p(X.data_ptr()), X.shape[0], dt, float(alpha),
                                        ctypes.c_void_p(sc.data_ptr()), ctypes.c_void_p(su.data_ptr()),
                                        ctypes.c_void_p(fl.data_ptr()), stream)


def test_noalloc_matches_insert_score_on_two_calls():
    lib = ace.load_library()
    w1 = workloads.kdd(seed=31, n=50_003)
    w2 = workloads.kdd(seed=32, n=20_000)
    d, K, L = w1["d"], w1["K"], w1["L"]
    ref = ace.Detector(d, K, L, seed=99, precision="fp32")
    new = ace.Detector(d, K, L, seed=99, precision="fp32")
    for w in (w1, w2):
        X = torch.from_numpy(w["X"]).cuda()
        n = X.shape[0]
        rs, ru, rf = ref.insert_score(X, 1.0)
        sc = torch.empty(n, dtype=torch.float64, device="cuda")
        su = torch.empty(n, dtype=torch.int32, device="cuda")
        fl = torch.empty(n, dtype=torch.uint8, device="cuda")
        assert _call_noalloc(lib, new, X, 1.0, sc, su, fl) == ace.ACE_OK, lib.ace_last_error()
        torch.cuda.synchronize()
        # the library's parity bar: integer outputs and binary64 scores bit-exact
        assert torch.equal(su, ru)
        assert torch.equal(sc, rs)
        assert torch.equal(fl, rf)
    assert np.array_equal(new.counts(), ref.counts())
    a, b = new.stats(), ref.stats()
    for k in ("n_ins", "n_scored", "Q", "S1", "S2", "mu", "sigma", "mu_ins"):
        assert a[k] == b[k], k


def test_noalloc_without_sums_output_and_bf16_input():
    w = workloads.highdim(seed=33, n=3000)
    d, K, L = w["d"], w["K"], w["L"]
    X = torch.from_numpy(w["X"].view(np.int16)).cuda()
    ref = ace.Detector(d, K, L, seed=7, precision="fp32")
    new = ace.Detector(d, K, L, seed=7, precision="fp32")
    rs, _, rf = ref.insert_score(X, 0.5, sums=False)
    sc, _, fl = new.insert_score_noalloc(X, 0.5, sums=False)
    torch.cuda.synchronize()
    assert torch.equal(sc, rs) and torch.equal(fl, rf)


def test_noalloc_rejects_batches_beyond_the_static_scratch():
    lib = ace.load_library()
    d, K, L = 4, 16, 64  # 128 bytes of ids per point
    det = ace.Detector(d, K, L, seed=1)
    n = ace.NOALLOC_SCRATCH_BYTES // (L * 2) + 1
    X = torch.zeros((n, d), dtype=torch.float32, device="cuda")
    sc = torch.empty(n, dtype=torch.float64, device="cuda")
    su = torch.empty(n, dtype=torch.int32, device="cuda")
    fl = torch.empty(n, dtype=torch.uint8, device="cuda")
    assert _call_noalloc(lib, det, X, 1.0, sc, su, fl) == ace.ACE_ERR_ARG
    assert b"static scratch" in lib.ace_last_error()
    st = det.stats()
    assert st["n_ins"] == 0 and st["n_scored"] == 0 and int(det.counts().sum()) == 0


def test_noalloc_at_the_exact_limit_without_sums_and_one_past_it():
    """A batch whose scratch need equals ACE_NOALLOC_SCRATCH_BYTES exactly (K=16, L=62: 124 bytes
    of ids and 4 of sums per point, 2^18 points, no sums buffer, so the sums sit at the very end
    of the static array) runs and matches ace_insert_score bit for bit; one point more is
    refused and changes nothing."""
    lib = ace.load_library()
    d, K, L = 8, 16, 62
    n = ace.NOALLOC_SCRATCH_BYTES // (L * 2 + 4)
    assert n * (L * 2 + 4) == ace.NOALLOC_SCRATCH_BYTES and (n * L * 2) % 256 == 0
    rng = np.random.default_rng(3)
    X = torch.from_numpy(rng.standard_normal((n + 1, d)).astype(np.float32)).cuda()
    ref = ace.Detector(d, K, L, seed=5, precision="fp32")
    new = ace.Detector(d, K, L, seed=5, precision="fp32")
    rs, _, rf = ref.insert_score(X[:n], 1.0, sums=False)
    sc, _, fl = new.insert_score_noalloc(X[:n], 1.0, sums=False)
    torch.cuda.synchronize()
    assert torch.equal(sc, rs) and torch.equal(fl, rf)
    assert np.array_equal(new.counts(), ref.counts())
    with pytest.raises(ace.AceError) as e:
        new.insert_score_noalloc(X, 1.0, sums=False)
    assert e.value.code == ace.ACE_ERR_ARG
    assert new.stats()["n_ins"] == n


def test_noalloc_wide_ids_k_above_16():
    """K > 16 (4-byte ids) through the allocation-free entry point, twice in a row, against
    ace_insert_score: scores, sums and flags bit for bit."""
    d, K, L = 24, 20, 8
    rng = np.random.default_rng(4)
    ref = ace.Detector(d, K, L, seed=6, precision="fp32")
    new = ace.Detector(d, K, L, seed=6, precision="fp32")
    for n in (10_000, 3_001):
        X = torch.from_numpy(rng.standard_normal((n, d)).astype(np.float32)).cuda()
        rs, ru, rf = ref.insert_score(X, 1.0)
        sc, su, fl = new.insert_score_noalloc(X, 1.0)
        torch.cuda.synchronize()
        assert torch.equal(su, ru) and torch.equal(sc, rs) and torch.equal(fl, rf)
    a, b = new.stats(), ref.stats()
    for k in ("n_ins", "n_scored", "Q", "S1", "S2", "mu", "sigma"):
        assert a[k] == b[k], k


def test_noalloc_launches_are_timed_by_the_profiling_hook():
    """With the timing hook on, the entry point's three kernels are counted and timed like
    ace_insert_score's."""
    d, K, L = 16, 12, 8
    det = ace.Detector(d, K, L, seed=2, precision="fp32")
    X = torch.from_numpy(np.random.default_rng(5).standard_normal((5000, d)).astype(np.float32)).cuda()
    det.profile_read()
    det.profile(True)
    det.insert_score_noalloc(X, 1.0)
    det.profile(False)
    p = det.profile_read()
    for ph in ("hash", "score", "flags"):
        assert p[ph]["launches"] == 1 and p[ph]["timed"] == 1 and p[ph]["ms"] > 0.0, (ph, p[ph])
