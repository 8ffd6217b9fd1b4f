"""The per-phase timing hook that bench.py relies on: every kernel the library launches is
counted in its phase, events bracket the launches while the hook is on, and a phase mask
limits the events to the chosen phases without changing the launch counts."""
import pytest

from paper_1706_06664_gb300 import ace, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_profile_hook_counts_and_phase_mask(precision):
    w = workloads.kdd(seed=2, n=5000)
    det = ace.Detector(w["d"], w["K"], w["L"], seed=3, precision=precision)
    Xd = torch.from_numpy(w["X"]).cuda()
    det.insert_score(Xd, 1.0)
    torch.cuda.synchronize()
    det.profile_read()

    det.profile(True)
    det.insert_score(Xd, 1.0)
    det.profile(False)
    p = det.profile_read()
    # the binary32 engine fuses the insert into its hash kernel; the tensor-core engine runs the
    # deferred-table recheck and a separate insert pass
    expect = {"hash": 1, "score": 1, "flags": 1, "other": 0,
              "recheck": 1 if precision == "bf16" else 0, "insert": 1 if precision == "bf16" else 0}
    assert {k: v["launches"] for k, v in p.items()} == expect
    assert {k: v["timed"] for k, v in p.items()} == expect
    assert all(p[k]["ms"] > 0.0 for k, n in expect.items() if n)

    det.profile(True, phases=["hash"])
    det.insert_score(Xd, 1.0)
    det.profile(False)
    p = det.profile_read()
    assert {k: v["launches"] for k, v in p.items()} == expect
    assert {k: v["timed"] for k, v in p.items()} == {k: (1 if k == "hash" else 0) for k in expect}

    det.profile(True)  # no mask: every phase again
    det.insert_score(Xd, 1.0)
    det.profile(False)
    assert {k: v["timed"] for k, v in det.profile_read().items()} == expect
    det.close()
