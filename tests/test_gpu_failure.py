"""Failure detection without a GPU fault: the library's bounded device waits, made to run out on
events that never happen (a barrier phase that gets one of its two arrivals, a device flag that
nothing sets), give up after their limit, raise the timeout status and leave the context usable:
a detector run right after is still bit-identical to the oracle."""
import numpy as np
import pytest

import oracle
from paper_1706_06664_gb300 import ace, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _detector_still_exact():
    w = workloads.kdd(seed=31, n=3000)
    det = ace.Detector(w["d"], w["K"], w["L"], seed=4)
    ref = oracle.Detector(w["d"], w["K"], w["L"], W=det.projection())
    sc, su, fl = det.insert_score(torch.from_numpy(w["X"]).cuda(), 1.0)
    rs, ru, rf = ref.insert_score(w["X"], 1.0)
    torch.cuda.synchronize()
    assert np.array_equal(ace.u32(su), ru) and np.array_equal(fl.cpu().numpy(), rf)
    assert det.stats()["status"] == 0


@pytest.mark.parametrize("kind", [0, 1])
def test_bounded_wait_gives_up_and_context_survives(kind):
    limit = 20_000_000  # about 10 ms of SM cycles
    r = ace.wait_probe(kind, limit)
    assert r["status"] & ace.ACE_STATUS_TIMEOUT
    assert limit <= r["cycles"] < 50 * limit
    if kind == 0:
        assert r["aborted_cycles"] < limit // 10  # the abort flag ends a wait at once
    _detector_still_exact()


def test_wait_probe_arguments():
    for kind, limit in ((2, 10**6), (0, 10), (1, 10**10)):
        with pytest.raises(ace.AceError) as e:
            ace.wait_probe(kind, limit)
        assert e.value.code == ace.ACE_ERR_ARG
