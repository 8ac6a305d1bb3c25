"""Failure detection without a GPU fault: every device wait in the library is
bounded, reports FRAG_ETIMEOUT through the error word and leaves the context
usable.  The wait is made to run out on purpose by waiting on a counter that
nothing increments (no trap, no bad address, no endless loop)."""
import numpy as np
import pytest

import oracle
from paper_1803_04880_b300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fr():
    import paper_1803_04880_b300 as m
    m.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return m


def test_bounded_wait_reports_timeout_and_context_survives(fr):
    fr.sync_status()  # clean error word
    fr.check_wait_timeout(polls=2000)
    with pytest.raises(fr.FragError) as ei:
        fr.sync_status()
    assert ei.value.status == fr.FRAG_ETIMEOUT
    # the word is cleared and the context still runs the hot path exactly
    fr.sync_status()
    data = wl.random_bytes(70000, 3)
    key = fr.Key(wl.KEY)
    plan = fr.Plan(512, 3)
    d = torch.from_numpy(data).cuda()
    priv, pub = fr.protect(plan, key, 1, d)
    out = fr.recover(plan, key, 1, priv, pub, data.size)
    fr.sync_status()
    p_ref, u_ref = oracle.protect(data, 512, 3, wl.KEY, 1)
    assert np.array_equal(priv.cpu().numpy(), p_ref)
    assert np.array_equal(pub.cpu().numpy(), u_ref)
    assert np.array_equal(out.cpu().numpy(), data)


def test_timeout_on_a_side_stream_is_reported_there(fr):
    s = torch.cuda.Stream()
    fr.check_wait_timeout(polls=500, stream=s)
    with pytest.raises(fr.FragError) as ei:
        fr.sync_status(s)
    assert ei.value.status == fr.FRAG_ETIMEOUT
    fr.sync_status()


def test_box_load_wait_reports_timeout_and_context_survives(fr):
    """The fused kernel's wait for a TMA box load, on a barrier armed for
    bytes no copy delivers: it runs out, reports FRAG_ETIMEOUT with its own
    message, and a recover that loads its level-1 bands as boxes (one
    buffer, 2 levels, width 1024) still matches the oracle afterwards."""
    fr.sync_status()
    fr.check_box_wait_timeout(polls=1000)
    with pytest.raises(fr.FragError) as ei:
        fr.sync_status()
    assert ei.value.status == fr.FRAG_ETIMEOUT
    assert "TMA box" in str(ei.value)
    fr.sync_status()
    data = wl.random_bytes(1024 * 64, 9)
    key = fr.Key(wl.KEY)
    plan = fr.Plan(1024, 2)
    d = torch.from_numpy(data).cuda()
    priv, pub = fr.protect(plan, key, 2, d)
    out = fr.recover(plan, key, 2, priv, pub, data.size)
    fr.sync_status()
    p_ref, u_ref = oracle.protect(data, 1024, 2, wl.KEY, 2)
    assert np.array_equal(priv.cpu().numpy(), p_ref)
    assert np.array_equal(pub.cpu().numpy(), u_ref)
    assert np.array_equal(out.cpu().numpy(), data)
