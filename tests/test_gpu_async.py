"""rise_submit / rise_collect against the synchronous calls.

Two captures in flight must come back exactly as one rise_detect each, from
device or host samples; the queue has two places; and a call whose run
arrays overflow (forced here with a tiny run capacity) is run again at
collect time without disturbing the other queued call.
"""
import numpy as np
import pytest

from paper_2603_20481_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _caps():
    a = synth.make_capture(1 << 20, 20e6, 40, 91, fft_size=1024, hop=512,
                           bw_hz=(0.2e6, 3e6), dur_s=(0.5e-3, 5e-3), snr_db=(10, 25))
    b = synth.single_capture(92)
    return a, b


def _want(caps):
    from paper_2603_20481_gb300 import rise
    with rise.Detector(0) as d:
        d.set_option(rise.OPT_GRAPH, 0)
        return [d.detect(torch.from_numpy(c.iq).cuda(), 1024, 512) for c in caps]


def test_two_in_flight_match_single_calls(det):
    caps = _caps()
    want = _want(caps)
    xs = [torch.from_numpy(c.iq).cuda() for c in caps]
    for _ in range(3):                          # the third round replays graphs
        det.submit(xs[0], 1024, 512)
        det.submit(xs[1], 1024, 512)
        np.testing.assert_array_equal(det.collect(), want[0])
        np.testing.assert_array_equal(det.collect(), want[1])
    # host samples: pinned tensors and a plain numpy array
    pinned = [torch.from_numpy(c.iq).pin_memory() for c in caps]
    for src in (pinned, [c.iq for c in caps]):
        det.submit(src[0], 1024, 512)
        det.submit(src[1], 1024, 512)
        np.testing.assert_array_equal(det.collect(), want[0])
        np.testing.assert_array_equal(det.collect(), want[1])


def test_queue_limits(det):
    import ctypes
    from paper_2603_20481_gb300 import rise
    a, b = _caps()
    x = torch.from_numpy(a.iq).cuda()
    n = ctypes.c_int64(0)
    assert rise.lib().rise_collect(det._h, None, 0, ctypes.byref(n)) == rise.RISE_EINVAL
    det.submit(x, 1024, 512)
    det.submit(x, 1024, 512)
    with pytest.raises(rise.RiseError) as e:
        det.submit(x, 1024, 512)
    assert e.value.code == rise.RISE_EAGAIN
    # the synchronous calls refuse while calls are queued
    with pytest.raises(rise.RiseError):
        det.detect(x, 1024, 512)
    with pytest.raises(rise.RiseError):
        det.detect_batch([x], [1024], [512])
    a1, a2 = det.collect(), det.collect()
    np.testing.assert_array_equal(a1, a2)
    np.testing.assert_array_equal(det.detect(x, 1024, 512), a1)


def test_run_overflow_is_run_again():
    from paper_2603_20481_gb300 import rise
    caps = _caps()
    want = _want(caps)
    xs = [torch.from_numpy(c.iq).cuda() for c in caps]
    with rise.Detector(0) as d:
        d.set_option(rise.OPT_RUN_CAPACITY, 1024)
        got = d.detect(xs[0], 1024, 512)         # synchronous: relabel in place
        v = np.zeros(4, np.int64)
        rise.lib().rise_debug_export(d._h, rise.DBG_CCL, v.ctypes.data, 32)
        assert v[0] > 1024 and v[3] > v[0]       # it overflowed and grew
        np.testing.assert_array_equal(got, want[0])
    with rise.Detector(0) as d:
        d.set_option(rise.OPT_RUN_CAPACITY, 1024)
        d.submit(xs[0], 1024, 512)                 # overflows
        d.submit(xs[1], 1024, 512)                 # queued behind it
        np.testing.assert_array_equal(d.collect(), want[0])
        np.testing.assert_array_equal(d.collect(), want[1])
