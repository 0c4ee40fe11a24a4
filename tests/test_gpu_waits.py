"""Bounded device waits run out without harm.

Every wait of the labelling stage has a bound: a single-pass scan tile polls
its predecessors' published sums at most RISE_OPT_SCAN_WAIT_LIMIT times, and
a union-find walk takes at most RISE_OPT_UNION_LIMIT steps.  When a bound is
reached the kernel records it in the call's status and returns, so the call
ends with RISE_ETIMEOUT, no GPU fault or hang occurs, and the next call on
the same context returns the usual boxes.  The scan case is forced with the
test-only RISE_OPT_TEST_WITHHOLD (one tile of the box-slot scan publishes
nothing, so every later tile's wait runs out after a short limit); the
union-find case with a limit of one step on a mask whose components are
chains of 61 runs.  Every index a timed-out kernel touches stays in range:
the box-slot scan bounds its writes by the run and box counts, and a walk
that gives up returns an ancestor, which is a valid run.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_20481_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _stripes(T, F, seed):
    # 3-wide vertical stripes 3 apart, cut every 64 rows: tens of thousands of
    # runs (many box-slot scan tiles), components 61 runs tall
    rng = np.random.default_rng(seed)
    q = np.full((T, F), 50, np.uint8)
    cols = (np.arange(F) % 6) < 3
    rows = (np.arange(T) % 64) < 61
    q[np.ix_(rows, cols)] = rng.integers(200, 256, size=(rows.sum(), cols.sum()))
    return q


def _thr():
    from paper_2603_20481_gb300 import rise
    kw = dict(psd_offset_db=-math.inf, power_offset_db=-math.inf)
    return rise.default_thresholds(**kw), oracle.params(**kw)


def test_scan_wait_runs_out_and_the_context_recovers():
    from paper_2603_20481_gb300 import rise
    q = _stripes(512, 1024, 3)
    thr_g, thr_r = _thr()
    want = oracle.detect_image(q, thr_r)
    img = torch.from_numpy(q).cuda()
    with rise.Detector(0) as d:
        np.testing.assert_array_equal(d.detect_image(img, thr_g), want)
        runs = int(d.debug(rise.DBG_CCL, 0, 0)[0])
        assert runs > 4 * 2048                         # several box-slot scan tiles
        d.set_option(rise.OPT_SCAN_WAIT_LIMIT, 64)
        d.set_option(rise.OPT_TEST_WITHHOLD, 0)
        for _ in range(2):
            with pytest.raises(rise.RiseError) as e:
                d.detect_image(img, thr_g)
            assert e.value.code == rise.RISE_ETIMEOUT
        d.set_option(rise.OPT_TEST_WITHHOLD, -1)
        d.set_option(rise.OPT_SCAN_WAIT_LIMIT, 0)      # back to the default bound
        for _ in range(2):
            np.testing.assert_array_equal(d.detect_image(img, thr_g), want)


def test_union_walk_limit_runs_out_and_the_context_recovers():
    from paper_2603_20481_gb300 import rise
    q = _stripes(512, 1024, 4)
    thr_g, thr_r = _thr()
    want = oracle.detect_image(q, thr_r)
    img = torch.from_numpy(q).cuda()
    with rise.Detector(0) as d:
        d.set_option(rise.OPT_UNION_LIMIT, 1)
        with pytest.raises(rise.RiseError) as e:
            d.detect_image(img, thr_g)
        assert e.value.code == rise.RISE_ETIMEOUT
        d.set_option(rise.OPT_UNION_LIMIT, 0)
        np.testing.assert_array_equal(d.detect_image(img, thr_g), want)


def test_waits_run_out_on_the_capture_and_batch_paths():
    """The same through rise_detect (replayed graphs included) and
    rise_detect_batch: every call with the withheld tile times out, and the
    calls after it give the boxes of an untouched context."""
    from paper_2603_20481_gb300 import rise
    cap = synth.make_capture(1 << 20, 100e6, 40, 61, fft_size=1024, hop=512,
                             bw_hz=(0.2e6, 20e6), dur_s=(0.1e-3, 5e-3), snr_db=(0, 20),
                             tone_fraction=0.2)
    x = torch.from_numpy(cap.iq).cuda()
    caps = synth.batched_captures(8, 8100, n_range=(1 << 16, 1 << 18))
    xs = [torch.from_numpy(c.iq).cuda() for c in caps]
    Ns = [c.fft_size for c in caps]
    hops = [c.hop for c in caps]
    with rise.Detector(0) as ref:
        ref.set_option(rise.OPT_AUTOTUNE, 0)         # fixed launch shapes and schedules in both
        want = ref.detect(x, 1024, 512)
        want_b, want_o = ref.detect_batch(xs, Ns, hops)
        runs = int(ref.debug(rise.DBG_CCL, 0, 0)[0])
    assert runs > 2048                                 # the batch's scan has a second tile
    with rise.Detector(0) as d:
        d.set_option(rise.OPT_AUTOTUNE, 0)
        d.detect(x, 1024, 512)
        d.set_option(rise.OPT_SCAN_WAIT_LIMIT, 64)
        d.set_option(rise.OPT_TEST_WITHHOLD, 0)
        for _ in range(3):                             # the third call replays a graph
            with pytest.raises(rise.RiseError) as e:
                d.detect_batch(xs, Ns, hops)
            assert e.value.code == rise.RISE_ETIMEOUT
        d.set_option(rise.OPT_UNION_LIMIT, 1)
        d.set_option(rise.OPT_TEST_WITHHOLD, -1)
        for _ in range(3):
            with pytest.raises(rise.RiseError) as e:
                d.detect(x, 1024, 512)
            assert e.value.code == rise.RISE_ETIMEOUT
        d.set_option(rise.OPT_UNION_LIMIT, 0)
        d.set_option(rise.OPT_SCAN_WAIT_LIMIT, 0)
        for _ in range(3):
            np.testing.assert_array_equal(d.detect(x, 1024, 512), want)
            b, o = d.detect_batch(xs, Ns, hops)
            np.testing.assert_array_equal(o, want_o)
            np.testing.assert_array_equal(b, want_b)


@pytest.mark.parametrize("N,hop,sched", [(1024, 512, 1), (4096, 2048, 1), (8192, 2048, 1), (8192, 2048, 2)])
def test_staged_copy_wait_runs_out_and_the_context_recovers(N, hop, sched):
    """The STFT's wait for a staged input copy: with RISE_OPT_TEST_WITHHOLD_COPY
    block 0 never issues the copy of one frame group, so its barrier wait runs
    out after RISE_OPT_COPY_WAIT_LIMIT polls; the block leaves (the halves of a
    schedule-2 block both leave, since no copy is issued without both), the
    call ends with RISE_ETIMEOUT on the single-capture and batch paths, and the
    next calls give the boxes of an untouched context.  No copy is in flight
    when a block leaves: the withheld one was never issued."""
    from paper_2603_20481_gb300 import rise
    cap = synth.make_capture(N * 64, 100e6, 12, 71 + N, fft_size=N, hop=hop,
                             bw_hz=(0.2e6, 20e6), dur_s=(0.05e-3, 0.3e-3), snr_db=(5, 20))
    x = torch.from_numpy(cap.iq).cuda()
    caps = synth.batched_captures(4, 8200 + N, n_range=(1 << 15, 1 << 17))
    xs = [torch.from_numpy(c.iq).cuda() for c in caps]
    Ns = [c.fft_size for c in caps]
    hops = [c.hop for c in caps]
    with rise.Detector(0) as d:
        d.set_option(rise.OPT_AUTOTUNE, 0)
        d.set_option(rise.OPT_FFT_SCHEDULE, sched)
        want = d.detect(x, N, hop)
        want_b, want_o = d.detect_batch(xs, Ns, hops)
        d.set_option(rise.OPT_COPY_WAIT_LIMIT, 1 << 14)
        d.set_option(rise.OPT_TEST_WITHHOLD_COPY, 0)   # the first copy of block 0
        for _ in range(2):
            with pytest.raises(rise.RiseError) as e:
                d.detect(x, N, hop)
            assert e.value.code == rise.RISE_ETIMEOUT
        with pytest.raises(rise.RiseError) as e:
            d.detect_batch(xs, Ns, hops)
        assert e.value.code == rise.RISE_ETIMEOUT
        d.set_option(rise.OPT_TEST_WITHHOLD_COPY, -1)
        d.set_option(rise.OPT_COPY_WAIT_LIMIT, 0)
        for _ in range(2):
            np.testing.assert_array_equal(d.detect(x, N, hop), want)
            b, o = d.detect_batch(xs, Ns, hops)
            np.testing.assert_array_equal(o, want_o)
            np.testing.assert_array_equal(b, want_b)


def test_limit_options_are_checked():
    from paper_2603_20481_gb300 import rise
    with rise.Detector(0) as d:
        for opt, bad in ((rise.OPT_SCAN_WAIT_LIMIT, -1), (rise.OPT_UNION_LIMIT, -5),
                         (rise.OPT_TEST_WITHHOLD, -2), (rise.OPT_UNION_LIMIT, 1 << 40),
                         (rise.OPT_COPY_WAIT_LIMIT, -1), (rise.OPT_COPY_WAIT_LIMIT, 1 << 40),
                         (rise.OPT_COPY_WAIT_LIMIT, 4095),
                         (rise.OPT_TEST_WITHHOLD_COPY, -2), (rise.OPT_BLOCKING_WAIT, 2),
                         (rise.OPT_BLOCKING_WAIT, -1)):
            with pytest.raises(rise.RiseError):
                d.set_option(opt, bad)
