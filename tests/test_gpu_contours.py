"""rise_contours: the shapes of the detected blocks against the oracle.

For the final mask of a call (taken from the GPU, whose bit-exactness against
the oracle's pipeline the parity tests already check), every run with its
component must equal the oracle's BFS labelling of that mask, and the
boundary mask the oracle's neighbour test; the runs of component k must
also rebuild box k (extent and area).  Shapes touching every image edge,
runs over many 32-bit words and blocks with holes are covered by a crafted
8-bit image; the queued calls, a run-array overflow with a call queued
behind it, and the error cases are covered on captures.
"""
import numpy as np
import pytest

import oracle
from paper_2603_20481_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _crafted(T=300, F=1024, seed=5):
    rng = np.random.default_rng(seed)
    q = rng.integers(0, 40, (T, F)).astype(np.uint8)

    def put(t0, t1, f0, f1, v=220):
        q[t0:t1 + 1, f0:f1 + 1] = v
    put(10, 60, F - 70, F - 1)          # touches the last column
    put(20, 40, 0, 45)                  # touches the first column
    put(100, 180, 200, 420)             # many words wide ...
    put(120, 160, 260, 360, 10)         # ... with a hole
    put(200, T - 1, 600, 640)           # touches the last row
    put(0, 5, 700, 900)                 # touches the first row
    for _ in range(40):
        t, f = rng.integers(0, T - 8), rng.integers(0, F - 8)
        put(t, t + rng.integers(3, 8), f, f + rng.integers(3, 8))
    return q


def _check(det, boxes, T, F):
    from paper_2603_20481_gb300 import rise
    runs, bnd = det.contours(T, F)
    mask = rise.unpack_mask(det.debug(rise.DBG_MASK3, T, F), F)
    np.testing.assert_array_equal(runs, oracle.component_runs(mask))
    np.testing.assert_array_equal(bnd, oracle.boundary(mask))
    # the runs of component k rebuild box k
    assert (runs[:, 0].max() + 1 if len(runs) else 0) == len(boxes)
    for k, b in enumerate(boxes):
        r = runs[runs[:, 0] == k]
        assert (r[:, 1].min(), r[:, 1].max(), r[:, 2].min(), r[:, 3].max()) == tuple(b[:4])
        assert int((r[:, 3] - r[:, 2] + 1).sum()) == b[5]
    return runs, bnd, mask


def test_crafted_image_shapes(det):
    q = _crafted()
    T, F = q.shape
    boxes = det.detect_image(torch.from_numpy(q).cuda())
    np.testing.assert_array_equal(boxes, oracle.detect_image(q))
    runs, bnd, mask = _check(det, boxes, T, F)
    assert (runs[:, 3] == F - 1).any() and (runs[:, 2] == 0).any()
    assert (runs[:, 1] == 0).any() and (runs[:, 1] == T - 1).any()
    assert ((runs[:, 3] - runs[:, 2]) > 64).any()
    assert bnd.sum() < mask.sum()      # interiors exist


def test_capture_and_without_boundary(det):
    cap = synth.single_capture(101)
    x = torch.from_numpy(cap.iq).cuda()
    boxes = det.detect(x, 1024, 512)
    T = oracle.num_frames(cap.iq.shape[0], 1024, 512)
    runs, _, _ = _check(det, boxes, T, 1024)
    runs2, none = det.contours(T, 1024, boundary=False)
    assert none is None
    np.testing.assert_array_equal(runs2, runs)


def test_queued_calls_and_overflow():
    """After two queued calls the shapes are the second's, also when the
    first overflowed its run arrays and was run again at collect time."""
    from paper_2603_20481_gb300 import rise
    a = synth.make_capture(1 << 20, 20e6, 40, 91, fft_size=1024, hop=512,
                           bw_hz=(0.2e6, 3e6), dur_s=(0.5e-3, 5e-3), snr_db=(10, 25))
    b = synth.single_capture(92)
    xs = [torch.from_numpy(c.iq).cuda() for c in (a, b)]
    T = oracle.num_frames(b.iq.shape[0], 1024, 512)
    with rise.Detector(0) as ref:
        ref.detect(xs[1], 1024, 512)
        want, _ = ref.contours(T, 1024)
    for run_cap in (0, 1024):
        with rise.Detector(0) as d:
            if run_cap:
                d.set_option(rise.OPT_RUN_CAPACITY, run_cap)
            d.submit(xs[0], 1024, 512)
            d.submit(xs[1], 1024, 512)
            with pytest.raises(rise.RiseError):
                d.contours(T, 1024)            # calls still queued
            d.collect()
            boxes = d.collect()
            got, _, _ = _check(d, boxes, T, 1024)
            np.testing.assert_array_equal(got, want)


def test_truncation_and_after_batch(det):
    import ctypes
    from paper_2603_20481_gb300 import rise
    cap = synth.single_capture(101)
    x = torch.from_numpy(cap.iq).cuda()
    det.detect(x, 1024, 512)
    T = oracle.num_frames(cap.iq.shape[0], 1024, 512)
    full, _ = det.contours(T, 1024, boundary=False)
    assert len(full) > 3
    part = np.zeros((3, 4), np.int32)
    n = ctypes.c_int64(0)
    rc = rise.lib().rise_contours(det._h, part.ctypes.data, 3, ctypes.byref(n), None)
    assert rc == rise.RISE_ETRUNC and n.value == len(full)
    np.testing.assert_array_equal(part, full[:3])
    det.detect_batch([x], [1024], [512])
    with pytest.raises(rise.RiseError):
        det.contours(T, 1024)
