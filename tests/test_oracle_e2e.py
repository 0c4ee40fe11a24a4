"""End-to-end checks of the oracle (CPU): the whole path is the composition
of its steps, and strong planted bursts come back as boxes that overlap
their ground truth (informational accuracy, as the paper itself reports a
mean IoU near 63%, Sec. VI-A)."""
import numpy as np
import pytest

import hand_images
import oracle
from paper_2603_20481_gb300 import synth


def _iou(a, b):
    t0, t1 = max(a[0], b[0]), min(a[1], b[1])
    f0, f1 = max(a[2], b[2]), min(a[3], b[3])
    if t1 < t0 or f1 < f0:
        return 0.0
    inter = (t1 - t0 + 1) * (f1 - f0 + 1)
    ua = (a[1] - a[0] + 1) * (a[3] - a[2] + 1)
    ub = (b[1] - b[0] + 1) * (b[3] - b[2] + 1)
    return inter / (ua + ub - inter)


def test_detect_is_the_composition_of_its_steps():
    cap = synth.make_capture(1 << 16, 20e6, 4, 77, fft_size=256, hop=128,
                             bw_hz=(1e6, 3e6), dur_s=(0.2e-3, 1e-3), snr_db=(10, 20),
                             tone_fraction=0.0)
    boxes, img, mx = oracle.detect(cap.iq, 256, 128)
    P = oracle.stft_power(cap.iq, 256, 128)
    assert mx == P.max()
    q = oracle.quantize(P, oracle.hi_db_of(mx))
    assert np.array_equal(q, img)
    assert np.array_equal(oracle.detect_image(q), boxes)
    # anchoring on hi_db equal to the capture max gives the same image
    b2, img2, _ = oracle.detect(cap.iq, 256, 128, oracle.params(range_mode=1, hi_db=oracle.hi_db_of(mx)))
    assert np.array_equal(img2, img) and np.array_equal(b2, boxes)


def test_strong_planted_bursts_are_found():
    hits, total = 0, 0
    for seed in (11, 12, 13):
        cap = synth.make_capture(1 << 18, 20e6, 5, seed, fft_size=512, hop=256,
                                 bw_hz=(1e6, 3e6), dur_s=(1e-3, 3e-3), snr_db=(12, 20),
                                 tone_fraction=0.0)
        gt = synth.gt_boxes(cap)
        boxes, _, _ = oracle.detect(cap.iq, 512, 256)
        for i, g in enumerate(gt):
            if any(_iou(g, h) > 0 for j, h in enumerate(gt) if j != i):
                continue            # overlapping emitters merge; skip them
            total += 1
            best = max((_iou(g, b[:4]) for b in boxes), default=0.0)
            hits += best >= 0.5
    assert total >= 8
    assert hits >= 0.8 * total



@pytest.mark.parametrize("F", [64, 256])
def test_hand_image_closed_form(F):
    """The block image of hand_images.block_image, worked through by hand:
    noise floor, offsets, power floor, per-column thresholds, final mask and
    the one box, all exact."""
    q, want, want_boxes = hand_images.block_image(F)
    boxes, ex = oracle.detect_image(q, extras=True)
    for k in ("D", "N0", "delta_psd", "delta_pow", "P_q"):
        assert ex[k] == want[k], k
    np.testing.assert_array_equal(ex["eff"], want["eff"])
    np.testing.assert_array_equal(ex["mask"], want["mask"])
    np.testing.assert_array_equal(boxes, want_boxes)
    # the Otsu step alone on a block column: the smallest of the tied splits
    h = np.zeros(256, np.uint32)
    h[100], h[200] = 54, 10
    assert oracle.otsu(h) == 100


def test_thread_count_does_not_change_results():
    """The oracle's parallel loops (frames, column groups, rows) give what one
    thread gives: the same image, anchor, histograms, masks and boxes."""
    cap = synth.make_capture(3 * 512 * 97 + 311, 20e6, 6, 99, fft_size=512, hop=384,
                             bw_hz=(0.5e6, 4e6), dur_s=(0.2e-3, 2e-3), snr_db=(5, 20),
                             tone_fraction=0.3)
    oracle.set_threads(1)
    try:
        one = oracle.detect(cap.iq, 512, 384)
        q = one[1]
        b1, ex1 = oracle.detect_image(q, extras=True)
        for n in (0, 3):
            oracle.set_threads(n)
            many = oracle.detect(cap.iq, 512, 384)
            assert many[2] == one[2]
            np.testing.assert_array_equal(many[1], one[1])
            np.testing.assert_array_equal(many[0], one[0])
            bn, exn = oracle.detect_image(q, extras=True)
            np.testing.assert_array_equal(bn, b1)
            for k in ("hist", "eff", "mask"):
                np.testing.assert_array_equal(exn[k], ex1[k])
    finally:
        oracle.set_threads(0)          # back to the default: every core
