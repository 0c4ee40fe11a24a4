"""rise_detect_batch against the FP64 oracle and against one rise_detect call
per capture.

A batch runs its own kernels (a persistent STFT over all captures of one FFT
size, batch-indexed histogram, floor, morphology and labelling), so every
capture is checked against the oracle directly, with the bars of the
single-capture parity tests: the float |X|^2 within 1e-4 relative, the anchor
within 1e-5, the 8-bit image equal to the oracle's quantiser applied to the
GPU's own power and within one level of the FP64 image on at most
ceil(1e-5 px) + 6 pixels, and the boxes bit-exact against the oracle run on
the capture's own 8-bit image.  A batch shares launches, not results: every
capture must also come out exactly as it does alone (same 8-bit anchor, noise
floor, Otsu thresholds, components), so the boxes are compared bit for bit
with rise_detect, capture by capture.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_20481_gb300 import synth

pytestmark = pytest.mark.gpu


def _oracle_check(det, xs, Ns, hops, boxes, offs, prm=None, power=True):
    """Every capture of the last batch against the oracle (see the module bars)."""
    from paper_2603_20481_gb300 import rise
    shapes = [(oracle.num_frames(int(x.numel()), N, h), N) for x, N, h in zip(xs, Ns, hops)]
    imgs = det.batch_debug(shapes, rise.DBG_BATCH_IMAGES)
    anchors = det.batch_debug(shapes, rise.DBG_BATCH_ANCHORS)
    pows = det.batch_debug(shapes, rise.DBG_BATCH_POWER) if power else [None] * len(xs)
    fixed = prm is not None and prm.range_mode == 1
    for c, (x, N, h, qg, Pg, Mg) in enumerate(zip(xs, Ns, hops, imgs, pows, anchors)):
        iq = x.cpu().numpy()
        want = oracle.detect_image(qg, prm)
        np.testing.assert_array_equal(boxes[offs[c]:offs[c + 1]], want, err_msg=f"capture {c}")
        boxes_r, qr, Mr = oracle.detect(iq, N, h, prm)
        d = qg.astype(np.int16) - qr.astype(np.int16)
        assert np.abs(d).max(initial=0) <= 1, f"capture {c}"
        assert np.count_nonzero(d) <= math.ceil(1e-5 * qg.size) + 6, f"capture {c}"
        if not fixed:
            assert abs(float(Mg) - Mr) <= 1e-5 * Mr, f"capture {c}"
        if Pg is not None:
            assert float(Mg) == float(Pg.max())
            T = qg.shape[0]
            rows = sorted({0, T // 2, T - 1})
            for t in rows:
                Pr = oracle.stft_power(iq, N, h, t, 1)
                floor = 1e-6 * Pr.mean(axis=1, keepdims=True)
                assert np.all(np.abs(Pg[t:t + 1].astype(np.float64) - Pr) <= 1e-4 * Pr + floor), \
                    f"capture {c} frame {t}"
            q_same = oracle.quantize(Pg.astype(np.float64), oracle.hi_db_of(float(Mg)),
                                     prm.level_db if prm is not None else 0.25)
            assert np.array_equal(q_same, qg), f"capture {c}"


def _batch(count, seed0, n_range=(1 << 13, 1 << 18), sizes=(256, 512, 1024, 2048)):
    return synth.batched_captures(count, seed0, sizes=sizes, n_range=n_range)


def _plain(det, xs, Ns, hops, thr=None):
    """One rise_detect per capture, each with the radix schedule the context's
    last batch ran for its FFT size (the two schedules round differently)."""
    from paper_2603_20481_gb300 import rise
    det.set_option(rise.OPT_FFT_SCHEDULE, -1)
    try:
        return [det.detect(x, N, h, thr) for x, N, h in zip(xs, Ns, hops)]
    finally:
        det.set_option(rise.OPT_FFT_SCHEDULE, 3)


def _check(boxes, offs, want):
    assert offs[0] == 0 and len(offs) == len(want) + 1
    assert offs[-1] == sum(len(w) for w in want) == len(boxes)
    for c, w in enumerate(want):
        np.testing.assert_array_equal(boxes[offs[c]:offs[c + 1]], w, err_msg=f"capture {c}")


def _to_gpu(caps, ragged=0):
    import torch
    xs = []
    for i, c in enumerate(caps):
        iq = c.iq
        if ragged and i % 3 == 1:
            iq = iq[: max(c.fft_size, iq.shape[0] - ragged - i)]   # ragged tail
        xs.append(torch.from_numpy(np.ascontiguousarray(iq)).cuda())
    return xs


def test_mixed_sizes_match_single_calls(det):
    caps = _batch(24, 7000)
    xs = _to_gpu(caps, ragged=777)
    Ns = [c.fft_size for c in caps]
    hops = [c.hop for c in caps]
    boxes, offs = det.detect_batch(xs, Ns, hops)
    info = det.batch_info()
    assert info[0] >= 2                                  # several FFT sizes -> several STFT groups
    _oracle_check(det, xs, Ns, hops, boxes, offs)
    _check(boxes, offs, _plain(det, xs, Ns, hops))


def test_odd_hops_and_unaligned_starts(det):
    # odd hops and a base that is only 8-byte aligned use the non-staged STFT
    import torch
    caps = _batch(6, 7100, n_range=(1 << 14, 1 << 16))
    xs, Ns, hops = [], [], []
    for i, c in enumerate(caps):
        t = torch.from_numpy(c.iq).cuda()
        if i % 2:
            t = torch.cat([torch.zeros(1, dtype=t.dtype, device=t.device), t])[1:]   # 8-byte offset
            assert t.data_ptr() % 16 == 8
        xs.append(t)
        Ns.append(c.fft_size)
        hops.append(c.fft_size // 2 + (1 if i % 3 == 0 else 0))
    boxes, offs = det.detect_batch(xs, Ns, hops)
    _oracle_check(det, xs, Ns, hops, boxes, offs)
    _check(boxes, offs, _plain(det, xs, Ns, hops))


def test_fixed_range_and_other_thresholds(det):
    from paper_2603_20481_gb300 import rise
    caps = _batch(8, 7200, n_range=(1 << 14, 1 << 17))
    xs = _to_gpu(caps)
    Ns = [c.fft_size for c in caps]
    hops = [c.hop for c in caps]
    for kw in (dict(range_mode=rise.RANGE_FIXED, hi_db=75.0),
               dict(level_db=0.5, psd_offset_db=1.0, power_offset_db=6.0, sg_half_window=3,
                    morph_order=1)):
        thr = rise.default_thresholds(**kw)
        boxes, offs = det.detect_batch(xs, Ns, hops, thr)
        _oracle_check(det, xs, Ns, hops, boxes, offs, oracle.params(**kw),
                      power=kw.get("range_mode", 0) == 0)
        _check(boxes, offs, _plain(det, xs, Ns, hops, thr))


def test_graph_replay_reads_fresh_inputs(det):
    # same composition twice: the second call replays the captured chain and
    # must still see the new samples and the new output
    import torch
    caps = _batch(10, 7300, n_range=(1 << 14, 1 << 17))
    Ns = [c.fft_size for c in caps]
    hops = [c.hop for c in caps]
    xs = _to_gpu(caps)
    b1, o1 = det.detect_batch(xs, Ns, hops)
    _check(b1, o1, _plain(det, xs, Ns, hops))
    # new contents in the same tensors (same pointers, same shapes)
    other = _batch(10, 7400, n_range=(1 << 14, 1 << 17))
    for x, c in zip(xs, other):
        n = min(x.numel(), c.iq.shape[0])
        x[:n].copy_(torch.from_numpy(c.iq[:n]))
    b2, o2 = det.detect_batch(xs, Ns, hops)
    assert det.batch_info()[1] == 1                       # run from the captured graph
    _oracle_check(det, xs, Ns, hops, b2, o2)
    _check(b2, o2, _plain(det, xs, Ns, hops))
    assert not (len(b1) == len(b2) and np.array_equal(b1, b2))
    # and once more with the first contents: a replay of the same graph
    for x, c in zip(xs, caps):
        n = min(x.numel(), c.iq.shape[0])
        x[:n].copy_(torch.from_numpy(c.iq[:n]))
    b3, o3 = det.detect_batch(xs, Ns, hops)
    assert det.batch_info()[1] == 1
    np.testing.assert_array_equal(b3, b1)
    np.testing.assert_array_equal(o3, o1)


def test_switches_give_the_same_boxes(det):
    from paper_2603_20481_gb300 import rise
    caps = _batch(12, 7500)
    xs = _to_gpu(caps)
    Ns = [c.fft_size for c in caps]
    hops = [c.hop for c in caps]
    ref, ro = det.detect_batch(xs, Ns, hops)
    ref_sched = det.batch_info()
    G = int(ref_sched[0])
    ref_sched = list(ref_sched[3 + G:3 + 3 * G])
    # (graphs, tuner, blocking wait): the host's way of waiting changes nothing
    for graph, tune, block in ((0, 0, 0), (0, 1, 0), (1, 0, 0), (1, 0, 1), (0, 0, 1)):
        with rise.Detector(0) as d2:
            d2.set_option(rise.OPT_BATCH_GRAPH, graph)
            d2.set_option(rise.OPT_AUTOTUNE, tune)
            d2.set_option(rise.OPT_BLOCKING_WAIT, block)
            for _ in range(2):
                b, o = d2.detect_batch(xs, Ns, hops)
                info = d2.batch_info()
                if list(info[3 + G:3 + 3 * G]) == ref_sched:   # same radix schedules: same bits
                    np.testing.assert_array_equal(o, ro)
                    np.testing.assert_array_equal(b, ref)
                else:
                    _oracle_check(d2, xs, Ns, hops, b, o)
            assert d2.batch_info()[1] == graph


def test_truncation_offsets_and_edge_cases(det):
    import ctypes
    import torch
    from paper_2603_20481_gb300 import rise
    caps = _batch(5, 7600, n_range=(1 << 15, 1 << 17))
    xs = _to_gpu(caps)
    Ns = [c.fft_size for c in caps]
    hops = [c.hop for c in caps]
    full, fo = det.detect_batch(xs, Ns, hops)
    assert fo[-1] > 3
    det._auto_grow = False
    try:
        b, o = det.detect_batch(xs, Ns, hops, cap=3)
        assert det.last_status == rise.RISE_ETRUNC
        np.testing.assert_array_equal(o, fo)
        np.testing.assert_array_equal(b, full[:3])
    finally:
        det._auto_grow = True
    # no captures
    offs = np.zeros(1, np.int64)
    assert rise.lib().rise_detect_batch(det._h, None, 0, None, None, 0, offs.ctypes.data) == 0
    assert offs[0] == 0
    # a capture of exactly one frame, next to normal ones
    one = torch.from_numpy(caps[0].iq[:Ns[0]].copy()).cuda()
    b, o = det.detect_batch([one] + xs, [Ns[0]] + Ns, [hops[0]] + hops)
    _check(b, o, _plain(det, [one] + xs, [Ns[0]] + Ns, [hops[0]] + hops))
    # rejected before any work: too short, too many frames, bad FFT size
    bad = [(xs[0], Ns[0] * 4096, hops[0]), (xs[0], Ns[0], 0), (xs[0], 300, 150)]
    for x, N, h in bad:
        with pytest.raises(rise.RiseError) as e:
            det.detect_batch([x], [N], [h])
        assert e.value.code == rise.RISE_EINVAL
    long = torch.zeros(rise.BATCH_MAX_ROWS * 256 + 256, dtype=torch.complex64, device="cuda")
    with pytest.raises(rise.RiseError):
        det.detect_batch([long], [256], [256])
    del long


@pytest.mark.slow
def test_many_uneven_captures(det):
    # 128 captures, 2^14..2^20 samples, every FFT size of the batched workload
    caps = _batch(128, 1000, n_range=(1 << 14, 1 << 20))
    xs = _to_gpu(caps)
    Ns = [c.fft_size for c in caps]
    hops = [c.hop for c in caps]
    boxes, offs = det.detect_batch(xs, Ns, hops)
    _oracle_check(det, xs, Ns, hops, boxes, offs)
    _check(boxes, offs, _plain(det, xs, Ns, hops))


def test_tune_cache_is_read_by_a_new_context(tmp_path, monkeypatch):
    """With RISE_TUNE_CACHE set, the first context tunes the composition and
    appends one line; a second context runs it from the file without tuning;
    a cached line asking for radix schedule 1 in every group is run as
    written and still matches the oracle."""
    from paper_2603_20481_gb300 import rise
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("RISE_TUNE_CACHE", str(path))
    caps = _batch(10, 7800, n_range=(1 << 14, 1 << 17), sizes=(512, 1024, 2048))
    xs = _to_gpu(caps)
    Ns = [c.fft_size for c in caps]
    hops = [c.hop for c in caps]
    with rise.Detector(0) as d1:
        b1, o1 = d1.detect_batch(xs, Ns, hops)
        assert d1.batch_info()[63] == 0
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("rise-tune 1 ")
    with rise.Detector(0) as d2:
        b2, o2 = d2.detect_batch(xs, Ns, hops)
        assert d2.batch_info()[63] == 1                  # from the file, no tuning
    assert path.read_text().splitlines() == lines
    np.testing.assert_array_equal(b2, b1)
    np.testing.assert_array_equal(o2, o1)
    f = lines[0].split()
    G = int(f[4])
    f[5 + G:5 + 2 * G] = ["1"] * G
    path.write_text(" ".join(f) + "\n")
    with rise.Detector(0) as d3:
        b3, o3 = d3.detect_batch(xs, Ns, hops)
        info = d3.batch_info()
        assert int(info[0]) == G and all(info[3 + G:3 + 2 * G] == 1)
        assert sorted(set(int(v) for v in info[3 + 2 * G:3 + 3 * G])) == [512, 1024, 2048]
        _oracle_check(d3, xs, Ns, hops, b3, o3)


def test_intermediates_are_dropped_by_the_next_call(det):
    from paper_2603_20481_gb300 import rise
    caps = _batch(3, 7700, n_range=(1 << 13, 1 << 14))
    xs = _to_gpu(caps)
    Ns = [c.fft_size for c in caps]
    hops = [c.hop for c in caps]
    det.detect_batch(xs, Ns, hops)
    shapes = [(oracle.num_frames(int(x.numel()), N, h), N) for x, N, h in zip(xs, Ns, hops)]
    det.batch_debug(shapes)
    det.detect(xs[0], Ns[0], hops[0])          # overwrites the image buffer
    with pytest.raises(rise.RiseError):
        det.batch_debug(shapes)


def test_replay_after_the_tables_grew():
    """A small composition, a larger one (its tables outgrow the staging
    blob, which moves), then the small one again: the small batch's graph
    must not be replayed with the old blob's address; every call equals the
    per-capture calls."""
    from paper_2603_20481_gb300 import rise
    caps_s = _batch(2, 3100)
    caps_b = _batch(96, 3200, n_range=(1 << 12, 1 << 14))
    small, big = _to_gpu(caps_s), _to_gpu(caps_b)
    args_s = ([c.fft_size for c in caps_s], [c.hop for c in caps_s])
    args_b = ([c.fft_size for c in caps_b], [c.hop for c in caps_b])
    with rise.Detector(0) as d:
        d.set_option(rise.OPT_AUTOTUNE, 0)
        want_s = _plain(d, small, *args_s)
        want_b = _plain(d, big, *args_b)
        for xs, args, want in ((small, args_s, want_s), (small, args_s, want_s), (big, args_b, want_b),
                               (big, args_b, want_b), (small, args_s, want_s), (small, args_s, want_s)):
            boxes, offs = d.detect_batch(xs, *args)
            _check(boxes, offs, want)
