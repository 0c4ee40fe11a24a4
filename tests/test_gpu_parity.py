"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars:
* spectrogram: |P_gpu - P_ref| <= 1e-4 P_ref + 1e-6 * mean of the frame's P_ref;
* 8-bit image: at most ceil(1e-5 * pixels) pixels differ, each by one level,
  and the GPU's levels equal the oracle's quantiser applied to the GPU's own
  float power with the GPU's anchor (the decision taken in the same precision);
* from the 8-bit image on (histograms, column statistics, every mask stage,
  boxes): bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_20481_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rise():
    from paper_2603_20481_gb300 import rise
    return rise


def _thr_pair(**kw):
    rise = _rise()
    return rise.default_thresholds(**kw), oracle.params(**kw)


def _gpu_detect(det, iq_np, N, hop, thr=None, keep=True):
    rise = _rise()
    det.set_option(rise.OPT_KEEP_POWER, int(keep))
    det.set_option(rise.OPT_KEEP_MASKS, int(keep))
    x = torch.from_numpy(iq_np).cuda()
    boxes = det.detect(x, N, hop, thr)
    torch.cuda.synchronize()
    return boxes


def _check_power(Pg, Pr):
    floor = 1e-6 * Pr.mean(axis=1, keepdims=True)
    bad = np.abs(Pg.astype(np.float64) - Pr) > 1e-4 * Pr + floor
    assert not bad.any(), f"{bad.sum()} spectrogram bins off, worst rel {np.max(np.abs(Pg - Pr) / (Pr + floor))}"


def _check_image(qg, qr):
    """Levels differ by at most one; returns how many pixels differ.  The
    1e-5 bar is a rate: it is asserted on pooled and full-size images
    (test_image_level_mismatch_rate, test_wideband_full_size), where the
    count is large enough to measure it; a single small image only gets a
    Poisson-tail guard."""
    d = qg.astype(np.int16) - qr.astype(np.int16)
    nd = int(np.count_nonzero(d))
    assert np.abs(d).max(initial=0) <= 1
    assert nd <= math.ceil(1e-5 * qg.size) + 6, f"{nd} of {qg.size} pixels differ"
    return nd


STFT_CASES = [
    # (N, hop, n, fs, seed)
    (256, 128, 256 * 37 + 77, 20e6, 1),
    (256, 1, 2000, 20e6, 2),
    (512, 512, 512 * 300 + 11, 20e6, 3),
    (1024, 1024, 1 << 18, 20e6, 4),
    (1024, 300, 100003, 20e6, 5),
    (2048, 1024, 2048 * 40 + 5, 61.44e6, 6),
    (4096, 2048, 4096 * 40 + 123, 100e6, 7),
    (8192, 2048, 8192 * 12 + 9, 100e6, 8),
    (4096, 4096, 4096, 100e6, 9),          # T = 1
]


@pytest.mark.parametrize("N,hop,n,fs,seed", STFT_CASES)
def test_spectrogram_and_image_parity(det, N, hop, n, fs, seed):
    rise = _rise()
    cap = synth.make_capture(n, fs, 6, 500 + seed, fft_size=N, hop=hop,
                             bw_hz=(fs / 200, fs / 20), dur_s=(n / fs / 20, n / fs / 3),
                             snr_db=(5, 25), tone_fraction=0.3)
    T = oracle.num_frames(n, N, hop)
    boxes_g = _gpu_detect(det, cap.iq, N, hop)
    Pg = det.debug(rise.DBG_POWER_F32, T, N)
    qg = det.debug(rise.DBG_IMAGE_U8, T, N)
    Mg = float(det.debug(rise.DBG_MAXPOW, T, N)[0])
    Pr = oracle.stft_power(cap.iq, N, hop)
    _check_power(Pg, Pr)
    assert Mg == float(Pg.max())
    # same-precision decision: the oracle's quantiser on the GPU's float power
    q_same = oracle.quantize(Pg.astype(np.float64), oracle.hi_db_of(Mg))
    assert np.array_equal(q_same, qg)
    # against the FP64 path end to end
    boxes_r, qr, Mr = oracle.detect(cap.iq, N, hop)
    assert abs(Mg - Mr) <= 1e-5 * Mr
    nd = _check_image(qg, qr)
    # from the image on, bit-exact: the oracle on the GPU's own image
    assert np.array_equal(boxes_g, oracle.detect_image(qg))
    if nd == 0:
        assert np.array_equal(boxes_g, boxes_r)


@pytest.mark.parametrize("sched", [0, 1, 2])
@pytest.mark.parametrize("N,hop,n,fs,seed", [c for c in STFT_CASES if c[0] in (512, 1024, 2048, 8192)]
                         + [(8192, 2047, 8192 * 9 + 5, 100e6, 10),   # odd hop: the unstaged loads
                            (512, 255, 512 * 200 + 7, 20e6, 11)])
def test_other_radix_schedules_match_the_oracle(det, N, hop, n, fs, seed, sched):
    """Every radix schedule under the same bars, whichever one is the
    library's for the size: 0 (the radix-r pass last), 1 (the radix-r pass
    first) and 2 (the frame split into two half-size transforms, N = 512 and
    8192, the halves decoupled at 8192; other sizes run schedule 0 for
    it)."""
    rise = _rise()
    cap = synth.make_capture(n, fs, 6, 500 + seed, fft_size=N, hop=hop,
                             bw_hz=(fs / 200, fs / 20), dur_s=(n / fs / 20, n / fs / 3),
                             snr_db=(5, 25), tone_fraction=0.3)
    T = oracle.num_frames(n, N, hop)
    det.set_option(rise.OPT_FFT_SCHEDULE, sched)
    try:
        boxes_g = _gpu_detect(det, cap.iq, N, hop)
        Pg = det.debug(rise.DBG_POWER_F32, T, N)
        qg = det.debug(rise.DBG_IMAGE_U8, T, N)
        Mg = float(det.debug(rise.DBG_MAXPOW, T, N)[0])
    finally:
        det.set_option(rise.OPT_FFT_SCHEDULE, 3)   # the default
    _check_power(Pg, oracle.stft_power(cap.iq, N, hop))
    q_same = oracle.quantize(Pg.astype(np.float64), oracle.hi_db_of(Mg))
    assert np.array_equal(q_same, qg)
    _, qr, Mr = oracle.detect(cap.iq, N, hop)
    assert abs(Mg - Mr) <= 1e-5 * Mr
    _check_image(qg, qr)
    assert np.array_equal(boxes_g, oracle.detect_image(qg))


def test_image_level_mismatch_rate(det):
    """At most 1e-5 of pixels may differ by one 8-bit level from the FP64
    oracle (the fp32 FFT's rounding puts a few pixels on the other side of a
    level edge).  Pooled over the STFT cases plus 1024 x 1024 and
    1023 x 4096 captures, about 11 million pixels."""
    rise = _rise()
    det.set_option(rise.OPT_KEEP_POWER, 0)
    det.set_option(rise.OPT_KEEP_MASKS, 0)
    caps = [(synth.make_capture(n, fs, 6, 500 + seed, fft_size=N, hop=hop,
                                bw_hz=(fs / 200, fs / 20), dur_s=(n / fs / 20, n / fs / 3),
                                snr_db=(5, 25), tone_fraction=0.3), N, hop)
            for N, hop, n, fs, seed in STFT_CASES]
    caps += [(synth.single_capture(101), 1024, 1024), (synth.single_capture(103), 1024, 1024)]
    for seed in range(2):
        caps.append((synth.make_capture(1 << 21, 100e6, 20, 700 + seed, fft_size=4096, hop=2048,
                                        bw_hz=(0.1e6, 20e6), dur_s=(0.5e-3, 5e-3),
                                        snr_db=(-3, 25), tone_fraction=0.25), 4096, 2048))
    px = diff = 0
    for cap, N, hop in caps:
        T = oracle.num_frames(cap.iq.shape[0], N, hop)
        det.detect(torch.from_numpy(cap.iq).cuda(), N, hop)
        qg = det.debug(rise.DBG_IMAGE_U8, T, N)
        _, qr, _ = oracle.detect(cap.iq, N, hop)
        d = qg.astype(np.int16) - qr.astype(np.int16)
        assert np.abs(d).max(initial=0) <= 1
        px += qg.size
        diff += int(np.count_nonzero(d))
    assert px > 10_000_000
    assert diff <= 1e-5 * px, f"{diff} of {px} pixels differ ({diff / px:.2e})"


def _image_stage_check(det, q, thr_g, thr_r):
    rise = _rise()
    det.set_option(rise.OPT_KEEP_MASKS, 1)
    T, F = q.shape
    boxes_g = det.detect_image(torch.from_numpy(q).cuda(), thr_g)
    boxes_r, ex = oracle.detect_image(q, thr_r, extras=True)
    hist_g = det.debug(rise.DBG_HIST, T, F)
    assert np.array_equal(hist_g, ex["hist"])
    cols = det.debug(rise.DBG_COLSTATS, T, F)
    st = oracle.column_thresholds(ex["hist"], T, thr_r)
    assert np.array_equal(cols["S"], st["S"])
    assert np.array_equal(cols["Shat"], st["Shat"])
    assert np.array_equal(cols["keep"], st["keep"].astype(np.int32))
    assert np.array_equal(cols["otsu"], st["otsu"])
    assert np.array_equal(cols["eff"], st["eff"])
    fl = det.debug(rise.DBG_FLOOR, T, F)
    assert fl[:5].tolist() == [st["N0"], st["delta_psd"], st["delta_pow"], st["P_q"], st["D"]]
    M0 = oracle.threshold(q, st["eff"])
    M1, M2, M3 = oracle.morph_chain(M0, thr_r.morph_order)
    for what, ref in ((rise.DBG_MASK0, M0), (rise.DBG_MASK1, M1), (rise.DBG_MASK2, M2),
                      (rise.DBG_MASK3, M3)):
        got = rise.unpack_mask(det.debug(what, T, F), F)
        assert np.array_equal(got, ref), f"mask stage {what - rise.DBG_MASK0}"
    assert np.array_equal(boxes_g, boxes_r)
    return boxes_g


def test_image_path_bit_exact_on_oracle_images(det):
    cap = synth.single_capture(101)
    _, q, _ = oracle.detect(cap.iq, 1024, 1024)
    for kw in ({}, dict(morph_order=1), dict(sg_half_window=2, level_db=0.5),
               dict(psd_offset_db=-math.inf), dict(power_offset_db=-math.inf),
               dict(psd_offset_db=3.0, power_offset_db=4.0)):
        thr_g, thr_r = _thr_pair(**kw)
        _image_stage_check(det, q, thr_g, thr_r)


@pytest.mark.parametrize("T,F,seed", [(1, 256, 1), (2, 512, 2), (1000, 512, 3), (37, 8192, 4),
                                      (300, 2048, 5), (129, 256, 6), (5000, 256, 7)])
def test_image_path_random_structures(det, T, F, seed):
    rng = np.random.default_rng(seed)
    q = rng.integers(90, 150, size=(T, F)).astype(np.uint8)
    # blocks, stripes and speckle to exercise strips, merges and long components
    for _ in range(12):
        t0, f0 = rng.integers(0, T), rng.integers(0, F)
        q[t0:t0 + rng.integers(1, max(2, T // 3)), f0:f0 + rng.integers(1, F // 4)] = rng.integers(180, 256)
    q[:, rng.integers(0, F - 3):][:, :3] = 220                 # a full-height line
    q[rng.random((T, F)) < 0.01] = 250
    for kw in ({}, dict(psd_offset_db=-math.inf, power_offset_db=-math.inf), dict(morph_order=1)):
        thr_g, thr_r = _thr_pair(**kw)
        _image_stage_check(det, q, thr_g, thr_r)


def _stripes(T, F, seed):
    # 3-wide vertical stripes 3 apart (they survive closing and opening), cut
    # every 64 rows by a 3-row gap, on a flat background (a constant column has
    # no Otsu split): F/6 runs in most rows, so a strip holds more runs than
    # fit in shared memory
    rng = np.random.default_rng(seed)
    q = np.full((T, F), 50, np.uint8)
    cols = (np.arange(F) % 6) < 3
    rows = (np.arange(T) % 64) < 61
    q[np.ix_(rows, cols)] = rng.integers(200, 256, size=(rows.sum(), cols.sum()))
    return q


def test_dense_foreground_many_components(det):
    thr_g, thr_r = _thr_pair(psd_offset_db=-math.inf, power_offset_db=-math.inf)
    q = _stripes(2048, 4096, 12)
    b = _image_stage_check(det, q, thr_g, thr_r)
    assert b.shape[0] > 10000
    # uniform random levels: ~half the pixels pass Otsu, the closing joins them
    rng = np.random.default_rng(13)
    q = rng.integers(0, 256, size=(1024, 2048)).astype(np.uint8)
    _image_stage_check(det, q, thr_g, thr_r)


def test_range_paths_and_fixed_anchor_agree(det):
    rise = _rise()
    cap = synth.make_capture(1 << 19, 100e6, 10, 33, fft_size=2048, hop=1024,
                             bw_hz=(1e6, 10e6), dur_s=(0.2e-3, 2e-3), snr_db=(5, 20))
    x = torch.from_numpy(cap.iq).cuda()
    T = oracle.num_frames(cap.iq.shape[0], 2048, 1024)
    out = {}
    for path in (1, 2):
        det.set_option(rise.OPT_RANGE_PATH, path)
        out[path] = (det.detect(x, 2048, 1024), det.debug(rise.DBG_IMAGE_U8, T, 2048).copy())
    det.set_option(rise.OPT_RANGE_PATH, 0)
    assert np.array_equal(out[1][0], out[2][0]) and np.array_equal(out[1][1], out[2][1])
    # a fixed anchor at 3 dB below the max clips the top levels
    Mg = float(det.debug(rise.DBG_MAXPOW, T, 2048)[0])
    hi = oracle.hi_db_of(Mg) - 3.0
    thr_g, thr_r = _thr_pair(range_mode=1, hi_db=hi)
    bg = det.detect(x, 2048, 1024, thr_g)
    qg = det.debug(rise.DBG_IMAGE_U8, T, 2048)
    br, qr, _ = oracle.detect(cap.iq, 2048, 1024, thr_r)
    _check_image(qg, qr)
    assert np.array_equal(bg, oracle.detect_image(qg, thr_r))


@pytest.mark.parametrize("N,hop,sched", [(8192, 2048, 2), (8192, 2048, 1), (8192, 2048, 0),
                                         (512, 256, 2), (512, 256, 1), (1024, 512, 0), (4096, 1024, 0)])
def test_every_epilogue_under_every_schedule(det, N, hop, sched):
    """The four STFT epilogues under each radix schedule: range path 1 (the
    anchor from a store-free MAX pass, then the QUANT pass writing the 8-bit
    image) against path 2 (POWER, then the quantising histogram), bit for
    bit; a fixed range with the float power kept (QUANT_POWER) against the
    oracle: power within the float bar, image within one level, boxes equal
    to the oracle on the GPU image."""
    rise = _rise()
    n = N * 40 + hop // 3
    cap = synth.make_capture(n, 50e6, 8, 900 + N + sched, fft_size=N, hop=hop,
                             bw_hz=(0.5e6, 8e6), dur_s=(n / 50e6 / 20, n / 50e6 / 4), snr_db=(5, 25),
                             tone_fraction=0.3)
    x = torch.from_numpy(cap.iq).cuda()
    T = oracle.num_frames(n, N, hop)
    det.set_option(rise.OPT_FFT_SCHEDULE, sched)
    try:
        out = {}
        for path in (1, 2):
            det.set_option(rise.OPT_RANGE_PATH, path)
            out[path] = (det.detect(x, N, hop), det.debug(rise.DBG_IMAGE_U8, T, N).copy(),
                         float(det.debug(rise.DBG_MAXPOW, T, N)[0]))
        det.set_option(rise.OPT_RANGE_PATH, 0)
        for a, b in zip(out[1], out[2]):
            assert np.array_equal(a, b)
        hi = oracle.hi_db_of(out[2][2]) - 2.0
        thr_g, thr_r = _thr_pair(range_mode=1, hi_db=hi)
        det.set_option(rise.OPT_KEEP_POWER, 1)
        bg = det.detect(x, N, hop, thr_g)
        Pg = det.debug(rise.DBG_POWER_F32, T, N)
        qg = det.debug(rise.DBG_IMAGE_U8, T, N)
    finally:
        det.set_option(rise.OPT_KEEP_POWER, 0)
        det.set_option(rise.OPT_RANGE_PATH, 0)
        det.set_option(rise.OPT_FFT_SCHEDULE, 3)
    _check_power(Pg, oracle.stft_power(cap.iq, N, hop))
    _, qr, _ = oracle.detect(cap.iq, N, hop, thr_r)
    _check_image(qg, qr)
    assert np.array_equal(bg, oracle.detect_image(qg, thr_r))


def test_degenerate_inputs(det):
    rise = _rise()
    # all-zero capture: every level 0, no boxes
    z = np.zeros(1 << 14, np.complex64)
    b = _gpu_detect(det, z, 1024, 512)
    assert b.shape == (0, 8)
    q = det.debug(rise.DBG_IMAGE_U8, oracle.num_frames(1 << 14, 1024, 512), 1024)
    assert not q.any()
    # constant image: no Otsu split anywhere
    img = torch.full((64, 256), 77, dtype=torch.uint8, device="cuda")
    assert det.detect_image(img).shape == (0, 8)



def test_hand_block_image_closed_form(det):
    """The image of hand_images.block_image through the CUDA path: noise
    floor, offsets, power floor, per-column thresholds, final mask and box
    against values worked out by hand, not against the oracle."""
    import hand_images
    rise = _rise()
    q, want, want_boxes = hand_images.block_image(256)
    det.set_option(rise.OPT_KEEP_MASKS, 1)
    T, F = q.shape
    boxes = det.detect_image(torch.from_numpy(q).cuda())
    fl = det.debug(rise.DBG_FLOOR, T, F)
    assert fl[:5].tolist() == [want["N0"], want["delta_psd"], want["delta_pow"], want["P_q"], want["D"]]
    cols = det.debug(rise.DBG_COLSTATS, T, F)
    assert np.array_equal(cols["eff"], want["eff"])
    assert np.array_equal(rise.unpack_mask(det.debug(rise.DBG_MASK3, T, F), F), want["mask"])
    assert np.array_equal(boxes, want_boxes)

def test_truncation_and_invalid_arguments(det):
    rise = _rise()
    q = _stripes(512, 1024, 3)
    thr_g, thr_r = _thr_pair(psd_offset_db=-math.inf, power_offset_db=-math.inf)
    full = oracle.detect_image(q, thr_r)
    assert full.shape[0] > 10
    img = torch.from_numpy(q).cuda()
    det._auto_grow = False
    try:
        part = det.detect_image(img, thr_g, cap=7)
        assert det.last_status == rise.RISE_ETRUNC
        assert np.array_equal(part, full[:7])
    finally:
        det._auto_grow = True
    x = torch.zeros(5000, dtype=torch.complex64, device="cuda")
    for args in ((x, 1000, 500), (x, 128, 64), (x, 16384, 100), (x, 1024, 0), (x, 1024, 1025),
                 (x[:1000], 1024, 512)):
        with pytest.raises(rise.RiseError) as e:
            det.detect(*args)
        assert e.value.code == rise.RISE_EINVAL
    with pytest.raises(rise.RiseError):
        det.detect(x, 1024, 512, rise.default_thresholds(level_db=0.0))
    with pytest.raises(rise.RiseError):
        det.detect(x, 1024, 512, rise.default_thresholds(morph_order=2))


def test_single_capture_full_config(det):
    # 2^20 samples, FFT 1024, hop 1024: the whole path against the oracle
    cap = synth.single_capture(101)
    boxes_g = _gpu_detect(det, cap.iq, 1024, 1024, keep=False)
    boxes_r, qr, _ = oracle.detect(cap.iq, 1024, 1024)
    qg = det.debug(_rise().DBG_IMAGE_U8, 1024, 1024)
    nd = _check_image(qg, qr)
    assert np.array_equal(boxes_g, oracle.detect_image(qg))
    if nd == 0:
        assert np.array_equal(boxes_g, boxes_r)


def test_host_entry_point_matches_device_entry_point(det):
    cap = synth.single_capture(102)
    bd = _gpu_detect(det, cap.iq, 1024, 512, keep=False)
    pinned = torch.from_numpy(cap.iq).pin_memory()
    bh = det.detect_host(pinned, 1024, 512)
    assert np.array_equal(bd, bh)


@pytest.mark.slow
def test_wideband_full_size_sampled(det):
    """2^26 samples, FFT 4096, hop 2048 (the bench workload, same launch path):
    sampled frames against the oracle's spectrogram, the full image within the
    quantisation budget, and boxes bit-exact against the oracle on the GPU image."""
    rise = _rise()
    cap = synth.wideband_capture(102)
    N, hop = 4096, 2048
    T = oracle.num_frames(cap.iq.shape[0], N, hop)
    det.set_option(rise.OPT_KEEP_POWER, 0)
    det.set_option(rise.OPT_KEEP_MASKS, 0)
    x = torch.from_numpy(cap.iq).cuda()
    boxes_g = det.detect(x, N, hop)
    qg = det.debug(rise.DBG_IMAGE_U8, T, N)
    Mg = float(det.debug(rise.DBG_MAXPOW, T, N)[0])
    boxes_r, qr, Mr = oracle.detect(cap.iq, N, hop)
    assert abs(Mg - Mr) <= 1e-5 * Mr
    # the whole 32767 x 4096 image within the level budget
    d = qg.astype(np.int16) - qr.astype(np.int16)
    assert np.abs(d).max() <= 1
    assert np.count_nonzero(d) <= 1e-5 * d.size
    # sampled frames: the spectrogram itself within tolerance
    rng = np.random.default_rng(0)
    det.set_option(rise.OPT_KEEP_POWER, 1)
    det.detect(x, N, hop)
    Pg_rows = det.debug(rise.DBG_POWER_F32, T, N)
    det.set_option(rise.OPT_KEEP_POWER, 0)
    for t in np.unique(np.concatenate([[0, T - 1], rng.integers(0, T, 30)])):
        _check_power(Pg_rows[t:t + 1], oracle.stft_power(cap.iq, N, hop, int(t), 1))
    # from the image on, bit-exact
    assert np.array_equal(boxes_g, oracle.detect_image(qg))


@pytest.mark.slow
def test_stress_full_size_sampled(det):
    """2^28 samples, FFT 8192, hop 2048 (T = 131069, 1.07 G pixels; 1024
    emitters, half of them fragmented, 16 running the whole capture): the
    anchor and sampled frames against the oracle's spectrogram and levels, and
    boxes bit-exact against the oracle on the GPU's own image."""
    rise = _rise()
    cap = synth.stress_capture(105)
    N, hop = 8192, 2048
    T = oracle.num_frames(cap.iq.shape[0], N, hop)
    det.set_option(rise.OPT_KEEP_POWER, 1)
    det.set_option(rise.OPT_KEEP_MASKS, 0)
    x = torch.from_numpy(cap.iq).cuda()
    boxes_g = det.detect(x, N, hop)
    del x
    qg = det.debug(rise.DBG_IMAGE_U8, T, N)
    Pg = det.debug(rise.DBG_POWER_F32, T, N)
    Mg = float(det.debug(rise.DBG_MAXPOW, T, N)[0])
    det.set_option(rise.OPT_KEEP_POWER, 0)
    # the anchor is the largest float power, and the oracle agrees on its value
    arg = int(np.argmax(Pg))
    ta, fa = divmod(arg, N)
    assert Pg.flat[arg] == Mg
    Pa = oracle.stft_power(cap.iq, N, hop, ta, 1)[0]
    assert abs(Pa[fa] - Mg) <= 1e-4 * Pa[fa]
    hi = oracle.hi_db_of(Pa[fa])
    # sampled frames (the anchor's frame, both ends, random ones): power and levels
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([[0, ta, T - 1], rng.integers(0, T, 200)]))
    px = diff = 0
    for t in rows:
        Pr = oracle.stft_power(cap.iq, N, hop, int(t), 1)
        _check_power(Pg[t:t + 1], Pr)
        # the GPU's levels are the quantiser on its own float power and anchor
        assert np.array_equal(qg[t:t + 1], oracle.quantize(Pg[t:t + 1].astype(np.float64),
                                                           oracle.hi_db_of(Mg)))
        d = qg[t:t + 1].astype(np.int16) - oracle.quantize(Pr, hi).astype(np.int16)
        assert np.abs(d).max(initial=0) <= 1
        px += d.size
        diff += int(np.count_nonzero(d))
    assert diff <= math.ceil(1e-5 * px) + 6, f"{diff} of {px} sampled pixels differ"
    del Pg
    # from the image on, bit-exact (the oracle labels the whole 1.07 G-pixel image)
    boxes_r = oracle.detect_image(qg)
    assert len(boxes_g) > 1000
    assert np.array_equal(boxes_g, boxes_r)


def test_repeated_calls_replay_a_graph(det):
    """The third identical call replays the captured launches; its boxes and
    intermediates equal a context with graphs off, and changed arguments
    (thresholds, another buffer) are not served from the old graph."""
    rise = _rise()
    cap = synth.single_capture(104)
    N, hop = 1024, 512
    x = torch.from_numpy(cap.iq).cuda()
    det.set_option(rise.OPT_KEEP_POWER, 0)
    det.set_option(rise.OPT_KEEP_MASKS, 0)
    with rise.Detector(0) as d0:
        d0.set_option(rise.OPT_GRAPH, 0)
        want = d0.detect(x, N, hop)
        thr = rise.default_thresholds(power_offset_db=6.0)
        want6 = d0.detect(x, N, hop, thr)
        assert d0.graph_info()[0] == 0
    got = [det.detect(x, N, hop) for _ in range(3)]
    assert det.graph_info()[0] == 1
    for g in got:
        np.testing.assert_array_equal(g, want)
    g6 = det.detect(x, N, hop, thr)
    assert det.graph_info()[0] == 0
    np.testing.assert_array_equal(g6, want6)
    # same shape, new contents in the same buffer: the replay reads them
    cap2 = synth.single_capture(105)
    x.copy_(torch.from_numpy(cap2.iq))
    with rise.Detector(0) as d0:
        d0.set_option(rise.OPT_GRAPH, 0)
        want2 = d0.detect(x, N, hop)
    for _ in range(3):
        got2 = det.detect(x, N, hop)
    assert det.graph_info()[0] == 1
    np.testing.assert_array_equal(got2, want2)
