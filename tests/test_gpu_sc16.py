"""16-bit integer I/Q (sc16) input.

A sc16 sample (I, Q) means (I + iQ) * 2^-15, which float represents exactly,
so the sc16 path must give bit-identical spectra, images and boxes to the
complex64 path on the same samples (whose parity with the oracle is checked
in test_gpu_parity.py) -- from device or host memory, with the staged and
the direct frame loads.
"""
import numpy as np
import pytest

import oracle
from paper_2603_20481_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _sc16(iq, seed=0):
    """Quantise to int16 (a radio's sc16) and the exactly equal complex64."""
    peak = max(np.abs(iq.real).max(), np.abs(iq.imag).max())
    s = 0.7 * 32767.0 / peak
    q = np.empty((iq.shape[0], 2), np.int16)
    q[:, 0] = np.round(iq.real * s)
    q[:, 1] = np.round(iq.imag * s)
    f = (q[:, 0].astype(np.float32) + 1j * q[:, 1].astype(np.float32)) * np.float32(2.0 ** -15)
    return q, f.astype(np.complex64)


def _run(det, iq, N, hop):
    from paper_2603_20481_gb300 import rise
    det.set_option(rise.OPT_KEEP_POWER, 1)
    det.submit(iq, N, hop)
    b = det.collect()
    T = (iq.shape[0] - N) // hop + 1
    return b, det.debug(rise.DBG_POWER_F32, T, N), det.debug(rise.DBG_IMAGE_U8, T, N)


@pytest.mark.parametrize("N,hop,n,sched", [(1024, 512, 1 << 20, 1), (4096, 2048, 1 << 21, 1),
                                           (256, 129, 50000, 1), (2048, 1000, 300001, 1),
                                           (2048, 1000, 300001, 0), (8192, 2048, 1 << 19, 1),
                                           (8192, 2048, 1 << 19, 2), (512, 257, 70001, 2)])
def test_sc16_equals_complex64_on_the_same_samples(det, N, hop, n, sched):
    from paper_2603_20481_gb300 import rise
    cap = synth.make_capture(n, 50e6, 12, 300 + N, fft_size=N, hop=hop,
                             bw_hz=(0.5e6, 5e6), dur_s=(n / 50e6 / 20, n / 50e6 / 4),
                             snr_db=(5, 25))
    q, f = _sc16(cap.iq)
    det.set_option(rise.OPT_FFT_SCHEDULE, sched)   # the same radix schedule for both inputs
    try:
        want = _run(det, torch.from_numpy(f).cuda(), N, hop)
        for src in (torch.from_numpy(q).cuda(), torch.from_numpy(q).pin_memory(), q):
            got = _run(det, src, N, hop)
            for g, w in zip(got, want):
                np.testing.assert_array_equal(g, w)
    finally:
        det.set_option(rise.OPT_FFT_SCHEDULE, 3)
    assert len(want[0]) > 0


def test_sc16_against_the_oracle(det):
    cap = synth.single_capture(121)
    q, f = _sc16(cap.iq)
    boxes, _, img = _run(det, torch.from_numpy(q).cuda(), 1024, 1024)
    _, qr, _ = oracle.detect(f, 1024, 1024)
    d = img.astype(np.int16) - qr.astype(np.int16)
    assert np.abs(d).max() <= 1 and np.count_nonzero(d) <= 16
    np.testing.assert_array_equal(boxes, oracle.detect_image(img))


def test_sc16_alignment_is_checked(det):
    from paper_2603_20481_gb300 import rise
    q, _ = _sc16(synth.single_capture(122).iq)
    t = torch.from_numpy(q).cuda().view(-1)[1:-1]            # 2-byte aligned start
    assert t.data_ptr() % 4 == 2
    rc = rise.lib().rise_submit(det._h, __import__("ctypes").c_void_p(t.data_ptr()), rise.IQ_SC16,
                                t.numel() // 2, 1024, 1024, None, 16)
    assert rc == rise.RISE_EINVAL
    rc = rise.lib().rise_submit(det._h, __import__("ctypes").c_void_p(q.ctypes.data), 8,
                                q.shape[0], 1024, 1024, None, 16)
    assert rc == rise.RISE_EINVAL                             # unknown flag
