"""Seeded synthetic IQ captures with planted emitters.

This module only generates inputs.  It draws complex white Gaussian noise,
pure tones and band-limited noise bursts, adds them into one complex64
capture, and reports where it planted each emitter.  None of the detection
method's arithmetic (windowing, STFT, quantisation, thresholds, morphology,
labelling) lives here, so the CUDA path and the FP64 oracle can both take
their inputs from it without sharing any of the method.

The emitters stand in for the paper's RFSynth / over-the-air captures
(Sec. V, "Signal generation"), which are not available: the shapes follow
the paper's scenarios (narrowband bursts a few MHz wide, wideband bursts
tens of MHz wide, time-gated transmissions) and the SNR convention of
Sec. VI-A-2 (signal power over noise power in the occupied bandwidth).

Noise has unit power, E|x|^2 = 1, spread over the whole sampled band.
* burst: white complex noise band-limited to [f_lo, f_hi] by masking its
  DFT; in-band power = SNR * (f_hi - f_lo) / fs, i.e. SNR over the noise
  that falls in the same bandwidth.
* tone: A * exp(2*pi*i*f*t/fs + phi) with A^2 = SNR / fft_size, i.e. SNR
  against the noise that falls in one FFT bin.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

try:  # scipy's pocketfft takes complex64 natively and threads
    import scipy.fft as _fft

    def _inv(x):
        return _fft.ifft(x, workers=-1)

    def _fast_len(n):
        return _fft.next_fast_len(n)
except Exception:  # pragma: no cover - numpy fallback for the generator only
    def _inv(x):
        return np.fft.ifft(x).astype(np.complex64)

    def _fast_len(n):
        return 1 << max(0, (n - 1).bit_length())


@dataclass
class Emitter:
    kind: str                 # "tone" or "burst"
    start: int                # first sample, inclusive
    stop: int                 # one past the last sample
    f_lo_hz: float            # occupied band, Hz, baseband (-fs/2 .. fs/2)
    f_hi_hz: float
    snr_db: float
    gaps: List[Tuple[int, int]] = field(default_factory=list)  # muted [a, b) ranges

    def segments(self) -> List[Tuple[int, int]]:
        """Sample ranges in which the emitter is on (its fragments)."""
        segs, cur = [], self.start
        for a, b in sorted(self.gaps):
            if a > cur:
                segs.append((cur, a))
            cur = max(cur, b)
        if cur < self.stop:
            segs.append((cur, self.stop))
        return segs


@dataclass
class Capture:
    iq: np.ndarray            # complex64 [n]
    fs: float
    emitters: List[Emitter]
    seed: int
    fft_size: int
    hop: int


def _loguniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def _band_noise(rng, length: int, f_lo: float, f_hi: float, fs: float,
                power: float) -> np.ndarray:
    """Complex Gaussian noise with a flat spectrum on [f_lo, f_hi] Hz, scaled to
    `power`: independent Gaussian DFT coefficients on the in-band bins of a
    transform of fast length L >= length, inverse transform, first `length`
    samples (the DFT of white Gaussian noise is white Gaussian, so this is
    band-masked white noise drawn directly in the frequency domain)."""
    L = _fast_len(max(1, length))
    k0 = math.ceil(f_lo * L / fs)
    k1 = max(k0, math.floor(f_hi * L / fs))
    m = k1 - k0 + 1
    W = np.zeros(L, np.complex64)
    coef = rng.standard_normal((m, 2), dtype=np.float32).view(np.complex64).reshape(m)
    W[np.arange(k0, k1 + 1) % L] = coef
    b = _inv(W)[:length].astype(np.complex64)
    p = float(np.mean(np.abs(b) ** 2)) if length else 0.0
    if p > 0:
        b *= np.float32(math.sqrt(power / p))
    return b


def make_capture(n: int, fs: float, n_emitters: int, seed: int, *,
                 fft_size: int, hop: int,
                 bw_hz: Tuple[float, float] = (0.2e6, 5e6),
                 dur_s: Tuple[float, float] = (1e-3, 20e-3),
                 snr_db: Tuple[float, float] = (0.0, 20.0),
                 tone_fraction: float = 0.5,
                 fragment_fraction: float = 0.0,
                 fragments: Tuple[int, int] = (2, 20),
                 gap_frames: Tuple[int, int] = (1, 3),
                 full_length: int = 0,
                 full_length_bw_hz: Tuple[float, float] = (20e3, 200e3)) -> Capture:
    """One capture of `n` complex64 samples at `fs` with planted emitters.

    Start times and centre frequencies are uniform; durations and
    bandwidths are log-uniform in their ranges; SNR is uniform in dB.
    `fragment_fraction` of the bursts are gated into 2..20 fragments whose
    gaps last `gap_frames` hops; `full_length` extra narrowband bursts run
    over the whole capture.
    """
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal((n, 2), dtype=np.float32)
         * np.float32(math.sqrt(0.5))).view(np.complex64).reshape(n)
    emitters: List[Emitter] = []
    n_tones = int(round(n_emitters * tone_fraction))
    for i in range(n_emitters + full_length):
        full = i >= n_emitters
        kind = "tone" if (i < n_tones) else "burst"
        if full:
            length = n
            start = 0
        else:
            length = int(min(n, max(16, round(_loguniform(rng, *dur_s) * fs))))
            start = int(rng.integers(0, max(1, n - length + 1)))
        snr = float(rng.uniform(*snr_db))
        snr_lin = 10.0 ** (snr / 10.0)
        if kind == "tone":
            fc = float(rng.uniform(-0.45 * fs, 0.45 * fs))
            amp = math.sqrt(snr_lin / fft_size)
            ph = float(rng.uniform(0, 2 * math.pi))
            t = np.arange(length, dtype=np.float64)
            sig = (amp * np.exp(1j * (2 * math.pi * fc / fs * t + ph))).astype(np.complex64)
            em = Emitter("tone", start, start + length, fc, fc, snr)
        else:
            bw = float(_loguniform(rng, *(full_length_bw_hz if full else bw_hz)))
            bw = min(bw, 0.9 * fs)
            fc = float(rng.uniform(-0.5 * fs + bw / 2, 0.5 * fs - bw / 2))
            sig = _band_noise(rng, length, fc - bw / 2, fc + bw / 2, fs,
                              snr_lin * bw / fs)
            em = Emitter("burst", start, start + length, fc - bw / 2, fc + bw / 2, snr)
            if (not full) and fragment_fraction > 0 and rng.uniform() < fragment_fraction:
                k = int(rng.integers(fragments[0], fragments[1] + 1))
                cuts = np.sort(rng.integers(1, max(2, length - 1), size=k - 1))
                for c in cuts:
                    g = int(rng.integers(gap_frames[0], gap_frames[1] + 1)) * hop
                    a = int(c)
                    b = min(length, a + g)
                    sig[a:b] = 0
                    em.gaps.append((start + a, start + b))
        x[start:start + length] += sig
        emitters.append(em)
    return Capture(iq=x, fs=fs, emitters=emitters, seed=seed, fft_size=fft_size, hop=hop)


def gt_boxes(cap: Capture, fft_size: Optional[int] = None,
             hop: Optional[int] = None) -> List[Tuple[int, int, int, int]]:
    """Ground-truth boxes (t0, t1, f0, f1), inclusive, one per fragment.

    Rows are the frames that overlap the fragment by at least half a frame;
    columns are the frequency cells (DC at column N/2) whose centre lies in
    the emitter's band (a tone is given +-1 cell).
    """
    N = fft_size or cap.fft_size
    H = hop or cap.hop
    n = cap.iq.shape[0]
    T = (n - N) // H + 1
    out = []
    for em in cap.emitters:
        lo, hi = em.f_lo_hz, em.f_hi_hz
        if em.kind == "tone":
            lo -= cap.fs / N
            hi += cap.fs / N
        f = np.arange(N)
        centre = (f - N // 2) * cap.fs / N
        cols = np.nonzero((centre >= lo) & (centre <= hi))[0]
        if cols.size == 0:
            continue
        for a, b in em.segments():
            t = np.arange(max(0, a // H - 2), min(T, b // H + 2))
            ov = np.minimum(t * H + N, b) - np.maximum(t * H, a)
            rows = t[ov >= N // 2]
            if rows.size:
                out.append((int(rows[0]), int(rows[-1]), int(cols[0]), int(cols[-1])))
    return out


# ---------------------------------------------------------------------------
# Named workloads (seeded)
# ---------------------------------------------------------------------------

def single_capture(seed: int = 101, n: int = 1 << 20) -> Capture:
    """2^20 samples at 20 MS/s, 8 emitters (4 tones, 4 bursts), FFT 1024, hop 1024."""
    return make_capture(n, 20e6, 8, seed, fft_size=1024, hop=1024,
                        bw_hz=(0.2e6, 5e6), dur_s=(1e-3, 20e-3), snr_db=(0.0, 20.0),
                        tone_fraction=0.5)


def wideband_capture(seed: int = 102, n: int = 1 << 26) -> Capture:
    """2^26 samples at 100 MS/s, 128 emitters, SNR -3..25 dB, 0.1-20 MHz, FFT 4096, hop 2048."""
    return make_capture(n, 100e6, 128, seed, fft_size=4096, hop=2048,
                        bw_hz=(0.1e6, 20e6), dur_s=(0.5e-3, 20e-3), snr_db=(-3.0, 25.0),
                        tone_fraction=0.25)


def stress_capture(seed: int = 105, n: int = 1 << 28) -> Capture:
    """2^28 samples, FFT 8192 / hop 2048, 1024 emitters at -5..10 dB, half fragmented,
    plus 16 full-length narrowband emitters."""
    return make_capture(n, 100e6, 1024, seed, fft_size=8192, hop=2048,
                        bw_hz=(0.1e6, 10e6), dur_s=(0.2e-3, 5e-3), snr_db=(-5.0, 10.0),
                        tone_fraction=0.1, fragment_fraction=0.5, fragments=(2, 20),
                        gap_frames=(1, 3), full_length=16)


def batched_captures(count: int = 256, seed0: int = 1000,
                     sizes: Sequence[int] = (256, 512, 1024, 2048),
                     n_range: Tuple[int, int] = (1 << 16, 1 << 22)) -> List[Capture]:
    """`count` captures of log-uniform length, FFT size drawn per capture, hop = N/2,
    4..64 emitters each (seed of capture i = seed0 + i)."""
    caps = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(round(_loguniform(rng, *n_range)))
        N = int(rng.choice(np.asarray(sizes)))
        n = max(n, N)
        k = int(rng.integers(4, 65))
        fs = 100e6
        dur = (max(16, n // 64) / fs, max(32, n // 2) / fs)
        caps.append(make_capture(n, fs, k, seed0 + 100000 + i, fft_size=N, hop=N // 2,
                                 bw_hz=(0.2e6, 20e6), dur_s=dur, snr_db=(0.0, 20.0),
                                 tone_fraction=0.25))
    return caps


def served_chunk(stream: int, k: int, n: int = 614400, fs: float = 61.44e6,
                 fft_size: int = 2048, hop: int = 1024) -> Capture:
    """Chunk k of radio `stream`: 10 ms at 61.44 MS/s (seed 4000 + 64*stream + k)."""
    seed = 4000 + 64 * stream + k
    rng = np.random.default_rng(seed)
    m = int(rng.integers(2, 9))
    return make_capture(n, fs, m, seed + 7919, fft_size=fft_size, hop=hop,
                        bw_hz=(0.2e6, 20e6), dur_s=(0.2e-3, 8e-3), snr_db=(0.0, 20.0),
                        tone_fraction=0.25)
