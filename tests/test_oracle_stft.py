"""Pins of the oracle's STFT, power and 8-bit image (CPU only).

The oracle's FFT is checked against the DFT's definition evaluated by brute
force, against numpy's FFT, against Parseval's theorem and against the
closed-form spectrum of an on-bin tone under a periodic Hann window; the
quantiser against levels placed exactly at its boundaries.
"""
import math

import numpy as np
import pytest

import oracle


def _direct_dft(x):
    n = np.arange(x.shape[0])
    W = np.exp(-2j * np.pi * np.outer(n, n) / x.shape[0])
    return W @ x


@pytest.mark.parametrize("N", [1, 2, 4, 8, 16, 32, 64])
def test_fft_is_the_dft_by_brute_force(N):
    rng = np.random.default_rng(N)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    assert np.allclose(oracle.fft(x), _direct_dft(x), rtol=0, atol=1e-12 * max(1, N))


@pytest.mark.parametrize("N", [128, 256, 1024, 4096, 8192])
def test_fft_matches_numpy(N):
    rng = np.random.default_rng(7 + N)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    ref = np.fft.fft(x)
    assert np.max(np.abs(oracle.fft(x) - ref)) <= 1e-12 * np.sqrt(N) * np.max(np.abs(ref))


def test_fft_rejects_non_power_of_two():
    with pytest.raises(RuntimeError):
        oracle.fft(np.ones(12, complex))


def test_hann_is_periodic():
    N = 1024
    w = oracle.hann(N)
    assert w[0] == 0.0 and abs(w[N // 2] - 1.0) < 1e-15
    assert np.allclose(w[1:], w[1:][::-1], atol=1e-15)          # w[m] = w[N-m]
    assert abs(w.sum() - N / 2) < 1e-9                           # coherent gain 1/2
    assert abs((w ** 2).sum() - 3 * N / 8) < 1e-9                # energy 3N/8


@pytest.mark.parametrize("N", [256, 1024, 4096])
def test_parseval_per_frame(N):
    rng = np.random.default_rng(N)
    iq = (rng.standard_normal(3 * N) + 1j * rng.standard_normal(3 * N)).astype(np.complex64)
    hop = N // 2
    P = oracle.stft_power(iq, N, hop)
    w = oracle.hann(N)
    for t in range(P.shape[0]):
        seg = iq[t * hop:t * hop + N].astype(np.complex128) * w
        assert abs(P[t].sum() - N * np.sum(np.abs(seg) ** 2)) <= 1e-9 * P[t].sum()


@pytest.mark.parametrize("N,k0", [(256, 3), (1024, -100), (4096, 1000), (8192, 0)])
def test_on_bin_tone_under_hann_closed_form(N, k0):
    # x[m] = A exp(2 pi i k0 m / N): periodic Hann gives |X| = A N / 2 at k0,
    # A N / 4 at k0 +- 1 and zero elsewhere.
    A = 0.75
    m = np.arange(2 * N)
    iq = (A * np.exp(2j * np.pi * k0 * m / N)).astype(np.complex64)
    P = oracle.stft_power(iq.astype(np.complex64), N, N)
    col = (k0 % N + N // 2) % N       # DC sits in column N/2
    for row in P:
        assert abs(row[col] - (A * N / 2) ** 2) <= 1e-6 * (A * N / 2) ** 2
        for d in (-1, 1):
            c = (col + d) % N
            assert abs(row[c] - (A * N / 4) ** 2) <= 1e-6 * (A * N / 2) ** 2
        rest = np.delete(row, [col, (col - 1) % N, (col + 1) % N])
        assert rest.max() <= 1e-8 * (A * N / 2) ** 2   # float32 input rounding only


def test_frames_follow_the_hop_and_count():
    N, hop = 512, 200
    rng = np.random.default_rng(3)
    iq = (rng.standard_normal(5000) + 1j * rng.standard_normal(5000)).astype(np.complex64)
    T = oracle.num_frames(iq.shape[0], N, hop)
    assert T == (5000 - 512) // 200 + 1
    P = oracle.stft_power(iq, N, hop)
    assert P.shape == (T, N)
    # frame t is the window at sample t*hop: shifting the capture by one hop shifts the rows
    P2 = oracle.stft_power(iq[hop:], N, hop)
    assert np.array_equal(P[1:1 + P2.shape[0]], P2)
    # a constant (DC) capture puts all energy in column N/2
    dc = np.ones(N, np.complex64)
    Pdc = oracle.stft_power(dc, N, N)[0]
    assert Pdc.argmax() == N // 2
    assert oracle.num_frames(N - 1, N, 1) == 0


def test_quantiser_levels_at_exact_boundaries():
    lvl, hi = 0.25, 37.0
    # level j is reached exactly at dB = hi + (j - 255.5) * lvl
    js = np.arange(1, 256)
    edges = 10.0 ** ((hi + (js - 255.5) * lvl) / 10.0)
    above = oracle.quantize(edges * (1 + 1e-9), hi, lvl)
    below = oracle.quantize(edges * (1 - 1e-9), hi, lvl)
    assert np.array_equal(above.astype(int), js)
    assert np.array_equal(below.astype(int), js - 1)
    top = 10.0 ** (hi / 10.0)
    assert oracle.quantize(np.array([top, top * 1e6, 0.0, 1e-300]), hi, lvl).tolist() == [255, 255, 0, 0]


def test_quantiser_is_monotone():
    P = np.sort(np.random.default_rng(1).exponential(size=20000)) * 1e3
    q = oracle.quantize(P, 10 * math.log10(P.max()), 0.25)
    assert np.all(np.diff(q.astype(int)) >= 0) and q[-1] == 255


def test_energy_table_closed_form():
    E = oracle.energy_table(0.25)
    assert int(E[255]) == 1 << 32
    assert int(E[255 - 40]) == round(2 ** 32 / 10)      # -10 dB
    assert int(E[255 - 120]) == round(2 ** 32 / 1000)   # -30 dB
    exact = 2.0 ** 32 * 10.0 ** ((np.arange(256) - 255) * 0.25 / 10)
    assert np.all(np.abs(E.astype(np.float64) - exact) <= 0.5)
    # no entry sits near a rounding tie, so any faithful evaluation rounds alike
    frac = exact - np.floor(exact)
    assert np.all(np.abs(frac - 0.5) > 1e-4)
