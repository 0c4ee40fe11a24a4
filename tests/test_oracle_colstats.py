"""Pins of the oracle's column statistics (CPU only): Savitzky-Golay weights,
noise floor N0, theta_PSD pruning, Otsu's threshold and the power floor.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sg_quadratic_coeffs.txt")


def _golden_sg():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            v = [int(x) for x in line.split()]
            rows.append((v[0], v[1], v[2:]))
    return rows


@pytest.mark.parametrize("m,norm,w", _golden_sg())
def test_sg_weights_match_the_published_table(m, norm, w):
    c, D = oracle.sg_coeffs(m)
    # c / D must equal w / norm for every tap
    for i in range(m + 1):
        assert c[i] * norm == w[i] * D
    assert c[0] + 2 * c[1:].sum() == D


def _stats_for_S(S, T=1, m=5, **kw):
    """Column thresholds for a histogram whose column sums are exactly S."""
    F = len(S)
    hist = np.zeros((F, 256), np.uint32)
    # put T rows per column: realise sum S_f with levels in 0..255
    for f, s in enumerate(S):
        assert 0 <= s <= 255 * T
        full, rem = divmod(int(s), 255)
        hist[f, 255] += full
        if rem:
            hist[f, rem] += 1
        hist[f, 0] += T - full - (1 if rem else 0)
    return oracle.column_thresholds(hist, T, oracle.params(sg_half_window=m, **kw))


def test_sg_reproduces_quadratics_exactly():
    F, T, m = 64, 1000, 5
    f = np.arange(F)
    S = 3 * (f - 20) ** 2 + 7 * f + 1000
    st = _stats_for_S(S, T=T, m=m)
    D = st["D"]
    assert np.array_equal(st["Shat"][m:F - m], D * S[m:F - m])
    assert np.all(st["Shat"][:m] == 0) and np.all(st["Shat"][F - m:] == 0)


def test_noise_floor_is_lowest_local_minimum():
    F, T = 80, 400
    f = np.arange(F)
    # two dips: a shallow one at 20 and a deeper one at 55, both wide enough to survive smoothing
    S = 40000 - 8000 * np.exp(-((f - 20) / 4.0) ** 2) - 15000 * np.exp(-((f - 55) / 4.0) ** 2)
    S = np.round(S).astype(np.int64)
    st = _stats_for_S(S, T=T)
    Sh = st["Shat"]
    assert st["N0"] == Sh[5:F - 5].min() == Sh[55]
    # a monotone PSD has no interior local minimum: N0 falls back to the global minimum
    S2 = np.linspace(30000, 50000, F).round().astype(np.int64)
    st2 = _stats_for_S(S2, T=T)
    assert st2["N0"] == st2["Shat"][5]


def test_constant_psd_floor_and_pruning():
    F, T = 32, 100
    S = np.full(F, 130 * T, np.int64)
    st = _stats_for_S(S, T=T)
    D = st["D"]
    assert st["N0"] == D * 130 * T
    # +0.5 dB (the default) = 2 levels above the floor: a flat PSD is pruned everywhere
    assert st["delta_psd"] == 2 * D * T
    assert st["keep"].sum() == 0 and np.all(st["eff"] == 256)
    # -inf switches both thresholds off
    st = _stats_for_S(S, T=T, psd_offset_db=-np.inf, power_offset_db=-np.inf)
    assert st["keep"].sum() == F and st["P_q"] == 0


def _sigma_b(h):
    """Textbook between-class variance (Otsu 1979, Eq. 18) for every split theta."""
    v = np.arange(256, dtype=np.float64)
    p = h / h.sum()
    w0 = np.cumsum(p)
    mu_t = np.cumsum(v * p)
    mu_T = mu_t[-1]
    with np.errstate(divide="ignore", invalid="ignore"):
        sb = (mu_T * w0 - mu_t) ** 2 / (w0 * (1 - w0))
    sb[(w0 <= 0) | (w0 >= 1 - 1e-15)] = -1
    return sb[:255]


def test_otsu_matches_float_definition_on_random_histograms():
    rng = np.random.default_rng(11)
    for trial in range(300):
        h = np.zeros(256, np.uint32)
        k = rng.integers(2, 40)
        h[rng.integers(0, 256, size=k)] = rng.integers(1, 5000, size=k)
        sb = _sigma_b(h.astype(np.float64))
        th = oracle.otsu(h)
        if sb.max() < 0:
            assert th == -1
            continue
        best = sb.max()
        ties = np.nonzero(sb >= best * (1 - 1e-12))[0]
        assert th in ties
        assert th == ties.min() or sb[ties.min()] < best * (1 - 1e-14)


def test_otsu_tie_break_smallest_theta():
    h = np.zeros(256, np.uint32)
    h[50] = 1000
    h[200] = 1000
    # every theta in [50, 199] gives the same split, so the smallest wins
    assert oracle.otsu(h) == 50


def test_otsu_two_gaussian_modes():
    v = np.arange(256)
    h = (4000 * np.exp(-((v - 80) / 10.0) ** 2) + 1500 * np.exp(-((v - 170) / 8.0) ** 2)).round()
    th = oracle.otsu(h.astype(np.uint32))
    assert 100 <= th <= 150


def test_otsu_degenerate_columns():
    h = np.zeros(256, np.uint32)
    h[77] = 5000
    assert oracle.otsu(h) == -1                 # one occupied level: no split
    h[255] = 1
    assert oracle.otsu(h) == 77                 # the only split with both classes occupied
    assert oracle.otsu(np.zeros(256, np.uint32)) == -1


def test_thresholds_are_invariant_to_a_level_shift_and_to_stacking_rows():
    rng = np.random.default_rng(5)
    T, F = 300, 48
    q = rng.integers(60, 120, size=(T, F)).astype(np.uint8)
    q[100:180, 10:20] += 60        # a bright block
    q[:, 30:33] += 20
    base = oracle.column_thresholds(oracle.column_hist(q), T)
    # adding c to every level adds c to Otsu, the power floor and eff; pruning is unchanged
    c = 9
    sh = oracle.column_thresholds(oracle.column_hist(q + c), T)
    assert np.array_equal(sh["keep"], base["keep"])
    kept = base["keep"] == 1
    assert np.array_equal(sh["otsu"][kept], base["otsu"][kept] + c)
    assert sh["P_q"] == base["P_q"] + c
    assert np.array_equal(sh["eff"][kept], base["eff"][kept] + c)
    # stacking the image on itself doubles every count: nothing changes
    q2 = np.vstack([q, q])
    st = oracle.column_thresholds(oracle.column_hist(q2), 2 * T)
    for key in ("keep", "otsu", "eff"):
        assert np.array_equal(st[key], base[key])
    assert st["P_q"] == base["P_q"]
    # eff is 256 on pruned columns, else max(otsu + 1, P_q)
    e = base["eff"]
    assert np.all(e[~kept] == 256)
    ok = kept & (base["otsu"] >= 0)
    assert np.array_equal(e[ok], np.maximum(base["otsu"][ok] + 1, base["P_q"]))
