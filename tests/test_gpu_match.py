"""rise_match_boxes (Eqs. 2-3 on the GPU) against the oracle's exhaustive
count: best (intersection, union) of every box, N_t and N_f, bit-exact, on
random sets larger than one staged tile and on real detections against the
planted emitters; P_d rises with SNR on a sweep."""
import numpy as np
import pytest

import oracle
from paper_2603_20481_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

THETAS = [0.0, 0.1, 0.25, 1.0 / 3.0, 0.4, 0.5, 0.75, 0.9, 1.0]


def _rand(rng, n, T=2000, F=1024):
    t0 = rng.integers(0, T, n)
    f0 = rng.integers(0, F, n)
    return np.stack([t0, t0 + rng.integers(0, 200, n), f0, f0 + rng.integers(0, 120, n)], 1)


def _check(det, gt, d):
    got = det.match(gt, d, THETAS)
    want = oracle.match(gt, d, THETAS)
    for k in ("n_t", "n_f", "gt_best", "det_best"):
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)
    return got


@pytest.mark.parametrize("ng,nd", [(0, 5), (7, 0), (1, 1), (300, 2500), (2600, 1700)])
def test_random_sets_match_the_oracle(det, ng, nd):
    rng = np.random.default_rng(ng * 7 + nd)
    gt = _rand(rng, ng).reshape(-1, 4)
    d = _rand(rng, nd).reshape(-1, 4)
    if ng and nd:
        d[: min(ng, nd) // 3] = gt[: min(ng, nd) // 3]     # exact hits: IoU 1
    _check(det, gt, d)


def test_ties_at_the_threshold(det):
    a = np.array([[0, 9, 0, 9]])
    d = np.array([[0, 4, 0, 9], [0, 9, 0, 9], [50, 51, 50, 51]])
    r = _check(det, a, d)
    i = THETAS.index(0.5)
    assert r["n_t"][i] == 1 and r["n_f"][i] == 1       # the half box is neither at 1/2


def test_invalid_arguments(det):
    from paper_2603_20481_gb300 import rise
    with pytest.raises(rise.RiseError):
        det.match(np.array([[5, 4, 0, 1]]), np.zeros((0, 4)), [0.5])   # empty box
    with pytest.raises(rise.RiseError):
        det.match(np.zeros((0, 4)), np.zeros((0, 4)), [1.5])


def test_detections_against_planted_emitters_and_snr_sweep(det):
    pd = []
    for snr in (0.0, 6.0, 12.0, 18.0):
        caps = [synth.make_capture(1 << 20, 20e6, 10, 777 + k, fft_size=1024, hop=512,
                                   bw_hz=(1e6, 4e6), dur_s=(2e-3, 10e-3), snr_db=(snr, snr),
                                   tone_fraction=0.0) for k in range(3)]
        nt = ng = 0
        for cap in caps:
            boxes = det.detect(torch.from_numpy(cap.iq).cuda(), 1024, 512)
            gt = np.array(synth.gt_boxes(cap), dtype=np.int64).reshape(-1, 4)
            r = _check(det, gt, boxes)
            nt += r["n_t"][THETAS.index(0.5)]
            ng += gt.shape[0]
        pd.append(nt / ng)
    assert pd[-1] > 0.7 and pd[-1] >= pd[0]
