"""Images whose detection is worked out by hand from Sec. IV-B (shared by the
oracle's pin and the GPU check of the same image)."""
from decimal import Decimal, getcontext

import numpy as np


def block_image(F: int):
    """A 64 x F image of level 100 with a 10 x 10 block of level 200 at rows
    10..19, columns 30..39, and what the default thresholds make of it:

    - column sums S_f: 64 * 100 = 6400 off the block, 54 * 100 + 10 * 200 =
      7400 on it;
    - quadratic SG (m = 5, c = 267, 252, 207, 132, 27, -108, D = 1287)
      leaves a flat run at D * 6400 and dips where only the -108 tap reaches
      the block (f = 25 and f = 44): N0 = 1287 * 6400 - 108 * 1000;
    - with the default offsets (0.5 dB and 10 dB at 0.25 dB a level),
      Delta_psd = 2 * D * T and Delta_pow = 40 * D * T; only the block's
      columns reach N0 + Delta_psd;
    - P_q = ceil((N0 + Delta_pow) / (D T)) = ceil(138.69) = 139;
    - Otsu on a block column: every split between 100 and 199 scores the
      same, the smallest wins (theta = 100), so eff = max(101, 139) = 139;
    - the MOs leave a solid 10 x 10 block unchanged: one component, whose
      energy is 100 pixels of round(2^32 * 10^((200 - 255) * 0.25 / 10)).

    Returns (q, expected dict, expected boxes int64 [1, 8]).
    """
    T = 64
    q = np.full((T, F), 100, np.uint8)
    q[10:20, 30:40] = 200
    D = 1287
    N0 = D * 6400 - 108 * 1000
    dpsd, dpow = 2 * D * T, 40 * D * T
    P_q = -(-(N0 + dpow) // (D * T))
    assert P_q == 139
    eff = np.full(F, 256, np.int32)
    eff[30:40] = 139
    mask = np.zeros((T, F), np.uint8)
    mask[10:20, 30:40] = 1
    getcontext().prec = 50
    e200 = int((Decimal(2) ** 32 * (Decimal(10) ** (Decimal(200 - 255) * Decimal("0.25") / 10)))
               .to_integral_value())
    boxes = np.array([[10, 19, 30, 39, 10 * F + 30, 100, 100 * 200, 100 * e200]], np.int64)
    want = dict(D=D, N0=N0, delta_psd=dpsd, delta_pow=dpow, P_q=P_q, eff=eff, mask=mask)
    return q, want, boxes
