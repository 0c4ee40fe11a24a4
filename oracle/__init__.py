"""FP64 CPU oracle of the RISE IQ -> boxes path -- TEST INFRASTRUCTURE.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It shares no code with the CUDA
library (`paper_2603_20481_gb300`): the arithmetic lives in
`rise_oracle.c` (plain loops, double precision), and this module only
marshals numpy arrays into it.

Boxes come back as int64 arrays of shape (n, 8) with columns
(t0, t1, f0, f1, anchor, area, sum_q, energy_fx), rows in anchor order.
"""
from __future__ import annotations

import ctypes as C
import math
from typing import Dict, Optional, Tuple

import numpy as np

from . import build as _build

RO_DILATE3, RO_ERODE3, RO_DILATE1x3, RO_ERODE1x3 = 0, 1, 2, 3
BOX_COLS = ("t0", "t1", "f0", "f1", "anchor", "area", "sum_q", "energy_fx")


class Params(C.Structure):
    _fields_ = [("range_mode", C.c_int), ("hi_db", C.c_double), ("level_db", C.c_double),
                ("psd_offset_db", C.c_double), ("power_offset_db", C.c_double),
                ("sg_half_window", C.c_int), ("morph_order", C.c_int)]


class _Box(C.Structure):
    _fields_ = [("t0", C.c_int32), ("t1", C.c_int32), ("f0", C.c_int32), ("f1", C.c_int32),
                ("anchor", C.c_int64), ("area", C.c_int64), ("sum_q", C.c_uint64),
                ("energy_fx", C.c_uint64)]


_BOX_DTYPE = np.dtype([("t0", "<i4"), ("t1", "<i4"), ("f0", "<i4"), ("f1", "<i4"),
                       ("anchor", "<i8"), ("area", "<i8"), ("sum_q", "<u8"),
                       ("energy_fx", "<u8")])
assert _BOX_DTYPE.itemsize == C.sizeof(_Box) == 48

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        P = C.c_void_p
        i64, i32, dbl = C.c_int64, C.c_int, C.c_double
        sig = {
            "ro_fft": (i32, [P, P, i32]),
            "ro_hann": (None, [i32, P]),
            "ro_num_frames": (i64, [i64, i32, i32]),
            "ro_stft_power": (i32, [P, i64, i32, i32, i64, i64, P]),
            "ro_max_power": (i32, [P, i64, i32, i32, P]),
            "ro_quantize": (None, [P, i64, dbl, dbl, P]),
            "ro_energy_table": (None, [dbl, P]),
            "ro_column_hist": (None, [P, i64, i32, P]),
            "ro_sg_coeffs": (i32, [i32, P, P]),
            "ro_otsu": (i32, [P]),
            "ro_column_thresholds": (i32, [P, i64, i32, P, P, P, P, P, P, P]),
            "ro_threshold": (None, [P, i64, i32, P, P]),
            "ro_morph": (i32, [P, P, i64, i32, i32]),
            "ro_morph_chain": (i32, [P, i64, i32, i32, P, P, P]),
            "ro_ccl_boxes": (i32, [P, P, i64, i32, dbl, P, i64, P]),
            "ro_detect_image": (i32, [P, i64, i32, P, P, i64, P, P, P, P, P]),
            "ro_detect": (i32, [P, i64, i32, i32, P, P, i64, P, P, P]),
            "ro_match": (i32, [P, i64, P, i64, P, i32, P, P, P, P]),
            "ro_label": (i32, [P, i64, i32, P]),
            "ro_component_runs": (i32, [P, i64, i32, P, i64, P]),
            "ro_boundary": (None, [P, i64, i32, P]),
            "ro_set_threads": (i32, [i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def params(range_mode: int = 0, hi_db: float = 0.0, level_db: float = 0.25,
           psd_offset_db: float = 0.5, power_offset_db: float = 10.0,
           sg_half_window: int = 5, morph_order: int = 0) -> Params:
    """Detection parameters; the defaults are the documented ones."""
    return Params(range_mode, hi_db, level_db, psd_offset_db, power_offset_db,
                  sg_half_window, morph_order)


def _check(rc: int, what: str):
    if rc not in (0, -3):
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def set_threads(n: int) -> int:
    """Host threads of the oracle's parallel loops (n < 1: every core).
    Returns the count in effect (1 without OpenMP).  Results do not depend
    on it."""
    return int(lib().ro_set_threads(int(n)))


def fft(x: np.ndarray) -> np.ndarray:
    z = np.ascontiguousarray(x, dtype=np.complex128)
    re = np.ascontiguousarray(z.real)
    im = np.ascontiguousarray(z.imag)
    _check(lib().ro_fft(_p(re), _p(im), re.shape[0]), "fft")
    return re + 1j * im


def hann(N: int) -> np.ndarray:
    w = np.empty(N, np.float64)
    lib().ro_hann(N, _p(w))
    return w


def num_frames(n: int, N: int, hop: int) -> int:
    return int(lib().ro_num_frames(n, N, hop))


def _iq(iq: np.ndarray) -> np.ndarray:
    iq = np.ascontiguousarray(iq)
    if iq.dtype != np.complex64:
        raise TypeError("iq must be complex64")
    return iq


def stft_power(iq: np.ndarray, N: int, hop: int, t0: int = 0,
               nt: Optional[int] = None) -> np.ndarray:
    iq = _iq(iq)
    T = num_frames(iq.shape[0], N, hop)
    if nt is None:
        nt = T - t0
    P = np.empty((nt, N), np.float64)
    _check(lib().ro_stft_power(_p(iq), iq.shape[0], N, hop, t0, nt, _p(P)), "stft_power")
    return P


def max_power(iq: np.ndarray, N: int, hop: int) -> float:
    iq = _iq(iq)
    out = np.zeros(1, np.float64)
    _check(lib().ro_max_power(_p(iq), iq.shape[0], N, hop, _p(out)), "max_power")
    return float(out[0])


def quantize(P: np.ndarray, hi_db: float, level_db: float = 0.25) -> np.ndarray:
    P = np.ascontiguousarray(P, dtype=np.float64)
    q = np.empty(P.shape, np.uint8)
    lib().ro_quantize(_p(P), P.size, hi_db, level_db, _p(q))
    return q


def energy_table(level_db: float = 0.25) -> np.ndarray:
    E = np.empty(256, np.uint64)
    lib().ro_energy_table(level_db, _p(E))
    return E


def column_hist(q: np.ndarray) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.uint8)
    T, F = q.shape
    h = np.empty((F, 256), np.uint32)
    lib().ro_column_hist(_p(q), T, F, _p(h))
    return h


def sg_coeffs(m: int) -> Tuple[np.ndarray, int]:
    c = np.zeros(m + 1, np.int64)
    D = np.zeros(1, np.int64)
    _check(lib().ro_sg_coeffs(m, _p(c), _p(D)), "sg_coeffs")
    return c, int(D[0])


def otsu(h: np.ndarray) -> int:
    h = np.ascontiguousarray(h, dtype=np.uint32)
    assert h.shape == (256,)
    return int(lib().ro_otsu(_p(h)))


def column_thresholds(hist: np.ndarray, T: int, prm: Optional[Params] = None) -> Dict:
    prm = prm or params()
    hist = np.ascontiguousarray(hist, dtype=np.uint32)
    F = hist.shape[0]
    S = np.zeros(F, np.uint64)
    Sh = np.zeros(F, np.int64)
    keep = np.zeros(F, np.uint8)
    th = np.zeros(F, np.int32)
    eff = np.zeros(F, np.int32)
    info = np.zeros(5, np.int64)
    _check(lib().ro_column_thresholds(_p(hist), T, F, C.byref(prm), _p(S), _p(Sh), _p(keep),
                                      _p(th), _p(eff), _p(info)), "column_thresholds")
    return dict(S=S, Shat=Sh, keep=keep, otsu=th, eff=eff, N0=int(info[0]),
                delta_psd=int(info[1]), delta_pow=int(info[2]), P_q=int(info[3]),
                D=int(info[4]))


def threshold(q: np.ndarray, eff: np.ndarray) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.uint8)
    eff = np.ascontiguousarray(eff, dtype=np.int32)
    T, F = q.shape
    m = np.empty_like(q)
    lib().ro_threshold(_p(q), T, F, _p(eff), _p(m))
    return m


def morph(mask: np.ndarray, op: int) -> np.ndarray:
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    T, F = mask.shape
    out = np.empty_like(mask)
    _check(lib().ro_morph(_p(mask), _p(out), T, F, op), "morph")
    return out


def morph_chain(M0: np.ndarray, order: int = 0) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    M0 = np.ascontiguousarray(M0, dtype=np.uint8)
    T, F = M0.shape
    M1, M2, M3 = (np.empty_like(M0) for _ in range(3))
    _check(lib().ro_morph_chain(_p(M0), T, F, order, _p(M1), _p(M2), _p(M3)), "morph_chain")
    return M1, M2, M3


def _boxes_to_array(raw: np.ndarray, n: int) -> np.ndarray:
    out = np.empty((n, 8), np.int64)
    for j, name in enumerate(BOX_COLS):
        out[:, j] = raw[name][:n].astype(np.int64)
    return out


def ccl_boxes(mask: np.ndarray, q: np.ndarray, level_db: float = 0.25,
              cap: Optional[int] = None) -> np.ndarray:
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    q = np.ascontiguousarray(q, dtype=np.uint8)
    T, F = mask.shape
    cap = cap if cap is not None else max(16, (T * F + 1) // 2)
    raw = np.zeros(cap, _BOX_DTYPE)
    n = np.zeros(1, np.int64)
    rc = lib().ro_ccl_boxes(_p(mask), _p(q), T, F, level_db, _p(raw), cap, _p(n))
    _check(rc, "ccl")
    if rc == -3:
        raise RuntimeError(f"oracle box capacity {cap} too small ({int(n[0])} boxes)")
    return _boxes_to_array(raw, int(n[0]))


def _box_cap(T: int, F: int) -> int:
    return max(1024, min(T * F // 4 + 16, 1 << 24))


def detect_image(q: np.ndarray, prm: Optional[Params] = None, extras: bool = False):
    prm = prm or params()
    q = np.ascontiguousarray(q, dtype=np.uint8)
    T, F = q.shape
    cap = _box_cap(T, F)
    raw = np.zeros(cap, _BOX_DTYPE)
    n = np.zeros(1, np.int64)
    hist = np.empty((F, 256), np.uint32) if extras else None
    eff = np.empty(F, np.int32) if extras else None
    info = np.zeros(5, np.int64)
    mask = np.empty_like(q) if extras else None
    rc = lib().ro_detect_image(_p(q), T, F, C.byref(prm), _p(raw), cap, _p(n), _p(hist),
                               _p(eff), _p(info), _p(mask))
    _check(rc, "detect_image")
    if rc == -3:
        raise RuntimeError(f"oracle box capacity {cap} too small ({int(n[0])} boxes)")
    boxes = _boxes_to_array(raw, int(n[0]))
    if not extras:
        return boxes
    return boxes, dict(hist=hist, eff=eff, mask=mask, N0=int(info[0]), delta_psd=int(info[1]),
                       delta_pow=int(info[2]), P_q=int(info[3]), D=int(info[4]))


def detect(iq: np.ndarray, N: int, hop: int, prm: Optional[Params] = None):
    """Whole path from complex64 IQ.  Returns (boxes, image u8 [T, N], max power)."""
    prm = prm or params()
    iq = _iq(iq)
    T = num_frames(iq.shape[0], N, hop)
    if T < 1:
        raise ValueError("capture shorter than one frame")
    cap = _box_cap(T, N)
    raw = np.zeros(cap, _BOX_DTYPE)
    n = np.zeros(1, np.int64)
    img = np.empty((T, N), np.uint8)
    mx = np.zeros(1, np.float64)
    rc = lib().ro_detect(_p(iq), iq.shape[0], N, hop, C.byref(prm), _p(raw), cap, _p(n),
                         _p(img), _p(mx))
    _check(rc, "detect")
    if rc == -3:
        raise RuntimeError(f"oracle box capacity {cap} too small ({int(n[0])} boxes)")
    return _boxes_to_array(raw, int(n[0])), img, float(mx[0])


def hi_db_of(max_power: float) -> float:
    """Anchor of the 8-bit range for a capture whose largest |X|^2 is max_power."""
    return 10.0 * math.log10(max_power) if max_power > 0 else -math.inf


def match(gt: np.ndarray, det: np.ndarray, thetas) -> Dict:
    """Detection quality (Sec. III-A-2, Eqs. 2-3) of detections against ground
    truth: boxes as (t0, t1, f0, f1) inclusive rows (extra columns ignored).
    Returns n_t, n_f per threshold, P_d = n_t / N_gt, P_fa = n_f / N_d, and the
    best (intersection, union) pair of every box."""
    g = np.ascontiguousarray(np.asarray(gt)[:, :4], dtype=np.int32).reshape(-1, 4)
    d = np.ascontiguousarray(np.asarray(det)[:, :4], dtype=np.int32).reshape(-1, 4)
    th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).reshape(-1))
    nt = np.zeros(th.shape[0], np.int64)
    nf = np.zeros(th.shape[0], np.int64)
    gb = np.zeros((g.shape[0], 2), np.int64)
    db = np.zeros((d.shape[0], 2), np.int64)
    _check(lib().ro_match(_p(g), g.shape[0], _p(d), d.shape[0], _p(th), th.shape[0], _p(nt), _p(nf),
                          _p(gb), _p(db)), "match")
    return {"n_t": nt, "n_f": nf, "gt_best": gb, "det_best": db,
            "p_d": nt / max(1, g.shape[0]), "p_fa": nf / max(1, d.shape[0])}


def label(mask: np.ndarray) -> np.ndarray:
    """Component of every pixel (box order), -1 for background."""
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    T, F = m.shape
    out = np.empty((T, F), np.int64)
    _check(lib().ro_label(_p(m), T, F, _p(out)), "label")
    return out


def component_runs(mask: np.ndarray) -> np.ndarray:
    """Foreground runs in raster order: int32 (n, 4) = component, row, first, last column."""
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    T, F = m.shape
    cap = (T * F + 1) // 2 + 1
    runs = np.empty((cap, 4), np.int32)
    n = np.zeros(1, np.int64)
    _check(lib().ro_component_runs(_p(m), T, F, _p(runs), cap, _p(n)), "component_runs")
    return runs[: int(n[0])].copy()


def boundary(mask: np.ndarray) -> np.ndarray:
    """Foreground pixels with a background 4-neighbour (outside counts as background)."""
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    T, F = m.shape
    out = np.empty((T, F), np.uint8)
    lib().ro_boundary(_p(m), T, F, _p(out))
    return out
