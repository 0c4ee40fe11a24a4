"""The C-ABI library loads and exports every function include/rise.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rise.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(rise_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_abi():
    names = _declared()
    for must in ("rise_create", "rise_destroy", "rise_detect", "rise_detect_image",
                 "rise_detect_host", "rise_strerror", "rise_thresholds_default"):
        assert must in names


def test_library_exports_every_declared_function(built_lib):
    so = ctypes.CDLL(built_lib)
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing
    from paper_2603_20481_gb300 import rise
    assert set(rise.EXPORTS) == set(_declared())


def test_defaults_and_strerror_without_a_gpu(built_lib):
    from paper_2603_20481_gb300 import rise
    t = rise.default_thresholds()
    assert (t.range_mode, t.level_db, t.psd_offset_db, t.power_offset_db,
            t.sg_half_window, t.morph_order) == (0, 0.25, 0.5, 10.0, 5, 0)
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert rise.strerror(code) != "unknown status"


def test_box_and_struct_layouts_match_the_oracle():
    import oracle
    from paper_2603_20481_gb300 import rise
    assert rise.BOX_DTYPE == oracle._BOX_DTYPE
    assert [f[0] for f in rise.Thresholds._fields_] == [f[0] for f in oracle.Params._fields_]


def test_boxes_widen_on_the_host(built_lib):
    """rise_boxes_widen is host code: rise_box records to int64 rows in the
    column order t0, t1, f0, f1, anchor, area, sum_q, energy_fx."""
    import numpy as np
    from paper_2603_20481_gb300 import rise
    rng = np.random.default_rng(5)
    raw = np.zeros(37, rise.BOX_DTYPE)
    cols = ("t0", "t1", "f0", "f1", "anchor", "area", "sum_q", "energy_fx")
    for name in cols:
        hi = 2 ** 31 - 1 if raw.dtype[name].itemsize == 4 else 2 ** 62
        raw[name] = rng.integers(0, hi, size=raw.shape[0], dtype=np.int64).astype(raw.dtype[name])
    out = rise.boxes_from_raw(raw, raw.shape[0])
    assert out.dtype == np.int64 and out.shape == (37, 8)
    for j, name in enumerate(cols):
        np.testing.assert_array_equal(out[:, j], raw[name].astype(np.int64))
    assert rise.boxes_from_raw(raw, 0).shape == (0, 8)


def test_arguments_rejected_before_any_device_call(built_lib):
    """Invalid arguments are refused before the library touches CUDA, so
    these calls are safe with no GPU present."""
    import numpy as np
    from paper_2603_20481_gb300 import rise
    L = rise.lib()
    offs = np.zeros(2, np.int64)
    assert L.rise_detect_batch(None, None, 0, None, None, 0, offs.ctypes.data) == rise.RISE_EINVAL
    for N, hop in ((1000, 500), (128, 64), (2048, 0), (2048, 4096)):
        with pytest.raises(rise.RiseError) as e:
            rise.Server(N, hop, max_chunk=8192, max_streams=1)
        assert e.value.code == rise.RISE_EINVAL
