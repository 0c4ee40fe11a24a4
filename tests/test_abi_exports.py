"""The C-ABI library loads and exports every function include/rise.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re

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
