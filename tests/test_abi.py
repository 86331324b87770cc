"""CPU checks of the C ABI: the library loads and exports every entry point
declared in include/msd.h (no compute calls: there is no GPU here)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(msd_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1409_8186_gb300 import build
    lib = build.build()
    import ctypes
    h = ctypes.CDLL(lib)
    names = declared_entry_points()
    assert len(names) >= 10
    missing = [n for n in sorted(names) if not hasattr(h, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1409_8186_gb300 import msd
    assert set(msd.EXPORTED) == declared_entry_points()
    for n in msd.EXPORTED:
        assert callable(getattr(msd, n))


def test_last_error_is_empty_string_initially():
    from paper_1409_8186_gb300 import msd
    assert isinstance(msd.msd_last_error(), str)
