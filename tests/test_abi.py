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


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of msd_opts and msd_stats have the size and field
    offsets that a C compiler gives the header's structs (a field added to
    one side only would shift every later field of the other)."""
    import ctypes
    import shutil
    import subprocess
    import pytest
    from paper_1409_8186_gb300 import msd
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "msd.h"', 'int main(void) {']
    for st in (msd.msd_opts, msd.msd_stats):
        name = st.__name__
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            a, b, c = ln.split()
            got[(a, b)] = int(c)
    for st in (msd.msd_opts, msd.msd_stats):
        name = st.__name__
        assert got[(name, "size")] == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, (name, f)
