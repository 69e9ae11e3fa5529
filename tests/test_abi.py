"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/*.h declares (no GPU needed: nothing is called)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for mt in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(svdup_\w+)\s*\(", src, flags=re.M):
            names.add(mt.group(1))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for n in ("svdup_create", "svdup_update", "svdup_sync", "svdup_destroy", "svdup_error_string"):
        assert n in names


def test_library_builds_and_exports_every_symbol():
    from paper_1707_08369_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in sorted(_declared()):
        assert hasattr(lib, n), "libsvdup.so does not export %s" % n


def test_error_strings_without_gpu():
    import paper_1707_08369_gb300 as sv
    from paper_1707_08369_gb300 import build
    build.build()
    sv.load()
    assert sv.error_string(sv.OK) == "ok"
    assert "converge" in sv.error_string(sv.ENOCONV)
    assert sv.error_string(12345) == "unknown error"
