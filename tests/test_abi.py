"""CPU checks of the C-ABI boundary: the library builds, loads, and exports
every entry point that include/adsx.h declares.  No compute calls (no GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as f:
                txt = f.read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(adsx_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2303_09855_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert {"adsx_build_index", "adsx_search", "adsx_free_index", "adsx_last_error"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_mirror_the_c_abi():
    from paper_2303_09855_gb300 import adsx
    for n in _declared():
        assert hasattr(adsx, n[len("adsx_"):]), n


def test_last_error_is_empty_string_initially():
    from paper_2303_09855_gb300 import adsx, build
    build.build()
    assert isinstance(adsx.last_error(), str)
