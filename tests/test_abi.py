"""CPU-side checks of the C ABI: the library builds, loads and exports every declared call."""
import os
import re

from paper_2505_03755_gb300 import EXPORTS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(las_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_call():
    import __graft_entry__ as g
    g.build()
    from paper_2505_03755_gb300 import load_library
    lib = load_library()
    decl = declared_functions()
    assert decl, "no declarations found"
    missing = [n for n in sorted(decl) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(EXPORTS) <= decl


def test_status_strings():
    from paper_2505_03755_gb300 import load_library
    lib = load_library()
    for code in range(7):
        assert lib.las_status_str(code)
