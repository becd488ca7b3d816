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


def test_binding_shape_checks():
    """The binding rejects a buffer of the wrong shape before any pointer reaches the library
    (which cannot see the size of a device buffer)."""
    import numpy as np
    import pytest
    import torch
    from paper_2505_03755_gb300.las import _shape_check
    _shape_check(torch.zeros(4, 3, dtype=torch.float64), (4, 3), "C")
    _shape_check(torch.zeros(2, 2, 2, dtype=torch.float64), 8, "dm1s")   # flat count
    _shape_check(torch.zeros((), dtype=torch.float64), 1, "E")
    _shape_check(np.zeros((5, 5)), (5, 5), "h")
    with pytest.raises(ValueError):
        _shape_check(torch.zeros(3, 4, dtype=torch.float64), (4, 3), "C")     # transposed
    with pytest.raises(ValueError):
        _shape_check(torch.zeros(4, 2, dtype=torch.float64), (4, 3), "G")     # too small
    with pytest.raises(ValueError):
        _shape_check(torch.zeros(7, dtype=torch.float64), 8, "dm2")
    with pytest.raises(ValueError):
        _shape_check(torch.zeros(12, dtype=torch.float64), (4, 3), "C")       # flat for a matrix


def test_header_is_c99_and_a_c_client_links(tmp_path):
    """include/las.h compiles as strict C99 and a C program linked against liblasdf.so gets
    the documented argument errors from the calls that check before any device work."""
    import shutil
    import subprocess
    import pytest
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import __graft_entry__ as g
    g.build()
    pkg = os.path.join(ROOT, "paper_2505_03755_gb300")
    exe = str(tmp_path / "abi_from_c")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_from_c.c"),
                    "-L", pkg, "-llasdf", "-Wl,-rpath," + pkg, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "ok"


def test_no_cpu_fallback(monkeypatch, tmp_path):
    """Without the compiled library, or with host tensors, the product path raises instead of
    computing anything on the CPU."""
    import types
    import pytest
    import torch
    from paper_2505_03755_gb300 import las
    monkeypatch.setattr(las, "_lib", None)
    with pytest.raises(RuntimeError, match="not found"):
        las.load_library(str(tmp_path / "liblasdf.so"))
    monkeypatch.undo()
    import __graft_entry__ as g
    g.build()
    n, X = 6, 4
    B = torch.zeros(X * n * (n + 1) // 2, dtype=torch.float64)          # a host tensor
    with pytest.raises(TypeError, match="CUDA"):
        las.LasDF(B, n, X, n, 2, [], stream=types.SimpleNamespace(cuda_stream=0))
