"""The C-ABI library builds, loads without a GPU, and exports every function
declared in include/cil.h (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(cil_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("cil_knn", "cil_radius_search", "cil_estimate_normals",
                     "cil_icp_point_to_plane", "cil_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1807_00399_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_status_strings_without_gpu():
    import paper_1807_00399_gb300 as cil

    L = cil.lib()
    for code, name in cil.STATUS.items():
        assert L.cil_status_string(code).decode() == name


def test_argument_errors_need_no_gpu():
    import paper_1807_00399_gb300 as cil

    L = cil.lib()
    # k out of range and negative sizes are rejected before any CUDA call
    assert L.cil_knn(None, 10, None, 10, 0, None, None, None) == 1
    assert L.cil_knn(None, 10, None, 10, 33, None, None, None) == 1
    assert L.cil_knn(None, -1, None, 10, 5, None, None, None) == 1
    assert L.cil_estimate_normals(None, 10, 0, None, None, None, None) == 1
    assert L.cil_icp_point_to_plane(None, -5, None, None, 10, None, 1, 0.1, None, None, None) == 1
    L.cil_icp_sums.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_float,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p]
    assert L.cil_icp_sums(None, 0, None, None, 0, None, 1, 0.1, None, None, None, None, None) == 1


def test_package_fails_loudly_without_library(monkeypatch, tmp_path):
    # no silent fallback: when the library cannot be produced, loading raises
    import importlib

    import paper_1807_00399_gb300 as cil
    from paper_1807_00399_gb300 import build

    monkeypatch.setattr(cil, "_lib", None)
    monkeypatch.setattr(build, "build", lambda *a, **k: str(tmp_path / "missing.so"))
    with pytest.raises(OSError):
        cil.lib()
    monkeypatch.setattr(cil, "_lib", None)
    importlib.reload(build)
