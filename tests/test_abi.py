"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/vb.h (host-only checks: no GPU is needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_15124_gb300 import native
    path = native.compile_library()
    return ctypes.CDLL(path)


def _declared():
    src = open(os.path.join(ROOT, "include", "vb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:vb_status|size_t|int64_t|const char\*)\s+(vb_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    import paper_2104_15124_gb300 as vb
    assert set(_declared()) == set(vb.EXPORTED)


def test_report_struct_matches_the_header():
    # the ctypes mirror of vb_report: same fields, same order, same widths
    import paper_2104_15124_gb300 as vb
    src = open(os.path.join(ROOT, "include", "vb.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} vb_report;", src, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(int32_t|int64_t)\s+(\w+);", body)
    want = [(name, ctypes.c_int32 if ty == "int32_t" else ctypes.c_int64) for ty, name in fields]
    assert [(n, t) for n, t in vb.Report._fields_] == want
    assert ctypes.sizeof(vb.Report) <= 256   # the context's device report block


def test_status_strings(lib):
    f = lib.vb_status_string
    f.restype = ctypes.c_char_p
    f.argtypes = [ctypes.c_int32]
    assert f(0) == b"ok"
    assert f(-3) == b"workspace too small"
    assert f(-42) == b"unknown status"


def test_workspace_sizes_are_host_only_and_grow(lib):
    import paper_2104_15124_gb300 as vb
    L = vb.lib()
    p = vb.KnnParams(32, 16, 0, 1)
    a = L.vb_knn_workspace(2000, 2, ctypes.byref(p))
    b = L.vb_knn_workspace(20000, 2, ctypes.byref(p))
    assert 0 < a < b
    assert L.vb_graph_workspace(1000, 8) < L.vb_graph_workspace(1000, 16)
    bp = vb.BuildParams(p, 0, vb.OpParams(1.0, -0.25, 2.0), -10.0, 4.0, 0.25, 0)
    assert L.vb_build_workspace(50000, 3, ctypes.byref(bp)) >= L.vb_graph_workspace(50000, 32)


def test_product_does_not_reach_the_oracle():
    # the package and its sources never import or load the oracle
    pkg = os.path.join(ROOT, "paper_2104_15124_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, flags=re.M), f
                assert "knn_bf" not in txt, f
