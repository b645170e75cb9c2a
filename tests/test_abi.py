"""CPU-side checks of the C ABI: the library builds, loads, and exports every
entry point that include/cdc.h declares; struct layouts match; errors are
reported without touching a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cdc.h")


@pytest.fixture(scope="module")
def libcdc():
    from paper_1908_01949_gb300 import build as B
    path = B.build()
    return C.CDLL(path), path


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cdc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_five_paper_calls():
    names = declared_functions()
    for n in ("cdc_load_geometry", "cdc_load_field", "cdc_hough_seeds", "cdc_scan_seeds", "cdc_refine_seeds"):
        assert n in names


def test_library_exports_every_declared_symbol(libcdc):
    L, path = libcdc
    for n in declared_functions():
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (cdc_[a-z0-9_]+)", out))
    assert set(declared_functions()) <= exported


def test_binding_covers_every_entry_point():
    from paper_1908_01949_gb300 import _lib
    assert sorted(_lib.EXPORTS) == declared_functions()
    for n in _lib.EXPORTS:
        if n.startswith("cdc_") and n not in ("cdc_create", "cdc_destroy", "cdc_last_error"):
            assert hasattr(_lib.Context, n)


def test_every_entry_point_has_a_declared_signature():
    """ctypes passes undeclared integer arguments as 32-bit ints, which would cut
    64-bit device pointers: every exported call carries its argument types, and
    as many as the header's declaration has parameters."""
    from paper_1908_01949_gb300 import _lib
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    L = _lib.lib()
    for n in _lib.EXPORTS:
        decl = re.search(r"\b" + n + r"\s*\(([^)]*)\)", src).group(1)
        n_params = 0 if decl.strip() in ("", "void") else decl.count(",") + 1
        assert getattr(L, n).argtypes is not None, n
        assert len(getattr(L, n).argtypes) == n_params, (n, len(getattr(L, n).argtypes), n_params)


def test_struct_layouts_match_header():
    from paper_1908_01949_gb300 import _lib
    assert C.sizeof(_lib.cdc_grid) == 60
    assert C.sizeof(_lib.cdc_scan_params) == 40
    assert C.sizeof(_lib.cdc_candidate) == 28
    assert C.sizeof(_lib.cdc_hough_params) == 13 * 4 + 60
    assert C.sizeof(_lib.cdc_refine_params) == 32
    assert C.sizeof(_lib.cdc_scan_config) == 12
    # compile a probe against the header and compare sizes/offsets
    probe = r'''
#include <stdio.h>
#include <stddef.h>
#include "cdc.h"
int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %d\n", sizeof(cdc_grid), sizeof(cdc_scan_params),
 sizeof(cdc_candidate), sizeof(cdc_hough_params), sizeof(cdc_refine_params),
 offsetof(cdc_hough_params, grid_template), offsetof(cdc_scan_params, max_drift), sizeof(cdc_scan_config),
 CDC_SCAN_CONFIGS); return 0;}
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(src, "w").write(probe)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        vals = [int(x) for x in subprocess.check_output([exe]).split()]
    assert vals == [C.sizeof(_lib.cdc_grid), C.sizeof(_lib.cdc_scan_params), C.sizeof(_lib.cdc_candidate),
                    C.sizeof(_lib.cdc_hough_params), C.sizeof(_lib.cdc_refine_params),
                    _lib.cdc_hough_params.grid_template.offset, _lib.cdc_scan_params.max_drift.offset,
                    C.sizeof(_lib.cdc_scan_config), _lib.CDC_SCAN_CONFIGS]


def test_null_context_is_an_argument_error(libcdc):
    L, _ = libcdc
    L.cdc_last_error.restype = C.c_char_p
    assert L.cdc_last_error(None) == b"NULL context"
    L.cdc_create.argtypes = [C.c_void_p, C.c_int]
    assert L.cdc_create(None, 0) == -1
    L.cdc_scan_seeds.restype = C.c_int
    assert L.cdc_scan_seeds(*([None] * 17)) == -1
    assert L.cdc_load_geometry(None, 0, None, None, None, None, C.c_double(0), C.c_double(0), C.c_double(0)) == -1
    assert L.cdc_set_scan_config(None, None) == -1
    assert L.cdc_get_scan_config(None, None) == -1
    assert L.cdc_tune_scan(*([None] * 11)) == -1


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1908_01949_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        _lib.lib()
