"""The C-ABI library (no GPU needed): it builds, loads, and exports every
function the public header declares; the binding's mirror of fmm_stats_t
matches the header field for field.  No compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fmm_layered.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(fmm_layered_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def library():
    import shutil
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    from paper_1902_05132_gb300 import _build
    _build.build()
    import paper_1902_05132_gb300 as pkg
    return pkg.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("fmm_layered_create", "fmm_layered_eval", "fmm_layered_eval_batched", "fmm_layered_destroy",
                 "fmm_layered_stats", "fmm_layered_last_error", "fmm_layered_direct"):
        assert must in names, names


def test_library_exports_every_declared_symbol(library):
    names = _declared_functions()
    missing = [n for n in names if not hasattr(library, n)]
    assert not missing, missing
    import paper_1902_05132_gb300 as pkg
    assert sorted(pkg.EXPORTED) == names


def test_stats_struct_matches_header(library):
    import paper_1902_05132_gb300 as pkg
    text = open(HEADER).read()
    body = re.search(r"typedef struct \{(.*?)\} fmm_stats_t;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", " ", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, rest = decl.split(None, 1)
        for name in rest.split(","):
            fields.append((name.strip(), ctype))
    cmap = {"int": ctypes.c_int, "long": ctypes.c_long, "double": ctypes.c_double}
    assert [(n, cmap[t]) for n, t in fields] == list(pkg.Stats._fields_)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_1902_05132_gb300 as pkg
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="missing"):
        pkg.lib()


def test_create_without_device_reports_an_error(library):
    # without a GPU the create call must fail with an error code, not crash
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    k = np.array([1.0, 1.5])
    d = np.array([0.0])
    h = ctypes.c_void_p()
    rc = library.fmm_layered_create(2, k.ctypes.data, d.ctypes.data, None, 4, 16, 0, ctypes.byref(h))
    assert rc != 0 and not h.value
    assert library.fmm_layered_last_error(None)
