"""The C ABI library on the CPU: it loads, exports every function that
include/*.h declares, and rejects bad arguments before any device work."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def v():
    from paper_2504_04564_gb300 import build
    build.build()
    import paper_2504_04564_gb300 as v
    return v


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(vdbc_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(v):
    names = declared_functions()
    assert len(names) >= 15
    L = ctypes.CDLL(v.LIB_PATH)
    for n in sorted(names):
        assert hasattr(L, n), n
    # and the binding covers the same surface
    assert names == set(v.SIGNATURES), names ^ set(v.SIGNATURES)


def test_version_and_empty_error(v):
    assert v.vdbc_version().startswith("vdbc ")
    assert "sm_103a" in v.vdbc_version()


def test_invalid_arguments_rejected_without_device(v):
    L = v.lib()
    h = ctypes.c_void_p()
    assert L.vdbc_encode(None, None, None, ctypes.byref(h)) == v.ERR_INVALID_ARG
    import numpy as np
    vol = np.zeros((4, 4, 4), dtype=np.float32)
    d = v.make_dense(vol)
    for ratio in (0.5, float("nan"), float("inf")):
        p = v.EncodeParams(ratio, 2, 0, 8, 0)
        assert L.vdbc_encode(ctypes.byref(d), ctypes.byref(p), None, ctypes.byref(h)) == v.ERR_INVALID_ARG
        assert "ratio" in v.vdbc_last_error()
    p = v.EncodeParams(2.0, 9, 0, 8, 0)
    assert L.vdbc_encode(ctypes.byref(d), ctypes.byref(p), None, ctypes.byref(h)) == v.ERR_INVALID_ARG
    p = v.EncodeParams(2.0, 2, 5, 8, 0)
    assert L.vdbc_encode(ctypes.byref(d), ctypes.byref(p), None, ctypes.byref(h)) == v.ERR_INVALID_ARG
    d.dims[0] = 0
    p = v.EncodeParams(2.0, 2, 0, 8, 0)
    assert L.vdbc_encode(ctypes.byref(d), ctypes.byref(p), None, ctypes.byref(h)) == v.ERR_INVALID_ARG
    assert L.vdbc_render(None, None, None, 1, 0, None, 1, None) == v.ERR_INVALID_ARG


def test_grid_load_rejects_bad_files_on_host(v, tmp_path):
    """A missing, foreign, truncated or corrupted file is refused before any
    device work (the checks run on the host)."""
    L = v.lib()
    h = ctypes.c_void_p()
    assert L.vdbc_grid_load(str(tmp_path / "missing.vdbc").encode(), None, ctypes.byref(h)) == v.ERR_INVALID_ARG
    bad = tmp_path / "bad.vdbc"
    bad.write_bytes(b"NOTAGRID" + bytes(200))
    assert L.vdbc_grid_load(str(bad).encode(), None, ctypes.byref(h)) == v.ERR_FORMAT
    short = tmp_path / "short.vdbc"
    short.write_bytes(b"VDBCGRD1" + (1).to_bytes(4, "little"))
    assert L.vdbc_grid_load(str(short).encode(), None, ctypes.byref(h)) == v.ERR_FORMAT
    assert h.value is None
