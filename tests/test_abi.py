"""The C ABI library on the CPU: it loads, exports every function that
include/*.h declares, and rejects bad arguments before any device work."""
import ctypes
import glob
import os
import re

import pytest

from gridfile import write_grid_file

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def v():
    import paper_2504_04564_gb300 as v
    from paper_2504_04564_gb300 import build
    build.build(checked=v.CHECKED, sanitize=v.SANITIZE)
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


def fabricated_file(v, path, **counts):
    """A checksummed one-brick 8^3 FP32 file whose block is 256 zero bytes at
    offset 0 for every table (the layout of no real grid)."""
    info = v.GridInfo()
    info.dims[:] = [8, 8, 8]
    info.macrocell = 8
    info.n_bricks = 1
    info.n_tiles = 1
    for k, x in counts.items():
        setattr(info, k, x)
    write_grid_file(path, dict(magic=b"VDBCGRD1", version=2, offsets=[0] * 16,
                               info=bytearray(bytes(info)), active=b"\x00", block=bytearray(256)))


def test_grid_load_checks_the_layout_on_host(v, tmp_path):
    """Counts that no grid could have, or tables not where the counts put
    them, are refused with FORMAT on the host (no device here)."""
    L = v.lib()
    h = ctypes.c_void_p()
    path = str(tmp_path / "fab.vdbc")
    fabricated_file(v, path)
    assert L.vdbc_grid_load(path.encode(), None, ctypes.byref(h)) == v.ERR_FORMAT
    assert "do not match" in v.vdbc_last_error()
    for bad in (dict(n_tiles=0), dict(n_leaves=-1), dict(n_upper=1 << 31), dict(n_neural=3)):
        fabricated_file(v, path, **bad)
        assert L.vdbc_grid_load(path.encode(), None, ctypes.byref(h)) == v.ERR_FORMAT, bad
        assert "counts" in v.vdbc_last_error(), (bad, v.vdbc_last_error())
    assert h.value is None


@pytest.fixture(scope="module")
def checked_lib():
    from paper_2504_04564_gb300 import build
    L = ctypes.CDLL(build.build(checked=True))
    L.vdbc_version.restype = ctypes.c_char_p
    return L


def test_checked_build_exports_the_same_surface(v, checked_lib):
    """libvdbc_checked.so (VDBC_CHECKED=1) declares itself and exports every
    function of include/*.h, and rejects bad arguments the same way."""
    for n in sorted(declared_functions()):
        assert hasattr(checked_lib, n), n
    assert checked_lib.vdbc_version().decode().endswith("checked")
    assert not v.vdbc_version().endswith("checked")
    h = ctypes.c_void_p()
    assert checked_lib.vdbc_encode(None, None, None, ctypes.byref(h)) == v.ERR_INVALID_ARG


def test_null_arguments_rejected_on_every_entry_point(v):
    """Every entry point that takes a handle or an output refuses a null one
    with INVALID_ARG before any device work (so this runs without a GPU)."""
    L = v.lib()
    h = ctypes.c_void_p()
    n64 = ctypes.c_int64()
    n32 = ctypes.c_int32()
    calls = [
        lambda: L.vdbc_grid_get_info(None, None),
        lambda: L.vdbc_grid_decode(None, None, 1, None),
        lambda: L.vdbc_grid_active_bricks(None, None),
        lambda: L.vdbc_grid_macrocells(None, None, None),
        lambda: L.vdbc_grid_save(None, b"/nonexistent"),
        lambda: L.vdbc_grid_load(None, None, ctypes.byref(h)),
        lambda: L.vdbc_render_stats_get(None, None, None),
        lambda: L.vdbc_volume_create(None, 0, 8, None, ctypes.byref(h)),
        lambda: L.vdbc_render_dense(None, None, None, 1, 0, None, 1, None),
        lambda: L.vdbc_volume_render_stats_get(None, None, None),
        lambda: L.vdbc_batch_create(None, 0, 0, None, ctypes.byref(h)),
        lambda: L.vdbc_batch_render_frames(None, 1, None),
        lambda: L.vdbc_batch_reset(None, None),
        lambda: L.vdbc_batch_get_tuning(None, None),
        lambda: L.vdbc_batch_stats_get(None, None, None),
        lambda: L.vdbc_batch_state_size(None, ctypes.byref(n64)),
        lambda: L.vdbc_batch_get_state(None, ctypes.byref(n32), None, None),
        lambda: L.vdbc_batch_set_state(None, 0, None, None),
        lambda: L.vdbc_learn(None, None, None, ctypes.byref(h), None),
        lambda: L.vdbc_learn_loss_grad(None, None, None, 1, None, None, None, None),
        lambda: L.vdbc_learn_get_params(None, None),
        lambda: L.vdbc_select_bricks_noalloc(None, None, None, None, None, None),
        lambda: L.vdbc_compare(None, None, 1, 1, 1, None, None),
    ]
    for i, call in enumerate(calls):
        assert call() == v.ERR_INVALID_ARG, i
        assert v.vdbc_last_error(), i
    L.vdbc_grid_free(None)
    L.vdbc_volume_free(None)
    L.vdbc_batch_free(None)


def test_noalloc_size_limit_is_checked_before_device_work(v):
    """The allocation-free selection's brick limit, argument-only: a
    1024 x 1024 x 2048 descriptor (exactly 65,536 bricks) passes the size
    check and only then meets the device checks (which fail here, with no
    GPU); one more brick along any axis is refused for its size.  No kernel
    can run on either path: the descriptor's pointer is a dummy."""
    import numpy as np
    L = v.lib()
    dummy = np.zeros(8, dtype=np.int64)
    ptr = dummy.ctypes.data
    p = v.EncodeParams(4.0, 2, 0, 8, 0)
    for dims, refused in (((1024, 1024, 2048), False), ((1025, 1024, 2048), True), ((1024, 1056, 2048), True),
                          ((1024, 1024, 2049), True)):
        d = v.Dense()
        d.dims[0], d.dims[1], d.dims[2] = dims
        d.on_device = 1
        d.data = ptr
        st = L.vdbc_select_bricks_noalloc(ctypes.byref(d), ctypes.byref(p), ptr, ptr, ptr, None)
        assert st != v.OK
        assert ("65536" in v.vdbc_last_error()) == refused, (dims, v.vdbc_last_error())


def test_header_is_c11_and_a_c_program_links_and_runs(v, tmp_path):
    """include/vdbc.h compiles as C11 with every warning an error, and a C
    program on it links against the library and runs: it renders where a GPU
    is present and otherwise exits with the library's error message."""
    import subprocess
    exe = str(tmp_path / "encode_render")
    lib_dir = os.path.dirname(v.LIB_PATH)
    lib_name = os.path.basename(v.LIB_PATH)[3:-3]
    r = subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I" + os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c", "encode_render.c"), "-L" + lib_dir, "-l" + lib_name,
                        "-Wl,-rpath," + lib_dir, "-o", exe], stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    assert r.returncode == 0, r.stdout
    r = subprocess.run([exe], stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=300)
    if r.returncode == 0:
        assert "paths" in r.stdout
    else:
        assert r.returncode == 1 and r.stdout.strip(), r.stdout
