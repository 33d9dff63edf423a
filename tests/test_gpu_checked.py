"""Bounds checking of the tree: the node-table validation of vdbc_grid_load,
and the VDBC_CHECKED build (libvdbc_checked.so), whose every lookup checks
each node, leaf and tile index before it loads through it.

No test lets a kernel follow a bad index.  A corrupted file goes either to
the validating load, whose device pass only reads the tables and which
refuses the file before any lookup, or (with VDBC_FAULT=bounds) to the
checked build alone, run in a child process that first confirms it holds the
checked library; there each lookup tests the index, reads the background
instead and raises the device error word."""
import os
import subprocess
import sys

import numpy as np
import pytest

from gridfile import NEURAL, TILE, read_grid_file, table, write_grid_file

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2504_04564_gb300 as v
    import volgen
    from volgen import scenes
    return dict(torch=torch, v=v, vg=volgen, sc=scenes, dev=torch.device("cuda:0"))


def saved_grid(env, tmp_path, ratio=1.0):
    torch, v, vg = env["torch"], env["v"], env["vg"]
    host = vg.generate_host(vg.make_params("blobs", (40, 36, 44), 3))
    vol = torch.from_numpy(host).to(env["dev"])
    g = v.vdbc_encode(vol, ratio)
    dec = torch.empty_like(vol)
    v.vdbc_grid_decode(g, dec)
    path = str(tmp_path / "good.vdbc")
    v.vdbc_grid_save(g, path)
    return g, dec.cpu().numpy(), path


def expect_format_error(v, path, words):
    with pytest.raises(v.VdbcError) as ex:
        g = v.vdbc_grid_load(path)
        g.close()
    assert ex.value.status == v.ERR_FORMAT, ex.value
    assert words in str(ex.value), str(ex.value)


def test_load_validates_every_node_entry(env, tmp_path):
    """A checksummed file whose root, upper or lower table names a child, a
    leaf or a tile past the end of its table is refused with FORMAT, and so is
    a header whose counts do not give the file's table layout; the intact
    file round-trips."""
    v = env["v"]
    g, _, path = saved_grid(env, tmp_path)
    info = g.info
    rewritten = str(tmp_path / "same.vdbc")
    write_grid_file(rewritten, read_grid_file(path))
    v.vdbc_grid_load(rewritten).close()       # the test's own writer gives a valid file
    cases = []
    f = read_grid_file(path)
    low = table(f, 2, info.n_lower * 4096)
    leaf_at = int(np.flatnonzero(low & TILE == 0)[0])
    cases.append((2, leaf_at, info.n_leaves))                     # leaf past the last leaf
    tile_at = int(np.flatnonzero(low & TILE)[0])
    cases.append((2, tile_at, TILE | info.n_tiles))               # tile past the last tile
    cases.append((2, leaf_at, NEURAL | 0))                    # a neural entry in a plain grid
    up = table(f, 1, info.n_upper * 32768)
    cases.append((1, int(np.flatnonzero(up & TILE == 0)[0]), info.n_lower))   # lower node past the last
    cases.append((0, 0, info.n_upper))                            # upper node past the last
    for k, at, value in cases:
        f = read_grid_file(path)
        t = table(f, k, at + 1)
        t[at] = value
        bad = str(tmp_path / ("bad_%d_%d.vdbc" % (k, at)))
        write_grid_file(bad, f)
        expect_format_error(v, bad, "outside their tables")
    # header counts that do not match the block's layout
    f = read_grid_file(path)
    gi = v.GridInfo.from_buffer(f["info"])
    gi.n_leaves += 1
    del gi
    bad = str(tmp_path / "counts.vdbc")
    write_grid_file(bad, f)
    expect_format_error(v, bad, "do not match")
    f = read_grid_file(path)
    gi = v.GridInfo.from_buffer(f["info"])
    gi.n_tiles = -1
    del gi
    write_grid_file(bad, f)
    expect_format_error(v, bad, "counts")


def child(args, extra_env, timeout=600):
    e = dict(os.environ)
    e.update(extra_env)
    e["PYTHONPATH"] = ROOT + os.pathsep + e.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_child.py")] + args, env=e, cwd=ROOT,
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT, timeout=timeout)
    assert r.returncode == 0, r.stdout.decode()[-4000:]


def test_checked_build_computes_the_same_bits(env, tmp_path):
    """Encode, decode, PT/EA/ISO renders of FP32/FP16/FP8 grids, a learned
    grid and a batch: the checked build returns bit-identical outputs with a
    clean error word, so its checks change nothing on a valid grid; its
    tracker event counters (VDBC_STATS) agree with the render's own counts."""
    import checked_child
    torch, v = env["torch"], env["v"]
    assert not v.vdbc_version().endswith("checked")
    out = str(tmp_path / "checked.npz")
    child(["workload", out], {"VDBC_CHECKED": "1"})
    got = np.load(out)
    want = checked_child.run_workload(v, torch, env["vg"], env["sc"])
    assert set(got.files) == set(want)
    for k in sorted(want):
        a, b = np.asarray(want[k]), got[k]
        if k.startswith("events"):
            # the plain build counts no events; the checked build (VDBC_STATS)
            # counts every path fetched once, a free flight per lookup at
            # least, more loop iterations than flights, one to eight accessor
            # queries per lookup, and tree descents for only some of them
            ev, lookups, paths = [int(x) for x in b[:8]], int(b[8]), int(b[9])
            assert not np.any(a[:8]) and int(a[8]) == lookups and int(a[9]) == paths, (k, a, b)
            assert ev[5] == paths and ev[4] > 0 and ev[3] >= lookups > 0, (k, ev, lookups, paths)
            assert ev[0] >= ev[3] and ev[1] > 0 and ev[2] == 0, (k, ev)
            assert lookups <= ev[6] <= 8 * lookups and 0 < ev[7] < ev[6], (k, ev, lookups)
        elif k.startswith("flags"):
            assert int(a) == 0 and int(b) == 0, (k, a, b)
        elif k == "n_neural":
            assert int(a) == int(b) > 0
        else:
            assert a.shape == b.shape and np.array_equal(a.view(np.uint32), b.view(np.uint32)), k


def test_checked_build_reports_a_bad_leaf_index(env, tmp_path):
    """One lower entry of a saved grid points one past the last leaf.  The
    plain build refuses the file at load; the checked build, told to skip the
    load-time validation, decodes every other voxel exactly, reads the bad
    leaf as the background, reports DEVICE_FLAG from the decode and from a
    render whose ray crosses that leaf, and stays usable."""
    v = env["v"]
    g, dec, path = saved_grid(env, tmp_path)
    info = g.info
    f = read_grid_file(path)
    low = table(f, 2, info.n_lower * 4096)
    dims = tuple(info.dims)
    nl = [(d + 7) // 8 for d in dims]
    # a leaf with density worth marching through, in the first layer along z
    # (the ray enters it before any opacity builds up): the brightest there
    best, at = -1.0, -1
    for q in np.flatnonzero(low & TILE == 0):
        li, lj, lk = q % 16, (q // 16) % 16, q // 256      # one lower node covers the whole volume
        if li >= nl[0] or lj >= nl[1] or lk != 0:
            continue
        m = float(dec[lk * 8:lk * 8 + 8, lj * 8:lj * 8 + 8, li * 8:li * 8 + 8].max())
        if m > best:
            best, at = m, int(q)
    assert info.n_lower == 1 and at >= 0 and best > 0.1
    li, lj, lk = at % 16, (at // 16) % 16, at // 256
    low[at] = info.n_leaves
    bad = str(tmp_path / "bad_leaf.vdbc")
    write_grid_file(bad, f)
    expect_format_error(v, bad, "outside their tables")
    out = str(tmp_path / "bad.npz")
    x, y = li * 8 + 3, lj * 8 + 3
    child(["bad", bad, out, str(x), str(y)], {"VDBC_CHECKED": "1", "VDBC_FAULT": "bounds"})
    r = np.load(out)
    assert int(r["decode_status"]) == v.ERR_DEVICE_FLAG
    assert int(r["render_status"]) == v.ERR_DEVICE_FLAG
    B = np.array([int(r["background_bits"])], dtype=np.uint32).view(np.float32)[0]
    want = dec.copy()
    want[lk * 8:lk * 8 + 8, lj * 8:lj * 8 + 8, li * 8:li * 8 + 8] = B
    assert np.array_equal(r["decode"].view(np.uint32), want.view(np.uint32))
    assert np.isfinite(r["after"]).all() and float(r["after"][0, 0, 3]) > 0.0
