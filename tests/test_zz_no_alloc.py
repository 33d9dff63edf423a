"""The allocation-free brick selection, vdbc_select_bricks_noalloc.

It serves callers that cannot allocate device memory while they run (a
renderer inside a host application that owns the device-memory budget, or a
frame loop that cannot absorb the device synchronization of cudaMalloc).  It
must give exactly what the selection inside vdbc_encode gives, which is the
oracle's Algorithm 1: the background value, the activated bricks and the
counts.  Two calls in a row on different volumes check that the shared
scratch left by one call does not leak into the next.

"Allocates nothing" is checked two ways: the calls run with VDBC_FAULT=oom,
which makes every device allocation of the library fail (so a call that
allocated would return OOM), and the device's free memory is unchanged
across every call but the first one on the device (which may load the
library's device image).

This file is collected last so that a run stopping at its first failure has
run every other test before it.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

_first_call_done = []


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__ as g
    g.build()
    import oracle
    import paper_2504_04564_gb300 as v
    import volgen
    return dict(torch=torch, v=v, vg=volgen, orc=oracle, dev=torch.device("cuda:0"))


def select_without_alloc(env, vol, ratio, metric, monkeypatch):
    torch, v = env["torch"], env["v"]
    nz, ny, nx = vol.shape
    nb = ((nx + 31) // 32) * ((ny + 31) // 32) * ((nz + 31) // 32)
    b = torch.full((1,), -1, dtype=torch.int32, device=env["dev"])
    active = torch.full((nb,), 7, dtype=torch.uint8, device=env["dev"])
    counts = torch.full((3,), -1, dtype=torch.int64, device=env["dev"])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("VDBC_FAULT", "oom")
    try:
        v.vdbc_select_bricks_noalloc(vol, ratio, b, active, counts, metric=metric)
        torch.cuda.synchronize()
    finally:
        monkeypatch.delenv("VDBC_FAULT")
    free1 = torch.cuda.mem_get_info()[0]
    if _first_call_done:
        assert free1 == free0
    _first_call_done.append(True)
    return (int(b.cpu().numpy().view(np.uint32)[0]), active.cpu().numpy(), counts.cpu().numpy())


def test_noalloc_selection_equals_encode_twice_in_a_row(env, monkeypatch):
    torch, v, vg = env["torch"], env["v"], env["vg"]
    cases = [("turbulence", (96, 80, 72), 6.0, 2), ("blobs", (130, 64, 40), 4.0, 3),
             ("turbulence", (96, 80, 72), 2.5, 1)]
    for kind, dims, ratio, metric in cases:
        vol = torch.from_numpy(vg.generate_host(vg.make_params(kind, dims, 5))).to(env["dev"])
        grid = v.vdbc_encode(vol, ratio, metric=metric)
        info = grid.info
        want_active = v.vdbc_grid_active_bricks(grid)
        for call in range(2):
            bits, active, counts = select_without_alloc(env, vol, ratio, metric, monkeypatch)
            assert bits == info.background_bits
            assert np.array_equal(active, want_active)
            assert counts[0] == info.n_nonempty and counts[1] == info.n_active and counts[2] == 0


def _tie_volume(dims, levels=37):
    """One or two non-background voxels per 32^3 brick from a few values:
    scores tie across hundreds of bricks at the budget edge."""
    nx, ny, nz = dims
    v = np.zeros((nz, ny, nx), dtype=np.float32)
    bx, by, bz = (nx + 31) // 32, (ny + 31) // 32, (nz + 31) // 32
    k, j, i = np.meshgrid(np.arange(bz), np.arange(by), np.arange(bx), indexing="ij")
    b = (k * by + j) * bx + i
    lvl = (1 + (i * 7 + j * 3 + k * 5) % levels).astype(np.float32) / levels
    keep = b % 5 != 0
    x, y, z = np.minimum(i * 32 + 3, nx - 1), np.minimum(j * 32 + 5, ny - 1), np.minimum(k * 32 + 2, nz - 1)
    v[z[keep], y[keep], x[keep]] = lvl[keep]
    neg = keep & (b % 3 == 0)
    v[z[neg], np.minimum(j * 32 + 9, ny - 1)[neg], np.minimum(i * 32 + 17, nx - 1)[neg]] = -lvl[neg] / 2
    return v


def test_noalloc_selection_equals_the_oracle_above_4096_bricks(env, monkeypatch):
    """4290 bricks (the selection's branch for more than 4096 keys) with tied
    scores at the budget edge, then the cloud generator's content at 4488
    bricks: B, the activated set and the counts equal the oracle's encode."""
    torch, orc, vg = env["torch"], env["orc"], env["vg"]
    cloud = vg.generate_torch(vg.make_params("cloud", (1040, 544, 256), 0)).cpu().numpy()
    for host, ratio, metric in ((_tie_volume((4160, 1056, 8)), 10.0, 2), (_tie_volume((4160, 1056, 8)), 3.0, 1),
                                (cloud, 10.0, 2), (cloud, 4.0, 3)):
        e = orc.encode(host, ratio, metric=metric)
        vol = torch.from_numpy(host).to(env["dev"])
        for call in range(2):
            bits, active, counts = select_without_alloc(env, vol, ratio, metric, monkeypatch)
            assert bits == e["background_bits"]
            assert np.array_equal(active, e["active"])
            assert counts[0] == int((e["empty"] == 0).sum()) and counts[1] == e["n_active"] and counts[2] == 0
        del vol


def test_noalloc_flags_a_non_finite_volume_and_recovers(env, monkeypatch):
    """A NaN anywhere sets the third count (the other outputs are then not
    defined); the next call on a finite volume is exact again, so the flag
    does not stay in the shared scratch."""
    torch, orc, vg = env["torch"], env["orc"], env["vg"]
    host = _tie_volume((4160, 1056, 8))
    bad = host.copy()
    bad[5, 700, 4000] = np.nan
    _, _, counts = select_without_alloc(env, torch.from_numpy(bad).to(env["dev"]), 10.0, 2, monkeypatch)
    assert counts[2] != 0
    e = orc.encode(host, 10.0)
    bits, active, counts = select_without_alloc(env, torch.from_numpy(host).to(env["dev"]), 10.0, 2, monkeypatch)
    assert counts[2] == 0 and bits == e["background_bits"] and np.array_equal(active, e["active"])


def _raw_call(env, dims, outs):
    v = env["v"]
    d = v.Dense()
    d.dims[0], d.dims[1], d.dims[2] = dims
    d.on_device = 1
    d.data = outs[0]
    p = v.EncodeParams(4.0, 2, 0, 8, 0)
    return v.lib().vdbc_select_bricks_noalloc(ctypes.byref(d), ctypes.byref(p), outs[1], outs[2], outs[3], None)


def test_noalloc_size_limit_boundary(env):
    """1024 x 1024 x 2048 voxels are exactly 65,536 bricks and pass the size
    check (the call then refuses a host counts_out, so no kernel runs); one
    more brick along x is refused for its size."""
    torch, v = env["torch"], env["v"]
    buf = torch.zeros(16, dtype=torch.int64, device=env["dev"])
    host = np.zeros(4, dtype=np.int64)
    dptr = buf.data_ptr()
    st = _raw_call(env, (1024, 1024, 2048), (dptr, dptr, dptr, host.ctypes.data))
    assert st == v.ERR_INVALID_ARG and "counts_out is not device memory" in v.vdbc_last_error()
    st = _raw_call(env, (1025, 1024, 2048), (dptr, dptr, dptr, dptr))
    assert st == v.ERR_INVALID_ARG and "65536" in v.vdbc_last_error()


def test_noalloc_checks_its_outputs(env, monkeypatch):
    """Outputs that kernels would write out of bounds or into host memory are
    refused: by the binding (kind, dtype, length) and by the C side (host
    memory, misalignment)."""
    torch, v = env["torch"], env["v"]
    vol = torch.zeros((40, 40, 70), dtype=torch.float32, device=env["dev"])     # 3 x 2 x 2 = 12 bricks
    b = torch.zeros(1, dtype=torch.int32, device=env["dev"])
    a = torch.zeros(12, dtype=torch.uint8, device=env["dev"])
    c = torch.zeros(3, dtype=torch.int64, device=env["dev"])
    with pytest.raises(ValueError):
        v.vdbc_select_bricks_noalloc(vol, 4.0, b, a[:11], c)
    with pytest.raises(TypeError):
        v.vdbc_select_bricks_noalloc(vol, 4.0, b, a.cpu(), c)
    with pytest.raises(TypeError):
        v.vdbc_select_bricks_noalloc(vol, 4.0, b, a, c.to(torch.int32))
    host = np.zeros(16, dtype=np.uint8)
    dptr = c.data_ptr()
    st = _raw_call(env, (70, 40, 40), (vol.data_ptr(), b.data_ptr(), host.ctypes.data, dptr))
    assert st == v.ERR_INVALID_ARG and "active_out is not device memory" in v.vdbc_last_error()
    st = _raw_call(env, (70, 40, 40), (vol.data_ptr(), b.data_ptr(), a.data_ptr(), dptr + 4))
    assert st == v.ERR_INVALID_ARG and "aligned" in v.vdbc_last_error()
    bits, active, counts = select_without_alloc(env, vol, 4.0, 2, monkeypatch)
    assert counts[1] == 0 and not active.any()
