"""The allocation-free brick selection, vdbc_select_bricks_noalloc.

It serves callers that cannot allocate device memory while they run (a
renderer inside a host application that owns the device-memory budget, or a
frame loop that cannot absorb the device synchronization of cudaMalloc).  It
must give exactly what the selection inside vdbc_encode gives: the background
value, the activated bricks and the counts.  Two calls in a row on different
volumes check that the shared scratch left by one call does not leak into the
next.  This file is collected last so that a run stopping at its first failure
has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2504_04564_gb300 as v
    import volgen
    return dict(torch=torch, v=v, vg=volgen, dev=torch.device("cuda:0"))


def select_without_alloc(env, vol, ratio, metric):
    torch, v = env["torch"], env["v"]
    nz, ny, nx = vol.shape
    nb = ((nx + 31) // 32) * ((ny + 31) // 32) * ((nz + 31) // 32)
    b = torch.full((1,), -1, dtype=torch.int32, device=env["dev"])
    active = torch.full((nb,), 7, dtype=torch.uint8, device=env["dev"])
    counts = torch.full((3,), -1, dtype=torch.int64, device=env["dev"])
    v.vdbc_select_bricks_noalloc(vol, ratio, b, active, counts, metric=metric)
    torch.cuda.synchronize()
    return (int(b.cpu().numpy().view(np.uint32)[0]), active.cpu().numpy(), counts.cpu().numpy())


def test_noalloc_selection_equals_encode_twice_in_a_row(env):
    torch, v, vg = env["torch"], env["v"], env["vg"]
    cases = [("turbulence", (96, 80, 72), 6.0, 2), ("blobs", (130, 64, 40), 4.0, 3),
             ("turbulence", (96, 80, 72), 2.5, 1)]
    for kind, dims, ratio, metric in cases:
        vol = torch.from_numpy(vg.generate_host(vg.make_params(kind, dims, 5))).to(env["dev"])
        grid = v.vdbc_encode(vol, ratio, metric=metric)
        info = grid.info
        want_active = v.vdbc_grid_active_bricks(grid)
        for call in range(2):
            free0 = torch.cuda.mem_get_info()[0]
            bits, active, counts = select_without_alloc(env, vol, ratio, metric)
            assert torch.cuda.mem_get_info()[0] == free0 or call == 0
            assert bits == info.background_bits
            assert np.array_equal(active, want_active)
            assert counts[0] == info.n_nonempty and counts[1] == info.n_active and counts[2] == 0


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    """66,000 bricks (2048 x 1024 x 1056 voxels) exceed the fixed 65,536-brick
    scratch: the call refuses before touching the GPU."""
    torch, v = env["torch"], env["v"]
    d = v.Dense()
    d.dims[0], d.dims[1], d.dims[2] = 2048, 1024, 1056
    d.on_device = 1
    buf = torch.zeros(16, dtype=torch.int64, device=env["dev"])
    d.data = buf.data_ptr()
    p = v.EncodeParams(4.0, 2, 0, 8, 0)
    st = v.lib().vdbc_select_bricks_noalloc(ctypes.byref(d), ctypes.byref(p), buf.data_ptr(), buf.data_ptr(),
                                            buf.data_ptr(), None)
    assert st == v.ERR_INVALID_ARG
    assert "65536" in v.vdbc_last_error()
