"""Host-side fault injection (VDBC_FAULT) on the GPU build, with no GPU
fault: the library's bounded waits time out on work that is merely slow,
and corrupt files are refused before any device work.

Timeouts: the stream is first given a few tens of milliseconds of torch's
bounded sleep kernel, so the call's own work is still queued when its wait
(limit 0 under VDBC_FAULT=timeout) looks.  The call must return
VDBC_ERR_TIMEOUT without freeing what that work uses; once the caller has
synchronized the stream, the output buffer holds what the call would have
given and every handle works as before.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SLEEP_CYCLES = 100_000_000      # about 50 ms at the GB300's 2 GHz SM clock


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2504_04564_gb300 as v
    import volgen
    from volgen import scenes
    vol = volgen.generate_torch(volgen.make_params("turbulence", (96, 80, 72), 3))
    grid = v.vdbc_encode(vol, 4.0, macrocell=16)
    torch.cuda.synchronize()
    return dict(torch=torch, v=v, vg=volgen, sc=scenes, vol=vol, grid=grid)


def busy_stream(torch):
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        torch.cuda._sleep(SLEEP_CYCLES)
    return s


def scene(env, w=96, h=64):
    v, sc = env["v"], env["sc"]
    cam = v.make_camera(*sc.pinhole_orbit((96, 80, 72), w, h))
    med = v.make_medium(v.MODE_PT, **sc.pt_medium_args())
    return cam, med


def test_timed_out_render_keeps_its_queued_copy_valid(env, monkeypatch):
    torch, v, grid = env["torch"], env["v"], env["grid"]
    cam, med = scene(env)
    want = np.zeros((64, 96, 4), dtype=np.float32)
    v.vdbc_render(grid, cam, med, 4, 9, want)
    out = torch.full((64, 96, 4), -1.0, dtype=torch.float32).pin_memory()   # an asynchronous D2H target
    s = busy_stream(torch)
    monkeypatch.setenv("VDBC_FAULT", "timeout")
    with pytest.raises(v.VdbcError) as ex:
        v.vdbc_render(grid, cam, med, 4, 9, out, stream=s)
    monkeypatch.delenv("VDBC_FAULT")
    assert ex.value.status == v.ERR_TIMEOUT
    s.synchronize()
    assert np.array_equal(out.numpy(), want)
    again = np.zeros_like(want)
    v.vdbc_render(grid, cam, med, 4, 9, again)             # the grid is usable as before
    assert np.array_equal(again, want)


def test_timed_out_decode_keeps_its_queued_copy_valid(env, monkeypatch):
    torch, v, grid, vol = env["torch"], env["v"], env["grid"], env["vol"]
    want = np.empty(tuple(vol.shape), dtype=np.float32)
    v.vdbc_grid_decode(grid, want)
    out = torch.full(tuple(vol.shape), -1.0, dtype=torch.float32).pin_memory()
    s = busy_stream(torch)
    monkeypatch.setenv("VDBC_FAULT", "timeout")
    with pytest.raises(v.VdbcError) as ex:
        v.vdbc_grid_decode(grid, out, stream=s)
    monkeypatch.delenv("VDBC_FAULT")
    assert ex.value.status == v.ERR_TIMEOUT
    s.synchronize()
    assert np.array_equal(out.numpy().view(np.uint32), want.view(np.uint32))


def test_timed_out_learn_returns_no_grid_and_releases_it_later(env, monkeypatch):
    """The learned grid a timed-out vdbc_learn would have returned is released
    only after its queued work; later calls (which run that release) work."""
    torch, v, grid = env["torch"], env["v"], env["grid"]
    timed_out = 0
    for _ in range(3):
        s = torch.cuda.Stream()
        monkeypatch.setenv("VDBC_FAULT", "timeout")
        try:
            g, _ = v.vdbc_learn(grid, steps=3, samples_per_leaf=16, stream=s)
            g.close()
        except v.VdbcError as ex:
            assert ex.status == v.ERR_TIMEOUT
            timed_out += 1
        finally:
            monkeypatch.delenv("VDBC_FAULT")
        s.synchronize()
    assert timed_out >= 1
    g, losses = v.vdbc_learn(grid, steps=3, samples_per_leaf=16)
    assert np.isfinite(losses).all() and g.info.n_neural + g.info.n_leaves > 0
    g.close()


def test_injected_format_fault_refuses_a_good_file(env, monkeypatch, tmp_path):
    v, grid = env["v"], env["grid"]
    path = str(tmp_path / "g.vdbc")
    v.vdbc_grid_save(grid, path)
    monkeypatch.setenv("VDBC_FAULT", "format")
    with pytest.raises(v.VdbcError) as ex:
        v.vdbc_grid_load(path)
    assert ex.value.status == v.ERR_FORMAT
    monkeypatch.delenv("VDBC_FAULT")
    g = v.vdbc_grid_load(path)
    assert g.info.as_dict() == grid.info.as_dict()
    g.close()
