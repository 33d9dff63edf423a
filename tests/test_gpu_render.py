"""GPU renderer parity against the FP64 CPU oracle with the shared Philox RNG.

Tolerances: emission-absorption marching max abs 1e-4 per channel; path
tracing mean abs 1e-4 per channel (FP32 tracking against FP64: rare branch
flips of single paths are expected and bounded by the mean).  The dense
hardware texture filters with 8-bit weights, so it is compared by PSNR.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EA_MAX_ABS = 1e-4
PT_MEAN_ABS = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__ as g
    g.build()
    import oracle
    import paper_2504_04564_gb300 as v
    import volgen
    from volgen import scenes
    return dict(torch=torch, v=v, orc=oracle, vg=volgen, sc=scenes, dev=torch.device("cuda:0"))


def gpu_image(env, target, cam_args, med, spp, seed, dense=False):
    torch, v = env["torch"], env["v"]
    out = torch.full((cam_args[2], cam_args[1], 4), -1.0, dtype=torch.float32, device=env["dev"])
    cam = v.make_camera(*cam_args)
    if dense:
        v.vdbc_render_dense(target, cam, med, spp, seed, out)
    else:
        v.vdbc_render(target, cam, med, spp, seed, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def oracle_image(env, D, cam_args, mode, spp, seed, macrocell=8, threads=8, **kw):
    orc = env["orc"]
    mx = orc.macrocell_minmax(D, macrocell)[1] if mode == 1 else None
    med = orc.make_medium(mode, macrocell=macrocell, **kw)
    return orc.render_image(D, mx, orc.make_camera(*cam_args), med, spp, seed, threads=threads)


def encoded(env, kind, dims, seed, ratio, payload=0):
    torch, v, orc, vg = env["torch"], env["v"], env["orc"], env["vg"]
    host = vg.generate_host(vg.make_params(kind, dims, seed))
    grid = v.vdbc_encode(torch.from_numpy(host).to(env["dev"]), ratio, payload=payload)
    e = orc.encode(host, ratio, payload=payload)
    D = orc.decode_dense(host, e["active"], e["background_bits"], payload)
    return host, grid, D


# ------------------------------------------------------------------ EA
def test_ea_blobs64_ortho_matches_oracle(env):
    """64^3 blobs at 1:4, EA step 0.5, linear-ramp TF, 128^2 ortho on +z."""
    v, sc = env["v"], env["sc"]
    w = sc.BLOBS_64_EA
    host, grid, D = encoded(env, w["kind"], w["dims"], w["seed"], w["ratio"])
    cam = sc.ortho_plus_z(w["dims"], w["width"], w["height"])
    tf = sc.linear_ramp_tf()
    got = gpu_image(env, grid, cam, v.make_medium(v.MODE_EA, tf=tf, step=w["step"]), 1, 0)
    ref = oracle_image(env, D, cam, 0, 1, 0, tf=tf, step=w["step"])
    assert np.abs(got - ref).max() <= EA_MAX_ABS
    assert ref[..., 3].max() > 0.5          # not an empty picture


@pytest.mark.parametrize("payload", [0, 1, 2])
def test_ea_pinhole_ragged_image(env, payload):
    v, sc = env["v"], env["sc"]
    dims = (53, 41, 70)
    host, grid, D = encoded(env, "turbulence", dims, 2, 3.0, payload)
    cam = sc.pinhole_orbit(dims, 67, 45)      # 3015 pixels: not a multiple of the block
    tf = sc.linear_ramp_tf(64) * np.float32([1.0, 0.7, 0.4, 0.3])
    got = gpu_image(env, grid, cam, v.make_medium(v.MODE_EA, tf=tf, step=0.37), 1, 0)
    ref = oracle_image(env, D, cam, 0, 1, 0, tf=tf, step=0.37)
    assert np.abs(got - ref).max() <= EA_MAX_ABS


def test_ea_dense_linear_equals_oracle_on_input(env):
    torch, v, sc, vg = env["torch"], env["v"], env["sc"], env["vg"]
    dims = (48, 40, 36)
    host = vg.generate_host(vg.make_params("blobs", dims, 6))
    vol = v.vdbc_volume_create(torch.from_numpy(host).to(env["dev"]), v.FILTER_LINEAR)
    cam = sc.ortho_plus_z(dims, 50, 40)
    tf = sc.linear_ramp_tf()
    got = gpu_image(env, vol, cam, v.make_medium(v.MODE_EA, tf=tf, step=0.5), 1, 0, dense=True)
    ref = oracle_image(env, host, cam, 0, 1, 0, tf=tf, step=0.5)
    assert np.abs(got - ref).max() <= EA_MAX_ABS


# ------------------------------------------------------------------ PT
@pytest.mark.parametrize("payload", [0, 1, 2])
def test_pt_turbulence_matches_oracle(env, payload):
    v, sc = env["v"], env["sc"]
    dims = (96, 96, 96)
    host, grid, D = encoded(env, "turbulence", dims, 1, 4.0, payload)
    cam = sc.pinhole_orbit(dims, 48, 40)
    med = sc.pt_medium_args()
    got = gpu_image(env, grid, cam, v.make_medium(v.MODE_PT, **med), 4, 123)
    ref = oracle_image(env, D, cam, 1, 4, 123, **med)
    err = np.abs(got[..., :3] - ref[..., :3]).mean(axis=(0, 1))
    assert np.all(err <= PT_MEAN_ABS), err
    assert ref[..., 0].std() > 0.01          # a lit, non-trivial picture
    st = v.vdbc_render_stats_get(grid)
    assert st.paths == 48 * 40 * 4 and st.error_flags == 0 and st.lookups > 48 * 40 * 4


@pytest.mark.parametrize("macrocell", [16, 5, 48, 56, 100, 128])
def test_pt_macrocell_sizes_match_oracle(env, macrocell):
    """Majorant macrocells of other sizes (the benchmarks use 56^3 and 128^3)
    change the free flights but not the parity with the oracle; 100 and 128
    leave partial cells at the volume's far faces, 128 one cell across y and z."""
    torch, v, orc, vg, sc = env["torch"], env["v"], env["orc"], env["vg"], env["sc"]
    dims = (112, 96, 80)
    host = vg.generate_host(vg.make_params("turbulence", dims, 4))
    grid = v.vdbc_encode(torch.from_numpy(host).to(env["dev"]), 6.0, macrocell=macrocell)
    e = orc.encode(host, 6.0)
    D = orc.decode_dense(host, e["active"], e["background_bits"])
    cam = sc.pinhole_orbit(dims, 40, 36)
    med = sc.pt_medium_args()
    got = gpu_image(env, grid, cam, v.make_medium(v.MODE_PT, **med), 4, 77)
    ref = oracle_image(env, D, cam, 1, 4, 77, macrocell=macrocell, **med)
    err = np.abs(got[..., :3] - ref[..., :3]).mean(axis=(0, 1))
    assert np.all(err <= PT_MEAN_ABS), err


def test_pt_blobs_lossless_vdb_equals_dense_linear(env):
    """At 1:1 the decoded grid is the input, so the grid render and the linear
    plain-form render run the same arithmetic on the same values."""
    torch, v, sc, vg = env["torch"], env["v"], env["sc"], env["vg"]
    dims = (64, 64, 64)
    host = vg.generate_host(vg.make_params("blobs", dims, 0))
    t = torch.from_numpy(host).to(env["dev"])
    grid = v.vdbc_encode(t, 1.0)
    vol = v.vdbc_volume_create(t, v.FILTER_LINEAR)
    cam = sc.pinhole_orbit(dims, 40, 40)
    med = v.make_medium(v.MODE_PT, **sc.pt_medium_args(density_scale=40.0))
    a = gpu_image(env, grid, cam, med, 8, 5)
    b = gpu_image(env, vol, cam, med, 8, 5, dense=True)
    assert np.array_equal(a, b)
    ref = oracle_image(env, host, cam, 1, 8, 5, **sc.pt_medium_args(density_scale=40.0))
    assert np.all(np.abs(a[..., :3] - ref[..., :3]).mean(axis=(0, 1)) <= PT_MEAN_ABS)


def test_pt_dense_texture_close_to_linear(env):
    torch, v, sc, vg = env["torch"], env["v"], env["sc"], env["vg"]
    dims = (80, 64, 72)
    host = vg.generate_host(vg.make_params("turbulence", dims, 3))
    t = torch.from_numpy(host).to(env["dev"])
    tex = v.vdbc_volume_create(t, v.FILTER_TEXTURE)
    lin = v.vdbc_volume_create(t, v.FILTER_LINEAR)
    cam = sc.pinhole_orbit(dims, 64, 64)
    med = v.make_medium(v.MODE_PT, **sc.pt_medium_args())
    a = gpu_image(env, tex, cam, med, 64, 9, dense=True)
    b = gpu_image(env, lin, cam, med, 64, 9, dense=True)
    mse = float(np.mean((a[..., :3] - b[..., :3]) ** 2))
    assert 10 * math.log10(1.0 / max(mse, 1e-30)) > 35.0


def test_pt_edge_cases(env):
    torch, v, sc = env["torch"], env["v"], env["sc"]
    med_args = sc.pt_medium_args()
    med = v.make_medium(v.MODE_PT, **med_args)
    # empty volume: every path escapes, every pixel is the environment
    z = np.zeros((20, 30, 10), dtype=np.float32)
    g = v.vdbc_encode(torch.from_numpy(z).to(env["dev"]), 1.0)
    img = gpu_image(env, g, sc.pinhole_orbit((10, 30, 20), 9, 7), med, 3, 1)
    assert np.allclose(img[..., :3], 0.25) and np.all(img[..., 3] == 1.0)
    # a single pixel, one sample; a single voxel volume
    one = np.full((1, 1, 1), 0.8, dtype=np.float32)
    g1 = v.vdbc_encode(torch.from_numpy(one).to(env["dev"]), 1.0)
    cam = sc.pinhole_orbit((1, 1, 1), 1, 1)
    got = gpu_image(env, g1, cam, med, 1, 3)
    ref = oracle_image(env, one, cam, 1, 1, 3, **med_args)
    assert np.abs(got - ref).max() < 1e-4
    # camera looking away: environment only
    cam = (1, 5, 4, (0.5, 0.5, -2.0), (0.5, 0.5, -3.0), (0, 1, 0), 30.0)
    g2 = v.vdbc_encode(torch.from_numpy(np.ones((8, 8, 8), np.float32)).to(env["dev"]), 1.0)
    assert np.allclose(gpu_image(env, g2, cam, med, 2, 0)[..., :3], 0.25)


def test_pt_white_furnace_gpu(env):
    torch, v, sc, vg = env["torch"], env["v"], env["sc"], env["vg"]
    dims = (40, 40, 40)
    host = vg.generate_host(vg.make_params("turbulence", dims, 7))
    g = v.vdbc_encode(torch.from_numpy(host).to(env["dev"]), 2.0)
    med = v.make_medium(v.MODE_PT, density_scale=30.0, albedo=1.0, g=0.5, max_bounces=4096,
                        sun_dir=(0, 0, 1), sun_rad=(0, 0, 0), env_rad=(0.6, 0.6, 0.6))
    img = gpu_image(env, g, sc.pinhole_orbit(dims, 32, 32), med, 4, 2)
    assert np.allclose(img[..., :3], 0.6, atol=1e-6)


def test_loop_bound_sets_device_flag(env):
    """A cell whose majorant is positive (one voxel on its dilated border) but
    whose density is zero along the ray, with a majorant so large that every
    Woodcock step underflows against t: the walk cannot leave the cell, hits
    the per-cell step bound, stops the path and raises the kernel's error word;
    the host reports DEVICE_FLAG (no trap) and the context stays usable."""
    torch, v = env["torch"], env["v"]
    vol = np.zeros((8, 8, 16), dtype=np.float32)     # nz=8, ny=8, nx=16: two macrocells along x
    vol[4, 4, 8] = 1.0                                # inside cell 1, on cell 0's dilated border
    g = v.vdbc_encode(torch.from_numpy(vol).to(env["dev"]), 1.0)
    assert v.vdbc_grid_macrocells(g)[1][0] == 1.0
    M = 16.0
    # orthographic 1x1 camera on +z through index (2, 4): inside cell 0, density 0 there
    cam = v.make_camera(v.CAM_ORTHO, 1, 1, ((2 + 0.5) / M, (4 + 0.5) / M, -1.0), ((2 + 0.5) / M, (4 + 0.5) / M, 0.0),
                        (0, 1, 0), 0.01)
    med = v.make_medium(v.MODE_PT, density_scale=3e38, albedo=0.0, max_bounces=1, env_rad=(1, 1, 1))
    out = np.zeros((1, 1, 4), dtype=np.float32)
    with pytest.raises(v.VdbcError) as ex:
        v.vdbc_render(g, cam, med, 1, 0, out)
    assert ex.value.status == v.ERR_DEVICE_FLAG
    ok = v.make_medium(v.MODE_PT, density_scale=1.0, albedo=0.0, max_bounces=1, env_rad=(1, 1, 1))
    v.vdbc_render(g, cam, ok, 1, 0, out)
    assert abs(out[0, 0, 0] - 1.0) < 1e-6


def test_philox_device_matches_oracle_and_published_vectors(env):
    import os
    v, orc = env["v"], env["orc"]
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for r in rows:
        vals = [int(x, 16) for x in r]
        got = v.vdbc_philox([vals[:4]], vals[4:6])[0]
        assert list(got) == vals[6:10]
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = np.array([0xDEADBEEF, 0x12345678], dtype=np.uint32)
    got = v.vdbc_philox(ctr, key)
    for i in range(0, 4096, 97):
        assert np.array_equal(got[i], orc.philox(ctr[i], key))


def test_full_size_turbulence_sampled_pixels(env):
    """The benchmark's launch configuration (512^3 medium at 1:10, 1024^2, 16
    spp, one launch): 256 sampled pixels against the FP64 oracle."""
    torch, v, orc, vg, sc = env["torch"], env["v"], env["orc"], env["vg"], env["sc"]
    w = sc.TURBULENCE_512
    p = vg.make_params(w["kind"], w["dims"], w["seed"])
    host = vg.generate_host(p)
    grid = v.vdbc_encode(vg.generate_torch(p), w["ratio"], macrocell=w["macrocell"])
    cam_args = sc.pinhole_orbit(w["dims"], w["width"], w["height"])
    out = torch.empty((w["height"], w["width"], 4), dtype=torch.float32, device=env["dev"])
    v.vdbc_render(grid, v.make_camera(*cam_args), v.make_medium(v.MODE_PT, **w["medium"]), w["spp"], 2024, out)
    img = out.cpu().numpy().reshape(-1, 4).astype(np.float64)
    e = orc.encode(host, w["ratio"])
    D = orc.decode_dense(host, e["active"], e["background_bits"])
    mx = orc.macrocell_minmax(D, w["macrocell"])[1]
    rng = np.random.default_rng(11)
    pix = np.sort(rng.choice(w["width"] * w["height"], 256, replace=False))
    ref = orc.render_pixels(D, mx, orc.make_camera(*cam_args), orc.make_medium(1, macrocell=w["macrocell"], **w["medium"]),
                            w["spp"], 2024, pix, threads=8)
    err = np.abs(img[pix, :3] - ref[:, :3]).mean(axis=0)
    assert np.all(err <= PT_MEAN_ABS), err


def test_pt_coarse_level_changes_no_image(env, monkeypatch):
    """The coarse DDA level (opt-in, VDBC_PT_COARSE=1) crosses empty 8^3 blocks
    of macrocells in one step, landing where cell-by-cell stepping lands: the
    images are bit-identical with and without it, and match the oracle."""
    torch, v, orc, vg, sc = env["torch"], env["v"], env["orc"], env["vg"], env["sc"]
    dims = (128, 112, 120)
    host = vg.generate_host(vg.make_params("blobs", dims, 6))
    grid = v.vdbc_encode(torch.from_numpy(host).to(env["dev"]), 4.0, macrocell=4)
    cam = sc.pinhole_orbit(dims, 48, 40)
    med = v.make_medium(v.MODE_PT, **sc.pt_medium_args(density_scale=30.0))
    monkeypatch.setenv("VDBC_PT_COARSE", "1")
    on = gpu_image(env, grid, cam, med, 8, 3)
    monkeypatch.setenv("VDBC_PT_COARSE", "0")
    off = gpu_image(env, grid, cam, med, 8, 3)
    assert np.array_equal(on, off)
    e = orc.encode(host, 4.0)
    D = orc.decode_dense(host, e["active"], e["background_bits"])
    ref = oracle_image(env, D, cam, 1, 8, 3, macrocell=4, **sc.pt_medium_args(density_scale=30.0))
    assert np.all(np.abs(on[..., :3] - ref[..., :3]).mean(axis=(0, 1)) <= PT_MEAN_ABS)


def test_pt_lookup_modes_and_work_chunks_change_no_image(env, monkeypatch):
    """The stencil modes (one-leaf path per lane, one path per warp, up to four
    leaves at once, the accessor at depth 2) fetch the same eight values and
    interpolate them in the same order, and the work chunks and the work order
    (tile first or sample first) only change which lane renders which path
    (the per-pixel sums are integers): every variant renders the default image
    bit for bit, with the same lookup count."""
    torch, v, vg, sc = env["torch"], env["v"], env["vg"], env["sc"]
    dims = (120, 104, 112)
    host = vg.generate_host(vg.make_params("turbulence", dims, 8))
    grid = v.vdbc_encode(torch.from_numpy(host).to(env["dev"]), 6.0, macrocell=16)
    cam = sc.pinhole_orbit(dims, 64, 48)
    med = v.make_medium(v.MODE_PT, **sc.pt_medium_args())
    base = gpu_image(env, grid, cam, med, 8, 5)
    lookups = v.vdbc_render_stats_get(grid).lookups
    for name, values in (("VDBC_PT_LOOKUP", ["11", "12", "22", "24"]), ("VDBC_PT_CHUNK", ["32", "64", "128", "256"]),
                         ("VDBC_PT_ORDER", ["sample"])):
        for val in values:
            monkeypatch.setenv(name, val)
            img = gpu_image(env, grid, cam, med, 8, 5)
            assert np.array_equal(img, base), (name, val)
            assert v.vdbc_render_stats_get(grid).lookups == lookups, (name, val)
        monkeypatch.delenv(name)
    grid.close()


def test_render_stats_time_the_tracker_kernel(env):
    """kernel_ms: CUDA events around the tracker's launch, positive for every mode."""
    torch, v, vg, sc = env["torch"], env["v"], env["vg"], env["sc"]
    dims = (48, 40, 44)
    host = vg.generate_host(vg.make_params("blobs", dims, 1))
    t = torch.from_numpy(host).to(env["dev"])
    grid = v.vdbc_encode(t, 2.0)
    vol = v.vdbc_volume_create(t, v.FILTER_TEXTURE)
    cam = v.make_camera(*sc.pinhole_orbit(dims, 32, 24))
    out = torch.zeros(24, 32, 4, device=env["dev"])
    for med, spp in ((v.make_medium(v.MODE_PT, **sc.pt_medium_args()), 4),
                     (v.make_medium(v.MODE_EA, tf=sc.linear_ramp_tf(), step=0.5), 1),
                     (v.make_medium(v.MODE_ISO, step=0.5, iso=0.3), 1)):
        v.vdbc_render(grid, cam, med, spp, 1, out)
        st = v.vdbc_render_stats_get(grid)
        assert 0.0 < st.kernel_ms < 1e4
        v.vdbc_render_dense(vol, cam, med, spp, 1, out)
        assert 0.0 < v.vdbc_volume_render_stats_get(vol).kernel_ms < 1e4


def test_concurrent_calls_on_two_threads(env):
    """Two host threads, each on its own stream, encode from pinned host
    memory and path trace into host memory at the same time, as the
    end-to-end benchmark does: every image equals the one-thread render of
    the same grid and samples, and no call fails."""
    import threading

    torch, v, vg, sc = env["torch"], env["v"], env["vg"], env["sc"]
    dims = (96, 80, 72)
    vols = [torch.from_numpy(vg.generate_host(vg.make_params("turbulence", dims, s))).pin_memory() for s in (5, 6)]
    cam = v.make_camera(*sc.pinhole_orbit(dims, 48, 40))
    med = v.make_medium(v.MODE_PT, **sc.pt_medium_args(density_scale=30.0, max_bounces=6))
    want = []
    for vol in vols:
        g = v.vdbc_encode(vol, 6.0, macrocell=16)
        img = np.zeros((40, 48, 4), dtype=np.float32)
        v.vdbc_render(g, cam, med, 4, 11, img)
        want.append(img)
        g.close()
    got = [[], []]
    errors = []

    def worker(i):
        try:
            torch.cuda.set_device(env["dev"])
            st = torch.cuda.Stream(device=env["dev"])
            for _ in range(4):
                g = v.vdbc_encode(vols[i], 6.0, macrocell=16, stream=st.cuda_stream)
                img = np.zeros((40, 48, 4), dtype=np.float32)
                v.vdbc_render(g, cam, med, 4, 11, img, stream=st.cuda_stream)
                g.close()
                got[i].append(img)
        except Exception as ex:     # reported on the test's thread
            errors.append(ex)

    ts = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    for i in range(2):
        assert len(got[i]) == 4
        for img in got[i]:
            assert np.array_equal(img.view(np.uint32), want[i].view(np.uint32))


def test_pt_across_the_root_boundary_matches_oracle(env):
    """A volume 8192 voxels long (the largest edge; two root-table entries
    along x), path traced by an orthographic camera that looks along +y at
    the 64 voxels around x = 4096, where lookups switch root entries: mean abs
    error per channel within the path-tracing tolerance of the FP64 oracle."""
    torch, v, vg = env["torch"], env["v"], env["vg"]
    dims = (8192, 4, 6)
    host = vg.generate_host(vg.make_params("turbulence", dims, 3))
    grid = v.vdbc_encode(torch.from_numpy(host).to(env["dev"]), 2.0, macrocell=16)
    assert grid.info.n_upper == 2
    orc = env["orc"]
    e = orc.encode(host, 2.0)
    D = orc.decode_dense(host, e["active"], e["background_bits"])
    M = 8192.0
    xc, zc = (4095.5 + 0.5) / M, (2.5 + 0.5) / M
    cam = (v.CAM_ORTHO, 64, 6, (xc, -1.0, zc), (xc, 0.0, zc), (0, 0, 1), 6.0 / M)
    kw = env["sc"].pt_medium_args(density_scale=3000.0, g=0.5, max_bounces=4)
    img = gpu_image(env, grid, cam, v.make_medium(v.MODE_PT, **kw), 8, 5)
    ref = oracle_image(env, D, cam, 1, 8, 5, macrocell=16, **kw)
    assert img[..., 3].min() > 0.0
    err = np.abs(img[..., :3] - ref[..., :3]).mean(axis=(0, 1))
    assert np.all(err <= PT_MEAN_ABS), err
    assert np.abs(img[..., :3] - 0.25).max() > 1e-3       # the medium is seen, not just the environment


def test_bad_cameras_and_media_rejected_before_any_launch(env):
    """A camera without a basis or a medium out of range is refused with
    INVALID_ARG before any device work; the same grid renders afterwards."""
    torch, v, sc = env["torch"], env["v"], env["sc"]
    dims = (24, 20, 28)
    g = v.vdbc_encode(torch.from_numpy(env["vg"].generate_host(env["vg"].make_params("blobs", dims, 2))).to(env["dev"]),
                      2.0)
    out = torch.zeros(6, 8, 4, device=env["dev"])
    good_cam = sc.pinhole_orbit(dims, 8, 6)
    pt = sc.pt_medium_args()
    nan = float("nan")
    bad_cams = [
        (1, 8, 6, (0.5, 0.5, 0.5), (0.5, 0.5, 0.5), (0, 1, 0), 40.0),      # look == eye
        (1, 8, 6, (0.5, 2.0, 0.5), (0.5, 0.0, 0.5), (0, 1, 0), 40.0),      # up along the view
        (1, 8, 6, (nan, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), 40.0),      # non-finite eye
        (1, 8, 6, (0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 0, 0), 40.0),      # zero up
        (1, 8, 6, (0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), 180.0),     # field of view
        (0, 8, 6, (0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), float("inf")),  # ortho height
        (1, 0, 6, (0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), 40.0),      # width 0
        (1, 16385, 6, (0.5, 0.5, 2.0), (0.5, 0.5, 0.5), (0, 1, 0), 40.0),  # width too large
    ]
    for cam in bad_cams:
        with pytest.raises(v.VdbcError) as ex:
            v.vdbc_render(g, v.make_camera(*cam), v.make_medium(v.MODE_PT, **pt), 1, 0, out)
        assert ex.value.status == v.ERR_INVALID_ARG, cam
    bad_media = [
        (v.make_medium(v.MODE_PT, **dict(pt, density_scale=float("inf"))), 1),
        (v.make_medium(v.MODE_PT, **dict(pt, density_scale=-1.0)), 1),
        (v.make_medium(v.MODE_PT, **dict(pt, albedo=1.5)), 1),
        (v.make_medium(v.MODE_PT, **dict(pt, g=1.0)), 1),
        (v.make_medium(v.MODE_PT, **dict(pt, max_bounces=0)), 1),
        (v.make_medium(v.MODE_PT, **dict(pt, sun_dir=(0, 0, 0))), 1),
        (v.make_medium(v.MODE_PT, **dict(pt, env_rad=(nan, 0, 0))), 1),
        (v.make_medium(v.MODE_PT, **pt), 0),
        (v.make_medium(v.MODE_EA, tf=sc.linear_ramp_tf(), step=0.5), 2),
        (v.make_medium(v.MODE_EA, tf=sc.linear_ramp_tf()[:1], step=0.5), 1),
        (v.make_medium(v.MODE_EA, tf=sc.linear_ramp_tf(), step=0.0), 1),
        (v.make_medium(v.MODE_ISO, step=0.5, iso=nan), 1),
    ]
    for med, spp in bad_media:
        with pytest.raises(v.VdbcError) as ex:
            v.vdbc_render(g, v.make_camera(*good_cam), med, spp, 0, out)
        assert ex.value.status == v.ERR_INVALID_ARG, (med.mode, spp)
    v.vdbc_render(g, v.make_camera(*good_cam), v.make_medium(v.MODE_PT, **pt), 2, 0, out)
    torch.cuda.synchronize()
    assert np.isfinite(out.cpu().numpy()).all() and v.vdbc_render_stats_get(g).paths == 8 * 6 * 2
