"""The ISO-surface marcher on the GPU against the FP64 oracle's plain march.

The GPU skips macrocells whose range excludes the iso value; the oracle looks
up every sample.  Agreement: the hit masks and, on pixels both hit, the
normal colours.  An FP32 sample that lands within rounding of the iso value
can flip the inside test and move a crossing, so a few pixels may differ;
the bound is 0.5 % of the pixels, and 1e-3 max-abs on the others (the
bisection pins the hit to step / 2^12, the normal is a smooth function of
it).  Skipping is exact: images are bit-identical across macrocell sizes,
and the grid render equals the linear dense render of the same values.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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


def gpu_iso(env, target, cam_args, iso=0.5, step=0.5, dense=False):
    torch, v = env["torch"], env["v"]
    out = torch.full((cam_args[2], cam_args[1], 4), -1.0, dtype=torch.float32, device=env["dev"])
    med = v.make_medium(v.MODE_ISO, step=step, iso=iso)
    (v.vdbc_render_dense if dense else v.vdbc_render)(target, v.make_camera(*cam_args), med, 1, 0, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def oracle_iso(env, D, cam_args, iso=0.5, step=0.5):
    orc = env["orc"]
    return orc.render_image(D, None, orc.make_camera(*cam_args), orc.make_medium(orc.MODE_ISO, step=step, iso=iso),
                            1, 0, threads=8)


def compare(got, ref):
    hit_g, hit_r = got[..., 3] == 1.0, ref[..., 3] == 1.0
    assert np.all((got[..., 3] == 0.0) | hit_g)
    assert np.all(got[~hit_g] == 0.0)
    differ = hit_g != hit_r
    assert differ.mean() <= 0.005
    both = hit_g & hit_r
    d = np.abs(got[both][:, :3] - ref[both][:, :3]).max(axis=1)
    print("\nISO: %d pixels hit by both, hit masks differ on %.4f, colour max-abs > 1e-3 on %.4f, median %.2g"
          % (both.sum(), differ.mean(), np.mean(d > 1e-3), np.median(d)))
    assert np.mean(d > 1e-3) <= 0.005
    return int(both.sum()), float(differ.mean())


@pytest.mark.parametrize("payload,ratio", [(0, 4.0), (1, 2.0), (2, 1.0)])
def test_iso_matches_oracle(env, payload, ratio):
    torch, v, orc, vg, sc = env["torch"], env["v"], env["orc"], env["vg"], env["sc"]
    dims = (64, 64, 64)
    host = vg.generate_host(vg.make_params("blobs", dims, 0))
    grid = v.vdbc_encode(torch.from_numpy(host).to(env["dev"]), ratio, payload=payload)
    e = orc.encode(host, ratio, payload=payload)
    D = orc.decode_dense(host, e["active"], e["background_bits"], payload)
    for iso in (0.3, 0.5):
        cam = sc.pinhole_orbit(dims, 72, 56)
        got = gpu_iso(env, grid, cam, iso=iso)
        ref = oracle_iso(env, D, cam, iso=iso)
        hits, _ = compare(got, ref)
        assert hits > 300


def test_iso_sphere_and_ragged_image(env):
    torch, v, orc, sc = env["torch"], env["v"], env["orc"], env["sc"]
    dims = (45, 38, 51)
    z, y, x = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
    r = np.sqrt((x - 22.0) ** 2 + (y - 18.5) ** 2 + (z - 25.0) ** 2)
    host = np.clip(1.0 - r / 34.0, 0.0, 1.0).astype(np.float32)
    grid = v.vdbc_encode(torch.from_numpy(host).to(env["dev"]), 1.0)
    cam = sc.pinhole_orbit(dims, 61, 47)
    got = gpu_iso(env, grid, cam, step=0.3)
    ref = oracle_iso(env, host, cam, step=0.3)
    hits, _ = compare(got, ref)
    assert hits > 500


def test_iso_skipping_is_exact_across_macrocell_sizes(env):
    """Different macrocell grids skip different samples; the image cannot change."""
    torch, v, vg, sc = env["torch"], env["v"], env["vg"], env["sc"]
    dims = (80, 72, 64)
    host = torch.from_numpy(vg.generate_host(vg.make_params("turbulence", dims, 4))).to(env["dev"])
    cam = sc.pinhole_orbit(dims, 64, 48)
    imgs = [gpu_iso(env, v.vdbc_encode(host, 3.0, macrocell=mc), cam, iso=0.35) for mc in (4, 8, 16, 64)]
    for im in imgs[1:]:
        assert np.array_equal(im, imgs[0])
    assert (imgs[0][..., 3] == 1.0).sum() > 200


def test_iso_grid_equals_dense_linear(env):
    torch, v, vg, sc = env["torch"], env["v"], env["vg"], env["sc"]
    dims = (64, 64, 64)
    host = torch.from_numpy(vg.generate_host(vg.make_params("blobs", dims, 2))).to(env["dev"])
    grid = v.vdbc_encode(host, 1.0)
    vol = v.vdbc_volume_create(host, v.FILTER_LINEAR)
    cam = sc.pinhole_orbit(dims, 40, 40)
    assert np.array_equal(gpu_iso(env, grid, cam), gpu_iso(env, vol, cam, dense=True))


def test_iso_edge_cases(env):
    torch, v, sc = env["torch"], env["v"], env["sc"]
    dims = (16, 16, 16)
    zero = torch.zeros(16, 16, 16, device=env["dev"])
    grid = v.vdbc_encode(zero, 1.0)
    assert np.all(gpu_iso(env, grid, sc.pinhole_orbit(dims, 9, 7)) == 0.0)
    one = v.vdbc_encode(torch.ones(1, 1, 1, device=env["dev"]), 1.0)
    assert np.all(gpu_iso(env, one, sc.pinhole_orbit((1, 1, 1), 5, 5)) == 0.0)   # inside everywhere
    with pytest.raises(v.VdbcError):
        out = torch.zeros(4, 4, 4, device=env["dev"])
        v.vdbc_render(grid, v.make_camera(*sc.pinhole_orbit(dims, 4, 4)), v.make_medium(v.MODE_ISO, step=0.5), 2, 0,
                      out)
