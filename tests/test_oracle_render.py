"""Pins of the oracle's renderer (Section 4 plus the project's EA marcher and
ratio tracker).

Closed forms: trilinear reproduction of linear fields, the EA slab
C = c (1 - exp(-a L)), Beer-Lambert transmittance exp(-sigma d) for both the
delta-tracking escape fraction and the ratio-tracking estimator, the
single-scattering slab integral, the white furnace, the Henyey-Greenstein
normalization and mean cosine.  Brute force: ray/box clipping and the DDA
cell sequence against dense sampling along the ray.
"""
import math

import numpy as np
import pytest


def const_volume(dims, c):
    nx, ny, nz = dims
    return np.full((nz, ny, nx), c, dtype=np.float32)


def ortho_z(orc, dims, w, h):
    """Orthographic camera looking down +z, the image covering the x-y extent."""
    nx, ny, nz = dims
    M = max(dims)
    cx, cy = 0.5 * nx / M, 0.5 * ny / M
    return orc.make_camera(orc.CAM_ORTHO, w, h, (cx, cy, -1.0), (cx, cy, 0.0), (0, 1, 0), ny / M)


# ------------------------------------------------------------------ sampler
def test_trilinear_reproduces_linear_fields(orc):
    rng = np.random.default_rng(0)
    nx, ny, nz = 13, 9, 11
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    a, b, c, d = 0.3, -0.7, 0.11, 2.0
    f = (a * x + b * y + c * z + d).astype(np.float64)
    vol = f.astype(np.float32)
    for _ in range(200):
        p = rng.uniform([0, 0, 0], [nx - 1, ny - 1, nz - 1])
        exact = a * p[0] + b * p[1] + c * p[2] + d
        assert abs(orc.trilinear(vol, p) - exact) < 1e-5
    # at voxel centres it returns the voxel; outside it clamps to the edge
    assert orc.trilinear(vol, [3, 4, 5]) == float(vol[5, 4, 3])
    assert orc.trilinear(vol, [-0.4, 0, 0]) == float(vol[0, 0, 0])
    assert orc.trilinear(vol, [nx - 0.6, ny - 1, nz - 1]) == float(vol[-1, -1, -1])


def test_macrocell_minmax_brute_force(orc):
    rng = np.random.default_rng(3)
    nx, ny, nz = 20, 17, 9
    vol = rng.random((nz, ny, nx)).astype(np.float32)
    mn, mx = orc.macrocell_minmax(vol, 8)
    nc = [(n + 7) // 8 for n in (nx, ny, nz)]
    for cz in range(nc[2]):
        for cy in range(nc[1]):
            for cx in range(nc[0]):
                sl = vol[max(cz * 8 - 1, 0):min(cz * 8 + 9, nz), max(cy * 8 - 1, 0):min(cy * 8 + 9, ny),
                         max(cx * 8 - 1, 0):min(cx * 8 + 9, nx)]
                c = (cz * nc[1] + cy) * nc[0] + cx
                assert mn[c] == sl.min() and mx[c] == sl.max()


def test_majorant_bounds_every_reconstructed_value(orc):
    """The one-voxel dilation makes the cell max bound the trilinear value
    anywhere inside the cell."""
    rng = np.random.default_rng(4)
    dims = (30, 25, 19)
    vol = rng.random(dims[::-1]).astype(np.float32)
    _, mx = orc.macrocell_minmax(vol, 8)
    nc = [(n + 7) // 8 for n in dims]
    for _ in range(3000):
        p = rng.uniform(-0.5, np.array(dims) - 0.5)
        c = [min(int(math.floor((p[a] + 0.5) / 8)), nc[a] - 1) for a in range(3)]
        cid = (c[2] * nc[1] + c[1]) * nc[0] + c[0]
        assert orc.trilinear(vol, p) <= mx[cid] + 1e-7


# ------------------------------------------------------------------ geometry
def test_clip_box_brute_force(orc):
    rng = np.random.default_rng(5)
    dims = (20, 11, 7)
    lo, hi = -0.5, np.array(dims) - 0.5
    for _ in range(300):
        o = rng.uniform(-15, 30, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        hit, tin, tout = orc.clip_box(dims, o, d)
        ts = np.linspace(0, 60, 60001)
        pts = o[None, :] + ts[:, None] * d[None, :]
        inside = np.all((pts >= lo) & (pts <= hi), axis=1)
        if not inside.any():
            assert not hit or tout - tin < 2e-3
            continue
        assert hit
        assert abs(ts[inside][0] - tin) < 2e-3 and abs(min(ts[inside][-1], 60) - min(tout, 60)) < 2e-3


def test_dda_cells_match_dense_sampling(orc):
    rng = np.random.default_rng(6)
    dims = (37, 29, 18)
    S = 8
    nc = [(n + S - 1) // S for n in dims]
    for _ in range(200):
        o = rng.uniform(-0.5, np.array(dims) - 0.5)
        d = rng.normal(size=3)
        if rng.random() < 0.2:
            d[rng.integers(3)] = 0.0     # axis-parallel components
        d /= np.linalg.norm(d)
        hit, tin, tout = orc.clip_box(dims, o, d)
        cells, t0, t1 = orc.dda_cells(dims, S, o, d, tin, tout)
        # consecutive, contiguous segments covering [tin, tout]
        assert t0[0] == tin and abs(t1[-1] - tout) < 1e-9
        assert np.all(np.abs(t0[1:] - t1[:-1]) < 1e-9)
        ts = np.linspace(tin, tout, 4000)[1:-1]
        want = []
        for t in ts:
            p = o + t * d
            c = [min(max(int(math.floor((p[a] + 0.5) / S)), 0), nc[a] - 1) for a in range(3)]
            cid = (c[2] * nc[1] + c[1]) * nc[0] + c[0]
            if not want or want[-1] != cid:
                want.append(cid)
        got = [c for c, a, b in zip(cells, t0, t1) if b - a > 1e-6]
        # every cell the segment visits appears, in order (tiny slivers may be missed by sampling)
        it = iter(got)
        assert all(any(c == g for g in it) for c in want)


def test_onb_orthonormal(orc):
    rng = np.random.default_rng(7)
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        b1 = np.zeros(3)
        b2 = np.zeros(3)
        orc.lib().or_onb(orc._p(np.ascontiguousarray(n)), orc._p(b1), orc._p(b2))
        m = np.stack([b1, b2, n])
        assert np.allclose(m @ m.T, np.eye(3), atol=1e-12)


# ------------------------------------------------------------------ phase function
@pytest.mark.parametrize("g", [-0.5, 0.0, 0.6, 0.8, 0.95])
def test_hg_normalized_and_mean_cosine(orc, g):
    L = orc.lib()
    mus = np.linspace(-1, 1, 200001)
    p = np.array([L.or_hg_eval(m, g) for m in mus[::20]])
    integral = 2 * math.pi * np.trapezoid(p, mus[::20])
    assert abs(integral - 1.0) < 2e-3
    # inverse-CDF sampling: E[mu] = g (stratified xi)
    xi = (np.arange(200000) + 0.5) / 200000
    s = np.array([L.or_hg_sample_mu(g, x) for x in xi])
    assert abs(s.mean() - g) < 1e-4
    # and the sampled histogram follows the density
    counts, edges = np.histogram(s, bins=20, range=(-1, 1))
    prob = []
    for a, b in zip(edges[:-1], edges[1:]):
        m = np.linspace(a, b, 2001)
        prob.append(2 * math.pi * np.trapezoid([L.or_hg_eval(x, g) for x in m], m))
    assert np.allclose(counts / s.size, prob, rtol=1e-3, atol=2e-5)


# ------------------------------------------------------------------ camera
def test_ortho_camera_pixel_centres(orc):
    dims = (64, 64, 64)
    cam = ortho_z(orc, dims, 128, 128)
    for px, py in ((0, 0), (127, 0), (5, 77)):
        o, d = orc.camera_ray(cam, dims, px, py, 0.5, 0.5)
        assert np.allclose(d, [0, 0, 1])
        # right = forward x up = -x for a camera looking down +z (right-handed
        # look-at); world x = 1 - (px + 1/2) / 128 -> index = world * 64 - 1/2
        assert abs(o[0] - ((127 - px + 0.5) / 2 - 0.5)) < 1e-12
        assert abs(o[1] - ((127 - py + 0.5) / 2 - 0.5)) < 1e-12


def test_pinhole_camera_geometry(orc):
    """A pinhole camera's rays start at the eye; the image centre looks at
    `look`; the top and right image edges lie at half the vertical field of
    view (times the aspect ratio, on tangents) from it; the top row leans
    toward `up` and the right column toward forward x up."""
    dims = (40, 30, 20)
    M = 40.0
    eye, look, up, fov = (0.9, 0.7, -0.4), (0.45, 0.3, 0.2), (0.0, 1.0, 0.0), 50.0
    w, h = 64, 48
    cam = orc.make_camera(orc.CAM_PINHOLE, w, h, eye, look, up, fov)
    fwd = np.subtract(look, eye)
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    for px, py, jx, jy in ((0, 0, 0.5, 0.5), (17, 30, 0.2, 0.9), (63, 47, 0.5, 0.5)):
        o, d = orc.camera_ray(cam, dims, px, py, jx, jy)
        assert np.allclose(o, np.array(eye) * M - 0.5, atol=1e-12) and abs(np.linalg.norm(d) - 1) < 1e-12
    o, d = orc.camera_ray(cam, dims, w // 2 - 1, h // 2 - 1, 1.0, 1.0)      # the exact image centre
    assert np.allclose(d, fwd, atol=1e-12)
    t = math.tan(math.radians(fov / 2))
    _, top = orc.camera_ray(cam, dims, w // 2 - 1, 0, 1.0, 0.0)               # top edge, centre column
    assert abs(np.dot(top, upv) / np.dot(top, fwd) - t) < 1e-12 and abs(np.dot(top, right)) < 1e-12
    _, rgt = orc.camera_ray(cam, dims, w - 1, h // 2 - 1, 1.0, 1.0)           # right edge, centre row
    assert abs(np.dot(rgt, right) / np.dot(rgt, fwd) - t * w / h) < 1e-12 and abs(np.dot(rgt, upv)) < 1e-12


# ------------------------------------------------------------------ EA marcher
@pytest.mark.parametrize("c,alpha_scale", [(0.5, 0.02), (1.0, 0.2), (0.25, 0.0)])
def test_ea_constant_slab_closed_form(orc, c, alpha_scale):
    dims = (16, 16, 64)
    vol = const_volume(dims, c)
    tf = np.zeros((256, 4), dtype=np.float32)
    ramp = np.arange(256) / 255.0
    tf[:, 0] = ramp
    tf[:, 1] = 0.5 * ramp
    tf[:, 2] = 1.0
    tf[:, 3] = alpha_scale * ramp
    med = orc.make_medium(orc.MODE_EA, tf=tf, step=0.5)
    cam = ortho_z(orc, dims, 8, 8)
    img = orc.render_image(vol, None, cam, med, 1, 0)
    rgba = np.interp(c * 255, np.arange(256), tf[:, 0]), np.interp(c * 255, np.arange(256), tf[:, 1])
    a = alpha_scale * c
    # samples at t = (k + 1/2) * 0.5 over the 64-voxel depth: 128 steps of 0.5
    opacity = 1.0 - math.exp(-a * 64.0)
    assert np.allclose(img[..., 0], c * opacity, atol=1e-12)
    assert np.allclose(img[..., 1], 0.5 * c * opacity, atol=1e-12)
    assert np.allclose(img[..., 2], opacity, atol=1e-12)
    assert np.allclose(img[..., 3], opacity, atol=1e-12)


# ------------------------------------------------------------------ tracking
def test_delta_tracking_escape_is_beer_lambert(orc):
    """albedo 0, environment 1: each path returns 1 if it escapes, so the image
    mean estimates exp(-sigma d) for the 64-voxel slab."""
    dims = (16, 16, 64)
    c, scale = 0.5, 2.0
    vol = const_volume(dims, c)
    _, mx = orc.macrocell_minmax(vol, 8)
    med = orc.make_medium(orc.MODE_PT, density_scale=scale, albedo=0.0, max_bounces=1, macrocell=8,
                          env_rad=(1, 1, 1))
    cam = ortho_z(orc, dims, 32, 32)
    img = orc.render_image(vol, mx, cam, med, 64, 1)
    # sigma per index unit = scale * c / M, M = 64, over 64 index units
    T = math.exp(-scale * c)
    n = 32 * 32 * 64
    assert abs(img[..., 0].mean() - T) < 4 * math.sqrt(T * (1 - T) / n)


@pytest.mark.parametrize("macrocell", [8, 128])
def test_ratio_tracking_mean_is_beer_lambert(orc, macrocell):
    dims = (16, 16, 64)
    c, scale = 0.8, 3.0
    vol = const_volume(dims, c)
    _, mx = orc.macrocell_minmax(vol, macrocell)
    med = orc.make_medium(orc.MODE_PT, density_scale=scale, macrocell=macrocell)
    T = math.exp(-scale * c)
    est = [orc.ratio_transmittance(vol, mx, med, [8, 8, -0.5], [0, 0, 1], s, 0, 9) for s in range(2000)]
    # constant medium with a tight majorant: every step multiplies by exactly 0
    # or the walk never stops inside; here sigma == majorant so T is 0 or 1
    est = np.array(est)
    assert abs(est.mean() - T) < 4 * math.sqrt(T * (1 - T) / est.size)


def test_ratio_tracking_loose_majorant_unbiased(orc):
    """A majorant 3x the density: the estimator takes fractional values and
    its mean is still exp(-sigma d)."""
    dims = (16, 16, 64)
    vol = const_volume(dims, 0.3)
    mx = np.full(2 * 2 * 8, 0.9, dtype=np.float32)      # loose bound, 8^3 cells
    med = orc.make_medium(orc.MODE_PT, density_scale=4.0, macrocell=8)
    T = math.exp(-4.0 * 0.3)
    est = np.array([orc.ratio_transmittance(vol, mx, med, [3, 4, -0.5], [0, 0, 1], s, 1, 3)
                    for s in range(4000)])
    assert len(np.unique(est)) > 10
    assert abs(est.mean() - T) < 4 * est.std() / math.sqrt(est.size)


def test_single_scattering_slab_closed_form(orc):
    """One scattering event, sun behind the camera (backscatter, mu = -1):
    E[L] = albedo p(-1) E_sun (1 - exp(-2 sigma L)) / 2."""
    dims = (16, 16, 64)
    c, scale, albedo, g, esun = 0.5, 1.5, 0.8, 0.4, 2.0
    vol = const_volume(dims, c)
    _, mx = orc.macrocell_minmax(vol, 8)
    med = orc.make_medium(orc.MODE_PT, density_scale=scale, albedo=albedo, g=g, max_bounces=1,
                          macrocell=8, sun_dir=(0, 0, -1), sun_rad=(esun, esun, esun))
    cam = ortho_z(orc, dims, 32, 32)
    img = orc.render_image(vol, mx, cam, med, 64, 2)
    tau = scale * c                 # optical depth of the slab
    p = orc.lib().or_hg_eval(-1.0, g)
    want = albedo * p * esun * (1 - math.exp(-2 * tau)) / 2
    vals = img[..., 0].ravel()
    assert abs(vals.mean() - want) < 4 * vals.std() / math.sqrt(vals.size) + 1e-12


def test_white_furnace(orc):
    """albedo 1, no light but a constant environment L: every path escapes
    with weight 1, so every pixel equals L."""
    dims = (24, 20, 28)
    rng = np.random.default_rng(8)
    vol = rng.random(dims[::-1]).astype(np.float32)
    _, mx = orc.macrocell_minmax(vol, 8)
    med = orc.make_medium(orc.MODE_PT, density_scale=20.0, albedo=1.0, g=0.3, max_bounces=100000,
                          macrocell=8, env_rad=(0.7, 0.7, 0.7))
    M = max(dims)
    cam = orc.make_camera(orc.CAM_PINHOLE, 16, 16, (1.5, 0.9, -1.2),
                          (0.5 * dims[0] / M, 0.5 * dims[1] / M, 0.5 * dims[2] / M), (0, 1, 0), 30)
    img = orc.render_image(vol, mx, cam, med, 8, 3)
    assert np.allclose(img[..., :3], 0.7, atol=1e-12)


def test_image_independent_of_macrocell_size(orc, vg):
    """Tracking is unbiased for any valid majorant: 8^3 macrocells and one
    global cell give the same image mean within Monte Carlo error."""
    dims = (32, 32, 32)
    vol = vg.generate_host(vg.make_params("blobs", dims, 1))
    med8 = orc.make_medium(orc.MODE_PT, density_scale=30.0, albedo=0.9, g=0.6, max_bounces=8,
                           macrocell=8, sun_dir=(0.6, 0.6, 0.52915), sun_rad=(3, 3, 3),
                           env_rad=(0.25, 0.25, 0.25))
    medG = orc.make_medium(orc.MODE_PT, density_scale=30.0, albedo=0.9, g=0.6, max_bounces=8,
                           macrocell=64, sun_dir=(0.6, 0.6, 0.52915), sun_rad=(3, 3, 3),
                           env_rad=(0.25, 0.25, 0.25))
    _, m8 = orc.macrocell_minmax(vol, 8)
    _, mG = orc.macrocell_minmax(vol, 64)
    cam = orc.make_camera(orc.CAM_PINHOLE, 24, 24, (1.4, 1.1, 1.6), (0.5, 0.5, 0.5), (0, 1, 0), 35)
    a = orc.render_image(vol, m8, cam, med8, 64, 10, threads=4)[..., 0]
    b = orc.render_image(vol, mG, cam, medG, 64, 11, threads=4)[..., 0]
    diff = (a - b).ravel()
    assert abs(diff.mean()) < 4 * diff.std() / math.sqrt(diff.size)


# ------------------------------------------------------------------ ISO surface marcher
def _iso_image(orc, vol, cam_args, iso=0.5, step=0.5):
    cam = orc.make_camera(*cam_args)
    med = orc.make_medium(orc.MODE_ISO, step=step, iso=iso)
    return orc.render_image(np.ascontiguousarray(vol, np.float32), None, cam, med, 1, 0)


def _ortho(dims, w, h):
    from volgen import scenes
    return scenes.ortho_plus_z(dims, w, h)


@pytest.mark.parametrize("grad", [(0.0, 0.0, 1.0), (1.0, 2.0, 3.0), (-2.0, 0.5, 1.5)])
def test_iso_linear_field_normals_are_exact(orc, grad):
    """Trilinear reconstruction of a linear field is the field, so the
    iso-surface is a plane and every hit pixel shows -grad/|grad|."""
    dims = (24, 20, 28)
    z, y, x = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
    g = np.asarray(grad)
    vol = (g[0] * x + g[1] * y + g[2] * z) / 40.0 + 0.5 - (g[0] * 11.5 + g[1] * 9.5 + g[2] * 13.5) / 40.0
    img = _iso_image(orc, vol, _ortho(dims, 20, 18))
    n = -g / np.linalg.norm(g)
    hit = img[..., 3] == 1.0
    assert hit.mean() > 0.5
    want = 0.5 * (n + 1.0)
    # away from the clamped border the central differences see the plane exactly
    core = img[4:-4, 4:-4]
    core_hit = core[..., 3] == 1.0
    assert core_hit.any()
    assert np.allclose(core[core_hit][:, :3], want, atol=1e-9)
    assert np.all(img[~hit] == 0.0)


def test_iso_constant_fields_miss(orc):
    dims = (16, 16, 16)
    for value in (0.2, 0.9):    # all outside, and all inside: no change along any ray
        img = _iso_image(orc, np.full(dims[::-1], value, np.float32), _ortho(dims, 12, 12))
        assert np.all(img == 0.0)


def test_iso_takes_the_first_of_two_slabs(orc):
    """Two slabs along z; +z rays meet the near face of the first one, whose
    normal is -z; a ray reversed along -z meets the far slab's back face."""
    dims = (16, 16, 48)
    vol = np.zeros(dims[::-1], np.float32)
    vol[10:18] = 1.0
    vol[30:40] = 1.0
    img = _iso_image(orc, vol, _ortho(dims, 10, 10))
    assert np.all(img[..., 3] == 1.0)
    assert np.allclose(img[..., :3], [0.5, 0.5, 0.0], atol=1e-12)
    from volgen import scenes
    ex, ey, ez = scenes.world_extent(dims)
    back = (0, 10, 10, (0.5 * ex, 0.5 * ey, ez + 1.0), (0.5 * ex, 0.5 * ey, ez), (0, 1, 0), ey)
    img = _iso_image(orc, vol, back)
    assert np.allclose(img[..., :3], [0.5, 0.5, 1.0], atol=1e-12)


def test_iso_sphere_matches_the_analytic_surface(orc):
    """f = clamp(1 - |p - c| / R): the 0.5 surface is the sphere of radius R/2;
    the shaded normal of each hit pixel follows the analytic intersection."""
    dims = (48, 48, 48)
    c, R = np.array([23.5, 23.5, 23.5]), 36.0
    z, y, x = np.meshgrid(np.arange(48), np.arange(48), np.arange(48), indexing="ij")
    r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    vol = np.clip(1.0 - r / R, 0.0, 1.0).astype(np.float32)
    cam_args = _ortho(dims, 24, 24)
    img = _iso_image(orc, vol, cam_args, step=0.25)
    cam = orc.make_camera(*cam_args)
    rs = R / 2
    checked = 0
    for py in range(24):
        for px in range(24):
            o, d = orc.camera_ray(cam, dims, px, py)
            oc = o - c
            b = np.dot(oc, d)
            disc = b * b - (np.dot(oc, oc) - rs * rs)
            if disc < 4.0:          # grazing rays: leave them out
                assert img[py, px, 3] == 0.0 or disc > 0
                continue
            t = -b - np.sqrt(disc)
            n = (o + t * d - c) / rs
            assert img[py, px, 3] == 1.0
            assert np.max(np.abs(img[py, px, :3] - 0.5 * (n + 1))) < 0.03
            checked += 1
    assert checked > 100
