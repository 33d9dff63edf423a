"""Pins of the oracle's multi-bounce path: the scattered direction, and
closed forms of whole random walks that depend on it.

Section 4: a path scatters until it leaves the medium (here: until a fixed
number of events, with no Russian roulette).  The new direction is drawn
around the incoming one: polar cosine mu from the Henyey-Greenstein phase
function, azimuth phi uniform.

* or_scatter_dir on its own: |d'| = 1, d.d' = mu exactly, d'(phi1).d'(phi2)
  = mu^2 + (1 - mu^2) cos(phi1 - phi2) (a circle of radius sin(theta) about
  d, traced once per 2 pi), and the mean of d' over a uniform azimuth is mu d.
* Whole paths on a line (the rod model of transport theory): an orthographic
  camera looks along +z through a slab of constant density (optical depth
  tau0) with a constant environment and no light.  Each path returns
  a^n for its n scattering events (a the albedo).
    - g -> +1 (every event keeps the direction): n is Poisson(tau0), so the
      pixel mean is exp(-tau0 (1 - a)).
    - g -> -1 (every event reverses it): the expected weight u(t) of a walker
      moving + and v(t) of one moving - at optical depth t obey
      u' = u - a v, v' = a u - v with u(tau0) = 1, v(0) = 1, so
      u(0) = (k + a sinh(k tau0)) / (sinh(k tau0) + k cosh(k tau0)),
      k = sqrt(1 - a^2).
* Mirror symmetry: with a uniform azimuth the walk has no preferred side, so
  the two halves of a mirror-symmetric scene render alike.
* Adam (Kingma and Ba 2015) past its first step: with a constant gradient c
  every bias-corrected step is lr c / (|c| + eps); with gradients c, -c, c
  steps 2 and 3 move by lr (1 - b1)/(1 + b1) and
  lr (1 - b1 + b1^2)/(1 + b1 + b1^2) (times the sign), because the second
  moments then equal c^2 (1 - b2^t) exactly.

Each group also runs once on a copy of the oracle with a planted mistake
(tests/plant.py) and must fail there: mu along b1 instead of d, the azimuth
not scaled to a full turn, beta1 in place of beta2 in the bias correction.
"""
import math

import numpy as np
import pytest

from plant import planted_library


def const_volume(dims, c):
    nx, ny, nz = dims
    return np.full((nz, ny, nx), c, dtype=np.float32)


def ortho_z(orc, dims, w, h):
    nx, ny, nz = dims
    M = max(dims)
    cx, cy = 0.5 * nx / M, 0.5 * ny / M
    return orc.make_camera(orc.CAM_ORTHO, w, h, (cx, cy, -1.0), (cx, cy, 0.0), (0, 1, 0), ny / M)


# ------------------------------------------------------------------ the direction itself
def _random_dirs(rng, n):
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    # the basis' two branches and its singular neighbourhood
    extra = np.array([[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0], [0, 1e-9, -1], [1e-7, 0, 1]], dtype=np.float64)
    extra /= np.linalg.norm(extra, axis=1, keepdims=True)
    return np.concatenate([d, extra])


def scatter_dir_violations(orc):
    """Largest violation of each geometric property over random cases."""
    rng = np.random.default_rng(11)
    worst = dict(norm=0.0, polar=0.0, circle=0.0, mean=0.0)
    for d in _random_dirs(rng, 60):
        for mu in (-1.0, -0.73, -0.2, 0.0, 0.31, 0.9, 1.0):
            phis = rng.uniform(0, 2 * math.pi, size=3)
            outs = [orc.scatter_dir(d, mu, p) for p in phis]
            for o in outs:
                worst["norm"] = max(worst["norm"], abs(np.linalg.norm(o) - 1.0))
                worst["polar"] = max(worst["polar"], abs(float(o @ d) - mu))
            c = float(outs[0] @ outs[1])
            want = mu * mu + (1 - mu * mu) * math.cos(phis[0] - phis[1])
            worst["circle"] = max(worst["circle"], abs(c - want))
            grid = [orc.scatter_dir(d, mu, 2 * math.pi * k / 64) for k in range(64)]
            worst["mean"] = max(worst["mean"], float(np.abs(np.mean(grid, axis=0) - mu * d).max()))
    return worst


def test_scatter_dir_geometry(orc):
    w = scatter_dir_violations(orc)
    assert w["norm"] < 1e-12
    assert w["polar"] < 1e-12
    assert w["circle"] < 1e-12
    assert w["mean"] < 1e-12


# ------------------------------------------------------------------ whole walks on a line
ROD_DIMS = (16, 16, 64)


def rod_image(orc, g, albedo, tau0, spp=64, seed=5):
    vol = const_volume(ROD_DIMS, 1.0)
    _, mx = orc.macrocell_minmax(vol, 8)
    # optical depth along z: density_scale * 1.0 * nz / M = density_scale
    # the light (zero radiance) stands across the line: the phase function at
    # cosine +-1 would divide by (1 - |g|)^2, which rounds to 0 at |g| -> 1
    med = orc.make_medium(orc.MODE_PT, density_scale=tau0, albedo=albedo, g=g, max_bounces=400, macrocell=8,
                          sun_dir=(1, 0, 0), env_rad=(1, 1, 1))
    cam = ortho_z(orc, ROD_DIMS, 16, 16)
    return orc.render_image(vol, mx, cam, med, spp, seed)[..., 0].ravel()


def rod_forward_z(orc, albedo=0.7, tau0=2.0):
    vals = rod_image(orc, 1.0 - 1e-9, albedo, tau0)
    want = math.exp(-tau0 * (1.0 - albedo))
    return (vals.mean() - want) / (vals.std() / math.sqrt(vals.size) + 1e-12)


def rod_backward_z(orc, albedo=0.7, tau0=2.0):
    vals = rod_image(orc, -(1.0 - 1e-9), albedo, tau0)
    k = math.sqrt(1.0 - albedo * albedo)
    s, c = math.sinh(k * tau0), math.cosh(k * tau0)
    want = (k + albedo * s) / (s + k * c)
    return (vals.mean() - want) / (vals.std() / math.sqrt(vals.size) + 1e-12)


def test_rod_forward_scattering_closed_form(orc):
    assert abs(rod_forward_z(orc)) < 4.5


def test_rod_back_scattering_closed_form(orc):
    assert abs(rod_backward_z(orc)) < 4.5


def test_rod_closed_forms_are_distinct():
    """The two closed forms differ by far more than the tests' noise (about
    0.004 at 16x16 pixels x 64 spp), so each test can tell them apart."""
    a, tau0 = 0.7, 2.0
    k = math.sqrt(1 - a * a)
    back = (k + a * math.sinh(k * tau0)) / (math.sinh(k * tau0) + k * math.cosh(k * tau0))
    fwd = math.exp(-tau0 * (1 - a))
    assert abs(back - fwd) > 0.03
    # and both reduce to Beer-Lambert without scattering weight (a -> 0)
    assert abs((1 + 0) / (math.sinh(tau0) + math.cosh(tau0)) - math.exp(-tau0)) < 1e-15


# ------------------------------------------------------------------ mirror symmetry (uniform azimuth)
def halves_z(orc):
    """Left minus right half of a scene symmetric under x -> -x, in units of
    its standard error."""
    dims = (32, 16, 16)
    vol = const_volume(dims, 1.0)
    _, mx = orc.macrocell_minmax(vol, 8)
    med = orc.make_medium(orc.MODE_PT, density_scale=6.0, albedo=0.85, g=0.5, max_bounces=200, macrocell=8,
                          env_rad=(1, 1, 1))
    cam = ortho_z(orc, dims, 32, 16)
    img = orc.render_image(vol, mx, cam, med, 32, 7)[..., 0]
    left, right = img[:, :16].ravel(), img[:, 16:].ravel()
    se = math.sqrt(left.var() / left.size + right.var() / right.size)
    return (left.mean() - right.mean()) / se


def test_uniform_azimuth_mirror_symmetry(orc):
    assert abs(halves_z(orc)) < 4.5


# ------------------------------------------------------------------ Adam past step 1
def adam_errors(orc):
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-8
    errs = []
    # constant gradient: every step moves by lr c / (|c| + eps)
    c = np.array([0.37, -2.5, 1e-3, 4.0])
    p = np.zeros(4); m = np.zeros(4); v = np.zeros(4)
    for t in range(1, 6):
        before = p.copy()
        orc.adam_step(p, c, m, v, t, lr=lr, beta1=b1, beta2=b2, eps=eps)
        errs.append(np.abs((before - p) - lr * c / (np.abs(c) + eps)).max())
    # gradients c, -c, c: closed-form step sizes at t = 2 and 3 (hand-derived,
    # second moments c^2 (1 - b2^t) exactly); eps is set to 0 here
    c = np.array([0.5, -1.5, 3.0])
    p = np.zeros(3); m = np.zeros(3); v = np.zeros(3)
    orc.adam_step(p, c, m, v, 1, lr=lr, beta1=b1, beta2=b2, eps=0.0)
    before = p.copy()
    orc.adam_step(p, -c, m, v, 2, lr=lr, beta1=b1, beta2=b2, eps=0.0)
    errs.append(np.abs((p - before) - lr * (1 - b1) / (1 + b1) * np.sign(c)).max())
    before = p.copy()
    orc.adam_step(p, c, m, v, 3, lr=lr, beta1=b1, beta2=b2, eps=0.0)
    errs.append(np.abs((before - p) - lr * (1 - b1 + b1 * b1) / (1 + b1 + b1 * b1) * np.sign(c)).max())
    return max(errs)


def test_adam_steps_two_and_three_closed_form(orc):
    assert adam_errors(orc) < 1e-15


# ------------------------------------------------------------------ the pins catch planted mistakes
def test_pins_catch_mu_along_b1(orc, tmp_path):
    lib = planted_library(tmp_path, "render.c",
                          "st * sin(phi) * b2[a] + mu * dir[a];", "st * sin(phi) * b2[a] + mu * b1[a];")
    with orc.library(lib):
        w = scatter_dir_violations(orc)
        assert w["polar"] > 1e-3 and w["mean"] > 1e-3
        assert not abs(rod_forward_z(orc)) < 4.5     # (a NaN fails the pin too)


def test_pins_catch_a_partial_azimuth(orc, tmp_path):
    lib = planted_library(tmp_path, "render.c", "double phi = 2.0 * M_PI * xi[1];", "double phi = xi[1];")
    with orc.library(lib):
        assert not abs(halves_z(orc)) < 4.5


def test_pins_catch_beta1_in_the_second_moment_correction(orc, tmp_path):
    lib = planted_library(tmp_path, "mlp.c", "c2 = 1.0 - pow(beta2, (double)step)",
                          "c2 = 1.0 - pow(beta1, (double)step)")
    with orc.library(lib):
        assert adam_errors(orc) > 1e-4
