"""Pins of the oracle's encoder (Section 3.1, Algorithm 1, Eq. f1-f3; Section 3.2.1).

Each test checks the oracle against something other than itself: brute force
on tiny inputs, numpy reductions, hand-computed values, the paper's printed
invariants (lossless at 1:1, the linear rate map, the worst-case overhead,
the metric ranking) and the tree descent against the definition of D.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def bits(x):
    return int(np.float32(x).view(np.uint32))


def pad_bricks(v, fill):
    nz, ny, nx = v.shape
    P = [((n + 31) // 32) * 32 for n in (nz, ny, nx)]
    out = np.full(P, fill, dtype=v.dtype)
    out[:nz, :ny, :nx] = v
    return out


def numpy_brick_minmax(v):
    """Per-brick min/max by reshaping a padded copy (pads with NaN, ignored)."""
    nz, ny, nx = v.shape
    p = pad_bricks(v.astype(np.float64), np.nan)
    bz, by, bx = p.shape[0] // 32, p.shape[1] // 32, p.shape[2] // 32
    r = p.reshape(bz, 32, by, 32, bx, 32)
    return np.nanmin(r, axis=(1, 3, 5)).ravel(), np.nanmax(r, axis=(1, 3, 5)).ravel()


# ------------------------------------------------------------------ background
def test_background_is_mode_for_plain_arrays(orc):
    rng = np.random.default_rng(1)
    for trial in range(20):
        vals = rng.choice(np.float32([0.0, 0.25, -1.5, 3.0, 1e-20]), size=1000,
                          p=[0.4, 0.2, 0.2, 0.1, 0.1])
        u, c = np.unique(vals.view(np.uint32), return_counts=True)
        # the mode's upper 16 bits are also the most frequent upper bin here
        assert orc.background_bits(vals) == int(u[np.argmax(c)])


def test_background_two_level_definition(orc):
    # upper bin 0x3f80 (1.0..) holds 3 distinct values once each (3 in total);
    # upper bin 0x4000 (2.0..) holds one value twice: the winning upper bin is
    # 0x3f80 and inside it the tie goes to the smallest pattern.
    a = np.float32(1.0).view(np.uint32)
    vals = np.array([a, a + 1, a + 2, bits(2.0), bits(2.0)], dtype=np.uint32).view(np.float32)
    assert orc.background_bits(vals) == int(a)
    # ties between upper bins go to the smaller pattern as well
    vals = np.float32([5.0, 5.0, -5.0, -5.0])
    assert orc.background_bits(vals) == bits(5.0)
    # -0 and +0 are different bit patterns
    vals = np.float32([-0.0, -0.0, 0.0])
    assert orc.background_bits(vals) == bits(-0.0)


# ------------------------------------------------------------------ ranges
@pytest.mark.parametrize("dims", [(40, 33, 17), (64, 64, 64), (1, 1, 1), (70, 5, 33)])
def test_brick_ranges_match_numpy(orc, dims):
    rng = np.random.default_rng(sum(dims))
    nx, ny, nz = dims
    v = rng.normal(size=(nz, ny, nx)).astype(np.float32)
    lo, hi = orc.brick_ranges(v)
    mn, mx = numpy_brick_minmax(v)
    assert np.array_equal(lo.view(np.float32).astype(np.float64), mn)
    assert np.array_equal(hi.view(np.float32).astype(np.float64), mx)
    nb = orc.brick_grid(dims)
    assert list(nb) == [math.ceil(d / 32) for d in dims]


def test_brick_range_orders_signed_zero(orc):
    v = np.zeros((32, 32, 32), dtype=np.float32)
    v[3, 4, 5] = -0.0
    lo, hi = orc.brick_ranges(v)
    assert int(lo[0]) == bits(-0.0) and int(hi[0]) == bits(0.0)


# ------------------------------------------------------------------ scores
def test_scores_hand_values(orc):
    lo = np.float32([0.0, 0.5, -1.0, 2.0, 0.25]).view(np.uint32)
    hi = np.float32([0.0, 1.5, 3.0, 2.0, 0.25]).view(np.uint32)
    B = bits(0.25)
    f1, e = orc.brick_scores(lo, hi, B, orc.F1)
    f2, _ = orc.brick_scores(lo, hi, B, orc.F2)
    f3, _ = orc.brick_scores(lo, hi, B, orc.F3)
    # closest / farthest / median point of [lo,hi] to B, written out by hand
    assert f1.tolist() == [0.25, 0.25, 1.25, 1.75, 0.0]
    assert f2.tolist() == [0.25, 1.25, 2.75, 1.75, 0.0]
    assert f3.tolist() == [0.25, 0.75, 0.75, 1.75, 0.0]
    assert e.tolist() == [0, 0, 0, 0, 1]


# ------------------------------------------------------------------ budget
@pytest.mark.parametrize("dims,ratio,expect", [
    ((64, 64, 64), 4, 2),            # 8 bricks at 1:4
    ((512, 512, 512), 10, 409),      # 4096 bricks at 1:10
    ((994, 676, 1225), 10, 2745),    # 27,456 bricks
    ((1987, 1351, 2449), 10, 20859),  # 208,593 bricks
    ((1987, 1351, 2449), 20, 10429),
    ((40, 33, 17), 1, 4),
])
def test_budget_linear_map(orc, dims, ratio, expect):
    nb = int(np.prod(orc.brick_grid(dims)))
    assert orc.brick_budget(nb, ratio, orc.FP32) == expect
    # the linear map of Algorithm 1: floor(numBricks * quality), quality = 1/ratio
    assert expect == math.floor(nb / ratio)


def test_budget_quantized_buys_more_bricks(orc):
    nb = 4096
    n32 = orc.brick_budget(nb, 10, orc.FP32)
    n16 = orc.brick_budget(nb, 10, orc.FP16)
    n8 = orc.brick_budget(nb, 10, orc.FP8)
    assert n16 == math.floor(nb * 131072 / (10 * (65536 + 512)))
    assert n8 == math.floor(nb * 131072 / (10 * (32768 + 512)))
    assert n32 < n16 < n8
    # payload bytes never exceed the (padded) dense bytes / ratio
    for n, bb in ((n32, 131072), (n16, 66048), (n8, 33280)):
        assert n * bb <= nb * 131072 / 10


# ------------------------------------------------------------------ selection
def brute_select(f, empty, n):
    order = sorted([i for i in range(f.size) if not empty[i]], key=lambda i: (-f[i], i))
    a = np.zeros(f.size, dtype=np.uint8)
    a[order[:n]] = 1
    return a


def test_select_matches_brute_force(orc):
    rng = np.random.default_rng(7)
    for trial in range(50):
        n = int(rng.integers(1, 60))
        f = rng.choice([0.0, 0.5, 1.0, 2.0, rng.random()], size=n)  # many ties
        empty = (rng.random(n) < 0.3).astype(np.uint8)
        k = int(rng.integers(0, n + 3))
        a, take = orc.select(f, empty, k)
        assert np.array_equal(a, brute_select(f, empty, k))
        assert take == min(k, int((empty == 0).sum()))


def test_select_keeps_largest_distance_first(orc, vg):
    """Reading of the sort direction: bricks farthest from B are kept first."""
    v = vg.generate_host(vg.make_params("blobs", (64, 64, 64), 0))
    e = orc.encode(v, 4.0)
    kept = e["f"][e["active"] == 1]
    dropped = e["f"][(e["active"] == 0) & (e["empty"] == 0)]
    assert kept.size == 2
    assert dropped.size == 0 or kept.min() >= dropped.max()


# ------------------------------------------------------------------ decode / tree
def definitional_D(v, active, B):
    """D(x) = V(x) in an activated brick or at the two extreme corners, B elsewhere."""
    nz, ny, nx = v.shape
    nb = [math.ceil(n / 32) for n in (nx, ny, nz)]
    a = active.reshape(nb[2], nb[1], nb[0]).astype(bool)
    mask = np.repeat(np.repeat(np.repeat(a, 32, 0), 32, 1), 32, 2)[:nz, :ny, :nx].copy()
    mask[0, 0, 0] = True
    mask[-1, -1, -1] = True
    return np.where(mask, v, np.float32(np.uint32(B).view(np.float32)))


@pytest.mark.parametrize("dims", [(40, 33, 17), (64, 64, 64), (9, 70, 3)])
@pytest.mark.parametrize("ratio", [1, 2.5, 6])
def test_decode_dense_matches_definition_fp32(orc, vg, dims, ratio):
    v = vg.generate_host(vg.make_params("blobs", dims, 3))
    e = orc.encode(v, ratio)
    D = orc.decode_dense(v, e["active"], e["background_bits"])
    ref = definitional_D(v, e["active"], e["background_bits"])
    assert np.array_equal(D.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("payload", [0, 1, 2])
@pytest.mark.parametrize("dims", [(40, 33, 17), (9, 70, 3), (8192, 3, 2), (2, 8192, 3), (3, 2, 8192)])
def test_tree_descent_equals_decode_every_voxel(orc, vg, dims, payload):
    """Every voxel through the tree equals the definitional decode; the
    8192-long volumes (the largest edge the encoder takes) span two entries of
    the root table along one axis each."""
    v = vg.generate_host(vg.make_params("blobs", dims, 5))
    e = orc.encode(v, 2.0, payload=payload)
    D = orc.decode_dense(v, e["active"], e["background_bits"], payload)
    t = orc.Tree(v, e["active"], e["background_bits"], payload)
    nx, ny, nz = dims
    got = np.array([[[t.value(i, j, k) for i in range(nx)] for j in range(ny)] for k in range(nz)],
                   dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), D.view(np.uint32))
    if max(dims) > 4096:
        assert t.counts()["root"] == 2


def test_prune_keeps_values_and_collapses_constant_leaves(orc):
    v = np.zeros((64, 64, 64), dtype=np.float32)
    v[:32, :32, :32] = 0.5          # one brick, constant: all its leaves prune to tiles
    v[40:44, 40:44, 40:44] = 0.75   # a non-constant brick
    e = orc.encode(v, 1.0)
    assert e["n_active"] == 2
    t = orc.Tree(v, e["active"], e["background_bits"])
    c = t.counts()
    # the constant brick collapses to 64 leaf-level tiles of value 0.5; the
    # other brick keeps the 8 leaves touched by the 4^3 cube (4 voxels at an
    # offset of 40 = 5*8 fall in one leaf) and 56 leaves that equal B are pruned
    assert c["lower_tiles"] == 64 and c["leaves"] == 1
    assert t.value(3, 3, 3) == 0.5 and t.value(41, 41, 41) == 0.75 and t.value(50, 50, 50) == 0.0
    D = orc.decode_dense(v, e["active"], e["background_bits"])
    assert np.array_equal(D, v)


def test_corners_always_present(orc):
    v = np.zeros((40, 33, 17), dtype=np.float32)
    v[0, 0, 0] = 0.3
    v[-1, -1, -1] = 0.7
    v[5, 5, 5] = 0.9
    e = orc.encode(v, 1000.0)          # budget 0: nothing activated
    assert e["n_active"] == 0
    D = orc.decode_dense(v, e["active"], e["background_bits"])
    assert D[0, 0, 0] == np.float32(0.3) and D[-1, -1, -1] == np.float32(0.7)
    assert D[5, 5, 5] == 0.0
    t = orc.Tree(v, e["active"], e["background_bits"])
    assert t.counts()["leaves"] == 2
    assert t.value(0, 0, 0) == np.float32(0.3) and t.value(16, 32, 39) == np.float32(0.7)


# ------------------------------------------------------------------ invariants of the paper
@pytest.mark.parametrize("kind,dims", [("blobs", (64, 64, 64)), ("turbulence", (96, 80, 72)),
                                       ("noise", (48, 40, 33)), ("blobs", (40, 33, 17))])
def test_lossless_at_one_to_one(orc, vg, kind, dims):
    """Section 5.1: at 1:1 only empty bricks are dropped, so D == V (MSE 0, PSNR inf)."""
    v = vg.generate_host(vg.make_params(kind, dims, 11))
    for metric in (orc.F1, orc.F2, orc.F3):
        e = orc.encode(v, 1.0, metric=metric)
        D = orc.decode_dense(v, e["active"], e["background_bits"])
        assert np.array_equal(D.view(np.uint32), v.view(np.uint32))
        assert orc.mse(D, v) == 0.0 and orc.psnr(D, v) == float("inf")


def test_quality_monotone_in_rate(orc, vg):
    """Table tab:stats: the error never grows as the rate moves toward 1:1."""
    v = vg.generate_host(vg.make_params("turbulence", (128, 128, 128), 2))
    prev = None
    for ratio in (64, 20, 10, 6, 5, 4, 2, 1):
        e = orc.encode(v, ratio)
        D = orc.decode_dense(v, e["active"], e["background_bits"])
        m = orc.mse(D, v)
        if prev is not None:
            assert m <= prev
        prev = m
    assert prev == 0.0


def test_size_saturates_at_nonempty_count(orc, vg):
    """Table tab:rates (Aneurism 16 MB at 1:4..1:1): once every non-empty brick
    is active, lowering the rate adds nothing."""
    v = vg.generate_host(vg.make_params("blobs", (128, 128, 128), 4))
    nonempty = None
    sizes = []
    for ratio in (4, 2, 1.5, 1):
        e = orc.encode(v, ratio)
        nonempty = int((e["empty"] == 0).sum())
        sizes.append(e["n_active"])
        assert e["n_active"] == min(e["budget"], nonempty)
    assert sizes[-1] == nonempty


def test_tree_payload_within_budget(orc, vg):
    v = vg.generate_host(vg.make_params("turbulence", (96, 96, 96), 9))
    for ratio in (10, 4, 2):
        e = orc.encode(v, ratio)
        t = orc.Tree(v, e["active"], e["background_bits"])
        c = t.counts()
        assert c["leaves"] <= 64 * e["n_active"] + 2
        assert e["n_active"] * 131072 <= (e["lo"].size * 131072) / ratio


def test_worst_case_overhead_dense_noise(orc, vg):
    """Table tab:worstcase: losslessly encoding dense noise costs at most 10 %
    more than the dense array once the volume is large (the paper's 256^3
    row is 67 MB vs 71 MB).  Bytes here: 2 KiB per 8^3 FP32 leaf, 16 KiB per
    16^3 lower node, 128 KiB per 32^3 upper node."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_tab_worstcase.txt"))
            if l.strip() and not l.startswith("#")]
    paper = {int(r[0]): float(r[2]) / float(r[1]) for r in rows}
    assert all(paper[e] <= 1.10 for e in (256, 512, 1024, 2048))
    n = 256
    v = vg.generate_host(vg.make_params("noise", (n, n, n), 1))
    e = orc.encode(v, 1.0)
    assert e["n_active"] == (n // 32) ** 3
    t = orc.Tree(v, e["active"], e["background_bits"])
    c = t.counts()
    total = c["leaves"] * 2048 + c["lower"] * 16384 + c["upper"] * 131072 + c["root"] * 8
    dense = n ** 3 * 4
    assert dense <= total <= 1.10 * dense


def test_metric_ranking_farthest_and_median_beat_closest(orc, vg):
    """Figure fig:distance: f2 (farthest) and f3 (median) give a PSNR at least
    that of f1 (closest) at the same rate."""
    v = vg.generate_host(vg.make_params("turbulence", (128, 128, 128), 0))
    for ratio in (8, 5):
        p = {}
        for metric in (orc.F1, orc.F2, orc.F3):
            e = orc.encode(v, ratio, metric=metric)
            D = orc.decode_dense(v, e["active"], e["background_bits"])
            p[metric] = orc.psnr(D, v)
        assert p[orc.F2] >= p[orc.F1] and p[orc.F3] >= p[orc.F1]


def test_psnr_convention_against_paper_table(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_tab_stats.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 23
    for name, rate, m, p, ok in rows:
        m, p = float(m), float(p)
        e = math.floor(math.log10(m))
        mlo, mhi = m - 0.5 * 10.0 ** e, m + 0.5 * 10.0 ** e
        dec = len(rows[0][3].split(".")[1]) if "." in str(p) and p < 100 else 0
        half = 0.5 * 10.0 ** (-dec)
        # the MSE values whose PSNR rounds to the printed one
        lo_m, hi_m = 10.0 ** (-(p + half) / 10.0), 10.0 ** (-(p - half) / 10.0)
        consistent = max(mlo, lo_m) <= min(mhi, hi_m)
        assert consistent == (ok == "1"), (name, rate)
        if ok == "1":
            # and the oracle's psnr() of an MSE inside the overlap rounds to the printed value
            mm = max(mlo, lo_m) * 0.5 + min(mhi, hi_m) * 0.5
            a = np.zeros(1)
            b = np.full(1, math.sqrt(mm))
            assert abs(orc.psnr(a, b) - p) <= half + 1e-9
