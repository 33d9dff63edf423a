"""GPU encoder parity against the CPU oracle (bit-exact: the background value,
the activated brick set, every decoded voxel, the macrocell ranges, the leaf
count), plus the input generator's device build against its host build."""
import os

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
    return dict(torch=torch, v=v, orc=oracle, vg=volgen, dev=torch.device("cuda:0"))


def encode_both(env, host, ratio, metric=2, payload=0, macrocell=8, offset=0):
    """offset > 0 places the volume `offset` floats into a device buffer, so
    that its base is off a 16-byte boundary (the encoder's scalar loads)."""
    torch, v, orc = env["torch"], env["v"], env["orc"]
    if offset:
        flat = torch.zeros(host.size + offset, dtype=torch.float32, device=env["dev"])
        vol = flat[offset:].view(host.shape)
        vol.copy_(torch.from_numpy(host))
    else:
        vol = torch.from_numpy(host).to(env["dev"])
    grid = v.vdbc_encode(vol, ratio, metric=metric, payload=payload, macrocell=macrocell)
    e = orc.encode(host, ratio, metric=metric, payload=payload)
    return vol, grid, e


def check_encoding(env, host, ratio, metric=2, payload=0, macrocell=8, offset=0):
    torch, v, orc = env["torch"], env["v"], env["orc"]
    vol, grid, e = encode_both(env, host, ratio, metric, payload, macrocell, offset)
    info = grid.info
    assert info.background_bits == e["background_bits"]
    assert info.n_bricks == e["lo"].size
    assert info.budget == e["budget"] and info.n_active == e["n_active"]
    assert info.n_nonempty == int((e["empty"] == 0).sum())
    assert np.array_equal(v.vdbc_grid_active_bricks(grid), e["active"])
    D = orc.decode_dense(host, e["active"], e["background_bits"], payload)
    dec = torch.empty_like(vol)
    v.vdbc_grid_decode(grid, dec)
    got = dec.cpu().numpy()
    assert np.array_equal(got.view(np.uint32), D.view(np.uint32))
    # host-output decode path as well
    got2 = np.empty_like(host)
    v.vdbc_grid_decode(grid, got2)
    assert np.array_equal(got2.view(np.uint32), D.view(np.uint32))
    # leaf count after prune equals the oracle tree's
    t = orc.Tree(host, e["active"], e["background_bits"], payload)
    c = t.counts()
    assert info.n_leaves == c["leaves"]
    assert info.n_lower == c["lower"] and info.n_upper == c["upper"]
    # macrocell min/max of the decoded grid
    mn, mx = v.vdbc_grid_macrocells(grid)
    omn, omx = orc.macrocell_minmax(D, macrocell)
    assert np.array_equal(mn, omn) and np.array_equal(mx, omx)
    return grid, e, D


@pytest.mark.parametrize("dims", [(64, 64, 64), (40, 33, 17), (97, 70, 33), (1, 1, 1), (3, 70, 9), (130, 8, 129)])
@pytest.mark.parametrize("ratio", [1.0, 4.0, 10.0])
def test_encoder_bit_exact_fp32(env, dims, ratio):
    host = env["vg"].generate_host(env["vg"].make_params("blobs", dims, 1))
    check_encoding(env, host, ratio)


@pytest.mark.parametrize("dims", [(8192, 4, 5), (4, 8192, 5), (4, 5, 8192)])
@pytest.mark.parametrize("payload", [0, 1, 2])
def test_encoder_bit_exact_largest_edge(env, dims, payload):
    """Volumes 8192 voxels long (the largest edge the encoder takes) along each
    axis: two entries of the root table along that axis, crossed by the tree
    descent of every decoded voxel and by the macrocells."""
    host = env["vg"].generate_host(env["vg"].make_params("turbulence", dims, 3))
    grid, e, D = check_encoding(env, host, 2.0, payload=payload, macrocell=16)
    assert grid.info.n_upper == 2


@pytest.mark.parametrize("dims", [(64, 64, 64), (97, 70, 33), (1, 1, 1), (130, 8, 129)])
@pytest.mark.parametrize("offset", [1, 3])
def test_encoder_bit_exact_unaligned_base(env, dims, offset):
    """The brick passes' scalar loads on a volume that starts off a 16-byte
    boundary (offset floats into a buffer), also for widths whose aligned
    volumes take the float4 loads: the same bits as the oracle."""
    host = env["vg"].generate_host(env["vg"].make_params("turbulence", dims, 4))
    check_encoding(env, host, 4.0, offset=offset)


@pytest.mark.parametrize("metric", [1, 2, 3])
@pytest.mark.parametrize("payload", [1, 2])
def test_encoder_bit_exact_metrics_and_quantized_payloads(env, metric, payload):
    host = env["vg"].generate_host(env["vg"].make_params("turbulence", (96, 80, 72), 3))
    check_encoding(env, host, 6.0, metric=metric, payload=payload)


@pytest.mark.parametrize("macrocell,payload", [(4, 0), (8, 0), (13, 0), (33, 0), (48, 0), (56, 0), (64, 0), (64, 1),
                                               (48, 2), (96, 0), (128, 0), (128, 2)])
def test_macrocell_sizes(env, macrocell, payload):
    """Cells above 4096 dilated voxels take the block-per-cell kernels: the
    input-based one for FP32 leaves (which takes a whole active brick's range
    from pass 1 and reads only partial bricks; 33, 48, 56 and 64 cover whole
    bricks, 64 the clipped ones at the volume's edges too; 96 and 128, the
    largest, overlap up to five and six bricks along an axis), the tree-based
    one for FP16/FP8."""
    host = env["vg"].generate_host(env["vg"].make_params("turbulence", (150, 97, 131), 2))
    check_encoding(env, host, 2.0, payload=payload, macrocell=macrocell)


def test_macrocell_128_six_bricks_per_axis(env):
    """A 128-voxel cell dilated by one voxel overlaps six 32^3 bricks along each
    axis once the volume reaches past 256 voxels: the 216 parts the input-based
    kernel lists at most.  At 1:2 most bricks are active, cut by the cell
    faces; the ranges equal the oracle's on the decoded grid."""
    v, orc = env["v"], env["orc"]
    host = env["vg"].generate_host(env["vg"].make_params("turbulence", (262, 259, 261), 5))
    vol, grid, e = encode_both(env, host, 2.0, 2, 0, 128, 0)
    D = orc.decode_dense(host, e["active"], e["background_bits"], 0)
    mn, mx = v.vdbc_grid_macrocells(grid)
    omn, omx = orc.macrocell_minmax(D, 128)
    assert mn.size == 3 * 3 * 3
    assert np.array_equal(mn, omn) and np.array_equal(mx, omx)
    grid.close()


def tie_volume(dims, levels=37):
    """One non-background voxel per 32^3 brick (two, one of them negative, in
    every third brick; every fifth brick empty), drawn from `levels` values:
    thousands of bricks share a few (lo, hi) ranges, so the scores tie at the
    selection's budget edge and the lower brick index must decide."""
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
    x2, y2 = np.minimum(i * 32 + 17, nx - 1), np.minimum(j * 32 + 9, ny - 1)
    v[z[neg], y2[neg], x2[neg]] = -lvl[neg] / 2
    return v


@pytest.mark.parametrize("metric", [1, 2, 3])
@pytest.mark.parametrize("ratio", [10.0, 3.0])
def test_selection_above_4096_bricks_with_ties(env, metric, ratio):
    """More than 4096 bricks (4290 here) take the selection's branch that
    keeps the keys in global memory; with scores tied across hundreds of
    bricks, the activated set must be the oracle's exactly (Algorithm 1:
    largest f first, ties to the lower brick index)."""
    host = tie_volume((4160, 1056, 8))
    grid, e, D = check_encoding(env, host, ratio, metric=metric, macrocell=16)
    assert e["lo"].size == 4290
    f = e["f"][e["active"] == 1]
    rest = e["f"][(e["active"] == 0) & (e["empty"] == 0)]
    assert rest.size and f.size and f.min() == rest.max()     # the budget edge falls inside a tie


def test_encoder_bit_exact_cloud_above_4096_bricks(env):
    """The cloud generator at 1040 x 544 x 256 (4488 bricks), made on the
    device (the generator's host and device builds are bit-identical): B, the
    activated bricks, every decoded voxel and the macrocells at 1:10."""
    vg = env["vg"]
    vol = vg.generate_torch(vg.make_params("cloud", (1040, 544, 256), 0))
    host = vol.cpu().numpy()
    del vol
    grid, e, D = check_encoding(env, host, 10.0, macrocell=64)
    assert e["lo"].size == 4488 and grid.info.n_active == e["n_active"] > 0


def test_degenerate_volumes(env):
    vg = env["vg"]
    # all zero: every brick is empty, only the (background) corners remain -> no leaves
    z = np.zeros((37, 20, 45), dtype=np.float32)
    grid, e, D = check_encoding(env, z, 1.0)
    assert grid.info.n_leaves == 0 and grid.info.n_active == 0
    # constant non-zero bricks prune to tiles; ties in f everywhere
    c = np.zeros((64, 64, 64), dtype=np.float32)
    c[:32] = 0.5
    grid, e, D = check_encoding(env, c, 1.0)
    assert grid.info.n_leaves == 0 and grid.info.n_tiles > 1
    # corner values differing from the background with nothing activated
    k = np.zeros((40, 33, 17), dtype=np.float32)
    k[0, 0, 0], k[-1, -1, -1], k[20, 20, 10] = 0.3, 0.7, 0.9
    grid, e, D = check_encoding(env, k, 1000.0)
    assert grid.info.n_active == 0 and grid.info.n_leaves == 2
    # both corners inside one leaf
    s = np.arange(27, dtype=np.float32).reshape(3, 3, 3) / 27
    check_encoding(env, s, 100.0)
    # dense noise, lossless (the paper's worst case)
    n = vg.generate_host(vg.make_params("noise", (64, 64, 64), 5))
    grid, e, D = check_encoding(env, n, 1.0)
    assert grid.info.n_active == 8 and grid.info.n_leaves == 512


def candidate_lattice(dims):
    """The 16 x 8 x 8 voxel lattice spanning the volume on which the encoder
    draws its candidate for a majority background pattern."""
    nx, ny, nz = dims
    m = np.zeros((nz, ny, nx), dtype=bool)
    for i in range(1024):
        m[(i >> 7) * (nz - 1) // 7, ((i >> 4) & 7) * (ny - 1) // 7, (i & 15) * (nx - 1) // 15] = True
    return m


@pytest.mark.parametrize("case", ["wrong_candidate", "exact_half", "no_majority"])
@pytest.mark.parametrize("offset", [0, 1])
def test_background_without_a_sampled_majority(env, case, offset):
    """B where the encoder's majority shortcut cannot decide it: the sampled
    candidate is not the majority pattern (zeros hold 70 % of the voxels, the
    sampled lattice holds 1.0); the candidate holds exactly half of the
    voxels (no strict majority: level 1 ties between two bins and takes the
    smaller); no pattern repeats at all.  Aligned rows and rows off a 16-byte
    boundary take the two load modes of both passes."""
    rng = np.random.default_rng(5)
    dims = (96, 80, 72)
    n = dims[0] * dims[1] * dims[2]
    lat = candidate_lattice(dims)
    if case == "wrong_candidate":
        host = np.where(rng.random(n).reshape(lat.shape) < 0.7, 0.0, rng.random(n).reshape(lat.shape))
        host[lat] = 1.0
    elif case == "exact_half":
        order = np.concatenate([np.flatnonzero(lat), rng.permutation(np.flatnonzero(~lat))])
        host = np.full(n, 0.5)
        host[order[: n // 2]] = 0.0
        host = host.reshape(lat.shape)
    else:
        host = rng.random(n).reshape(lat.shape) + 0.5
    host = np.ascontiguousarray(host.astype(np.float32))
    grid, e, _ = check_encoding(env, host, 10.0, offset=offset)
    if case != "no_majority":
        assert e["background_bits"] == 0


def test_encoder_rejects_non_finite(env):
    torch, v = env["torch"], env["v"]
    a = np.zeros((16, 16, 16), dtype=np.float32)
    a[3, 4, 5] = np.inf
    with pytest.raises(v.VdbcError) as ex:
        v.vdbc_encode(torch.from_numpy(a).to(env["dev"]), 2.0)
    assert ex.value.status == v.ERR_INVALID_ARG


def test_host_input_equals_device_input(env):
    v = env["v"]
    host = env["vg"].generate_host(env["vg"].make_params("blobs", (70, 64, 50), 9))
    g1 = v.vdbc_encode(host, 4.0)
    vol, g2, _ = encode_both(env, host, 4.0)
    a = np.empty_like(host)
    b = np.empty_like(host)
    v.vdbc_grid_decode(g1, a)
    v.vdbc_grid_decode(g2, b)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_save_load_roundtrip_and_corruption(env, tmp_path):
    v = env["v"]
    host = env["vg"].generate_host(env["vg"].make_params("turbulence", (64, 48, 80), 4))
    g1 = v.vdbc_encode(host, 3.0, payload=1)
    path = str(tmp_path / "g.vdbc")
    v.vdbc_grid_save(g1, path)
    g2 = v.vdbc_grid_load(path)
    assert g2.info.as_dict() == g1.info.as_dict()
    a = np.empty_like(host)
    b = np.empty_like(host)
    v.vdbc_grid_decode(g1, a)
    v.vdbc_grid_decode(g2, b)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert np.array_equal(v.vdbc_grid_macrocells(g1)[1], v.vdbc_grid_macrocells(g2)[1])
    raw = bytearray(open(path, "rb").read())
    raw[len(raw) // 2] ^= 0x40
    bad = str(tmp_path / "bad.vdbc")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(v.VdbcError) as ex:
        v.vdbc_grid_load(bad)
    assert ex.value.status == v.ERR_FORMAT


def test_injected_allocation_failure(env, monkeypatch):
    """Host-side fault injection: VDBC_FAULT=oom refuses every device allocation
    before it is made; the call reports OOM and the context stays usable."""
    v = env["v"]
    host = env["vg"].generate_host(env["vg"].make_params("blobs", (32, 32, 32), 0))
    monkeypatch.setenv("VDBC_FAULT", "oom")
    with pytest.raises(v.VdbcError) as ex:
        v.vdbc_encode(host, 1.0)
    assert ex.value.status == v.ERR_OOM
    monkeypatch.delenv("VDBC_FAULT")
    g = v.vdbc_encode(host, 1.0)        # one 32^3 brick: the budget at 1:1 is that brick
    assert g.info.n_active == 1


def test_device_generator_matches_host(env):
    torch, vg = env["torch"], env["vg"]
    for kind, dims in (("blobs", (64, 64, 64)), ("turbulence", (72, 64, 80)), ("cloud", (66, 45, 81)),
                       ("noise", (33, 17, 9))):
        p = vg.make_params(kind, dims, 2)
        h = vg.generate_host(p)
        d = vg.generate_torch(p).cpu().numpy()
        assert np.array_equal(h.view(np.uint32), d.view(np.uint32)), kind


def test_full_size_turbulence_encoding(env):
    """The 512^3 medium at 1:10, as the benchmark encodes it: B, the 409
    activated bricks and sampled decoded voxels against the oracle."""
    torch, v, orc, vg = env["torch"], env["v"], env["orc"], env["vg"]
    p = vg.make_params("turbulence", (512, 512, 512), 0)
    host = vg.generate_host(p)
    vol = vg.generate_torch(p)
    grid = v.vdbc_encode(vol, 10.0)
    e = orc.encode(host, 10.0)
    assert grid.info.n_active == 409 == e["n_active"]
    assert grid.info.background_bits == e["background_bits"]
    assert np.array_equal(v.vdbc_grid_active_bricks(grid), e["active"])
    dec = torch.empty_like(vol)
    v.vdbc_grid_decode(grid, dec)
    D = orc.decode_dense(host, e["active"], e["background_bits"])
    got = dec.cpu().numpy()
    assert np.array_equal(got.view(np.uint32), D.view(np.uint32))
