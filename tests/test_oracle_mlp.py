"""Pins of the oracle's learned leaf decoder (a project extension the paper
prints no values for).  The backward pass is pinned to the forward
by central finite differences, the forward to networks built by hand whose
output is known in closed form, and Adam to the closed form of its first
step."""
import numpy as np
import pytest


def layout(orc):
    n_in, h = orc.MLP_IN, orc.MLP_HID
    sizes = [h * n_in, h, h * h, h, h, 1]
    offs = np.cumsum([0] + sizes)
    return dict(W1=(offs[0], (h, n_in)), b1=(offs[1], (h,)), W2=(offs[2], (h, h)), b2=(offs[3], (h,)),
                w3=(offs[4], (h,)), b3=(offs[5], (1,)))


def view(p, lay, name):
    o, shape = lay[name]
    return p[o:o + int(np.prod(shape))].reshape(shape)


def test_parameter_count(orc):
    assert orc.mlp_num_params() == 32 * 19 + 32 + 32 * 32 + 32 + 32 + 1 == 1729


def test_forward_closed_form_networks(orc):
    lay = layout(orc)
    p = np.zeros(orc.mlp_num_params())
    # zero weights: the output is the last bias
    view(p, lay, "b3")[0] = 0.37
    x = np.random.default_rng(0).random((10, 19))
    assert np.allclose(orc.mlp_forward(p, x), 0.37, atol=0, rtol=0)
    # y = relu(2 u - 1) + 3 z_4 (z_4 >= 0) through explicit weights
    W1, b1, W2, w3 = view(p, lay, "W1"), view(p, lay, "b1"), view(p, lay, "W2"), view(p, lay, "w3")
    W1[0, 0], b1[0] = 2.0, -1.0
    W1[1, 3 + 4] = 3.0
    W2[0, 0] = 1.0
    W2[1, 1] = 1.0
    w3[0], w3[1] = 1.0, 1.0
    view(p, lay, "b3")[0] = 0.0
    want = np.maximum(2 * x[:, 0] - 1, 0) + 3 * x[:, 7]
    assert np.allclose(orc.mlp_forward(p, x), want, atol=1e-15)


@pytest.mark.parametrize("seed", [1, 2])
def test_gradients_match_finite_differences(orc, seed):
    rng = np.random.default_rng(seed)
    n = 7
    p = rng.normal(0, 0.4, orc.mlp_num_params())
    x = rng.random((n, 19))
    t = rng.random(n)
    loss, gp, gx = orc.mlp_loss_grad(p, x, t)
    h = 1e-6
    idx = rng.choice(p.size, 60, replace=False)
    for i in idx:
        q = p.copy(); q[i] += h
        lp = orc.mlp_loss_grad(q, x, t)[0]
        q[i] -= 2 * h
        lm = orc.mlp_loss_grad(q, x, t)[0]
        assert abs((lp - lm) / (2 * h) - gp[i]) <= 1e-6 * max(1.0, abs(gp[i]))
    for s in range(n):
        for k in (0, 2, 3, 10, 18):
            y = x.copy(); y[s, k] += h
            lp = orc.mlp_loss_grad(p, y, t)[0]
            y[s, k] -= 2 * h
            lm = orc.mlp_loss_grad(p, y, t)[0]
            assert abs((lp - lm) / (2 * h) - gx[s, k]) <= 1e-6 * max(1.0, abs(gx[s, k]))
    # and the loss is the mean squared error of the forward pass
    assert abs(loss - np.mean((orc.mlp_forward(p, x) - t) ** 2)) < 1e-14


def test_adam_first_step_closed_form(orc):
    rng = np.random.default_rng(3)
    p0 = rng.normal(size=50)
    g = rng.normal(size=50)
    p = p0.copy(); m = np.zeros(50); v = np.zeros(50)
    orc.adam_step(p, g, m, v, 1, lr=0.01)
    # step 1: m_hat = g, v_hat = g^2, so the update is lr * g / (|g| + eps)
    assert np.allclose(p, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_training_fits_a_smooth_leaf(orc):
    """Gradient descent with the oracle's own pieces fits one smooth leaf:
    the loss falls by more than 10x (a sanity check of the whole loop)."""
    rng = np.random.default_rng(4)
    p = rng.normal(0, 0.3, orc.mlp_num_params())
    z = rng.normal(0, 0.1, 16)
    x = orc.leaf_inputs(z)
    t = 0.5 + 0.3 * np.sin(3 * x[:, 0]) * x[:, 1]
    m = np.zeros_like(p); v = np.zeros_like(p)
    l0 = orc.mlp_loss_grad(p, x, t)[0]
    for step in range(1, 301):
        loss, gp, gx = orc.mlp_loss_grad(p, x, t)
        orc.adam_step(p, gp, m, v, step, lr=3e-3)
    assert loss < l0 / 10


def test_bf16_rounding_matches_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.normal(size=20000), rng.normal(size=2000) * 1e-30, [0.0, 1.0, 1.0 / 7, 3.0 / 7]])
    xs = xs.astype(np.float32)
    want = torch.from_numpy(xs).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([orc.round_bf16(float(x)) for x in xs], dtype=np.float32)
    assert np.array_equal(got, want)


def test_bf16_forward_close_to_full_precision(orc):
    """The bf16 forward differs from the FP64 one by the rounding of its
    operands only: a few bf16 ulps on a well-scaled network."""
    rng = np.random.default_rng(6)
    p = rng.normal(0, 0.3, orc.mlp_num_params())
    x = rng.random((200, 19))
    a = orc.mlp_forward(p, x)
    b = orc.mlp_forward_bf16(p, x)
    assert np.abs(a - b).max() < 0.05 * max(1.0, np.abs(a).max())
    # exact on inputs and weights that bf16 represents, when no activation needs rounding
    q = np.zeros_like(p)
    q[0] = 1.0              # W1[0,0]
    q[32 * 19 + 32] = 1.0   # W2[0,0]
    q[32 * 19 + 32 + 32 * 32 + 32] = 2.0  # w3[0]
    xx = np.zeros((3, 19)); xx[:, 0] = [0.5, 0.25, 0.75]
    assert np.array_equal(orc.mlp_forward_bf16(q, xx), 2.0 * xx[:, 0])


def _u_network(orc):
    """y = u (the voxel's x position in its leaf / 7) through explicit weights."""
    lay = layout(orc)
    p = np.zeros(orc.mlp_num_params())
    view(p, lay, "W1")[0, 0] = 1.0
    view(p, lay, "W2")[0, 0] = 1.0
    view(p, lay, "w3")[0] = 1.0
    return p, lay


def test_learned_leaf_closed_forms(orc):
    rng = np.random.default_rng(3)
    src = rng.random(512).astype(np.float32) * 5 - 1
    _, scale, offset = orc.quantize_leaf(src, orc.FP16)
    assert scale == np.float32(src.max()) - np.float32(src.min()) and offset == src.min()
    lay = layout(orc)
    z = rng.random(16).astype(np.float32)
    # constant networks: y = b3, clamped to [0, 1]
    for b3, want in ((0.25, 0.25), (2.0, 1.0), (-1.0, 0.0)):
        p = np.zeros(orc.mlp_num_params())
        view(p, lay, "b3")[0] = b3
        out = orc.learned_leaf(p, z, src)
        assert np.all(out == np.float32(np.float64(offset) + np.float64(scale) * want))
    # y = u: bf16 rounding of i/7 shows in the output, the latent does not
    p, _ = _u_network(orc)
    out = orc.learned_leaf(p, z, src)
    i = np.arange(512) & 7
    u_bf16 = np.array([orc.round_bf16(np.float32(k / 7.0)) for k in range(8)])
    want = (np.float64(offset) + np.float64(scale) * u_bf16[i]).astype(np.float32)
    assert np.array_equal(out, want)
    assert not np.array_equal(u_bf16, np.arange(8) / 7.0)     # the rounding is visible


def test_learned_leaf_latent_is_rounded_once_to_bf16(orc):
    # y = z_0 through the network: the latent is stored in bf16, one rounding of
    # its FP32 value.  z_0 = 1/2 + 2^-9 + 2^-13 rounds up to 1/2 + 2^-8 in bf16,
    # while a detour through FP16 would land on the bf16 midpoint and tie to 1/2.
    lay = layout(orc)
    p = np.zeros(orc.mlp_num_params())
    view(p, lay, "W1")[0, 3] = 1.0
    view(p, lay, "W2")[0, 0] = 1.0
    view(p, lay, "w3")[0] = 1.0
    src = np.linspace(0, 1, 512, dtype=np.float32)
    z = np.zeros(16, dtype=np.float32)
    z[0] = np.float32(0.5 + 2.0 ** -9 + 2.0 ** -13)
    out = orc.learned_leaf(p, z, src)
    assert orc.round_bf16(z[0]) == 0.5 + 2.0 ** -8
    assert orc.round_bf16(orc.round_fp16(z[0])) == 0.5
    assert np.all(out == np.float32(0.5 + 2.0 ** -8))       # offset 0, scale 1


def test_tree_leaf_matches_decode(orc, vg):
    vol = vg.generate_host(vg.make_params("blobs", (40, 36, 44), 0))
    enc = orc.encode(vol, 4.0)
    tree = orc.Tree(vol, enc["active"], enc["background_bits"])
    dec = orc.decode_dense(vol, enc["active"], enc["background_bits"])
    B = np.uint32(enc["background_bits"]).view(np.float32)
    nz, ny, nx = vol.shape
    n = 0
    for lk in range((nz + 7) // 8):
        for lj in range((ny + 7) // 8):
            for li in range((nx + 7) // 8):
                leaf = tree.leaf(li, lj, lk)
                blk = dec[lk * 8:lk * 8 + 8, lj * 8:lj * 8 + 8, li * 8:li * 8 + 8]
                if leaf is None:
                    # a tile: the decoded region is constant
                    assert np.all(blk.view(np.uint32) == blk.reshape(-1)[0].view(np.uint32))
                    continue
                n += 1
                cube = leaf.reshape(8, 8, 8)
                ez, ey, ex = blk.shape
                assert np.array_equal(cube[:ez, :ey, :ex].view(np.uint32), blk.view(np.uint32))
                outside = np.ones((8, 8, 8), bool)
                outside[:ez, :ey, :ex] = False
                assert np.all(cube[outside] == B)
    assert n == tree.counts()["leaves"] and n > 0


def test_learned_decode_all_raw_is_the_fp16_grid(orc, vg):
    vol = vg.generate_host(vg.make_params("blobs", (40, 36, 44), 1))
    enc = orc.encode(vol, 2.0)
    nl = 5 * 5 * 6
    force = np.full(nl, 2, np.uint8)
    out, kinds = orc.learned_decode(vol, enc["active"], enc["background_bits"], np.zeros(orc.mlp_num_params()),
                                    np.zeros((nl, 16), np.float32), force)
    want = orc.decode_dense(vol, enc["active"], enc["background_bits"], orc.FP16)
    assert np.array_equal(out.view(np.uint32), want.view(np.uint32))
    assert int((kinds == 2).sum()) == orc.Tree(vol, enc["active"], enc["background_bits"]).counts()["leaves"]


def _representable_case(orc, rng):
    """A network, inputs and targets on which every value the bf16 gradient
    rounds is already a bf16 number: sparse weights of +-1/2, +-1, inputs in
    {0, 1/2, 1}, and targets that put the errors at +-1/4 or +-1/2."""
    lay = layout(orc)
    p = np.zeros(orc.mlp_num_params())
    W1, b1, W2, b2 = view(p, lay, "W1"), view(p, lay, "b1"), view(p, lay, "W2"), view(p, lay, "b2")
    w3, b3 = view(p, lay, "w3"), view(p, lay, "b3")
    vals = np.array([-1.0, -0.5, 0.5, 1.0])
    for i in range(32):
        for k in rng.choice(19, 3, replace=False):
            W1[i, k] = rng.choice(vals)
        for k in rng.choice(32, 3, replace=False):
            W2[i, k] = rng.choice(vals)
    b1[:] = rng.choice([-0.25, 0.0, 0.25, 0.5], 32)
    b2[:] = rng.choice([-0.25, 0.0, 0.25], 32)
    w3[:] = rng.choice(vals, 32)
    b3[0] = 0.25
    x = rng.choice([0.0, 0.5, 1.0], (4, 19))
    y = orc.mlp_forward(p, x)
    t = y - rng.choice([-0.5, -0.25, 0.25, 0.5], 4)
    return p, x, t


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bf16_gradient_is_exact_on_representable_networks(orc, seed):
    p, x, t = _representable_case(orc, np.random.default_rng(seed))
    l0, g0, gx0 = orc.mlp_loss_grad(p, x, t)
    l1, g1, gx1 = orc.mlp_loss_grad_bf16(p, x, t)
    assert l1 == l0
    assert np.array_equal(g1, g0) and np.array_equal(gx1, gx0)
    assert np.abs(g0).max() > 0


def test_bf16_gradient_loss_is_the_bf16_forward_mse(orc):
    rng = np.random.default_rng(5)
    p = rng.normal(0, 0.4, orc.mlp_num_params())
    x = rng.random((40, 19))
    t = rng.random(40)
    loss, _, _ = orc.mlp_loss_grad_bf16(p, x, t)
    y = orc.mlp_forward_bf16(p, x)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-6)


def test_bf16_gradient_close_to_exact_gradient(orc):
    """bf16 operands move the gradient by about 2^-8 relative: a transposed
    weight, a wrong mask or a dropped term would move it by order one."""
    rng = np.random.default_rng(6)
    p = rng.normal(0, 0.4, orc.mlp_num_params())
    x = rng.random((200, 19))
    t = rng.random(200)
    _, g0, gx0 = orc.mlp_loss_grad(p, x, t)
    _, g1, gx1 = orc.mlp_loss_grad_bf16(p, x, t)
    assert np.abs(g1 - g0).max() <= 2e-2 * np.abs(g0).max()
    # a single sample's input gradient can move further where bf16 operands flip
    # the sign of a pre-activation near zero (its ReLU mask); most samples do not
    far = np.abs(gx1 - gx0).max(axis=1) > 2e-2 * np.abs(gx0).max()
    assert far.mean() <= 0.1
    assert np.abs(g1 - g0).max() > 0          # the rounding is there
