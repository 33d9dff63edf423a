"""vdbc_compare, the FP64 image and volume error reduction, against numpy in
FP64 (the same sums in another order: agreement to 1e-12 relative)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2504_04564_gb300 as v
    return dict(torch=torch, v=v)


@pytest.mark.parametrize("shape,stride,channels", [((97, 131, 4), 4, 3), ((1,), 1, 1), ((33, 17, 29), 1, 1),
                                                   ((1024, 1024, 4), 4, 3), ((5, 4), 4, 4)])
def test_compare_matches_numpy_fp64(env, shape, stride, channels):
    torch, v = env["torch"], env["v"]
    rng = np.random.default_rng(sum(shape))
    a = rng.random(shape, dtype=np.float32)
    b = (a + rng.normal(0, 0.01, shape)).astype(np.float32)
    st = v.vdbc_compare(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), stride=stride, channels=channels)
    d = (a.astype(np.float64) - b.astype(np.float64)).reshape(-1, stride)[:, :channels]
    mse = float(np.mean(d * d))
    assert st.n == d.size
    assert math.isclose(st.mse, mse, rel_tol=1e-12)
    assert math.isclose(st.mean_abs, float(np.mean(np.abs(d))), rel_tol=1e-12)
    assert st.max_abs == float(np.max(np.abs(d)))
    assert math.isclose(st.psnr, 10 * math.log10(1 / mse), rel_tol=1e-12)


def test_compare_equal_arrays_and_repeatability(env):
    torch, v = env["torch"], env["v"]
    a = torch.rand((300, 200, 4), device="cuda")
    st = v.vdbc_compare(a, a.clone(), stride=4, channels=3)
    assert st.mse == 0.0 and st.max_abs == 0.0 and math.isinf(st.psnr)
    b = a + 1e-3 * torch.rand_like(a)
    r = [v.vdbc_compare(a, b, stride=4, channels=3).as_dict() for _ in range(3)]
    assert r[0] == r[1] == r[2]            # a fixed summation order
