"""Pins of the oracle's FP16 / FP8(E4M3) leaf codecs (a project extension:
the paper stores FP32 leaves, so the pins are the formats' own definitions).

The rounding is checked against the format definitions decoded bit field by
bit field (IEEE 754 binary16; OCP FP8 E4M3 with no infinities), exhaustively
over every code, and against numpy's float16 and torch's float8_e4m3fn casts.
"""
import numpy as np
import pytest


def decode_fields(code, ebits, mbits, bias, fn_nan=False):
    """Value of a minifloat code from its sign / exponent / fraction fields."""
    s = (code >> (ebits + mbits)) & 1
    e = (code >> mbits) & ((1 << ebits) - 1)
    m = code & ((1 << mbits) - 1)
    if fn_nan and e == (1 << ebits) - 1 and m == (1 << mbits) - 1:
        return float("nan")
    if not fn_nan and e == (1 << ebits) - 1:
        return float("nan") if m else (-1.0) ** s * float("inf")
    if e == 0:
        v = m * 2.0 ** (1 - bias - mbits)
    else:
        v = (1.0 + m * 2.0 ** (-mbits)) * 2.0 ** (e - bias)
    return -v if s else v


def finite_values(ebits, mbits, bias, fn_nan):
    vals = []
    for c in range(1 << (1 + ebits + mbits)):
        v = decode_fields(c, ebits, mbits, bias, fn_nan)
        if np.isfinite(v) and not (v == 0 and c != 0):
            vals.append(v)
    return np.array(sorted(set(vals)))


@pytest.mark.parametrize("fmt", ["fp16", "e4m3"])
def test_every_code_rounds_to_itself_and_midpoints_to_even(orc, fmt):
    if fmt == "fp16":
        vals = finite_values(5, 10, 15, False)
        rnd = orc.round_fp16
        mbits = 10
    else:
        vals = finite_values(4, 3, 7, True)
        rnd = orc.round_e4m3
        mbits = 3
    pos = vals[vals >= 0]
    for v in pos:
        assert rnd(float(np.float32(v))) == np.float32(v)
    # midpoints between neighbours go to the one with an even fraction field;
    # positive codes are consecutive integers in value order, so the index in
    # `pos` is the code itself and its parity is the fraction's last bit
    for idx in range(len(pos) - 1):
        a, b = pos[idx], pos[idx + 1]
        mid = 0.5 * (a + b)
        if np.float32(mid) != mid:
            continue               # not representable in FP32: no exact tie to test
        r = rnd(float(mid))
        even = a if idx % 2 == 0 else b
        assert r == np.float32(even), (fmt, a, b, r)


def test_fp16_matches_numpy(orc):
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.random(20000), rng.random(2000) * 1e-4, rng.random(2000) * 7e4,
                         -rng.random(2000), [0.0, 1.0, 65504.0, 65519.0, 65520.0, 6e-8, 3e-8]])
    for x in xs.astype(np.float32):
        want = np.float32(np.float16(x))
        got = orc.round_fp16(float(x))
        assert got == want or (np.isinf(got) and np.isinf(want)), x


def test_e4m3_matches_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.random(20000), rng.random(2000) * 1e-2, rng.random(2000) * 440.0,
                         -rng.random(2000), [0.0, 1.0, 448.0, 2.0 ** -9, 2.0 ** -10, 0.0625]])
    xs = xs.astype(np.float32)
    want = torch.from_numpy(xs).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    got = np.array([orc.round_e4m3(float(x)) for x in xs], dtype=np.float32)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("payload,half_step", [(1, 2.0 ** -11), (2, 2.0 ** -4)])
def test_leaf_quantization_error_bound(orc, payload, half_step):
    """decode = fmaf(scale, code, off) stays within half a code step of t in
    [0,1] (times scale), plus FP32 rounding."""
    rng = np.random.default_rng(payload)
    for trial in range(50):
        leaf = (rng.random(512) * rng.choice([1e-3, 1.0, 100.0]) + rng.normal()).astype(np.float32)
        q, s, o = orc.quantize_leaf(leaf, payload)
        assert o == leaf.min() and np.float32(s) == np.float32(leaf.max() - leaf.min())
        err = np.abs(q.astype(np.float64) - leaf.astype(np.float64))
        bound = s * half_step + 4 * np.finfo(np.float32).eps * np.abs(leaf).max()
        assert err.max() <= bound
        assert q[np.argmin(leaf)] == o          # code 0 decodes to the offset exactly


def test_constant_leaf_quantizes_to_itself(orc):
    leaf = np.full(512, 0.3, dtype=np.float32)
    for payload in (1, 2):
        q, s, o = orc.quantize_leaf(leaf, payload)
        assert s == 0.0 and np.array_equal(q, leaf)
