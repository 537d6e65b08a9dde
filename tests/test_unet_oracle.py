"""Pins of the U-Net oracle (oracle/unet.py) against brute force, library
routines and closed forms; CPU only."""
import itertools
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle.unet as U  # noqa: E402
import synth  # noqa: E402


def test_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(200000) * np.exp(rng.uniform(-20, 20, 200000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16(x.astype(np.float64)), ref)


def test_bf16_ties_to_even():
    # 1 + 2^-8 lies half way between 1 and 1 + 2^-7: even mantissa is 1
    assert U.bf16(np.array([1 + 2.0 ** -8]))[0] == 1.0
    # 1 + 3 * 2^-8 lies half way between 1 + 2^-7 and 1 + 2^-6: even is 1 + 2^-6
    assert U.bf16(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6
    # values with 8 significant bits are kept
    k = np.arange(-255, 256, dtype=np.float64)
    assert np.array_equal(U.bf16(k * 2.0 ** -5), k * 2.0 ** -5)
    assert U.bf16(np.array([0.0]))[0] == 0.0


def _conv3x3_loops(x, w, b, relu):
    B, H, W, Ci = x.shape
    Co = w.shape[0]
    out = np.zeros((B, H, W, Co))
    for n, y, xx, co in itertools.product(range(B), range(H), range(W), range(Co)):
        s = float(b[co])
        for dy, dx, ci in itertools.product(range(3), range(3), range(Ci)):
            yy, xs = y + dy - 1, xx + dx - 1
            if 0 <= yy < H and 0 <= xs < W:
                s += float(x[n, yy, xs, ci]) * float(w[co, ci, dy, dx])
        out[n, y, xx, co] = max(s, 0.0) if relu else s
    return out


@pytest.mark.parametrize("relu", [True, False])
def test_conv3x3_brute_force(relu):
    rng = np.random.default_rng(1)
    x = rng.integers(-8, 9, (2, 4, 5, 3)) / 8.0
    w = rng.integers(-8, 9, (2, 3, 3, 3)) / 16.0
    b = rng.integers(-4, 5, 2) / 8.0
    ref = _conv3x3_loops(x, w, b, relu)
    # small integers over powers of two: every sum is exact, so is bf16
    assert np.array_equal(U.conv3x3(x, w, b, relu), U.bf16(ref))


def test_conv3x3_matches_scipy_correlate():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 9, 7, 2))
    w = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    got = U.conv3x3(x, w, b, relu=False)
    for co in range(3):
        ref = b[co] + sum(signal.correlate2d(x[0, :, :, ci], w[co, ci], mode="same", boundary="fill")
                          for ci in range(2))
        np.testing.assert_allclose(got[0, :, :, co], U.bf16(ref), rtol=2 ** -7, atol=1e-12)


def test_conv3x3_delta_kernels():
    rng = np.random.default_rng(3)
    x = U.bf16(rng.uniform(0, 1, (1, 6, 5, 2)))
    w = np.zeros((2, 2, 3, 3))
    w[0, 0, 1, 1] = 1.0           # centre tap: identity of channel 0
    w[1, 1, 0, 2] = 1.0           # tap (dy, dx) = (-1, +1): shift of channel 1
    out = U.conv3x3(x, w, np.zeros(2), relu=True)
    assert np.array_equal(out[..., 0], x[..., 0])
    shifted = np.zeros_like(x[..., 1])
    shifted[:, 1:, :-1] = x[:, :-1, 1:, 1]
    assert np.array_equal(out[..., 1], shifted)


def test_maxpool_brute_force():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 6, 4, 3))
    got = U.maxpool2(x)
    for n, y, xx, c in itertools.product(range(2), range(3), range(2), range(3)):
        assert got[n, y, xx, c] == max(x[n, 2 * y + i, 2 * xx + j, c] for i in range(2) for j in range(2))


def test_upconv_brute_force():
    rng = np.random.default_rng(5)
    x = rng.integers(-8, 9, (1, 3, 2, 4)) / 8.0
    w = rng.integers(-8, 9, (4, 3, 2, 2)) / 8.0
    b = rng.integers(-4, 5, 3) / 4.0
    got = U.upconv2(x, w, b)
    for y, xx, co in itertools.product(range(6), range(4), range(3)):
        s = b[co] + sum(x[0, y // 2, xx // 2, ci] * w[ci, co, y % 2, xx % 2] for ci in range(4))
        assert got[0, y, xx, co] == U.bf16(np.array([s]))[0]


def test_head_argmax_first_on_ties():
    x = np.zeros((1, 1, 2, 2))
    w = np.zeros((3, 2, 1, 1))
    b = np.array([0.5, 0.5, 0.25])
    logits, lab = U.head(x, w, b)
    assert lab.tolist() == [[[0, 0]]] and logits.dtype == np.float32


def test_forward_zero_weights_gives_head_bias():
    """All-zero weights and biases except the head bias: every activation is 0,
    so every pixel's scores are the head bias and its label is their argmax."""
    wts = {k: (np.zeros_like(w), np.zeros_like(b)) for k, (w, b) in synth.unet_weights(4, 2, 0).items()}
    hw, hb = wts["head"]
    wts["head"] = (hw, np.array([0.0, 0.25, -1.0], np.float32))
    chips = synth.chips_from_scene(synth.scene(256, 256, 1)[0], 1)
    logits, lab = U.forward(chips, wts, depth=2)
    assert logits.shape == (1, 256, 256, 3)
    assert np.all(lab == 1)
    assert np.all(logits == np.array([0.0, 0.25, -1.0], np.float32))


def test_weights_exact_in_bf16():
    for name, (w, b) in synth.unet_weights(8, 4, 1).items():
        assert np.array_equal(U.bf16(w.astype(np.float64)), w), name
        assert np.array_equal(U.bf16(b.astype(np.float64)), b), name


def test_prep_filtered_closed_forms():
    """V' = V leaves the chip unchanged; V' = 0 gives black; V' = 2V doubles
    grey pixels; every c' <= V' and the largest channel becomes V'."""
    rng = np.random.default_rng(9)
    chips = rng.integers(0, 256, (1, 256, 256, 3)).astype(np.uint8)
    v = chips.max(axis=-1)
    assert np.array_equal(U.prep_filtered(chips, v), U.prep(chips))
    assert not U.prep_filtered(chips, np.zeros_like(v)).any()
    grey = np.repeat(rng.integers(0, 128, (1, 256, 256, 1)).astype(np.uint8), 3, axis=-1)
    got = U.prep_filtered(grey, (2 * grey[..., 0]).astype(np.uint8))
    assert np.array_equal(got, 2 * U.prep(grey))
    vp = rng.integers(0, 256, v.shape).astype(np.uint8)
    cf = np.round(U.prep_filtered(chips, vp) * 256).astype(np.int64)
    assert (cf <= vp[..., None]).all()
    assert np.array_equal(cf.max(axis=-1)[v > 0], vp[v > 0])
    # brute force on a few pixels, exact fractions
    from fractions import Fraction
    for (y, x) in [(0, 0), (17, 200), (255, 255), (128, 3)]:
        for c in range(3):
            V = int(v[0, y, x])
            want = 0 if V == 0 else int(Fraction(int(chips[0, y, x, c]) * int(vp[0, y, x]), V) + Fraction(1, 2))
            assert cf[0, y, x, c] == want
