"""Pins of the CPU oracle against things other than itself.

Each test checks one function of the oracle against a textbook or library
definition, a closed form the paper fixes, a hand-labelled tile, or a
brute force on tiny inputs -- never against a retyped copy of its own
formula.  No GPU is needed.
"""
import colorsys
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grey(v):
    v = np.asarray(v, np.uint8)
    return np.repeat(v[:, :, None], 3, axis=2)


# --------------------------------------------------------------------------
# HSV conversion (Sec. III-B: HSV colour space, 8-bit convention implied by
# the class bounds H <= 185, S, V <= 255).
# --------------------------------------------------------------------------
def test_hsv_golden_cases():
    cases = json.load(open(os.path.join(GOLDEN, "hsv_cases.json")))["cases"]
    for c in cases:
        assert oracle.hsv(*c["rgb"]) == tuple(c["hsv"]), c


def test_hsv_matches_colorsys_within_rounding():
    """Python's colorsys is the library definition of HSV (hue in [0,1),
    S = (max-min)/max, V = max).  The oracle must be its value scaled to
    H/2-degrees and 0..255 and rounded to the nearest integer."""
    rng = np.random.default_rng(123)
    cols = rng.integers(0, 256, (20000, 3))
    extra = [(v, v, v) for v in range(256)] + [(255, 0, 0), (0, 255, 0), (0, 0, 255),
                                                (1, 0, 0), (0, 1, 0), (0, 0, 1), (255, 254, 255)]
    for r, g, b in list(map(tuple, cols)) + extra:
        h, s, v = oracle.hsv(r, g, b)
        hf, sf, vf = colorsys.rgb_to_hsv(r / 255.0, g / 255.0, b / 255.0)
        assert v == max(r, g, b)
        assert abs(v - vf * 255.0) < 1e-9
        assert 0 <= s <= 255 and abs(s - sf * 255.0) <= 0.5 + 1e-9, (r, g, b, s, sf * 255)
        assert 0 <= h <= 179
        target = hf * 180.0
        dist = min(abs(h - target), abs(h + 180 - target), abs(h - 180 - target))
        assert dist <= 0.5 + 1e-9, (r, g, b, h, target)


def test_hsv_rounding_is_half_up_on_exact_ties():
    """Exact ties found by rational arithmetic on the library definition:
    hue/2 = k + 1/2 or 255 d / V = k + 1/2 must round up."""
    found_h = found_s = 0
    for (r, g, b) in [(60, 1, 0), (2, 1, 1), (120, 2, 0), (6, 3, 3), (200, 80, 200), (10, 5, 5)]:
        mx, mn = max(r, g, b), min(r, g, b)
        d = mx - mn
        s_exact = Fraction(255 * d, mx) if mx else Fraction(0)
        h, s, _ = oracle.hsv(r, g, b)
        if s_exact.denominator == 2:
            found_s += 1
            assert s == int(s_exact + Fraction(1, 2))
        # colorsys on Fractions of the inputs gives the exact hue fraction
        # (only + - * / and max/min are used before the final modulo).
        rc, gc, bc = (Fraction(mx - x, d) if d else 0 for x in (r, g, b))
        if d:
            if r == mx:
                hh = bc - gc
            elif g == mx:
                hh = 2 + rc - bc
            else:
                hh = 4 + gc - rc
            half_deg = (hh * 30) % 180  # hue (sixths of a turn) -> degrees / 2
            if half_deg.denominator == 2:
                found_h += 1
                assert h == int(half_deg + Fraction(1, 2)) % 180
    assert found_h >= 1 and found_s >= 1


# --------------------------------------------------------------------------
# uint16 reflectance -> 8 bit (the paper is silent; reading: round half up
# of v * 255 / scale, clamped).
# --------------------------------------------------------------------------
def test_u16_to_u8_against_fractions():
    for scale in (10000, 4095, 1):
        for v in list(range(0, 70)) + list(range(9900, 10100)) + [65535, 32767, 5000, 19607]:
            exact = Fraction(v * 255, scale)
            want = min(255, int(exact + Fraction(1, 2)))
            assert oracle.u16_to_u8(v, scale) == want, (v, scale)


def test_u16_roundtrip_of_u8_values():
    for v in range(256):
        v16 = int(Fraction(v * 10000, 255) + Fraction(1, 2))
        assert oracle.u16_to_u8(v16, 10000) == v


# --------------------------------------------------------------------------
# Noise filter: 3x3 median with replicated border == scipy's median_filter.
# --------------------------------------------------------------------------
def test_median_matches_scipy_nearest():
    from scipy.ndimage import median_filter
    rng = np.random.default_rng(5)
    for h in range(1, 10):
        for w in range(1, 8):
            V = rng.integers(0, 256, (h, w)).astype(np.uint8)
            want = median_filter(V, size=3, mode="nearest")
            np.testing.assert_array_equal(oracle.median3x3(V), want)
    V = rng.integers(0, 256, (37, 29)).astype(np.uint8)
    np.testing.assert_array_equal(oracle.median3x3(V), median_filter(V, size=3, mode="nearest"))


def test_median_special_cases():
    V = np.full((6, 7), 42, np.uint8)
    np.testing.assert_array_equal(oracle.median3x3(V), V)
    V[3, 3] = 255
    np.testing.assert_array_equal(oracle.median3x3(V), np.full((6, 7), 42, np.uint8))
    V = np.zeros((1, 1), np.uint8) + 9
    assert oracle.median3x3(V)[0, 0] == 9


# --------------------------------------------------------------------------
# Otsu: brute force over every t with the textbook between-class variance
# sigma_B^2 = w0 w1 (mu0 - mu1)^2 (class probabilities and means), exact.
# --------------------------------------------------------------------------
def _otsu_textbook(hist, fallback):
    N = sum(hist)
    best, best_t = None, None
    for t in range(255):
        n0 = sum(hist[: t + 1])
        n1 = N - n0
        if n0 == 0 or n1 == 0:
            continue
        m0 = Fraction(sum(k * hist[k] for k in range(t + 1)), n0)
        m1 = Fraction(sum(k * hist[k] for k in range(t + 1, 256)), n1)
        var_b = Fraction(n0, N) * Fraction(n1, N) * (m0 - m1) ** 2
        if best is None or var_b > best:
            best, best_t = var_b, t
    return fallback if best_t is None else best_t


def _otsu_within_class(hist, fallback):
    """Equivalent definition: minimise the within-class variance."""
    N = sum(hist)
    best, best_t = None, None
    vals = np.repeat(np.arange(256), hist)
    for t in range(255):
        a, b = vals[vals <= t], vals[vals > t]
        if len(a) == 0 or len(b) == 0:
            continue
        wv = Fraction(len(a), N) * _var(a) + Fraction(len(b), N) * _var(b)
        if best is None or wv < best:
            best, best_t = wv, t
    return fallback if best_t is None else best_t


def _var(a):
    n = len(a)
    m = Fraction(int(a.sum()), n)
    return sum((Fraction(int(x)) - m) ** 2 for x in a) / n


def test_otsu_against_textbook_bruteforce():
    rng = np.random.default_rng(7)
    for trial in range(60):
        hist = [0] * 256
        k = rng.integers(1, 6)
        for _ in range(int(rng.integers(1, 40))):
            hist[int(rng.integers(0, 256)) if k > 3 else int(rng.integers(0, 32) * 8)] += 1
        lo = min(i for i, c in enumerate(hist) if c)
        got = oracle.otsu(hist, lo)
        assert got == _otsu_textbook(hist, lo), hist


def test_otsu_against_within_class_variance():
    rng = np.random.default_rng(8)
    for trial in range(15):
        hist = np.zeros(256, np.int64)
        for v in rng.integers(0, 256, int(rng.integers(2, 25))):
            hist[v] += 1
        lo = int(np.nonzero(hist)[0][0])
        assert oracle.otsu(hist, lo) == _otsu_within_class(list(hist), lo)


def test_otsu_special_cases():
    h = np.zeros(256, np.uint64)
    h[77] = 10
    assert oracle.otsu(h, 77) == 77          # constant: no split, fallback
    h[200] = 3
    assert oracle.otsu(h, 77) == 77          # two values a<b: every t in [a,b-1] ties -> a
    h = np.zeros(256, np.uint64)
    h[255] = 5
    assert oracle.otsu(h, 255) == 255
    h = np.zeros(256, np.uint64)
    assert oracle.otsu(h, 0) == 0            # empty chip
    # a full 512x512 chip worth of pixels must not overflow
    h = np.zeros(256, np.uint64)
    h[0] = 131072
    h[255] = 131072
    assert oracle.otsu(h, 0) == 0


# --------------------------------------------------------------------------
# Min-max normalisation: lo -> 0, hi -> 255, round half up, monotone.
# --------------------------------------------------------------------------
def test_stretch_against_fractions():
    for lo, hi in [(0, 255), (60, 180), (10, 11), (0, 1), (3, 250), (100, 164)]:
        prev = -1
        for v in range(lo, hi + 1):
            exact = Fraction((v - lo) * 255, hi - lo)
            got = oracle.stretch(v, lo, hi)
            assert got == int(exact + Fraction(1, 2))
            assert got >= prev
            prev = got
        assert oracle.stretch(lo, lo, hi) == 0 and oracle.stretch(hi, lo, hi) == 255
    for v in range(256):
        assert oracle.stretch(v, 0, 255) == v


# --------------------------------------------------------------------------
# Class thresholds (Sec. III-B): with the filter off and the default ranges
# the label is a closed form of V alone: water V<=30, thin 31..204, thick
# >=205; the three ranges do not intersect, so nothing is masked.  Checked
# on all 2^24 RGB colours.
# --------------------------------------------------------------------------
@pytest.mark.slow
def test_thresholds_exhaustive_colour_cube():
    r = np.arange(256, dtype=np.uint8)
    cube = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(4096, 4096, 3)
    labels, counts, chip_counts, _ = oracle.label(cube, {"filter": 0, "chip": 256})
    V = cube.max(axis=2)
    want = np.where(V <= 30, 2, np.where(V <= 204, 1, 0)).astype(np.uint8)
    np.testing.assert_array_equal(labels, want)
    assert counts[3] == 0
    assert int(counts.sum()) == 1 << 24
    np.testing.assert_array_equal(counts, np.bincount(want.ravel(), minlength=4))
    np.testing.assert_array_equal(chip_counts.sum(axis=(0, 1)), counts)


def test_threshold_boundary_pixels():
    px = [((0, 0, 30), 2), ((0, 0, 31), 1), ((204, 0, 0), 1), ((205, 205, 205), 0),
          ((0, 0, 0), 2), ((255, 255, 255), 0), ((0, 204, 0), 1), ((0, 205, 0), 0)]
    img = np.array([[c for c, _ in px]], np.uint8)
    labels, counts, _, _ = oracle.label(img, {"filter": 0, "chip": 8})
    assert list(labels[0]) == [l for _, l in px]


# --------------------------------------------------------------------------
# Hand-labelled tiles.
# --------------------------------------------------------------------------
def _golden_cases():
    return json.load(open(os.path.join(GOLDEN, "worked_4x4.json")))["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_worked_tiles(case):
    img = np.array(case["rgb"], np.uint8) if "rgb" in case else _grey(case["v"])
    labels, counts, chip_counts, stats = oracle.label(img, case["params"])
    np.testing.assert_array_equal(labels, np.array(case["labels"], np.uint8))
    assert list(counts) == case["counts"]
    if "chip_counts" in case:
        np.testing.assert_array_equal(chip_counts, np.array(case["chip_counts"]))
    if "stats" in case:
        for k, v in case["stats"].items():
            assert stats[0][k] == v, (k, stats[0])


# --------------------------------------------------------------------------
# Invariants of the method.
# --------------------------------------------------------------------------
def test_counts_sum_and_chip_sum():
    img, _ = synth.scene(300, 410, 3, n_floes=8)
    for chip in (4, 37, 128, 256):
        labels, counts, chip_counts, _ = oracle.label(img, {"chip": chip})
        assert int(counts.sum()) == 300 * 410
        np.testing.assert_array_equal(chip_counts.sum(axis=(0, 1)), counts)
        np.testing.assert_array_equal(np.bincount(labels.ravel(), minlength=4), counts)


def test_locality_pixels_outside_chip_do_not_matter():
    img, _ = synth.scene(200, 200, 4, n_floes=6)
    base, _, _, _ = oracle.label(img, {"chip": 64})
    img2 = img.copy()
    rng = np.random.default_rng(0)
    mask = np.ones((200, 200), bool)
    mask[64:128, 64:128] = False           # chip (1,1) untouched
    img2[mask] = rng.integers(0, 256, (mask.sum(), 3))
    other, _, _, _ = oracle.label(img2, {"chip": 64})
    np.testing.assert_array_equal(other[64:128, 64:128], base[64:128, 64:128])


def test_chip_aligned_crop_equals_region_of_full_result():
    img, _ = synth.scene(320, 330, 5, n_floes=9)
    full, _, cc, _ = oracle.label(img, {"chip": 64})
    crop = np.ascontiguousarray(img[64:256, 128:330])
    part, _, cc2, _ = oracle.label(crop, {"chip": 64})
    np.testing.assert_array_equal(part, full[64:256, 128:330])
    np.testing.assert_array_equal(cc2, cc[1:4, 2:6])


def test_u16_path_equals_u8_path_without_nodata():
    img, _ = synth.scene(150, 170, 6, n_floes=5)
    img16 = np.array([[[int(Fraction(int(v) * 10000, 255) + Fraction(1, 2)) for v in px]
                       for px in row] for row in img[:20, :30]], np.uint16)
    a, ca, _, _ = oracle.label(np.ascontiguousarray(img[:20, :30]), {"chip": 16})
    b, cb, _, _ = oracle.label(img16, {"chip": 16})
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(ca, cb)


def test_u16_nodata_is_masked_and_left_out_of_statistics():
    img16, _ = synth.scene(64, 64, 7, n_floes=4, dtype=np.uint16)
    nod = (img16.max(axis=2) == 0)
    assert nod.any() and not nod.all()
    labels, counts, _, stats = oracle.label(img16, {"chip": 64})
    assert (labels[nod] == 3).all()
    assert stats[0]["n"] == int((~nod).sum())
    all0 = np.zeros((8, 8, 3), np.uint16)
    labels, counts, _, _ = oracle.label(all0, {"chip": 8})
    assert (labels == 3).all() and list(counts) == [0, 0, 0, 64]


def test_bgr_order_only_moves_hue():
    img, _ = synth.scene(64, 64, 8, n_floes=4)
    a, ca, _, _ = oracle.label(img, {"chip": 32})
    b, cb, _, _ = oracle.label(np.ascontiguousarray(img[:, :, ::-1]), {"chip": 32, "bgr": 1})
    np.testing.assert_array_equal(a, b)


def test_hue_range_matches_colorsys():
    """Random colours with the filter off and a hue window on the thin class:
    the oracle's decision equals the one taken on colorsys' hue (rounded),
    away from rounding ties."""
    rng = np.random.default_rng(9)
    cols = rng.integers(0, 256, (1, 4000, 3)).astype(np.uint8)
    p = {"filter": 0, "chip": 256, "lo": [[0, 0, 205], [40, 60, 31], [0, 0, 0]],
         "hi": [[185, 255, 255], [100, 200, 204], [185, 255, 30]]}
    labels, _, _, _ = oracle.label(cols, p)
    checked = 0
    for i, (r, g, b) in enumerate(cols[0]):
        hf, sf, vf = colorsys.rgb_to_hsv(r / 255, g / 255, b / 255)
        h, s, v = hf * 180, sf * 255, vf * 255
        if min(abs(h - round(h) - 0.5), abs(h - round(h) + 0.5)) < 1e-6:
            continue
        if min(abs(s - round(s) - 0.5), abs(s - round(s) + 0.5)) < 1e-6:
            continue
        hr, sr = int(np.floor(h + 0.5)) % 180, int(np.floor(s + 0.5))
        if v >= 205:
            want = 0
        elif v >= 31:
            want = 1 if (40 <= hr <= 100 and 60 <= sr <= 200) else 3
        else:
            want = 2
        assert labels[0, i] == want, (r, g, b, hr, sr)
        checked += 1
    assert checked > 3500


def test_invalid_params_rejected():
    assert oracle.params_valid({})
    assert not oracle.params_valid({"chip": 3})
    assert not oracle.params_valid({"chip": 513})
    assert not oracle.params_valid({"lo": [[10, 0, 0], [0, 0, 0], [0, 0, 0]],
                                    "hi": [[5, 255, 255], [185, 255, 204], [185, 255, 30]]})
    assert not oracle.params_valid({"u16_scale": 0})
    assert not oracle.params_valid({"mm_min_range": 0})


# --------------------------------------------------------------------------
# Confusion counts (Sec. IV-A evaluation metrics) == numpy bincount.
# --------------------------------------------------------------------------
def test_confusion_matches_bincount():
    rng = np.random.default_rng(10)
    a = rng.integers(0, 4, (70, 90)).astype(np.uint8)
    b = rng.integers(0, 4, (70, 90)).astype(np.uint8)
    conf, chip_conf = oracle.confusion(a, b, chip=32)
    want = np.bincount((a.astype(int) * 4 + b).ravel(), minlength=16).reshape(4, 4)
    np.testing.assert_array_equal(conf, want)
    np.testing.assert_array_equal(chip_conf.sum(axis=(0, 1)), conf)
    sub = np.bincount((a[32:64, 64:90].astype(int) * 4 + b[32:64, 64:90]).ravel(), minlength=16)
    np.testing.assert_array_equal(chip_conf[1, 2].ravel(), sub)


# --------------------------------------------------------------------------
# The filter's corrected value V' (the U-Net's filtered input is built from it).
# --------------------------------------------------------------------------
def test_vprime_is_v_without_filter():
    img, _ = synth.scene(130, 170, 4, n_floes=5)
    vp = oracle.filtered_value(img, {"filter": 0})
    assert np.array_equal(vp, img.max(axis=2))


def test_vprime_worked_example_endpoints():
    """Ex1 of the hand-labelled tiles: lo = 60 stretches to 0, hi = 180 to 255
    (min-max normalisation, Sec. III-B)."""
    case = next(c for c in _golden_cases() if c["name"] == "ex1_two_levels_stretched")
    vp = oracle.filtered_value(_grey(case["v"]), case["params"])
    assert np.array_equal(vp, np.array([[0, 0, 255, 255]] * 4, np.uint8))


def test_vprime_decides_the_class():
    """With the default ranges (H and S unconstrained) and no absdiff mask, a
    pixel's label is the class whose V range holds its V'."""
    img, _ = synth.scene(400, 300, 6, n_floes=9, n_haze=2, n_shadow=2)
    labels, _, _, _ = oracle.label(img)
    vp = oracle.filtered_value(img)
    expect = np.where(vp >= 205, 0, np.where(vp >= 31, 1, 2)).astype(np.uint8)
    assert np.array_equal(labels, expect)


def test_vprime_nodata_is_zero():
    img, _ = synth.scene(200, 260, 8, n_floes=4, dtype=np.uint16)
    vp = oracle.filtered_value(img)
    nodata = (img == 0).all(axis=2)
    assert nodata.any() and not vp[nodata].any()
