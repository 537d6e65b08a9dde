"""The seeded synthetic inputs follow their stated recipe (the stand-in for
the paper's Sentinel-2 scenes): deterministic per seed, class colours around
the stated means with the stated noise, shadows halve and thin cloud
brightens, the uint16 form is the scaled uint8 form with a nodata wedge,
and the uneven-tile shapes stay in their ranges.  CPU only."""
import numpy as np

import synth


def test_same_seed_same_bytes_other_seed_other_bytes():
    a, ta = synth.scene(200, 240, 9, n_floes=6)
    b, tb = synth.scene(200, 240, 9, n_floes=6)
    c, _ = synth.scene(200, 240, 10, n_floes=6)
    assert np.array_equal(a, b) and np.array_equal(ta, tb)
    assert not np.array_equal(a, c)


def test_class_colours_and_noise_without_shadow_or_haze():
    img, truth = synth.scene(600, 600, 3, n_floes=30, n_haze=0, n_shadow=0)
    assert set(np.unique(truth)) <= {0, 1, 2}
    for k in range(3):
        px = img[truth == k].astype(np.float64)
        if len(px) < 1000:
            continue
        assert np.all(np.abs(px.mean(0) - synth.CLASS_MEANS[k]) < 1.0), (k, px.mean(0))
        if k == 1:  # thin ice is far from both clip bounds: the noise is plain N(0, 8), rounded
            assert np.all(np.abs(px.std(0) - synth.NOISE_SIGMA) < 0.3), px.std(0)


def test_shadow_halves_and_haze_brightens():
    base, _ = synth.scene(300, 300, 5, n_floes=10, n_haze=0, n_shadow=0)
    sh, _ = synth.scene(300, 300, 5, n_floes=10, n_haze=0, n_shadow=2)
    hz, _ = synth.scene(300, 300, 5, n_floes=10, n_haze=1, n_shadow=0)   # one blob: at most +40
    # same floes and noise (drawn before the shadows and the blobs)
    changed = np.any(sh != base, axis=2)
    assert changed.any()
    assert np.array_equal(sh[changed], base[changed] // 2)
    up = hz.astype(np.int16) - base.astype(np.int16)
    assert up.min() >= 0 and up.max() <= synth.HAZE_AMPLITUDE
    assert (up > 0).any()


def test_uint16_is_scaled_uint8_with_a_nodata_wedge():
    img8, _ = synth.scene(128, 160, 11, n_floes=5)
    img16, _ = synth.scene(128, 160, 11, n_floes=5, dtype=np.uint16)
    assert img16.dtype == np.uint16
    nodata = np.all(img16 == 0, axis=2)
    assert nodata[0, 0] and not nodata[-1, -1]
    want = np.rint(img8.astype(np.float64) * 10000.0 / 255.0).astype(np.uint16)
    assert np.array_equal(img16[~nodata], want[~nodata])
    # the wedge is the triangle y + x < k
    ys, xs = np.nonzero(nodata)
    k = int((ys + xs).max()) + 1
    yy, xx = np.mgrid[:128, :160]
    assert np.array_equal(nodata, (yy + xx) < k)


def test_uneven_tile_shapes_stay_in_range():
    shapes = synth.uneven_tile_shapes(64)
    assert len(shapes) == 64
    for H, W, seed in shapes:
        s, o = min(H, W), max(H, W)
        assert s in synth.TILE_SIDES
        assert s <= o <= 2 * s
    assert len({(H, W) for H, W, _ in shapes}) > 10
