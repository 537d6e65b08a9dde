"""Parity of the CUDA labeler (through the C ABI) with the CPU oracle.

Bit-exact: labels, per-request counts and per-chip counts must be identical
(0 mismatched pixels).  Inputs are seeded synthetic scenes (see synth/) and
random small shapes that cover ragged chips, odd widths, unaligned rows and
the degenerate cases of the method.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sil():
    import paper_2403_13135_gb300 as m
    return m


def _to_dev(img, pad_bytes=0, offset_bytes=0):
    """Device copy of an H x W x 3 array with optional row padding and a
    misaligned base (offset into a larger buffer); returns (tensor view,
    backing buffer)."""
    H, W, _ = img.shape
    es = img.dtype.itemsize
    row = W * 3 * es + pad_bytes
    buf = torch.zeros(offset_bytes + H * row + 64, dtype=torch.uint8, device="cuda")
    host = np.zeros(offset_bytes + H * row + 64, np.uint8)
    for y in range(H):
        host[offset_bytes + y * row: offset_bytes + y * row + W * 3 * es] = img[y].view(np.uint8).ravel()
    buf.copy_(torch.from_numpy(host))
    if es == 1:
        view = torch.as_strided(buf, (H, W, 3), (row, 3, 1), offset_bytes)
    else:
        assert offset_bytes % 2 == 0 and row % 2 == 0
        view = torch.as_strided(buf.view(torch.int16), (H, W, 3), (row // 2, 3, 1), offset_bytes // 2)
    return view, buf


def _check(sil, img, p=None, pad=0, off=0, want_labels=True):
    p = dict(p or {})
    dev, keep = _to_dev(img, pad, off)
    lab, cnt, cc = sil.label(dev, p, labels=want_labels, chip_counts=True)
    torch.cuda.synchronize()
    olab, ocnt, occ, _ = oracle.label(img, p)
    if want_labels:
        got = lab.cpu().numpy()
        bad = int((got != olab).sum())
        assert bad == 0, f"{bad} mismatched pixels (shape {img.shape}, params {p})"
    np.testing.assert_array_equal(cnt.cpu().numpy().astype(np.uint64), ocnt)
    np.testing.assert_array_equal(cc.cpu().numpy().astype(np.uint32), occ)


def test_tile_512_seed0(sil):
    img, _ = synth.tile_512(0)
    _check(sil, img)


def test_tile_512_no_filter_and_no_median(sil):
    img, _ = synth.tile_512(0)
    _check(sil, img, {"filter": 0})
    _check(sil, img, {"median": 0})


@pytest.mark.parametrize("chip", [4, 5, 16, 37, 64, 128, 200, 256])
def test_chip_sizes(sil, chip):
    img, _ = synth.scene(301, 283, 11, n_floes=7)
    _check(sil, img, {"chip": chip})


@pytest.mark.parametrize("chip", [257, 300, 512])
def test_large_chips_generic_path(sil, chip):
    img, _ = synth.scene(530, 610, 12, n_floes=7)
    _check(sil, img, {"chip": chip})


@pytest.mark.parametrize("shape", [(1, 1), (1, 300), (300, 1), (2, 2), (3, 17), (17, 3),
                                   (255, 257), (256, 256), (257, 255), (16, 16), (5, 33)])
def test_degenerate_and_ragged_shapes(sil, shape):
    img, _ = synth.scene(shape[0], shape[1], 13, n_floes=3)
    _check(sil, img)


@pytest.mark.parametrize("pad,off", [(0, 1), (0, 3), (5, 0), (13, 7), (1, 15), (16, 0)])
def test_unaligned_rows(sil, pad, off):
    img, _ = synth.scene(270, 260, 14, n_floes=5)
    _check(sil, img, pad=pad, off=off)


def test_random_small_images_many_params(sil):
    rng = np.random.default_rng(99)
    for trial in range(25):
        H, W = int(rng.integers(1, 90)), int(rng.integers(1, 90))
        img = rng.integers(0, 256, (H, W, 3)).astype(np.uint8)
        p = {"chip": int(rng.integers(4, 64)), "mm_min_range": int(rng.integers(1, 120)),
             "mm_min_frac_den": int(rng.integers(1, 40)), "v_trunc": int(rng.integers(100, 256)),
             "max_shift": int(rng.integers(0, 256)), "median": int(rng.integers(0, 2)),
             "filter": int(rng.integers(0, 2))}
        _check(sil, img, p, pad=int(rng.integers(0, 9)), off=int(rng.integers(0, 16)))


def test_hue_saturation_ranges(sil):
    """Narrowed H/S ranges switch on the per-pixel H/S decision."""
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, (200, 230, 3)).astype(np.uint8)
    p = {"chip": 64, "lo": [[0, 0, 180], [40, 60, 31], [90, 0, 0]],
         "hi": [[185, 40, 255], [100, 200, 204], [150, 255, 40]]}
    _check(sil, img, p)
    _check(sil, img, dict(p, filter=0))
    _check(sil, img, dict(p, bgr=1), off=5)
    _check(sil, img, dict(p, chip=300))


def test_bgr_flag(sil):
    img, _ = synth.scene(128, 160, 15, n_floes=4)
    _check(sil, img, {"bgr": 1})


def test_counts_only_mode(sil):
    img, _ = synth.tile_512(0)
    _check(sil, img, want_labels=False)


def test_u16_with_nodata(sil):
    img16, _ = synth.scene(300, 270, 16, n_floes=6, dtype=np.uint16)
    assert (img16.max(axis=2) == 0).any()
    _check(sil, img16)
    _check(sil, img16, {"chip": 64}, pad=2, off=2)
    _check(sil, img16, {"u16_scale": 4095})
    _check(sil, img16, {"chip": 300})
    p = {"lo": [[0, 0, 180], [40, 60, 31], [0, 0, 0]], "hi": [[185, 40, 255], [100, 200, 204], [185, 255, 40]]}
    _check(sil, img16, p)


def test_all_nodata_u16(sil):
    _check(sil, np.zeros((40, 50, 3), np.uint16), {"chip": 16})


def test_constant_images(sil):
    for v in (0, 30, 31, 204, 205, 255):
        _check(sil, np.full((70, 90, 3), v, np.uint8), {"chip": 32})


def test_worked_tiles_on_gpu(sil):
    import json, os
    cases = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_4x4.json")))["cases"]
    for c in cases:
        img = np.array(c["rgb"], np.uint8) if "rgb" in c else \
            np.repeat(np.array(c["v"], np.uint8)[:, :, None], 3, axis=2)
        dev, keep = _to_dev(img)
        lab, cnt, cc = sil.label(dev, c["params"], chip_counts=True)
        assert lab.cpu().numpy().tolist() == c["labels"], c["name"]
        assert cnt.cpu().numpy().tolist() == c["counts"], c["name"]


def test_invalid_arguments_rejected(sil):
    img = torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(sil.SilError):
        sil.label(img, {"chip": 2})
    with pytest.raises(sil.SilError):
        sil.label(img, {"lo": [[200, 0, 0], [0, 0, 31], [0, 0, 0]]})
    cnt = torch.empty(4, dtype=torch.int64, device="cuda")
    p = sil.params()
    import ctypes
    st = sil.sil_label(img.data_ptr(), 8, 8, 10, sil.SIL_U8, ctypes.byref(p), None, 8, cnt.data_ptr(), None, None)
    assert st == sil.SIL_EINVAL
    st = sil.sil_label(img.data_ptr(), 0, 8, 24, sil.SIL_U8, ctypes.byref(p), None, 8, cnt.data_ptr(), None, None)
    assert st == sil.SIL_EINVAL
    st = sil.sil_label(None, 8, 8, 24, sil.SIL_U8, ctypes.byref(p), None, 8, cnt.data_ptr(), None, None)
    assert st == sil.SIL_EINVAL


def test_host_buffer_entry_point(sil):
    img, _ = synth.scene(333, 517, 17, n_floes=6)
    lab, cnt, cc = sil.label_host(img, None, chip_counts=True)
    olab, ocnt, occ, _ = oracle.label(img)
    assert int((lab != olab).sum()) == 0
    np.testing.assert_array_equal(cnt, ocnt)
    np.testing.assert_array_equal(cc, occ)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_host_entry_point_striped(sil, dtype):
    """The host entry point pipelines stripes of whole chip rows (copy in,
    label, copy out on three streams): a tall image of many stripes, host
    rows with padding, a label pitch wider than W, a chip of 100."""
    img, _ = synth.scene(2900, 300, 5, n_floes=8, dtype=dtype)
    bpp = img.dtype.itemsize * 3
    host = np.zeros((2900, 300 * bpp + 16), np.uint8)
    host[:, :300 * bpp] = img.view(np.uint8).reshape(2900, 300 * bpp)
    view = host[:, :300 * bpp].view(img.dtype).reshape(2900, 300, 3)
    assert view.strides[0] == 300 * bpp + 16
    p = dict(oracle.params_default(), chip=100)
    pp = sil.params(chip=100)
    lab = np.full((2900, 320), 7, np.uint8)
    cnt = np.zeros(4, np.uint64)
    cc = np.zeros((29, 3, 4), np.uint32)
    import ctypes
    dt = sil.SIL_U8 if dtype == np.uint8 else sil.SIL_U16
    sil.check(sil.sil_label_host(view.ctypes.data, 2900, 300, view.strides[0], dt, ctypes.byref(pp),
                                 lab.ctypes.data, 320, cnt.ctypes.data, cc.ctypes.data, None))
    olab, ocnt, occ, _ = oracle.label(np.ascontiguousarray(view), p)
    assert int((lab[:, :300] != olab).sum()) == 0
    assert np.all(lab[:, 300:] == 7)          # bytes past W untouched
    np.testing.assert_array_equal(cnt, ocnt)
    np.testing.assert_array_equal(cc, occ)


def test_full_scene_sampled_chips(sil):
    """The 10980 x 10980 scene in the benchmark's launch configuration:
    per-chip counts of sampled chips and their labels against the oracle run
    on the chip-aligned crops (a chip's labels depend on that chip alone);
    totals against the sum of chip counts."""
    img, _ = synth.full_scene(1)
    H, W, _ = img.shape
    dev = torch.from_numpy(img).cuda()
    lab, cnt, cc = sil.label(dev, None, chip_counts=True)
    torch.cuda.synchronize()
    cc = cc.cpu().numpy().astype(np.int64)
    cnt = cnt.cpu().numpy()
    assert int(cnt.sum()) == H * W
    np.testing.assert_array_equal(cc.sum(axis=(0, 1)), cnt)
    gy, gx = cc.shape[:2]
    rng = np.random.default_rng(3)
    picks = {(0, 0), (gy - 1, gx - 1), (0, gx - 1), (gy - 1, 0)}
    while len(picks) < 16:
        picks.add((int(rng.integers(0, gy)), int(rng.integers(0, gx))))
    lab_h = lab.cpu().numpy()
    for (cy, cx) in sorted(picks):
        y0, x0 = cy * 256, cx * 256
        crop = np.ascontiguousarray(img[y0:y0 + 256, x0:x0 + 256])
        olab, ocnt, occ, _ = oracle.label(crop)
        np.testing.assert_array_equal(cc[cy, cx], occ[0, 0].astype(np.int64))
        assert int((lab_h[y0:y0 + 256, x0:x0 + 256] != olab).sum()) == 0, (cy, cx)


def test_same_result_any_stream_and_repeat(sil):
    img, _ = synth.tile_512(0)
    dev = torch.from_numpy(img).cuda()
    a, ca, _ = sil.label(dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b, cb, _ = sil.label(dev, stream=s)
    s.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(ca, cb)


@pytest.mark.parametrize("case", ["u8", "u16_nodata", "chip100", "chip300", "filter_off", "narrow_h"])
def test_vprime_matches_oracle(sil, case):
    """sil_label_v: the filter's corrected value V' of every pixel, bit-exact,
    and the same labels and counts as sil_label."""
    p = {}
    dtype = np.uint16 if case == "u16_nodata" else np.uint8
    img, _ = synth.scene(700, 530, 31, n_floes=7, n_haze=2, n_shadow=2, dtype=dtype)
    if case == "chip100":
        p = {"chip": 100}
    elif case == "chip300":
        p = {"chip": 300}
    elif case == "filter_off":
        p = {"filter": 0}
    elif case == "narrow_h":
        p = {"lo": [[0, 0, 205], [60, 0, 31], [0, 0, 0]]}
    dev = torch.from_numpy(img).cuda()
    lab, vp, cnt = sil.label_v(dev, p)
    lab1, cnt1, _ = sil.label(dev, p)
    torch.cuda.synchronize()
    ovp = oracle.filtered_value(img, p)
    assert int((vp.cpu().numpy() != ovp).sum()) == 0
    assert torch.equal(lab, lab1) and torch.equal(cnt, cnt1)


def test_image_beyond_4gib(sil):
    """A 38000 x 38000 u8 image (4.33 GB in, 1.44 GB of labels): byte offsets
    past 2^32 in every address of the last chip rows.  The image tiles a
    2000 x 2000 scene (a period that is not a multiple of the chip, so the
    chips differ) with a different scene in its bottom-right corner; sampled
    chips there and elsewhere against the oracle on chip-aligned crops, the
    totals against the sum of the chip counts, and the host entry point equal
    to the device one."""
    base, _ = synth.scene(2000, 2000, 5, n_floes=30, n_haze=2, n_shadow=2)
    img = np.tile(base, (19, 19, 1))
    H, W, _ = img.shape
    corner, _ = synth.scene(600, 900, 7, n_floes=6, n_haze=1, n_shadow=1)
    img[H - 600:, W - 900:] = corner
    assert (H - 1) * W * 3 > 2 ** 32
    dev = torch.from_numpy(img).cuda()
    lab, cnt, cc = sil.label(dev, None, chip_counts=True)
    torch.cuda.synchronize()
    del dev
    cnt = cnt.cpu().numpy()
    cc = cc.cpu().numpy().astype(np.int64)
    lab_h = lab.cpu().numpy()
    del lab
    assert int(cnt.sum()) == H * W
    np.testing.assert_array_equal(cc.sum(axis=(0, 1)), cnt)
    gy, gx = cc.shape[:2]
    assert (gy, gx) == (149, 149)
    picks = {(0, 0), (0, gx - 1), (gy - 1, 0), (gy - 1, gx - 1), (gy - 2, gx - 3),
             (gy - 3, gx - 2), (gy - 1, gx - 4), (gy // 2, gx // 2)}
    rng = np.random.default_rng(8)
    while len(picks) < 16:
        picks.add((int(rng.integers(0, gy)), int(rng.integers(0, gx))))
    for (cy, cx) in sorted(picks):
        y0, x0 = cy * 256, cx * 256
        crop = np.ascontiguousarray(img[y0:y0 + 256, x0:x0 + 256])
        olab, _, occ, _ = oracle.label(crop)
        np.testing.assert_array_equal(cc[cy, cx], occ[0, 0].astype(np.int64))
        assert int((lab_h[y0:y0 + 256, x0:x0 + 256] != olab).sum()) == 0, (cy, cx)
    hlab, hcnt, hcc = sil.label_host(img, None, chip_counts=True)
    assert np.array_equal(hlab, lab_h)
    np.testing.assert_array_equal(hcnt.astype(np.uint64), cnt.astype(np.uint64))
    np.testing.assert_array_equal(hcc.astype(np.int64), cc)


@pytest.mark.parametrize("case", ["chip256", "chip256_counts_only", "chip100", "chip8", "one_wave_limit"])
def test_split_chips_match_oracle(sil, case):
    """Requests with few chips (four CTAs per chip fit in one wave of
    resident CTAs) are labelled by clusters of four CTAs, one row slice each,
    with the histogram summed across the cluster; "one_wave_limit" has the
    largest such chip count on this GPU, plus one (whole-chip path).  Whole
    images against the oracle: labels, V', counts and chip counts
    bit-exact."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    p = {}
    if case.startswith("chip256"):
        H, W = 1000, 1500                          # 4 x 6 chips, ragged edges
    elif case == "chip100":
        H, W, p = 700, 530, {"chip": 100}
    elif case == "chip8":
        H, W, p = 64, 61, {"chip": 8}
    else:
        n = (2 * sms) // 4 + 1                     # two CTAs per SM on this GPU
        H, W, p = 64, 64 * n - 5, {"chip": 64}
    img, _ = synth.scene(H, W, 47, n_floes=9, n_haze=2, n_shadow=2)
    dev = torch.from_numpy(img).cuda()
    want_labels = case != "chip256_counts_only"
    lab, vp, cnt, cc = sil.label_v(dev, p, labels=want_labels, chip_counts=True)
    torch.cuda.synchronize()
    olab, ocnt, occ, _ = oracle.label(img, p)
    if want_labels:
        assert int((lab.cpu().numpy() != olab).sum()) == 0
    np.testing.assert_array_equal(vp.cpu().numpy(), oracle.filtered_value(img, p))
    np.testing.assert_array_equal(cnt.cpu().numpy().astype(np.uint64), ocnt)
    np.testing.assert_array_equal(cc.cpu().numpy().astype(np.uint32), occ)
