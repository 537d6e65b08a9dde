"""Confusion counts and the metrics derived from them (Sec. IV-A
evaluation metrics), the colour render of the label map (Sec. III-A colours)
and the export of (image chip, colour-mask chip) training pairs on the GPU,
against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from oracle import metrics as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sil():
    import paper_2403_13135_gb300 as m
    return m


def test_confusion_matches_oracle(sil):
    rng = np.random.default_rng(21)
    for (H, W, chip) in [(300, 517, 256), (64, 64, 16), (1, 1, 4), (513, 77, 100)]:
        a = rng.integers(0, 4, (H, W)).astype(np.uint8)
        b = rng.integers(0, 4, (H, W)).astype(np.uint8)
        conf, cc = sil.confusion(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), chip, chip_conf=True)
        torch.cuda.synchronize()
        oconf, occ = oracle.confusion(a, b, chip)
        np.testing.assert_array_equal(conf.cpu().numpy().astype(np.uint64), oconf)
        np.testing.assert_array_equal(cc.cpu().numpy().astype(np.uint32), occ)


def test_confusion_of_labels_against_floe_truth(sil):
    """f1 use: labels of a synthetic scene against its floe ground truth."""
    img, truth = synth.tile_512(0)
    lab, _, _ = sil.label(torch.from_numpy(img).cuda())
    conf, _ = sil.confusion(lab, torch.from_numpy(truth).cuda())
    torch.cuda.synchronize()
    olab, _, _, _ = oracle.label(img)
    oconf, _ = oracle.confusion(olab, truth, 256)
    np.testing.assert_array_equal(conf.cpu().numpy().astype(np.uint64), oconf)
    assert int(conf.sum()) == 512 * 512


def test_render_palette(sil):
    lab = np.array([[0, 1, 2, 3], [3, 2, 1, 0]], np.uint8)
    rgb = sil.render(torch.from_numpy(lab).cuda()).cpu().numpy()
    assert np.array_equal(rgb, M.render(lab))
    img, _ = synth.scene(301, 283, 8, n_floes=6)
    olab, _, _, _ = oracle.label(img)
    rgb = sil.render(torch.from_numpy(olab).cuda()).cpu().numpy()
    assert np.array_equal(rgb, M.render(olab))


def test_metrics_of_labels_against_floe_truth(sil):
    """Sec. IV-A metrics of the auto-labels against the generator's floe
    truth: confusion counts on the GPU, metrics from them, equal to the
    oracle's labels, confusion and metric definitions."""
    img, truth = synth.scene(1000, 900, 23, n_floes=15, n_haze=3, n_shadow=3)
    lab, _, _ = sil.label(torch.from_numpy(img).cuda())
    conf, _ = sil.confusion(lab, torch.from_numpy(truth).cuda())
    torch.cuda.synchronize()
    got = sil.metrics(conf)
    olab, _, _, _ = oracle.label(img)
    oconf, _ = oracle.confusion(olab, truth, 256)
    want = M.metrics(oconf)
    assert got["accuracy"] == pytest.approx(want["accuracy"], abs=1e-12)
    np.testing.assert_allclose(got["f1"], want["f1"], atol=1e-12)
    np.testing.assert_allclose(got["matrix"], want["matrix"], atol=1e-12)
    assert got["accuracy"] > 0.5  # the synthetic classes are separable by V


@pytest.mark.parametrize("shape,chip,k0,n", [((700, 530), 256, 0, None), ((700, 530), 256, 4, 3),
                                             ((333, 517), 100, 0, None), ((61, 64), 8, 5, 40)])
def test_export_chips_matches_oracle(sil, shape, chip, k0, n):
    """Training pairs: every exported image chip equals the scene's chip grid
    (zero past the edges) and every mask chip the oracle's labels in the
    paper's colours, chip for chip."""
    img, _ = synth.scene(shape[0], shape[1], 29, n_floes=7, n_haze=2, n_shadow=2)
    dev = torch.from_numpy(img).cuda()
    p = {"chip": chip} if chip != 256 else None
    lab, _, _ = sil.label(dev, p)
    chips, masks = sil.export_chips(dev, lab, chip, k0, n)
    torch.cuda.synchronize()
    olab, _, _, _ = oracle.label(img, p)
    want_chips = M.chip_grid(img, chip)
    want_masks = M.chip_grid(M.render(olab), chip)
    end = len(want_chips) if n is None else k0 + n
    assert np.array_equal(chips.cpu().numpy(), want_chips[k0:end])
    assert np.array_equal(masks.cpu().numpy(), want_masks[k0:end])


def test_export_rejects_bad_ranges(sil):
    img = torch.zeros((300, 300, 3), dtype=torch.uint8, device="cuda")
    lab = torch.zeros((300, 300), dtype=torch.uint8, device="cuda")
    with pytest.raises(sil.SilError):
        sil.export_chips(img, lab, 256, 3, 2)    # the grid has 4 chips
    with pytest.raises(sil.SilError):
        sil.export_chips(img, lab, 2, 0, 1)      # chip below 4
