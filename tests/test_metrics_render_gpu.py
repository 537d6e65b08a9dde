"""Confusion counts (Sec. IV-A evaluation metrics) and the colour render of
the label map (Sec. III-A colours) on the GPU, against the oracle / numpy."""
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
    pal = {0: (255, 0, 0), 1: (0, 0, 255), 2: (0, 255, 0), 3: (0, 0, 0)}
    for y in range(2):
        for x in range(4):
            assert tuple(rgb[y, x]) == pal[int(lab[y, x])]
