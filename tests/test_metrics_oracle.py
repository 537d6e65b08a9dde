"""Pins of the evaluation oracle (oracle/metrics.py): the colour masks
against the paper's label colours (Sec. III-A), the chip grid against
slicing, and the metrics of Sec. IV-A against a hand-worked case and against
scikit-learn's definitions on random label maps."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import metrics as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "metrics_worked.json")


def test_render_is_the_papers_legend():
    # red snow-covered/thick ice, blue thin/young ice, green open water
    lab = np.array([[0, 1], [2, 3]], np.uint8)
    rgb = M.render(lab)
    assert rgb.tolist() == [[[255, 0, 0], [0, 0, 255]], [[0, 255, 0], [0, 0, 0]]]
    assert rgb.dtype == np.uint8 and rgb.shape == (2, 2, 3)


def test_chip_grid_zero_pads_the_edges():
    img = np.arange(5 * 7 * 3, dtype=np.uint8).reshape(5, 7, 3)
    g = M.chip_grid(img, 4)
    assert g.shape == (4, 4, 4, 3)
    assert np.array_equal(g[0], img[:4, :4])
    assert np.array_equal(g[1, :, :3], img[:4, 4:7]) and not g[1, :, 3:].any()
    assert np.array_equal(g[2, :1], img[4:5, :4]) and not g[2, 1:].any()
    assert np.array_equal(g[3, :1, :3], img[4:5, 4:7])


def test_metrics_hand_worked_case():
    case = json.load(open(GOLDEN))
    m = M.metrics(case["conf"])
    fr = lambda p: float(Fraction(p[0], p[1]))
    assert m["accuracy"] == pytest.approx(fr(case["accuracy"]), abs=1e-15)
    for k in range(3):
        assert m["precision"][k] == pytest.approx(fr(case["precision"][k]), abs=1e-15)
        assert m["recall"][k] == pytest.approx(fr(case["recall"][k]), abs=1e-15)
        assert m["f1"][k] == pytest.approx(fr(case["f1"][k]), abs=1e-15)
    assert m["macro_f1"] == pytest.approx(np.mean([fr(f) for f in case["f1"]]), abs=1e-15)
    assert m["weighted_recall"] == pytest.approx(np.mean([fr(r) for r in case["recall"]]), abs=1e-15)
    np.testing.assert_allclose(m["matrix"], case["matrix"], atol=1e-15)
    np.testing.assert_allclose(m["matrix"][:, :3].sum(axis=0), 1.0)   # columns add up to 100 %
    assert m["support"].tolist() == case["support"]


def test_metrics_degenerate_cases():
    # a perfect classification: diagonal matrix, every score 1
    m = M.metrics(np.diag([5, 7, 9, 0]))
    assert m["accuracy"] == 1.0 and np.allclose(m["f1"], 1.0)
    assert np.allclose(m["matrix"][:3, :3], np.eye(3))
    # a class never predicted and never present: its scores are 0
    c = np.zeros((4, 4)); c[0, 0] = 4; c[2, 2] = 6
    m = M.metrics(c)
    assert m["precision"][1] == 0 and m["recall"][1] == 0 and m["f1"][1] == 0
    assert m["accuracy"] == 1.0


def test_metrics_against_sklearn_on_random_maps():
    sk = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(4)
    for trial in range(20):
        ref = rng.integers(0, 4, (37, 41)).astype(np.uint8)
        pred = np.where(rng.random(ref.shape) < 0.7, ref, rng.integers(0, 4, ref.shape)).astype(np.uint8)
        conf, _ = oracle.confusion(pred, ref, chip=16)
        m = M.metrics(conf)
        keep = ref.ravel() < 3
        yt, yp = ref.ravel()[keep], pred.ravel()[keep]
        p, r, f, s = sk.precision_recall_fscore_support(yt, yp, labels=[0, 1, 2], zero_division=0)
        np.testing.assert_allclose(m["precision"], p, atol=1e-12)
        np.testing.assert_allclose(m["recall"], r, atol=1e-12)
        np.testing.assert_allclose(m["f1"], f, atol=1e-12)
        assert m["accuracy"] == pytest.approx(sk.accuracy_score(yt, yp), abs=1e-12)
        for avg, key in (("macro", "macro"), ("weighted", "weighted")):
            pa, ra, fa, _ = sk.precision_recall_fscore_support(yt, yp, labels=[0, 1, 2], average=avg,
                                                               zero_division=0)
            assert m[f"{key}_precision"] == pytest.approx(pa, abs=1e-12)
            assert m[f"{key}_recall"] == pytest.approx(ra, abs=1e-12)
            assert m[f"{key}_f1"] == pytest.approx(fa, abs=1e-12)
        cm = sk.confusion_matrix(yt, yp, labels=[0, 1, 2, 3], normalize="true")  # rows: true class
        np.testing.assert_allclose(m["matrix"][:, :3], cm[:3].T, atol=1e-12)


def test_library_metrics_equal_the_oracle():
    """sil_metrics_from_confusion (host code of the library, no GPU) against
    the oracle's definitions on the worked case and random counts."""
    sil = pytest.importorskip("paper_2403_13135_gb300")
    case = json.load(open(GOLDEN))
    rng = np.random.default_rng(9)
    confs = [np.array(case["conf"], np.uint64), np.diag([5, 7, 9, 0]).astype(np.uint64),
             np.zeros((4, 4), np.uint64)]
    confs += [rng.integers(0, 10 ** 6, (4, 4)).astype(np.uint64) for _ in range(30)]
    confs += [(rng.random((4, 4)) < 0.4) * rng.integers(0, 50, (4, 4)).astype(np.uint64) for _ in range(30)]
    for c in confs:
        got, want = sil.metrics(c), M.metrics(c)
        for k in ("accuracy", "macro_precision", "macro_recall", "macro_f1", "weighted_precision",
                  "weighted_recall", "weighted_f1"):
            assert got[k] == pytest.approx(want[k], rel=1e-12, abs=1e-15), k
        for k in ("precision", "recall", "f1"):
            np.testing.assert_allclose(got[k], want[k], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(got["matrix"], want["matrix"], rtol=1e-12, atol=1e-15)
        assert got["support"] == want["support"].tolist()
    with pytest.raises(sil.SilError):
        import ctypes
        sil.check(sil._lib.sil_metrics_from_confusion(None, ctypes.byref(sil.sil_metrics())))
