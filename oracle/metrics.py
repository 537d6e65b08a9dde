"""CPU oracle of the evaluation outputs -- TEST INFRASTRUCTURE ONLY.

Only the tests and ``__graft_entry__.smoke()`` may import this module; the
product library never loads it.  Plain numpy, written from the definitions:

* ``render``: the paper's colour masks (Sec. III-A, the label colours of the
  manual and auto labels: red for snow-covered / thick ice, blue for thin /
  young ice, green for open water); masked pixels (code 3) black.
* ``chip_grid``: a scene cut into its chip grid anchored at (0, 0), zero past
  the right and bottom edges (Sec. III-C cuts scenes into 256 x 256 images).
* ``metrics``: Sec. IV-A "Evaluation Metrics" -- accuracy, precision,
  recall and F1 score, and the confusion matrix whose element in row A and
  column B is the number of samples predicted as A over the number of
  samples of class B, so that each column adds up to 100 %.

Readings where the paper is silent: the three classes are the paper's
(thick ice, thin ice, open water); pixels whose reference is masked (code 3)
are left out of every metric; a prediction of "masked" counts as a miss of
the pixel's reference class (it appears in row 3 of the matrix); the single
precision / recall / F1 figures are the unweighted means over the classes
(macro), the support-weighted means are given as well; a precision, recall
or F1 whose denominator is zero is 0.
"""
from __future__ import annotations

import numpy as np

# Sec. III-A: red thick ice, blue thin ice, green open water; masked black.
PALETTE = np.array([[255, 0, 0],
                    [0, 0, 255],
                    [0, 255, 0],
                    [0, 0, 0]], dtype=np.uint8)
N_CLASSES = 3


def render(labels: np.ndarray) -> np.ndarray:
    """[..., H, W] label codes 0..3 -> [..., H, W, 3] uint8 colour masks."""
    lab = np.asarray(labels)
    assert lab.min() >= 0 and lab.max() <= 3
    return PALETTE[lab]


def chip_grid(img: np.ndarray, chip: int = 256) -> np.ndarray:
    """[H, W, ...] -> [gy * gx, chip, chip, ...], row-major over the grid,
    zero past the edges."""
    H, W = img.shape[:2]
    gy, gx = -(-H // chip), -(-W // chip)
    out = np.zeros((gy * gx, chip, chip) + img.shape[2:], dtype=img.dtype)
    for k in range(gy * gx):
        cy, cx = divmod(k, gx)
        part = img[cy * chip:(cy + 1) * chip, cx * chip:(cx + 1) * chip]
        out[k, :part.shape[0], :part.shape[1]] = part
    return out


def _div(a, b):
    return a / b if b else 0.0


def metrics(conf) -> dict:
    """Metrics of a 4 x 4 confusion count matrix conf[pred][ref]."""
    c = np.asarray(conf, dtype=np.float64).reshape(4, 4)
    cols = c[:, :N_CLASSES]            # reference masked: left out
    total = cols.sum()
    col_sum = cols.sum(axis=0)         # pixels of each reference class
    row_sum = cols.sum(axis=1)         # pixels predicted as each code
    tp = np.array([c[k, k] for k in range(N_CLASSES)])
    prec = np.array([_div(tp[k], row_sum[k]) for k in range(N_CLASSES)])
    rec = np.array([_div(tp[k], col_sum[k]) for k in range(N_CLASSES)])
    f1 = np.array([_div(2 * prec[k] * rec[k], prec[k] + rec[k]) for k in range(N_CLASSES)])
    matrix = np.zeros((4, 4))
    for b in range(N_CLASSES):
        if col_sum[b]:
            matrix[:, b] = c[:, b] / col_sum[b]
    w = col_sum / total if total else np.zeros(N_CLASSES)
    return {
        "accuracy": _div(tp.sum(), total),
        "precision": prec, "recall": rec, "f1": f1,
        "macro_precision": prec.mean(), "macro_recall": rec.mean(), "macro_f1": f1.mean(),
        "weighted_precision": float((prec * w).sum()), "weighted_recall": float((rec * w).sum()),
        "weighted_f1": float((f1 * w).sum()),
        "matrix": matrix, "support": col_sum.astype(np.uint64),
    }
