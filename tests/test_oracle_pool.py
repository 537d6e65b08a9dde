"""The multi-core oracle runner of the full-size parity tests: stripes of
whole chip rows and crops give the same labels, counts and chip counts as
the oracle on the whole image (chips are anchored at the image origin, so a
stripe that starts on the chip grid holds the same chips)."""
import numpy as np

import oracle
import synth
from oracle_pool import OraclePool, digest


def test_stripes_and_crops_equal_whole_image():
    img, _ = synth.scene(700, 530, 21, n_floes=6, n_haze=1, n_shadow=1)
    lab, cnt, cc, _ = oracle.label(img)
    with OraclePool(cores=2) as pool:
        dig, scnt, scc = pool.label_stripes(img)
        assert dig == [digest(lab[y:y + 256]) for y in range(0, 700, 256)]
        np.testing.assert_array_equal(scnt, cnt)
        np.testing.assert_array_equal(scc, cc)
        boxes = [(0, 0, 700, 530), (13, 7, 100, 300), (256, 256, 444, 274)]
        res = pool.label_crops(img, boxes, {"chip": 64})
        for (y, x, h, w), (d, c, ccc) in zip(boxes, res):
            ol, oc, occ, _ = oracle.label(np.ascontiguousarray(img[y:y + h, x:x + w]), {"chip": 64})
            assert d == digest(ol)
            np.testing.assert_array_equal(c, oc)
            np.testing.assert_array_equal(ccc, occ)
        # a different label map gives a different digest
        lab2 = lab.copy()
        lab2[5, 5] ^= 1
        assert digest(lab2) != digest(lab)
