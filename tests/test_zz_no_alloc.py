"""The batched entry point that allocates nothing (sil_label_batch_noalloc),
for callers that may not allocate device memory: through the C ABI, two
calls in a row, each checked bit for bit against sil_label_batch (the entry
point that keeps its scratch in a context).  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _batch(shapes, seed):
    imgs = [synth.scene(h, w, seed + i, n_floes=4)[0] for i, (h, w) in enumerate(shapes)]
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    return imgs, dev


def _outputs(sil, imgs):
    labs = [torch.full(im.shape[:2], 7, dtype=torch.uint8, device="cuda") for im in imgs]
    cnts = [torch.full((4,), -1, dtype=torch.int64, device="cuda") for _ in imgs]
    ccs = [torch.full((-(-im.shape[0] // 256), -(-im.shape[1] // 256), 4), -1, dtype=torch.int32,
                      device="cuda") for im in imgs]
    return labs, cnts, ccs


def test_noalloc_matches_context_batch_twice():
    import paper_2403_13135_gb300 as sil
    p = sil.params()
    ctx = sil.Context()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    batches = [_batch([(300, 517), (256, 256), (64, 1000), (1, 1), (513, 40)], 900),
               _batch([(1000, 700), (17, 33), (256, 700)], 950)]
    for imgs, dev in batches:  # two calls in a row, different batches
        ref = _outputs(sil, imgs)
        got = _outputs(sil, imgs)
        t_ref = sil.make_tiles(dev, *ref)
        t_got = sil.make_tiles(dev, *got)
        sil.check(sil.sil_label_batch(t_ref, len(imgs), sil.SIL_U8, ctypes.byref(p), ctx.handle, stream))
        st = sil.sil_label_batch_noalloc(t_got, len(imgs), sil.SIL_U8, ctypes.byref(p), stream)
        assert st == sil.SIL_OK, sil.sil_last_error()
        torch.cuda.synchronize()
        for a, b in zip(ref[0], got[0]):
            assert torch.equal(a, b)
        for a, b in zip(ref[1], got[1]):
            assert torch.equal(a, b)
        for a, b in zip(ref[2], got[2]):
            assert torch.equal(a, b)
    ctx.close()


def test_noalloc_rejects_more_tiles_than_its_scratch_holds():
    import paper_2403_13135_gb300 as sil
    p = sil.params()
    img = torch.zeros((4, 4, 3), dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    tiles = sil.make_tiles([img] * 257, None, [cnt] * 257, None)
    st = sil.sil_label_batch_noalloc(tiles, 257, sil.SIL_U8, ctypes.byref(p), None)
    assert st == sil.SIL_EINVAL
    assert b"256" in sil.sil_last_error()
