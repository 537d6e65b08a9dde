"""The batched entry point that allocates nothing (sil_label_batch_noalloc),
for callers that may not allocate device memory: through the C ABI, two
calls in a row, each checked bit for bit against sil_label_batch (the entry
point that keeps its scratch in a context), for every kernel instance it
can take (8-bit, 16-bit, narrowed H/S ranges, chips above the resident
size) and at its 256-tile limit.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HS_PARAMS = {"lo": [[0, 0, 180], [40, 60, 31], [0, 0, 0]],
             "hi": [[185, 40, 255], [100, 200, 204], [185, 255, 40]]}


def _batch(shapes, seed, dtype=np.uint8):
    imgs = [synth.scene(h, w, seed + i, n_floes=4, dtype=dtype)[0] for i, (h, w) in enumerate(shapes)]
    # uint16 images travel as int16 tensors (same bytes)
    dev = [torch.from_numpy(im.view(np.int16) if im.dtype == np.uint16 else im).cuda() for im in imgs]
    return imgs, dev


def _outputs(imgs, chip):
    labs = [torch.full(im.shape[:2], 7, dtype=torch.uint8, device="cuda") for im in imgs]
    cnts = [torch.full((4,), -1, dtype=torch.int64, device="cuda") for _ in imgs]
    ccs = [torch.full((-(-im.shape[0] // chip), -(-im.shape[1] // chip), 4), -1, dtype=torch.int32,
                      device="cuda") for im in imgs]
    return labs, cnts, ccs


CASES = {
    "u8": (np.uint8, {}, [[(300, 517), (256, 256), (64, 1000), (1, 1), (513, 40)],
                          [(1000, 700), (17, 33), (256, 700)]]),
    "u16": (np.uint16, {}, [[(300, 270), (150, 170), (2, 9)], [(513, 257), (40, 50)]]),
    "hs_ranges": (np.uint8, HS_PARAMS, [[(200, 230), (64, 64)], [(300, 100), (7, 500)]]),
    "chip512": (np.uint8, {"chip": 512}, [[(530, 610), (600, 300)], [(1100, 40)]]),
    "256_tiles": (np.uint8, {"chip": 16}, [[(20 + i % 7, 30 + i % 11) for i in range(256)],
                                          [(9 + i % 5, 12 + i % 3) for i in range(256)]]),
}


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_matches_context_batch_twice(case):
    import paper_2403_13135_gb300 as sil
    dtype, pd, shape_lists = CASES[case]
    p = sil.params(**pd)
    dt = sil.SIL_U8 if dtype == np.uint8 else sil.SIL_U16
    ctx = sil.Context()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for k, shapes in enumerate(shape_lists):  # two calls in a row, different batches
        imgs, dev = _batch(shapes, 900 + 50 * k, dtype)
        ref = _outputs(imgs, p.chip)
        got = _outputs(imgs, p.chip)
        t_ref = sil.make_tiles(dev, *ref)
        t_got = sil.make_tiles(dev, *got)
        sil.check(sil.sil_label_batch(t_ref, len(imgs), dt, ctypes.byref(p), ctx.handle, stream))
        st = sil.sil_label_batch_noalloc(t_got, len(imgs), dt, ctypes.byref(p), stream)
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


def test_noalloc_refuses_a_capturing_stream():
    """Its descriptors are copied from the call's stack, which a recorded copy
    would read after the call returned: while the stream is being captured
    the call returns SIL_EINVAL and enqueues nothing; afterwards it works."""
    import paper_2403_13135_gb300 as sil
    p = sil.params()
    img = torch.from_numpy(synth.scene(40, 50, 3)[0]).cuda()
    cnt = torch.full((4,), -1, dtype=torch.int64, device="cuda")
    tiles = sil.make_tiles([img], None, [cnt], None)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            st = sil.sil_label_batch_noalloc(tiles, 1, sil.SIL_U8, ctypes.byref(p),
                                             ctypes.c_void_p(s.cuda_stream))
            msg = sil.sil_last_error()
            # something for the graph to hold
            cnt.add_(0)
        finally:
            g.capture_end()
    assert st == sil.SIL_EINVAL
    assert b"captur" in msg
    st = sil.sil_label_batch_noalloc(tiles, 1, sil.SIL_U8, ctypes.byref(p), None)
    assert st == sil.SIL_OK, sil.sil_last_error()
    torch.cuda.synchronize()
    assert int(cnt.sum()) == 40 * 50
