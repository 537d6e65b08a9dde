"""Batched (persistent kernel + CUDA graph) and served (continuous batching)
labelling: results identical to single-request labelling and the oracle,
alone and in a mix."""
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


def _tiles(n, seed=0, sides=(17, 64, 128, 200, 256, 300, 513)):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        H = int(rng.choice(sides))
        W = int(rng.integers(1, 2 * H))
        img, _ = synth.scene(H, W, 5000 + i, n_floes=4)
        out.append(img)
    return out


def _run_batch(sil, ctx, imgs, p=None, dt=None):
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    C = sil._as_params(p).chip
    labs = [torch.full(im.shape[:2], 255, dtype=torch.uint8, device="cuda") for im in imgs]
    cnts = [torch.empty(4, dtype=torch.int64, device="cuda") for _ in imgs]
    ccs = [torch.empty((-(-im.shape[0] // C), -(-im.shape[1] // C), 4), dtype=torch.int32, device="cuda")
           for im in imgs]
    tiles = sil.make_tiles(dev, labs, cnts, ccs)
    sil.label_batch(ctx, tiles, len(imgs), sil.SIL_U8 if dt is None else dt, p)
    torch.cuda.synchronize()
    return [l.cpu().numpy() for l in labs], [c.cpu().numpy() for c in cnts], [c.cpu().numpy() for c in ccs]


def test_batch_matches_single_and_oracle(sil):
    imgs = _tiles(24)
    ctx = sil.Context()
    labs, cnts, ccs = _run_batch(sil, ctx, imgs)
    for im, l, c, cc in zip(imgs, labs, cnts, ccs):
        ol, oc, occ, _ = oracle.label(im)
        assert int((l != ol).sum()) == 0
        np.testing.assert_array_equal(c.astype(np.uint64), oc)
        np.testing.assert_array_equal(cc.astype(np.uint32), occ)
    ctx.close()


def test_batch_graph_replay_and_autotune(sil):
    imgs = _tiles(12, seed=1)
    ctx = sil.Context()
    a = _run_batch(sil, ctx, imgs)
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    labs = [torch.empty(im.shape[:2], dtype=torch.uint8, device="cuda") for im in imgs]
    cnts = [torch.empty(4, dtype=torch.int64, device="cuda") for _ in imgs]
    tiles = sil.make_tiles(dev, labs, cnts, None)
    best = sil.autotune(ctx, tiles, len(imgs))
    assert best["schedule"] in (sil.SCHED_STRIDE, sil.SCHED_QUEUE, sil.SCHED_PER_CHIP)
    assert best["threads"] in (256, 320) and best["us"] > 0
    # the last candidate the tuner ran (fixed-stride persistent CTAs of 320
    # threads) left its outputs in the buffers: they equal the default's
    torch.cuda.synchronize()
    for i in range(len(imgs)):
        assert np.array_equal(labs[i].cpu().numpy(), a[0][i])
        assert np.array_equal(cnts[i].cpu().numpy(), a[1][i])
    assert sil.batch_tuning(ctx, tiles, len(imgs)) == (best, True)
    for _ in range(3):  # the same batch replays its cached graph
        sil.label_batch(ctx, tiles, len(imgs))
    torch.cuda.synchronize()
    for i in range(len(imgs)):
        assert np.array_equal(labs[i].cpu().numpy(), a[0][i])
        assert np.array_equal(cnts[i].cpu().numpy(), a[1][i])
    ctx.close()


def test_autotune_cache_persists_by_batch_class(sil, tmp_path, monkeypatch):
    """The tuned schedule is saved under the batch's class and a new context
    loads it; a batch of another class stays untuned."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("SIL_AUTOTUNE_CACHE", str(cache))
    imgs = _tiles(8, seed=4)
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    labs = [torch.empty(im.shape[:2], dtype=torch.uint8, device="cuda") for im in imgs]
    cnts = [torch.empty(4, dtype=torch.int64, device="cuda") for _ in imgs]
    tiles = sil.make_tiles(dev, labs, cnts, None)
    ctx = sil.Context()
    assert sil.batch_tuning(ctx, tiles, len(imgs))[1] is False
    best = sil.autotune(ctx, tiles, len(imgs))
    ctx.close()
    lines = cache.read_text().splitlines()
    assert len(lines) == 1
    key, sched, _ctas, threads, _us = lines[0].split()
    assert (int(sched), int(threads)) == (best["schedule"], best["threads"])
    assert key.startswith(torch.cuda.get_device_name(0).replace(" ", "_"))
    ctx2 = sil.Context()
    got, tuned = sil.batch_tuning(ctx2, tiles, len(imgs))
    assert tuned and (got["schedule"], got["threads"]) == (best["schedule"], best["threads"])
    # one tile of 4096 x 4096: another class (tile and chip counts)
    big = torch.zeros((4096, 4096, 3), dtype=torch.uint8, device="cuda")
    cb = torch.empty(4, dtype=torch.int64, device="cuda")
    t2 = sil.make_tiles([big], None, [cb], None)
    assert sil.batch_tuning(ctx2, t2, 1)[1] is False
    sil.label_batch(ctx2, t2, 1)
    torch.cuda.synchronize()
    assert int(cb[2]) == 4096 * 4096  # black: all open water
    ctx2.close()


def test_batch_other_variants(sil):
    imgs = _tiles(6, seed=2)
    ctx = sil.Context()
    for p in ({"chip": 64}, {"chip": 300}, {"lo": [[0, 0, 180], [40, 60, 31], [0, 0, 0]],
                                            "hi": [[185, 40, 255], [100, 200, 204], [185, 255, 40]]}):
        labs, cnts, ccs = _run_batch(sil, ctx, imgs, p)
        for im, l, c in zip(imgs, labs, cnts):
            ol, oc, _, _ = oracle.label(im, p)
            assert int((l != ol).sum()) == 0, p
            np.testing.assert_array_equal(c.astype(np.uint64), oc)
    imgs16 = [synth.scene(150, 170, 77 + i, n_floes=3, dtype=np.uint16)[0] for i in range(3)]
    labs, cnts, ccs = _run_batch(sil, ctx, imgs16, None, sil.SIL_U16)
    for im, l, c in zip(imgs16, labs, cnts):
        ol, oc, _, _ = oracle.label(im)
        assert int((l != ol).sum()) == 0
        np.testing.assert_array_equal(c.astype(np.uint64), oc)
    ctx.close()


def test_server_alone_equals_mix_and_oracle(sil):
    imgs = _tiles(20, seed=3)
    # alone: one request at a time
    alone = []
    with sil.Server(max_inflight=8) as srv:
        for im in imgs:
            lab = np.empty(im.shape[:2], np.uint8)
            cc = np.zeros((-(-im.shape[0] // 256), -(-im.shape[1] // 256), 4), np.uint32)
            rid = srv.submit(im, lab, cc)
            r = srv.wait(rid, 60000)
            assert r["status"] == sil.SIL_OK
            alone.append((lab, r["counts"], cc))
    # in the mix: everything submitted at once, small memory budget so that
    # admission waits for earlier requests to finish
    budget = 3 * max(im.nbytes for im in imgs)
    with sil.Server(max_inflight=6, mem_budget=budget, max_batch=4) as srv:
        ids, outs = [], []
        for im in imgs:
            lab = np.empty(im.shape[:2], np.uint8)
            cc = np.zeros((-(-im.shape[0] // 256), -(-im.shape[1] // 256), 4), np.uint32)
            ids.append(srv.submit(im, lab, cc))
            outs.append((lab, cc))
        res = [srv.wait(i, 60000) for i in ids]
    for im, (lab, cc), r, (alab, acnt, acc) in zip(imgs, outs, res, alone):
        assert r["status"] == sil.SIL_OK
        assert np.array_equal(lab, alab)
        assert r["counts"] == acnt
        assert np.array_equal(cc, acc)
        ol, oc, occ, _ = oracle.label(im)
        assert np.array_equal(lab, ol)
        assert r["counts"] == [int(x) for x in oc]
        assert r["t_submit_ms"] <= r["t_admit_ms"] <= r["t_done_ms"]


def test_server_ring_takes_requests_while_running(sil):
    """Requests submitted back to back are published to the device ring and
    taken up by the running persistent kernel: far fewer kernel launches than
    requests, every result equal to the oracle's."""
    imgs = _tiles(40, seed=6)
    with sil.Server(max_inflight=64, idle_timeout_us=200000) as srv:
        outs = []
        for im in imgs:
            lab = np.empty(im.shape[:2], np.uint8)
            outs.append((srv.submit(im, lab), lab))
        res = [(srv.wait(i, 60000), lab) for i, lab in outs]
        st = srv.stats()
    assert st["kernel_launches"] < len(imgs) // 2, st
    assert st["chips_published"] == sum(-(-im.shape[0] // 256) * -(-im.shape[1] // 256) for im in imgs)
    for im, (r, lab) in zip(imgs, res):
        assert r["status"] == sil.SIL_OK
        ol, oc, _, _ = oracle.label(im)
        assert np.array_equal(lab, ol) and r["counts"] == [int(x) for x in oc]


def test_server_ring_ready_wait_runs_out(sil):
    """Failure detection without a GPU fault: the test hook publishes a
    request without its ready word, so the kernel's bounded wait for it runs
    out (ready_timeout_ms) and it ends with SIL_ETIMEOUT; the requests before
    and after it, and later ones on the same server, are labelled correctly."""
    import time
    imgs = _tiles(4, seed=7)
    with sil.Server(max_inflight=8, ready_timeout_ms=300) as srv:
        la = np.empty(imgs[0].shape[:2], np.uint8)
        ra = srv.wait(srv.submit(imgs[0], la), 60000)
        srv.set_fault(True)
        t0 = time.monotonic()
        rb_id = srv.submit(imgs[1], np.empty(imgs[1].shape[:2], np.uint8))
        lc = np.empty(imgs[2].shape[:2], np.uint8)
        rc_id = srv.submit(imgs[2], lc)
        rb = srv.wait(rb_id, 60000)
        tb = time.monotonic() - t0
        rc = srv.wait(rc_id, 60000)
        ld = np.empty(imgs[3].shape[:2], np.uint8)
        rd = srv.wait(srv.submit(imgs[3], ld), 60000)
    assert rb["status"] == sil.SIL_ETIMEOUT
    assert 0.3 <= tb < 30, tb
    for im, r, lab in ((imgs[0], ra, la), (imgs[2], rc, lc), (imgs[3], rd, ld)):
        assert r["status"] == sil.SIL_OK
        ol, oc, _, _ = oracle.label(im)
        assert np.array_equal(lab, ol) and r["counts"] == [int(x) for x in oc]


def test_server_faults_are_reported(sil):
    """Host-side failures: a request that can never fit the memory budget,
    an invalid request, cancelling a queued request, a wait that runs out,
    an unknown id.  Nothing here faults or stalls the GPU."""
    img, _ = synth.scene(2000, 2000, 9, n_floes=5)
    with sil.Server(max_inflight=1, mem_budget=2 * img.nbytes + (1 << 20)) as srv:
        with pytest.raises(sil.SilError) as e:
            srv.submit(np.zeros((3000, 3000, 3), np.uint8))  # never fits the budget
        assert e.value.status == sil.SIL_EBUSY
        with pytest.raises(sil.SilError) as e:
            srv.submit(np.zeros((0, 5, 3), np.uint8))       # empty image
        assert e.value.status == sil.SIL_EINVAL
        ids = [srv.submit(img) for _ in range(5)]
        # one slot: the last request is still queued -> it can be cancelled
        assert srv.cancel(ids[-1]) == sil.SIL_OK
        # the fourth has not run yet either: a zero-length wait runs out
        with pytest.raises(sil.SilError) as e:
            srv.wait(ids[-2], 0)
        assert e.value.status == sil.SIL_ETIMEOUT
        for i in ids[:-1]:
            assert srv.wait(i, 60000)["status"] == sil.SIL_OK
        assert srv.wait(ids[-1], 60000)["status"] == sil.SIL_ECANCELED
        assert srv.poll(123456789)["status"] == sil.SIL_EINVAL
        # requests still queued when the server is closed are cancelled
        for _ in range(3):
            srv.submit(img)
