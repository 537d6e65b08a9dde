"""U-Net inference on the GPU (tcgen05 implicit-GEMM convolutions) against
the float64 oracle of oracle/unet.py on seeded chips and weights.

Bounds, from the arithmetic: both sides round every stored activation to
bfloat16 (8 significant bits); the GPU sums bf16 x bf16 products in float32,
the oracle exactly.  Each layer is checked in isolation on the GPU's own
input of that layer: an output may then differ from the oracle's by one
bfloat16 ulp (the two sums straddle a rounding boundary) plus the float32
summation error bound, element by element.  The end-to-end scores, where
differences compound over the layers, are compared by relative L2; labels
where the oracle's best score beats the second by more than the score
difference bound (elsewhere either label is a correct argmax of scores
within rounding)."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import oracle.unet as U  # noqa: E402
import synth  # noqa: E402


@pytest.fixture(scope="module")
def sil():
    import paper_2403_13135_gb300 as m
    return m


def _chips(n, seed):
    img, _ = synth.scene(1024, 1024, seed, n_floes=12, n_haze=2, n_shadow=2)
    return synth.chips_from_scene(img, n, seed)


def _oracle_chain(chips, wts, depth):
    """Every layer's output activation of the oracle, in the library's order."""
    x = U.prep(chips)
    outs, skips = [], []
    for lvl in range(depth):
        x = U.conv3x3(x, *wts[f"enc{lvl}_0"]); outs.append(x)
        x = U.conv3x3(x, *wts[f"enc{lvl}_1"]); outs.append(x)
        skips.append(x)
        x = U.maxpool2(x)
    x = U.conv3x3(x, *wts["bott_0"]); outs.append(x)
    x = U.conv3x3(x, *wts["bott_1"]); outs.append(x)
    for lvl in reversed(range(depth)):
        x = U.upconv2(x, *wts[f"up{lvl}"]); outs.append(x)
        x = np.concatenate([x, skips[lvl]], axis=-1)
        x = U.conv3x3(x, *wts[f"dec{lvl}_0"]); outs.append(x)
        x = U.conv3x3(x, *wts[f"dec{lvl}_1"]); outs.append(x)
    logits, labels = U.head(x, *wts["head"])
    return outs, logits, labels


def _run(sil, F, depth, chips, wts, max_batch=None):
    cfg = sil.unet_config(F, depth, max_batch or len(chips))
    net = sil.UNet(cfg, list(wts.values()))
    dev = torch.from_numpy(chips).cuda()
    lab = torch.empty(chips.shape[:3], dtype=torch.uint8, device="cuda")
    lg = torch.empty(chips.shape[:3] + (3,), dtype=torch.float32, device="cuda")
    net.forward(dev, lab, lg)
    torch.cuda.synchronize()
    return net, lab.cpu().numpy(), lg.cpu().numpy()


def _ulp_bf16(v):
    m, e = np.frexp(np.abs(v))
    return np.ldexp(1.0, e - 8)


def _layer_names(depth):
    names = []
    for lvl in range(depth):
        names += [f"enc{lvl}_0", f"enc{lvl}_1"]
    names += ["bott_0", "bott_1"]
    for lvl in reversed(range(depth)):
        names += [f"up{lvl}", f"dec{lvl}_0", f"dec{lvl}_1"]
    return names + ["head"]


def _abs_conv3x3(x, w, b):
    """sum of |terms| of each 3x3 convolution output: |x| * |w| + |b|."""
    B, H, W, Ci = x.shape
    xp = np.zeros((B, H + 2, W + 2, Ci))
    xp[:, 1:H + 1, 1:W + 1, :] = np.abs(x)
    out = np.zeros((B, H, W, w.shape[0])) + np.abs(b)
    for dy in range(3):
        for dx in range(3):
            out += xp[:, dy:dy + H, dx:dx + W, :] @ np.abs(np.asarray(w[:, :, dy, dx], np.float64)).T
    return out


def _abs_upconv2(x, w, b):
    B, H, W, Ci = x.shape
    out = np.zeros((B, 2 * H, 2 * W, w.shape[1]))
    for i in range(2):
        for j in range(2):
            out[:, i::2, j::2, :] = np.abs(x) @ np.abs(np.asarray(w[:, :, i, j], np.float64))
    return out + np.abs(b)


@pytest.mark.parametrize("F,depth,n", [(16, 2, 2), (32, 4, 1), (16, 5, 3), (32, 5, 1), (64, 5, 1),
                                       (64, 3, 1)])
def test_unet_each_layer_against_oracle(sil, F, depth, n):
    """Every layer in isolation: the oracle's layer i applied to the GPU's own
    input of that layer (its layer i-1 output, max-pooled or concatenated
    with the skip as the network does) must agree with the GPU's output
    element by element.  The GPU sums bf16 x bf16 products in float32, the
    oracle exactly, and both round the result to bf16: the two agree within
    one bf16 ulp of the oracle's value, plus twice the float32 summation
    error bound (K + 2) 2^-24 sum|terms| (K terms per output), which only
    matters where the sum cancels.  Depth 5 is the paper's network (28
    convolution layers); its 8 x 8 bottleneck maps are tiled two chips at a
    time, and n = 3 leaves the last such tile half empty."""
    chips = _chips(n, 11 + F + depth)
    wts = synth.unet_weights(F, depth, seed=F + depth)
    net, lab, lg = _run(sil, F, depth, chips, wts)
    assert net.error_count() == 0
    names = _layer_names(depth)
    assert len(names) == sil._lib.sil_unet_num_layers(depth) == 5 * depth + 3
    gpu = {}
    for i, nm in enumerate(names[:-1]):
        gpu[nm] = net.tensor(i).float().cpu().numpy().astype(np.float64)
    x0 = net.tensor(-1).float().cpu().numpy()
    assert np.array_equal(x0[..., :3], U.prep(chips)) and not x0[..., 3:].any()
    exact_frac = []
    for i, nm in enumerate(names[:-1]):
        w, b = wts[nm]
        if nm == "enc0_0":
            x = U.prep(chips)
        elif nm.startswith("enc") and nm.endswith("_0"):
            x = U.maxpool2(gpu[f"enc{int(nm[3:-2]) - 1}_1"])
        elif nm.endswith("_1"):
            x = gpu[nm[:-1] + "0"]
        elif nm == "bott_0":
            x = U.maxpool2(gpu[f"enc{depth - 1}_1"])
        elif nm.startswith("up"):
            lvl = int(nm[2:])
            x = gpu["bott_1"] if lvl == depth - 1 else gpu[f"dec{lvl + 1}_1"]
        else:  # dec l_0: [upsampled, skip]
            lvl = int(nm[3:-2])
            x = np.concatenate([gpu[f"up{lvl}"], gpu[f"enc{lvl}_1"]], axis=-1)
        if nm.startswith("up"):
            ref, S, K = U.upconv2(x, w, b), _abs_upconv2(x, w, b), x.shape[-1]
        else:
            ref, S, K = U.conv3x3(x, w, b), _abs_conv3x3(x, w, b), 9 * x.shape[-1]
        g = gpu[nm]
        assert g.shape == ref.shape, (nm, g.shape, ref.shape)
        bound = _ulp_bf16(ref) + 2.0 * (K + 2) * 2.0 ** -24 * S
        d = np.abs(g - ref)
        bad = d > bound
        assert not bad.any(), (nm, int(bad.sum()), float(d.max()))
        exact_frac.append(float(np.mean(d == 0)))
    assert min(exact_frac) > 0.8, exact_frac
    # the head (float32 scores) on the GPU's own last activation
    hw, hb = wts["head"]
    ref_lg, _ = U.head(gpu["dec0_1"], hw, hb)
    S = np.abs(gpu["dec0_1"]) @ np.abs(hw.reshape(3, -1).astype(np.float64)).T + np.abs(hb)
    hb_bound = (F + 2) * 2.0 ** -24 * S + np.abs(ref_lg.astype(np.float64)) * 2.0 ** -23
    assert np.all(np.abs(lg.astype(np.float64) - ref_lg.astype(np.float64)) <= hb_bound)
    # labels: the argmax of those scores wherever the top two are apart by
    # more than the score bound
    srt = np.sort(ref_lg.astype(np.float64), axis=-1)
    clear = (srt[..., -1] - srt[..., -2]) > 2 * hb_bound.max(axis=-1)
    assert clear.mean() > 0.9
    assert np.array_equal(lab[clear], np.argmax(ref_lg, axis=-1)[clear])


@pytest.mark.parametrize("F,depth,n", [(16, 2, 2), (32, 5, 1)])
def test_unet_chain_against_oracle(sil, F, depth, n):
    """The whole network, GPU against the oracle run end to end on the same
    chips (differences compound over the layers): scores within 3e-2
    relative L2, labels equal where the oracle's top score clears the second
    by twice the largest score difference."""
    chips = _chips(n, 5 + F)
    wts = synth.unet_weights(F, depth, seed=F)
    net, lab, lg = _run(sil, F, depth, chips, wts)
    outs, ref_lg, ref_lab = _oracle_chain(chips, wts, depth)
    rel = np.linalg.norm(lg - ref_lg) / np.linalg.norm(ref_lg)
    assert rel < 3e-2, rel
    bound = np.abs(lg - ref_lg).max()
    srt = np.sort(ref_lg, axis=-1)
    clear = (srt[..., -1] - srt[..., -2]) > 2 * bound
    assert clear.mean() > 0.5
    assert np.array_equal(lab[clear], ref_lab[clear])
    assert net.error_count() == 0


def test_unet_batch_independent(sil):
    """A chip's scores do not depend on the batch it is in (bit-exact)."""
    F, depth = 16, 3
    chips = _chips(5, 3)
    wts = synth.unet_weights(F, depth, seed=7)
    net5, lab5, lg5 = _run(sil, F, depth, chips, wts)
    net1, lab1, lg1 = _run(sil, F, depth, chips[2:3], wts, max_batch=8)
    assert np.array_equal(lg5[2:3], lg1) and np.array_equal(lab5[2:3], lab1)
    assert net5.error_count() == 0 and net1.error_count() == 0


def test_unet_rejects_bad_arguments(sil):
    cfg = sil.unet_config(32, 4, 2)
    wts = list(synth.unet_weights(32, 4, 0).values())
    with pytest.raises(sil.SilError):
        sil.UNet(sil.unet_config(32, 6, 2), list(synth.unet_weights(32, 6, 0).values()))
    net = sil.UNet(cfg, wts)
    dev = torch.zeros((3, 256, 256, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(sil.SilError):
        net.forward(dev)                 # 3 > max_batch
    with pytest.raises(sil.SilError):
        sil.UNet(sil.unet_config(24, 4, 2), wts)  # width not in {16, 32, 64}
    with pytest.raises(ValueError):
        sil.UNet(cfg, wts[:-1])


def test_unet_bounded_wait_runs_out_and_recovers(sil):
    """Failure detection without a GPU fault: the test hook leaves one stage's
    input load out, so that layer's wait for it runs out (bounded, about
    1.3 s); the kernel counts the error and returns, and the next forward on
    the same network and context gives the same scores as before, bit for
    bit."""
    F, depth = 16, 2
    chips = _chips(2, 21)
    wts = synth.unet_weights(F, depth, seed=3)
    net, lab0, lg0 = _run(sil, F, depth, chips, wts)
    assert net.error_count() == 0
    shapes = sil.unet_layer_shapes(net.cfg)
    # the first layer with 32 input channels reads by tensor map
    layer = next(i for i, (s, k) in enumerate(shapes) if k == sil.UNET_CONV3 and s[1] == 32)
    with pytest.raises(sil.SilError):
        net.set_fault(0)                 # the first layer gathers: no hook there
    net.set_fault(layer)
    dev = torch.from_numpy(chips).cuda()
    lab = torch.empty(chips.shape[:3], dtype=torch.uint8, device="cuda")
    lg = torch.empty(chips.shape[:3] + (3,), dtype=torch.float32, device="cuda")
    net.forward(dev, lab, lg)
    errors = net.error_count()           # synchronises
    assert errors > 0
    net.set_fault(-1)
    net.forward(dev, lab, lg)
    torch.cuda.synchronize()
    assert net.error_count() == errors   # no new errors
    assert np.array_equal(lg.cpu().numpy(), lg0) and np.array_equal(lab.cpu().numpy(), lab0)


def test_unet_on_filtered_chips(sil):
    """The paper's inferencing workflow: the scene is labelled with the
    filter's V' kept (sil_label_v), chips are cut with their V', and the
    U-Net runs on the filtered chips.  V' bit-exact against the oracle on the
    same chips, the filtered input exact, the scores within the bf16 bound."""
    img, _ = synth.scene(768, 512, 41, n_floes=10, n_haze=3, n_shadow=2)
    dev = torch.from_numpy(img).cuda()
    _, vp, _ = sil.label_v(dev, None, labels=False)
    torch.cuda.synchronize()
    vp = vp.cpu().numpy()
    pos = [(0, 0), (1, 1), (2, 0)]
    chips = np.stack([img[256 * y:256 * y + 256, 256 * x:256 * x + 256] for y, x in pos])
    vps = np.stack([vp[256 * y:256 * y + 256, 256 * x:256 * x + 256] for y, x in pos])
    # V' of a chip depends on that chip alone: the oracle on each chip
    ovps = np.stack([oracle.filtered_value(np.ascontiguousarray(c)) for c in chips])
    assert np.array_equal(vps, ovps)
    F, depth = 16, 2
    wts = synth.unet_weights(F, depth, seed=5)
    net = sil.UNet(sil.unet_config(F, depth, len(chips)), list(wts.values()))
    lg = torch.empty(chips.shape[:3] + (3,), dtype=torch.float32, device="cuda")
    net.forward(torch.from_numpy(chips).cuda(), None, lg, vprime=torch.from_numpy(vps).cuda())
    torch.cuda.synchronize()
    x0 = net.tensor(-1).float().cpu().numpy()
    assert np.array_equal(x0[..., :3], U.prep_filtered(chips, ovps)) and not x0[..., 3:].any()
    ref, _ = U.forward(chips, wts, depth=depth, vprime_u8=ovps)
    got = lg.cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 3e-2
    assert net.error_count() == 0


def test_unet_label_scene_matches_chips(sil):
    """sil_unet_label_scene: the scene's chip grid (zero past the edges) with
    its V', max_batch chips at a time, labels written back -- equal, bit for
    bit, to cutting the same chips by hand and running them one batch each."""
    img, _ = synth.scene(700, 530, 43, n_floes=9, n_haze=2, n_shadow=2)
    H, W, _ = img.shape
    dev = torch.from_numpy(img).cuda()
    _, vp, _ = sil.label_v(dev, None, labels=False)
    F, depth = 16, 2
    wts = synth.unet_weights(F, depth, seed=6)
    net = sil.UNet(sil.unet_config(F, depth, 4), list(wts.values()))   # 9 chips: batches 4, 4, 1
    lab = net.label_scene(dev, vprime=vp)
    torch.cuda.synchronize()
    assert net.error_count() == 0
    vp_h = vp.cpu().numpy()
    gy, gx = -(-H // 256), -(-W // 256)
    chips = np.zeros((gy * gx, 256, 256, 3), np.uint8)
    vps = np.zeros((gy * gx, 256, 256), np.uint8)
    for k in range(gy * gx):
        cy, cx = divmod(k, gx)
        part = img[cy * 256:cy * 256 + 256, cx * 256:cx * 256 + 256]
        chips[k, :part.shape[0], :part.shape[1]] = part
        vps[k, :part.shape[0], :part.shape[1]] = vp_h[cy * 256:cy * 256 + 256, cx * 256:cx * 256 + 256]
    want = np.zeros((gy * 256, gx * 256), np.uint8)
    for k0 in range(0, gy * gx, 4):
        c = torch.from_numpy(chips[k0:k0 + 4]).cuda()
        lb = torch.empty(c.shape[:3], dtype=torch.uint8, device="cuda")
        net.forward(c, lb, vprime=torch.from_numpy(vps[k0:k0 + 4]).cuda())
        torch.cuda.synchronize()
        for i, l in enumerate(lb.cpu().numpy()):
            cy, cx = divmod(k0 + i, gx)
            want[cy * 256:cy * 256 + 256, cx * 256:cx * 256 + 256] = l
    assert np.array_equal(lab.cpu().numpy(), want[:H, :W])
