"""U-Net training step on the GPU (Sec. III-C "U-Net Model Training" and
"Distributed U-Net Model Training using Horovod Framework") against the
float64 training oracle of oracle/unet_train.py.

Every step of the backward pass is checked in isolation on the GPU's own
inputs of that step (its stored activations and the activation gradient it
received), so that a wrong index, sign or transposed operand in any one
kernel fails here:

* weight and bias gradients (f32 sums of bf16 products over the P pixels
  of the batch) against the exact sums, within 8 sqrt(P) 2^-24 of the sum
  of the absolute terms (the probabilistic bound of float32 summation);
* each activation gradient the GPU stores in bf16 against the exact
  gradient rounded to bf16: at most one bf16 ulp apart (the two values can
  straddle a rounding boundary) plus 1e-5 of the sum of absolute terms.

The whole chain is then compared with the oracle's backward pass on the
same activations (differences compound over the layers: relative L2), and
Adam, the re-packing of the updated weights, the decrease of the loss and
the equivalence of averaged per-worker gradients with the full-batch
gradient are checked."""
import numpy as np
import pytest

import oracle.unet as U
import oracle.unet_train as T
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sil():
    import paper_2403_13135_gb300 as m
    return m


def _names(depth):
    names = []
    for lvl in range(depth):
        names += [f"enc{lvl}_0", f"enc{lvl}_1"]
    names += ["bott_0", "bott_1"]
    for lvl in reversed(range(depth)):
        names += [f"up{lvl}", f"dec{lvl}_0", f"dec{lvl}_1"]
    return names + ["head"]


def _f64(t):
    return t.float().cpu().numpy().astype(np.float64)


def _ulp(v):
    _, e = np.frexp(np.abs(v))
    return np.ldexp(1.0, e - 8)


def _batch(sil, n, seed, masked=True):
    img, _ = synth.scene(1024, 1024, seed, n_floes=12, n_haze=2, n_shadow=2)
    chips = synth.chips_from_scene(img, n, seed)
    dev = torch.from_numpy(chips).cuda()
    lab = torch.stack([sil.label(dev[i])[0] for i in range(n)])  # the labeler's auto-labels
    if not masked:
        lab = torch.where(lab == 3, torch.full_like(lab, 2), lab)
    return chips, dev, lab.contiguous()


class Run:
    """One backward pass and everything the checks read back."""

    def __init__(self, sil, F, depth, n, seed):
        self.F, self.depth, self.n = F, depth, n
        self.wts = synth.unet_weights(F, depth, seed=seed)
        self.names = _names(depth)
        self.idx = {k: i for i, k in enumerate(self.names)}
        cfg = sil.unet_config(F, depth, n)
        self.tr = sil.Trainer(cfg, list(self.wts.values()))
        self.chips, self.dev, self.lab_dev = _batch(sil, n, seed)
        self.grads, self.loss = self.tr.backward(self.dev, self.lab_dev)
        lg = torch.empty((n, 256, 256, 3), dtype=torch.float32, device="cuda")
        self.tr.net.forward(self.dev, logits=lg)      # the same scores the step used
        torch.cuda.synchronize()
        self.logits = lg.cpu().numpy().astype(np.float64)
        self.labels = self.lab_dev.cpu().numpy()
        self.g = self.tr.unflatten(self.grads)        # [(dw, db)] per layer
        self.act = {k: _f64(self.tr.net.tensor(i)) for i, k in enumerate(self.names[:-1])}
        self.act["x0"] = _f64(self.tr.net.tensor(-1))[..., :3]
        self.sil = sil

    def dsl(self, name):
        return _f64(self.tr.grad_tensor(self.sil.UNET_GRAD_LAYER, self.idx[name]))

    def gcat(self, lvl):
        return _f64(self.tr.grad_tensor(self.sil.UNET_GRAD_CAT, lvl))

    def gpool(self, lvl):
        return _f64(self.tr.grad_tensor(self.sil.UNET_GRAD_POOL, lvl))

    def input_of(self, name):
        D = self.depth
        if name.startswith("enc"):
            lvl, j = int(name[3]), int(name[5])
            if j == 1:
                return self.act[f"enc{lvl}_0"]
            return self.act["x0"] if lvl == 0 else U.maxpool2(self.act[f"enc{lvl - 1}_1"])
        if name == "bott_0":
            return U.maxpool2(self.act[f"enc{D - 1}_1"])
        if name == "bott_1":
            return self.act["bott_0"]
        if name.startswith("up"):
            lvl = int(name[2])
            return self.act["bott_1"] if lvl == D - 1 else self.act[f"dec{lvl + 1}_1"]
        lvl, j = int(name[3]), int(name[5])
        if j == 1:
            return self.act[f"dec{lvl}_0"]
        return np.concatenate([self.act[f"up{lvl}"], self.act[f"enc{lvl}_1"]], axis=-1)


def _check_param(got, want, bound, what, terms):
    err = np.abs(got - want)
    tol = 8.0 * np.sqrt(terms) * 2.0 ** -24 * bound + 1e-30
    bad = err > tol
    assert not bad.any(), f"{what}: {bad.sum()} of {bad.size} beyond the bound, worst {err.max():.3g}"


def _check_bf16(got, exact, bound, what):
    err = np.abs(got - U.bf16(exact))
    tol = _ulp(exact) + 1e-5 * bound
    bad = err > tol
    assert not bad.any(), f"{what}: {bad.sum()} of {bad.size} beyond one ulp, worst {err.max():.3g}"


def _conv_step(r, name, ds, target, mask):
    """Weight / bias gradient and the dgrad of 3x3 layer `name` from the
    GPU's ds; target: the GPU's stored gradient at the layer's input."""
    w = U.bf16(r.wts[name][0])
    x = r.input_of(name)
    dx, dw, db = T.conv3x3_backward(x, w, ds)
    adx, adw, adb = T.conv3x3_backward(np.abs(x), np.abs(w), np.abs(ds))
    gw, gb = r.g[r.idx[name]]
    _check_param(gw, dw, adw, name + " dw", ds[..., 0].size)
    _check_param(gb, db, adb, name + " db", ds[..., 0].size)
    if target is None:
        return
    if mask is not None:
        dx = np.where(mask > 0, dx, 0.0)
    _check_bf16(target, dx, adx, name + " dx")


@pytest.fixture(scope="module", params=[(16, 2, 2), (16, 5, 1), (32, 3, 2)],
                ids=["F16-d2-n2", "F16-d5-n1", "F32-d3-n2"])
def run(sil, request):
    F, depth, n = request.param
    return Run(sil, F, depth, n, seed=40 + depth)


def test_loss_and_head(run):
    loss, dz = T.softmax_ce(run.logits, run.labels)
    assert float(run.loss.item()) == pytest.approx(loss, rel=2e-5)
    hw, _ = run.wts["head"]
    y = run.act["dec0_1"]
    dx, dw, db = T.head_backward(y, hw, dz)
    adx, adw, adb = T.head_backward(np.abs(y), np.abs(hw), np.abs(dz))
    gw, gb = run.g[run.idx["head"]]
    _check_param(gw, dw, adw, "head dw", dz[..., 0].size)
    _check_param(gb, db, adb, "head db", dz[..., 0].size)
    _check_bf16(run.dsl("dec0_1"), np.where(y > 0, dx, 0.0), adx, "head dx")


def test_decoder_steps(run):
    D = run.depth
    for lvl in range(D):
        _conv_step(run, f"dec{lvl}_1", run.dsl(f"dec{lvl}_1"), run.dsl(f"dec{lvl}_0"),
                   run.act[f"dec{lvl}_0"])
        _conv_step(run, f"dec{lvl}_0", run.dsl(f"dec{lvl}_0"), run.gcat(lvl), None)
        # the transposed convolution's gradient is the first half of the
        # concatenation's
        gc = run.gcat(lvl)
        half = gc.shape[-1] // 2
        dup = run.dsl(f"up{lvl}")
        assert np.array_equal(dup, gc[..., :half])
        name = f"up{lvl}"
        w = U.bf16(run.wts[name][0])
        x = run.input_of(name)
        dx, dw, db = T.upconv2_backward(x, w, dup)
        adx, adw, adb = T.upconv2_backward(np.abs(x), np.abs(w), np.abs(dup))
        gw, gb = run.g[run.idx[name]]
        _check_param(gw, dw, adw, name + " dw", x[..., 0].size)
        _check_param(gb, db, adb, name + " db", x[..., 0].size)
        below = "bott_1" if lvl == D - 1 else f"dec{lvl + 1}_1"
        _check_bf16(run.dsl(below), np.where(x > 0, dx, 0.0), adx, name + " dx")


def test_bottleneck_and_encoder_steps(run):
    D = run.depth
    _conv_step(run, "bott_1", run.dsl("bott_1"), run.dsl("bott_0"), run.act["bott_0"])
    _conv_step(run, "bott_0", run.dsl("bott_0"), run.gpool(D - 1), None)
    for lvl in reversed(range(D)):
        # pooling share (first maximum of each window) + skip share, masked
        y = run.act[f"enc{lvl}_1"]
        gc = run.gcat(lvl)
        g = T.maxpool2_backward(y, run.gpool(lvl)) + gc[..., gc.shape[-1] // 2:]
        _check_bf16(run.dsl(f"enc{lvl}_1"), np.where(y > 0, g, 0.0), np.abs(g), f"pool{lvl} bwd")
        _conv_step(run, f"enc{lvl}_1", run.dsl(f"enc{lvl}_1"), run.dsl(f"enc{lvl}_0"),
                   run.act[f"enc{lvl}_0"])
        _conv_step(run, f"enc{lvl}_0", run.dsl(f"enc{lvl}_0"),
                   run.gpool(lvl - 1) if lvl else None, None)


def test_whole_chain_against_oracle(run):
    """The oracle's backward pass on the GPU's activations, with every
    stored activation gradient rounded to bf16: every parameter gradient
    within 1e-2 relative L2 (rounding differences compound over the
    layers)."""
    D = run.depth
    acts = dict(run.act)
    for lvl in range(D):
        acts[f"pool{lvl}"] = U.maxpool2(acts[f"enc{lvl}_1"])
        acts[f"cat{lvl}"] = np.concatenate([acts[f"up{lvl}"], acts[f"enc{lvl}_1"]], axis=-1)
    wts = {k: (U.bf16(w) if k != "head" else w.astype(np.float64), b) for k, (w, b) in run.wts.items()}
    loss, grads = T.backward_network(acts, run.logits, run.labels, wts, D, rb=U.bf16)
    assert float(run.loss.item()) == pytest.approx(loss, rel=2e-5)
    for k, (dw, db) in grads.items():
        gw, gb = run.g[run.idx[k]]
        for got, want, what in ((gw, dw, "w"), (gb, db, "b")):
            rel = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-30)
            assert rel < 1e-2, (k, what, rel)


def test_adam_steps_and_repacked_weights(sil, run):
    """Two Adam steps against the oracle's update on the same gradients;
    the network's next forward pass uses the updated weights rounded to
    bf16: scores identical to a network created from them."""
    tr = sil.Trainer(sil.unet_config(run.F, run.depth, run.n), list(run.wts.values()))
    p = tr.params().cpu().numpy().astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t in (1, 2):
        grads, _ = tr.backward(run.dev, run.lab_dev)
        g = grads.cpu().numpy().astype(np.float64)
        tr.adam(grads, lr=1e-3)
        p, m, v = T.adam_step(p, g, m, v, t, 1e-3)
        got = tr.params().cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(got, p, rtol=1e-6, atol=1e-8)
        p = got
    fresh = sil.UNet(sil.unet_config(run.F, run.depth, run.n), tr.unflatten(tr.params()))
    a = torch.empty((run.n, 256, 256, 3), dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    tr.net.forward(run.dev, logits=a)
    fresh.forward(run.dev, logits=b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_set_params_restarts(sil, run):
    tr = sil.Trainer(sil.unet_config(run.F, run.depth, run.n), list(run.wts.values()))
    p0 = tr.params()
    grads, _ = tr.backward(run.dev, run.lab_dev)
    tr.adam(grads)
    assert not torch.equal(tr.params(), p0)
    tr.set_params(p0)
    assert torch.equal(tr.params(), p0) and tr.t == 0
    g2, _ = tr.backward(run.dev, run.lab_dev)
    assert torch.equal(g2, grads)    # same weights, same batch: same gradient


def test_loss_decreases_on_auto_labels(sil):
    """The paper's workflow: the labeler's auto-labels train the U-Net."""
    wts = synth.unet_weights(16, 3, seed=5)
    tr = sil.Trainer(sil.unet_config(16, 3, 4), list(wts.values()))
    _, dev, lab = _batch(sil, 4, 6)
    losses = []
    for _ in range(40):
        losses.append(float(tr.step(dev, lab, lr=2e-3).item()))
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.7 * losses[0], losses


def test_averaged_worker_gradients_equal_the_full_batch(sil):
    """Data parallelism as the paper's Horovod training does it: with every
    pixel labelled, the mean of two workers' gradients (one chip each) is the
    gradient of the two-chip batch."""
    wts = synth.unet_weights(16, 2, seed=9)
    tr = sil.Trainer(sil.unet_config(16, 2, 2), list(wts.values()))
    _, dev, lab = _batch(sil, 2, 10, masked=False)
    full, lf = tr.backward(dev, lab)
    full = full.clone()
    a, la = tr.backward(dev[:1].contiguous(), lab[:1].contiguous())
    a = a.clone()
    b, lb = tr.backward(dev[1:].contiguous(), lab[1:].contiguous())
    avg = (a + b) / 2
    scale = full.abs().max()
    assert torch.allclose(avg, full, rtol=1e-3, atol=1e-4 * float(scale))
    assert float(lf.item()) == pytest.approx((float(la.item()) + float(lb.item())) / 2, rel=1e-5)


def test_trainer_rejects_bad_arguments(sil):
    wts = synth.unet_weights(16, 1, seed=1)
    tr = sil.Trainer(sil.unet_config(16, 1, 1), list(wts.values()))
    chips = torch.zeros((2, 256, 256, 3), dtype=torch.uint8, device="cuda")
    lab = torch.zeros((2, 256, 256), dtype=torch.uint8, device="cuda")
    with pytest.raises(sil.SilError):
        tr.backward(chips, lab)                      # n above max_batch
    g = torch.zeros(tr.num_params, device="cuda")
    with pytest.raises(sil.SilError):
        tr.adam(g, lr=1e-3, t=0)
    with pytest.raises(sil.SilError):
        tr.grad_tensor(sil.UNET_GRAD_LAYER, 0)       # no backward pass yet
    tr.backward(chips[:1], lab[:1])
    with pytest.raises(sil.SilError):
        tr.grad_tensor(sil.UNET_GRAD_LAYER, len(tr.shapes) - 1)   # the head keeps none
    with pytest.raises(sil.SilError):
        tr.grad_tensor(sil.UNET_GRAD_CAT, 1)         # depth 1: level 0 only
