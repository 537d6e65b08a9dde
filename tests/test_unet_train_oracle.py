"""Pins of the training-step oracle (oracle/unet_train.py), CPU only: every
backward function against PyTorch's autograd in float64 on random tensors
(an independent implementation of the same derivatives), the whole
network's gradients against autograd and against finite differences, the
max pool's tie rule and Adam against its closed-form first step and
PyTorch's optimizer."""
import numpy as np
import pytest

import oracle.unet as U
import oracle.unet_train as T
import synth

torch = pytest.importorskip("torch")
F_ = torch.nn.functional


def _t(a):
    return torch.tensor(np.asarray(a, np.float64), dtype=torch.float64, requires_grad=True)


def _nchw(x):
    return x.permute(0, 3, 1, 2)


def _nhwc(x):
    return x.permute(0, 2, 3, 1)


def test_softmax_ce_against_torch():
    rng = np.random.default_rng(1)
    z = rng.normal(size=(2, 5, 7, 3))
    lab = rng.integers(0, 4, (2, 5, 7))          # code 3: masked, left out
    loss, dz = T.softmax_ce(z, lab)
    zt = _t(z)
    lt = F_.cross_entropy(zt.reshape(-1, 3), torch.tensor(lab.reshape(-1)), ignore_index=3)
    lt.backward()
    assert loss == pytest.approx(lt.item(), rel=1e-12)
    np.testing.assert_allclose(dz, zt.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_conv3x3_backward_against_torch():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 6, 5, 3))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    ds = rng.normal(size=(2, 6, 5, 4))
    dx, dw, db = T.conv3x3_backward(x, w, ds)
    xt, wt, bt = _t(x), _t(w), _t(b)
    s = _nhwc(F_.conv2d(_nchw(xt), wt, bt, padding=1))
    (s * torch.tensor(ds)).sum().backward()
    np.testing.assert_allclose(dx, xt.grad.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(dw, wt.grad.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(db, bt.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_upconv2_backward_against_torch():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 3, 4, 5))
    w = rng.normal(size=(5, 2, 2, 2))            # [Ci, Co, 2, 2]
    b = rng.normal(size=2)
    dy = rng.normal(size=(2, 6, 8, 2))
    dx, dw, db = T.upconv2_backward(x, w, dy)
    xt, wt, bt = _t(x), _t(w), _t(b)
    y = _nhwc(F_.conv_transpose2d(_nchw(xt), wt, bt, stride=2))
    (y * torch.tensor(dy)).sum().backward()
    np.testing.assert_allclose(dx, xt.grad.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(dw, wt.grad.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(db, bt.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_maxpool_backward_against_torch_and_tie_rule():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(2, 6, 8, 3))            # continuous: no ties
    dy = rng.normal(size=(2, 3, 4, 3))
    dx = T.maxpool2_backward(x, dy)
    xt = _t(x)
    y = _nhwc(F_.max_pool2d(_nchw(xt), 2))
    (y * torch.tensor(dy)).sum().backward()
    np.testing.assert_allclose(dx, xt.grad.numpy(), rtol=0, atol=0)
    # ties go to the first maximum in the order (0,0), (0,1), (1,0), (1,1)
    x = np.array([[[1.0], [1.0]], [[0.0], [1.0]]])[None]     # window [[1, 1], [0, 1]]
    dx = T.maxpool2_backward(x, np.array([[[[5.0]]]]))
    assert dx[0, :, :, 0].tolist() == [[5.0, 0.0], [0.0, 0.0]]
    x = np.array([[[0.0], [2.0]], [[2.0], [1.0]]])[None]     # first max at (0,1)
    dx = T.maxpool2_backward(x, np.array([[[[3.0]]]]))
    assert dx[0, :, :, 0].tolist() == [[0.0, 3.0], [0.0, 0.0]]


def test_head_backward_against_torch():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(2, 4, 3, 6))
    w = rng.normal(size=(3, 6, 1, 1))
    b = rng.normal(size=3)
    dz = rng.normal(size=(2, 4, 3, 3))
    dx, dw, db = T.head_backward(x, w, dz)
    xt, wt, bt = _t(x), _t(w), _t(b)
    z = _nhwc(F_.conv2d(_nchw(xt), wt, bt))
    (z * torch.tensor(dz)).sum().backward()
    np.testing.assert_allclose(dx, xt.grad.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(dw, wt.grad.numpy(), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(db, bt.grad.numpy(), rtol=1e-10, atol=1e-12)


def _exact(monkeypatch):
    """The oracle's forward without bfloat16 rounding (exact derivatives)."""
    monkeypatch.setattr(U, "bf16", lambda v: np.asarray(v, np.float64))


def _torch_unet_loss(x0, wts, depth, lab):
    """The same network built from PyTorch ops (float64)."""
    P = {k: (_t(w), _t(b)) for k, (w, b) in wts.items()}
    x = _nchw(torch.tensor(x0))
    skips = []
    for lvl in range(depth):
        for j in (0, 1):
            w, b = P[f"enc{lvl}_{j}"]
            x = F_.relu(F_.conv2d(x, w, b, padding=1))
        skips.append(x)
        x = F_.max_pool2d(x, 2)
    for j in (0, 1):
        w, b = P[f"bott_{j}"]
        x = F_.relu(F_.conv2d(x, w, b, padding=1))
    for lvl in reversed(range(depth)):
        w, b = P[f"up{lvl}"]
        x = F_.conv_transpose2d(x, w, b, stride=2)
        x = torch.cat([x, skips[lvl]], dim=1)
        for j in (0, 1):
            w, b = P[f"dec{lvl}_{j}"]
            x = F_.relu(F_.conv2d(x, w, b, padding=1))
    w, b = P["head"]
    z = _nhwc(F_.conv2d(x, w, b))
    loss = F_.cross_entropy(z.reshape(-1, 3), torch.tensor(lab.reshape(-1)), ignore_index=3)
    return loss, P


def _small_net(seed):
    F, depth = 4, 2
    wts = synth.unet_weights(F, depth, seed=seed)
    rng = np.random.default_rng(seed)
    x0 = rng.random((2, 16, 16, 3))
    lab = rng.integers(0, 4, (2, 16, 16))
    return F, depth, wts, x0, lab


def test_network_gradients_against_torch_autograd(monkeypatch):
    _exact(monkeypatch)
    F, depth, wts, x0, lab = _small_net(7)
    acts, logits = T.forward_saved(x0, wts, depth)
    loss, grads = T.backward_network(acts, logits, lab, wts, depth)
    lt, P = _torch_unet_loss(x0, wts, depth, lab)
    lt.backward()
    assert loss == pytest.approx(lt.item(), rel=1e-10)
    assert set(grads) == set(P)
    for k, (w, b) in P.items():
        np.testing.assert_allclose(grads[k][0], w.grad.numpy(), rtol=1e-8, atol=1e-12, err_msg=k)
        np.testing.assert_allclose(grads[k][1], b.grad.numpy(), rtol=1e-8, atol=1e-12, err_msg=k)


def test_network_gradients_against_finite_differences(monkeypatch):
    _exact(monkeypatch)
    F, depth, wts, x0, lab = _small_net(8)
    acts, logits = T.forward_saved(x0, wts, depth)
    _, grads = T.backward_network(acts, logits, lab, wts, depth)
    rng = np.random.default_rng(9)
    h = 1e-6
    for name in ("enc0_0", "enc1_1", "bott_0", "up1", "dec0_0", "head"):
        w, b = wts[name]
        for _ in range(3):
            idx = tuple(int(rng.integers(0, s)) for s in w.shape)
            wp = {k: (v[0].astype(np.float64).copy(), v[1].astype(np.float64).copy()) for k, v in wts.items()}
            wm = {k: (v[0].astype(np.float64).copy(), v[1].astype(np.float64).copy()) for k, v in wts.items()}
            wp[name][0][idx] += h
            wm[name][0][idx] -= h
            lp = T.softmax_ce(T.forward_saved(x0, wp, depth)[1], lab)[0]
            lm = T.softmax_ce(T.forward_saved(x0, wm, depth)[1], lab)[0]
            fd = (lp - lm) / (2 * h)
            assert grads[name][0][idx] == pytest.approx(fd, rel=1e-4, abs=1e-8), (name, idx)


def test_adam_first_step_closed_form_and_torch():
    rng = np.random.default_rng(10)
    p0 = rng.normal(size=20)
    g = rng.normal(size=20)
    lr = 1e-3
    p1, m, v = T.adam_step(p0, g, np.zeros(20), np.zeros(20), 1, lr)
    # m_hat = g, v_hat = g^2 on the first step
    np.testing.assert_allclose(p1, p0 - lr * g / (np.abs(g) + T.ADAM_EPS), rtol=1e-12)
    # five steps against PyTorch's Adam
    pt = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=lr, betas=(T.ADAM_B1, T.ADAM_B2), eps=T.ADAM_EPS)
    p, m, v = p0.copy(), np.zeros(20), np.zeros(20)
    for t in range(1, 6):
        gt = rng.normal(size=20)
        opt.zero_grad()
        pt.grad = torch.tensor(gt)
        opt.step()
        p, m, v = T.adam_step(p, gt, m, v, t, lr)
    np.testing.assert_allclose(p, pt.detach().numpy(), rtol=1e-12, atol=1e-15)


def test_average_gradients_is_the_mean():
    a = {"x": (np.array([1.0, 2.0]), np.array([3.0]))}
    b = {"x": (np.array([3.0, 6.0]), np.array([5.0]))}
    avg = T.average_gradients([a, b])
    assert avg["x"][0].tolist() == [2.0, 4.0] and avg["x"][1].tolist() == [4.0]
