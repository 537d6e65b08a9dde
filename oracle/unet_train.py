"""CPU oracle of the U-Net training step -- TEST INFRASTRUCTURE ONLY.

Only the tests may import this module; the product library never loads it.
Plain numpy in float64, channels-last (NHWC), one function per layer's
backward pass, written from the definitions, for the training the paper
describes in Sec. III-C "U-Net Model Training" and "Distributed U-Net Model
Training using Horovod Framework":

* loss: categorical cross-entropy of the three class scores against the
  reference label of every pixel, averaged over the pixels of the batch;
* optimizer: Adam (Kingma and Ba): m <- b1 m + (1 - b1) g,
  v <- b2 v + (1 - b2) g^2, p <- p - lr m_hat / (sqrt(v_hat) + eps) with
  m_hat = m / (1 - b1^t), v_hat = v / (1 - b2^t); the paper trained with
  TensorFlow, whose defaults are lr 1e-3, b1 0.9, b2 0.999, eps 1e-7;
* data parallelism: each worker computes the gradient of its own batch and
  the workers' gradients are averaged (ring all-reduce) before the
  optimizer step; initial weights are broadcast from rank 0.

Readings where the paper is silent: the paper's dropout layers (rates 0.1 to
0.3, positions not given) are left out, so a step is deterministic; pixels
whose reference label is 3 (masked) are left out of the loss; a 2x2 max
pool sends its gradient to the first maximum of its window in the order
(0,0), (0,1), (1,0), (1,1).

Rounding, to match a device that stores activations and activation
gradients in bfloat16: ``rb`` (default identity) is applied to every stored
activation gradient; parameter gradients are exact.
"""
from __future__ import annotations

import numpy as np

from . import unet as U

ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-7


def _ident(x):
    return x


def softmax_ce(logits: np.ndarray, labels: np.ndarray):
    """Mean cross-entropy over pixels whose label is 0..2 and its gradient
    with respect to the scores: (softmax - onehot) / count (0 elsewhere)."""
    z = np.asarray(logits, np.float64)
    lab = np.asarray(labels)
    keep = lab < 3
    zmax = z.max(axis=-1, keepdims=True)
    e = np.exp(z - zmax)
    sm = e / e.sum(axis=-1, keepdims=True)
    n = max(int(keep.sum()), 1)
    idx = np.where(keep, lab, 0).astype(np.int64)
    logp = np.log(np.take_along_axis(sm, idx[..., None], axis=-1))[..., 0]
    loss = -float((logp * keep).sum()) / n
    onehot = np.zeros_like(sm)
    np.put_along_axis(onehot, idx[..., None], 1.0, axis=-1)
    dz = (sm - onehot) * keep[..., None] / n
    return loss, dz


def head_backward(x, w, dz):
    """1x1 head: scores = x . w^T + b; returns dx, dw [3, F, 1, 1], db."""
    w2 = np.asarray(w, np.float64).reshape(w.shape[0], w.shape[1])
    dx = dz @ w2
    dw = (dz.reshape(-1, dz.shape[-1]).T @ np.asarray(x, np.float64).reshape(-1, x.shape[-1])).reshape(w.shape)
    db = dz.reshape(-1, dz.shape[-1]).sum(axis=0)
    return dx, dw, db


def relu_backward(y, dy):
    """Gradient through ReLU given its output y: dy where y > 0."""
    return np.where(np.asarray(y) > 0, dy, 0.0)


def conv3x3_backward(x, w, ds):
    """3x3 convolution, zero padding 1: s[y, x, co] = b[co] +
    sum_{dy,dx,ci} x[y+dy-1, x+dx-1, ci] w[co, ci, dy, dx].  Given ds
    (gradient at s): dx, dw [Co, Ci, 3, 3], db."""
    B, H, W, Ci = x.shape
    Co = w.shape[0]
    xp = np.zeros((B, H + 2, W + 2, Ci))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros((Co, Ci, 3, 3))
    for dy in range(3):
        for dx_ in range(3):
            win = xp[:, dy:dy + H, dx_:dx_ + W, :]
            dw[:, :, dy, dx_] = np.einsum("bhwo,bhwc->oc", ds, win)
            dxp[:, dy:dy + H, dx_:dx_ + W, :] += ds @ np.asarray(w[:, :, dy, dx_], np.float64)
    db = ds.reshape(-1, Co).sum(axis=0)
    return dxp[:, 1:H + 1, 1:W + 1, :], dw, db


def maxpool2_backward(x, dy):
    """2x2 max pool, stride 2: the gradient of each window goes to its first
    maximum in the order (0,0), (0,1), (1,0), (1,1)."""
    B, H, W, C = x.shape
    xw = x.reshape(B, H // 2, 2, W // 2, 2, C).transpose(0, 1, 3, 2, 4, 5).reshape(B, H // 2, W // 2, 4, C)
    first = np.argmax(xw, axis=3)  # numpy's argmax returns the first maximum
    dxw = np.zeros_like(xw)
    np.put_along_axis(dxw, first[:, :, :, None, :], dy[:, :, :, None, :], axis=3)
    return dxw.reshape(B, H // 2, W // 2, 2, 2, C).transpose(0, 1, 3, 2, 4, 5).reshape(B, H, W, C)


def upconv2_backward(x, w, dy):
    """2x2 stride-2 transposed convolution: y[2y+i, 2x+j, co] = b[co] +
    sum_ci x[y, x, ci] w[ci, co, i, j].  Given dy: dx, dw [Ci, Co, 2, 2], db."""
    dx = np.zeros(x.shape)
    dw = np.zeros(w.shape)
    for i in range(2):
        for j in range(2):
            g = dy[:, i::2, j::2, :]
            dx += g @ np.asarray(w[:, :, i, j], np.float64).T
            dw[:, :, i, j] = np.einsum("bhwc,bhwo->co", x, g)
    db = dy.reshape(-1, dy.shape[-1]).sum(axis=0)
    return dx, dw, db


def forward_saved(x0, weights: dict, depth: int):
    """The forward pass of oracle.unet on prepared input x0 (float64 NHWC),
    keeping every activation the backward pass reads.  Returns
    (acts dict, logits)."""
    a = {"x0": x0}
    x = x0
    for lvl in range(depth):
        x = U.conv3x3(x, *weights[f"enc{lvl}_0"]); a[f"enc{lvl}_0"] = x
        x = U.conv3x3(x, *weights[f"enc{lvl}_1"]); a[f"enc{lvl}_1"] = x
        x = U.maxpool2(x); a[f"pool{lvl}"] = x
    x = U.conv3x3(x, *weights["bott_0"]); a["bott_0"] = x
    x = U.conv3x3(x, *weights["bott_1"]); a["bott_1"] = x
    for lvl in reversed(range(depth)):
        x = U.upconv2(x, *weights[f"up{lvl}"]); a[f"up{lvl}"] = x
        x = np.concatenate([x, a[f"enc{lvl}_1"]], axis=-1); a[f"cat{lvl}"] = x
        x = U.conv3x3(x, *weights[f"dec{lvl}_0"]); a[f"dec{lvl}_0"] = x
        x = U.conv3x3(x, *weights[f"dec{lvl}_1"]); a[f"dec{lvl}_1"] = x
    hw, hb = weights["head"]
    logits = x @ np.asarray(hw, np.float64).reshape(3, -1).T + np.asarray(hb, np.float64)
    return a, logits


def backward_network(acts: dict, logits, labels, weights: dict, depth: int, rb=_ident):
    """Loss and every parameter's gradient (name -> (dw, db)) of one batch,
    from the saved activations of forward_saved.  The decoder is walked from
    the head down to the bottleneck, the encoder from the bottleneck up; the
    gradient of each encoder level's output is the sum of its skip share
    (from the decoder's concatenation) and its pooling share.  ``rb`` rounds
    each stored activation gradient (identity: exact)."""
    loss, dz = softmax_ce(logits, labels)
    grads = {}
    dx, dw, db = head_backward(acts["dec0_1"], weights["head"][0], dz)
    grads["head"] = (dw, db)
    dy = rb(dx)                      # gradient at dec0_1's output
    skip = {}
    for lvl in range(depth):         # decoder, level 0 (top) to depth - 1
        ds = relu_backward(acts[f"dec{lvl}_1"], dy)
        dx, dw, db = conv3x3_backward(acts[f"dec{lvl}_0"], weights[f"dec{lvl}_1"][0], ds)
        grads[f"dec{lvl}_1"] = (dw, db)
        dy = rb(dx)
        ds = relu_backward(acts[f"dec{lvl}_0"], dy)
        dx, dw, db = conv3x3_backward(acts[f"cat{lvl}"], weights[f"dec{lvl}_0"][0], ds)
        grads[f"dec{lvl}_0"] = (dw, db)
        dx = rb(dx)
        half = dx.shape[-1] // 2
        dup, skip[lvl] = dx[..., :half], dx[..., half:]
        up_in = acts["bott_1"] if lvl == depth - 1 else acts[f"dec{lvl + 1}_1"]
        dx, dw, db = upconv2_backward(up_in, weights[f"up{lvl}"][0], dup)
        grads[f"up{lvl}"] = (dw, db)
        dy = rb(dx)                  # gradient at up_in
    # bottleneck (dy = gradient at bott_1's output)
    ds = relu_backward(acts["bott_1"], dy)
    dx, dw, db = conv3x3_backward(acts["bott_0"], weights["bott_1"][0], ds)
    grads["bott_1"] = (dw, db)
    dy = rb(dx)
    ds = relu_backward(acts["bott_0"], dy)
    dx, dw, db = conv3x3_backward(acts[f"pool{depth - 1}"], weights["bott_0"][0], ds)
    grads["bott_0"] = (dw, db)
    dy = rb(dx)                      # gradient at pool(depth - 1)
    for lvl in reversed(range(depth)):   # encoder, deepest first
        dy = rb(maxpool2_backward(acts[f"enc{lvl}_1"], dy) + skip[lvl])
        ds = relu_backward(acts[f"enc{lvl}_1"], dy)
        dx, dw, db = conv3x3_backward(acts[f"enc{lvl}_0"], weights[f"enc{lvl}_1"][0], ds)
        grads[f"enc{lvl}_1"] = (dw, db)
        dy = rb(dx)
        ds = relu_backward(acts[f"enc{lvl}_0"], dy)
        x_in = acts["x0"] if lvl == 0 else acts[f"pool{lvl - 1}"]
        dx, dw, db = conv3x3_backward(x_in, weights[f"enc{lvl}_0"][0], ds)
        grads[f"enc{lvl}_0"] = (dw, db)
        dy = rb(dx)                  # gradient at pool(lvl - 1) (unused at level 0)
    return loss, grads


def adam_step(p, g, m, v, t: int, lr: float = 1e-3, b1: float = ADAM_B1, b2: float = ADAM_B2,
              eps: float = ADAM_EPS):
    """One Adam update (step t >= 1); returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def average_gradients(per_worker: list) -> dict:
    """Data-parallel reduction: the mean of the workers' gradients, name by
    name (what the ring all-reduce of the Horovod optimizer computes)."""
    n = len(per_worker)
    out = {}
    for k in per_worker[0]:
        out[k] = tuple(sum(g[k][i] for g in per_worker) / n for i in range(2))
    return out
