"""CPU oracle of the U-Net inference on filtered chips -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module; the product library never loads it.

Plain numpy in float64, channels-last (NHWC), one function per layer type,
following the encoder-decoder of Sec. III-C "U-Net Model Inferencing"
(256 x 256 chips, as the paper splits its scenes) and Sec. III-C "U-Net
Model Training" (a U-Net).  The paper fixes neither the widths nor the
precision, so the readings are:

* input: the chip's R, G, B bytes scaled by 1/256 (exact in bfloat16); the
  filtered input (Sec. III-C feeds the filtered image to the U-Net) first
  scales each pixel's R, G, B by V'/V, V = max(R, G, B) and V' the filter's
  corrected value (HSV with V replaced, H and S kept), rounded half up to an
  integer: c' = floor((2 c V' + V) / (2 V)), 0 when V = 0;
* encoder: 4 levels of two 3x3 convolutions (zero padding 1, bias, ReLU)
  followed by 2x2 max pooling; widths F, 2F, 4F, 8F; a bottleneck of two
  3x3 convolutions of width 16F;
* decoder: per level a 2x2 stride-2 transposed convolution (bias, no
  activation) halving the width, concatenation [upsampled, skip] along the
  channels, two 3x3 convolutions (bias, ReLU);
* head: 1x1 convolution to 3 class scores (thick ice, thin ice, open
  water), kept in float32; label = index of the largest score (the first on
  ties);
* every stored activation is rounded to bfloat16 (round to nearest, ties to
  even), the storage format of the GPU path; sums are exact (float64).

Weights use PyTorch layouts: conv [Co, Ci, kh, kw], transposed conv
[Ci, Co, 2, 2], head [3, F, 1, 1]; biases [Co].
"""
from __future__ import annotations

import numpy as np

N_CLASSES = 3


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 value (8 significant bits, ties to even),
    returned as float64.  x = m 2^e with 0.5 <= |m| < 1, so m 2^8 rounded to
    an integer (half to even) keeps 8 significant bits."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def prep(chips_u8: np.ndarray) -> np.ndarray:
    """[B, 256, 256, 3] uint8 -> [B, 256, 256, 3] float64 activations v / 256."""
    return np.asarray(chips_u8, dtype=np.float64) / 256.0


def prep_filtered(chips_u8: np.ndarray, vprime_u8: np.ndarray) -> np.ndarray:
    """[B, 256, 256, 3] uint8 chips and their [B, 256, 256] V' -> the filtered
    chips' activations c' / 256, c' = floor((2 c V' + V) / (2 V)) (0 if V = 0)."""
    c = np.asarray(chips_u8, dtype=np.int64)
    v = c.max(axis=-1, keepdims=True)
    vp = np.asarray(vprime_u8, dtype=np.int64)[..., None]
    cf = np.where(v > 0, (2 * c * vp + v) // np.maximum(2 * v, 1), 0)
    return cf.astype(np.float64) / 256.0


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray, relu: bool = True) -> np.ndarray:
    """3x3 convolution with zero padding 1: out[.., y, x, co] =
    b[co] + sum_{dy,dx,ci} in[.., y+dy-1, x+dx-1, ci] w[co, ci, dy, dx];
    then ReLU and bfloat16 rounding."""
    B, H, W, Ci = x.shape
    Co = w.shape[0]
    assert w.shape == (Co, Ci, 3, 3)
    xp = np.zeros((B, H + 2, W + 2, Ci))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    out = np.zeros((B, H, W, Co))
    for dy in range(3):
        for dx in range(3):
            out += xp[:, dy:dy + H, dx:dx + W, :] @ np.asarray(w[:, :, dy, dx], np.float64).T
    out += np.asarray(b, np.float64)
    if relu:
        out = np.maximum(out, 0.0)
    return bf16(out)


def maxpool2(x: np.ndarray) -> np.ndarray:
    """2x2 max pooling, stride 2 (H and W even)."""
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).max(axis=(2, 4))


def upconv2(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """2x2 stride-2 transposed convolution: out[.., 2y+i, 2x+j, co] =
    b[co] + sum_ci in[.., y, x, ci] w[ci, co, i, j]; bfloat16 rounding."""
    B, H, W, Ci = x.shape
    Co = w.shape[1]
    assert w.shape == (Ci, Co, 2, 2)
    out = np.zeros((B, 2 * H, 2 * W, Co))
    for i in range(2):
        for j in range(2):
            out[:, i::2, j::2, :] = x @ np.asarray(w[:, :, i, j], np.float64)
    out += np.asarray(b, np.float64)
    return bf16(out)


def head(x: np.ndarray, w: np.ndarray, b: np.ndarray):
    """1x1 convolution to class scores (float32) and the label (first max)."""
    Co, Ci = w.shape[0], w.shape[1]
    logits = (x @ np.asarray(w.reshape(Co, Ci), np.float64).T + np.asarray(b, np.float64))
    logits = logits.astype(np.float32)
    return logits, np.argmax(logits, axis=-1).astype(np.uint8)


def forward(chips_u8: np.ndarray, weights: dict, depth: int = 4, vprime_u8=None):
    """The whole network on [B, 256, 256, 3] uint8 chips (filtered by their
    [B, 256, 256] V' when vprime_u8 is given).
    weights: 'enc{l}_{0,1}' / 'bott_{0,1}' / 'dec{l}_{0,1}' conv (w, b),
    'up{l}' transposed conv (w, b), 'head' (w, b).
    Returns (logits [B, H, W, 3] float32, labels [B, H, W] uint8)."""
    x = prep(chips_u8) if vprime_u8 is None else prep_filtered(chips_u8, vprime_u8)
    skips = []
    for lvl in range(depth):
        x = conv3x3(x, *weights[f"enc{lvl}_0"])
        x = conv3x3(x, *weights[f"enc{lvl}_1"])
        skips.append(x)
        x = maxpool2(x)
    x = conv3x3(x, *weights["bott_0"])
    x = conv3x3(x, *weights["bott_1"])
    for lvl in reversed(range(depth)):
        x = upconv2(x, *weights[f"up{lvl}"])
        x = np.concatenate([x, skips[lvl]], axis=-1)
        x = conv3x3(x, *weights[f"dec{lvl}_0"])
        x = conv3x3(x, *weights[f"dec{lvl}_1"])
    return head(x, *weights["head"])
