"""Seeded synthetic Sentinel-2-like sea-ice scenes.

This module only draws input images; it holds none of the labeling
arithmetic and imports neither the oracle nor the CUDA library, so both
sides can be fed the same bytes.  It stands in for the paper's data
(Sec. III-A: 66 Ross Sea scenes, bands 2/3/4 at 10 m, split into 256 x 256
chips), which is not available here.

Recipe (one scene, H x W, seed s):
  * Voronoi floes: ``n_floes`` seeds uniform over the scene, one class per
    floe drawn uniformly from {thick ice, thin ice, open water}.  For scenes
    above 16 Mpx the nearest-seed map is taken on a 4x coarser grid and
    repeated (floe edges on a 4-pixel raster).
  * Pixel colour = class mean + round(N(0, 8)) per channel, clipped to
    [0, 255]; means (R, G, B): water (20, 30, 45), thin (120, 130, 140),
    thick (230, 235, 240).
  * Shadows: ``n_shadow`` ellipses, random centre and angle, semi-axes
    U[W/16, W/6]; inside, every channel v <- floor(v / 2).
  * Thin cloud: ``n_haze`` blobs, applied after the shadows; every channel
    v <- min(255, v + round(40 exp(-r^2 / (2 sigma^2)))), sigma ~ U[W/16, W/4].
  * The floe class map is returned as ground truth (codes 0 thick, 1 thin,
    2 water).
  * uint16 variant: round(v8 * 10000 / 255) per channel, plus a nodata
    wedge (all channels 0) in one corner, as at the edge of an S2 swath.

Generation is deterministic for a given seed on a given machine (numpy
PCG64).  Floating-point exp() may round differently across CPU
architectures, so nothing compares generator output against stored bytes.
"""
from __future__ import annotations

import numpy as np

CLASS_MEANS = np.array([[230, 235, 240],   # 0 thick / snow-covered ice
                        [120, 130, 140],   # 1 young / thin ice
                        [20, 30, 45]],     # 2 open water
                       dtype=np.int16)
NOISE_SIGMA = 8.0
HAZE_AMPLITUDE = 40.0


def _voronoi(rng, H, W, n_floes):
    ys = rng.uniform(0, H, n_floes)
    xs = rng.uniform(0, W, n_floes)
    cls = rng.integers(0, 3, n_floes).astype(np.uint8)
    f = 4 if H * W > 16_000_000 else 1
    hc, wc = -(-H // f), -(-W // f)
    cy = (np.arange(hc, dtype=np.float64) + 0.5) * f
    cx = (np.arange(wc, dtype=np.float64) + 0.5) * f
    try:
        from scipy.spatial import cKDTree
        tree = cKDTree(np.stack([ys, xs], 1))
        gy, gx = np.meshgrid(cy, cx, indexing="ij")
        _, idx = tree.query(np.stack([gy.ravel(), gx.ravel()], 1), workers=-1)
        idx = idx.reshape(hc, wc)
    except ImportError:  # pragma: no cover - plain numpy fallback
        idx = np.zeros((hc, wc), np.int64)
        best = np.full((hc, wc), np.inf)
        for i in range(n_floes):
            d = (cy[:, None] - ys[i]) ** 2 + (cx[None, :] - xs[i]) ** 2
            m = d < best
            best[m] = d[m]
            idx[m] = i
    truth = cls[idx]
    if f > 1:
        truth = np.repeat(np.repeat(truth, f, 0), f, 1)[:H, :W]
    return np.ascontiguousarray(truth)


def scene(H: int, W: int, seed: int, n_floes: int = 20, n_haze: int = 1,
          n_shadow: int = 1, dtype=np.uint8, chunk_rows: int = 1024):
    """Return (img[H, W, 3], truth[H, W] uint8).  dtype uint8 or uint16."""
    rng = np.random.Generator(np.random.PCG64(seed))
    truth = _voronoi(rng, H, W, max(1, n_floes))
    img = np.empty((H, W, 3), np.uint8)
    for r0 in range(0, H, chunk_rows):
        r1 = min(H, r0 + chunk_rows)
        noise = rng.standard_normal((r1 - r0, W, 3), dtype=np.float32)
        noise *= NOISE_SIGMA
        v = CLASS_MEANS[truth[r0:r1]] + np.rint(noise).astype(np.int16)
        np.clip(v, 0, 255, out=v)
        img[r0:r1] = v.astype(np.uint8)
        del noise, v

    side = float(min(H, W))
    for _ in range(n_shadow):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        a, b = rng.uniform(side / 16, side / 6, 2)
        th = rng.uniform(0, np.pi)
        r = int(np.ceil(max(a, b)))
        y0, y1 = max(0, int(cy) - r), min(H, int(cy) + r + 1)
        x0, x1 = max(0, int(cx) - r), min(W, int(cx) + r + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = np.arange(y0, y1, dtype=np.float64)[:, None] - cy
        xx = np.arange(x0, x1, dtype=np.float64)[None, :] - cx
        u = xx * np.cos(th) + yy * np.sin(th)
        w = -xx * np.sin(th) + yy * np.cos(th)
        inside = (u / a) ** 2 + (w / b) ** 2 <= 1.0
        sub = img[y0:y1, x0:x1]
        sub[inside] //= 2

    for _ in range(n_haze):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        sg = rng.uniform(side / 16, side / 4)
        r = int(np.ceil(4 * sg))
        y0, y1 = max(0, int(cy) - r), min(H, int(cy) + r + 1)
        x0, x1 = max(0, int(cx) - r), min(W, int(cx) + r + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = np.arange(y0, y1, dtype=np.float64)[:, None] - cy
        xx = np.arange(x0, x1, dtype=np.float64)[None, :] - cx
        inc = np.rint(HAZE_AMPLITUDE * np.exp(-(yy * yy + xx * xx) / (2 * sg * sg)))
        inc = inc.astype(np.int16)[:, :, None]
        sub = img[y0:y1, x0:x1].astype(np.int16) + inc
        np.minimum(sub, 255, out=sub)
        img[y0:y1, x0:x1] = sub.astype(np.uint8)

    if dtype == np.uint16:
        img16 = np.rint(img.astype(np.float32) * (10000.0 / 255.0)).astype(np.uint16)
        k = int(rng.uniform(0.1, 0.3) * (H + W))
        yy = np.arange(H)[:, None]
        xx = np.arange(W)[None, :]
        img16[(yy + xx) < k] = 0
        return img16, truth
    return img, truth


# The workloads the benchmarks and tests use, by name.
def tile_512(seed: int = 0, dtype=np.uint8):
    """512 x 512 tile: 20 floes, one thin-cloud blob, one shadow ellipse."""
    return scene(512, 512, seed, n_floes=20, n_haze=1, n_shadow=1, dtype=dtype)


def full_scene(seed: int = 1, side: int = 10980, dtype=np.uint8):
    """A full Sentinel-2 tile (10980 x 10980 at 10 m): 200 floes, 5-15 haze
    blobs and 3-8 shadow ellipses."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    n_haze = int(rng.integers(5, 16))
    n_shadow = int(rng.integers(3, 9))
    return scene(side, side, seed, n_floes=200, n_haze=n_haze, n_shadow=n_shadow,
                 dtype=dtype)


TILE_SIDES = (128, 256, 512, 1024, 2048)


def uneven_tile_shapes(n: int = 512, base_seed: int = 1000):
    """Shapes of the uneven-tile batch: side in {128 ... 2048}, the other side
    round(side * U[1, 2]), orientation random; one seed per tile."""
    out = []
    for i in range(n):
        rng = np.random.Generator(np.random.PCG64(base_seed + i))
        s = int(rng.choice(TILE_SIDES))
        o = int(round(s * rng.uniform(1.0, 2.0)))
        if rng.integers(0, 2):
            out.append((s, o, base_seed + i))
        else:
            out.append((o, s, base_seed + i))
    return out


def uneven_tile(H: int, W: int, seed: int, dtype=np.uint8):
    """One tile of the uneven batch: floes scale with area (at least 3)."""
    n_floes = max(3, int(round(200 * H * W / (10980 * 10980))))
    return scene(H, W, seed, n_floes=n_floes, n_haze=1, n_shadow=1, dtype=dtype)


def unet_layer_shapes(F: int = 32, depth: int = 4) -> dict:
    """Weight shapes of the U-Net (PyTorch layouts) for base width F: name ->
    (weight shape, kind) with kind 'conv3' (3x3, ReLU), 'up' (2x2 stride-2
    transposed) or 'head' (1x1 to 3 classes)."""
    shapes = {}
    w = [F << l for l in range(depth + 1)]
    cin = 3
    for lvl in range(depth):
        shapes[f"enc{lvl}_0"] = ((w[lvl], cin, 3, 3), "conv3")
        shapes[f"enc{lvl}_1"] = ((w[lvl], w[lvl], 3, 3), "conv3")
        cin = w[lvl]
    shapes["bott_0"] = ((w[depth], w[depth - 1], 3, 3), "conv3")
    shapes["bott_1"] = ((w[depth], w[depth], 3, 3), "conv3")
    for lvl in reversed(range(depth)):
        shapes[f"up{lvl}"] = ((w[lvl + 1], w[lvl], 2, 2), "up")
        shapes[f"dec{lvl}_0"] = ((w[lvl], 2 * w[lvl], 3, 3), "conv3")
        shapes[f"dec{lvl}_1"] = ((w[lvl], w[lvl], 3, 3), "conv3")
    shapes["head"] = ((3, F, 1, 1), "head")
    return shapes


def unet_weights(F: int = 32, depth: int = 4, seed: int = 0) -> dict:
    """Seeded random U-Net weights (random init; no trained weights exist
    here).  Every value is k * 2^-m with |k| <= 127, so it is exact in
    bfloat16: weights k ~ round(32 N(0, 1)) with 2^-m ~ std / 32 for a
    He-style std (sqrt(2 / fan_in), sqrt(1 / fan_in) without ReLU); biases
    k / 1024 with k uniform in [-8, 8].  Returns name -> (w, b) float32."""
    rng = np.random.default_rng(seed)
    out = {}
    for name, (shape, kind) in unet_layer_shapes(F, depth).items():
        if kind == "conv3":
            std = np.sqrt(2.0 / (shape[1] * 9))
        elif kind == "up":
            std = np.sqrt(1.0 / shape[0])
        else:
            std = np.sqrt(1.0 / shape[1])
        m = int(round(np.log2(32.0 / std)))
        k = np.clip(np.round(rng.standard_normal(shape) * 32.0), -127, 127)
        co = shape[1] if kind == "up" else shape[0]
        kb = rng.integers(-8, 9, size=co)
        out[name] = ((k * 2.0 ** -m).astype(np.float32), (kb / 1024.0).astype(np.float32))
    return out


def chips_from_scene(img: np.ndarray, n: int, seed: int = 0, chip: int = 256) -> np.ndarray:
    """n whole chip x chip crops of an H x W x 3 scene at random chip-grid
    positions (chips cut as the paper cuts its scenes), [n, chip, chip, 3]."""
    rng = np.random.default_rng(seed)
    gy, gx = img.shape[0] // chip, img.shape[1] // chip
    out = np.empty((n, chip, chip, img.shape[2]), dtype=img.dtype)
    for i in range(n):
        cy, cx = int(rng.integers(gy)), int(rng.integers(gx))
        out[i] = img[cy * chip:(cy + 1) * chip, cx * chip:(cx + 1) * chip]
    return out


def crop_tiles(img: np.ndarray, shapes, seed: int = 0):
    """The uneven-tile batch as crops of one scene: for each (h, w, _) of
    ``shapes`` a crop of that size (clamped to the scene) at a seeded random
    position.  Returns (tiles, boxes) with boxes[i] = (y, x, h, w); the
    tiles are contiguous copies."""
    rng = np.random.default_rng(seed)
    H, W = img.shape[:2]
    tiles, boxes = [], []
    for (h, w, _s) in shapes:
        h, w = min(h, H), min(w, W)
        y = int(rng.integers(0, H - h + 1))
        x = int(rng.integers(0, W - w + 1))
        tiles.append(np.ascontiguousarray(img[y:y + h, x:x + w]))
        boxes.append((y, x, h, w))
    return tiles, boxes


def colour_cube() -> np.ndarray:
    """Every 24-bit RGB colour once: a 4096 x 4096 x 3 uint8 image whose pixel
    i = 4096 y + x has R = i >> 16, G = (i >> 8) & 255, B = i & 255."""
    i = np.arange(1 << 24, dtype=np.uint32)
    img = np.empty((1 << 24, 3), np.uint8)
    img[:, 0] = i >> 16
    img[:, 1] = (i >> 8) & 255
    img[:, 2] = i & 255
    return img.reshape(4096, 4096, 3)
