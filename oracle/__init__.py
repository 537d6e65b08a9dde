"""CPU oracle of the sea-ice auto-labeling path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library never loads it, and it never loads the product library.

The arithmetic lives in ``sil_oracle.c`` (plain single-threaded C, integer
only, one function per step of the method, each citing its passage of the
paper).  This module compiles it with gcc and wraps it with ctypes; it adds
no arithmetic of its own.

Functions
---------
params_default()            -> dict of parameters (paper defaults)
hsv(r, g, b)                -> (h, s, v), Sec. III-B HSV convention
u16_to_u8(v, scale)         -> int, 8-bit value of a uint16 reflectance
median3x3(V)                -> 3x3 median of a 2-D uint8 array, clamped border
otsu(hist, fallback)        -> Otsu threshold of a 256-bin histogram
stretch(v, lo, hi)          -> min-max normalised value
label(img, params, ...)     -> (labels, counts, chip_counts, chip_stats)
filtered_value(img, params) -> V' plane (the filter's corrected value)
confusion(pred, ref, chip)  -> (conf[4][4], chip_conf[gy][gx][4][4])
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sil_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libsil_oracle.so")
_lock = threading.Lock()
_lib = None


class OracleParams(ctypes.Structure):
    """Mirror of ``sil_oracle_params`` in sil_oracle.c."""

    _fields_ = [
        ("lo", (ctypes.c_uint8 * 3) * 3),
        ("hi", (ctypes.c_uint8 * 3) * 3),
        ("filter", ctypes.c_int32),
        ("chip", ctypes.c_int32),
        ("median", ctypes.c_int32),
        ("mm_min_range", ctypes.c_int32),
        ("mm_min_frac_den", ctypes.c_int32),
        ("v_trunc", ctypes.c_int32),
        ("max_shift", ctypes.c_int32),
        ("bgr", ctypes.c_int32),
        ("u16_scale", ctypes.c_int32),
    ]


class ChipStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("n", "lo", "hi", "t", "n0", "n1", "gate")]


_SCALAR_FIELDS = ("filter", "chip", "median", "mm_min_range", "mm_min_frac_den",
                  "v_trunc", "max_shift", "bgr", "u16_scale")


def build(force: bool = False) -> str:
    """Compile sil_oracle.c into libsil_oracle.so next to it (gcc, -O2)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared",
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    lib.sil_oracle_params_default.argtypes = [ctypes.POINTER(OracleParams)]
    lib.sil_oracle_params_check.argtypes = [ctypes.POINTER(OracleParams)]
    lib.sil_oracle_u16_to_u8.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.sil_oracle_hsv.argtypes = [ctypes.c_int] * 3 + [ctypes.POINTER(ctypes.c_int)] * 3
    lib.sil_oracle_hsv.restype = None
    lib.sil_oracle_median3x3.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    lib.sil_oracle_median3x3.restype = None
    lib.sil_oracle_otsu.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.sil_oracle_stretch.argtypes = [ctypes.c_int] * 3
    lib.sil_oracle_label.argtypes = [
        ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
        ctypes.POINTER(OracleParams), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
        ctypes.c_void_p, ctypes.c_void_p]
    lib.sil_oracle_label_v.argtypes = [
        ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
        ctypes.POINTER(OracleParams), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
        ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.sil_oracle_label_v.restype = ctypes.c_int
    lib.sil_oracle_confusion.argtypes = [
        ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
        ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    _lib = lib
    return lib


def params_default() -> dict:
    """Parameters with the paper's class ranges and the filter defaults."""
    lib = _load()
    p = OracleParams()
    lib.sil_oracle_params_default(ctypes.byref(p))
    return _to_dict(p)


def _to_dict(p: OracleParams) -> dict:
    d = {"lo": [[p.lo[k][c] for c in range(3)] for k in range(3)],
         "hi": [[p.hi[k][c] for c in range(3)] for k in range(3)]}
    for f in _SCALAR_FIELDS:
        d[f] = getattr(p, f)
    return d


def _from_dict(d: dict) -> OracleParams:
    merged = params_default()
    merged.update(d or {})
    p = OracleParams()
    for k in range(3):
        for c in range(3):
            p.lo[k][c] = int(merged["lo"][k][c])
            p.hi[k][c] = int(merged["hi"][k][c])
    for f in _SCALAR_FIELDS:
        setattr(p, f, int(merged[f]))
    return p


def params_valid(d: dict) -> bool:
    return _load().sil_oracle_params_check(ctypes.byref(_from_dict(d))) == 0


def hsv(r: int, g: int, b: int):
    lib = _load()
    h, s, v = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    lib.sil_oracle_hsv(int(r), int(g), int(b), ctypes.byref(h), ctypes.byref(s), ctypes.byref(v))
    return h.value, s.value, v.value


def u16_to_u8(v: int, scale: int = 10000) -> int:
    return _load().sil_oracle_u16_to_u8(int(v), int(scale))


def median3x3(V: np.ndarray) -> np.ndarray:
    V = np.ascontiguousarray(V, dtype=np.uint8)
    assert V.ndim == 2
    out = np.empty_like(V)
    _load().sil_oracle_median3x3(V.ctypes.data, V.shape[0], V.shape[1], out.ctypes.data)
    return out


def otsu(hist, fallback: int) -> int:
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    assert h.shape == (256,)
    return _load().sil_oracle_otsu(h.ctypes.data, int(fallback))


def stretch(v: int, lo: int, hi: int) -> int:
    return _load().sil_oracle_stretch(int(v), int(lo), int(hi))


def label(img: np.ndarray, params: dict | None = None, *, pitch: int | None = None,
          H: int | None = None, W: int | None = None, want_labels: bool = True):
    """Run the oracle on an H x W x 3 uint8 or uint16 image.

    ``img`` may also be a 1-D uint8 buffer with explicit ``pitch``/``H``/``W``
    (bytes per row; the dtype is then taken from ``params['_dtype']``).
    Returns (labels[H, W] uint8 or None, counts[4] uint64,
    chip_counts[gy, gx, 4] uint32, stats list of dicts).
    """
    lib = _load()
    p = _from_dict(params)
    if img.ndim == 3:
        H, W = img.shape[0], img.shape[1]
        assert img.shape[2] == 3
        dtype = 0 if img.dtype == np.uint8 else 1
        assert img.dtype in (np.uint8, np.uint16)
        buf = np.ascontiguousarray(img)
        pitch = buf.strides[0]
    else:
        assert pitch is not None and H is not None and W is not None
        dtype = int((params or {}).get("_dtype", 0))
        buf = np.ascontiguousarray(img, dtype=np.uint8)
    C = p.chip
    gy, gx = -(-H // C), -(-W // C)
    labels = np.empty((H, W), np.uint8) if want_labels else None
    counts = np.zeros(4, np.uint64)
    chip_counts = np.zeros((gy, gx, 4), np.uint32)
    stats = (ChipStats * (gy * gx))()
    rc = lib.sil_oracle_label(buf.ctypes.data, H, W, pitch, dtype, ctypes.byref(p),
                              labels.ctypes.data if want_labels else None, W,
                              counts.ctypes.data, chip_counts.ctypes.data, stats)
    if rc != 0:
        raise ValueError("sil_oracle_label: invalid arguments")
    st = [{f: getattr(s, f) for f in ("n", "lo", "hi", "t", "n0", "n1", "gate")} for s in stats]
    return labels, counts, chip_counts, st


def filtered_value(img: np.ndarray, params: dict | None = None) -> np.ndarray:
    """The filter's corrected value V' of every pixel of an H x W x 3 uint8 or
    uint16 image (the value the class ranges are applied to: V after the
    median, the gated min-max stretch and the truncation; V itself when the
    filter is off; 0 for nodata), H x W uint8."""
    lib = _load()
    p = _from_dict(params)
    assert img.ndim == 3 and img.shape[2] == 3 and img.dtype in (np.uint8, np.uint16)
    H, W = img.shape[0], img.shape[1]
    buf = np.ascontiguousarray(img)
    vp = np.empty((H, W), np.uint8)
    counts = np.zeros(4, np.uint64)
    rc = lib.sil_oracle_label_v(buf.ctypes.data, H, W, buf.strides[0], 0 if img.dtype == np.uint8 else 1,
                                ctypes.byref(p), None, W, vp.ctypes.data, W, counts.ctypes.data,
                                None, None)
    if rc != 0:
        raise ValueError("sil_oracle_label_v: invalid arguments")
    return vp


def confusion(pred: np.ndarray, ref: np.ndarray, chip: int = 256):
    """Confusion counts conf[pred][ref] (4 x 4) and per-chip copies."""
    lib = _load()
    pred = np.ascontiguousarray(pred, dtype=np.uint8)
    ref = np.ascontiguousarray(ref, dtype=np.uint8)
    assert pred.shape == ref.shape and pred.ndim == 2
    H, W = pred.shape
    gy, gx = -(-H // chip), -(-W // chip)
    conf = np.zeros(16, np.uint64)
    chip_conf = np.zeros((gy, gx, 16), np.uint32)
    rc = lib.sil_oracle_confusion(pred.ctypes.data, W, ref.ctypes.data, W, H, W, chip,
                                  conf.ctypes.data, chip_conf.ctypes.data)
    if rc != 0:
        raise ValueError("sil_oracle_confusion: invalid arguments")
    return conf.reshape(4, 4), chip_conf.reshape(gy, gx, 4, 4)
