"""Python binding of libsil, the GB300 sea-ice auto-labeler.

Argument marshalling only: every step of the labelling runs in the CUDA
kernels of ``libsil.so`` behind the C ABI declared in ``include/sil.h``.
PyTorch supplies device memory and streams.  Importing this package loads
``libsil.so`` and raises ``ImportError`` if it is missing -- there is no CPU
fallback.

Same names as the C ABI (``sil_label``, ``sil_label_batch``, ...) taking
integer pointers; plus helpers (``label``, ``label_host``, ``label_batch``,
``Server``) that take torch tensors / numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsil.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libsil.so not built ({LIB_PATH}); run python paper_2403_13135_gb300/build.py")
_lib = ctypes.CDLL(LIB_PATH)

SIL_OK, SIL_EINVAL, SIL_ENOMEM, SIL_ECUDA, SIL_ETIMEOUT, SIL_EBUSY, SIL_ECANCELED = range(7)
SIL_U8, SIL_U16 = 0, 1
THICK, THIN, WATER, MASKED = 0, 1, 2, 3


class SilError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.sil_status_string(status).decode()} ({status}): {msg}")
        self.status = status


class sil_params(ctypes.Structure):
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


class sil_tile(ctypes.Structure):
    _fields_ = [
        ("img", ctypes.c_void_p),
        ("H", ctypes.c_int64), ("W", ctypes.c_int64), ("pitch_bytes", ctypes.c_int64),
        ("labels", ctypes.c_void_p), ("label_pitch", ctypes.c_int64),
        ("counts", ctypes.c_void_p), ("chip_counts", ctypes.c_void_p),
    ]


class sil_tuning(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("us", ctypes.c_float)]


SCHED_STRIDE, SCHED_QUEUE, SCHED_PER_CHIP = 0, 1, 2


class sil_metrics(ctypes.Structure):
    _fields_ = [("accuracy", ctypes.c_double), ("precision", ctypes.c_double * 3),
                ("recall", ctypes.c_double * 3), ("f1", ctypes.c_double * 3),
                ("macro_precision", ctypes.c_double), ("macro_recall", ctypes.c_double),
                ("macro_f1", ctypes.c_double), ("weighted_precision", ctypes.c_double),
                ("weighted_recall", ctypes.c_double), ("weighted_f1", ctypes.c_double),
                ("matrix", (ctypes.c_double * 4) * 4), ("support", ctypes.c_uint64 * 3)]


class sil_server_config(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
        ("device_mem_budget", ctypes.c_int64), ("max_batch", ctypes.c_int32),
        ("want_labels", ctypes.c_int32), ("ready_timeout_ms", ctypes.c_int32),
        ("idle_timeout_us", ctypes.c_int32),
    ]


class sil_request_result(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_int64), ("status", ctypes.c_int32),
        ("counts", ctypes.c_uint64 * 4),
        ("t_submit_ms", ctypes.c_double), ("t_admit_ms", ctypes.c_double),
        ("t_done_ms", ctypes.c_double),
    ]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_SIGS = {
    "sil_params_default": ([ctypes.POINTER(sil_params)], _I32),
    "sil_params_validate": ([ctypes.POINTER(sil_params)], _I32),
    "sil_status_string": ([_I32], ctypes.c_char_p),
    "sil_last_error": ([], ctypes.c_char_p),
    "sil_version": ([], ctypes.c_int),
    "sil_label": ([_P, _I64, _I64, _I64, _I32, ctypes.POINTER(sil_params), _P, _I64, _P, _P, _P], _I32),
    "sil_label_host": ([_P, _I64, _I64, _I64, _I32, ctypes.POINTER(sil_params), _P, _I64, _P, _P, _P], _I32),
    "sil_label_v": ([_P, _I64, _I64, _I64, _I32, ctypes.POINTER(sil_params), _P, _I64, _P, _I64, _P, _P,
                     _P], _I32),
    "sil_ctx_create": ([ctypes.POINTER(_P), _I32], _I32),
    "sil_ctx_destroy": ([_P], None),
    "sil_label_batch": ([ctypes.POINTER(sil_tile), _I32, _I32, ctypes.POINTER(sil_params), _P, _P], _I32),
    "sil_autotune": ([ctypes.POINTER(sil_tile), _I32, _I32, ctypes.POINTER(sil_params), _P, _P,
                      ctypes.POINTER(_I32)], _I32),
    "sil_autotune_ex": ([ctypes.POINTER(sil_tile), _I32, _I32, ctypes.POINTER(sil_params), _P, _P,
                         ctypes.POINTER(sil_tuning)], _I32),
    "sil_batch_tuning": ([ctypes.POINTER(sil_tile), _I32, _I32, ctypes.POINTER(sil_params), _P,
                          ctypes.POINTER(sil_tuning), ctypes.POINTER(_I32)], _I32),
    "sil_label_batch_noalloc": ([ctypes.POINTER(sil_tile), _I32, _I32, ctypes.POINTER(sil_params), _P], _I32),
    "sil_server_config_default": ([ctypes.POINTER(sil_server_config)], _I32),
    "sil_server_create": ([ctypes.POINTER(_P), ctypes.POINTER(sil_server_config), _I32,
                           ctypes.POINTER(sil_params)], _I32),
    "sil_server_submit": ([_P, _P, _I64, _I64, _I64, _P, _I64, _P, ctypes.POINTER(_I64)], _I32),
    "sil_server_wait": ([_P, _I64, _I64, ctypes.POINTER(sil_request_result)], _I32),
    "sil_server_poll": ([_P, _I64, ctypes.POINTER(sil_request_result)], _I32),
    "sil_server_cancel": ([_P, _I64], _I32),
    "sil_server_destroy": ([_P], None),
    "sil_server_stats": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)], _I32),
    "sil_server_set_fault": ([_P, _I32], _I32),
    "sil_confusion": ([_P, _I64, _P, _I64, _I64, _I64, _I32, _P, _P, _P], _I32),
    "sil_render": ([_P, _I64, _I64, _I64, _P, _I64, _P], _I32),
    "sil_metrics_from_confusion": ([_P, ctypes.POINTER(sil_metrics)], _I32),
    "sil_export_chips": ([_P, _I64, _I64, _I64, _P, _I64, _I32, _I64, _I64, _P, _P, _P], _I32),
    "sil_unet_config_default": ([ctypes.c_void_p], _I32),
    "sil_unet_num_layers": ([_I32], _I32),
    "sil_unet_layer_shape": ([_P, _I32, ctypes.POINTER(_I64), ctypes.POINTER(_I32)], _I32),
    "sil_unet_flops_per_chip": ([_P], _I64),
    "sil_unet_create": ([ctypes.POINTER(_P), _P, ctypes.POINTER(ctypes.POINTER(ctypes.c_float)),
                         ctypes.POINTER(ctypes.POINTER(ctypes.c_float)), _I32], _I32),
    "sil_unet_destroy": ([_P], None),
    "sil_unet_forward": ([_P, _P, _I32, _P, _P, _P], _I32),
    "sil_unet_forward_filtered": ([_P, _P, _P, _I32, _P, _P, _P], _I32),
    "sil_unet_label_scene": ([_P, _P, _I64, _I64, _I64, _P, _I64, _P, _I64, _P], _I32),
    "sil_unet_error_count": ([_P, ctypes.POINTER(ctypes.c_uint32)], _I32),
    "sil_unet_set_fault": ([_P, _I32], _I32),
    "sil_unet_tensor_shape": ([_P, _I32, ctypes.POINTER(_I64)], _I32),
    "sil_unet_copy_tensor": ([_P, _I32, _P, _P], _I32),
    "sil_unet_trainer_create": ([ctypes.POINTER(_P), _P, ctypes.POINTER(ctypes.POINTER(ctypes.c_float)),
                                 ctypes.POINTER(ctypes.POINTER(ctypes.c_float)), _I32], _I32),
    "sil_unet_trainer_destroy": ([_P], None),
    "sil_unet_trainer_net": ([_P], _P),
    "sil_unet_trainer_num_params": ([_P], _I64),
    "sil_unet_trainer_param_offset": ([_P, _I32, ctypes.POINTER(_I64), ctypes.POINTER(_I64)], _I32),
    "sil_unet_trainer_backward": ([_P, _P, _P, _I32, _P, _P, _P], _I32),
    "sil_unet_trainer_adam": ([_P, _P, ctypes.c_float, _I32, _P], _I32),
    "sil_unet_trainer_get_params": ([_P, _P, _P], _I32),
    "sil_unet_trainer_set_params": ([_P, _P, _P], _I32),
    "sil_unet_trainer_grad_shape": ([_P, _I32, _I32, ctypes.POINTER(_I64)], _I32),
    "sil_unet_trainer_copy_grad": ([_P, _I32, _I32, _P, _P], _I32),
}
EXPORTED = tuple(_SIGS)

for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name, None)
    if _f is None:
        continue
    _f.argtypes = _args
    _f.restype = _res
    globals()[_name] = _f


def check(status: int) -> None:
    if status != SIL_OK:
        raise SilError(status, (_lib.sil_last_error() or b"").decode())


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------
def params(**overrides) -> sil_params:
    """Default parameters (paper class ranges, filter F1) with overrides;
    ``lo`` / ``hi`` take 3 x 3 nested lists."""
    p = sil_params()
    check(_lib.sil_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        if k.startswith("_"):
            continue
        if k in ("lo", "hi"):
            arr = getattr(p, k)
            for a in range(3):
                for b in range(3):
                    arr[a][b] = int(v[a][b])
        else:
            setattr(p, k, int(v))
    return p


def _as_params(p) -> sil_params:
    if p is None:
        return params()
    if isinstance(p, sil_params):
        return p
    return params(**dict(p))


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _img_geometry(img):
    """(H, W, pitch_bytes, dtype) of an H x W x 3 uint8/uint16 tensor whose
    rows may be padded (stride(0) >= 3 W)."""
    import torch
    assert img.dim() == 3 and img.shape[2] == 3, "image must be H x W x 3"
    assert img.stride(2) == 1 and img.stride(1) == 3, "pixels must be interleaved"
    if img.dtype == torch.uint8:
        dt, es = SIL_U8, 1
    elif img.dtype in (torch.uint16, torch.int16):
        dt, es = SIL_U16, 2
    else:
        raise TypeError(f"unsupported dtype {img.dtype}")
    return img.shape[0], img.shape[1], img.stride(0) * es, dt


def label(img, p=None, *, labels=True, chip_counts=False, out_labels=None,
          out_counts=None, out_chip_counts=None, stream=None):
    """Label one device image (torch CUDA tensor H x W x 3, uint8 or uint16).

    Returns (labels uint8 H x W or None, counts uint64[4] as int64 tensor,
    chip_counts int32 [gy, gx, 4] or None).  Asynchronous on ``stream``."""
    import torch
    H, W, pitch, dt = _img_geometry(img)
    pp = _as_params(p)
    C = pp.chip
    gy, gx = -(-H // C), -(-W // C)
    dev = img.device
    lab = None
    if labels:
        lab = out_labels if out_labels is not None else torch.empty((H, W), dtype=torch.uint8, device=dev)
    cnt = out_counts if out_counts is not None else torch.empty(4, dtype=torch.int64, device=dev)
    cc = None
    if chip_counts:
        cc = out_chip_counts if out_chip_counts is not None else torch.empty((gy, gx, 4), dtype=torch.int32, device=dev)
    check(_lib.sil_label(img.data_ptr(), H, W, pitch, dt, ctypes.byref(pp),
                         lab.data_ptr() if lab is not None else None,
                         lab.stride(0) if lab is not None else W,
                         cnt.data_ptr(), cc.data_ptr() if cc is not None else None,
                         _stream_handle(stream)))
    return lab, cnt, cc


def label_v(img, p=None, *, labels=True, chip_counts=False, stream=None):
    """Like ``label`` plus the filter's corrected value V' of every pixel
    (uint8 H x W; sil_label_v).  Returns (labels or None, vprime, counts),
    and the chip counts as a fourth item when ``chip_counts``."""
    import torch
    H, W, pitch, dt = _img_geometry(img)
    pp = _as_params(p)
    dev = img.device
    lab = torch.empty((H, W), dtype=torch.uint8, device=dev) if labels else None
    vp = torch.empty((H, W), dtype=torch.uint8, device=dev)
    cnt = torch.empty(4, dtype=torch.int64, device=dev)
    cc = None
    if chip_counts:
        cc = torch.empty((-(-H // pp.chip), -(-W // pp.chip), 4), dtype=torch.int32, device=dev)
    check(_lib.sil_label_v(img.data_ptr(), H, W, pitch, dt, ctypes.byref(pp),
                           lab.data_ptr() if lab is not None else None, W, vp.data_ptr(), W,
                           cnt.data_ptr(), cc.data_ptr() if cc is not None else None,
                           _stream_handle(stream)))
    return (lab, vp, cnt, cc) if chip_counts else (lab, vp, cnt)


def label_host(img: np.ndarray, p=None, *, labels=True, chip_counts=False, stream=None):
    """Label a HOST image (numpy H x W x 3 uint8/uint16, ideally in pinned
    memory); returns numpy (labels, counts uint64[4], chip_counts)."""
    assert img.ndim == 3 and img.shape[2] == 3
    H, W = img.shape[:2]
    dt = SIL_U8 if img.dtype == np.uint8 else SIL_U16
    pp = _as_params(p)
    C = pp.chip
    gy, gx = -(-H // C), -(-W // C)
    lab = np.empty((H, W), np.uint8) if labels else None
    cnt = np.zeros(4, np.uint64)
    cc = np.zeros((gy, gx, 4), np.uint32) if chip_counts else None
    check(_lib.sil_label_host(img.ctypes.data, H, W, img.strides[0], dt, ctypes.byref(pp),
                              lab.ctypes.data if lab is not None else None, W,
                              cnt.ctypes.data, cc.ctypes.data if cc is not None else None,
                              _stream_handle(stream)))
    return lab, cnt, cc


class Context:
    """Owns a sil_ctx (batch work queue, graph cache, autotune results)."""

    def __init__(self, device: int | None = None):
        import torch
        if device is None:
            device = torch.cuda.current_device()
        self.handle = ctypes.c_void_p()
        check(_lib.sil_ctx_create(ctypes.byref(self.handle), int(device)))

    def close(self):
        if self.handle:
            _lib.sil_ctx_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_tiles(imgs, labels=None, counts=None, chip_counts=None):
    """ctypes array of sil_tile for lists of device tensors."""
    n = len(imgs)
    arr = (sil_tile * n)()
    for i, im in enumerate(imgs):
        H, W, pitch, _ = _img_geometry(im)
        t = arr[i]
        t.img = im.data_ptr()
        t.H, t.W, t.pitch_bytes = H, W, pitch
        lab = labels[i] if labels is not None else None
        t.labels = lab.data_ptr() if lab is not None else None
        t.label_pitch = lab.stride(0) if lab is not None else W
        t.counts = counts[i].data_ptr()
        cc = chip_counts[i] if chip_counts is not None else None
        t.chip_counts = cc.data_ptr() if cc is not None else None
    return arr


def label_batch(ctx: Context, tiles, n: int, dt: int = SIL_U8, p=None, stream=None):
    pp = _as_params(p)
    check(_lib.sil_label_batch(tiles, int(n), int(dt), ctypes.byref(pp), ctx.handle,
                               _stream_handle(stream)))


def _tuning_dict(t: sil_tuning) -> dict:
    return {"schedule": int(t.schedule), "ctas_per_sm": int(t.ctas_per_sm), "threads": int(t.threads),
            "us": float(t.us)}


def autotune(ctx: Context, tiles, n: int, dt: int = SIL_U8, p=None, stream=None) -> dict:
    """Time every schedule of the batched kernel on this batch
    (sil_autotune_ex); returns the winner as a dict (schedule, ctas_per_sm,
    threads, us), which ctx then uses for batches of the same class."""
    pp = _as_params(p)
    best = sil_tuning()
    check(_lib.sil_autotune_ex(tiles, int(n), int(dt), ctypes.byref(pp), ctx.handle,
                               _stream_handle(stream), ctypes.byref(best)))
    return _tuning_dict(best)


def batch_tuning(ctx: Context, tiles, n: int, dt: int = SIL_U8, p=None):
    """The schedule sil_label_batch would use for this batch, and whether it
    comes from a tuning: (dict, bool)."""
    pp = _as_params(p)
    t = sil_tuning()
    tuned = _I32(0)
    check(_lib.sil_batch_tuning(tiles, int(n), int(dt), ctypes.byref(pp), ctx.handle, ctypes.byref(t),
                                ctypes.byref(tuned)))
    return _tuning_dict(t), bool(tuned.value)


def confusion(pred, ref, chip: int = 256, chip_conf: bool = False, stream=None):
    """Confusion counts [pred][ref] of two device label maps (uint8 H x W)."""
    import torch
    H, W = pred.shape
    conf = torch.empty((4, 4), dtype=torch.int64, device=pred.device)
    cc = None
    if chip_conf:
        cc = torch.empty((-(-H // chip), -(-W // chip), 4, 4), dtype=torch.int32, device=pred.device)
    check(_lib.sil_confusion(pred.data_ptr(), pred.stride(0), ref.data_ptr(), ref.stride(0), H, W,
                             int(chip), conf.data_ptr(), cc.data_ptr() if cc is not None else None,
                             _stream_handle(stream)))
    return conf, cc


def render(labels, stream=None):
    """Colour image (H x W x 3 uint8, device) of a label map: thick red,
    thin blue, water green, masked black."""
    import torch
    H, W = labels.shape
    rgb = torch.empty((H, W, 3), dtype=torch.uint8, device=labels.device)
    check(_lib.sil_render(labels.data_ptr(), labels.stride(0), H, W, rgb.data_ptr(), 3 * W,
                          _stream_handle(stream)))
    return rgb


def metrics(conf) -> dict:
    """Sec. IV-A metrics of a 4 x 4 confusion count matrix [pred][ref]
    (host numpy or a torch tensor; sil_metrics_from_confusion)."""
    c = np.ascontiguousarray(np.asarray(conf.cpu() if hasattr(conf, "cpu") else conf,
                                        dtype=np.uint64).reshape(16))
    m = sil_metrics()
    check(_lib.sil_metrics_from_confusion(c.ctypes.data, ctypes.byref(m)))
    return {"accuracy": m.accuracy, "precision": list(m.precision), "recall": list(m.recall),
            "f1": list(m.f1), "macro_precision": m.macro_precision, "macro_recall": m.macro_recall,
            "macro_f1": m.macro_f1, "weighted_precision": m.weighted_precision,
            "weighted_recall": m.weighted_recall, "weighted_f1": m.weighted_f1,
            "matrix": [list(r) for r in m.matrix], "support": [int(v) for v in m.support]}


def export_chips(img, labels, chip: int = 256, k0: int = 0, n: int | None = None, stream=None):
    """Image chips and colour-mask chips of a device scene and its labels
    (sil_export_chips): chips k0 .. k0 + n - 1 of the chip grid, each
    [chip, chip, 3] uint8; returns (chips, masks) device tensors [n, ...]."""
    import torch
    H, W, pitch, dt = _img_geometry(img)
    assert dt == SIL_U8, "uint8 images"
    gy, gx = -(-H // chip), -(-W // chip)
    if n is None:
        n = gy * gx - k0
    chips = torch.empty((n, chip, chip, 3), dtype=torch.uint8, device=img.device)
    masks = torch.empty((n, chip, chip, 3), dtype=torch.uint8, device=img.device)
    check(_lib.sil_export_chips(img.data_ptr(), H, W, pitch, labels.data_ptr(), labels.stride(0),
                                int(chip), int(k0), int(n), chips.data_ptr(), masks.data_ptr(),
                                _stream_handle(stream)))
    return chips, masks


class Server:
    """Continuous-batching labelling server (sil_server_*).  Images are host
    numpy arrays (H x W x 3, uint8/uint16; pinned memory gives the fastest
    copies) kept alive here until their request completes."""

    def __init__(self, dt: int = SIL_U8, p=None, *, device: int = 0, max_inflight: int = 64,
                 mem_budget: int = 0, max_batch: int = 32, want_labels: bool = True,
                 ready_timeout_ms: int | None = None, idle_timeout_us: int | None = None):
        cfg = sil_server_config()
        check(_lib.sil_server_config_default(ctypes.byref(cfg)))
        if ready_timeout_ms is not None:
            cfg.ready_timeout_ms = int(ready_timeout_ms)
        if idle_timeout_us is not None:
            cfg.idle_timeout_us = int(idle_timeout_us)
        cfg.device, cfg.max_inflight, cfg.device_mem_budget = device, max_inflight, mem_budget
        cfg.max_batch, cfg.want_labels = max_batch, int(want_labels)
        self.dt = dt
        self.params = _as_params(p)
        self.handle = ctypes.c_void_p()
        check(_lib.sil_server_create(ctypes.byref(self.handle), ctypes.byref(cfg), dt,
                                     ctypes.byref(self.params)))
        self._keep = {}

    def submit(self, img: np.ndarray, labels: np.ndarray | None = None,
               chip_counts: np.ndarray | None = None) -> int:
        H, W = img.shape[:2]
        rid = _I64(0)
        check(_lib.sil_server_submit(self.handle, img.ctypes.data, H, W, img.strides[0],
                                     labels.ctypes.data if labels is not None else None,
                                     labels.strides[0] if labels is not None else W,
                                     chip_counts.ctypes.data if chip_counts is not None else None,
                                     ctypes.byref(rid)))
        self._keep[rid.value] = (img, labels, chip_counts)
        return rid.value

    @staticmethod
    def _result(r: sil_request_result) -> dict:
        return {"id": r.id, "status": r.status, "counts": [int(c) for c in r.counts],
                "t_submit_ms": r.t_submit_ms, "t_admit_ms": r.t_admit_ms, "t_done_ms": r.t_done_ms}

    def wait(self, rid: int, timeout_ms: int = -1) -> dict:
        """Result of request rid once it has completed ({'status': the
        request's own status, 'counts', times}); raises SilError with
        SIL_ETIMEOUT if it has not completed within timeout_ms."""
        res = sil_request_result()
        st = _lib.sil_server_wait(self.handle, rid, int(timeout_ms), ctypes.byref(res))
        if st != SIL_OK:
            raise SilError(st, (_lib.sil_last_error() or b"").decode())
        self._keep.pop(rid, None)
        return self._result(res)

    def poll(self, rid: int):
        """The result if request rid has completed, None if not yet;
        {'status': SIL_EINVAL} for an unknown id."""
        res = sil_request_result()
        st = _lib.sil_server_poll(self.handle, rid, ctypes.byref(res))
        if st == SIL_EBUSY:
            return None
        if st != SIL_OK:
            return {"id": rid, "status": st}
        self._keep.pop(rid, None)
        return self._result(res)

    def cancel(self, rid: int) -> int:
        return _lib.sil_server_cancel(self.handle, rid)

    def stats(self) -> dict:
        """{'kernel_launches', 'chips_published'} so far."""
        a, b = _I64(0), _I64(0)
        check(_lib.sil_server_stats(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return {"kernel_launches": a.value, "chips_published": b.value}

    def set_fault(self, skip_ready: bool) -> None:
        """Test hook: the next published request never gets its ready word
        (its chips' bounded device waits run out; it ends with SIL_ETIMEOUT)."""
        check(_lib.sil_server_set_fault(self.handle, int(bool(skip_ready))))

    def close(self):
        if self.handle:
            _lib.sil_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# U-Net inference on filtered chips (include/sil_unet.h)
# --------------------------------------------------------------------------
class sil_unet_config(ctypes.Structure):
    _fields_ = [("base_width", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("max_batch", ctypes.c_int32)]


UNET_CONV3, UNET_UP, UNET_HEAD = 0, 1, 2


def unet_config(base_width: int = 32, depth: int = 5, max_batch: int = 32) -> sil_unet_config:
    c = sil_unet_config()
    check(_lib.sil_unet_config_default(ctypes.byref(c)))
    c.base_width, c.depth, c.max_batch = int(base_width), int(depth), int(max_batch)
    return c


def unet_layer_shapes(cfg: sil_unet_config):
    """[(weight shape, kind)] in the library's layer order."""
    out = []
    nl = _lib.sil_unet_num_layers(cfg.depth)
    if nl < 0:
        raise SilError(SIL_EINVAL, f"U-Net depth {cfg.depth} out of range")
    for i in range(nl):
        dims = (_I64 * 4)()
        kind = _I32()
        check(_lib.sil_unet_layer_shape(ctypes.byref(cfg), i, dims, ctypes.byref(kind)))
        out.append((tuple(int(d) for d in dims), int(kind.value)))
    return out


def _weight_arrays(cfg, weights):
    """Host float32 arrays of (w, b) per layer, checked against the layer
    shapes, as the C arrays of pointers sil_unet_create takes."""
    shapes = unet_layer_shapes(cfg)
    if len(weights) != len(shapes):
        raise ValueError(f"{len(weights)} layers given, {len(shapes)} expected")
    keep = []
    W = (ctypes.POINTER(ctypes.c_float) * len(shapes))()
    B = (ctypes.POINTER(ctypes.c_float) * len(shapes))()
    for i, ((w, b), (shape, kind)) in enumerate(zip(weights, shapes)):
        w = np.ascontiguousarray(w, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float32)
        if w.shape != shape:
            raise ValueError(f"layer {i}: weight shape {w.shape}, expected {shape}")
        keep += [w, b]
        W[i] = w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        B[i] = b.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    return W, B, keep


class UNet:
    """A network on the current CUDA device.  ``weights``: list of (w, b)
    float32 numpy arrays in the library's layer order (PyTorch layouts)."""

    def __init__(self, cfg: sil_unet_config, weights, device: int = 0):
        W, B, keep = _weight_arrays(cfg, weights)
        self.cfg = cfg
        self.handle = _P()
        self._owner = None
        check(_lib.sil_unet_create(ctypes.byref(self.handle), ctypes.byref(cfg), W, B, int(device)))
        del keep

    @classmethod
    def _borrow(cls, handle, cfg, owner):
        """The network of a Trainer (owned, and freed, by the trainer)."""
        net = cls.__new__(cls)
        net.cfg, net.handle, net._owner = cfg, _P(handle), owner
        return net

    def __del__(self):
        if getattr(self, "handle", None) and getattr(self, "_owner", None) is None:
            _lib.sil_unet_destroy(self.handle)
        self.handle = None

    def flops_per_chip(self) -> int:
        return int(_lib.sil_unet_flops_per_chip(ctypes.byref(self.cfg)))

    def forward(self, chips, labels=None, logits=None, stream=None, vprime=None):
        """chips: cuda uint8 [n, 256, 256, 3]; labels: cuda uint8 [n, 256, 256]
        or None; logits: cuda float32 [n, 256, 256, 3] or None; vprime: cuda
        uint8 [n, 256, 256] (the filter's V') to run on the filtered chips."""
        n = int(chips.shape[0])
        check(_lib.sil_unet_forward_filtered(self.handle, chips.data_ptr(),
                                             vprime.data_ptr() if vprime is not None else None, n,
                                             labels.data_ptr() if labels is not None else None,
                                             logits.data_ptr() if logits is not None else None,
                                             _stream_handle(stream)))

    def set_fault(self, layer: int) -> None:
        """Test hook: make layer `layer`'s bounded wait run out (-1 clears)."""
        check(_lib.sil_unet_set_fault(self.handle, int(layer)))

    def label_scene(self, img, vprime=None, labels=None, stream=None):
        """U-Net labels of a whole device scene (H x W x 3 uint8), chip by chip,
        on the filtered chips when vprime (H x W uint8, from label_v) is given."""
        import torch
        H, W, pitch, dt = _img_geometry(img)
        if dt != SIL_U8:
            raise ValueError("label_scene takes uint8 RGB scenes")
        if labels is None:
            labels = torch.empty((H, W), dtype=torch.uint8, device=img.device)
        check(_lib.sil_unet_label_scene(self.handle, img.data_ptr(), H, W, pitch,
                                        vprime.data_ptr() if vprime is not None else None,
                                        vprime.stride(0) if vprime is not None else W,
                                        labels.data_ptr(), labels.stride(0), _stream_handle(stream)))
        return labels

    def error_count(self) -> int:
        v = ctypes.c_uint32()
        check(_lib.sil_unet_error_count(self.handle, ctypes.byref(v)))
        return int(v.value)

    def tensor(self, i: int, stream=None):
        """Copy of layer i's output activation (i = -1: the prepared input) as
        a cuda bfloat16 tensor [n, H, W, C]."""
        import torch
        dims = (_I64 * 4)()
        check(_lib.sil_unet_tensor_shape(self.handle, int(i), dims))
        out = torch.empty(tuple(int(d) for d in dims), dtype=torch.bfloat16, device="cuda")
        check(_lib.sil_unet_copy_tensor(self.handle, int(i), out.data_ptr(), _stream_handle(stream)))
        return out


# --------------------------------------------------------------------------
# U-Net training step and data-parallel plumbing (include/sil_unet.h)
# --------------------------------------------------------------------------
UNET_GRAD_LAYER, UNET_GRAD_CAT, UNET_GRAD_POOL = 0, 1, 2


class Trainer:
    """Training of a U-Net on the current CUDA device: ``backward`` gives the
    flat f32 gradient and the mean loss of a batch, ``adam`` applies one
    update with a (possibly averaged) gradient.  ``net`` is the trained
    network (forward pass, activations)."""

    def __init__(self, cfg: sil_unet_config, weights, device: int = 0):
        W, B, keep = _weight_arrays(cfg, weights)
        self.cfg = cfg
        self.handle = _P()
        check(_lib.sil_unet_trainer_create(ctypes.byref(self.handle), ctypes.byref(cfg), W, B,
                                           int(device)))
        del keep
        self.device = int(device)
        self.num_params = int(_lib.sil_unet_trainer_num_params(self.handle))
        self.net = UNet._borrow(_lib.sil_unet_trainer_net(self.handle), cfg, self)
        self.shapes = unet_layer_shapes(cfg)
        self.offsets = []
        for i in range(len(self.shapes)):
            wo, bo = _I64(), _I64()
            check(_lib.sil_unet_trainer_param_offset(self.handle, i, ctypes.byref(wo), ctypes.byref(bo)))
            self.offsets.append((int(wo.value), int(bo.value)))
        self.t = 0

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.sil_unet_trainer_destroy(self.handle)
            self.handle = None

    def _flat(self):
        import torch
        return torch.empty(self.num_params, dtype=torch.float32, device=f"cuda:{self.device}")

    def backward(self, chips, labels, grads=None, loss=None, stream=None):
        """chips: cuda uint8 [n, 256, 256, 3]; labels: cuda uint8 [n, 256, 256]
        (3: left out of the loss).  Returns (grads [num_params], loss [1])."""
        import torch
        grads = self._flat() if grads is None else grads
        loss = torch.empty(1, dtype=torch.float32, device=grads.device) if loss is None else loss
        check(_lib.sil_unet_trainer_backward(self.handle, chips.data_ptr(), labels.data_ptr(),
                                             int(chips.shape[0]), grads.data_ptr(), loss.data_ptr(),
                                             _stream_handle(stream)))
        return grads, loss

    def adam(self, grads, lr: float = 1e-3, t: int | None = None, stream=None) -> None:
        """One Adam step (t: the step number, default one past the last)."""
        self.t = self.t + 1 if t is None else int(t)
        check(_lib.sil_unet_trainer_adam(self.handle, grads.data_ptr(), float(lr), self.t,
                                         _stream_handle(stream)))

    def params(self, stream=None):
        out = self._flat()
        check(_lib.sil_unet_trainer_get_params(self.handle, out.data_ptr(), _stream_handle(stream)))
        return out

    def set_params(self, flat, stream=None) -> None:
        """Loads the flat master weights (cuda float32 [num_params]) and starts
        a fresh optimizer (moments zero, step count 0)."""
        check(_lib.sil_unet_trainer_set_params(self.handle, flat.data_ptr(), _stream_handle(stream)))
        self.t = 0

    def unflatten(self, flat) -> list:
        """[(w, b)] numpy float32 per layer from a flat vector."""
        a = flat.detach().cpu().numpy() if hasattr(flat, "detach") else np.asarray(flat)
        out = []
        for (shape, kind), (wo, bo) in zip(self.shapes, self.offsets):
            nw = int(np.prod(shape))
            nb = shape[1] if kind == UNET_UP else shape[0]
            out.append((a[wo:wo + nw].reshape(shape).copy(), a[bo:bo + nb].copy()))
        return out

    def grad_tensor(self, kind: int, i: int, stream=None):
        """A stored activation gradient of the last backward pass (kind
        UNET_GRAD_LAYER / CAT / POOL) as a cuda bfloat16 tensor [n, H, W, C]."""
        import torch
        dims = (_I64 * 4)()
        check(_lib.sil_unet_trainer_grad_shape(self.handle, int(kind), int(i), dims))
        out = torch.empty(tuple(int(d) for d in dims), dtype=torch.bfloat16, device=f"cuda:{self.device}")
        check(_lib.sil_unet_trainer_copy_grad(self.handle, int(kind), int(i), out.data_ptr(),
                                              _stream_handle(stream)))
        return out

    def step(self, chips, labels, lr: float = 1e-3, group=None, grads=None, loss=None, stream=None):
        """One data-parallel step: local gradient, average over the process
        group (none: this process alone), Adam.  Returns the local loss."""
        grads, loss = self.backward(chips, labels, grads, loss, stream)
        average_gradients_(grads, group)
        self.adam(grads, lr, stream=stream)
        return loss


def average_gradients_(grads, group=None):
    """In place: the mean of every rank's gradient (the all-reduce of the
    data-parallel optimizer).  No-op without an initialised process group."""
    import torch.distributed as dist
    if group is None and not (dist.is_available() and dist.is_initialized()):
        return grads
    world = dist.get_world_size(group)
    if world > 1:
        dist.all_reduce(grads, op=dist.ReduceOp.SUM, group=group)
        grads.div_(world)
    return grads


def broadcast_params_(trainer, src: int = 0, group=None):
    """Every rank takes rank `src`'s weights and restarts its optimizer."""
    import torch.distributed as dist
    flat = trainer.params()
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.broadcast(flat, src=src, group=group)
    trainer.set_params(flat)
    return flat
