"""The C-ABI library: loads, exports every function include/*.h declares,
and its host-only calls behave as documented.  No GPU needed."""
import ctypes
import os
import re

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sil():
    import paper_2403_13135_gb300 as m
    return m


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sil_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("sil_label", "sil_label_batch", "sil_ctx_create", "sil_server_submit",
                 "sil_params_default", "sil_status_string", "sil_unet_create", "sil_unet_forward"):
        assert must in names


def test_every_declared_function_is_exported(sil):
    lib = ctypes.CDLL(sil.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_declared()) <= set(sil.EXPORTED)


def test_params_layout_and_defaults_match_the_paper(sil):
    assert ctypes.sizeof(sil.sil_params) == 56
    p = sil.params()
    d = oracle.params_default()
    assert [[p.lo[k][c] for c in range(3)] for k in range(3)] == d["lo"]
    assert [[p.hi[k][c] for c in range(3)] for k in range(3)] == d["hi"]
    for f in ("filter", "chip", "median", "mm_min_range", "mm_min_frac_den", "v_trunc",
              "max_shift", "bgr", "u16_scale"):
        assert getattr(p, f) == d[f], f
    # Sec. III-B: thick (0,0,205)-(185,255,255), thin (0,0,31)-(185,255,204),
    # water (0,0,0)-(185,255,30)
    assert d["lo"] == [[0, 0, 205], [0, 0, 31], [0, 0, 0]]
    assert d["hi"] == [[185, 255, 255], [185, 255, 204], [185, 255, 30]]


def test_params_validation_agrees_with_oracle(sil):
    cases = [{}, {"chip": 3}, {"chip": 4}, {"chip": 512}, {"chip": 513}, {"filter": 2},
             {"mm_min_range": 0}, {"mm_min_frac_den": 0}, {"v_trunc": 256}, {"max_shift": -1},
             {"u16_scale": 0}, {"u16_scale": 65535}, {"bgr": 1},
             {"lo": [[10, 0, 0], [0, 0, 31], [0, 0, 0]], "hi": [[5, 255, 255], [185, 255, 204], [185, 255, 30]]}]
    for c in cases:
        p = sil.params(**c)
        ok = sil.sil_params_validate(ctypes.byref(p)) == sil.SIL_OK
        assert ok == oracle.params_valid(c), c
    p = sil.params(chip=3)
    assert sil.sil_params_validate(ctypes.byref(p)) == sil.SIL_EINVAL
    assert b"chip" in sil.sil_last_error()


def test_status_strings(sil):
    for s in range(7):
        assert sil.sil_status_string(s)
    assert sil.sil_status_string(99) == b"unknown status"
    assert sil.sil_version() == 2


def test_null_arguments_rejected_without_gpu(sil):
    assert sil.sil_params_default(None) == sil.SIL_EINVAL
    assert sil.sil_ctx_create(None, 0) == sil.SIL_EINVAL
    assert sil.sil_server_config_default(None) == sil.SIL_EINVAL
    p = sil.params()
    # no image -> invalid before any CUDA call
    st = sil.sil_label(None, 4, 4, 12, 0, ctypes.byref(p), None, 4, None, None, None)
    assert st == sil.SIL_EINVAL


def test_unet_host_calls_without_gpu(sil):
    """Layer shapes and flop count agree with the seeded generator's layer
    table; bad configs are rejected on the host."""
    import synth
    for F, depth in ((16, 1), (32, 4), (64, 3), (32, 5), (64, 5)):
        cfg = sil.unet_config(F, depth, 4)
        got = sil.unet_layer_shapes(cfg)
        ref = synth.unet_layer_shapes(F, depth)
        assert [s for s, _ in got] == [s for s, _ in ref.values()]
        kinds = {"conv3": sil.UNET_CONV3, "up": sil.UNET_UP, "head": sil.UNET_HEAD}
        assert [k for _, k in got] == [kinds[k] for _, k in ref.values()]
        # flops: 2 x multiply-adds over the layers at their output resolution
        flops, lvl = 0, {}
        for i, (name, (shape, kind)) in enumerate(ref.items()):
            if name.startswith("enc"):
                res = 256 >> int(name[3])
            elif name.startswith("bott"):
                res = 256 >> depth
            elif name.startswith("up") or name.startswith("dec"):
                res = 256 >> int(name[2] if name.startswith("up") else name[3])
            else:
                res = 256
            taps = 9 if kind == "conv3" else 1
            flops += 2 * res * res * shape[0] * shape[1] * taps
        assert sil._lib.sil_unet_flops_per_chip(ctypes.byref(cfg)) == flops
    bad = sil.sil_unet_config()
    bad.base_width, bad.depth, bad.max_batch = 24, 4, 1
    dims = (ctypes.c_int64 * 4)()
    kind = ctypes.c_int32()
    assert sil._lib.sil_unet_layer_shape(ctypes.byref(bad), 0, dims, ctypes.byref(kind)) == sil.SIL_EINVAL
    assert sil._lib.sil_unet_num_layers(5) == 28
    assert sil._lib.sil_unet_num_layers(6) == -1 and sil._lib.sil_unet_num_layers(0) == -1
    h = ctypes.c_void_p()
    assert sil._lib.sil_unet_create(ctypes.byref(h), ctypes.byref(bad), None, None, 0) == sil.SIL_EINVAL
