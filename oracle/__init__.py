"""Plain CPU oracle for the augmentation hot path (arXiv 1809.06839).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (``paper_1809_06839_gb300``) never imports it and shares
no code with it.

The arithmetic lives in ``alb_oracle.c`` (plain loops, float64 / exact
integers, built with ``-ffp-contract=off``); this module only marshals numpy
arrays through ctypes.  Every function is pinned by ``tests/test_oracle_*.py``
(closed forms, library routines, invariants, brute force).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "alb_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

# transform ids (same public numbering as the C-ABI)
HFLIP, VFLIP, RANDOM_CROP, PAD_TO_SIZE = 1, 2, 3, 4
BRIGHTNESS, CONTRAST, BRIGHTNESS_CONTRAST, GAMMA = 5, 6, 7, 8
SHIFT_RGB, SHIFT_HSV, GRAYSCALE, EQUALIZE = 9, 10, 11, 12
ROTATE, SHIFT_SCALE_ROTATE, RESIZE, RANDOM_SIZED_CROP = 13, 14, 15, 16
RANDOM_RESIZED_CROP, TRANSPOSE, ROT90, CHAIN = 17, 18, 19, 20
GRID_DISTORTION, ELASTIC = 21, 22


class Params(C.Structure):
    _fields_ = [
        ("tid", C.c_int32), ("apply", C.c_int32),
        ("in_h", C.c_int32), ("in_w", C.c_int32), ("out_h", C.c_int32), ("out_w", C.c_int32),
        ("y0", C.c_int32), ("x0", C.c_int32), ("ch", C.c_int32), ("cw", C.c_int32),
        ("flip", C.c_int32), ("k", C.c_int32),
        ("alpha", C.c_double), ("beta", C.c_double), ("gamma", C.c_double), ("sat", C.c_double),
        ("shift", C.c_double * 3),
        ("angle", C.c_double), ("scale", C.c_double), ("dx", C.c_double), ("dy", C.c_double),
        ("m", C.c_double * 6),
        ("q", C.c_int64 * 6),
    ]


class Cfg(C.Structure):
    _fields_ = [
        ("tid", C.c_int32), ("out_h", C.c_int32), ("out_w", C.c_int32), ("_pad", C.c_int32),
        ("p", C.c_double),
        ("lo", C.c_double * 4), ("hi", C.c_double * 4),
    ]


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile alb_oracle.c into oracle/_build/liboracle.so (gcc, no SIMD)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-fvisibility=hidden", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


def _declare(L):
    P = C.POINTER
    u8p = P(C.c_uint8)
    L.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
    L.orc_stream_words.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_int, P(C.c_uint32)]
    L.orc_stream_uniform01.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_int, P(C.c_double)]
    L.orc_stream_randint.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_int32, C.c_int,
                                     P(C.c_int32)]
    L.orc_sample_params.argtypes = [P(Cfg), C.c_uint64, C.c_uint64, C.c_uint32, C.c_int, C.c_int,
                                    P(Params)]
    L.orc_sample_params.restype = C.c_int
    L.orc_warp_geometry.argtypes = [P(Params), C.c_int, C.c_int]
    L.orc_output_shape.argtypes = [P(Params), C.c_int, C.c_int, P(C.c_int), P(C.c_int)]
    L.orc_build_lut.argtypes = [P(Params), u8p]
    L.orc_build_lut.restype = C.c_int
    L.orc_equalize_lut.argtypes = [P(C.c_uint64), u8p]
    L.orc_shift_hsv_pixel.argtypes = [P(C.c_double), u8p, u8p]
    for name in ("orc_apply_image", "orc_apply_mask"):
        f = getattr(L, name)
        f.argtypes = [P(Params), u8p, C.c_int, C.c_int, C.c_int, C.c_int64, u8p, C.c_int64]
        f.restype = C.c_int
    L.orc_apply_boxes.argtypes = [P(Params), C.c_int, C.c_int, P(C.c_float), C.c_int, P(C.c_float)]
    L.orc_apply_boxes.restype = C.c_int
    L.orc_grid_q5.argtypes = [P(Params), C.c_int, C.c_int64, C.c_int64]
    L.orc_grid_q5.restype = C.c_int64
    L.orc_grid_edge_inverse.argtypes = [P(Params), C.c_int, C.c_double, C.c_int64]
    L.orc_grid_edge_inverse.restype = C.c_double
    L.orc_grid_factor.argtypes = [P(Params), C.c_int]
    L.orc_grid_factor.restype = C.c_int32
    L.orc_grid_set_factor.argtypes = [P(Params), C.c_int, C.c_int32]
    L.orc_grid_set_factor.restype = None
    L.orc_elastic_point.argtypes = [P(Params), C.c_int64, P(C.c_int32), P(C.c_int32)]
    L.orc_elastic_point.restype = None
    L.orc_elastic_disp.argtypes = [P(Params), C.c_int64, C.c_int64, C.c_int, P(C.c_int32), P(C.c_int32)]
    L.orc_elastic_disp.restype = None
    L.orc_chain_mask.argtypes = [P(Params), u8p, C.c_int, C.c_int, C.c_int, C.c_int64, u8p, C.c_int64]
    L.orc_chain_mask.restype = C.c_int
    L.orc_chain_boxes.argtypes = [P(Params), P(C.c_float), C.c_int, P(C.c_float)]
    L.orc_chain_boxes.restype = C.c_int
    L.orc_sample_chain_box_safe.argtypes = [P(Cfg), C.c_uint64, C.c_uint64, C.c_uint32, C.c_int, C.c_int,
                                            P(C.c_float), C.c_int, P(Params)]
    L.orc_sample_chain_box_safe.restype = C.c_int
    L.orc_f32_to_bf16.argtypes = [C.c_float]
    L.orc_f32_to_bf16.restype = C.c_uint16
    L.orc_normalize_consts.argtypes = [P(C.c_double), P(C.c_double), P(C.c_float), P(C.c_float)]
    L.orc_chain_image.argtypes = [P(Params), P(C.c_double), P(C.c_double), u8p, C.c_int, C.c_int,
                                  C.c_int64, P(C.c_uint16)]
    L.orc_chain_image.restype = C.c_int
    L.orc_chain_image_jitter.argtypes = L.orc_chain_image.argtypes
    L.orc_chain_image_jitter.restype = C.c_int
    L.orc_jitter_mode1.argtypes = [P(Params), u8p, C.c_size_t]
    L.orc_jitter_mode1.restype = None
    L.orc_contrast_pivot.argtypes = [u8p, C.c_size_t]
    L.orc_contrast_pivot.restype = C.c_int
    L.orc_jitter_op.argtypes = [C.c_int, C.c_int]
    L.orc_jitter_op.restype = C.c_int
    dp = P(C.c_double)
    L.orc_warp_photo_fwd.argtypes = [C.c_int] * 5 + [dp] * 10
    L.orc_warp_photo_bwd.argtypes = [C.c_int] * 5 + [dp] * 13


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


# ---------------------------------------------------------------- sampler
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def stream_words(seed, stream_id, index, n):
    out = np.zeros(n, dtype=np.uint32)
    lib().orc_stream_words(seed, stream_id, index, n, _ptr(out, C.c_uint32))
    return out


def stream_uniform01(seed, stream_id, index, n):
    out = np.zeros(n, dtype=np.float64)
    lib().orc_stream_uniform01(seed, stream_id, index, n, _ptr(out, C.c_double))
    return out


def stream_randint(seed, stream_id, index, hi, n):
    out = np.zeros(n, dtype=np.int32)
    lib().orc_stream_randint(seed, stream_id, index, hi, n, _ptr(out, C.c_int32))
    return out


def make_cfg(tid, p=1.0, out_h=0, out_w=0, lo=(), hi=()) -> Cfg:
    c = Cfg()
    c.tid, c.out_h, c.out_w, c.p = tid, out_h, out_w, p
    for i, v in enumerate(lo):
        c.lo[i] = v
    for i, v in enumerate(hi):
        c.hi[i] = v
    return c


def sample_params(cfg: Cfg, seed: int, stream_id: int, index: int, h: int, w: int) -> Params:
    p = Params()
    rc = lib().orc_sample_params(C.byref(cfg), seed, stream_id, index, h, w, C.byref(p))
    if rc != 0:
        raise ValueError(f"orc_sample_params failed with status {rc}")
    return p


def warp_geometry(p: Params, h: int, w: int) -> Params:
    lib().orc_warp_geometry(C.byref(p), h, w)
    return p


def output_shape(p: Params, h: int, w: int):
    oh, ow = C.c_int(), C.c_int()
    lib().orc_output_shape(C.byref(p), h, w, C.byref(oh), C.byref(ow))
    return oh.value, ow.value


# ---------------------------------------------------------------- images
def build_lut(p: Params) -> np.ndarray:
    lut = np.zeros((3, 256), dtype=np.uint8)
    rc = lib().orc_build_lut(C.byref(p), _ptr(lut, C.c_uint8))
    if rc != 0:
        raise ValueError("no LUT for this transform")
    return lut


def equalize_lut(hist) -> np.ndarray:
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    lut = np.zeros(256, dtype=np.uint8)
    lib().orc_equalize_lut(_ptr(h, C.c_uint64), _ptr(lut, C.c_uint8))
    return lut


def shift_hsv_pixel(shift, rgb) -> np.ndarray:
    s = np.ascontiguousarray(shift, dtype=np.float64)
    i = np.ascontiguousarray(rgb, dtype=np.uint8)
    o = np.zeros(3, dtype=np.uint8)
    lib().orc_shift_hsv_pixel(_ptr(s, C.c_double), _ptr(i, C.c_uint8), _ptr(o, C.c_uint8))
    return o


def _apply(fn, p: Params, img: np.ndarray) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    squeeze = img.ndim == 2
    if squeeze:
        img = img[:, :, None]
    h, w, c = img.shape
    oh, ow = output_shape(p, h, w)
    out = np.zeros((oh, ow, c), dtype=np.uint8)
    rc = fn(C.byref(p), _ptr(img, C.c_uint8), h, w, c, w * c, _ptr(out, C.c_uint8), ow * c)
    if rc != 0:
        raise ValueError(f"oracle apply failed with status {rc}")
    return out[:, :, 0] if squeeze else out


def apply_image(p: Params, img: np.ndarray) -> np.ndarray:
    return _apply(lib().orc_apply_image, p, img)


def apply_mask(p: Params, mask: np.ndarray) -> np.ndarray:
    return _apply(lib().orc_apply_mask, p, mask)


def apply_boxes(p: Params, h: int, w: int, boxes: np.ndarray) -> np.ndarray:
    b = np.ascontiguousarray(boxes, dtype=np.float32).reshape(-1, 4)
    out = np.zeros_like(b)
    n = lib().orc_apply_boxes(C.byref(p), h, w, _ptr(b, C.c_float), b.shape[0], _ptr(out, C.c_float))
    if n < 0:
        raise ValueError("boxes are not defined for this transform")
    return out[:n]


# ---------------------------------------------------------------- grid / elastic helpers
def grid_q5(p: Params, axis: int, x: int, n: int) -> int:
    return int(lib().orc_grid_q5(C.byref(p), axis, x, n))


def grid_edge_inverse(p: Params, axis: int, e: float, n: int) -> float:
    return float(lib().orc_grid_edge_inverse(C.byref(p), axis, e, n))


def grid_factor(p: Params, slot: int) -> int:
    return int(lib().orc_grid_factor(C.byref(p), slot))


def grid_set_factor(p: Params, slot: int, d: int) -> None:
    lib().orc_grid_set_factor(C.byref(p), slot, d)


def elastic_point(p: Params, t: int):
    dx, dy = C.c_int32(), C.c_int32()
    lib().orc_elastic_point(C.byref(p), t, C.byref(dx), C.byref(dy))
    return dx.value, dy.value


def elastic_disp(p: Params, x: int, y: int, w: int):
    dx, dy = C.c_int32(), C.c_int32()
    lib().orc_elastic_disp(C.byref(p), x, y, w, C.byref(dx), C.byref(dy))
    return dx.value, dy.value


def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    f = lib().orc_f32_to_bf16
    flat = np.asarray(x, dtype=np.float32).ravel()
    return np.array([f(float(v)) for v in flat], dtype=np.uint16).reshape(np.shape(x))


IMAGENET_MEAN = (0.485, 0.456, 0.406)
IMAGENET_STD = (0.229, 0.224, 0.225)


def normalize_consts(mean=IMAGENET_MEAN, std=IMAGENET_STD):
    m = np.ascontiguousarray(mean, dtype=np.float64)
    s = np.ascontiguousarray(std, dtype=np.float64)
    k = np.zeros(3, dtype=np.float32)
    mm = np.zeros(3, dtype=np.float32)
    lib().orc_normalize_consts(_ptr(m, C.c_double), _ptr(s, C.c_double), _ptr(k, C.c_float),
                               _ptr(mm, C.c_float))
    return k, mm


def chain_image(p: Params, img: np.ndarray, mean=IMAGENET_MEAN, std=IMAGENET_STD, jitter: int = 0) -> np.ndarray:
    """bf16 bit patterns, shape (3, out_h, out_w).  jitter 0: fixed order,
    constant contrast pivot, float saturation; 1: the record's random order,
    image-mean contrast pivot, uint8 after each jitter op."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, w, _ = img.shape
    m = np.ascontiguousarray(mean, dtype=np.float64)
    s = np.ascontiguousarray(std, dtype=np.float64)
    out = np.zeros((3, p.out_h, p.out_w), dtype=np.uint16)
    fn = lib().orc_chain_image_jitter if jitter else lib().orc_chain_image
    rc = fn(C.byref(p), _ptr(m, C.c_double), _ptr(s, C.c_double), _ptr(img, C.c_uint8), h, w, w * 3,
            _ptr(out, C.c_uint16))
    if rc != 0:
        raise ValueError("chain failed")
    return out


def jitter_mode1(p: Params, img: np.ndarray) -> np.ndarray:
    """The three jitter ops of mode 1 in the record's order on a uint8 RGB image."""
    out = np.ascontiguousarray(img, dtype=np.uint8).copy()
    lib().orc_jitter_mode1(C.byref(p), _ptr(out, C.c_uint8), out.size // 3)
    return out


def contrast_pivot(img: np.ndarray) -> int:
    a = np.ascontiguousarray(img, dtype=np.uint8)
    return int(lib().orc_contrast_pivot(_ptr(a, C.c_uint8), a.size // 3))


def jitter_op(k: int, i: int) -> int:
    return int(lib().orc_jitter_op(k, i))


# ---------------------------------------------------------------- float path
def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def warp_photo_fwd(x, angle, scale, tx, ty, alpha, beta, gamma, want_warped=False, coords=64):
    """Float warp + photometric forward.  coords=64: source coordinates in
    float64 (the definition); coords=32: the float32 coordinate class (map
    entries rounded to float32 once, coordinates by float32 fused
    multiply-adds), everything else float64."""
    if coords not in (32, 64):
        raise ValueError("coords must be 32 or 64")
    x = _f64(x)
    B, Cc, H, W = x.shape
    args = [_f64(a) for a in (angle, scale, tx, ty, alpha, beta, gamma)]
    y = np.zeros_like(x)
    warped = np.zeros_like(x) if want_warped else None
    dp = C.POINTER(C.c_double)
    lib().orc_warp_photo_fwd(B, Cc, H, W, coords, _ptr(x, C.c_double), *[_ptr(a, C.c_double) for a in args],
                             _ptr(warped, C.c_double) if warped is not None else C.cast(None, dp),
                             _ptr(y, C.c_double))
    return (y, warped) if want_warped else y


def warp_photo_bwd(x, angle, scale, tx, ty, alpha, beta, gamma, gy, coords=64, want_abs=False):
    """Analytic adjoint: (dx, dparams[B][7]); with want_abs also the sums of
    the absolute values of each entry's terms, (adx, adparams)."""
    if coords not in (32, 64):
        raise ValueError("coords must be 32 or 64")
    x = _f64(x)
    gy = _f64(gy)
    B, Cc, H, W = x.shape
    args = [_f64(a) for a in (angle, scale, tx, ty, alpha, beta, gamma)]
    dx = np.zeros_like(x)
    dparams = np.zeros((B, 7), dtype=np.float64)
    adx = np.zeros_like(x) if want_abs else None
    adp = np.zeros((B, 7), dtype=np.float64) if want_abs else None
    nul = C.cast(None, C.POINTER(C.c_double))
    lib().orc_warp_photo_bwd(B, Cc, H, W, coords, _ptr(x, C.c_double), *[_ptr(a, C.c_double) for a in args],
                             _ptr(gy, C.c_double), _ptr(dx, C.c_double), _ptr(dparams, C.c_double),
                             _ptr(adx, C.c_double) if want_abs else nul, _ptr(adp, C.c_double) if want_abs else nul)
    return (dx, dparams, adx, adp) if want_abs else (dx, dparams)


# ---------------------------------------------------------------- chain targets
def chain_mask(p: Params, mask: np.ndarray) -> np.ndarray:
    """N-plane uint8 mask (H, W, N) through the chain's crop, nearest resize and flip."""
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    h, w, c = m.shape
    out = np.zeros((p.out_h, p.out_w, c), np.uint8)
    rc = lib().orc_chain_mask(C.byref(p), _ptr(m, C.c_uint8), h, w, c, w * c, _ptr(out, C.c_uint8), p.out_w * c)
    if rc != 0:
        raise ValueError("chain mask failed")
    return out


def chain_boxes(p: Params, boxes: np.ndarray) -> np.ndarray:
    b = np.ascontiguousarray(boxes, dtype=np.float32).reshape(-1, 4)
    out = np.zeros_like(b)
    n = lib().orc_chain_boxes(C.byref(p), _ptr(b, C.c_float), b.shape[0], _ptr(out, C.c_float))
    return out[:n]


def sample_chain_box_safe(cfg: Cfg, seed: int, stream_id: int, index: int, h: int, w: int,
                          boxes: np.ndarray) -> Params:
    b = np.ascontiguousarray(boxes, dtype=np.float32).reshape(-1, 4)
    p = Params()
    rc = lib().orc_sample_chain_box_safe(C.byref(cfg), seed, stream_id, index, h, w, _ptr(b, C.c_float),
                                         b.shape[0], C.byref(p))
    if rc != 0:
        raise ValueError(f"orc_sample_chain_box_safe failed with status {rc}")
    return p

