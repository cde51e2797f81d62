"""ctypes binding of libalb.so (include/alb.h), same names as the C ABI.

Argument marshalling only: every step of the augmentation path runs in the CUDA
kernels of libalb.so.  PyTorch supplies device memory and streams.  There is no
CPU fallback: loading fails loudly when the library is missing, and the calls
require CUDA tensors.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

from . import build as _build

# ---------------------------------------------------------------- constants
ALB_OK, ALB_EINVAL, ALB_ESHAPE, ALB_EALIGN, ALB_ECAPACITY, ALB_ECUDA, ALB_ETIMEOUT, ALB_EWORKSPACE = range(8)
HFLIP, VFLIP, RANDOM_CROP, PAD_TO_SIZE = 1, 2, 3, 4
BRIGHTNESS, CONTRAST, BRIGHTNESS_CONTRAST, GAMMA = 5, 6, 7, 8
SHIFT_RGB, SHIFT_HSV, GRAYSCALE, EQUALIZE = 9, 10, 11, 12
ROTATE, SHIFT_SCALE_ROTATE, RESIZE, RANDOM_SIZED_CROP = 13, 14, 15, 16
RANDOM_RESIZED_CROP, TRANSPOSE, ROT90, CHAIN = 17, 18, 19, 20
GRID_DISTORTION, ELASTIC = 21, 22
MODE_FUSED, MODE_PLAIN = 0, 1

GEOMETRIC = {HFLIP, VFLIP, RANDOM_CROP, PAD_TO_SIZE, ROTATE, SHIFT_SCALE_ROTATE, RESIZE, RANDOM_SIZED_CROP,
             RANDOM_RESIZED_CROP, TRANSPOSE, ROT90, GRID_DISTORTION, ELASTIC}
NAMES = {HFLIP: "HorizontalFlip", VFLIP: "VerticalFlip", RANDOM_CROP: "RandomCrop", PAD_TO_SIZE: "PadToSize",
         BRIGHTNESS: "Brightness", CONTRAST: "Contrast", BRIGHTNESS_CONTRAST: "BrightnessContrast",
         GAMMA: "Gamma", SHIFT_RGB: "ShiftRGB", SHIFT_HSV: "ShiftHSV", GRAYSCALE: "Grayscale",
         EQUALIZE: "Equalize", ROTATE: "Rotate", SHIFT_SCALE_ROTATE: "ShiftScaleRotate", RESIZE: "Resize",
         RANDOM_SIZED_CROP: "RandomSizedCrop", RANDOM_RESIZED_CROP: "RandomResizedCrop",
         TRANSPOSE: "Transpose", ROT90: "RandomRotate90", CHAIN: "Chain", GRID_DISTORTION: "GridDistortion",
         ELASTIC: "ElasticTransform"}


class Image(C.Structure):
    _fields_ = [("data", C.c_void_p), ("h", C.c_int32), ("w", C.c_int32), ("c", C.c_int32),
                ("reserved", C.c_int32), ("row_stride", C.c_int64)]


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


class SampleCfg(C.Structure):
    _fields_ = [("tid", C.c_int32), ("out_h", C.c_int32), ("out_w", C.c_int32), ("reserved", C.c_int32),
                ("p", C.c_double), ("lo", C.c_double * 4), ("hi", C.c_double * 4)]


class ChainCfg(C.Structure):
    _fields_ = [("out_h", C.c_int32), ("out_w", C.c_int32), ("mean", C.c_double * 3), ("std", C.c_double * 3),
                ("tile_h", C.c_int32), ("tile_w", C.c_int32), ("ctas_per_sm", C.c_int32), ("jitter", C.c_int32)]


assert C.sizeof(Image) == 32 and C.sizeof(Params) == 232 and C.sizeof(SampleCfg) == 88 and C.sizeof(ChainCfg) == 72


class AlbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libalb status {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()
P = C.POINTER
vp = C.c_void_p


def _declare(L):
    st = C.c_int
    L.alb_last_error.restype = C.c_char_p
    L.alb_version.restype = C.c_char_p
    L.alb_sample_params.argtypes = [P(SampleCfg), C.c_uint64, C.c_uint64, C.c_uint32, C.c_int32, C.c_int32,
                                    P(Params)]
    L.alb_sample_params.restype = st
    L.alb_sample_params_batch.argtypes = [P(SampleCfg), C.c_uint64, C.c_uint64, C.c_uint32, C.c_int32, vp, vp, vp,
                                          vp]
    L.alb_sample_params_batch.restype = st
    L.alb_output_shape.argtypes = [P(Params), C.c_int32, C.c_int32, P(C.c_int32), P(C.c_int32)]
    L.alb_output_shape.restype = st
    L.alb_workspace_size.argtypes = [C.c_int32, C.c_int32]
    L.alb_workspace_size.restype = C.c_size_t
    L.alb_apply.argtypes = [P(Params), P(Image), P(Image), P(Image), P(Image), vp, C.c_int32, vp, vp, vp,
                            C.c_size_t, vp]
    L.alb_apply.restype = st
    L.alb_apply_ragged.argtypes = [C.c_int32, C.c_int32, vp, vp, vp, vp, vp, vp, vp, C.c_int32, vp, vp, vp,
                                   C.c_size_t, vp, vp]
    L.alb_apply_ragged.restype = st
    L.alb_apply_ragged_static.argtypes = [C.c_int32, C.c_int32, vp, vp, vp, vp, vp]
    L.alb_apply_ragged_static.restype = st
    L.alb_selftest_bounded_wait.argtypes = [C.c_int32, vp, vp, vp, vp]
    L.alb_selftest_bounded_wait.restype = st
    L.alb_autotune_lookup.argtypes = [P(ChainCfg), C.c_int32, P(ChainCfg), P(C.c_int32)]
    L.alb_autotune_lookup.restype = st
    L.alb_autotune_save.argtypes = [C.c_char_p]
    L.alb_autotune_save.restype = st
    L.alb_autotune_load.argtypes = [C.c_char_p, P(C.c_int32)]
    L.alb_autotune_load.restype = st
    L.alb_bounds_violations.argtypes = [P(C.c_uint32), P(C.c_uint32), C.c_int32, P(C.c_int32)]
    L.alb_bounds_violations.restype = st
    L.alb_batch_workspace_size.argtypes = [P(ChainCfg), C.c_int32, C.c_int32]
    L.alb_batch_workspace_size.restype = C.c_size_t
    L.alb_apply_batch.argtypes = [P(ChainCfg), C.c_int32, vp, vp, vp, C.c_int32, vp, C.c_size_t, vp, vp]
    L.alb_apply_batch.restype = st
    L.alb_autotune_batch.argtypes = [P(ChainCfg), C.c_int32, vp, vp, vp, vp, C.c_size_t, C.c_int32, P(ChainCfg), vp]
    L.alb_autotune_batch.restype = st
    L.alb_apply_batch_targets.argtypes = [P(ChainCfg), C.c_int32, vp, vp, vp, vp, vp, vp, vp, C.c_int32, vp, vp,
                                          C.c_int32, vp, C.c_size_t, vp, vp]
    L.alb_apply_batch_targets.restype = st
    L.alb_sample_chain_box_safe.argtypes = [P(SampleCfg), C.c_uint64, C.c_uint64, C.c_uint32, C.c_int32, C.c_int32,
                                            P(C.c_float), C.c_int32, P(Params)]
    L.alb_sample_chain_box_safe.restype = st
    L.alb_sample_chain_box_safe_batch.argtypes = [P(SampleCfg), C.c_uint64, C.c_uint64, C.c_uint32, C.c_int32, vp,
                                                  vp, vp, C.c_int32, vp, vp, vp]
    L.alb_sample_chain_box_safe_batch.restype = st
    L.alb_f32_workspace_size.argtypes = [C.c_int32] * 4
    L.alb_f32_workspace_size.restype = C.c_size_t
    for name in ("alb_warp_affine_f32_fwd", "alb_photometric_f32_fwd"):
        f = getattr(L, name)
        f.argtypes = [C.c_int32] * 4 + [vp, vp, vp, vp]
        f.restype = st
    for name in ("alb_warp_affine_f32_bwd", "alb_photometric_f32_bwd"):
        f = getattr(L, name)
        f.argtypes = [C.c_int32] * 4 + [vp, vp, vp, vp, vp, vp, C.c_size_t, vp]
        f.restype = st


def bounds_checked() -> bool:
    """ALB_BOUNDS_CHECK=1 in the environment selects the bounds-checked build."""
    return os.environ.get("ALB_BOUNDS_CHECK", "") == "1"


def lib_path() -> str:
    return _build.CHECK_LIB if bounds_checked() else _build.LIB


def load(build_if_missing: bool = True):
    """Load libalb.so (building it in-tree with nvcc if needed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if bounds_checked():
                _build.build(check_bounds=True)
            elif not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"libalb.so not found at {path}; run paper_1809_06839_gb300.build.build()")
                _build.build()
            L = C.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


def _check(rc):
    if rc != ALB_OK:
        raise AlbError(rc, load().alb_last_error().decode())


def _cuda(t: torch.Tensor, what: str):
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor (libalb has no CPU path)")
    return t


def _stream(stream):
    if stream is None:
        return vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return vp(stream.cuda_stream)
    return vp(stream)


def _ptr(t):
    return None if t is None else vp(t.data_ptr())


# ---------------------------------------------------------------- descriptors
def image_desc(t: torch.Tensor) -> Image:
    """Descriptor of a uint8 (H, W, C) or (H, W) CUDA tensor with contiguous rows."""
    _cuda(t, "image")
    if t.dtype != torch.uint8:
        raise ValueError("images are uint8")
    if t.dim() == 2:
        h, w, c = t.shape[0], t.shape[1], 1
        if t.stride(1) != 1:
            raise ValueError("rows must be contiguous")
    else:
        h, w, c = t.shape
        if t.stride(2) != 1 or t.stride(1) != c:
            raise ValueError("pixels must be packed (HWC)")
    d = Image()
    d.data, d.h, d.w, d.c, d.reserved, d.row_stride = t.data_ptr(), h, w, c, 0, t.stride(0) if h > 0 else w * c
    return d


def descs_to_device(descs, device="cuda") -> torch.Tensor:
    """Pack a list of Image descriptors into a device buffer (n * 32 bytes)."""
    arr = (Image * len(descs))(*descs)
    host = torch.frombuffer(bytearray(arr), dtype=torch.uint8) if len(descs) else torch.zeros(0, dtype=torch.uint8)
    return host.to(device)


def params_to_device(params, device="cuda") -> torch.Tensor:
    arr = (Params * len(params))(*params)
    host = torch.frombuffer(bytearray(arr), dtype=torch.uint8) if len(params) else torch.zeros(0, dtype=torch.uint8)
    return host.to(device)


def params_from_device(buf: torch.Tensor):
    raw = bytes(buf.cpu().numpy().tobytes())
    n = len(raw) // C.sizeof(Params)
    return list((Params * n).from_buffer_copy(raw))


def sample_cfg(tid, p=1.0, out_h=0, out_w=0, lo=(), hi=()) -> SampleCfg:
    c = SampleCfg()
    c.tid, c.out_h, c.out_w, c.p = tid, out_h, out_w, p
    for i, v in enumerate(lo):
        c.lo[i] = v
    for i, v in enumerate(hi):
        c.hi[i] = v
    return c


IMAGENET_MEAN = (0.485, 0.456, 0.406)
IMAGENET_STD = (0.229, 0.224, 0.225)


def chain_cfg(out_h=224, out_w=224, mean=IMAGENET_MEAN, std=IMAGENET_STD, tile_h=0, tile_w=0, ctas_per_sm=0,
              jitter=0):
    c = ChainCfg()
    c.out_h, c.out_w = out_h, out_w
    for i in range(3):
        c.mean[i], c.std[i] = mean[i], std[i]
    c.tile_h, c.tile_w, c.ctas_per_sm, c.jitter = tile_h, tile_w, ctas_per_sm, jitter
    return c


# ---------------------------------------------------------------- the C ABI, same names
def alb_version() -> str:
    return load().alb_version().decode()


def alb_last_error() -> str:
    return load().alb_last_error().decode()


def alb_sample_params(cfg: SampleCfg, seed: int, stream_id: int, index: int, h: int, w: int) -> Params:
    p = Params()
    _check(load().alb_sample_params(C.byref(cfg), seed, stream_id, index, h, w, C.byref(p)))
    return p


def alb_sample_params_batch(cfg: SampleCfg, seed: int, stream_id: int, first_index: int, n: int,
                            images_dev: torch.Tensor, params_dev: torch.Tensor, dev_status=None, stream=None):
    _check(load().alb_sample_params_batch(C.byref(cfg), seed, stream_id, first_index, n, _ptr(images_dev),
                                          _ptr(params_dev), _ptr(dev_status), _stream(stream)))


def alb_output_shape(p: Params, h: int, w: int):
    oh, ow = C.c_int32(), C.c_int32()
    _check(load().alb_output_shape(C.byref(p), h, w, C.byref(oh), C.byref(ow)))
    return oh.value, ow.value


def alb_workspace_size(tid: int, n: int) -> int:
    return int(load().alb_workspace_size(tid, n))


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def alb_apply(p: Params, img: torch.Tensor, out: torch.Tensor | None = None, mask: torch.Tensor | None = None,
              mask_out: torch.Tensor | None = None, boxes: torch.Tensor | None = None,
              boxes_out: torch.Tensor | None = None, n_boxes_out: torch.Tensor | None = None,
              ws: torch.Tensor | None = None, stream=None):
    """Apply one transform to one image (and mask, boxes).  Allocates the
    output/workspace tensors that are not given; returns (out, mask_out,
    boxes_out, n_boxes_out)."""
    L = load()
    d_in = image_desc(img)
    oh, ow = alb_output_shape(p, d_in.h, d_in.w)
    if out is None:
        out = torch.empty((oh, ow, d_in.c), dtype=torch.uint8, device=img.device)
    d_out = image_desc(out)
    d_mi = d_mo = None
    if mask is not None:
        d_mi = image_desc(mask)
        geo = p.tid in GEOMETRIC
        if mask_out is None:
            shape = (oh, ow) if geo else (d_mi.h, d_mi.w)
            mask_out = torch.empty(shape + ((d_mi.c,) if mask.dim() == 3 else ()), dtype=torch.uint8,
                                   device=img.device)
        d_mo = image_desc(mask_out)
    nb = 0
    if boxes is not None:
        _cuda(boxes, "boxes")
        boxes = boxes.contiguous().float()
        nb = boxes.shape[0]
        if boxes_out is None:
            boxes_out = torch.empty_like(boxes)
        if n_boxes_out is None:
            n_boxes_out = torch.zeros(1, dtype=torch.int32, device=img.device)
    if ws is None:
        ws = workspace(alb_workspace_size(p.tid, 1), img.device)
    _check(L.alb_apply(C.byref(p), C.byref(d_in), C.byref(d_out), C.byref(d_mi) if d_mi else None,
                       C.byref(d_mo) if d_mo else None, _ptr(boxes), nb, _ptr(boxes_out), _ptr(n_boxes_out),
                       _ptr(ws), ws.numel(), _stream(stream)))
    return out, mask_out, boxes_out, n_boxes_out


def alb_apply_ragged(tid: int, n: int, params_dev, in_dev, out_dev, mask_in_dev=None, mask_out_dev=None,
                     boxes_dev=None, n_boxes_dev=None, box_cap=0, boxes_out_dev=None, n_boxes_out_dev=None,
                     ws=None, dev_status=None, stream=None):
    _check(load().alb_apply_ragged(tid, n, _ptr(params_dev), _ptr(in_dev), _ptr(out_dev), _ptr(mask_in_dev),
                                   _ptr(mask_out_dev), _ptr(boxes_dev), _ptr(n_boxes_dev), box_cap,
                                   _ptr(boxes_out_dev), _ptr(n_boxes_out_dev), _ptr(ws),
                                   0 if ws is None else ws.numel(), _ptr(dev_status), _stream(stream)))


def alb_apply_ragged_static(tid: int, n: int, params_dev, in_dev, out_dev, dev_status=None, stream=None):
    """alb_apply_ragged without a workspace: for callers that cannot allocate
    device memory; scratch is a static array inside libalb (<= 2048 images)."""
    _check(load().alb_apply_ragged_static(tid, n, _ptr(params_dev), _ptr(in_dev), _ptr(out_dev), _ptr(dev_status),
                                          _stream(stream)))


def alb_selftest_bounded_wait(spins: int, src_dev, out_dev, dev_status, stream=None):
    """Runs the bulk-copy kernels' timeout path on purpose (see alb.h)."""
    _check(load().alb_selftest_bounded_wait(spins, _ptr(src_dev), _ptr(out_dev), _ptr(dev_status), _stream(stream)))


def alb_autotune_lookup(cfg: ChainCfg, n: int):
    """The cached fused schedule for (current device, cfg, n), or None."""
    best = ChainCfg()
    found = C.c_int32(0)
    _check(load().alb_autotune_lookup(C.byref(cfg), n, C.byref(best), C.byref(found)))
    return best if found.value else None


def alb_autotune_save(path: str):
    _check(load().alb_autotune_save(os.fsencode(path)))


def alb_autotune_load(path: str) -> int:
    n = C.c_int32(0)
    _check(load().alb_autotune_load(os.fsencode(path), C.byref(n)))
    return n.value


def alb_bounds_violations(reset: bool = False):
    """(checked build?, violations counted, first failing source line)."""
    cnt, line, chk = C.c_uint32(0), C.c_uint32(0), C.c_int32(0)
    _check(load().alb_bounds_violations(C.byref(cnt), C.byref(line), int(reset), C.byref(chk)))
    return bool(chk.value), cnt.value, line.value


def alb_batch_workspace_size(cfg: ChainCfg, n: int, mode: int) -> int:
    return int(load().alb_batch_workspace_size(C.byref(cfg), n, mode))


def alb_apply_batch(cfg: ChainCfg, n: int, params_dev, in_dev, out_bf16: torch.Tensor, mode: int = MODE_FUSED,
                    ws=None, dev_status=None, stream=None):
    _cuda(out_bf16, "out")
    if ws is None:
        ws = workspace(alb_batch_workspace_size(cfg, n, mode), out_bf16.device)
    _check(load().alb_apply_batch(C.byref(cfg), n, _ptr(params_dev), _ptr(in_dev), _ptr(out_bf16), mode, _ptr(ws),
                                  ws.numel(), _ptr(dev_status), _stream(stream)))


def alb_autotune_batch(cfg: ChainCfg, n: int, params_dev, in_dev, out_bf16: torch.Tensor, ws=None, reps: int = 3,
                       stream=None) -> ChainCfg:
    """Times the fused kernel's candidate schedules on this batch, caches the
    fastest in the library and returns it (a copy of cfg with tile_h and
    ctas_per_sm set).  Synchronises the stream."""
    _cuda(out_bf16, "out")
    if ws is None:
        ws = workspace(alb_batch_workspace_size(cfg, n, MODE_FUSED), out_bf16.device)
    best = ChainCfg()
    _check(load().alb_autotune_batch(C.byref(cfg), n, _ptr(params_dev), _ptr(in_dev), _ptr(out_bf16), _ptr(ws),
                                     ws.numel(), reps, C.byref(best), _stream(stream)))
    return best


def alb_apply_batch_targets(cfg: ChainCfg, n: int, params_dev, in_dev, out_bf16: torch.Tensor, mask_in_dev=None,
                            mask_out_dev=None, boxes_dev=None, n_boxes_dev=None, box_cap=0, boxes_out_dev=None,
                            n_boxes_out_dev=None, mode: int = MODE_FUSED, ws=None, dev_status=None, stream=None):
    _cuda(out_bf16, "out")
    if ws is None:
        ws = workspace(alb_batch_workspace_size(cfg, n, mode), out_bf16.device)
    _check(load().alb_apply_batch_targets(C.byref(cfg), n, _ptr(params_dev), _ptr(in_dev), _ptr(out_bf16),
                                          _ptr(mask_in_dev), _ptr(mask_out_dev), _ptr(boxes_dev),
                                          _ptr(n_boxes_dev), box_cap, _ptr(boxes_out_dev), _ptr(n_boxes_out_dev),
                                          mode, _ptr(ws), ws.numel(), _ptr(dev_status), _stream(stream)))


def alb_sample_chain_box_safe(cfg: SampleCfg, seed: int, stream_id: int, index: int, h: int, w: int,
                              boxes) -> Params:
    import numpy as np
    b = np.ascontiguousarray(boxes, dtype=np.float32).reshape(-1, 4)
    p = Params()
    _check(load().alb_sample_chain_box_safe(C.byref(cfg), seed, stream_id, index, h, w,
                                            b.ctypes.data_as(C.POINTER(C.c_float)), b.shape[0], C.byref(p)))
    return p


def alb_sample_chain_box_safe_batch(cfg: SampleCfg, seed: int, stream_id: int, first_index: int, n: int, images_dev,
                                    boxes_dev, n_boxes_dev, box_cap: int, params_dev, dev_status=None, stream=None):
    _check(load().alb_sample_chain_box_safe_batch(C.byref(cfg), seed, stream_id, first_index, n, _ptr(images_dev),
                                                  _ptr(boxes_dev), _ptr(n_boxes_dev), box_cap, _ptr(params_dev),
                                                  _ptr(dev_status), _stream(stream)))


def alb_f32_workspace_size(B, Cc, H, W) -> int:
    return int(load().alb_f32_workspace_size(B, Cc, H, W))


def _f32_args(x, prm):
    _cuda(x, "x")
    if x.dtype != torch.float32 or not x.is_contiguous():
        raise ValueError("x must be a contiguous float32 NCHW CUDA tensor")
    B, Cc, H, W = x.shape
    return B, Cc, H, W


def alb_warp_affine_f32_fwd(x, prm, y=None, stream=None):
    B, Cc, H, W = _f32_args(x, prm)
    y = torch.empty_like(x) if y is None else y
    _check(load().alb_warp_affine_f32_fwd(B, Cc, H, W, _ptr(x), _ptr(prm.contiguous()), _ptr(y), _stream(stream)))
    return y


def alb_warp_affine_f32_bwd(x, prm, gy, gx=None, gprm=None, ws=None, stream=None):
    B, Cc, H, W = _f32_args(x, prm)
    gx = torch.empty_like(x) if gx is None else gx
    gprm = torch.empty((B, 4), dtype=torch.float32, device=x.device) if gprm is None else gprm
    ws = workspace(alb_f32_workspace_size(B, Cc, H, W), x.device) if ws is None else ws
    _check(load().alb_warp_affine_f32_bwd(B, Cc, H, W, _ptr(x), _ptr(prm.contiguous()), _ptr(gy.contiguous()),
                                          _ptr(gx), _ptr(gprm), _ptr(ws), ws.numel(), _stream(stream)))
    return gx, gprm


def alb_photometric_f32_fwd(x, prm, y=None, stream=None):
    B, Cc, H, W = _f32_args(x, prm)
    y = torch.empty_like(x) if y is None else y
    _check(load().alb_photometric_f32_fwd(B, Cc, H, W, _ptr(x), _ptr(prm.contiguous()), _ptr(y), _stream(stream)))
    return y


def alb_photometric_f32_bwd(x, prm, gy, gx=None, gprm=None, ws=None, stream=None):
    B, Cc, H, W = _f32_args(x, prm)
    gx = torch.empty_like(x) if gx is None else gx
    gprm = torch.empty((B, 3), dtype=torch.float32, device=x.device) if gprm is None else gprm
    ws = workspace(alb_f32_workspace_size(B, Cc, H, W), x.device) if ws is None else ws
    _check(load().alb_photometric_f32_bwd(B, Cc, H, W, _ptr(x), _ptr(prm.contiguous()), _ptr(gy.contiguous()),
                                          _ptr(gx), _ptr(gprm), _ptr(ws), ws.numel(), _stream(stream)))
    return gx, gprm
