"""Shared test helpers: parameter-record conversion between the oracle's and
the library's ctypes layouts (field by field, by name), workload configs and
oracle runs over ragged batches.  No method arithmetic lives here."""
import numpy as np

import oracle as O

FIELDS = ["tid", "apply", "in_h", "in_w", "out_h", "out_w", "y0", "x0", "ch", "cw", "flip", "k", "alpha", "beta",
          "gamma", "sat", "angle", "scale", "dx", "dy"]
ARRAYS = ["shift", "m", "q"]


def to_lib(op, alb):
    """Oracle Params -> library Params (same meaning, separate layouts)."""
    p = alb.Params()
    for f in FIELDS:
        setattr(p, f, getattr(op, f))
    for f in ARRAYS:
        for i, v in enumerate(getattr(op, f)):
            getattr(p, f)[i] = v
    return p


def same_params(a, b, rel_m=0.0):
    for f in FIELDS:
        if getattr(a, f) != getattr(b, f):
            return f"{f}: {getattr(a, f)} != {getattr(b, f)}"
    for f in ("shift", "q"):
        if list(getattr(a, f)) != list(getattr(b, f)):
            return f"{f}: {list(getattr(a, f))} != {list(getattr(b, f))}"
    ma, mb = np.array(list(a.m)), np.array(list(b.m))
    if np.any(np.abs(ma - mb) > rel_m * np.maximum(1.0, np.abs(ma))):
        return f"m: {ma} != {mb}"
    return None


# The per-transform suite: sampling configurations of each transform
# (ranges of the ImageNet-like per-transform workload).
def suite_cfgs():
    return {
        "HorizontalFlip": O.make_cfg(O.HFLIP, p=1.0),
        "VerticalFlip": O.make_cfg(O.VFLIP, p=1.0),
        "Rotate": O.make_cfg(O.ROTATE, lo=(-90.0,), hi=(90.0,)),
        "ShiftScaleRotate": O.make_cfg(O.SHIFT_SCALE_ROTATE, lo=(-0.0625, 0.9, -45.0), hi=(0.0625, 1.1, 45.0)),
        "Brightness": O.make_cfg(O.BRIGHTNESS, lo=(-20.0,), hi=(20.0,)),
        "Contrast": O.make_cfg(O.CONTRAST, lo=(0.8,), hi=(1.2,)),
        "Gamma": O.make_cfg(O.GAMMA, lo=(0.8,), hi=(1.2,)),
        "ShiftRGB": O.make_cfg(O.SHIFT_RGB, lo=(-20.0, -20.0, -20.0), hi=(20.0, 20.0, 20.0)),
        "ShiftHSV": O.make_cfg(O.SHIFT_HSV, lo=(-20.0, -30.0, -20.0), hi=(20.0, 30.0, 20.0)),
        "Grayscale": O.make_cfg(O.GRAYSCALE, p=1.0),
        "RandomCrop64": O.make_cfg(O.RANDOM_CROP, out_h=64, out_w=64),
        "PadToSize512": O.make_cfg(O.PAD_TO_SIZE, out_h=512, out_w=512),
        "Resize512": O.make_cfg(O.RESIZE, out_h=512, out_w=512),
        "RandomSizedCrop512": O.make_cfg(O.RANDOM_SIZED_CROP, out_h=512, out_w=512, lo=(0.25,), hi=(1.0,)),
        "Equalize": O.make_cfg(O.EQUALIZE, p=1.0),
    }


EXTRA_CFGS = {
    "BrightnessContrast": O.make_cfg(O.BRIGHTNESS_CONTRAST, lo=(0.8, -20.0), hi=(1.2, 20.0)),
    "Transpose": O.make_cfg(O.TRANSPOSE, p=1.0),
    "RandomRotate90": O.make_cfg(O.ROT90, p=1.0),
    "RandomResizedCrop224": O.make_cfg(O.RANDOM_RESIZED_CROP, out_h=224, out_w=224, lo=(0.08, 3 / 4),
                                       hi=(1.0, 4 / 3)),
    "HFlipHalf": O.make_cfg(O.HFLIP, p=0.5),
    "GridDistortion": O.make_cfg(O.GRID_DISTORTION, lo=(-0.3, 5), hi=(0.3, 5)),
    "ElasticTransform": O.make_cfg(O.ELASTIC, lo=(8.0, 4)),
}


def cfg_to_lib(oc, alb):
    c = alb.SampleCfg()
    c.tid, c.out_h, c.out_w, c.p = oc.tid, oc.out_h, oc.out_w, oc.p
    for i in range(4):
        c.lo[i], c.hi[i] = oc.lo[i], oc.hi[i]
    return c


CHAIN_CFG = dict(out_h=224, out_w=224, lo=(0.08, 3 / 4, 0.6), hi=(1.0, 4 / 3, 1.4))
