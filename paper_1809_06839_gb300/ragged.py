"""Device-side ragged batches for libalb: packs image descriptors and parameter
records into device arrays and allocates outputs sized by each record.
Marshalling only; all pixel work happens in libalb.so."""
from __future__ import annotations

import torch

from . import alb
from .synth import Ragged, empty_ragged


def descs(rb: Ragged):
    out = []
    for i, (h, w, c) in enumerate(rb.shapes):
        d = alb.Image()
        d.data = rb.flat.data_ptr() + rb.offsets[i]
        d.h, d.w, d.c, d.reserved, d.row_stride = h, w, c, 0, w * c
        out.append(d)
    return out


class DeviceBatch:
    """A ragged batch resident on the GPU plus its descriptor array."""

    def __init__(self, rb: Ragged):
        if not rb.flat.is_cuda:
            raise ValueError("DeviceBatch needs a CUDA-resident Ragged batch")
        self.rb = rb
        self.descs = descs(rb)
        self.dev = alb.descs_to_device(self.descs, rb.flat.device)

    def __len__(self):
        return len(self.rb)

    @property
    def nbytes(self):
        return self.rb.nbytes


def output_batch(params, in_shapes, device="cuda", channels=None) -> DeviceBatch:
    shapes = []
    for p, (h, w, c) in zip(params, in_shapes):
        oh, ow = alb.alb_output_shape(p, h, w)
        shapes.append((oh, ow, channels or c))
    return DeviceBatch(empty_ragged(shapes, device=device))


def mask_output_batch(params, in_shapes, device="cuda") -> DeviceBatch:
    shapes = []
    for p, (h, w, c) in zip(params, in_shapes):
        if p.tid in alb.GEOMETRIC:
            oh, ow = alb.alb_output_shape(p, h, w)
        else:
            oh, ow = h, w
        shapes.append((oh, ow, c))
    return DeviceBatch(empty_ragged(shapes, device=device))


def to_device(rb: Ragged, device="cuda") -> Ragged:
    return Ragged(rb.flat.to(device), list(rb.offsets), list(rb.shapes))
