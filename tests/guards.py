"""Guard bytes around kernel outputs: output images laid out with a guard
region after each one (and before the first), all pre-filled with a sentinel;
after the launch every byte outside the images must still hold it, so a
kernel that writes past an image's last byte (or before its first) fails
the test instead of passing silently."""
import torch

from paper_1809_06839_gb300.ragged import DeviceBatch
from paper_1809_06839_gb300.synth import Ragged
from paper_1809_06839_gb300 import alb

SENTINEL = 0xA5
GUARD = 512


def guarded_empty(shapes, device):
    offs, pos = [], GUARD
    for h, w, c in shapes:
        offs.append(pos)
        pos += (h * w * c + 255) // 256 * 256 + GUARD
    flat = torch.full((pos,), SENTINEL, dtype=torch.uint8, device=device)
    return Ragged(flat, offs, [tuple(s) for s in shapes])


def guarded_output_batch(params, in_shapes, device, mask=False):
    shapes = []
    for p, (h, w, c) in zip(params, in_shapes):
        if mask and p.tid not in alb.GEOMETRIC:
            oh, ow = h, w
        else:
            oh, ow = alb.alb_output_shape(p, h, w)
        shapes.append((oh, ow, c))
    return DeviceBatch(guarded_empty(shapes, device))


def assert_guards(batch, what=""):
    rb = batch.rb
    inside = torch.zeros(rb.flat.numel(), dtype=torch.bool, device=rb.flat.device)
    for o, (h, w, c) in zip(rb.offsets, rb.shapes):
        inside[o:o + h * w * c] = True
    bad = (rb.flat != SENTINEL) & ~inside
    n = int(bad.sum().item())
    assert n == 0, (what, "bytes written outside the output images", n)
