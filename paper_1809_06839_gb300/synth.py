"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This module holds none of the augmentation arithmetic: it only makes images,
masks and boxes with the shapes and statistics of the paper's workloads
(natural-image-like smooth textures, blob-structured label masks, boxes of
16-400 px), because the paper's benchmark images and datasets (Sec. III,
Table I; Mapillary Vistas, Inria, Figs. 2-3) are not available.

* value-noise texture: per image and channel, two lattices of uniform values
  in [0, 255] (spacing 64 px and 16 px, weights 0.7 / 0.3), each
  interpolated with smoothstep-weighted bilinear blending, rounded and
  clamped to uint8.
* blob label mask: argmax over ``n_classes`` single-octave value-noise
  fields (spacing 96 px) -> uint8 labels.
* boxes: n ~ U_int[1, 50], side lengths ~ U[16, 400] clipped to the image,
  top-left uniform so the box fits; float32 xyxy in pixel-edge coordinates.

Random lattice values come from numpy's ``default_rng`` keyed by
(seed, image index, stream), so CPU and GPU generation agree on the lattice;
the interpolation runs on the requested torch device.  Tests generate on the
CPU and copy bytes to the GPU, so both sides see identical inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

BASE_SEED = 1809


def _rng(seed: int, index: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(index), int(stream)])


def _smooth_field(lattice: torch.Tensor, h: int, w: int, spacing: int) -> torch.Tensor:
    """lattice (Ly, Lx, C) float32 -> (h, w, C) smoothstep-bilinear field."""
    dev = lattice.device
    ys = torch.arange(h, device=dev, dtype=torch.float32) / spacing
    xs = torch.arange(w, device=dev, dtype=torch.float32) / spacing
    iy = ys.floor().long()
    ix = xs.floor().long()
    ty = ys - iy.float()
    tx = xs - ix.float()
    ty = ty * ty * (3 - 2 * ty)
    tx = tx * tx * (3 - 2 * tx)
    a = lattice[iy][:, ix]
    b = lattice[iy][:, ix + 1]
    c = lattice[iy + 1][:, ix]
    d = lattice[iy + 1][:, ix + 1]
    ty = ty[:, None, None]
    tx = tx[None, :, None]
    top = a + (b - a) * tx
    bot = c + (d - c) * tx
    return top + (bot - top) * ty


def value_noise_image(h: int, w: int, index: int = 0, seed: int = BASE_SEED, channels: int = 3,
                      device="cpu") -> torch.Tensor:
    """uint8 (h, w, channels) smooth texture, deterministic in (seed, index)."""
    out = torch.zeros((h, w, channels), dtype=torch.float32, device=device)
    for octave, (spacing, weight) in enumerate(((64, 0.7), (16, 0.3))):
        ly, lx = h // spacing + 2, w // spacing + 2
        lat = _rng(seed, index, octave).uniform(0.0, 255.0, size=(ly, lx, channels))
        lat_t = torch.from_numpy(lat.astype(np.float32)).to(device)
        out += weight * _smooth_field(lat_t, h, w, spacing)
    return out.round().clamp_(0, 255).to(torch.uint8)


def blob_mask(h: int, w: int, index: int = 0, seed: int = BASE_SEED, n_classes: int = 20,
              device="cpu") -> torch.Tensor:
    """uint8 (h, w) label mask with blob-shaped regions of n_classes labels."""
    spacing = 96
    ly, lx = h // spacing + 2, w // spacing + 2
    lat = _rng(seed, index, 100).uniform(0.0, 1.0, size=(ly, lx, n_classes))
    lat_t = torch.from_numpy(lat.astype(np.float32)).to(device)
    return _smooth_field(lat_t, h, w, spacing).argmax(dim=2).to(torch.uint8)


def random_boxes(h: int, w: int, index: int = 0, seed: int = BASE_SEED, n_max: int = 50,
                 side_lo: float = 16.0, side_hi: float = 400.0) -> np.ndarray:
    """float32 (n, 4) xyxy boxes inside [0, w] x [0, h]."""
    r = _rng(seed, index, 200)
    n = int(r.integers(1, n_max + 1))
    bw = np.minimum(r.uniform(side_lo, side_hi, n), w)
    bh = np.minimum(r.uniform(side_lo, side_hi, n), h)
    x1 = r.uniform(0, 1, n) * (w - bw)
    y1 = r.uniform(0, 1, n) * (h - bh)
    return np.stack([x1, y1, x1 + bw, y1 + bh], axis=1).astype(np.float32)


def uniform_sizes(n: int, lo: int, hi: int, seed: int = BASE_SEED, stream: int = 300):
    """n (h, w) pairs, each side uniform in [lo, hi]."""
    r = _rng(seed, 0, stream)
    hw = r.integers(lo, hi + 1, size=(n, 2))
    return [(int(a), int(b)) for a, b in hw]


ALIGN = 256


@dataclass
class Ragged:
    """A ragged batch of HWC uint8 images packed in one flat buffer.

    Image i occupies ``flat[offsets[i] : offsets[i] + h*w*c]`` (contiguous rows,
    each image 256-byte aligned)."""
    flat: torch.Tensor
    offsets: list
    shapes: list            # (h, w, c)

    def __len__(self):
        return len(self.shapes)

    def image(self, i: int) -> torch.Tensor:
        h, w, c = self.shapes[i]
        o = self.offsets[i]
        return self.flat[o:o + h * w * c].view(h, w, c)

    @property
    def nbytes(self) -> int:
        return sum(h * w * c for h, w, c in self.shapes)


def layout(shapes) -> tuple[list, int]:
    offs, total = [], 0
    for h, w, c in shapes:
        offs.append(total)
        total += int(math.ceil(h * w * c / ALIGN)) * ALIGN
    return offs, max(total, ALIGN)


def empty_ragged(shapes, device="cpu", pin: bool = False) -> Ragged:
    offs, total = layout(shapes)
    flat = torch.empty(total, dtype=torch.uint8, device=device, pin_memory=pin)
    return Ragged(flat, offs, [tuple(s) for s in shapes])


def ragged_noise(sizes, seed: int = BASE_SEED, device="cpu", channels: int = 3,
                 first_index: int = 0) -> Ragged:
    shapes = [(h, w, channels) for h, w in sizes]
    rb = empty_ragged(shapes, device=device)
    for i, (h, w) in enumerate(sizes):
        rb.image(i).copy_(value_noise_image(h, w, first_index + i, seed, channels, device=device))
    return rb


def ragged_masks(sizes, seed: int = BASE_SEED, device="cpu", n_classes: int = 20) -> Ragged:
    shapes = [(h, w, 1) for h, w in sizes]
    rb = empty_ragged(shapes, device=device)
    for i, (h, w) in enumerate(sizes):
        rb.image(i).copy_(blob_mask(h, w, i, seed, n_classes, device=device)[:, :, None])
    return rb


def instance_stacks(sizes, planes, seed: int = BASE_SEED, device="cpu") -> Ragged:
    """Per image an N-plane instance stack (uint8 HWC, c = N): plane k is the
    binary mask (255) of blob class k of a 20-class blob label mask."""
    shapes = [(h, w, n) for (h, w), n in zip(sizes, planes)]
    rb = empty_ragged(shapes, device=device)
    for i, ((h, w), n) in enumerate(zip(sizes, planes)):
        lab = blob_mask(h, w, i, seed, 20, device=device)
        k = torch.arange(n, device=lab.device, dtype=lab.dtype)
        rb.image(i).copy_((lab[:, :, None] == k).to(torch.uint8) * 255)
    return rb


def float_images(b: int, c: int, h: int, w: int, seed: int = BASE_SEED, device="cpu") -> torch.Tensor:
    g = torch.Generator(device="cpu").manual_seed(seed)
    return torch.rand((b, c, h, w), generator=g, dtype=torch.float32).to(device)


def float_normal(shape, seed: int = BASE_SEED + 1, device="cpu") -> torch.Tensor:
    g = torch.Generator(device="cpu").manual_seed(seed)
    return torch.randn(shape, generator=g, dtype=torch.float32).to(device)
