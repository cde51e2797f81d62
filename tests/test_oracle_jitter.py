"""Pins of the oracle's colour jitter, mode 1 (random order of brightness,
contrast and saturation, a contrast pivot at the image mean, uint8 after each
op): exact rational arithmetic, closed forms of special factors, the
permutation order and the sampler's order draw."""
import itertools
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle as O
from paper_1809_06839_gb300 import synth
from test_oracle_targets import fmaf_exact

CHAIN = O.make_cfg(O.CHAIN, out_h=24, out_w=20, lo=(0.08, 3 / 4, 0.6), hi=(1.0, 4 / 3, 1.4))
NAMES = "BCS"


def rne_u8(q: Fraction) -> int:
    return max(0, min(255, round(q)))      # Python rounds a Fraction half to even


def grey_int(img):
    """Integer BT.601 grey per pixel, from the oracle's Grayscale transform
    (pinned exactly in test_oracle_color)."""
    p = O.sample_params(O.make_cfg(O.GRAYSCALE, p=1.0), 1, 2, 0, img.shape[0], img.shape[1])
    return O.apply_image(p, np.ascontiguousarray(img))[:, :, 0].astype(np.int64)


def pivot(img) -> int:
    g = grey_int(img)
    return round(Fraction(int(g.sum()), g.size))


def exact_op(op, x, p):
    if op == "B":
        return np.vectorize(lambda v: rne_u8(Fraction(p.beta) * int(v)))(x)
    if op == "C":
        m = pivot(x.astype(np.uint8))
        return np.vectorize(lambda v: rne_u8(m + Fraction(p.alpha) * (int(v) - m)))(x)
    s = float(np.float32(p.sat))
    out = np.zeros_like(x)
    for idx in np.ndindex(x.shape[:2]):
        R, G, B = (float(v) for v in x[idx])
        grey = fmaf_exact(np.float32(0.114), B, fmaf_exact(np.float32(0.587), G, float(np.float32(0.299) * np.float32(R))))
        for c in range(3):
            d = float(np.float32(float(x[idx][c])) - np.float32(grey))
            out[idx][c] = rne_u8(Fraction(fmaf_exact(s, d, grey)))
    return out


def test_permutation_index_lists_every_order_once():
    perms = [tuple(O.jitter_op(k, i) for i in range(3)) for k in range(6)]
    assert perms == list(itertools.permutations(range(3)))
    assert O.jitter_op(6, 0) == -1 and O.jitter_op(0, 3) == -1


@pytest.mark.parametrize("k", range(6))
def test_mode1_chain_is_composition_of_exact_steps(k):
    h, w = 60, 84
    img = synth.value_noise_image(h, w, 11 + k).numpy()
    p = O.sample_params(CHAIN, 1809, 20, k, h, w)
    p.k = k
    got = O.chain_image(p, img, jitter=1)
    r = O.Params()
    r.tid, r.apply, r.out_h, r.out_w, r.ch, r.cw = O.RESIZE, 1, 24, 20, p.ch, p.cw
    x = O.apply_image(r, np.ascontiguousarray(img[p.y0:p.y0 + p.ch, p.x0:p.x0 + p.cw])).astype(np.int64)
    if p.flip:
        x = x[:, ::-1]
    order = list(itertools.permutations(NAMES))[k]
    for op in order:
        x = exact_op(op, x, p)
    kc, mc = O.normalize_consts()
    ref = np.zeros((3, 24, 20), np.float32)
    for c in range(3):
        ref[c] = np.vectorize(lambda v: fmaf_exact(float(v), kc[c], mc[c]))(x[:, :, c])
    ref_bits = torch.from_numpy(ref).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(got, ref_bits)


@pytest.mark.parametrize("k", range(6))
def test_unit_factors_leave_the_image_unchanged(k):
    img = synth.value_noise_image(33, 47, k).numpy()
    p = O.Params()
    p.alpha = p.beta = p.sat = 1.0
    p.k = k
    assert np.array_equal(O.jitter_mode1(p, img), img)


def test_zero_contrast_first_gives_the_pivot_everywhere():
    img = synth.value_noise_image(41, 29, 5).numpy()
    p = O.Params()
    p.alpha, p.beta, p.sat, p.k = 0.0, 1.0, 1.0, 2      # C, B, S
    out = O.jitter_mode1(p, img)
    assert np.all(out == pivot(img))
    assert O.contrast_pivot(img) == pivot(img)


def test_contrast_pivot_follows_the_earlier_ops():
    img = synth.value_noise_image(37, 51, 8).numpy()
    p = O.Params()
    p.alpha, p.beta, p.sat = 0.0, 0.5, 1.0
    p.k = 0                                              # B then C: pivot of the darkened image
    dark = np.vectorize(lambda v: rne_u8(Fraction(0.5) * int(v)))(img).astype(np.uint8)
    assert np.all(O.jitter_mode1(p, img) == pivot(dark))
    p.k = 2                                              # C then B: half of the original pivot
    assert np.all(O.jitter_mode1(p, img) == rne_u8(Fraction(0.5) * pivot(img)))


@pytest.mark.parametrize("k", [0, 1])
def test_zero_brightness_first_gives_black(k):
    img = synth.value_noise_image(20, 30, 3).numpy()
    p = O.Params()
    p.alpha, p.beta, p.sat, p.k = 1.3, 0.0, 0.7, k
    assert not O.jitter_mode1(p, img).any()


@pytest.mark.parametrize("s", [0.0, 0.6, 1.4])
def test_saturation_of_grey_pixels_is_identity(s):
    v = np.arange(256, dtype=np.uint8)
    img = np.repeat(v[None, :, None], 3, axis=2)
    p = O.Params()
    p.alpha, p.beta, p.sat, p.k = 1.0, 1.0, s, 4
    assert np.array_equal(O.jitter_mode1(p, img), img)


def test_sampled_order_covers_all_permutations():
    ks = [O.sample_params(CHAIN, 3, 20, i, 300, 300).k for i in range(600)]
    counts = np.bincount(ks, minlength=6)
    assert len(counts) == 6 and counts.min() > 60          # ~100 each
