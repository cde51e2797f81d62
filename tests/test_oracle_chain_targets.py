"""Pins of the oracle's chain targets: instance-mask stacks and boxes through
the chain's crop / resize / flip, and the box-safe crop-window sampler."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1809_06839_gb300 import synth

CHAIN = O.make_cfg(O.CHAIN, out_h=224, out_w=224, lo=(0.08, 3 / 4, 0.6), hi=(1.0, 4 / 3, 1.4))
SMALL = O.make_cfg(O.CHAIN, out_h=40, out_w=56, lo=(0.08, 3 / 4, 0.6), hi=(1.0, 4 / 3, 1.4))


def resize_record(p):
    r = O.Params()
    r.tid, r.apply, r.out_h, r.out_w, r.ch, r.cw = O.RESIZE, 1, p.out_h, p.out_w, p.ch, p.cw
    return r


@pytest.mark.parametrize("planes", [1, 3, 8])
def test_chain_mask_is_crop_nearest_resize_then_flip(planes):
    h, w = 150, 211
    rng = np.random.default_rng(planes)
    mask = rng.integers(0, 2, (h, w, planes)).astype(np.uint8) * rng.integers(1, 255, planes).astype(np.uint8)
    for i in range(6):
        p = O.sample_params(SMALL, 17, 20, i, h, w)
        got = O.chain_mask(p, mask)
        win = np.ascontiguousarray(mask[p.y0:p.y0 + p.ch, p.x0:p.x0 + p.cw])
        ref = O.apply_mask(resize_record(p), win)        # nearest resize, pinned in test_oracle_geometric
        if p.flip:
            ref = ref[:, ::-1]
        assert np.array_equal(got, ref), i


def test_chain_boxes_compose_the_window_map_and_the_flip():
    h, w = 300, 420
    for i in range(20):
        p = O.sample_params(CHAIN, 5, 20, i, h, w)
        boxes = synth.random_boxes(h, w, i, 5)
        got = O.chain_boxes(p, boxes)
        r = resize_record(p)
        shifted = boxes - np.array([p.x0, p.y0, p.x0, p.y0], np.float32)
        ref = O.apply_boxes(r, p.ch, p.cw, np.clip(shifted, 0, [p.cw, p.ch, p.cw, p.ch]).astype(np.float32))
        if p.flip:
            ref = np.stack([224 - ref[:, 2], ref[:, 1], 224 - ref[:, 0], ref[:, 3]], axis=1)
        assert got.shape == ref.shape
        assert np.abs(got - ref).max(initial=0) <= 1e-4


def test_box_safe_window_contains_the_union():
    h, w = 333, 480
    rng = np.random.default_rng(0)
    lo_hits = hi_hits = 0
    for i in range(300):
        n = int(rng.integers(1, 6))
        x1 = rng.uniform(-20, w - 10, n); y1 = rng.uniform(-20, h - 10, n)
        boxes = np.stack([x1, y1, x1 + rng.uniform(2, 150, n), y1 + rng.uniform(2, 150, n)], 1).astype(np.float32)
        p = O.sample_chain_box_safe(CHAIN, 3, 20, i, h, w, boxes)
        c = np.clip(boxes, 0, [w, h, w, h])
        c = c[(c[:, 2] > c[:, 0]) & (c[:, 3] > c[:, 1])]
        ux1, uy1 = math.floor(c[:, 0].min()), math.floor(c[:, 1].min())
        ux2, uy2 = math.ceil(c[:, 2].max()), math.ceil(c[:, 3].max())
        assert 0 <= p.x0 <= ux1 and p.x0 + p.cw >= ux2 and p.x0 + p.cw <= w
        assert 0 <= p.y0 <= uy1 and p.y0 + p.ch >= uy2 and p.y0 + p.ch <= h
        lo_hits += p.x0 == 0
        hi_hits += p.x0 == ux1
        # every box inside the image stays whole: mapped, none dropped
        inside = boxes[(boxes[:, 0] >= 0) & (boxes[:, 1] >= 0) & (boxes[:, 2] <= w) & (boxes[:, 3] <= h)]
        out = O.chain_boxes(p, inside)
        assert len(out) == len(inside)
        sx, sy = 224 / p.cw, 224 / p.ch
        ext = np.stack([(inside[:, 0] - p.x0) * sx, (inside[:, 1] - p.y0) * sy,
                        (inside[:, 2] - p.x0) * sx, (inside[:, 3] - p.y0) * sy], 1)
        if p.flip:
            ext = np.stack([224 - ext[:, 2], ext[:, 1], 224 - ext[:, 0], ext[:, 3]], 1)
        assert np.abs(out - ext).max(initial=0) <= 1e-3
    assert lo_hits > 0 and hi_hits > 0


def test_box_safe_without_boxes_is_the_chain_sampler():
    for i in range(40):
        a = O.sample_chain_box_safe(CHAIN, 9, 20, i, 400, 500, np.zeros((0, 4), np.float32))
        b = O.sample_params(CHAIN, 9, 20, i, 400, 500)
        for f in ("x0", "y0", "ch", "cw", "flip", "k", "alpha", "beta", "sat", "out_h", "out_w", "apply"):
            assert getattr(a, f) == getattr(b, f), (i, f)
    # boxes entirely outside the image count as no boxes
    out = np.array([[-50, -50, -10, -10], [600, 10, 700, 20]], np.float32)
    a = O.sample_chain_box_safe(CHAIN, 9, 20, 3, 400, 500, out)
    b = O.sample_params(CHAIN, 9, 20, 3, 400, 500)
    assert (a.x0, a.y0, a.ch, a.cw) == (b.x0, b.y0, b.ch, b.cw)
