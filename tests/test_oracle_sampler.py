"""Pins of the oracle's parameter sampler: Philox4x32-10, the uniform and
integer draws built on it, the per-transform samplers and the warp geometry.
These run on the CPU only (no GPU, no CUDA library)."""
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, rhs = line.split("->")
        a = [int(v, 16) for v in lhs.split()]
        b = [int(v, 16) for v in rhs.split()]
        rows.append((a[:4], a[4:], b))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert list(O.philox4x32_10(ctr, key)) == expect


def test_stream_counter_layout():
    # block j of stream (seed, stream_id, index) is Philox((j, index, sid_lo, sid_hi), seed)
    seed, sid, idx = 0x0123456789ABCDEF, 0xFEDC_BA98_0000_0007, 42
    words = O.stream_words(seed, sid, idx, 12)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(3):
        blk = O.philox4x32_10([j, idx, sid & 0xFFFFFFFF, sid >> 32], key)
        assert list(words[4 * j:4 * j + 4]) == list(blk)


def test_uniform01_is_53_bit_grid():
    u = O.stream_uniform01(7, 1, 3, 20000)
    assert (u >= 0).all() and (u < 1).all()
    k = u * 2.0 ** 53
    assert np.array_equal(k, np.floor(k))           # exact multiples of 2^-53
    w = O.stream_words(7, 1, 3, 4)
    expect0 = ((int(w[0]) >> 5) * 2 ** 26 + (int(w[1]) >> 6)) / 2.0 ** 53
    assert u[0] == expect0
    assert abs(u.mean() - 0.5) < 0.01


def test_randint_power_of_two_is_high_bits():
    # for a range of 2^k the multiply-shift takes the k high bits, never rejects
    for k in (1, 5, 16):
        r = O.stream_randint(11, 2, 5, 2 ** k - 1, 64)
        w = O.stream_words(11, 2, 5, 64)
        assert np.array_equal(r.astype(np.int64), w.astype(np.int64) >> (32 - k))


def test_randint_rejection_removes_bias():
    # range 3*2^29: plain multiply-shift maps 3, 3 and 2 of every 8 words to
    # the residues 0, 1, 2 (mod 3) -> probability 1/4 for residue 2; with
    # Lemire's rejection (words = 0, 3 mod 8 rejected) each residue gets 1/3.
    n = 3 * 2 ** 29
    r = O.stream_randint(5, 9, 0, n - 1, 30000).astype(np.int64)
    assert r.min() >= 0 and r.max() <= n - 1
    frac2 = np.mean(r % 3 == 2)
    assert abs(frac2 - 1 / 3) < 0.02, frac2


def test_randint_bounds_and_coverage():
    r = O.stream_randint(3, 4, 5, 6, 5000)
    assert set(r.tolist()) == set(range(7))


def test_sampler_is_deterministic_and_keyed():
    cfg = O.make_cfg(O.SHIFT_SCALE_ROTATE, lo=(-0.0625, 0.9, -45), hi=(0.0625, 1.1, 45))
    a = O.sample_params(cfg, 1809, 14, 3, 400, 500)
    b = O.sample_params(cfg, 1809, 14, 3, 400, 500)
    c = O.sample_params(cfg, 1809, 14, 4, 400, 500)
    assert bytes(a) == bytes(b)
    assert bytes(a) != bytes(c)


@pytest.mark.parametrize("idx", range(40))
def test_sampler_ranges(idx):
    h, w = 333 + 4 * idx, 500 - 3 * idx
    s = O.sample_params(O.make_cfg(O.RANDOM_CROP, out_h=64, out_w=64), 1, 3, idx, h, w)
    assert 0 <= s.y0 <= h - 64 and 0 <= s.x0 <= w - 64 and (s.out_h, s.out_w) == (64, 64)
    s = O.sample_params(O.make_cfg(O.BRIGHTNESS_CONTRAST, lo=(0.8, -20), hi=(1.2, 20)), 1, 7, idx, h, w)
    assert 0.8 <= s.alpha < 1.2 and -20 <= s.beta < 20
    s = O.sample_params(O.make_cfg(O.SHIFT_SCALE_ROTATE, lo=(-0.0625, 0.9, -45), hi=(0.0625, 1.1, 45)),
                        1, 14, idx, h, w)
    assert -0.0625 <= s.dx < 0.0625 and -0.0625 <= s.dy < 0.0625
    assert 0.9 <= s.scale < 1.1 and -45 <= s.angle < 45
    s = O.sample_params(O.make_cfg(O.RANDOM_SIZED_CROP, out_h=512, out_w=512, lo=(0.25,), hi=(1.0,)),
                        1, 16, idx, h, w)
    m = min(h, w)
    assert np.ceil(0.25 * m) <= s.ch <= m and s.ch == s.cw
    assert 0 <= s.y0 <= h - s.ch and 0 <= s.x0 <= w - s.cw
    s = O.sample_params(O.make_cfg(O.PAD_TO_SIZE, out_h=512, out_w=512), 1, 4, idx, h, w)
    assert (s.out_h, s.out_w) == (512, 512) and s.y0 == (512 - h) // 2 and s.x0 == (512 - w) // 2


def test_probability_draw():
    cfg = O.make_cfg(O.HFLIP, p=0.5)
    hits = [O.sample_params(cfg, 9, 1, i, 10, 10).apply for i in range(4000)]
    assert abs(np.mean(hits) - 0.5) < 0.03
    assert all(O.sample_params(O.make_cfg(O.HFLIP, p=0.0), 9, 1, i, 10, 10).apply == 0 for i in range(50))
    assert all(O.sample_params(O.make_cfg(O.HFLIP, p=1.0), 9, 1, i, 10, 10).apply == 1 for i in range(50))


def test_rrc_distribution_and_fit():
    cfg = O.make_cfg(O.RANDOM_RESIZED_CROP, out_h=224, out_w=224, lo=(0.08, 3 / 4), hi=(1.0, 4 / 3))
    areas, ratios = [], []
    for i in range(3000):
        h, w = 256 + (i * 37) % 769, 256 + (i * 91) % 769
        p = O.sample_params(cfg, 1809, 17, i, h, w)
        assert 1 <= p.ch <= h and 1 <= p.cw <= w
        assert 0 <= p.y0 <= h - p.ch and 0 <= p.x0 <= w - p.cw
        areas.append(p.ch * p.cw / (h * w))
        ratios.append(p.cw / p.ch)
    areas, ratios = np.array(areas), np.array(ratios)
    # rounding of the sides moves area/ratio slightly outside the sampled ranges
    assert areas.min() > 0.07 and areas.max() <= 1.0
    assert ratios.min() > 0.7 and ratios.max() < 1.4
    # log-ratio is uniform: its mean is ~0
    assert abs(np.log(ratios).mean()) < 0.02


def test_rrc_fallback_centre_crop():
    # a 10 x 1000 strip: no sampled crop with aspect in [3/4, 4/3] fits, so the
    # fallback takes the full height and the widest allowed aspect, centred.
    cfg = O.make_cfg(O.RANDOM_RESIZED_CROP, out_h=8, out_w=8, lo=(0.9, 3 / 4), hi=(1.0, 4 / 3))
    p = O.sample_params(cfg, 1, 1, 0, 10, 1000)
    assert (p.ch, p.cw) == (10, 13)
    assert (p.y0, p.x0) == (0, (1000 - 13) // 2)


def _T(tx, ty):
    return np.array([[1, 0, tx], [0, 1, ty], [0, 0, 1]], dtype=np.float64)


@pytest.mark.parametrize("angle,scale,dx,dy,h,w", [
    (30.0, 1.0, 0.0, 0.0, 100, 140), (-45.0, 0.9, 0.05, -0.03, 333, 500),
    (90.0, 1.1, -0.0625, 0.0625, 64, 64), (0.0, 1.0, 0.0, 0.0, 7, 9)])
def test_warp_geometry_matches_matrix_composition(angle, scale, dx, dy, h, w):
    p = O.Params()
    p.tid, p.apply, p.angle, p.scale, p.dx, p.dy = O.SHIFT_SCALE_ROTATE, 1, angle, scale, dx, dy
    O.warp_geometry(p, h, w)
    t = np.deg2rad(angle)
    R = np.array([[np.cos(t), np.sin(t), 0], [-np.sin(t), np.cos(t), 0], [0, 0, 1]])
    S = np.diag([scale, scale, 1.0])
    cx, cy = (w - 1) / 2, (h - 1) / 2
    M = _T(cx + dx * w, cy + dy * h) @ S @ R @ _T(-cx, -cy)
    got = np.array(list(p.m)).reshape(2, 3)
    assert np.allclose(got, M[:2], atol=1e-9)
    # Q16 inverse is the rounded inverse of M
    Minv = np.linalg.inv(M)
    q = np.array(list(p.q), dtype=np.float64).reshape(2, 3)
    assert np.abs(q - np.rint(Minv[:2] * 65536)).max() <= 1
    # positive angle turns the image counter-clockwise on screen (y down):
    # a point right of the centre moves up.
    if angle > 0 and dx == 0 and dy == 0:
        px = M @ np.array([cx + 10, cy, 1.0])
        assert px[1] < cy
