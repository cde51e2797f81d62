"""Pins of the oracle's grid distortion and elastic transform (Sec. II-C):
identities, the grid map recomputed in exact rationals from the cell
definition, the elastic lattice recomputed from the pinned Philox, the
warps against scipy's bilinear interpolation, masks by numpy indexing and the
grid's box map by round trips."""
import bisect
from fractions import Fraction
from math import floor

import numpy as np
import pytest
from scipy import ndimage

import oracle as O
from paper_1809_06839_gb300 import synth

GRID = O.make_cfg(O.GRID_DISTORTION, lo=(-0.3, 5), hi=(0.3, 5))
ELASTIC = O.make_cfg(O.ELASTIC, lo=(6.0, 4))


def grid_record(h, w, seed=3, g=5):
    cfg = O.make_cfg(O.GRID_DISTORTION, lo=(-0.3, g), hi=(0.3, g))
    return O.sample_params(cfg, seed, 21, 0, h, w)


def grid_src_exact(p, axis, x, n):
    """The cell definition in exact rationals: output cells of equal width,
    source cells proportional to the factors, linear inside a cell."""
    g = p.k
    if n == 1:
        return Fraction(0)
    d = [O.grid_factor(p, 12 * axis + j) for j in range(g)]
    out_b = [Fraction(i * (n - 1), g) for i in range(g + 1)]
    src_b = [Fraction(0)]
    for j in range(g):
        src_b.append(src_b[-1] + Fraction((n - 1) * d[j], sum(d)))
    i = min(g - 1, bisect.bisect_right(out_b, Fraction(x)) - 1)
    t = (Fraction(x) - out_b[i]) / (out_b[i + 1] - out_b[i])
    return src_b[i] + t * (src_b[i + 1] - src_b[i])


def q5_half_up(v: Fraction) -> int:
    return floor(32 * v + Fraction(1, 2))


@pytest.mark.parametrize("n", [1, 2, 7, 64, 333, 500])
def test_grid_table_is_the_exact_cell_map(n):
    p = grid_record(n, n, seed=n)
    for axis in (0, 1):
        got = [O.grid_q5(p, axis, x, n) for x in range(n)]
        ref = [q5_half_up(grid_src_exact(p, axis, x, n)) for x in range(n)]
        assert got == ref
        assert got[0] == 0 and got[-1] == 32 * (n - 1)
        assert all(b >= a for a, b in zip(got, got[1:]))


def test_grid_equal_factors_is_identity():
    img = synth.value_noise_image(57, 83, 2).numpy()
    p = grid_record(57, 83)
    for slot in list(range(5)) + list(range(12, 17)):
        O.grid_set_factor(p, slot, 17000)
    assert np.array_equal(O.apply_image(p, img), img)
    m = img[:, :, :1].copy()
    assert np.array_equal(O.apply_mask(p, m), m)


def test_grid_sampler_ranges_and_cells():
    for i in range(50):
        p = O.sample_params(GRID, 9, 21, i, 300, 400)
        assert p.k == 5 and p.apply == 1
        for slot in list(range(5)) + list(range(12, 17)):
            assert round(16384 * 0.7) <= O.grid_factor(p, slot) <= round(16384 * 1.3)
    p = O.sample_params(O.make_cfg(O.GRID_DISTORTION, lo=(-0.1, 3), hi=(0.1, 3)), 9, 21, 0, 50, 50)
    assert p.k == 3
    with pytest.raises(ValueError):
        O.sample_params(O.make_cfg(O.GRID_DISTORTION, lo=(-0.1, 13), hi=(0.1, 13)), 9, 21, 0, 50, 50)


def test_grid_image_matches_scipy_bilinear_and_masks_are_nearest():
    h, w = 71, 93
    img = synth.value_noise_image(h, w, 4).numpy()
    p = grid_record(h, w, seed=5)
    got = O.apply_image(p, img).astype(np.int64)
    xs = np.array([O.grid_q5(p, 0, x, w) for x in range(w)]) / 32.0
    ys = np.array([O.grid_q5(p, 1, y, h) for y in range(h)]) / 32.0
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    for c in range(3):
        ref = ndimage.map_coordinates(img[:, :, c].astype(np.float64), [yy, xx], order=1, mode="nearest")
        assert np.abs(got[:, :, c] - ref).max() <= 1.0
    m = synth.value_noise_image(h, w, 6).numpy()[:, :, :1].copy()
    iy = (np.array([O.grid_q5(p, 1, y, h) for y in range(h)]) + 16) // 32
    ix = (np.array([O.grid_q5(p, 0, x, w) for x in range(w)]) + 16) // 32
    assert np.array_equal(O.apply_mask(p, m), m[iy][:, ix])


def test_grid_box_map_inverts_the_cell_map():
    h, w = 120, 160
    p = grid_record(h, w, seed=8)
    for axis, n in ((0, w), (1, h)):
        for e in np.linspace(0.5, n - 0.5, 37):
            x = O.grid_edge_inverse(p, axis, float(e), n) - 0.5
            back = grid_src_exact(p, axis, Fraction(x), n) if 0 <= x <= n - 1 else None
            if back is not None:
                assert abs(float(back) - (e - 0.5)) < 1e-9
        assert abs(O.grid_edge_inverse(p, axis, 0.5, n) - 0.5) < 1e-9
        assert abs(O.grid_edge_inverse(p, axis, n - 0.5, n) - (n - 0.5)) < 1e-9
    full = O.apply_boxes(p, h, w, np.array([[0, 0, w, h]], np.float32))
    assert np.allclose(full, [[0, 0, w, h]], atol=1e-4)


def test_elastic_lattice_follows_the_published_philox():
    p = O.sample_params(ELASTIC, 1809, 22, 7, 90, 110)
    assert p.k == 192 and p.cw == 4
    span = 2 * p.k + 1
    sid = 22
    for t in (0, 1, 5, 40, 77):
        ctr = [t, 7, sid & 0xFFFFFFFF, (sid >> 32) ^ 0x80000000]
        key = [1809 & 0xFFFFFFFF, 1809 >> 32]
        o = O.philox4x32_10(ctr, key)
        ref = (int((int(o[0]) * span) >> 32) - p.k, int((int(o[1]) * span) >> 32) - p.k)
        assert O.elastic_point(p, t) == ref


def test_elastic_displacement_is_the_rounded_bilinear_blend():
    h, w = 40, 52
    p = O.sample_params(ELASTIC, 5, 22, 1, h, w)
    S = 1 << p.cw
    nx = (w + S - 1) // S + 1
    for y in range(0, h, 3):
        for x in range(0, w, 5):
            ci, cj, fy, fx = y // S, x // S, y % S, x % S
            pts = [O.elastic_point(p, (ci + a) * nx + cj + b) for a in (0, 1) for b in (0, 1)]
            wts = [(S - fx) * (S - fy), fx * (S - fy), (S - fx) * fy, fx * fy]
            ref = tuple(floor(Fraction(sum(wt * pt[k] for wt, pt in zip(wts, pts)), S * S) + Fraction(1, 2)) for k in (0, 1))
            assert O.elastic_disp(p, x, y, w) == ref
            if fx == 0 and fy == 0:
                assert ref == pts[0]


def test_elastic_zero_amplitude_is_identity():
    img = synth.value_noise_image(45, 61, 3).numpy()
    p = O.sample_params(O.make_cfg(O.ELASTIC, lo=(0.0, 5)), 3, 22, 0, 45, 61)
    assert np.array_equal(O.apply_image(p, img), img)
    m = img[:, :, 1:2].copy()
    assert np.array_equal(O.apply_mask(p, m), m)


def test_elastic_image_matches_scipy_mirror_bilinear_and_masks_are_nearest():
    h, w = 64, 80
    img = synth.value_noise_image(h, w, 7).numpy()
    p = O.sample_params(ELASTIC, 11, 22, 2, h, w)
    got = O.apply_image(p, img).astype(np.int64)
    d = np.array([[O.elastic_disp(p, x, y, w) for x in range(w)] for y in range(h)])
    yy = np.arange(h)[:, None] + d[:, :, 1] / 32.0
    xx = np.arange(w)[None, :] + d[:, :, 0] / 32.0
    for c in range(3):
        ref = ndimage.map_coordinates(img[:, :, c].astype(np.float64), [yy, xx], order=1, mode="mirror")
        assert np.abs(got[:, :, c] - ref).max() <= 1.0
    m = synth.value_noise_image(h, w, 8).numpy()[:, :, :1].copy()

    def r101(i, n):
        i = np.abs(i) % (2 * (n - 1)) if n > 1 else np.zeros_like(i)
        return np.where(i >= n, 2 * (n - 1) - i, i)

    iy = r101(np.floor_divide(32 * np.arange(h)[:, None] + d[:, :, 1] + 16, 32), h)
    ix = r101(np.floor_divide(32 * np.arange(w)[None, :] + d[:, :, 0] + 16, 32), w)
    assert np.array_equal(O.apply_mask(p, m)[:, :, 0], m[iy, ix, 0])
    with pytest.raises(ValueError):
        O.apply_boxes(p, h, w, np.array([[1, 1, 5, 5]], np.float32))


def test_elastic_lattice_values_are_bounded_and_centred():
    p = O.sample_params(ELASTIC, 2, 22, 0, 500, 500)
    vals = np.array([O.elastic_point(p, t) for t in range(2000)])
    assert vals.min() >= -p.k and vals.max() <= p.k
    assert abs(vals.mean()) < 0.08 * p.k
