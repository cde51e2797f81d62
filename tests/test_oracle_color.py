"""Pins of the oracle's photometric transforms: LUT ops, Grayscale, ShiftHSV,
Equalize.  Independent references: exact rational arithmetic with Python
``fractions`` (whose ``round`` is round-half-even), the standard library's
``colorsys`` HSV conversion, and closed forms of special cases."""
import colorsys
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1809_06839_gb300 import synth


def P(tid, **kw):
    p = O.Params()
    p.tid, p.apply = tid, 1
    p.alpha, p.gamma, p.scale, p.sat = 1.0, 1.0, 1.0, 1.0
    for k, v in kw.items():
        if k == "shift":
            for i, s in enumerate(v):
                p.shift[i] = s
        else:
            setattr(p, k, v)
    return p


V = np.arange(256)


def sat(v):
    return max(0, min(255, v))


def test_lut_identities():
    for p in (P(O.BRIGHTNESS, beta=0.0), P(O.CONTRAST, alpha=1.0), P(O.GAMMA, gamma=1.0),
              P(O.SHIFT_RGB, shift=(0.0, 0.0, 0.0)), P(O.BRIGHTNESS_CONTRAST, alpha=1.0, beta=0.0)):
        assert np.array_equal(O.build_lut(p), np.tile(V, (3, 1)))


@pytest.mark.parametrize("beta", [-20, -3, 7, 19])
def test_integer_brightness_is_saturating_add(beta):
    lut = O.build_lut(P(O.BRIGHTNESS, beta=float(beta)))
    assert [int(v) for v in lut[0]] == [sat(v + beta) for v in range(256)]


def test_half_ties_round_to_even():
    lut = O.build_lut(P(O.BRIGHTNESS, beta=0.5))
    assert [int(v) for v in lut[0]] == [sat(v if v % 2 == 0 else v + 1) for v in range(256)]
    lut = O.build_lut(P(O.BRIGHTNESS, beta=-0.5))
    assert [int(v) for v in lut[0]] == [sat(v if v % 2 == 0 else v - 1) for v in range(256)]
    lut = O.build_lut(P(O.CONTRAST, alpha=0.5))      # v/2: odd v ties to even
    assert [int(v) for v in lut[0]] == [round(Fraction(v, 2)) for v in range(256)]


@pytest.mark.parametrize("seed", range(8))
def test_brightness_contrast_exact_rational(seed):
    r = np.random.default_rng(seed)
    a, b = float(r.uniform(0.8, 1.2)), float(r.uniform(-20, 20))
    lut = O.build_lut(P(O.BRIGHTNESS_CONTRAST, alpha=a, beta=b))
    for v in range(256):
        exact = Fraction(a) * v + Fraction(b)
        frac = exact - int(exact)
        if abs(frac - Fraction(1, 2)) < Fraction(1, 10 ** 9):
            continue   # a near-tie where float64 rounding may legitimately decide
        assert lut[0][v] == sat(round(exact)), (v, a, b)


def test_gamma_two_is_exact_square():
    lut = O.build_lut(P(O.GAMMA, gamma=2.0))
    assert [int(v) for v in lut[1]] == [round(Fraction(v * v, 255)) for v in range(256)]


@pytest.mark.parametrize("g", [0.8, 0.93, 1.07, 1.2])
def test_gamma_monotone_with_fixed_endpoints(g):
    lut = O.build_lut(P(O.GAMMA, gamma=g)).astype(int)
    assert lut[0][0] == 0 and lut[0][255] == 255
    assert (np.diff(lut[0]) >= 0).all()
    assert (lut[0] >= V).all() if g < 1 else (lut[0] <= V).all()


def test_shift_rgb_per_channel():
    lut = O.build_lut(P(O.SHIFT_RGB, shift=(5.0, -7.0, 12.0)))
    for c, s in enumerate((5, -7, 12)):
        assert [int(v) for v in lut[c]] == [sat(v + s) for v in range(256)]


def lattice16():
    g = np.arange(0, 256, 17, dtype=np.uint8)        # 16 levels incl. 0 and 255
    r, gg, b = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([r.ravel(), gg.ravel(), b.ravel()], axis=1).reshape(64, 64, 3)


def test_grayscale_exact_bt601():
    img = lattice16()
    got = O.apply_image(P(O.GRAYSCALE), img)
    for y in range(0, 64, 3):
        for x in range(64):
            r, g, b = (int(v) for v in img[y, x])
            e = round(Fraction(299 * r + 587 * g + 114 * b, 1000))
            assert list(got[y, x]) == [e, e, e]
    grey = np.repeat(np.arange(256, dtype=np.uint8).reshape(16, 16, 1), 3, axis=2)
    assert np.array_equal(O.apply_image(P(O.GRAYSCALE), grey), grey)


def test_shift_hsv_zero_is_identity():
    img = np.concatenate([lattice16().reshape(-1, 3),
                          np.random.default_rng(0).integers(0, 256, (4096, 3))]).astype(np.uint8)
    img = img.reshape(-1, 64, 3)
    assert np.array_equal(O.apply_image(P(O.SHIFT_HSV, shift=(0.0, 0.0, 0.0)), img), img)
    # a hue shift of 180 half-degrees (= 360 degrees) is also the identity
    assert np.array_equal(O.apply_image(P(O.SHIFT_HSV, shift=(180.0, 0.0, 0.0)), img), img)


def test_shift_hsv_grey_invariant_under_hue():
    grey = np.repeat(np.arange(256, dtype=np.uint8).reshape(16, 16, 1), 3, axis=2)
    assert np.array_equal(O.apply_image(P(O.SHIFT_HSV, shift=(13.7, 0.0, 0.0)), grey), grey)


@pytest.mark.parametrize("shift", [(10.0, 0.0, 0.0), (-20.0, 25.0, -15.0), (7.5, -30.0, 20.0)])
def test_shift_hsv_matches_colorsys(shift):
    rng = np.random.default_rng(3)
    px = rng.integers(0, 256, (3000, 3)).astype(np.uint8)
    got = O.apply_image(P(O.SHIFT_HSV, shift=shift), px.reshape(-1, 100, 3)).reshape(-1, 3)
    bad = 0
    for i, (r, g, b) in enumerate(px):
        h, s, v = colorsys.rgb_to_hsv(r / 255, g / 255, b / 255)
        h = (h + 2 * shift[0] / 360) % 1.0
        s = min(1.0, max(0.0, s + shift[1] / 255))
        v = min(1.0, max(0.0, v + shift[2] / 255))
        ref = np.array(colorsys.hsv_to_rgb(h, s, v)) * 255
        d = np.abs(got[i].astype(float) - ref)
        assert d.max() <= 0.5 + 1e-9 or (d.max() <= 1 and np.any(np.abs(ref % 1 - 0.5) < 1e-6))
        bad += int(d.max() > 0.5 + 1e-9)
    assert bad <= 3


def _hsv_shift_exact(shift, r, g, b):
    """The hexcone shift of one pixel in exact rationals (Smith's hexcone; hue
    shifted by 2 * shift[0] degrees, saturation and value by shift / 255,
    both clamped to [0, 1]); returns the three unrounded channel values."""
    F = Fraction
    mx, mn = max(r, g, b), min(r, g, b)
    chroma = mx - mn
    hue = F(0)
    if chroma > 0:
        if mx == r:
            hue = 60 * F(g - b, chroma)
        elif mx == g:
            hue = 60 * (F(b - r, chroma) + 2)
        else:
            hue = 60 * (F(r - g, chroma) + 4)
        if hue < 0:
            hue += 360
    sat = F(chroma, mx) if mx > 0 else F(0)
    val = F(mx, 255)
    h2 = (hue + 2 * F(shift[0])) % 360
    s2 = min(F(1), max(F(0), sat + F(shift[1]) / 255))
    v2 = min(F(1), max(F(0), val + F(shift[2]) / 255))
    c2 = v2 * s2
    hp = h2 / 60
    sector = int(hp)                       # hp >= 0
    fr = hp - 2 * (hp // 2)
    x = c2 * (1 - abs(fr - 1))
    m = v2 - c2
    rgb1 = [(c2, x, 0), (x, c2, 0), (0, c2, x), (0, x, c2), (x, 0, c2), (c2, 0, x)][min(sector, 5)]
    return [255 * (c + m) for c in rgb1]


@pytest.mark.parametrize("shift", [(10.0, 0.0, 0.0), (-20.0, 25.0, -15.0), (7.5, -30.0, 20.0), (-90.0, 60.0, 0.0),
                                   (33.3, -255.0, 40.0)])
def test_shift_hsv_matches_exact_rationals(shift):
    """Every pixel equals the exact rational result rounded to nearest (ties to
    even) and saturated, except where that exact value lies within 1e-9 of a
    half-integer: there the float64 oracle may round either way."""
    rng = np.random.default_rng(11)
    px = np.concatenate([lattice16().reshape(-1, 3), rng.integers(0, 256, (6000, 3))]).astype(np.uint8)
    n = (len(px) // 100) * 100
    px = px[:n]
    got = O.apply_image(P(O.SHIFT_HSV, shift=shift), px.reshape(-1, 100, 3)).reshape(-1, 3)
    ties = 0
    for i, (r, g, b) in enumerate(px.tolist()):
        for c, e in enumerate(_hsv_shift_exact(shift, r, g, b)):
            lo = int(e)                            # e >= 0
            near_tie = abs(e - lo - Fraction(1, 2)) < Fraction(1, 10 ** 9)
            ref = min(255, max(0, round(e)))       # Fraction.__round__: ties to even
            if near_tie:
                ties += 1
                assert int(got[i, c]) in (min(255, lo), min(255, lo + 1)), (shift, (r, g, b), c)
            else:
                assert int(got[i, c]) == ref, (shift, (r, g, b), c, float(e))
    assert ties <= 3 * len(px) // 100             # exact half-integers: under 1 % of the channel values


def test_equalize_uniform_histogram_is_identity():
    hist = np.full(256, 7, dtype=np.uint64)
    assert np.array_equal(O.equalize_lut(hist), V.astype(np.uint8))


@pytest.mark.parametrize("k", range(2, 11))
def test_equalize_equal_mass_levels_are_evenly_spread(k):
    rng = np.random.default_rng(k)
    levels = np.sort(rng.choice(256, size=k, replace=False))
    hist = np.zeros(256, dtype=np.uint64)
    hist[levels] = 5
    lut = O.equalize_lut(hist)
    assert [int(lut[v]) for v in levels] == [round(Fraction(255 * j, k - 1)) for j in range(k)]


def test_equalize_invariants_on_images():
    img = synth.value_noise_image(50, 70, 9).numpy()
    out = O.apply_image(P(O.EQUALIZE), img)
    for c in range(3):
        src, dst = img[:, :, c].ravel().astype(int), out[:, :, c].ravel().astype(int)
        order = np.argsort(src, kind="stable")
        assert (np.diff(dst[order]) >= 0).all()                  # monotone
        assert dst[src == src.min()].max() == 0                 # lowest level -> 0
        assert dst[src == src.max()].min() == 255               # highest level -> 255
    const = np.full((5, 6, 3), 77, dtype=np.uint8)
    assert np.array_equal(O.apply_image(P(O.EQUALIZE), const), const)


def test_equalize_brute_force_tiny_images():
    # every 2x2 single-channel image over 4 levels: LUT monotone, extremes map to 0/255
    from itertools import product
    for vals in product(range(4), repeat=4):
        hist = np.zeros(256, dtype=np.uint64)
        for v in vals:
            hist[v * 60] += 1
        lut = O.equalize_lut(hist).astype(int)
        occ = [v * 60 for v in sorted(set(vals))]
        mapped = [lut[o] for o in occ]
        if len(occ) == 1:
            assert mapped == occ
        else:
            assert mapped[0] == 0 and mapped[-1] == 255 and mapped == sorted(mapped)
