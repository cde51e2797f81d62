"""Pins of the oracle's geometric transforms (flips, crop, pad, dihedral maps,
Q5 bilinear warps and resizes, nearest masks).  Independent references:
numpy indexing, ``np.pad(mode='reflect')`` (edge not repeated = reflect-101),
``np.rot90``, scipy ``map_coordinates`` (bilinear, ``mode='mirror'`` =
reflect-101) and closed forms of special cases."""
import numpy as np
import pytest
from scipy import ndimage

import oracle as O
from paper_1809_06839_gb300 import synth


def P(tid, apply=1, **kw):
    p = O.Params()
    p.tid, p.apply = tid, apply
    p.scale, p.alpha, p.gamma, p.sat = 1.0, 1.0, 1.0, 1.0
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def rnd(h, w, c=3, seed=0):
    return np.random.default_rng(seed).integers(0, 256, size=(h, w, c), dtype=np.uint8)


def structured_8x8():
    ramp = np.arange(64, dtype=np.uint8).reshape(8, 8) * 4
    checker = ((np.indices((8, 8)).sum(0) % 2) * 255).astype(np.uint8)
    hot = np.zeros((8, 8), np.uint8)
    hot[2, 5] = 255
    return [np.stack([ramp, checker, hot], axis=2), rnd(8, 8, 3, 1), rnd(8, 8, 3, 2)]


@pytest.mark.parametrize("img", structured_8x8())
def test_flips_exhaustive_8x8(img):
    assert np.array_equal(O.apply_image(P(O.HFLIP), img), img[:, ::-1])
    assert np.array_equal(O.apply_image(P(O.VFLIP), img), img[::-1])
    assert np.array_equal(O.apply_image(P(O.TRANSPOSE), img), img.transpose(1, 0, 2))
    for k in range(4):
        assert np.array_equal(O.apply_image(P(O.ROT90, k=k), img), np.rot90(img, k))
    assert np.array_equal(O.apply_image(P(O.HFLIP, apply=0), img), img)


def test_flip_twice_is_identity():
    img = rnd(37, 53)
    for tid in (O.HFLIP, O.VFLIP, O.TRANSPOSE):
        assert np.array_equal(O.apply_image(P(tid), O.apply_image(P(tid), img)), img)


@pytest.mark.parametrize("c", [1, 3, 4])
def test_crop_is_slice(c):
    img = rnd(40, 50, c)
    p = P(O.RANDOM_CROP, out_h=17, out_w=23, y0=5, x0=19, ch=17, cw=23)
    assert np.array_equal(O.apply_image(p, img), img[5:22, 19:42])


@pytest.mark.parametrize("h,w,oh,ow", [(3, 5, 16, 16), (333, 417, 512, 512), (1, 4, 6, 9), (8, 8, 8, 8),
                                       (600, 20, 512, 512)])
def test_pad_is_numpy_reflect(h, w, oh, ow):
    img = rnd(h, w)
    OH, OW = max(h, oh), max(w, ow)
    top, left = (OH - h) // 2, (OW - w) // 2
    p = P(O.PAD_TO_SIZE, out_h=OH, out_w=OW, y0=top, x0=left)
    got = O.apply_image(p, img)
    if h == 1:   # a single row reflects onto itself
        ref = np.pad(img, ((0, 0), (left, OW - w - left), (0, 0)), mode="reflect")
        ref = np.repeat(ref, OH, axis=0)
    else:
        ref = np.pad(img, ((top, OH - h - top), (left, OW - w - left), (0, 0)), mode="reflect")
    assert np.array_equal(got, ref)
    # crop back at (top, left) is the identity
    back = O.apply_image(P(O.RANDOM_CROP, out_h=h, out_w=w, y0=top, x0=left, ch=h, cw=w), got)
    assert np.array_equal(back, img)


def ssr(angle=0.0, scale=1.0, dx=0.0, dy=0.0, h=8, w=8, tid=None):
    p = P(tid or O.SHIFT_SCALE_ROTATE, angle=angle, scale=scale, dx=dx, dy=dy)
    return O.warp_geometry(p, h, w)


def test_warp_identity_bit_exact():
    img = rnd(31, 45)
    assert np.array_equal(O.apply_image(ssr(h=31, w=45, tid=O.ROTATE), img), img)
    assert np.array_equal(O.apply_mask(ssr(h=31, w=45), img[:, :, :1]), img[:, :, :1])


@pytest.mark.parametrize("n", [9, 31])
def test_rotate_quarter_turns_on_odd_squares(n):
    img = rnd(n, n)
    # Q16 rounding snaps cos(90 deg) to exactly 0, so +-90 and 180 degrees are exact
    assert np.array_equal(O.apply_image(ssr(90.0, h=n, w=n), img), np.rot90(img, 1))
    assert np.array_equal(O.apply_image(ssr(-90.0, h=n, w=n), img), np.rot90(img, -1))
    assert np.array_equal(O.apply_image(ssr(180.0, h=n, w=n), img), np.rot90(img, 2))
    assert np.array_equal(O.apply_mask(ssr(90.0, h=n, w=n), img[:, :, 0]), np.rot90(img[:, :, 0], 1))


@pytest.mark.parametrize("sx,sy", [(3, 0), (-5, 2), (0, -7), (11, 13)])
def test_integer_shift_is_reflect101_translation(sx, sy):
    h, w = 24, 32
    img = rnd(h, w)
    got = O.apply_image(ssr(dx=sx / w, dy=sy / h, h=h, w=w), img)
    ext = np.pad(img, ((20, 20), (40, 40), (0, 0)), mode="reflect")
    ref = ext[20 - sy:20 - sy + h, 40 - sx:40 - sx + w]
    assert np.array_equal(got, ref)


def _scipy_bilinear(img, ys, xs, mode):
    out = np.zeros(ys.shape + (img.shape[2],))
    for k in range(img.shape[2]):
        out[..., k] = ndimage.map_coordinates(img[:, :, k].astype(np.float64), [ys, xs], order=1, mode=mode)
    return out


@pytest.mark.parametrize("angle,scale,dx,dy", [(17.3, 1.0, 0.0, 0.0), (-63.0, 1.08, 0.04, -0.02),
                                               (44.0, 0.91, -0.06, 0.06), (-89.0, 1.0, 0.0, 0.0)])
def test_warp_matches_scipy_bilinear_mirror(angle, scale, dx, dy):
    """The Q5 (1/32 px) quantised warp agrees with a float64 bilinear warp
    (scipy, reflect-101) to 1 LSB on a smooth image."""
    h, w = 61, 77
    img = synth.value_noise_image(h, w, 3).numpy()
    p = ssr(angle, scale, dx, dy, h, w)
    got = O.apply_image(p, img).astype(np.int64)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    q = np.array(list(p.q), dtype=np.float64) / 65536.0
    xs = q[0] * xx + q[1] * yy + q[2]
    ys = q[3] * xx + q[4] * yy + q[5]
    ref = _scipy_bilinear(img, ys, xs, "mirror")
    d = np.abs(got - ref)
    assert d.max() <= 1.0, d.max()


def test_warp_nearest_mask_agrees_with_rounded_coordinates():
    h, w = 40, 52
    m = synth.blob_mask(h, w, 1).numpy()
    p = ssr(33.0, 1.05, 0.03, -0.02, h, w)
    got = O.apply_mask(p, m)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.int64)
    q = np.array(list(p.q), dtype=np.int64)
    X = q[0] * xx + q[1] * yy + q[2]
    Y = q[3] * xx + q[4] * yy + q[5]
    ix = np.floor((X + 32768) / 65536).astype(np.int64)
    iy = np.floor((Y + 32768) / 65536).astype(np.int64)
    ext = np.pad(m, ((200, 200), (200, 200)), mode="reflect")
    assert np.array_equal(got, ext[iy + 200, ix + 200])


def test_resize_same_size_is_identity():
    img = rnd(23, 29)
    p = P(O.RESIZE, out_h=23, out_w=29, ch=23, cw=29)
    assert np.array_equal(O.apply_image(p, img), img)
    assert np.array_equal(O.apply_mask(p, img[:, :, :1]), img[:, :, :1])


def test_resize_downscale_by_two_is_rounded_box_mean():
    img = rnd(32, 48).astype(np.int64)
    p = P(O.RESIZE, out_h=16, out_w=24, ch=32, cw=48)
    got = O.apply_image(p, img.astype(np.uint8))
    s = img[0::2, 0::2] + img[0::2, 1::2] + img[1::2, 0::2] + img[1::2, 1::2]
    assert np.array_equal(got, (s + 2) // 4)     # round half up of the 2x2 mean
    # nearest picks the second of each pair
    assert np.array_equal(O.apply_mask(p, img[:, :, :1].astype(np.uint8))[:, :, 0], img[1::2, 1::2, 0])


def test_resize_upscale_by_two_closed_form():
    h, w = 6, 7
    img = rnd(h, w).astype(np.int64)
    p = P(O.RESIZE, out_h=2 * h, out_w=2 * w, ch=h, cw=w)
    got = O.apply_image(p, img.astype(np.uint8)).astype(np.int64)

    def taps(n):
        # output 2k+1 -> 24/32 on k, 8/32 on k+1; output 2k -> 8/32 on k-1, 24/32 on k
        W = np.zeros((2 * n, n), dtype=np.int64)
        for d in range(2 * n):
            k = d // 2
            if d == 0:
                W[d, 0] = 32
            elif d % 2 == 1:
                if k + 1 < n:
                    W[d, k], W[d, k + 1] = 24, 8
                else:
                    W[d, k] = 32
            else:
                W[d, k - 1], W[d, k] = 8, 24
        return W

    Wy, Wx = taps(h), taps(w)
    acc = np.einsum("yi,xj,ijc->yxc", Wy, Wx, img)
    assert np.array_equal(got, (acc + 512) // 1024)
    assert np.array_equal(O.apply_mask(p, img[:, :, :1].astype(np.uint8))[:, :, 0],
                          np.repeat(np.repeat(img[:, :, 0], 2, 0), 2, 1))


@pytest.mark.parametrize("h,w,oh,ow", [(333, 417, 512, 512), (500, 360, 64, 80), (50, 70, 77, 41)])
def test_resize_matches_scipy_half_pixel(h, w, oh, ow):
    img = synth.value_noise_image(h, w, 5).numpy()
    p = P(O.RESIZE, out_h=oh, out_w=ow, ch=h, cw=w)
    got = O.apply_image(p, img).astype(np.int64)
    ys = (np.arange(oh) + 0.5) * h / oh - 0.5
    xs = (np.arange(ow) + 0.5) * w / ow - 0.5
    yy, xx = np.meshgrid(np.clip(ys, 0, h - 1), np.clip(xs, 0, w - 1), indexing="ij")
    ref = _scipy_bilinear(img, yy, xx, "nearest")
    assert np.abs(got - ref).max() <= 1.0


def test_random_sized_crop_is_crop_then_resize():
    img = rnd(90, 120)
    p = P(O.RANDOM_SIZED_CROP, out_h=64, out_w=64, y0=11, x0=40, ch=57, cw=57)
    crop = img[11:68, 40:97]
    r = P(O.RESIZE, out_h=64, out_w=64, ch=57, cw=57)
    assert np.array_equal(O.apply_image(p, img), O.apply_image(r, crop))
    assert np.array_equal(O.apply_mask(p, img[:, :, :1]), O.apply_mask(r, crop[:, :, :1].copy()))


def test_photometric_leave_mask_unchanged():
    m = synth.blob_mask(20, 30, 2).numpy()
    for tid in (O.BRIGHTNESS, O.SHIFT_HSV, O.GRAYSCALE, O.EQUALIZE, O.GAMMA):
        assert np.array_equal(O.apply_mask(P(tid, beta=10.0), m), m)
