"""Pins of the oracle's box transforms, fused chain and float warp/photometric
path.  Independent references: closed forms, warped rasterised masks, exact
rational arithmetic (``fractions``) with a correctly rounded float32 step,
torch's bfloat16 cast, scipy ``map_coordinates`` (``grid-constant`` = zero
border), central finite differences and the adjoint (dot-product) identity."""
from fractions import Fraction

import numpy as np
import pytest
import torch
from scipy import ndimage

import oracle as O
from tolerances import coord_bound
from paper_1809_06839_gb300 import synth


def P(tid, apply=1, **kw):
    p = O.Params()
    p.tid, p.apply = tid, apply
    p.scale, p.alpha, p.gamma, p.sat = 1.0, 1.0, 1.0, 1.0
    for k, v in kw.items():
        setattr(p, k, v)
    return p


BOXES = np.array([[10.5, 4.0, 30.25, 20.0], [0.0, 0.0, 64.0, 48.0], [50.0, 40.0, 63.0, 47.5]], np.float32)


def test_box_flips_exact_and_involutive():
    h, w = 48, 64
    hb = O.apply_boxes(P(O.HFLIP), h, w, BOXES)
    assert np.array_equal(hb, np.stack([w - BOXES[:, 2], BOXES[:, 1], w - BOXES[:, 0], BOXES[:, 3]], 1))
    assert np.array_equal(O.apply_boxes(P(O.HFLIP), h, w, hb), BOXES)
    vb = O.apply_boxes(P(O.VFLIP), h, w, BOXES)
    assert np.array_equal(vb, np.stack([BOXES[:, 0], h - BOXES[:, 3], BOXES[:, 2], h - BOXES[:, 1]], 1))
    assert np.array_equal(O.apply_boxes(P(O.HFLIP, apply=0), h, w, BOXES), BOXES)


def test_box_crop_clip_and_drop():
    p = P(O.RANDOM_CROP, out_h=20, out_w=20, y0=30, x0=45, ch=20, cw=20)
    got = O.apply_boxes(p, 48, 64, BOXES)
    # box 0 lies outside the window -> dropped; box 1 clipped to the window
    assert np.array_equal(got, np.array([[0, 0, 19, 18], [5, 10, 18, 17.5]], np.float32))


def test_box_pad_then_crop_back():
    p = P(O.PAD_TO_SIZE, out_h=100, out_w=90, y0=26, x0=13)
    padded = O.apply_boxes(p, 48, 64, BOXES)
    assert np.array_equal(padded, BOXES + np.array([13, 26, 13, 26], np.float32))
    back = O.apply_boxes(P(O.RANDOM_CROP, out_h=48, out_w=64, y0=26, x0=13, ch=48, cw=64), 100, 90, padded)
    assert np.array_equal(back, BOXES)


def test_box_resize_scales():
    p = P(O.RESIZE, out_h=24, out_w=128, ch=48, cw=64)
    got = O.apply_boxes(p, 48, 64, BOXES)
    assert np.allclose(got, BOXES * np.array([2, 0.5, 2, 0.5], np.float32), atol=0)


def test_box_dihedral_matches_mask():
    h, w = 30, 44
    for p in (P(O.TRANSPOSE), P(O.ROT90, k=1), P(O.ROT90, k=2), P(O.ROT90, k=3)):
        box = np.array([[3, 5, 17, 11]], np.float32)
        m = np.zeros((h, w), np.uint8)
        m[5:11, 3:17] = 1
        wm = O.apply_mask(p, m)
        ys, xs = np.nonzero(wm)
        got = O.apply_boxes(p, h, w, box)[0]
        assert list(got) == [xs.min(), ys.min(), xs.max() + 1, ys.max() + 1]


def _warp(angle, scale, dx, dy, h, w):
    p = P(O.SHIFT_SCALE_ROTATE, angle=angle, scale=scale, dx=dx, dy=dy)
    return O.warp_geometry(p, h, w)


@pytest.mark.parametrize("angle,scale,dx,dy", [(0.0, 1.0, 0.0, 0.0), (30.0, 1.0, 0.0, 0.0),
                                               (-41.0, 1.07, 0.05, -0.04), (12.0, 0.92, -0.06, 0.02)])
def test_box_warp_follows_warped_mask(angle, scale, dx, dy):
    """The 4-corner box of a warped box encloses the nearest-warped raster of
    that box and is within ~1 px of its extent."""
    h, w = 120, 160
    p = _warp(angle, scale, dx, dy, h, w)
    box = np.array([[40, 30, 100, 80]], np.float32)
    m = np.zeros((h, w), np.uint8)
    m[30:80, 40:100] = 1
    wm = O.apply_mask(p, m)
    got = O.apply_boxes(p, h, w, box)[0]
    # only pixels reached without reflection count (the border reflects content)
    ys, xs = np.nonzero(wm)
    q = np.array(list(p.q), dtype=np.float64) / 65536
    sx = q[0] * xs + q[1] * ys + q[2]
    sy = q[3] * xs + q[4] * ys + q[5]
    inside = (sx > -0.5) & (sx < w - 0.5) & (sy > -0.5) & (sy < h - 0.5)
    xs, ys = xs[inside], ys[inside]
    ext = [xs.min(), ys.min(), xs.max() + 1, ys.max() + 1]
    # a pixel is set when its (rounded) centre falls in the box: the box holds
    # every set pixel centre, up to the 1/2 px of nearest rounding
    assert got[0] <= ext[0] + 0.5 + 0.5 and got[1] <= ext[1] + 0.5 + 0.5
    assert got[2] >= ext[2] - 0.5 - 0.5 and got[3] >= ext[3] - 0.5 - 0.5
    assert np.abs(np.array(ext) - got).max() <= 1.5
    # corners map through the forward matrix (built independently here)
    t = np.deg2rad(angle)
    cx, cy = (w - 1) / 2, (h - 1) / 2
    R = np.array([[np.cos(t), np.sin(t)], [-np.sin(t), np.cos(t)]]) * scale
    corners = np.array([[40, 30], [100, 30], [40, 80], [100, 80]], np.float64) - 0.5
    mapped = (corners - [cx, cy]) @ R.T + [cx + dx * w, cy + dy * h] + 0.5
    ref = [max(mapped[:, 0].min(), 0), max(mapped[:, 1].min(), 0),
           min(mapped[:, 0].max(), w), min(mapped[:, 1].max(), h)]
    assert np.abs(np.array(ref) - got).max() < 1e-4


# ------------------------------------------------------------ fused chain
def round_f32(q: Fraction) -> float:
    """Correctly rounded (half-even) float32 of an exact rational (normal range)."""
    if q == 0:
        return 0.0
    sign = -1 if q < 0 else 1
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    while Fraction(2) ** (e + 1) <= q:
        e += 1
    scaled = q / Fraction(2) ** (e - 23)
    n = round(scaled)
    return sign * float(n) * 2.0 ** (e - 23)


def fmaf_exact(a, b, c):
    return round_f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def test_round_f32_matches_numpy_on_doubles():
    rng = np.random.default_rng(0)
    for v in rng.uniform(-300, 300, 200):
        assert round_f32(Fraction(float(v))) == float(np.float32(v))


def test_bf16_cast_matches_torch():
    vals = np.random.default_rng(1).normal(0, 3, 5000).astype(np.float32)
    vals[:4] = [0.0, -0.0, 1.00390625, 1.01171875]   # exact bf16 ties
    ours = O.f32_to_bf16_bits(vals)
    ref = torch.from_numpy(vals).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)


@pytest.mark.parametrize("seed", range(3))
def test_chain_is_composition_of_pinned_steps(seed):
    h, w = 70, 90
    img = synth.value_noise_image(h, w, seed).numpy()
    cfg = O.make_cfg(O.CHAIN, out_h=24, out_w=20, lo=(0.08, 3 / 4, 0.6), hi=(1.0, 4 / 3, 1.4))
    p = O.sample_params(cfg, 1809, 20, seed, h, w)
    got = O.chain_image(p, img)
    # step 1: crop + resize (pinned in test_oracle_geometric)
    r = P(O.RESIZE, out_h=24, out_w=20, ch=p.ch, cw=p.cw)
    x = O.apply_image(r, np.ascontiguousarray(img[p.y0:p.y0 + p.ch, p.x0:p.x0 + p.cw]))
    if p.flip:
        x = x[:, ::-1]
    # step 3: brightness b then contrast c about 128, exact rational + half-even
    b, c = p.beta, p.alpha
    lut = np.zeros(256, np.int64)
    for v in range(256):
        e = Fraction(c) * (Fraction(b) * v - 128) + 128
        lut[v] = max(0, min(255, round(e)))
    x = lut[x]
    k, m = O.normalize_consts()
    s = np.float32(p.sat)
    ref = np.zeros((3, 24, 20), np.float32)
    for yy in range(24):
        for xx in range(20):
            R, G, B = (float(v) for v in x[yy, xx])
            grey = fmaf_exact(np.float32(0.114), B, fmaf_exact(np.float32(0.587), G, float(np.float32(0.299) * np.float32(R))))
            for ch in range(3):
                d = float(np.float32(float(x[yy, xx, ch])) - np.float32(grey))
                v = min(255.0, max(0.0, fmaf_exact(s, d, grey)))
                ref[ch, yy, xx] = fmaf_exact(v, k[ch], m[ch])
    ref_bits = torch.from_numpy(ref).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(got, ref_bits)


def test_normalize_consts_are_rounded_float64():
    k, m = O.normalize_consts()
    for c, (mu, sd) in enumerate(zip(O.IMAGENET_MEAN, O.IMAGENET_STD)):
        assert k[c] == np.float32(1.0 / (255.0 * sd)) and m[c] == np.float32(-mu / sd)


# ------------------------------------------------------------ float path
def fparams(B, seed=0, ident=False):
    r = np.random.default_rng(seed)
    if ident:
        z = np.zeros(B)
        return dict(angle=z, scale=np.ones(B), tx=z, ty=z, alpha=np.ones(B), beta=z, gamma=np.ones(B))
    return dict(angle=r.uniform(-30, 30, B), scale=r.uniform(0.9, 1.1, B), tx=r.uniform(-0.0625, 0.0625, B),
                ty=r.uniform(-0.0625, 0.0625, B), alpha=r.uniform(0.8, 1.2, B), beta=r.uniform(-0.1, 0.1, B),
                gamma=r.uniform(0.8, 1.2, B))


def test_float_identity():
    x = np.random.default_rng(0).uniform(0, 1, (2, 3, 9, 11))
    y = O.warp_photo_fwd(x, **fparams(2, ident=True))
    assert np.array_equal(y, x)


def test_float_integer_shift_zero_fill():
    B, C, H, W = 1, 2, 10, 12
    x = np.random.default_rng(1).uniform(0.1, 0.9, (B, C, H, W))
    p = fparams(B, ident=True)
    p["tx"] = np.array([3 / W])
    p["ty"] = np.array([-2 / H])
    y = O.warp_photo_fwd(x, **p)
    ref = np.zeros_like(x)
    ref[:, :, 0:H - 2, 3:W] = x[:, :, 2:H, 0:W - 3]
    assert np.allclose(y, ref, atol=1e-12)


def test_float_warp_matches_scipy_grid_constant():
    B, C, H, W = 2, 3, 21, 27
    x = np.random.default_rng(2).uniform(0, 1, (B, C, H, W))
    p = fparams(B, seed=5)
    y, warped = O.warp_photo_fwd(x, **p, want_warped=True)
    for b in range(B):
        t = np.deg2rad(p["angle"][b])
        s = p["scale"][b]
        cx, cy = (W - 1) / 2, (H - 1) / 2
        yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
        xp, yp = xx - cx - p["tx"][b] * W, yy - cy - p["ty"][b] * H
        sx = (np.cos(t) * xp - np.sin(t) * yp) / s + cx
        sy = (np.sin(t) * xp + np.cos(t) * yp) / s + cy
        for c in range(C):
            ref = ndimage.map_coordinates(x[b, c], [sy, sx], order=1, mode="grid-constant", cval=0.0)
            assert np.abs(warped[b, c] - ref).max() < 1e-12
            z = p["alpha"][b] * ref + p["beta"][b]
            yref = np.where(z > 0, np.clip(z, 0, 1) ** p["gamma"][b], 0)
            assert np.abs(y[b, c] - yref).max() < 1e-12


def test_float_adjoint_dot_product():
    """With identity photometrics and values in (0,1) the path is linear in x:
    <A x, g> == <x, A^T g>."""
    B, C, H, W = 2, 2, 13, 15
    rng = np.random.default_rng(3)
    x = rng.uniform(0.05, 0.5, (B, C, H, W))
    p = fparams(B, seed=7)
    p.update(alpha=np.ones(B), beta=np.zeros(B), gamma=np.ones(B))
    g = rng.normal(0, 1, x.shape)
    y = O.warp_photo_fwd(x, **p)
    dx, _ = O.warp_photo_bwd(x, **p, gy=g)
    lhs = float((y * g).sum())
    rhs = float((x * dx).sum())
    # the border zeros (z == 0) are outside the open interval and carry no gradient
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def test_float_gradients_match_finite_differences():
    B, C, H, W = 2, 3, 16, 16
    rng = np.random.default_rng(11)
    x = rng.uniform(0.15, 0.85, (B, C, H, W))
    p = fparams(B, seed=13)
    g = rng.normal(0, 1, x.shape)
    dx, dparams = O.warp_photo_bwd(x, **p, gy=g)

    def loss(xx, pp):
        return float((O.warp_photo_fwd(xx, **pp) * g).sum())

    names = ["angle", "scale", "tx", "ty", "alpha", "beta", "gamma"]
    # piecewise bilinear in the parameters: take the step size (of three) that
    # does not straddle a kink
    for b in range(B):
        for j, n in enumerate(names):
            an = dparams[b, j]
            errs = []
            for rel in (1e-6, 1e-7, 1e-8):
                hstep = rel * max(1.0, abs(p[n][b]))
                pp, pm = {k: v.copy() for k, v in p.items()}, {k: v.copy() for k, v in p.items()}
                pp[n][b] += hstep
                pm[n][b] -= hstep
                fd = (loss(x, pp) - loss(x, pm)) / (2 * hstep)
                errs.append(abs(fd - an) / max(1e-3, abs(fd)))
            assert min(errs) <= 1e-3, (b, n, errs, an)
    for (b, c, yy, xx) in [(0, 0, 5, 7), (1, 2, 8, 8), (0, 1, 12, 3), (1, 0, 2, 14)]:
        hstep = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[b, c, yy, xx] += hstep
        xm[b, c, yy, xx] -= hstep
        fd = (loss(xp, p) - loss(xm, p)) / (2 * hstep)
        assert abs(fd - dx[b, c, yy, xx]) <= 1e-3 * max(1e-3, abs(fd))


# ------------------------------------------------ float32 coordinate class
def test_float32_coordinates_exact_where_representable():
    # identity and integer shifts: every map entry and coordinate is exact in
    # float32, so the two classes give identical outputs
    B, C, H, W = 1, 2, 10, 12
    x = np.random.default_rng(1).uniform(0.1, 0.9, (B, C, H, W))
    for tx, ty in ((0.0, 0.0), (3 / W, -2 / H), (-5 / W, 4 / H)):
        p = fparams(B, ident=True)
        p["tx"], p["ty"] = np.array([tx]), np.array([ty])
        assert np.array_equal(O.warp_photo_fwd(x, **p, coords=32), O.warp_photo_fwd(x, **p, coords=64))


@pytest.mark.parametrize("H,W", [(512, 512), (333, 500), (37, 53)])
def test_float32_coordinates_within_rounding_bound(H, W):
    """The float32 class samples within the coordinate rounding bound of the
    float64 map: with inputs in [0,1] the bilinear value moves by at most
    |dsx| + |dsy| (slope <= 1 per pixel along each axis)."""
    B, C = 2, 1
    x = np.random.default_rng(4).uniform(0, 1, (B, C, H, W))
    p = fparams(B, seed=9)
    p.update(alpha=np.ones(B), beta=np.zeros(B), gamma=np.ones(B))
    _, w32 = O.warp_photo_fwd(x, **p, coords=32, want_warped=True)
    _, w64 = O.warp_photo_fwd(x, **p, coords=64, want_warped=True)
    for b in range(B):
        d = np.abs(w32[b] - w64[b]).max()
        assert d <= 2 * coord_bound(p, b, H, W), (b, d, coord_bound(p, b, H, W))
    assert np.abs(w32 - w64).max() > 0          # the classes do differ


def test_float32_coordinates_adjoint_dot_product():
    """The float32 class is linear in x for an affine photometric step with z
    inside (0,1): <y - beta, g> == <x, dx> / alpha * alpha."""
    B, C, H, W = 2, 2, 19, 23
    rng = np.random.default_rng(5)
    x = rng.uniform(0.0, 1.0, (B, C, H, W))
    p = fparams(B, seed=8)
    p.update(alpha=np.full(B, 0.5), beta=np.full(B, 0.25), gamma=np.ones(B))
    g = rng.normal(0, 1, x.shape)
    y = O.warp_photo_fwd(x, **p, coords=32)
    dx, _ = O.warp_photo_bwd(x, **p, gy=g, coords=32)
    lhs = float(((y - 0.25) * g).sum())
    rhs = float((x * dx).sum())
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def test_float32_coordinates_gradients_follow_the_float64_adjoint():
    """On a 16x16 image no sample changes cell between the classes, so the
    float32-class gradients equal the (finite-difference pinned) float64
    ones up to the coordinate rounding."""
    B, C, H, W = 2, 3, 16, 16
    rng = np.random.default_rng(11)
    x = rng.uniform(0.15, 0.85, (B, C, H, W))
    p = fparams(B, seed=13)
    g = rng.normal(0, 1, x.shape)
    dx64, dp64 = O.warp_photo_bwd(x, **p, gy=g)
    dx32, dp32 = O.warp_photo_bwd(x, **p, gy=g, coords=32)
    assert np.abs(dx32 - dx64).max() <= 1e-5
    assert np.all(np.abs(dp32 - dp64) <= 1e-5 * np.abs(dp64) + 1e-6), (dp32, dp64)


def test_absolute_term_sums():
    """The sums of absolute term values bound the gradients (triangle
    inequality) and equal them where every term is non-negative: with g >= 0
    and alpha > 0 the input adjoint, d alpha and d beta have only
    non-negative terms."""
    B, C, H, W = 2, 3, 21, 17
    rng = np.random.default_rng(12)
    x = rng.uniform(0.0, 1.0, (B, C, H, W))
    p = fparams(B, seed=14)
    g = rng.normal(0, 1, x.shape)
    for coords in (32, 64):
        dx, dp, adx, adp = O.warp_photo_bwd(x, **p, gy=g, coords=coords, want_abs=True)
        assert np.all(adx >= np.abs(dx) - 1e-12) and np.all(adp >= np.abs(dp) - 1e-12)
        assert np.all(adp[:, :4] > 0)
        dx, dp, adx, adp = O.warp_photo_bwd(x, **p, gy=np.abs(g), coords=coords, want_abs=True)
        assert np.allclose(adx, dx, rtol=1e-12, atol=0)
        assert np.allclose(adp[:, 4:6], dp[:, 4:6], rtol=1e-12, atol=0)
