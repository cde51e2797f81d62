"""Tolerances of the float path, derived from float32 rounding.

u = 2^-24 is the unit roundoff of float32.

* Coordinates.  A float32 warp rounds the six inverse-map entries to float32
  once and forms each source coordinate with two fused multiply-adds, so its
  coordinate differs from the float64 map's by at most
  3 u (|a00| (W-1) + |a01| (H-1) + max(|b0|, |b1|)) (first order; the
  entries' relative errors times the largest products plus the two
  roundings, bounded by three times the largest magnitude).  With inputs in
  [0,1] the bilinear value moves by at most |dsx| + |dsy|: twice that bound.
  This is the tolerance against the float64 coordinate class; it grows with
  the image (about 2.3e-4 at 512 x 512, 6e-5 at 128 x 96).
* Values.  Against the float32 coordinate class (the same sample cells) a
  forward value differs only by float32 rounding of the weights, the four
  products and the photometric step: 1e-5 absolute.
* Gradients.  Each gradient entry is a sum of terms t_i; a float32
  evaluation gets each term to within ~8 roundings and sums them in running
  float32 sums whose expected error grows with the square root of the chain
  length, so |got - ref| <= 1e-3 |ref| + 64 u sum_i |t_i| (the oracle returns
  sum_i |t_i| per entry).  A near-zero entry is thus checked at the float32
  resolution of its own terms, never against another entry's size.
"""
import numpy as np

U32 = 2.0 ** -24
FWD_ABS = 1e-5
GRAD_REL = 1e-3
GRAD_ULPS = 64


def coord_bound(p, b, H, W):
    """First-order bound on |s32 - s64| over every output pixel of image b."""
    t = np.deg2rad(p["angle"][b])
    s = p["scale"][b]
    cx, cy = (W - 1) / 2, (H - 1) / 2
    a00, a01 = np.cos(t) / s, -np.sin(t) / s
    ox, oy = cx + p["tx"][b] * W, cy + p["ty"][b] * H
    b0 = cx - (a00 * ox + a01 * oy)
    b1 = cy - (-a01 * ox + a00 * oy)
    m = abs(a00) * (W - 1) + abs(a01) * (H - 1)
    return 3 * U32 * (m + max(abs(b0), abs(b1))) * 1.001


def warped_bound(p, b, H, W):
    """Tolerance of a float32 warp's value against the float64 class."""
    return 2 * coord_bound(p, b, H, W) + 1e-6


def grad_excess(got, ref, absref):
    """Per entry: |got - ref| minus its tolerance (<= 0 passes)."""
    return np.abs(got - ref) - (GRAD_REL * np.abs(ref) + GRAD_ULPS * U32 * absref)


def grad_ok(got, ref, absref):
    return bool(np.all(grad_excess(got, ref, absref) <= 0))


def kink_free_grad(y_oracle_warped, alpha, beta, g, margin=1e-3):
    """Upstream gradient with the outputs near the photometric step's kinks
    (z = alpha w + beta within `margin` of 0 or 1: the clamp, and z^(gamma-1)
    for gamma < 1) set to zero, so neither side sums a term whose inclusion
    or conditioning depends on the last bits of the warped value."""
    B = g.shape[0]
    z = alpha.reshape(B, 1, 1, 1) * y_oracle_warped + beta.reshape(B, 1, 1, 1)
    near = (np.abs(z) < margin) | (np.abs(z - 1.0) < margin)
    out = g.copy()
    out[near] = 0.0
    return out
