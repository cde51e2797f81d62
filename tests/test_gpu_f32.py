"""GPU parity of the differentiable float32 warp and photometric kernels,
through torch.autograd and the C ABI.

The oracle is compared in two coordinate classes (tests/tolerances.py has
the derivations):
* the float32 coordinate class (map entries rounded to float32 once,
  coordinates by float32 fused multiply-adds: the same sample cells as a
  float32 warp): forward values within 1e-5, every gradient entry -- each
  pixel of the input gradient, each parameter of each image -- within
  1e-3 relative plus 64 float32 ulps of the sum of the absolute values of
  that entry's own terms;
* the float64 class (the definition): warped values within twice the
  coordinate rounding bound of the image's own size; gradients against
  float64 finite differences.
Outputs near the photometric step's kinks (z within 1e-3 of 0 or 1) get a
zero upstream gradient on both sides in the gradient comparisons."""
import numpy as np
import pytest
import torch

import oracle as O
from tolerances import FWD_ABS, U32, grad_excess, grad_ok, kink_free_grad, warped_bound

from paper_1809_06839_gb300 import alb, synth
from paper_1809_06839_gb300.autograd import AffineWarpFn, PhotometricFn, augment

pytestmark = pytest.mark.gpu
NAMES = ["angle", "scale", "tx", "ty", "alpha", "beta", "gamma"]


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    alb.load()
    return torch.device("cuda")


def params(B, seed):
    """The differentiable workload's parameter ranges."""
    r = np.random.default_rng(seed)
    return dict(angle=r.uniform(-30, 30, B), scale=r.uniform(0.9, 1.1, B), tx=r.uniform(-0.0625, 0.0625, B),
                ty=r.uniform(-0.0625, 0.0625, B), alpha=r.uniform(0.8, 1.2, B), beta=r.uniform(-0.1, 0.1, B),
                gamma=r.uniform(0.8, 1.2, B))


def f32(p):
    return {k: np.asarray(v, np.float32).astype(np.float64) for k, v in p.items()}


def t(v, dev):
    return torch.tensor(np.asarray(v, np.float32), device=dev)


def run_fwd_bwd(dev, x, p, g):
    xd = x.to(dev).requires_grad_(True)
    tp = {k: t(p[k], dev).requires_grad_(True) for k in p}
    y = augment(xd, *(tp[k] for k in NAMES))
    if g is not None:
        y.backward(torch.as_tensor(g, dtype=torch.float32).to(dev))
    return y.detach().cpu().numpy(), xd, tp


def check_grads(xd, tp, x, p, g, where=""):
    dx_ref, dp_ref, adx, adp = O.warp_photo_bwd(x, **p, gy=g, coords=32, want_abs=True)
    dx = xd.grad.cpu().numpy()
    ex = grad_excess(dx, dx_ref, adx)
    assert ex.max() <= 0, (where, "dx", np.unravel_index(ex.argmax(), ex.shape), ex.max())
    for j, k in enumerate(NAMES):
        got = tp[k].grad.cpu().numpy()
        assert grad_ok(got, dp_ref[:, j], adp[:, j]), (where, k, got, dp_ref[:, j], adp[:, j] * 64 * U32)
    return dp_ref


@pytest.mark.parametrize("B,C,H,W", [(3, 3, 37, 53), (2, 3, 128, 96), (2, 3, 512, 512), (1, 3, 509, 517)])
def test_forward_matches_oracle(dev, B, C, H, W):
    """Full-size images (3 x 512 x 512, and an odd 509 x 517) included."""
    x = synth.float_images(B, C, H, W, seed=5)
    p = f32(params(B, 6))
    y, _, _ = run_fwd_bwd(dev, x, p, None)
    ref = O.warp_photo_fwd(x.numpy(), **p, coords=32)
    assert np.abs(y - ref).max() <= FWD_ABS
    # the warp alone: float32 class to rounding, float64 class to the
    # coordinate bound of this image size
    w = AffineWarpFn.apply(x.to(dev), *(t(p[k], dev) for k in ("angle", "scale", "tx", "ty"))).cpu().numpy()
    ident = {**p, "alpha": np.ones(B), "beta": np.zeros(B), "gamma": np.ones(B)}
    _, w32 = O.warp_photo_fwd(x.numpy(), **ident, want_warped=True, coords=32)
    _, w64 = O.warp_photo_fwd(x.numpy(), **ident, want_warped=True, coords=64)
    assert np.abs(w - w32).max() <= FWD_ABS
    for b in range(B):
        assert np.abs(w[b] - w64[b]).max() <= warped_bound(p, b, H, W), b


@pytest.mark.parametrize("B,C,H,W", [(2, 3, 16, 16), (3, 3, 64, 48), (2, 3, 512, 512)])
def test_backward_matches_oracle_adjoint(dev, B, C, H, W):
    """Every input-gradient pixel and every parameter gradient on its own, at
    sizes up to the workload's 3 x 512 x 512, with the workload's ranges."""
    x = synth.float_images(B, C, H, W, seed=11).numpy()
    p = f32(params(B, 13))
    _, w32 = O.warp_photo_fwd(x, **p, want_warped=True, coords=32)
    g = kink_free_grad(w32, p["alpha"], p["beta"], synth.float_normal((B, C, H, W), seed=12).numpy())
    _, xd, tp = run_fwd_bwd(dev, torch.from_numpy(x), p, g)
    check_grads(xd, tp, x, p, g, (B, C, H, W))


def test_small_gradient_checked_on_its_own(dev):
    """Image 1's upstream gradient is 100x smaller than image 0's, so all of
    its gradients are 100x smaller; each is checked against its own terms,
    not against image 0's magnitude."""
    B, C, H, W = 2, 3, 96, 80
    x = synth.float_images(B, C, H, W, seed=51).numpy()
    p = f32(params(B, 52))
    _, w32 = O.warp_photo_fwd(x, **p, want_warped=True, coords=32)
    g = synth.float_normal((B, C, H, W), seed=53).numpy()
    g[1] *= 0.01
    g = kink_free_grad(w32, p["alpha"], p["beta"], g)
    _, xd, tp = run_fwd_bwd(dev, torch.from_numpy(x), p, g)
    dp_ref = check_grads(xd, tp, x, p, g, "small")
    _, adp0 = O.warp_photo_bwd(x, **p, gy=g, coords=32, want_abs=True)[2:]
    assert np.all(adp0[1] < 0.05 * adp0[0])          # the scales really differ


def test_gradients_match_finite_differences(dev):
    """Central float64 differences of the oracle's float64 forward against
    the CUDA backward, per parameter and image, rel 1e-3 plus the float32
    resolution of the entry's own terms."""
    B, C, H, W = 2, 3, 16, 16
    x = synth.float_images(B, C, H, W, seed=21).numpy().astype(np.float64)
    x = (0.15 + 0.7 * x).astype(np.float32).astype(np.float64)
    g = synth.float_normal((B, C, H, W), seed=22).numpy().astype(np.float64)
    p = f32(params(B, 23))
    _, w64 = O.warp_photo_fwd(x, **p, want_warped=True)
    g = kink_free_grad(w64, p["alpha"], p["beta"], g)
    _, xd, tp = run_fwd_bwd(dev, torch.from_numpy(x.astype(np.float32)), p, g)
    _, _, _, adp = O.warp_photo_bwd(x, **p, gy=g, want_abs=True)

    def loss(pp):
        return float((O.warp_photo_fwd(x, **pp) * g).sum())

    # the warp is piecewise bilinear in the parameters: a difference whose step
    # straddles a kink (a sample crossing a pixel boundary) is not a derivative,
    # so three step sizes are tried and the closest one is compared
    for j, k in enumerate(NAMES):
        for b in range(B):
            got = float(tp[k].grad[b])
            fds = []
            for rel in (1e-6, 1e-7, 1e-8):
                h = rel * max(1.0, abs(p[k][b]))
                pp = {kk: v.copy() for kk, v in p.items()}
                pm = {kk: v.copy() for kk, v in p.items()}
                pp[k][b] += h
                pm[k][b] -= h
                fds.append((loss(pp) - loss(pm)) / (2 * h))
            tol = [1e-3 * abs(fd) + 64 * U32 * adp[b, j] for fd in fds]
            assert min(abs(got - fd) - tl for fd, tl in zip(fds, tol)) <= 0, (k, b, got, fds)


def test_photometric_alone_and_clamp(dev):
    x = torch.linspace(-0.5, 1.5, 3 * 40 * 40, device=dev).reshape(1, 3, 40, 40)
    a, b, gm = t([1.1], dev), t([0.05], dev), t([0.9], dev)
    xr = x.clone().requires_grad_(True)
    y = PhotometricFn.apply(xr, a, b, gm)
    z = (1.1 * x.double() + 0.05).clamp(0, 1)
    assert torch.allclose(y.double(), z ** 0.9, atol=2e-6)
    y.sum().backward()
    zz = 1.1 * x.double() + 0.05
    inside = (zz > 0) & (zz < 1)
    ref = torch.where(inside, 0.9 * zz.clamp(1e-30) ** (0.9 - 1) * 1.1, torch.zeros_like(zz))
    assert torch.allclose(xr.grad.double(), ref, rtol=1e-4, atol=1e-5)


WARP_CASES = [
    # (B, C, H, W, angle range, scale range): odd widths take the 4-byte staging
    # path, C = 4 two channel groups, zoom 3 (backward box) and 0.3 (forward
    # box) overflow the staging buffer and read global memory
    (2, 1, 40, 61, (-30, 30), (0.9, 1.1)),
    (2, 4, 48, 64, (-30, 30), (0.9, 1.1)),
    (2, 3, 37, 53, (-30, 30), (0.9, 1.1)),
    (2, 3, 64, 64, (-20, 20), (3.0, 3.0)),
    (2, 3, 64, 64, (-20, 20), (0.3, 0.3)),
    (2, 3, 50, 52, (90, 90), (1.0, 1.0)),
    (2, 2, 33, 80, (180, 180), (1.05, 1.05)),
    (2, 3, 512, 512, (-30, 30), (0.3, 0.3)),
]


@pytest.mark.parametrize("B,C,H,W,ang,sc", WARP_CASES)
def test_warp_shapes_zoom_and_channel_groups(dev, B, C, H, W, ang, sc):
    x = synth.float_images(B, C, H, W, seed=31).numpy()
    r = np.random.default_rng(33)
    p = f32(dict(angle=r.uniform(*ang, B), scale=r.uniform(*sc, B), tx=r.uniform(-0.05, 0.05, B),
                 ty=r.uniform(-0.05, 0.05, B), alpha=r.uniform(0.8, 1.2, B), beta=r.uniform(-0.1, 0.1, B),
                 gamma=r.uniform(0.8, 1.2, B)))
    y, _, _ = run_fwd_bwd(dev, torch.from_numpy(x), p, None)
    ref, w32 = O.warp_photo_fwd(x, **p, want_warped=True, coords=32)
    assert np.abs(y - ref).max() <= FWD_ABS
    g = kink_free_grad(w32, p["alpha"], p["beta"], synth.float_normal((B, C, H, W), seed=32).numpy())
    _, xd, tp = run_fwd_bwd(dev, torch.from_numpy(x), p, g)
    check_grads(xd, tp, x, p, g, (C, H, W, ang, sc))


@pytest.mark.parametrize("W", [64, 61, 512])
def test_warp_backward_is_deterministic(dev, W):
    """The input adjoint is a gather in a fixed order and the parameter
    partials are reduced in a fixed order: two runs agree bit for bit."""
    B, C, H = 3, 3, 96
    x = synth.float_images(B, C, H, W, seed=41).to(dev)
    g = synth.float_normal((B, C, H, W), seed=42).to(dev)
    r = np.random.default_rng(43)
    wp = torch.tensor(np.stack([r.uniform(-30, 30, B), r.uniform(0.9, 1.1, B), r.uniform(-0.06, 0.06, B),
                                r.uniform(-0.06, 0.06, B)], 1), dtype=torch.float32, device=dev)
    ws = alb.workspace(alb.alb_f32_workspace_size(B, C, H, W), dev)
    outs = []
    for _ in range(2):
        gx = torch.full_like(x, float("nan"))
        gp = torch.full((B, 4), float("nan"), device=dev)
        alb.alb_warp_affine_f32_bwd(x, wp, g, gx, gp, ws)
        outs.append((gx, gp))
    torch.cuda.synchronize()
    assert torch.isfinite(outs[0][0]).all() and torch.isfinite(outs[0][1]).all()
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
