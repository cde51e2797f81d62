"""GPU parity of the differentiable float32 warp and photometric kernels: the
forward against the float64 oracle, the backward (input and parameter
gradients) against the oracle's analytic adjoint and against float64 finite
differences of the oracle, through torch.autograd.

Tolerances (derived from float32 rounding): the warp's source coordinate is
a short chain of float32 multiply-adds of magnitude <= ~2W, so its error is a
few ulp of 2W (~1e-4 px at W = 512); with inputs in [0,1] the warped value
moves by at most that much, so forward outputs agree to 2e-4 absolute.
Gradients sum O(H W) float32 terms per image and are compared with a
relative tolerance of 1e-3 (the workload's stated bound) plus a small
absolute floor for near-zero sums."""
import numpy as np
import pytest
import torch

import oracle as O

from paper_1809_06839_gb300 import alb, synth
from paper_1809_06839_gb300.autograd import AffineWarpFn, PhotometricFn, augment

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    alb.load()
    return torch.device("cuda")


def params(B, seed):
    r = np.random.default_rng(seed)
    return dict(angle=r.uniform(-30, 30, B), scale=r.uniform(0.9, 1.1, B), tx=r.uniform(-0.0625, 0.0625, B),
                ty=r.uniform(-0.0625, 0.0625, B), alpha=r.uniform(0.8, 1.2, B), beta=r.uniform(-0.1, 0.1, B),
                gamma=r.uniform(0.8, 1.2, B))


def f32(p):
    return {k: np.asarray(v, np.float32).astype(np.float64) for k, v in p.items()}


def t(v, dev):
    return torch.tensor(np.asarray(v, np.float32), device=dev)


@pytest.mark.parametrize("B,C,H,W", [(3, 3, 37, 53), (2, 3, 128, 96)])
def test_forward_matches_oracle(dev, B, C, H, W):
    x = synth.float_images(B, C, H, W, seed=5)
    p = f32(params(B, 6))
    xd = x.to(dev)
    y = augment(xd, *(t(p[k], dev) for k in ("angle", "scale", "tx", "ty", "alpha", "beta", "gamma")))
    ref = O.warp_photo_fwd(x.numpy(), **p)
    assert np.abs(y.cpu().numpy() - ref).max() < 2e-4
    w = AffineWarpFn.apply(xd, *(t(p[k], dev) for k in ("angle", "scale", "tx", "ty")))
    _, wref = O.warp_photo_fwd(x.numpy(), **{**p, "alpha": np.ones(B), "beta": np.zeros(B),
                                            "gamma": np.ones(B)}, want_warped=True)
    assert np.abs(w.cpu().numpy() - wref).max() < 2e-4


def close(got, ref, rel=1e-3, floor=1e-3):
    return np.all(np.abs(got - ref) <= rel * np.abs(ref) + floor)


@pytest.mark.parametrize("B,C,H,W", [(2, 3, 16, 16), (3, 3, 64, 48)])
def test_backward_matches_oracle_adjoint(dev, B, C, H, W):
    x = synth.float_images(B, C, H, W, seed=11)
    g = synth.float_normal((B, C, H, W), seed=12)
    p = f32(params(B, 13))
    xd = x.to(dev).requires_grad_(True)
    tp = {k: t(p[k], dev).requires_grad_(True) for k in p}
    y = augment(xd, tp["angle"], tp["scale"], tp["tx"], tp["ty"], tp["alpha"], tp["beta"], tp["gamma"])
    y.backward(g.to(dev))
    dx_ref, dp_ref = O.warp_photo_bwd(x.numpy(), **p, gy=g.numpy())
    # the float path's input gradient: absolute tolerance scaled by the largest entry
    dx = xd.grad.cpu().numpy()
    assert np.abs(dx - dx_ref).max() <= 2e-3 * max(1.0, np.abs(dx_ref).max())
    names = ["angle", "scale", "tx", "ty", "alpha", "beta", "gamma"]
    for j, k in enumerate(names):
        got = tp[k].grad.cpu().numpy()
        scale = np.abs(dp_ref[:, j]).max() + 1e-6
        assert close(got, dp_ref[:, j], rel=1e-3, floor=2e-3 * scale), (k, got, dp_ref[:, j])


def test_gradients_match_finite_differences(dev):
    """Central float64 differences of the oracle forward vs the CUDA backward."""
    B, C, H, W = 2, 3, 16, 16
    x = synth.float_images(B, C, H, W, seed=21).numpy().astype(np.float64)
    x = (0.15 + 0.7 * x).astype(np.float32).astype(np.float64)
    g = synth.float_normal((B, C, H, W), seed=22).numpy().astype(np.float64)
    p = f32(params(B, 23))
    xd = torch.tensor(x, dtype=torch.float32, device=dev, requires_grad=True)
    tp = {k: t(p[k], dev).requires_grad_(True) for k in p}
    y = augment(xd, tp["angle"], tp["scale"], tp["tx"], tp["ty"], tp["alpha"], tp["beta"], tp["gamma"])
    y.backward(torch.tensor(g, dtype=torch.float32, device=dev))

    def loss(pp):
        return float((O.warp_photo_fwd(x, **pp) * g).sum())

    # the warp is piecewise bilinear in the parameters: a difference whose step
    # straddles a kink (a sample crossing a pixel boundary) is not a derivative,
    # so several step sizes are tried and the closest one is compared
    for k in p:
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
            assert min(abs(got - fd) - 1e-3 * abs(fd) for fd in fds) <= 2e-3, (k, b, got, fds)


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
]


@pytest.mark.parametrize("B,C,H,W,ang,sc", WARP_CASES)
def test_warp_shapes_zoom_and_channel_groups(dev, B, C, H, W, ang, sc):
    x = synth.float_images(B, C, H, W, seed=31)
    g = synth.float_normal((B, C, H, W), seed=32)
    r = np.random.default_rng(33)
    # photometric offset kept positive (z = alpha w + beta >= 0.02): near z = 0
    # with gamma < 1 the composed gradient depends on the last bits of the
    # warped value through gamma z^(gamma-1) (a float32 warp moves z = 3e-6 by
    # 7% and a border pixel's tx gradient by 0.2), which would test the
    # conditioning of the composition rather than the warp
    p = f32(dict(angle=r.uniform(*ang, B), scale=r.uniform(*sc, B), tx=r.uniform(-0.05, 0.05, B),
                 ty=r.uniform(-0.05, 0.05, B), alpha=r.uniform(0.8, 1.2, B), beta=r.uniform(0.02, 0.1, B),
                 gamma=r.uniform(0.8, 1.2, B)))
    xd = x.to(dev).requires_grad_(True)
    tp = {k: t(p[k], dev).requires_grad_(True) for k in p}
    y = augment(xd, tp["angle"], tp["scale"], tp["tx"], tp["ty"], tp["alpha"], tp["beta"], tp["gamma"])
    assert np.abs(y.detach().cpu().numpy() - O.warp_photo_fwd(x.numpy(), **p)).max() < 2e-4
    y.backward(g.to(dev))
    dx_ref, dp_ref = O.warp_photo_bwd(x.numpy(), **p, gy=g.numpy())
    dx = xd.grad.cpu().numpy()
    assert np.abs(dx - dx_ref).max() <= 2e-3 * max(1.0, np.abs(dx_ref).max())
    for j, k in enumerate(["angle", "scale", "tx", "ty", "alpha", "beta", "gamma"]):
        got = tp[k].grad.cpu().numpy()
        scale = np.abs(dp_ref[:, j]).max() + 1e-6
        assert close(got, dp_ref[:, j], rel=1e-3, floor=2e-3 * scale), (k, got, dp_ref[:, j])


@pytest.mark.parametrize("W", [64, 61])
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
