"""GPU parity of the fused ragged-batch chain (RandomResizedCrop -> resize 224 ->
h-flip -> brightness/contrast -> saturation -> Normalize -> bf16 NCHW): the
persistent fused kernel, the plain one-step-per-launch path and the oracle
agree bit for bit."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import CHAIN_CFG, cfg_to_lib, to_lib

from paper_1809_06839_gb300 import alb, synth
from paper_1809_06839_gb300.ragged import DeviceBatch, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    alb.load()
    return torch.device("cuda")


def bits(t):
    return t.view(torch.int16).cpu().numpy().view(np.uint16)


def run_chain(din, lps, dev, mode, oh=224, ow=224, tile_h=0, jitter=0):
    n = len(lps)
    cfg = alb.chain_cfg(oh, ow, tile_h=tile_h, jitter=jitter)
    out = torch.empty((n, 3, oh, ow), dtype=torch.bfloat16, device=dev)
    alb.alb_apply_batch(cfg, n, alb.params_to_device(lps, dev), din.dev, out, mode)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("oh,ow", [(224, 224), (37, 61)])
def test_fused_plain_oracle_agree(dev, oh, ow):
    sizes = [(256 + (i * 97) % 769, 256 + (i * 193) % 769) for i in range(12)] + [(3, 900), (1024, 1024)]
    rb = synth.ragged_noise(sizes, seed=7)
    oc = O.make_cfg(O.CHAIN, **{**CHAIN_CFG, "out_h": oh, "out_w": ow})
    ops = [O.sample_params(oc, 7, 20, i, h, w) for i, (h, w) in enumerate(sizes)]
    lps = [to_lib(p, alb) for p in ops]
    din = DeviceBatch(to_device(rb, dev))
    fused = run_chain(din, lps, dev, alb.MODE_FUSED, oh, ow)
    plain = run_chain(din, lps, dev, alb.MODE_PLAIN, oh, ow)
    assert torch.equal(fused.view(torch.int16), plain.view(torch.int16))
    fb = bits(fused)
    for i in range(len(sizes)):
        ref = O.chain_image(ops[i], rb.image(i).numpy())
        assert np.array_equal(fb[i], ref), i


@pytest.mark.parametrize("tile_h", [1, 3, 8, 16])
def test_fused_band_heights(dev, tile_h):
    sizes = [(300, 400), (512, 256), (999, 1001)]
    rb = synth.ragged_noise(sizes, seed=3)
    oc = O.make_cfg(O.CHAIN, **CHAIN_CFG)
    ops = [O.sample_params(oc, 3, 20, i, h, w) for i, (h, w) in enumerate(sizes)]
    lps = [to_lib(p, alb) for p in ops]
    din = DeviceBatch(to_device(rb, dev))
    out = bits(run_chain(din, lps, dev, alb.MODE_FUSED, tile_h=tile_h))
    for i in range(len(sizes)):
        assert np.array_equal(out[i], O.chain_image(ops[i], rb.image(i).numpy()))


def test_autotuned_schedule_and_every_candidate_agree(dev):
    """The autotuner returns one of its candidate schedules, later zero-field
    calls use it, and every schedule writes the same bits as the oracle."""
    sizes = [(256 + (i * 131) % 769, 256 + (i * 71) % 769) for i in range(40)]
    rb = synth.ragged_noise(sizes, seed=11)
    oc = O.make_cfg(O.CHAIN, **CHAIN_CFG)
    ops = [O.sample_params(oc, 11, 20, i, h, w) for i, (h, w) in enumerate(sizes)]
    lps = [to_lib(p, alb) for p in ops]
    din = DeviceBatch(to_device(rb, dev))
    n = len(lps)
    pdev = alb.params_to_device(lps, dev)
    out = torch.empty((n, 3, 224, 224), dtype=torch.bfloat16, device=dev)
    best = alb.alb_autotune_batch(alb.chain_cfg(), n, pdev, din.dev, out, reps=2)
    torch.cuda.synchronize()
    assert best.tile_h in (2, 4, 8, 16, 32) and best.ctas_per_sm >= 1 and best.tile_w == 0
    ref = bits(out)
    for i in range(n):
        assert np.array_equal(ref[i], O.chain_image(ops[i], rb.image(i).numpy())), i
    cached = torch.empty_like(out)
    alb.alb_apply_batch(alb.chain_cfg(), n, pdev, din.dev, cached, alb.MODE_FUSED)
    for tile_h, per_sm in ((2, 1), (32, best.ctas_per_sm), (best.tile_h, best.ctas_per_sm), (5, 2)):
        o = torch.empty_like(out)
        alb.alb_apply_batch(alb.chain_cfg(tile_h=tile_h, ctas_per_sm=per_sm), n, pdev, din.dev, o, alb.MODE_FUSED)
        torch.cuda.synchronize()
        assert np.array_equal(bits(o), ref), (tile_h, per_sm)
    torch.cuda.synchronize()
    assert np.array_equal(bits(cached), ref)


def test_full_size_ragged_batch_sampled(dev):
    """4096 images, H, W ~ U[256, 1024], params from the device sampler; fused ==
    plain over the whole output; 24 sampled images against the oracle."""
    n = 4096
    sizes = synth.uniform_sizes(n, 256, 1024, seed=1809)
    rb = synth.ragged_noise(sizes, seed=1809, device=dev)
    din = DeviceBatch(rb)
    oc = O.make_cfg(O.CHAIN, **CHAIN_CFG)
    pdev = torch.zeros(n * 232, dtype=torch.uint8, device=dev)
    alb.alb_sample_params_batch(cfg_to_lib(oc, alb), 1809, 20, 0, n, din.dev, pdev)
    cfg = alb.chain_cfg()
    fused = torch.empty((n, 3, 224, 224), dtype=torch.bfloat16, device=dev)
    plain = torch.empty_like(fused)
    alb.alb_apply_batch(cfg, n, pdev, din.dev, fused, alb.MODE_FUSED)
    alb.alb_apply_batch(cfg, n, pdev, din.dev, plain, alb.MODE_PLAIN)
    torch.cuda.synchronize()
    assert torch.equal(fused.view(torch.int16), plain.view(torch.int16))
    fb = bits(fused[::171])
    for k, i in enumerate(range(0, n, 171)):
        h, w = sizes[i]
        op = O.sample_params(oc, 1809, 20, i, h, w)     # the oracle samples its own parameters
        ref = O.chain_image(op, rb.image(i).cpu().numpy())
        assert np.array_equal(fb[k], ref), i


@pytest.mark.parametrize("oh,ow", [(224, 224), (37, 61)])
def test_jitter_mode1_fused_plain_oracle_agree(dev, oh, ow):
    """Random op order and image-mean contrast pivot: fused == plain == oracle
    for every one of the six orders."""
    sizes = [(256 + (i * 97) % 769, 256 + (i * 193) % 769) for i in range(12)] + [(3, 900), (1024, 1024)]
    rb = synth.ragged_noise(sizes, seed=9)
    oc = O.make_cfg(O.CHAIN, **{**CHAIN_CFG, "out_h": oh, "out_w": ow})
    ops = [O.sample_params(oc, 9, 20, i, h, w) for i, (h, w) in enumerate(sizes)]
    for i, op in enumerate(ops):
        op.k = i % 6
    lps = [to_lib(p, alb) for p in ops]
    din = DeviceBatch(to_device(rb, dev))
    fused = run_chain(din, lps, dev, alb.MODE_FUSED, oh, ow, jitter=1)
    plain = run_chain(din, lps, dev, alb.MODE_PLAIN, oh, ow, jitter=1)
    assert torch.equal(fused.view(torch.int16), plain.view(torch.int16))
    fb = bits(fused)
    for i in range(len(sizes)):
        ref = O.chain_image(ops[i], rb.image(i).numpy(), jitter=1)
        assert np.array_equal(fb[i], ref), (i, ops[i].k)


def test_jitter_mode1_full_size_batch_sampled(dev):
    """4096 images, device-sampled records (order drawn per image), every
    schedule of the autotuner's pick; fused == plain; 24 images vs the oracle."""
    n = 4096
    sizes = synth.uniform_sizes(n, 256, 1024, seed=1810)
    rb = synth.ragged_noise(sizes, seed=1810, device=dev)
    din = DeviceBatch(rb)
    oc = O.make_cfg(O.CHAIN, **CHAIN_CFG)
    pdev = torch.zeros(n * 232, dtype=torch.uint8, device=dev)
    alb.alb_sample_params_batch(cfg_to_lib(oc, alb), 1810, 20, 0, n, din.dev, pdev)
    cfg = alb.chain_cfg(jitter=1)
    fused = torch.empty((n, 3, 224, 224), dtype=torch.bfloat16, device=dev)
    best = alb.alb_autotune_batch(cfg, n, pdev, din.dev, fused, reps=1)
    assert best.jitter == 1 and best.tile_h in (2, 4, 8, 16, 32)
    plain = torch.empty_like(fused)
    alb.alb_apply_batch(cfg, n, pdev, din.dev, fused, alb.MODE_FUSED)
    alb.alb_apply_batch(cfg, n, pdev, din.dev, plain, alb.MODE_PLAIN)
    torch.cuda.synchronize()
    assert torch.equal(fused.view(torch.int16), plain.view(torch.int16))
    fb = bits(fused[::171])
    for k, i in enumerate(range(0, n, 171)):
        h, w = sizes[i]
        op = O.sample_params(oc, 1810, 20, i, h, w)
        ref = O.chain_image(op, rb.image(i).cpu().numpy(), jitter=1)
        assert np.array_equal(fb[k], ref), i
