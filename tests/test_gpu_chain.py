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
    """The chain into an output with a guard image before and after it (a
    sentinel bit pattern that must survive the launch)."""
    n = len(lps)
    cfg = alb.chain_cfg(oh, ow, tile_h=tile_h, jitter=jitter)
    full = torch.full((n + 2, 3, oh, ow), -1, dtype=torch.int16, device=dev).view(torch.bfloat16)
    out = full[1:n + 1]
    alb.alb_apply_batch(cfg, n, alb.params_to_device(lps, dev), din.dev, out, mode)
    torch.cuda.synchronize()
    g = full.view(torch.int16)
    assert bool((g[0] == -1).all()) and bool((g[n + 1] == -1).all()), "chain wrote outside its output"
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


def test_autotune_cache_persists_to_json(dev, tmp_path):
    """The autotuner's pick is cached, written to JSON keyed by device name
    and SM count, and read back: a schedule edited in the file becomes the
    cached pick, and zero-field calls with it still write the oracle's bits."""
    import json
    sizes = [(300 + (i * 37) % 500, 280 + (i * 53) % 600) for i in range(24)]
    rb = synth.ragged_noise(sizes, seed=13)
    oc = O.make_cfg(O.CHAIN, **CHAIN_CFG)
    ops = [O.sample_params(oc, 13, 20, i, h, w) for i, (h, w) in enumerate(sizes)]
    lps = [to_lib(p, alb) for p in ops]
    din = DeviceBatch(to_device(rb, dev))
    n = len(lps)
    pdev = alb.params_to_device(lps, dev)
    out = torch.empty((n, 3, 224, 224), dtype=torch.bfloat16, device=dev)
    best = alb.alb_autotune_batch(alb.chain_cfg(), n, pdev, din.dev, out, reps=1)
    got = alb.alb_autotune_lookup(alb.chain_cfg(), n)
    assert got is not None and (got.tile_h, got.ctas_per_sm) == (best.tile_h, best.ctas_per_sm)
    assert alb.alb_autotune_lookup(alb.chain_cfg(out_h=17, out_w=19), n) is None
    path = tmp_path / "tune.json"
    alb.alb_autotune_save(str(path))
    doc = json.loads(path.read_text())
    assert doc["format"] == "alb-autotune-1"
    mine = [e for e in doc["entries"] if e["out_h"] == 224 and e["jitter"] == 0 and e["bucket"] == 5]
    assert len(mine) == 1 and mine[0]["rows_per_item"] == best.tile_h
    assert mine[0]["device"] == torch.cuda.get_device_name(dev)
    assert mine[0]["sms"] == torch.cuda.get_device_properties(dev).multi_processor_count
    mine[0]["rows_per_item"] = 4 if best.tile_h != 4 else 16
    mine[0]["ctas_per_sm"] = 1
    path.write_text(json.dumps(doc))
    assert alb.alb_autotune_load(str(path)) >= 1
    got = alb.alb_autotune_lookup(alb.chain_cfg(), n)
    assert (got.tile_h, got.ctas_per_sm) == (mine[0]["rows_per_item"], 1)
    o = torch.empty_like(out)
    alb.alb_apply_batch(alb.chain_cfg(), n, pdev, din.dev, o, alb.MODE_FUSED)
    torch.cuda.synchronize()
    ob = bits(o)
    for i in range(n):
        assert np.array_equal(ob[i], O.chain_image(ops[i], rb.image(i).numpy())), i


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


def test_chain_targets_masks_and_boxes(dev):
    """Instance-mask stacks (1 to 20 planes) and boxes through the chain,
    fused and plain, against the oracle; the images are unchanged by the
    targets; box-safe windows from the device sampler equal the oracle's."""
    from paper_1809_06839_gb300.ragged import mask_output_batch
    from helpers import same_params
    sizes = [(256 + (i * 97) % 769, 256 + (i * 193) % 769) for i in range(10)] + [(3, 900), (1024, 1024)]
    planes = [1, 3, 20, 8, 1, 5, 2, 20, 4, 1, 7, 3]
    n = len(sizes)
    rb = synth.ragged_noise(sizes, seed=12)
    rng = np.random.default_rng(12)
    mask_np = [(rng.integers(0, 2, (h, w, c)) * rng.integers(1, 256, c)).astype(np.uint8)
               for (h, w), c in zip(sizes, planes)]
    cap = 50
    boxes = np.zeros((n, cap, 4), np.float32)
    nb = np.zeros(n, np.int32)
    for i, (h, w) in enumerate(sizes):
        b = synth.random_boxes(h, w, i, 12)[: 1 + i * 3]
        boxes[i, :len(b)] = b
        nb[i] = len(b)
    oc = O.make_cfg(O.CHAIN, **CHAIN_CFG)
    din = DeviceBatch(to_device(rb, dev))
    bd, nbd = torch.from_numpy(boxes).to(dev), torch.from_numpy(nb).to(dev)
    pdev = torch.zeros(n * 232, dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    alb.alb_sample_chain_box_safe_batch(cfg_to_lib(oc, alb), 12, 20, 0, n, din.dev, bd, nbd, cap, pdev, status)
    got_p = alb.params_from_device(pdev)
    ops = [O.sample_chain_box_safe(oc, 12, 20, i, h, w, boxes[i, :nb[i]]) for i, (h, w) in enumerate(sizes)]
    for i in range(n):
        assert same_params(ops[i], got_p[i]) is None, i
    mdesc = []
    flat = []
    for m in mask_np:
        t = torch.from_numpy(m).to(dev)
        flat.append(t)
        mdesc.append(alb.image_desc(t))
    mi = alb.descs_to_device(mdesc, dev)
    results = {}
    for mode in (alb.MODE_FUSED, alb.MODE_PLAIN):
        outs = [torch.zeros((224, 224, c), dtype=torch.uint8, device=dev) for c in planes]
        mo = alb.descs_to_device([alb.image_desc(t) for t in outs], dev)
        img = torch.empty((n, 3, 224, 224), dtype=torch.bfloat16, device=dev)
        bo, nbo = torch.zeros_like(bd), torch.zeros_like(nbd)
        alb.alb_apply_batch_targets(alb.chain_cfg(), n, pdev, din.dev, img, mi, mo, bd, nbd, cap, bo, nbo, mode,
                                    dev_status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        results[mode] = (bits(img), [t.cpu().numpy() for t in outs], bo.cpu().numpy(), nbo.cpu().numpy())
    for mode, (ib, ms, bo, nbo) in results.items():
        for i, (h, w) in enumerate(sizes):
            assert np.array_equal(ib[i], O.chain_image(ops[i], rb.image(i).numpy())), (mode, i)
            assert np.array_equal(ms[i], O.chain_mask(ops[i], mask_np[i])), (mode, "mask", i)
            bref = O.chain_boxes(ops[i], boxes[i, :nb[i]])
            assert nbo[i] == len(bref) == nb[i], (mode, "boxes", i)       # box-safe windows keep every box
            assert np.abs(bo[i, :nbo[i]] - bref).max(initial=0) <= 1e-4


def test_chain_target_masks_of_the_wrong_size_are_rejected_on_device(dev):
    sizes = [(300, 400), (280, 260)]
    rb = synth.ragged_noise(sizes, seed=2)
    oc = O.make_cfg(O.CHAIN, **CHAIN_CFG)
    ops = [O.sample_params(oc, 2, 20, i, h, w) for i, (h, w) in enumerate(sizes)]
    din = DeviceBatch(to_device(rb, dev))
    good = torch.ones((300, 400, 2), dtype=torch.uint8, device=dev)
    bad = torch.ones((200, 260, 2), dtype=torch.uint8, device=dev)         # height differs from its image
    mi = alb.descs_to_device([alb.image_desc(good), alb.image_desc(bad)], dev)
    outs = [torch.full((224, 224, 2), 7, dtype=torch.uint8, device=dev) for _ in range(2)]
    mo = alb.descs_to_device([alb.image_desc(t) for t in outs], dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    img = torch.empty((2, 3, 224, 224), dtype=torch.bfloat16, device=dev)
    alb.alb_apply_batch_targets(alb.chain_cfg(), 2, alb.params_to_device([to_lib(o, alb) for o in ops], dev), din.dev,
                                img, mi, mo, dev_status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == alb.ALB_ESHAPE
    assert (outs[1] == 7).all()                                              # untouched
    assert np.array_equal(outs[0].cpu().numpy(), O.chain_mask(ops[0], good.cpu().numpy()))
