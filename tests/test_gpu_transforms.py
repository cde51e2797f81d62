"""GPU parity of every per-image transform (images, masks, boxes) and of the
device sampler against the oracle, through the C ABI.  Bit-exact for copies,
LUT/integer ops, Q5 warps/resizes and nearest masks; ShiftHSV (float32 on the
GPU, float64 in the oracle) within 1 LSB on at most 0.1 % of pixels; boxes
within 1e-4 px."""
import numpy as np
import pytest
import torch

import oracle as O
from guards import assert_guards, guarded_output_batch
from helpers import EXTRA_CFGS, cfg_to_lib, same_params, suite_cfgs, to_lib

from paper_1809_06839_gb300 import alb, synth
from paper_1809_06839_gb300.ragged import DeviceBatch, mask_output_batch, output_batch, to_device

pytestmark = pytest.mark.gpu

ALL = {**suite_cfgs(), **EXTRA_CFGS}
# sizes spanning several work items and ragged tails, plus degenerate 1-px axes
SIZES = [(333, 500), (129, 200), (64, 64), (17, 509), (300, 251), (1, 97), (88, 1), (1, 1), (257, 65)]
CROP_SIZES = [(333, 500), (129, 200), (64, 64), (300, 251), (65, 64), (500, 333)]


def sizes_for(name):
    return CROP_SIZES if name == "RandomCrop64" else SIZES


def hsv_ok(got, ref):
    d = np.abs(got.astype(np.int32) - ref.astype(np.int32))
    return d.max() <= 1 and (d > 0).mean() <= 1e-3


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    alb.load()
    return torch.device("cuda")


def run_ragged(name, sizes, seed, dev, with_mask=True, with_boxes=True, oc=None):
    oc = oc if oc is not None else ALL[name]
    rb = synth.ragged_noise(sizes, seed=seed)
    masks = synth.ragged_masks(sizes, seed=seed)
    ops = [O.sample_params(oc, seed, oc.tid, i, h, w) for i, (h, w) in enumerate(sizes)]
    lps = [to_lib(p, alb) for p in ops]
    din = DeviceBatch(to_device(rb, dev))
    dout = guarded_output_batch(lps, rb.shapes, dev)
    prm = alb.params_to_device(lps, dev)
    n = len(sizes)
    dmi = dmo = None
    if with_mask:
        dmi = DeviceBatch(to_device(masks, dev))
        dmo = guarded_output_batch(lps, masks.shapes, dev, mask=True)
    cap = 50
    boxes = np.zeros((n, cap, 4), np.float32)
    nb = np.zeros(n, np.int32)
    for i, (h, w) in enumerate(sizes):
        b = synth.random_boxes(h, w, i, seed)[:cap]
        boxes[i, :len(b)] = b
        nb[i] = len(b)
    bd = torch.from_numpy(boxes).to(dev)
    nbd = torch.from_numpy(nb).to(dev)
    bo = torch.zeros_like(bd)
    nbo = torch.zeros_like(nbd)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = alb.workspace(alb.alb_workspace_size(oc.tid, n), dev)
    alb.alb_apply_ragged(oc.tid, n, prm, din.dev, dout.dev, dmi.dev if dmi else None, dmo.dev if dmo else None,
                         bd if with_boxes else None, nbd if with_boxes else None, cap if with_boxes else 0,
                         bo if with_boxes else None, nbo if with_boxes else None, ws, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert_guards(dout, (name, "image"))
    if dmo is not None:
        assert_guards(dmo, (name, "mask"))
    return rb, masks, ops, dout, dmo, boxes, nb, bo.cpu().numpy(), nbo.cpu().numpy()


@pytest.mark.parametrize("name", sorted(ALL))
def test_ragged_transform_matches_oracle(dev, name):
    sizes = sizes_for(name)
    with_boxes = ALL[name].tid != O.ELASTIC           # boxes are not defined for the elastic field
    rb, masks, ops, dout, dmo, boxes, nb, bo, nbo = run_ragged(name, sizes, 1809, dev, with_boxes=with_boxes)
    for i, (h, w) in enumerate(sizes):
        img = rb.image(i).numpy()
        ref = O.apply_image(ops[i], img)
        got = dout.rb.image(i).cpu().numpy()
        assert got.shape == ref.shape
        if ops[i].tid == O.SHIFT_HSV:
            assert hsv_ok(got, ref), (name, i)
        else:
            assert np.array_equal(got, ref), (name, i, (got != ref).sum())
        mref = O.apply_mask(ops[i], masks.image(i).numpy())
        assert np.array_equal(dmo.rb.image(i).cpu().numpy(), mref), (name, "mask", i)
        if not with_boxes:
            continue
        bref = O.apply_boxes(ops[i], h, w, boxes[i, :nb[i]])
        assert nbo[i] == len(bref), (name, "boxes", i)
        assert np.abs(bo[i, :nbo[i]] - bref).max(initial=0) <= 1e-4


def test_resize_scale_classes_in_one_batch(dev):
    """One ragged Resize batch whose images fall in the three scale classes
    that the tile plans route apart -- windows within 17/16 of the output
    (enlargements and mild reductions), reductions up to about 2x, and
    stronger ones (on either axis) -- each through its own tile shape, checked
    against the oracle bit for bit with masks and boxes."""
    oc = O.make_cfg(O.RESIZE, out_h=200, out_w=160)
    sizes = [(150, 120), (210, 168), (200, 160), (1, 1), (380, 300), (250, 170), (1000, 150), (120, 700),
             (700, 20), (433, 351)]
    rb, masks, ops, dout, dmo, boxes, nb, bo, nbo = run_ragged("Resize200x160", sizes, 7, dev, oc=oc)
    for i, (h, w) in enumerate(sizes):
        ref = O.apply_image(ops[i], rb.image(i).numpy())
        got = dout.rb.image(i).cpu().numpy()
        assert got.shape == ref.shape == (200, 160, 3)
        assert np.array_equal(got, ref), (sizes[i], (got != ref).sum())
        assert np.array_equal(dmo.rb.image(i).cpu().numpy(), O.apply_mask(ops[i], masks.image(i).numpy())), sizes[i]
        bref = O.apply_boxes(ops[i], h, w, boxes[i, :nb[i]])
        assert nbo[i] == len(bref), sizes[i]
        assert np.abs(bo[i, :nbo[i]] - bref).max(initial=0) <= 1e-4


@pytest.mark.parametrize("name", sorted(ALL))
def test_device_sampler_matches_oracle(dev, name):
    oc = ALL[name]
    sizes = [(333 + (i * 29) % 168, 333 + (i * 53) % 168) for i in range(300)]
    descs = []
    for h, w in sizes:
        d = alb.Image()
        d.h, d.w, d.c, d.row_stride = h, w, 3, 3 * w
        descs.append(d)
    ddev = alb.descs_to_device(descs, dev)
    pdev = torch.zeros(len(sizes) * 232, dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    alb.alb_sample_params_batch(cfg_to_lib(oc, alb), 1809, oc.tid, 0, len(sizes), ddev, pdev, status)
    got = alb.params_from_device(pdev)
    assert int(status.item()) == 0
    for i, (h, w) in enumerate(sizes):
        ref = O.sample_params(oc, 1809, oc.tid, i, h, w)
        # cos/sin/log/exp on the device may differ from the host libm in the last
        # ulp: the forward matrix is compared to 1e-12; Q16 integers and every
        # other field must be identical
        err = same_params(ref, got[i], rel_m=1e-12)
        assert err is None, (name, i, err)


def test_single_image_apply_and_in_place(dev):
    img = synth.value_noise_image(77, 91, 3)
    op = O.sample_params(ALL["Gamma"], 5, 8, 0, 77, 91)
    g = img.to(dev)
    out, _, _, _ = alb.alb_apply(to_lib(op, alb), g)
    assert np.array_equal(out.cpu().numpy(), O.apply_image(op, img.numpy()))
    alb.alb_apply(to_lib(op, alb), g, out=g)            # in place
    assert np.array_equal(g.cpu().numpy(), O.apply_image(op, img.numpy()))
    with pytest.raises(alb.AlbError):
        hp = O.sample_params(ALL["HorizontalFlip"], 5, 1, 0, 77, 91)
        alb.alb_apply(to_lib(hp, alb), g, out=g)       # geometric in place is rejected


def test_empty_and_strided_images(dev):
    # zero-row image: a no-op; a padded row stride (a column slice) is honoured
    e = torch.empty((0, 5, 3), dtype=torch.uint8, device=dev)
    op = O.sample_params(ALL["VerticalFlip"], 1, 2, 0, 0 + 1, 5)
    alb.alb_apply(to_lib(op, alb), e, out=torch.empty_like(e))
    base = synth.value_noise_image(40, 80, 4)
    view = base.to(dev)[:, 10:60]                       # row stride 240 > 50*3
    op = O.sample_params(ALL["Rotate"], 1, 13, 0, 40, 50)
    out, _, _, _ = alb.alb_apply(to_lib(op, alb), view)
    assert np.array_equal(out.cpu().numpy(), O.apply_image(op, np.ascontiguousarray(base.numpy()[:, 10:60])))


def test_multichannel_mask_planes(dev):
    # N instance planes interleaved (c = 5) follow the image geometry bit-exactly
    h, w = 120, 150
    planes = torch.stack([synth.blob_mask(h, w, i, n_classes=2) for i in range(5)], dim=2).contiguous()
    img = synth.value_noise_image(h, w, 1)
    for name in ("ShiftScaleRotate", "RandomSizedCrop512", "PadToSize512", "HorizontalFlip", "Transpose"):
        op = O.sample_params(ALL[name], 3, 4, 0, h, w)
        _, mo, _, _ = alb.alb_apply(to_lib(op, alb), img.to(dev), mask=planes.to(dev))
        assert np.array_equal(mo.cpu().numpy(), O.apply_mask(op, planes.numpy())), name


def test_small_plain_workload_full_size(dev):
    """64 x 256x256 images + masks: HFlip -> Brightness/Contrast -> RandomCrop 224,
    bit-exact against the oracle for every image (the oracle takes seconds)."""
    n, seed = 64, 1809
    sizes = [(256, 256)] * n
    rb = synth.ragged_noise(sizes, seed=seed)
    masks = synth.ragged_masks(sizes, seed=seed)
    steps = [O.make_cfg(O.HFLIP, p=0.5), O.make_cfg(O.BRIGHTNESS_CONTRAST, lo=(0.8, -20.0), hi=(1.2, 20.0)),
             O.make_cfg(O.RANDOM_CROP, out_h=224, out_w=224)]
    cur = DeviceBatch(to_device(rb, dev))
    curm = DeviceBatch(to_device(masks, dev))
    ref = [rb.image(i).numpy() for i in range(n)]
    refm = [masks.image(i).numpy() for i in range(n)]
    for k, oc in enumerate(steps):
        shapes = cur.rb.shapes
        ops = [O.sample_params(oc, seed, 100 + k, i, s[0], s[1]) for i, s in enumerate(shapes)]
        lps = [to_lib(p, alb) for p in ops]
        nxt = output_batch(lps, shapes, dev)
        nxtm = mask_output_batch(lps, curm.rb.shapes, dev)
        ws = alb.workspace(alb.alb_workspace_size(oc.tid, n), dev)
        alb.alb_apply_ragged(oc.tid, n, alb.params_to_device(lps, dev), cur.dev, nxt.dev, curm.dev, nxtm.dev,
                             ws=ws)
        ref = [O.apply_image(ops[i], ref[i]) for i in range(n)]
        refm = [O.apply_mask(ops[i], refm[i]) for i in range(n)]
        cur, curm = nxt, nxtm
    torch.cuda.synchronize()
    for i in range(n):
        assert np.array_equal(cur.rb.image(i).cpu().numpy(), ref[i]), i
        assert np.array_equal(curm.rb.image(i).cpu().numpy(), refm[i]), i


@pytest.mark.parametrize("kind,arg", [("ssr", 0.3), ("ssr", 0.45), ("ssr", 1.7), ("rot", 45.0), ("rot", -90.0),
                                      ("resize", (37, 61)), ("resize", (700, 20)), ("resize", (1, 1)),
                                      ("resize", (333, 500))])
def test_resample_extremes(dev, kind, arg):
    """Footprints that overflow the staged box (strong down-scaling) take the
    direct-gather fallback inside the tiled kernel; both paths are exact."""
    sizes = [(333, 500), (129, 200), (64, 64), (17, 509), (1, 97)]
    rb = synth.ragged_noise(sizes, seed=4)
    masks = synth.ragged_masks(sizes, seed=4)
    ops = []
    for i, (h, w) in enumerate(sizes):
        p = O.Params()
        p.apply, p.scale, p.alpha, p.gamma, p.sat = 1, 1.0, 1.0, 1.0, 1.0
        if kind in ("ssr", "rot"):
            p.tid = O.SHIFT_SCALE_ROTATE
            p.angle = 17.0 + 11 * i if kind == "ssr" else arg
            p.scale = arg if kind == "ssr" else 1.0
            p.dx, p.dy = 0.03, -0.05
            O.warp_geometry(p, h, w)
        else:
            p.tid = O.RESIZE
            p.out_h, p.out_w, p.ch, p.cw = arg[0], arg[1], h, w
        ops.append(p)
    lps = [to_lib(p, alb) for p in ops]
    din = DeviceBatch(to_device(rb, dev))
    dmi = DeviceBatch(to_device(masks, dev))
    dout = guarded_output_batch(lps, rb.shapes, dev)
    dmo = guarded_output_batch(lps, masks.shapes, dev, mask=True)
    ws = alb.workspace(alb.alb_workspace_size(ops[0].tid, len(sizes)), dev)
    alb.alb_apply_ragged(ops[0].tid, len(sizes), alb.params_to_device(lps, dev), din.dev, dout.dev, dmi.dev, dmo.dev,
                         ws=ws)
    torch.cuda.synchronize()
    assert_guards(dout, kind)
    assert_guards(dmo, (kind, "mask"))
    for i in range(len(sizes)):
        assert np.array_equal(dout.rb.image(i).cpu().numpy(), O.apply_image(ops[i], rb.image(i).numpy())), (kind, i)
        assert np.array_equal(dmo.rb.image(i).cpu().numpy(), O.apply_mask(ops[i], masks.image(i).numpy())), (kind, i)


def test_inconsistent_descriptors_are_rejected_on_device(dev):
    """Descriptors the host cannot inspect (device arrays) are validated per
    image before any pixel is touched: a wrong output size, a crop window
    outside its image or a 1-channel image in an RGB slot record a status and
    the other images are still processed."""
    sizes = [(64, 80), (50, 70), (90, 40)]
    rb = synth.ragged_noise(sizes, seed=8)
    oc = ALL["RandomCrop64"]
    ops = [O.sample_params(O.make_cfg(O.RANDOM_CROP, out_h=32, out_w=32), 8, 3, i, h, w)
           for i, (h, w) in enumerate(sizes)]
    lps = [to_lib(p, alb) for p in ops]
    lps[1].y0 = 40                                          # window 40..72 outside the 50-row image
    din = DeviceBatch(to_device(rb, dev))
    dout = output_batch(lps, rb.shapes, dev)
    descs = list(dout.descs)
    descs[2].w = 31                                          # output narrower than the record says
    out_dev = alb.descs_to_device(descs, dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = alb.workspace(alb.alb_workspace_size(oc.tid, 3), dev)
    alb.alb_apply_ragged(oc.tid, 3, alb.params_to_device(lps, dev), din.dev, out_dev, ws=ws, dev_status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == alb.ALB_ESHAPE
    assert np.array_equal(dout.rb.image(0).cpu().numpy(), O.apply_image(ops[0], rb.image(0).numpy()))
    # a single-channel image in an RGB slot of a ragged photometric launch
    gray = synth.empty_ragged([(20, 30, 1)], device=dev)
    gin = DeviceBatch(gray)
    gout = DeviceBatch(synth.empty_ragged([(20, 30, 1)], device=dev))
    gp = to_lib(O.sample_params(ALL["Gamma"], 1, 8, 0, 20, 30), alb)
    status.zero_()
    ws = alb.workspace(alb.alb_workspace_size(alb.GAMMA, 1), dev)
    alb.alb_apply_ragged(alb.GAMMA, 1, alb.params_to_device([gp], dev), gin.dev, gout.dev, ws=ws, dev_status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == alb.ALB_EINVAL


@pytest.mark.parametrize("name", ["ShiftScaleRotate", "RandomSizedCrop512", "VerticalFlip", "Gamma"])
def test_ragged_masks_with_mixed_channel_counts(dev, name):
    """Ragged masks of 1 and 3 planes in one launch: single-plane masks take the
    specialised kernels, the others the general ones; all match the oracle."""
    oc = ALL[name]
    sizes = [(120, 150), (97, 64), (200, 131)]
    chans = [1, 3, 1]
    rb = synth.ragged_noise(sizes, seed=6)
    mshapes = [(h, w, c) for (h, w), c in zip(sizes, chans)]
    masks = synth.empty_ragged(mshapes)
    for i, (h, w) in enumerate(sizes):
        planes = [synth.blob_mask(h, w, 10 * i + j, n_classes=5) for j in range(chans[i])]
        masks.image(i).copy_(torch.stack(planes, dim=2))
    ops = [O.sample_params(oc, 6, oc.tid, i, h, w) for i, (h, w) in enumerate(sizes)]
    lps = [to_lib(p, alb) for p in ops]
    din = DeviceBatch(to_device(rb, dev))
    dout = output_batch(lps, rb.shapes, dev)
    dmi = DeviceBatch(to_device(masks, dev))
    dmo = mask_output_batch(lps, masks.shapes, dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = alb.workspace(alb.alb_workspace_size(oc.tid, 3), dev)
    alb.alb_apply_ragged(oc.tid, 3, alb.params_to_device(lps, dev), din.dev, dout.dev, dmi.dev, dmo.dev, ws=ws,
                         dev_status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    for i in range(3):
        assert np.array_equal(dmo.rb.image(i).cpu().numpy(), O.apply_mask(ops[i], masks.image(i).numpy())), i


def test_gamma_tables_exact_over_a_dense_gamma_grid(dev):
    """Every entry of 3000 gamma tables (gamma on a dense grid over [0.5, 2.0])
    equals the oracle's float64 definition: the device builds the tables in
    float32 and falls back to float64 near rounding points, so the grid
    exercises both branches."""
    from paper_1809_06839_gb300.synth import Ragged
    n = 3000
    gammas = np.linspace(0.5, 2.0, n)
    row = np.repeat(np.arange(256, dtype=np.uint8), 3)
    flat = torch.from_numpy(np.tile(row, n))
    rb = Ragged(flat.to(dev), [768 * i for i in range(n)], [(1, 256, 3)] * n)
    din = DeviceBatch(rb)
    ops = [O.sample_params(O.make_cfg(O.GAMMA, lo=(g,), hi=(g,)), 1, 2, i, 1, 256) for i, g in enumerate(gammas)]
    prm = alb.params_to_device([to_lib(o, alb) for o in ops], dev)
    dout = output_batch([to_lib(o, alb) for o in ops], rb.shapes, dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    alb.alb_apply_ragged(O.GAMMA, n, prm, din.dev, dout.dev, ws=alb.workspace(alb.alb_workspace_size(O.GAMMA, n), dev),
                         dev_status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    got = dout.rb.flat.cpu().numpy().reshape(n, 256, 3)
    for i in range(n):
        ref = O.apply_image(ops[i], row.reshape(1, 256, 3))[0]
        assert np.array_equal(got[i], ref), (i, gammas[i])


@pytest.mark.parametrize("name,cfg", [
    ("grid G=1", O.make_cfg(O.GRID_DISTORTION, lo=(-0.5, 1), hi=(0.5, 1))),
    ("grid G=12 strong", O.make_cfg(O.GRID_DISTORTION, lo=(-0.9, 12), hi=(0.9, 12))),
    ("elastic S=4 large", O.make_cfg(O.ELASTIC, lo=(40.0, 2))),
    ("elastic S=256", O.make_cfg(O.ELASTIC, lo=(3.0, 8))),
    ("elastic p=0.5", O.make_cfg(O.ELASTIC, p=0.5, lo=(5.0, 5))),
])
def test_distortion_extremes(dev, name, cfg):
    """Few and many grid cells with strong factors, dense and sparse elastic
    lattices with large displacements (taps reflected far outside), half the
    records not applied; images and masks bit-exact."""
    sizes = [(333, 500), (1, 97), (88, 1), (1, 1), (257, 65), (700, 40), (31, 900)]
    rb = synth.ragged_noise(sizes, seed=4)
    masks = synth.ragged_masks(sizes, seed=4)
    ops = [O.sample_params(cfg, 4, cfg.tid, i, h, w) for i, (h, w) in enumerate(sizes)]
    lps = [to_lib(p, alb) for p in ops]
    din, dmi = DeviceBatch(to_device(rb, dev)), DeviceBatch(to_device(masks, dev))
    dout, dmo = guarded_output_batch(lps, rb.shapes, dev), guarded_output_batch(lps, masks.shapes, dev, mask=True)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    n = len(sizes)
    alb.alb_apply_ragged(cfg.tid, n, alb.params_to_device(lps, dev), din.dev, dout.dev, dmi.dev, dmo.dev,
                         ws=alb.workspace(alb.alb_workspace_size(cfg.tid, n), dev), dev_status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert_guards(dout, name)
    assert_guards(dmo, (name, "mask"))
    for i in range(n):
        assert np.array_equal(dout.rb.image(i).cpu().numpy(), O.apply_image(ops[i], rb.image(i).numpy())), (name, i)
        assert np.array_equal(dmo.rb.image(i).cpu().numpy(), O.apply_mask(ops[i], masks.image(i).numpy())), (name, i)
