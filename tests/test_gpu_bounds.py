"""The bounds-checked build of the library (compiled with ALB_CHECK_BOUNDS):
every instrumented gather, staging copy and store tests its index against
its region, counts failures on the device and skips the access.  A fresh
process loads that build, runs the transforms (ragged sizes down to 1 px,
strong zoom, border-crossing warps, masks), the fused and plain chains and
the float warp, checks a sample against the oracle and reads the counters:
zero violations."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import oracle as O
from helpers import EXTRA_CFGS, suite_cfgs, to_lib, CHAIN_CFG
from paper_1809_06839_gb300 import alb, synth
from paper_1809_06839_gb300.ragged import DeviceBatch, mask_output_batch, output_batch, to_device
from paper_1809_06839_gb300.autograd import augment
dev = torch.device("cuda")
alb.load()
checked, _, _ = alb.alb_bounds_violations(reset=True)
assert checked, "not the checked build"
sizes = [(333, 500), (1, 97), (88, 1), (1, 1), (257, 65), (700, 40), (64, 64)]
rb = synth.ragged_noise(sizes, seed=3)
masks = synth.ragged_masks(sizes, seed=3)
din, dmi = DeviceBatch(to_device(rb, dev)), DeviceBatch(to_device(masks, dev))
cfgs = {**suite_cfgs(), **EXTRA_CFGS}
cfgs["ZoomOut"] = O.make_cfg(O.SHIFT_SCALE_ROTATE, lo=(0.05, 0.3, -80.0), hi=(0.05, 0.3, -80.0))
cfgs["ZoomIn"] = O.make_cfg(O.SHIFT_SCALE_ROTATE, lo=(-0.05, 3.0, 33.0), hi=(-0.05, 3.0, 33.0))
for name, oc in sorted(cfgs.items()):
    if name == "RandomCrop64":
        continue
    ops = [O.sample_params(oc, 3, oc.tid, i, h, w) for i, (h, w) in enumerate(sizes)]
    lps = [to_lib(p, alb) for p in ops]
    dout = output_batch(lps, rb.shapes, dev)
    dmo = mask_output_batch(lps, masks.shapes, dev)
    alb.alb_apply_ragged(oc.tid, len(sizes), alb.params_to_device(lps, dev), din.dev, dout.dev, dmi.dev, dmo.dev,
                         ws=alb.workspace(alb.alb_workspace_size(oc.tid, len(sizes)), dev))
    torch.cuda.synchronize()
    ref = O.apply_image(ops[0], rb.image(0).numpy())
    got = dout.rb.image(0).cpu().numpy()
    if oc.tid != O.SHIFT_HSV:
        assert np.array_equal(got, ref), name
# fused and plain chain, both jitter modes
csz = [(256 + (i * 97) % 769, 256 + (i * 193) % 769) for i in range(10)] + [(3, 900)]
crb = synth.ragged_noise(csz, seed=4)
cin = DeviceBatch(to_device(crb, dev))
oc = O.make_cfg(O.CHAIN, **CHAIN_CFG)
cops = [O.sample_params(oc, 4, 20, i, h, w) for i, (h, w) in enumerate(csz)]
cp = alb.params_to_device([to_lib(p, alb) for p in cops], dev)
for jit in (0, 1):
    for mode in (alb.MODE_FUSED, alb.MODE_PLAIN):
        out = torch.empty((len(csz), 3, 224, 224), dtype=torch.bfloat16, device=dev)
        alb.alb_apply_batch(alb.chain_cfg(jitter=jit), len(csz), cp, cin.dev, out, mode)
torch.cuda.synchronize()
# float warp forward
x = synth.float_images(2, 3, 96, 130, seed=5).to(dev)
for sc in (0.3, 1.0, 3.0):
    t = lambda v: torch.tensor(v, dtype=torch.float32, device=dev)
    augment(x, t([20.0, -70.0]), t([sc, sc]), t([0.03, -0.05]), t([0.01, 0.04]), t([1.0, 1.1]), t([0.0, 0.02]),
            t([1.0, 0.9]))
torch.cuda.synchronize()
checked, count, line = alb.alb_bounds_violations()
print("BOUNDS", count, line)
assert count == 0, (count, line)
'''


def test_checked_build_has_no_bounds_violations():
    env = dict(os.environ, ALB_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "BOUNDS 0 0" in r.stdout
