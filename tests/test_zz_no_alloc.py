"""The allocation-free entry point alb_apply_ragged_static, for callers that
cannot allocate device memory (so cannot pass a workspace): its output must
equal alb_apply_ragged's on the same inputs, on two calls in a row (the second
call reuses the static scratch the first one left behind).  Collected last so
that a stop-at-first-failure run has already run every other test; it also
passes alone in a fresh process."""
import numpy as np
import pytest
import torch

import oracle as O
from helpers import suite_cfgs, to_lib

from paper_1809_06839_gb300 import alb, synth
from paper_1809_06839_gb300.ragged import DeviceBatch, output_batch, to_device

pytestmark = pytest.mark.gpu

CASES = ["Equalize", "Gamma", "ShiftRGB", "HorizontalFlip", "Rotate", "PadToSize512"]


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    alb.load()
    return torch.device("cuda")


def batch(seed, n, dev):
    sizes = [(40 + (i * 37 + seed) % 300, 33 + (i * 53 + seed) % 280) for i in range(n)]
    return sizes, DeviceBatch(to_device(synth.ragged_noise(sizes, seed=seed), dev))


@pytest.mark.parametrize("name", CASES)
def test_static_scratch_matches_workspace_path(dev, name):
    oc = suite_cfgs()[name]
    for call, seed in enumerate((11, 12)):            # two calls in a row, different inputs
        n = 7 + 5 * call
        sizes, din = batch(seed, n, dev)
        lps = [to_lib(O.sample_params(oc, seed, oc.tid, i, h, w), alb) for i, (h, w) in enumerate(sizes)]
        prm = alb.params_to_device(lps, dev)
        ref = output_batch(lps, din.rb.shapes, dev)
        got = output_batch(lps, din.rb.shapes, dev)
        ws = alb.workspace(alb.alb_workspace_size(oc.tid, n), dev)
        alb.alb_apply_ragged(oc.tid, n, prm, din.dev, ref.dev, ws=ws)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        alb.alb_apply_ragged_static(oc.tid, n, prm, din.dev, got.dev, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        for i in range(n):
            assert np.array_equal(got.rb.image(i).cpu().numpy(), ref.rb.image(i).cpu().numpy()), (name, call, i)


def test_static_scratch_rejects_too_many_images(dev):
    with pytest.raises(alb.AlbError) as e:
        alb.alb_apply_ragged_static(alb.EQUALIZE, 2049, None, None, None)
    assert e.value.code == alb.ALB_ECAPACITY
    assert "2048" in alb.alb_last_error()
