"""Failure handling on the GPU without a GPU fault: the bounded wait of the
bulk-copy kernels gives up on a barrier phase that no copy will complete,
the drain waits for the copies that were issued, and the status word reads
ALB_ETIMEOUT; the context stays usable."""
import numpy as np
import pytest
import torch

from paper_1809_06839_gb300 import alb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    alb.load()
    return torch.device("cuda")


@pytest.mark.parametrize("spins", [1, 8, 256])
def test_bounded_wait_times_out_and_drains(dev, spins):
    src = torch.arange(32, dtype=torch.uint8, device=dev) * 7 + 3
    out = torch.zeros(32, dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    alb.alb_selftest_bounded_wait(spins, src, out, status)
    torch.cuda.synchronize()                        # the launch completed
    assert int(status.item()) == alb.ALB_ETIMEOUT
    assert torch.equal(out, src)                    # the issued copies landed before the CTA ended
    # the context is still usable: an ordinary transform runs afterwards
    x = torch.arange(2 * 3 * 3, dtype=torch.uint8, device=dev).reshape(2, 3, 3)
    p = alb.Params()
    p.tid, p.apply, p.in_h, p.in_w, p.out_h, p.out_w = alb.HFLIP, 1, 2, 3, 2, 3
    y, _, _, _ = alb.alb_apply(p, x)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), x.cpu().numpy()[:, ::-1])


def test_status_word_keeps_the_first_error(dev):
    src = torch.zeros(32, dtype=torch.uint8, device=dev)
    out = torch.zeros(32, dtype=torch.uint8, device=dev)
    status = torch.full((1,), alb.ALB_ESHAPE, dtype=torch.int32, device=dev)
    alb.alb_selftest_bounded_wait(4, src, out, status)
    torch.cuda.synchronize()
    assert int(status.item()) == alb.ALB_ESHAPE
