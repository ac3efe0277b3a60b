"""The bounded device-side waits of the tensor-core kernels (radial quadrature
and covariance): a wait that runs out latches FFB_ERR_TIMEOUT, the next
synchronising call returns and clears it, the kernel drains what it issued
and returns, and the plan computes normally afterwards.  The waits are made
to run out by a zero cycle budget (ffb_set_wait_budget); nothing here faults
or hangs the device."""
import numpy as np
import pytest
import torch

from paper_1412_0781_gb300 import FFBError, Plan, data

pytestmark = pytest.mark.gpu
FFB_ERR_TIMEOUT = -6


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _raises_timeout(fn):
    with pytest.raises(FFBError) as e:
        fn()
    assert e.value.status == FFB_ERR_TIMEOUT


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_wait_timeout_is_latched_cleared_and_recovered(dev, prec):
    spec = data.StackSpec(1024, 64, 32.0, 12, (1.0, 4.0), 0.2, 20141210)
    imgs, _, _ = data.blob_stack(spec, device=dev)
    gp = Plan(64, 0.5, 32.0, eps=1e-6, precision=prec)
    ref = gp.expand(imgs)
    gp.covariance(ref, reset=True)
    m_ref, C_ref = gp.cov_get()
    gp.sync()

    # radial quadrature: the producer / MMA / epilogue waits give up
    gp.set_wait_budget(0)
    scratch = torch.empty_like(ref)

    def expand_and_sync():
        gp.expand(imgs, out=scratch)
        gp.sync()
    _raises_timeout(expand_and_sync)
    gp.sync()                                 # the latch was cleared

    # covariance: the tile-buffer and accumulator waits give up
    def cov_and_sync():
        gp.covariance(ref, reset=True)
        gp.sync()
    _raises_timeout(cov_and_sync)
    gp.sync()

    # default budget again: the same results as before
    gp.set_wait_budget(-1)
    again = gp.expand(imgs)
    gp.covariance(again, reset=True)
    m, C = gp.cov_get()
    gp.sync()
    assert torch.equal(again, ref)
    assert torch.allclose(m, m_ref, rtol=1e-12, atol=0)
    Cn, Cr = C.cpu().numpy(), C_ref.cpu().numpy()
    assert np.max(np.abs(Cn - Cr)) <= 1e-9 * np.max(np.abs(Cr))
