"""R and c estimated from the images (Sec. V) on the GPU against the FP64
oracle: the mean radial variance, the radial power spectrum, the noise level,
and the resulting R and c."""
import math

import numpy as np
import pytest
import torch

from oracle import estimate as est
from oracle import fb
from paper_1412_0781_gb300 import FFBError, Plan, data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _compare(dev, x, L, sigma2=None, frac=0.999):
    plan = Plan(L, 0.5, L / 2, eps=1e-6)
    got = plan.estimate_support(x.to(dev).contiguous(), frac=frac, sigma2=sigma2)
    op = fb.make_plan(L, 0.5, L / 2)
    R, c, s2, V, P = est.estimate(op, x.double().numpy(), frac=frac, sigma2=sigma2)
    ev = np.max(np.abs(got["radial_variance"] - V)) / np.max(np.abs(V))
    ep = np.max(np.abs(got["radial_power"] - P)) / np.max(np.abs(P))
    print("L=%d radial variance err %.2e, radial power err %.2e, R %g/%g, c %g/%g" %
          (L, ev, ep, got["R"], R, got["c"], c))
    assert ev <= 1e-6
    assert ep <= 1e-5
    assert abs(got["sigma2"] - s2) <= 1e-6 * max(s2, 1e-30)
    assert got["R"] == R
    assert got["c"] == c
    plan.close()
    return got


def test_estimate_tiny_stack(dev):
    imgs, _, _ = data.blob_stack(data.TINY)
    _compare(dev, imgs, 32)                       # separate-kernel NUFFT path


def test_estimate_l64_stack_fused_path(dev):
    spec = data.StackSpec(300, 64, 32.0, 12, (1.0, 4.0), 0.5, 4242)
    imgs, _, s2 = data.blob_stack(spec)
    got = _compare(dev, imgs, 64)                 # shared-memory grid path
    assert abs(got["sigma2"] / s2 - 1.0) < 0.05


def test_estimate_gaussian_closed_form(dev):
    L, s = 32, 2.0
    i = torch.arange(L, dtype=torch.float64) - L // 2
    G = torch.exp(-(i[:, None] ** 2 + i[None, :] ** 2) / (2 * s * s))
    a = torch.from_numpy(np.random.default_rng(4).standard_normal(50))
    x = (a[:, None, None] * G[None]).float()
    got = _compare(dev, x, L, sigma2=0.0)
    assert abs(got["R"] - s * math.sqrt(math.log(1000.0))) <= 1.0


def test_estimate_l128_sample(dev):
    spec = data.FP32_L128
    imgs, _, _ = data.blob_stack(spec, n=48)
    _compare(dev, imgs, 128)


def test_estimate_rejects_bad_arguments(dev):
    plan = Plan(32, 0.5, 16.0)
    x = torch.zeros((4, 32, 32), device=dev)
    with pytest.raises(FFBError):
        plan.estimate_support(x, frac=0.0)
    with pytest.raises(FFBError):
        plan.estimate_support(x[:0].contiguous())
