"""End-to-end entry point with host buffers (ffb_expand_cov_host): images in
host memory stream to the device in parts through a ring of device buffers,
are expanded (Alg. 1 steps 3-4) and accumulated into the covariance (Alg. 2
steps 1-4), and the mean and blocks come back to host memory.  Checked
against the device-buffer path (ffb_expand, ffb_covariance, ffb_cov_get) on
the same images: several parts with a ragged last one and more parts than
device slots, continuation with reset = 0, pageable host memory, and the
BF16x3 precision at L = 128.  The coefficients are the same per image; the
covariance sums run over other image ranges, so the statistics agree to the
streaming tolerance of the accumulator (relative 1e-6)."""
import numpy as np
import pytest
import torch

from paper_1412_0781_gb300 import Plan, FFBError, data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def stack(L, n, dev):
    spec = data.StackSpec(n, L, L / 2, 8, (1.0, L / 16), 1 / 10, 1412 + L)
    imgs, _, _ = data.blob_stack(spec, device=dev)
    return imgs


def device_stats(plan, d_imgs):
    coef = plan.expand(d_imgs)
    plan.covariance(coef, reset=True)
    m, C = plan.cov_get()
    return m.cpu().numpy(), C.cpu().numpy()


def test_host_call_matches_device_path_over_many_parts(dev):
    plan = Plan(64, 0.5, 32.0, eps=1e-6, precision="fp32")
    n = 7 * plan.chunk + 37            # four parts of two chunks, the last ragged
    d_imgs = stack(64, n, dev)
    h_imgs = d_imgs.cpu().pin_memory()
    m1, C1 = device_stats(plan, d_imgs)
    for _ in range(2):                 # a second call reuses the plan's buffers
        m2, C2 = plan.expand_cov_host(h_imgs, reset=True)
        assert rel(C2.numpy(), C1) < 1e-6 and rel(m2.numpy(), m1) < 1e-6
    # continuation: two calls, the second with reset = 0, equal one call
    k = 3 * plan.chunk + 11
    plan.expand_cov_host(h_imgs[:k], reset=True)
    m3, C3 = plan.expand_cov_host(h_imgs[k:], reset=False)
    assert rel(C3.numpy(), C1) < 1e-6 and rel(m3.numpy(), m1) < 1e-6
    # pageable host memory gives the same statistics
    m4, C4 = plan.expand_cov_host(d_imgs.cpu(), reset=True)
    assert rel(C4.numpy(), C1) < 1e-6 and rel(m4.numpy(), m1) < 1e-6
    plan.close()


def test_host_call_bf16x3_l128(dev):
    plan = Plan(128, 0.5, 64.0, eps=1e-6, precision="bf16x3")
    n = 5 * plan.chunk + 19
    d_imgs = stack(128, n, dev)
    m1, C1 = device_stats(plan, d_imgs)
    out_m = torch.empty(plan.p[0], dtype=torch.float64).pin_memory()
    out_C = torch.empty(plan.cov_total, dtype=torch.float64).pin_memory()
    m2, C2 = plan.expand_cov_host(d_imgs.cpu().pin_memory(), reset=True, mean_out=out_m, C_out=out_C)
    assert m2.data_ptr() == out_m.data_ptr() and C2.data_ptr() == out_C.data_ptr()
    assert rel(C2.numpy(), C1) < 1e-6 and rel(m2.numpy(), m1) < 1e-6
    plan.close()


def test_host_call_arguments(dev):
    plan = Plan(64, 0.5, 32.0, eps=1e-6, precision="fp32")
    with pytest.raises(FFBError):      # nothing accumulated, statistics asked for
        plan.expand_cov_host(torch.empty((0, 64, 64)), reset=True)
    with pytest.raises(TypeError):     # device tensors go through expand / covariance
        plan.expand_cov_host(torch.empty((4, 64, 64), device=dev), reset=True)
    plan.close()
