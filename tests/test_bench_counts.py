"""The benchmark's roofline arithmetic (bench.py, host only): the algorithmic
work per image it divides by the kernels' event times, the derived FP32 peak,
and the executed work of the tensor-core ring DFT, at the L = 128 workload
(n_xi = 128, n_theta = 512, P = 4848, sum p_k^2 = 190,224).  The counts follow
the method: the interpolation at the taps the accuracy needs
(w_a = ceil(log10(1/eps)) + 1 = 7 at eps = 1e-6, 5 flop per tap), the
real-input oversampled 2-D FFT, the Hermitian half-ring DFT of Eq. 1DFFT,
4 P n_xi for the quadrature of Eq. a and 2 sum p_k^2 for the covariance of
Eqs. ck, ck_0."""
import math
import types

import pytest

import bench


def plan_l128():
    # the sizes of the L = 128 plan (c = 1/2, R = 64, literal sampling
    # criterion) that the counts read; p_k is set where a test needs it
    return types.SimpleNamespace(n_xi=128, n_theta=512, N=256, L=128, w=8, P=4848, p=[],
                                 polar_variant=2)


def test_algorithmic_counts_at_l128():
    plan = plan_l128()
    f = bench.algorithmic_flops(plan, eps=1e-6)
    fft2 = 2.5 * 256 * 256 * math.log2(256 * 256) / 2
    interp = 128 * 256 * 7 * 7 * 5
    assert f["grid_interp"] == pytest.approx(fft2 + interp)
    assert f["grid_interp"] / 1e6 == pytest.approx(9.339, abs=1e-3)
    assert f["ring_fft"] / 1e6 == pytest.approx(1.4746, abs=1e-4)       # 128 x 2.5 x 512 x 9
    assert f["bessel"] == 4.0 * 4848 * 128                                # 2.48 MFLOP
    # the covariance count is 2 sum p_k^2 over the plan's blocks
    plan.p = [5, 3]
    assert bench.algorithmic_flops(plan)["covariance"] == 2.0 * (25 + 9)


def test_accuracy_width_follows_eps():
    plan = plan_l128()
    lo = bench.algorithmic_flops(plan, eps=1e-6)["grid_interp"]
    hi = bench.algorithmic_flops(plan, eps=1e-5)["grid_interp"]   # w_a = 6
    assert lo - hi == pytest.approx(128 * 256 * (49 - 36) * 5)


def test_fp32_peak_and_tensor_ring_dft():
    assert bench.fp32_peak_tflops(152, 2070) == pytest.approx(80.54784)
    on, exe = bench.tc_ring_dft(plan_l128(), "bf16x3")
    assert on and exe == 2 * 3 * 128 * 192 * 256 * 2                     # 75.5 MFLOP per image
    assert not bench.tc_ring_dft(plan_l128(), "tf32x3")[0]
    small = types.SimpleNamespace(n_xi=64, n_theta=256, polar_variant=2)
    assert not bench.tc_ring_dft(small, "bf16x3")[0]


def test_frac_reproduces_from_counts():
    """frac = algorithmic flops x images / kernel time / peak, the way the
    line's roofline is formed: 9.339 MFLOP x 100,000 images in 65.6 ms at
    80.55 TFLOP/s is 0.177."""
    plan = plan_l128()
    f = bench.algorithmic_flops(plan)["grid_interp"]
    achieved = f * 100000 / 65.6e-3 / 1e12
    assert achieved / bench.fp32_peak_tflops(152, 2070) == pytest.approx(0.1767, abs=5e-4)
