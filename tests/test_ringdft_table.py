"""Host logic of the ring DFT that runs on the tensor cores (Eq. 1DFFT at
n_theta = 512 with BF16x3): the tables the plan builds on the host (exported
as ffb_ringdft_table; no GPU needed).

For a ring of a real image F(theta + pi) = conj F(theta), so with the half
ring f_l = u_l + i v_l, l < n_theta/2, the transform of Eq. 1DFFT is
F_k = 2 s sum_l u_l e^{-i k theta_l} for even k and
F_k = 2 s sum_l v_l (sin k theta_l + i cos k theta_l) for odd k, s = 2 pi /
n_theta: two real contractions with the even-k and the odd-k table.
Checked here:
  * the tables against that closed form, hi + lo within the bf16 split's
    bound 2^-17 of each entry, columns above k_max zero;
  * the contraction of conjugate-completed random rings with the tables
    against the oracle's plain ring DFT of the full rings;
  * the BF16x3 form (hi-hi + hi-lo + lo-hi with the rings split the same way)
    within 2e-5 relative L2 of the exact transform;
  * unsupported sizes rejected."""
import math
import types

import numpy as np
import pytest

from oracle import fb


@pytest.fixture(scope="module")
def ffb():
    from paper_1412_0781_gb300 import build
    build.build()
    from paper_1412_0781_gb300 import ffb as mod
    return mod


def bf16(x):
    """Round to bfloat16 (nearest even) and return float64."""
    a = np.asarray(x, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("n_theta,k_max", [(512, 182), (512, 150), (256, 85)])
def test_tables_match_the_closed_form(ffb, n_theta, k_max):
    hi, lo = ffb.ringdft_table(n_theta, k_max)
    T = hi.astype(np.float64) + lo.astype(np.float64)
    s = 2.0 * math.pi / n_theta
    th = 2.0 * math.pi * np.arange(n_theta // 2) / n_theta
    for par in (0, 1):
        for col in range(192):
            k, c = 2 * (col // 2) + par, col % 2
            if k > k_max:
                assert not T[par, col].any()
                continue
            if par == 0:
                want = -2 * s * np.sin(k * th) if c else 2 * s * np.cos(k * th)
            else:
                want = 2 * s * np.cos(k * th) if c else 2 * s * np.sin(k * th)
            assert np.all(np.abs(T[par, col] - want) <= 2.0 ** -17 * np.abs(want) + 1e-12)
            assert np.array_equal(bf16(hi[par, col]), hi[par, col].astype(np.float64))


def test_contraction_equals_the_oracle_ring_dft(ffb):
    n_theta, k_max = 512, 182
    hi, lo = ffb.ringdft_table(n_theta, k_max)
    T = hi.astype(np.float64) + lo.astype(np.float64)
    rng = np.random.default_rng(1412)
    half = rng.standard_normal((6, n_theta // 2)) + 1j * rng.standard_normal((6, n_theta // 2))
    full = np.concatenate([half, np.conj(half)], axis=1)          # F(theta + pi) = conj F(theta)
    want = fb.ring_dft(types.SimpleNamespace(n_theta=n_theta, k_max=k_max), full)
    De, Do = half.real @ T[0].T, half.imag @ T[1].T               # (rings, 192)
    got = np.zeros_like(want)
    for e in range(96):
        if 2 * e <= k_max:
            got[:, 2 * e] = De[:, 2 * e] + 1j * De[:, 2 * e + 1]
        if 2 * e + 1 <= k_max:
            got[:, 2 * e + 1] = Do[:, 2 * e] + 1j * Do[:, 2 * e + 1]
    # the tables carry the bf16 split's error (2^-17 per entry)
    assert np.linalg.norm(got - want) <= 2e-5 * np.linalg.norm(want)
    # and the exact tables reproduce the oracle to rounding
    th = 2.0 * math.pi * np.arange(n_theta // 2) / n_theta
    s = 2.0 * math.pi / n_theta
    k = np.arange(k_max + 1)
    E = 2 * s * np.exp(-1j * np.outer(th, k))
    exact = np.where(k % 2 == 0, half.real @ E, 1j * (half.imag @ E))
    assert np.abs(exact - want).max() <= 1e-12 * np.abs(want).max()


def test_bf16x3_form_within_its_bound(ffb):
    n_theta, k_max = 512, 182
    hi, lo = (t.astype(np.float64) for t in ffb.ringdft_table(n_theta, k_max))
    rng = np.random.default_rng(2)
    u = rng.standard_normal((8, n_theta // 2)) * np.exp(rng.uniform(-3, 3, (8, 1)))
    uh = bf16(u)
    ul = bf16(u - uh)
    exact = u @ (hi[0] + lo[0]).T
    x3 = uh @ hi[0].T + uh @ lo[0].T + ul @ hi[0].T
    assert np.linalg.norm(x3 - exact) <= 2e-5 * np.linalg.norm(exact)


def test_unsupported_sizes_rejected(ffb):
    with pytest.raises(ffb.FFBError):
        ffb.ringdft_table(511, 100)       # odd ring length
    with pytest.raises(ffb.FFBError):
        ffb.ringdft_table(1024, 200)      # k_max beyond the 192-column tables
