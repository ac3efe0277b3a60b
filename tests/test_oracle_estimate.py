"""Pins of the oracle's estimation of R and c (Sec. V) against closed forms,
special cases and invariances -- none of them re-types the oracle's own
formulas."""
import math

import numpy as np

from oracle import estimate as est
from oracle import fb


def _plan(L):
    return fb.make_plan(L, 0.5, L / 2)


def test_delta_pair_closed_form():
    """I_1 = delta_0, I_2 = -delta_0: mean 0, variance 1 at the centre pixel
    only, and |F(delta)| = 1 at every frequency, so the normalised power is
    1/L^2 on every radius."""
    L = 16
    x = np.zeros((2, L, L))
    x[0, L // 2, L // 2] = 1.0
    x[1, L // 2, L // 2] = -1.0
    m, v = est.mean_and_variance(x)
    assert np.all(m == 0.0)
    V = est.radial_variance(v)
    assert V[0] == 1.0 and np.all(V[1:] == 0.0)
    assert est.corner_noise(v) == 0.0
    P = est.radial_power(_plan(L), x, m)
    assert np.max(np.abs(P - 1.0 / L ** 2)) < 1e-15


def test_gaussian_blob_power_closed_form():
    """+-G with G(i) = exp(-|i|^2 / (2 s^2)): for s = 2 the sampled sum equals
    the continuous transform 2 pi s^2 exp(-2 pi^2 s^2 xi^2) up to aliasing of
    order exp(-2 pi^2 s^2) ~ 1e-34 (Poisson summation), so P(xi) =
    (2 pi s^2)^2 exp(-4 pi^2 s^2 xi^2) / L^2 at every polar radius."""
    L, s = 32, 2.0
    r2 = est.pixel_radius(L) ** 2
    G = np.exp(-r2 / (2 * s * s))
    x = np.stack([G, -G])
    plan = _plan(L)
    P = est.radial_power(plan, x, np.zeros((L, L)))
    ref = (2 * math.pi * s * s) ** 2 * np.exp(-4 * math.pi ** 2 * s * s * plan.xi ** 2) / L ** 2
    assert np.max(np.abs(P - ref)) <= 1e-12 * ref.max()


def test_white_noise_is_flat_at_sigma2():
    """Pure noise of variance 4: the radial variance, the corner estimate and
    the radial power all sit at 4 within their sampling error (no spurious
    structure)."""
    L, n, s2 = 32, 400, 4.0
    rng = np.random.default_rng(3)
    x = math.sqrt(s2) * rng.standard_normal((n, L, L))
    plan = _plan(L)
    R, c, sig, V, P = est.estimate(plan, x)
    assert abs(sig / s2 - 1.0) < 0.02
    assert np.max(np.abs(V[4:] / s2 - 1.0)) < 0.06
    assert np.max(np.abs(P / s2 - 1.0)) < 0.05


def test_ring_support_is_found_exactly():
    """Images +-ring(r0) (the pixels with round(|i|) = r0), no noise: all the
    variance sits on ring r0, so the cumulative excess jumps there and R = r0."""
    L, r0 = 32, 11
    ring = (np.rint(est.pixel_radius(L)) == r0).astype(float)
    rng = np.random.default_rng(0)
    a = rng.choice([-1.0, 1.0], size=64)
    a -= a.mean()
    x = a[:, None, None] * ring[None]
    R, c, sig, V, P = est.estimate(_plan(L), x, sigma2=0.0)
    assert R == r0
    assert np.argmax(V) == r0 and np.count_nonzero(V > 1e-12) == 1


def test_scale_and_offset_invariance():
    """R and c do not change when the stack is scaled (noise level scaled
    with it) or shifted by a constant image (removed by the mean)."""
    from paper_1412_0781_gb300 import data
    spec = data.TINY
    imgs, _, _ = data.blob_stack(spec, n=60)
    x = imgs.double().numpy()
    plan = _plan(spec.L)
    base = est.estimate(plan, x, sigma2=1.0)
    scaled = est.estimate(plan, 3.0 * x, sigma2=9.0)
    shifted = est.estimate(plan, x + 5.0 * np.ones((spec.L, spec.L)), sigma2=1.0)
    assert base[0] == scaled[0] == shifted[0]
    assert base[1] == scaled[1] == shifted[1]
    assert np.allclose(scaled[3], 9 * base[3], rtol=1e-12, atol=1e-12)


def test_half_plane_angles_suffice_for_real_images():
    """|F(-xi)| = |F(xi)| for real images: averaging the power over theta in
    [0, pi) equals the average over the whole circle (the GPU path uses the
    half ring)."""
    L = 32
    plan = _plan(L)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, L, L))
    F = fb.ndft_polar(plan, x)
    full = (np.abs(F) ** 2).mean(axis=(0, 2))
    half = (np.abs(F[:, :, : plan.n_theta // 2]) ** 2).mean(axis=(0, 2))
    assert np.max(np.abs(full - half) / full) < 1e-12


def test_gaussian_stack_cutoffs_closed_form():
    """a_n G(i) with G a centred Gaussian of s = 2 px and zero-mean random
    amplitudes, no noise: the variance map is var(a) G^2 = var(a)
    exp(-|i|^2 / s^2), whose integral int_0^r exp(-r^2/s^2) r dr reaches
    99.9 % at r = s sqrt(ln 1000) = 5.26; the power is proportional to
    exp(-4 pi^2 s^2 xi^2), whose xi dxi integral reaches 99.9 % at
    xi = sqrt(ln 1000 / (4 pi^2 s^2)) = 0.209.  The discrete estimates land
    within one ring and one Gauss-Legendre node of these."""
    L, s = 32, 2.0
    G = np.exp(-est.pixel_radius(L) ** 2 / (2 * s * s))
    rng = np.random.default_rng(4)
    a = rng.standard_normal(50)
    x = a[:, None, None] * G[None]
    plan = _plan(L)
    R, c, sig, V, P = est.estimate(plan, x, sigma2=0.0)
    r_star = s * math.sqrt(math.log(1000.0))
    xi_star = math.sqrt(math.log(1000.0) / (4 * math.pi ** 2 * s * s))
    assert abs(R - r_star) <= 1.0
    j = int(np.searchsorted(plan.xi, xi_star))
    assert plan.xi[max(j - 1, 0)] <= c <= plan.xi[min(j + 1, plan.n_xi - 1)]


def test_blob_stack_support():
    """The TINY stack (blobs within 0.6 R of the centre, zeroed for r >= R =
    16, noise everywhere): R lands inside the support and the corner noise
    estimate matches the generator's variance."""
    from paper_1412_0781_gb300 import data
    spec = data.TINY
    imgs, _, s2 = data.blob_stack(spec)
    R, c, sig, V, P = est.estimate(_plan(spec.L), imgs.double().numpy())
    assert 5 <= R <= 16
    assert abs(sig / s2 - 1.0) < 0.1
