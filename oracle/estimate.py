"""FP64 oracle of the estimation of the support radius R and the band limit c
from a stack of noisy images (test infrastructure only; see
``oracle/__init__.py``).

Sec. V (the experiment on the simulated ribosome projections) estimates R and
c before the expansion: subtract the mean image, average the per-pixel
variance over angles (mean radial variance), subtract the noise variance and
accumulate with the Jacobian weight r dr; R is where the cumulative fraction
reaches 99.9 %.  The same is done in the Fourier domain with the angular
average of the mean power spectrum and the weight xi dxi, giving c.

Readings (the paper states the procedure, not its discretisation):
* radial bins are the rounded pixel radius r = round(|i|), r = 0 .. L/2 - 1
  (the rings fully inside the image), pixel grid i = a - L//2;
* the noise variance, when not given, is the mean variance of the pixels with
  |i| >= L/2 (the corners outside the inscribed disk, where the particle has no
  support);
* the power spectrum is sampled on the polar grid of a plan (Gauss-Legendre
  radii xi_j on [0, c_plan], all n_theta angles, direct NDFT) and normalised
  by L^2, so that white noise of variance s^2 gives the level s^2; the xi dxi
  integral is the plan's radial quadrature sum_j (.) xi_j w_j;
* the excess over the noise level is clipped at zero before accumulating, and
  the estimate is the first bin (radius, node) at which the cumulative excess
  reaches the fraction of its total.
"""
import numpy as np

from . import fb


def pixel_radius(L):
    i = np.arange(L) - L // 2
    return np.sqrt(i[:, None] ** 2 + i[None, :] ** 2)


def mean_and_variance(images):
    """mean image and per-pixel variance (1/n normalisation), two passes."""
    x = np.asarray(images, dtype=np.float64)
    m = x.mean(axis=0)
    v = ((x - m) ** 2).mean(axis=0)
    return m, v


def radial_variance(v):
    """mean of the variance map over each ring round(|i|) = r, r < L/2."""
    L = v.shape[0]
    rb = np.rint(pixel_radius(L)).astype(int)
    out = np.zeros(L // 2)
    for r in range(L // 2):
        out[r] = v[rb == r].mean()
    return out


def corner_noise(v):
    """mean variance of the pixels with |i| >= L/2."""
    L = v.shape[0]
    return float(v[pixel_radius(L) >= L / 2].mean())


def radial_power(plan, images, mean_image):
    """P(xi_j) = (1 / (n n_theta L^2)) sum_n sum_l |F(I_n - mean)(xi_j, theta_l)|^2."""
    x = np.asarray(images, dtype=np.float64) - mean_image[None]
    F = fb.ndft_polar(plan, x)                         # (n, n_xi, n_theta)
    return (np.abs(F) ** 2).mean(axis=(0, 2)) / plan.L ** 2


def cumulative_cut(values, weights, level, frac):
    """first index at which sum_{<= index} max(values - level, 0) weights
    reaches frac of the total (-1 when the total is zero)."""
    ex = np.maximum(np.asarray(values) - level, 0.0) * np.asarray(weights)
    cum = np.cumsum(ex)
    if cum[-1] <= 0.0:
        return -1
    return int(np.argmax(cum >= frac * cum[-1]))


def estimate(plan, images, frac=0.999, sigma2=None):
    """(R, c, sigma2, radial variance, radial power) of a stack; plan fixes
    L and the polar grid of the power spectrum (c = 1/2, R = L/2 covers the
    whole band)."""
    m, v = mean_and_variance(images)
    V = radial_variance(v)
    s2 = corner_noise(v) if sigma2 is None else float(sigma2)
    P = radial_power(plan, images, m)
    r = np.arange(plan.L // 2, dtype=np.float64)
    iR = cumulative_cut(V, r, s2, frac)
    ic = cumulative_cut(P, plan.xi * plan.w, s2, frac)
    R = float(iR) if iR >= 0 else 0.0
    c = float(plan.xi[ic]) if ic >= 0 else 0.0
    return R, c, s2, V, P
