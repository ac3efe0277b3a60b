"""Seeded synthetic inputs: Gaussian-blob images plus white noise.

This module holds no arithmetic of the method itself: it only draws the test
and benchmark images, and both the CUDA path and the FP64 oracle consume
exactly the float32 arrays it returns.

Recipe (one stack):
* ``n_blobs`` isotropic Gaussians per image, A exp(-|x - x0|^2 / (2 s^2)),
  centres uniform in area inside the disk of radius 0.6 R (r = 0.6 R sqrt(u)),
  widths s uniform in ``width`` (pixels), amplitudes A ~ N(1, 0.3^2);
* the clean image is set to zero wherever r >= R (pixel radius measured from
  the grid centre i = 0, pixel index i = -ceil((L-1)/2) .. floor((L-1)/2),
  first array axis = i1 = x, second = i2 = y);
* white Gaussian noise of variance sigma^2 = P_s / SNR on all L^2 pixels, with
  P_s the mean of clean^2 over all n L^2 pixels of the stack.

Random numbers come from one ``torch.Generator`` seeded with ``seed``; blob
parameters are drawn for the whole stack first, noise chunk by chunk in image
order, so a given (seed, chunk) reproduces the same stack on the same device.
"""
from dataclasses import dataclass
import math

import torch


@dataclass(frozen=True)
class StackSpec:
    n: int
    L: int
    R: float
    n_blobs: int
    width: tuple
    snr: float
    seed: int
    c: float = 0.5


# Workload recipes (seed 20141203 + recipe index).
TINY = StackSpec(n=200, L=32, R=16.0, n_blobs=6, width=(1.5, 4.0), snr=1 / 5, seed=20141203)
FP32_L128 = StackSpec(n=20000, L=128, R=64.0, n_blobs=12, width=(2.0, 8.0), snr=1 / 20, seed=20141204)
PRECISION_L128 = StackSpec(n=100000, L=128, R=64.0, n_blobs=12, width=(2.0, 8.0), snr=1 / 10, seed=20141205)
DIFF_L256 = StackSpec(n=4096, L=256, R=128.0, n_blobs=12, width=(4.0, 16.0), snr=1 / 10, seed=20141207)


def batching_stacks(S=48, n_range=(500, 20000), sizes=(64, 96, 128, 180, 256), seed=20141206):
    """The batching workload: S independent stacks, stack s drawn from a
    numpy generator seeded with ``seed``: L uniform in ``sizes``, R = L/2,
    c = 1/2, n uniform in ``n_range`` (inclusive), SNR uniform in [1/50, 1/5];
    12 blobs of widths [2, 8] L/128 px; the stack's own images use seed
    ``seed + 1000 s``.  Returns a list of StackSpec."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for s in range(S):
        L = int(rng.choice(sizes))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        snr = float(rng.uniform(1 / 50, 1 / 5))
        out.append(StackSpec(n, L, L / 2, 12, (2.0 * L / 128, 8.0 * L / 128), snr, seed + 1000 * s))
    return out


def pixel_index(L, device="cpu", dtype=torch.float64):
    return torch.arange(L, device=device, dtype=dtype) - (L // 2)


def blob_stack(spec, n=None, device="cpu", chunk=2048):
    """Return (images float32 (n, L, L), clean float32 (n, L, L), sigma2 float).

    ``chunk`` fixes how the noise is drawn (part of the seeded recipe); the
    blob rendering is split independently so that its float64 temporaries
    stay near 256 MB."""
    n = spec.n if n is None else n
    L, R = spec.L, float(spec.R)
    g = torch.Generator(device=device)
    g.manual_seed(spec.seed)
    f64 = torch.float64
    u = torch.rand((n, spec.n_blobs), generator=g, device=device, dtype=f64)
    v = torch.rand((n, spec.n_blobs), generator=g, device=device, dtype=f64)
    rad = 0.6 * R * torch.sqrt(u)
    ang = 2.0 * math.pi * v
    x0 = rad * torch.cos(ang)
    y0 = rad * torch.sin(ang)
    lo, hi = spec.width
    s = lo + (hi - lo) * torch.rand((n, spec.n_blobs), generator=g, device=device, dtype=f64)
    amp = 1.0 + 0.3 * torch.randn((n, spec.n_blobs), generator=g, device=device, dtype=f64)

    idx = pixel_index(L, device)
    X1 = idx[:, None].expand(L, L)
    X2 = idx[None, :].expand(L, L)
    inside = (X1 * X1 + X2 * X2) < R * R
    clean = torch.empty((n, L, L), device=device, dtype=torch.float32)
    power = torch.zeros((), device=device, dtype=f64)
    rchunk = max(1, (1 << 25) // (spec.n_blobs * L * L))
    for s0 in range(0, n, rchunk):
        s1 = min(n, s0 + rchunk)
        dx = X1[None, None] - x0[s0:s1, :, None, None]
        dy = X2[None, None] - y0[s0:s1, :, None, None]
        ss = s[s0:s1, :, None, None]
        img = (amp[s0:s1, :, None, None] * torch.exp(-(dx * dx + dy * dy) / (2.0 * ss * ss))).sum(1)
        img = img * inside
        power += (img * img).sum()
        clean[s0:s1] = img.to(torch.float32)
    p_s = float(power) / (n * L * L)
    sigma2 = p_s / spec.snr
    sigma = math.sqrt(sigma2)
    images = torch.empty_like(clean)
    for s0 in range(0, n, chunk):
        s1 = min(n, s0 + chunk)
        noise = torch.randn((s1 - s0, L, L), generator=g, device=device, dtype=torch.float32)
        images[s0:s1] = clean[s0:s1] + sigma * noise
    return images, clean, sigma2


def white_noise(n, L, seed, sigma=1.0, device="cpu"):
    """n images of i.i.d. N(0, sigma^2) pixels, float32."""
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return sigma * torch.randn((n, L, L), generator=g, device=device, dtype=torch.float32)


def support_mask(L, R, device="cpu"):
    """Boolean (L, L) mask of pixels with radius < R."""
    idx = pixel_index(L, device)
    return (idx[:, None] ** 2 + idx[None, :] ** 2) < R * R


def random_coefficients(n, P, p0, seed, device="cpu"):
    """Complex64 (n, P) standard normal coefficients with Im of the first p0
    (the k = 0 block) set to zero."""
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    re = torch.randn((n, P), generator=g, device=device, dtype=torch.float32)
    im = torch.randn((n, P), generator=g, device=device, dtype=torch.float32)
    im[:, :p0] = 0.0
    return torch.complex(re, im)
