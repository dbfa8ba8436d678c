"""Seeded synthetic inputs shared by the tests, the benchmark and the serving loop.

This module holds none of the method's arithmetic (no Philox, no bonds, no
labeling): it only makes the workloads' raw inputs on the host with numpy /
scipy, so the GPU path and the oracle can be handed identical arrays.

* :func:`blurred_noise_image` -- the image-segmentation workload: white
  Gaussian noise, Gaussian blur (sigma = 3, truncated at 4 sigma, reflecting
  edges), quantised to 8 levels with equal-probability bins (thresholds at
  the standard-normal quantiles k/8 of the standardised field).
* :func:`batched_replicas` -- the batched workload: 512 replicas, L
  log-uniform in [64, 2048] rounded to a multiple of 32, beta spread linearly
  over [0.9, 1.1] beta_c, seed = replica id.
* :func:`poisson_arrivals` -- request arrival times of a Poisson stream.
"""
import math

import numpy as np


def blurred_noise_image(H, W, seed, levels=8, sigma=3.0):
    from scipy.ndimage import gaussian_filter
    from scipy.stats import norm
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((H, W), dtype=np.float32)
    blur = gaussian_filter(noise, sigma=sigma, mode="reflect", truncate=4.0)
    z = (blur - blur.mean()) / max(float(blur.std()), 1e-12)
    cuts = norm.ppf(np.arange(1, levels) / levels).astype(np.float32)
    return np.searchsorted(cuts, z).astype(np.uint8)


def batched_replicas(n=512, seed=2024, L_min=64, L_max=2048, beta_c=0.5 * math.log(1 + math.sqrt(2))):
    """List of dicts (L, beta, seed) for n independent Ising replicas."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(L_min), math.log(L_max), size=n)
    Ls = np.clip(32 * np.round(np.exp(u) / 32), L_min, L_max).astype(int)
    betas = beta_c * (0.9 + 0.2 * np.arange(n) / max(n - 1, 1))
    return [{"L": int(L), "beta": float(b), "seed": int(r)} for r, (L, b) in enumerate(zip(Ls, betas))]


def poisson_arrivals(rate, n, seed=0):
    """n arrival times (seconds) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def random_mask(H, W, p, seed):
    """Packed bond mask with every bond bit open independently with probability p
    (numpy generator; for label tests with densities other than 1/2)."""
    rng = np.random.default_rng(seed)
    N = H * W
    east = rng.random(N) < p
    north = rng.random(N) < p
    i = np.arange(N)
    bits = (east.astype(np.uint8) | (north.astype(np.uint8) << 1)) << (2 * (i & 3)).astype(np.uint8)
    m = np.zeros((N + 3) // 4, dtype=np.uint8)
    np.bitwise_or.at(m, i >> 2, bits)
    return m
