"""Seeded synthetic training windows shaped like a Viola-Jones face set.

This module only draws input data: uint8 windows and 0/1 labels.  It holds
none of the boosting arithmetic and is the one module that both the CUDA path
(tests, bench) and the CPU oracle's tests take their inputs from.

The paper trains on 24x24 face / non-face windows (Sec. 2.2: 4916 faces and
7960 non-faces; the introduction quotes about 5000 and 10,000).  That set is not
available here, so windows are drawn from two generators:

* positive ("face"): a fixed template -- background 128, a dark band (64) over
  a bright band (192) across the middle rows -- scaled by a random contrast
  c ~ U(0.7, 1.3), shifted by a random offset o ~ U(-20, 20), plus white
  Gaussian noise of standard deviation ``POS_NOISE_STD`` smoothed by a
  Gaussian of sigma 1 (radius 3 sigma, reflecting boundary);
* negative: uniform noise U(0, 255) smoothed by a Gaussian whose sigma is
  drawn from U(0.5, 3).

Pixels are rounded and clipped to [0, 255].  Sample order is shuffled so that
labels are interleaved.  RNG: numpy PCG64.

``POS_NOISE_STD`` is the one free parameter of the recipe.  With a small noise
amplitude (25, 100 or 300) one Haar feature separates the two classes perfectly
(round-1 error 0), which ends boosting after one round.  At 800 the smoothed
noise (about 226 grey levels before clipping) keeps the classes overlapping for
every single feature: the round-1 error is about 0.12 on the 10x10 workload and
about 0.047 on the 24x24 / 15k workload.
"""

from __future__ import annotations

import numpy as np
from scipy.ndimage import gaussian_filter

# Standard deviation of the white noise added to positives before smoothing.
POS_NOISE_STD = 800.0


def _template(h: int, w: int) -> np.ndarray:
    t = np.full((h, w), 128.0)
    t[h // 4: h // 2, :] = 64.0
    t[h // 2: (3 * h) // 4, :] = 192.0
    return t


def make_windows(n_pos: int, n_neg: int, h: int = 24, w: int = 24, seed: int = 1306,
                 pos_noise_std: float | None = None, shuffle: bool = True):
    """Return (pixels uint8 [N, h, w], labels uint8 [N]) with N = n_pos + n_neg."""
    if pos_noise_std is None:
        pos_noise_std = POS_NOISE_STD
    rng = np.random.Generator(np.random.PCG64(seed))
    n = n_pos + n_neg
    px = np.empty((n, h, w), dtype=np.uint8)
    tmpl = _template(h, w)
    if n_pos:
        c = rng.uniform(0.7, 1.3, size=n_pos)
        o = rng.uniform(-20.0, 20.0, size=n_pos)
        g = rng.normal(0.0, pos_noise_std, size=(n_pos, h, w))
        g = gaussian_filter(g, sigma=(0.0, 1.0, 1.0), mode="reflect", truncate=3.0)
        img = 128.0 + c[:, None, None] * (tmpl[None] - 128.0) + o[:, None, None] + g
        px[:n_pos] = np.clip(np.rint(img), 0, 255).astype(np.uint8)
    for k in range(n_neg):
        sig = rng.uniform(0.5, 3.0)
        u = rng.uniform(0.0, 255.0, size=(h, w))
        img = gaussian_filter(u, sigma=sig, mode="reflect", truncate=3.0)
        px[n_pos + k] = np.clip(np.rint(img), 0, 255).astype(np.uint8)
    y = np.concatenate([np.ones(n_pos, np.uint8), np.zeros(n_neg, np.uint8)])
    if shuffle:
        perm = rng.permutation(n)
        px, y = px[perm], y[perm]
    return np.ascontiguousarray(px), np.ascontiguousarray(y)


# Named workloads.  Seeds are 1306 + workload number.
WORKLOADS = {
    "tiny_10x10": dict(n_pos=200, n_neg=400, h=10, w=10, seed=1306, rounds=10),
    "paper_24x24_15k": dict(n_pos=5000, n_neg=10000, h=24, w=24, seed=1307, rounds=200),
    "precision_24x24_15k": dict(n_pos=5000, n_neg=10000, h=24, w=24, seed=1308, rounds=300),
    # the search kernel's profiling case: the same 15k windows at 16x16, so
    # the sorted table (32,384 features, 0.97 GB) is larger than L2 but small
    "search_16x16_15k": dict(n_pos=5000, n_neg=10000, h=16, w=16, seed=1309, rounds=20),
}


def workload(name: str):
    """Pixels, labels and round count of a named workload."""
    cfg = dict(WORKLOADS[name])
    rounds = cfg.pop("rounds")
    px, y = make_windows(**cfg)
    return px, y, rounds


def log_uniform_weights(n: int, seed: int, lo: float = 1e-12, hi: float = 1.0) -> np.ndarray:
    """Weights drawn log-uniformly in [lo, hi] (FP32), for the precision workload."""
    rng = np.random.Generator(np.random.PCG64(seed))
    e = rng.uniform(np.log(lo), np.log(hi), size=n)
    return np.exp(e).astype(np.float32)


def batch_jobs(n_jobs: int, seed: int, n_lo: int = 2000, n_hi: int = 20000,
               pos_lo: float = 0.2, pos_hi: float = 0.5, h: int = 24, w: int = 24):
    """Job shapes of the batching workload: list of (n_pos, n_neg, h, w, seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    jobs = []
    for k in range(n_jobs):
        n = int(rng.integers(n_lo, n_hi + 1))
        frac = rng.uniform(pos_lo, pos_hi)
        n_pos = max(1, min(n - 1, int(round(frac * n))))
        jobs.append((n_pos, n - n_pos, h, w, seed * 1000 + k))
    return jobs
