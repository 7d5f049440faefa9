"""Seeded synthetic inputs for the BOAC hot path.

This module holds random draws and phantom painting only -- none of the
method's arithmetic (no Legendre boundary, no projector, no MLEM).  It is the
one module that both the CUDA path's tests/benchmark and the CPU oracle's
tests read their inputs from.

The paper's phantoms (Fig. 3) are not published, so these stand in for them:
a brain of uniform activity 1.0 with four seeded ellipses at 4.0 (clipped to
the brain), 0 in the cranium and outside; the caller passes the brain mask it
got from its own rasteriser.  Measured sinograms are Poisson draws of an
expected sinogram (again computed by the caller) scaled to a total count.
Streams are spawned from one ``SeedSequence`` per workload in a fixed order:
[phantom, noise, candidates].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Legendre coefficients of the true head boundary (cm) and tissue values
# (mu_b, mu_c in cm^-1, cranium thickness dR in cm).
C_TRUE = (8.0, 0.3, -0.6, 0.2, -0.1, 0.05)
TISSUE = (0.15, 0.25, 0.6)


@dataclass(frozen=True)
class Workload:
    name: str
    n: int                 # image side (pixels); bins per view = n
    dx: float              # pixel size (cm); bin pitch = dx
    V: int                 # views over 360 deg
    K: int                 # MLEM iterations
    B: int                 # candidates
    counts: float          # total counts of the measured sinogram
    sigma_rel: float = 0.15
    sigma_abs: float = 0.05
    seed: int = 0
    extra: dict = field(default_factory=dict)


# The five workloads the hot path is exercised on.
SMALL = Workload("mlem64_v60", 64, 0.4, 60, 20, 1, 2e5)
BATCHED = Workload("bo_batch128_v120", 128, 0.2, 120, 50, 256, 1e6)
GRAD = Workload("grad128_v120", 128, 0.2, 120, 10, 64, 1e6, extra={"ckpt_every": 2})
RAGGED_CLASSES = ((64, 0.4, 60), (96, 25.6 / 96, 90), (128, 0.2, 120))
RAGGED = Workload("ragged512", 0, 0.0, 0, 0, 512, 0.0,
                  extra={"classes": RAGGED_CLASSES, "mix": (1, 1, 2), "k_range": (20, 80)})
LARGE = Workload("slices256_v180", 256, 0.1, 180, 100, 32, 5e6, extra={"slices": 64})


def streams(seed: int):
    """Independent generators for [phantom, noise, candidates]."""
    ss = np.random.SeedSequence(seed)
    return [np.random.default_rng(s) for s in ss.spawn(3)]


def ellipses(rng: np.random.Generator, c0: float, count: int = 4):
    """Ellipse parameters: centre uniform in the disk of radius c0/2,
    semi-axes U(0.5, 2) cm, orientation U(0, pi)."""
    out = []
    for _ in range(count):
        rad = 0.5 * c0 * np.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2.0 * np.pi)
        cx, cy = rad * np.cos(ang), rad * np.sin(ang)
        a, b = rng.uniform(0.5, 2.0, size=2)
        th = rng.uniform(0.0, np.pi)
        out.append((cx, cy, a, b, th))
    return out


def paint_activity(n: int, dx: float, brain_mask: np.ndarray, ells,
                   background: float = 1.0, hot: float = 4.0) -> np.ndarray:
    """Activity image: ``background`` on the brain mask, ``hot`` inside the
    ellipses (clipped to the mask), 0 elsewhere.  Pixel (i, j) has centre
    x = (j - c) dx, y = (i - c) dx with c = (n - 1) / 2."""
    c = (n - 1) / 2.0
    x = (np.arange(n) - c) * dx
    X, Y = np.meshgrid(x, x)  # X varies along columns, Y along rows
    img = np.where(brain_mask, background, 0.0)
    for cx, cy, a, b, th in ells:
        xr = (X - cx) * np.cos(th) + (Y - cy) * np.sin(th)
        yr = -(X - cx) * np.sin(th) + (Y - cy) * np.cos(th)
        inside = (xr / a) ** 2 + (yr / b) ** 2 <= 1.0
        img = np.where(inside & brain_mask, hot, img)
    return img


def poisson_sinogram(rng: np.random.Generator, expected: np.ndarray, total: float) -> np.ndarray:
    """Poisson draw of ``expected`` rescaled to ``total`` expected counts."""
    expected = np.asarray(expected, dtype=np.float64)
    lam = expected * (total / expected.sum())
    return rng.poisson(lam).astype(np.float64)


def candidates(rng: np.random.Generator, B: int, c_true=C_TRUE,
               sigma_rel: float = 0.15, sigma_abs: float = 0.05) -> np.ndarray:
    """B coefficient vectors c_k + N(0, sigma_rel |c_k| + sigma_abs)."""
    c = np.asarray(c_true, dtype=np.float64)
    sd = sigma_rel * np.abs(c) + sigma_abs
    return c[None, :] + rng.normal(size=(B, 6)) * sd[None, :]


def tissue_candidates(rng: np.random.Generator, B: int, tissue=TISSUE,
                      spread: float = 0.2) -> np.ndarray:
    """B (mu_b, mu_c, dR) triples, each value times U(1 - spread, 1 + spread)."""
    t = np.asarray(tissue, dtype=np.float64)
    return t[None, :] * rng.uniform(1.0 - spread, 1.0 + spread, (B, 3))


def ragged_schedule(rng: np.random.Generator, B: int = 512, mix=(1, 1, 2), k_range=(20, 80)):
    """Size class per candidate in the given ratio (shuffled) and iteration
    counts uniform on k_range (inclusive)."""
    tot = sum(mix)
    cls = np.concatenate([np.full(B * m // tot, i, dtype=np.int32) for i, m in enumerate(mix)])
    cls = np.concatenate([cls, np.full(B - cls.size, len(mix) - 1, dtype=np.int32)])
    rng.shuffle(cls)
    K = rng.integers(k_range[0], k_range[1] + 1, size=B).astype(np.int32)
    return cls, K


def slice_coefficients(rng: np.random.Generator, n_slices: int, base=C_TRUE) -> np.ndarray:
    """Per-slice true head coefficients for the large-slice workload:
    c_0 ~ U(6, 9) cm, c_1..c_5 = base_k x U(0.5, 1.5)."""
    c = np.empty((n_slices, 6))
    c[:, 0] = rng.uniform(6.0, 9.0, n_slices)
    c[:, 1:] = np.asarray(base[1:])[None, :] * rng.uniform(0.5, 1.5, (n_slices, 5))
    return c
