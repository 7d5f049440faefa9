"""Seeded test problems built on the CPU with the oracle and the shared
synthetic-input module (never with the CUDA path), in float32-representable
values so that the CUDA path and the oracle see identical inputs."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import oracle
from paper_2109_11920_gb300 import synth

F32 = np.float32


def f32(x) -> float:
    return float(F32(x))


@dataclass
class Problem:
    n: int
    dx: float          # float32-rounded pixel size
    V: int
    tissue: tuple      # float32-rounded (mu_b, mu_c, dR)
    mu_true: np.ndarray
    F_true: np.ndarray
    S: np.ndarray      # measured sinogram [V, n] (integer counts)
    coefs: np.ndarray  # candidate coefficients [B, 6], float32 values
    mu: np.ndarray     # candidate attenuation maps [B, n, n] (oracle, CENTER)

    @property
    def geom(self) -> oracle.Geometry:
        return oracle.Geometry(self.n, self.dx, self.V)


def make_problem(n: int, dx: float, V: int, counts: float, B: int, seed: int = 0,
                 mode: int = oracle.CENTER, c_true=synth.C_TRUE) -> Problem:
    dx = f32(dx)
    tissue = tuple(f32(t) for t in synth.TISSUE)
    mu_b, mu_c, dR = tissue
    ph, noise, cand = synth.streams(seed)
    c_true = np.array(c_true, dtype=F32).astype(np.float64)
    g = oracle.Geometry(n, dx, V)
    mu_true = oracle.rasterize(n, dx, mu_b, mu_c, dR, c_true, oracle.CENTER)
    F_true = synth.paint_activity(n, dx, mu_true == mu_b, synth.ellipses(ph, c_true[0]))
    S = synth.poisson_sinogram(noise, oracle.project(g, mu_true, F_true), counts)
    coefs = synth.candidates(cand, B, c_true).astype(F32).astype(np.float64)
    mu = np.stack([oracle.rasterize(n, dx, mu_b, mu_c, dR, c, mode) for c in coefs])
    return Problem(n, dx, V, tissue, mu_true, F_true, S, coefs, mu)


def center_tie_mask(n: int, dx: float, coef, dR: float, tol: float = 1e-9) -> np.ndarray:
    """Pixels whose centre lies within ``tol`` cm of a class boundary of Eq. 4
    (r = R(theta) or r = R(theta) + dR, R clamped at 0), computed here in
    float64 with numpy's Legendre series -- independently of the oracle and
    of the CUDA path.  Only at these pixels may two correct float64
    evaluations of R (different polynomial recursions) pick different
    classes."""
    c = (n - 1) / 2.0
    jj, ii = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64))
    x, y = (jj - c) * dx, (ii - c) * dx
    r = np.hypot(x, y)
    z = np.where(r > 0, x / np.where(r > 0, r, 1.0), 1.0)
    R = np.maximum(np.polynomial.legendre.legval(z, np.asarray(coef, dtype=np.float64)), 0.0)
    return (np.abs(r - R) < tol) | (np.abs(r - (R + max(dR, 0.0))) < tol)


def assert_center_classes(mu, ref, n, dx, coef, dR, tol=1e-9):
    """CENTER-mode rasterisation (Eq. 4) is a class decision: the CUDA map
    must equal the oracle's bit for bit at every pixel that is not a tie
    (``center_tie_mask``)."""
    mu = np.asarray(mu)
    ref32 = np.asarray(ref).astype(F32)
    differ = mu != ref32
    ties = center_tie_mask(n, dx, coef, dR, tol)
    bad = differ & ~ties
    assert not bad.any(), (f"{int(bad.sum())} pixels differ away from a boundary, first at "
                           f"{np.argwhere(bad)[:3].tolist()}")
    return int(differ.sum()), int(ties.sum())


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
