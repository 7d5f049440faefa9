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


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
