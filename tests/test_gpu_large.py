"""256 x 256 images (too large for one SM's shared memory: the fused kernel
keeps their images in a per-CTA region of the workspace), against the FP64
oracle, including the large-slice workload at full size."""
import numpy as np
import pytest
import torch

import oracle
from paper_2109_11920_gb300 import Geom, synth
from paper_2109_11920_gb300 import api as boac
from problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("V", [16, 18])  # four and two views per sample grid
def test_mlem_256_small(cuda, V):
    p = make_problem(256, 0.1, V, 2e5, B=3, seed=21)
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    F = torch.ones(3, 256, 256, device=cuda)
    F, L = boac.boac_mlem(g, mu, S, F, 4)
    Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu, p.S, 4)
    for b in range(3):
        assert rel_l2(F[b].cpu().numpy(), Fo[b]) < 1e-4
        assert abs(float(L[b]) - Lo[b]) < 1e-6 * abs(Lo[b])


def test_large_slice_workload_sampled(cuda):
    """64 slices of 256^2 (0.1 cm, 180 views, 5e6 counts, own head and
    phantom per slice) x 32 candidates, 100 MLEM iterations, one ragged call
    whose candidates point at their slice's sinogram; the last candidate of
    the last slice is checked against the FP64 oracle."""
    wl = synth.LARGE
    n_sl, per = wl.extra["slices"], wl.B
    rng = np.random.default_rng(wl.seed)
    c_sl = synth.slice_coefficients(rng, n_sl)
    probs = [make_problem(wl.n, wl.dx, wl.V, wl.counts, B=per, seed=s, c_true=c_sl[s]) for s in range(n_sl)]
    g = Geom.make(wl.n, probs[0].dx, wl.V)
    mus, Ss, cls, K = [], [], [], []
    for p in probs:
        for b in range(per):
            mus.append(torch.tensor(p.mu[b], dtype=torch.float32))
            Ss.append(torch.tensor(p.S, dtype=torch.float32))  # same slice: same sinogram
            cls.append(0)
            K.append(wl.K)
    batch = boac.RaggedBatch([g], cls, K, mus, Ss, device=cuda)
    L = boac.boac_mlem_ragged(batch).cpu().numpy()
    assert np.all(np.isfinite(L))
    last = len(cls) - 1
    p = probs[-1]
    Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu[per - 1:per], p.S, wl.K)
    assert rel_l2(batch.image(last).cpu().numpy(), Fo[0]) < 1e-4
    assert abs(L[last] - Lo[0]) < 1e-6 * abs(Lo[0])
