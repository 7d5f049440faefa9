"""The batched evaluation captured in a CUDA graph (BatchedEvaluator) gives
the same scores and images as direct calls, replay after replay."""
import numpy as np
import pytest
import torch

from paper_2109_11920_gb300 import Geom, Tissue, synth
from paper_2109_11920_gb300 import api as boac
from problems import make_problem

pytestmark = pytest.mark.gpu


def test_batched_evaluator_replays_match_direct_calls(cuda):
    p = make_problem(128, 0.2, 120, 1e6, B=24, seed=9)
    g, t = Geom.make(p.n, p.dx, p.V), Tissue(*p.tissue)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    ev = boac.BatchedEvaluator(g, t, S, B=24, K=6)
    rng = np.random.default_rng(0)
    for rep in range(3):
        c = torch.tensor(synth.candidates(rng, 24).astype(np.float32), device=cuda)
        L = ev.evaluate(c).clone()
        F = ev.F.clone()
        mu = boac.boac_rasterize_mu(g, t, c)
        Fd = torch.ones(24, p.n, p.n, device=cuda)
        Fd, Ld = boac.boac_mlem(g, mu, S, Fd, 6)
        torch.testing.assert_close(L, Ld, rtol=0, atol=0)
        torch.testing.assert_close(F, Fd, rtol=0, atol=0)


def test_batched_evaluator_with_the_cluster_kernel(cuda):
    """256 x 256 images run the cluster kernel (a record kernel, a memset and
    a cluster launch per call); captured in a graph they replay to the same
    bits as direct calls."""
    p = make_problem(256, 0.1, 16, 2e5, B=6, seed=11)
    g, t = Geom.make(p.n, p.dx, p.V), Tissue(*p.tissue)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    ev = boac.BatchedEvaluator(g, t, S, B=6, K=3)
    rng = np.random.default_rng(1)
    for rep in range(2):
        c = torch.tensor(synth.candidates(rng, 6).astype(np.float32), device=cuda)
        L = ev.evaluate(c).clone()
        F = ev.F.clone()
        mu = boac.boac_rasterize_mu(g, t, c)
        Fd, Ld = boac.boac_mlem(g, mu, S, torch.ones(6, p.n, p.n, device=cuda), 3)
        torch.testing.assert_close(L, Ld, rtol=0, atol=0)
        torch.testing.assert_close(F, Fd, rtol=0, atol=0)
