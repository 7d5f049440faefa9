"""The fused kernel's cluster mode (launch configurations 9-16): a cluster
of 2, 3, 4, 6, 8, 9, 12 or 16 CTAs per candidate, each CTA on its share of the sample
grids, the back-projections summed across the cluster every iteration.
Checked against the FP64 oracle (images 1e-4, scores 1e-6 relative, as
every MLEM path), with more candidates than clusters (a cluster then runs
several candidates one after the other) and K = 0."""
import numpy as np
import pytest
import torch

import oracle
from paper_2109_11920_gb300 import Geom
from paper_2109_11920_gb300 import api as boac
from problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu

SHAPES = [(64, 0.4, 60), (96, 25.6 / 96, 90), (128, 0.2, 120)]


def run_split(p, dev, K, config, B=None):
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu if B is None else p.mu[:B], dtype=torch.float32, device=dev)
    Bn = mu.shape[0]
    S = torch.tensor(p.S, dtype=torch.float32, device=dev)
    batch = boac.RaggedBatch([g], [0] * Bn, [K] * Bn, list(mu), [S] * Bn, device=dev)
    L = boac.boac_mlem_ragged(batch, config=[config])
    return batch.F_pool.view(Bn, p.n, p.n).cpu().numpy(), L.cpu().numpy()


@pytest.mark.parametrize("config", [9, 10, 11, 12, 13, 14, 15, 16])
@pytest.mark.parametrize("shape", SHAPES)
def test_cluster_split_against_oracle(cuda, shape, config):
    p = make_problem(*shape, counts=2e5, B=3, seed=17)
    g = Geom.make(p.n, p.dx, p.V)
    if not boac.config_valid(g, config):
        pytest.skip("view count below one grid per rank")
    K = 6
    F, L = run_split(p, cuda, K, config)
    Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu, p.S, K)
    for b in range(3):
        assert rel_l2(F[b], Fo[b]) < 1e-4, b
        assert abs(L[b] - Lo[b]) < 1e-6 * abs(Lo[b]), b


def test_cluster_split_more_candidates_than_clusters(cuda):
    """40 candidates on clusters of 8 CTAs (configuration 13; at most
    152 / 8 = 19 resident):
    each cluster runs several candidates; sampled ones against the oracle,
    the rest against the one-CTA kernel."""
    p = make_problem(64, 0.4, 60, 2e5, B=40, seed=19)
    K = 3
    F, L = run_split(p, cuda, K, 13)
    F1, L1 = run_split(p, cuda, K, 4)  # one CTA of 8n threads per candidate
    assert rel_l2(F, F1) < 1e-5
    np.testing.assert_allclose(L, L1, rtol=1e-6)
    for b in (0, 17, 39):
        Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu[b][None], p.S, K)
        assert rel_l2(F[b], Fo[0]) < 1e-4, b
        assert abs(L[b] - Lo[0]) < 1e-6 * abs(Lo[0]), b


def test_cluster_split_zero_iterations(cuda):
    p = make_problem(128, 0.2, 120, 2e5, B=2, seed=23)
    F, L = run_split(p, cuda, 0, 13)
    np.testing.assert_array_equal(F, np.ones_like(F))  # F^0 unchanged
    for b in range(2):
        Lo = oracle.score(p.geom, p.mu[b], p.S, np.ones((p.n, p.n)))
        assert abs(L[b] - Lo) < 1e-6 * abs(Lo)


def test_default_path_for_small_batches_is_the_cluster_mode(cuda):
    """boac_mlem's own choice for 1, 5 and 16 candidates at 128 x 128 (the
    cluster mode) against the oracle."""
    p = make_problem(128, 0.2, 120, 2e5, B=16, seed=31)
    g = Geom.make(p.n, p.dx, p.V)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    K = 5
    for B in (1, 5, 16):
        mu = torch.tensor(p.mu[:B], dtype=torch.float32, device=cuda)
        F, L = boac.boac_mlem(g, mu, S, torch.ones(B, p.n, p.n, device=cuda), K)
        F, L = F.cpu().numpy(), L.cpu().numpy()
        for b in sorted({0, B - 1}):
            Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu[b][None], p.S, K)
            assert rel_l2(F[b], Fo[0]) < 1e-4, (B, b)
            assert abs(L[b] - Lo[0]) < 1e-6 * abs(Lo[0]), (B, b)
