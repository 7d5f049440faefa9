"""The cluster kernel for 256 x 256 images (bands of rows over the CTAs of a
thread-block cluster) against the FP64 oracle and the one-CTA kernel: every
cluster size, grids whose base view is turned by a quarter, a batch large
enough that the work split cuts candidates between clusters, and bit-exact
repeats."""
import numpy as np
import pytest
import torch

import oracle
from paper_2109_11920_gb300 import Geom, _lib
from paper_2109_11920_gb300 import api as boac
from problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu


def ragged_one_class(p, g, K, cuda, cands=None):
    idx = range(p.mu.shape[0]) if cands is None else cands
    mus = [torch.tensor(p.mu[b], dtype=torch.float32) for b in idx]
    Ss = [torch.tensor(p.S, dtype=torch.float32) for _ in idx]
    return boac.RaggedBatch([g], [0] * len(mus), [K] * len(mus), mus, Ss, device=cuda)


@pytest.mark.parametrize("cfg", [6, 7, 8])
def test_every_cluster_size_matches_the_oracle(cuda, cfg):
    # 16 views: grids at 0, 22.5, 45 and 67.5 degrees (the last one with a
    # base view turned by a quarter)
    p = make_problem(256, 0.1, 16, 2e5, B=2, seed=41)
    g = Geom.make(p.n, p.dx, p.V)
    K = 3
    batch = ragged_one_class(p, g, K, cuda)
    L = boac.boac_mlem_ragged(batch, config=[cfg]).cpu().numpy()
    Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu, p.S, K)
    for b in range(2):
        assert rel_l2(batch.image(b).cpu().numpy(), Fo[b]) < 1e-4
        assert abs(L[b] - Lo[b]) < 1e-6 * abs(Lo[b])


def test_cluster_kernel_agrees_with_the_one_cta_kernel(cuda):
    p = make_problem(256, 0.1, 24, 2e5, B=2, seed=43)
    g = Geom.make(p.n, p.dx, p.V)
    K = 4
    out = {}
    for cfg in (4, 6, 7, 8):  # one-CTA kernel (1024 threads, four views per grid), clusters
        batch = ragged_one_class(p, g, K, cuda)
        L = boac.boac_mlem_ragged(batch, config=[cfg]).cpu().numpy()
        out[cfg] = (batch.F_pool.cpu().numpy().copy(), L)
    F4, L4 = out[4]
    for cfg in (6, 7, 8):
        F, L = out[cfg]
        assert rel_l2(F, F4) < 1e-5, cfg
        np.testing.assert_allclose(L, L4, rtol=1e-6, atol=0)


def test_default_256_path_views_180(cuda):
    """The large-slice geometry (180 views: base views on both sides of 45
    degrees) on a cluster of 5 CTAs and through boac_mlem's default (for one
    candidate the unfused kernels), against the oracle."""
    p = make_problem(256, 0.1, 180, 5e5, B=1, seed=45)
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    F, L = boac.boac_mlem(g, mu, S, torch.ones(1, 256, 256, device=cuda), 2)
    batch = ragged_one_class(p, g, 2, cuda)
    Lc = boac.boac_mlem_ragged(batch, config=[6]).cpu().numpy()
    Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu, p.S, 2)
    for F_run, L_run in ((F[0].cpu().numpy(), float(L[0])), (batch.image(0).cpu().numpy(), float(Lc[0]))):
        assert rel_l2(F_run, Fo[0]) < 1e-4
        assert abs(L_run - Lo[0]) < 1e-6 * abs(Lo[0])


def test_work_split_over_clusters_and_repeatability(cuda):
    """More candidates than resident clusters with 3 iterations each: the
    even split cuts candidates between clusters (hand-over through F in
    global memory); results equal the oracle on sampled candidates and are
    bit-identical on a second run."""
    B = 61
    p = make_problem(256, 0.1, 8, 1e5, B=B, seed=47)
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    K = 3
    ws = boac.workspace(g, B, _lib.OP_MLEM, cuda)
    F1, L1 = boac.boac_mlem(g, mu, S, torch.ones(B, 256, 256, device=cuda), K, ws=ws)
    assert boac.boac_workspace_status(ws) == 0
    F2, L2 = boac.boac_mlem(g, mu, S, torch.ones(B, 256, 256, device=cuda), K, ws=ws)
    assert torch.equal(F1, F2) and torch.equal(L1, L2)
    picks = [0, 1, 29, 30, B - 1]
    Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu[picks], p.S, K)
    for i, b in enumerate(picks):
        assert rel_l2(F1[b].cpu().numpy(), Fo[i]) < 1e-4, b
        assert abs(float(L1[b]) - Lo[i]) < 1e-6 * abs(Lo[i]), b


def test_zero_iterations_and_lone_candidate(cuda):
    """K = 0: the score of the initial image; one candidate on one cluster
    (and through boac_mlem's default)."""
    p = make_problem(256, 0.1, 8, 1e5, B=1, seed=49)
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    F0 = torch.full((1, 256, 256), 0.5, device=cuda)
    Lo = oracle.loglik(p.S, oracle.project(p.geom, p.mu[0], np.full((256, 256), 0.5)))
    F, L = boac.boac_mlem(g, mu, S, F0.clone(), 0)
    assert torch.equal(F, F0)
    assert abs(float(L[0]) - Lo) < 1e-6 * abs(Lo)
    for cfg in (6, 7, 8):
        batch = boac.RaggedBatch([g], [0], [0], [mu[0]], [S], device=cuda)
        batch.F_pool.fill_(0.5)
        Lc = boac.boac_mlem_ragged(batch, config=[cfg])
        assert torch.equal(batch.image(0), F0[0]), cfg
        assert abs(float(Lc[0]) - Lo) < 1e-6 * abs(Lo), cfg


def test_largest_view_count(cuda):
    """720 views (the library's maximum): 180 sample grids per iteration,
    the largest exponent table per CTA."""
    p = make_problem(256, 0.1, 720, 1e6, B=1, seed=51)
    g = Geom.make(p.n, p.dx, p.V)
    batch = ragged_one_class(p, g, 2, cuda)
    L = boac.boac_mlem_ragged(batch, config=[6]).cpu().numpy()
    Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu, p.S, 2)
    assert rel_l2(batch.image(0).cpu().numpy(), Fo[0]) < 1e-4
    assert abs(float(L[0]) - Lo[0]) < 1e-6 * abs(Lo[0])


@pytest.mark.parametrize("n,dx,V,cfg1", [(128, 0.2, 120, 4), (64, 0.4, 60, 2)])
def test_cluster_kernel_small_images(cuda, n, dx, V, cfg1):
    """128 x 128 and 64 x 64 images on clusters of 2, 4 or 8 CTAs (configs
    6-8) against the oracle and the one-CTA kernel."""
    p = make_problem(n, dx, V, 1e6, B=3, seed=61)
    g = Geom.make(p.n, p.dx, p.V)
    K = 4
    out = {}
    for cfg in (cfg1, 6, 7, 8):
        batch = ragged_one_class(p, g, K, cuda)
        L = boac.boac_mlem_ragged(batch, config=[cfg]).cpu().numpy()
        out[cfg] = (batch.F_pool.cpu().numpy().copy(), L)
    Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu, p.S, K)
    F4, L4 = out[cfg1]
    for cfg in (6, 7, 8):
        F, L = out[cfg]
        assert rel_l2(F, F4) < 1e-5, cfg
        np.testing.assert_allclose(L, L4, rtol=1e-6, atol=0)
        for b in range(3):
            assert rel_l2(F[b * n * n:(b + 1) * n * n], Fo[b].ravel()) < 1e-4, (cfg, b)
            assert abs(L[b] - Lo[b]) < 1e-6 * abs(Lo[b]), (cfg, b)
