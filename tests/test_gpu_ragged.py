"""Ragged batches (mixed image sizes and iteration counts in one call), the
per-class launch-shape autotuner and CUDA-graph capture, on the GPU, against
the uniform entry point and the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2109_11920_gb300 import Geom, synth
from paper_2109_11920_gb300 import api as boac
from paper_2109_11920_gb300 import autotune
from problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu

CLASSES = [(64, 0.4, 60), (96, 25.6 / 96, 90), (128, 0.2, 120)]


def one_candidate(g, mu, S, K, cfg, dev):
    """The same candidate alone through the ragged entry point at launch
    configuration cfg: (F, L)."""
    b1 = boac.RaggedBatch([g], [0], [K], [mu], [S], device=dev)
    L = boac.boac_mlem_ragged(b1, config=[cfg])
    return b1.F_pool.view(g.n, g.n), float(L[0])


def build(dev, cls, K, seed0=100, counts=2e5):
    """One oracle-built problem per candidate (own phantom, noise, coefficients)."""
    probs = [make_problem(*CLASSES[c], counts=counts, B=1, seed=seed0 + i) for i, c in enumerate(cls)]
    geoms = [Geom.make(n, float(np.float32(dx)), V) for n, dx, V in CLASSES]
    mu = [torch.tensor(p.mu[0], dtype=torch.float32, device=dev) for p in probs]
    S = [torch.tensor(p.S, dtype=torch.float32, device=dev) for p in probs]
    batch = boac.RaggedBatch(geoms, cls, K, mu, S, device=dev)
    return batch, probs


def test_ragged_matches_uniform_and_oracle(cuda):
    """Mixed classes and iteration counts in one call: at a fixed launch
    configuration per class every candidate equals its one-candidate call bit
    for bit; it agrees with boac_mlem's own choice for one candidate (the
    unfused kernels) to float rounding, and one per class with the oracle."""
    cls = [0, 1, 2, 2, 1, 0, 2, 0, 1, 2, 2, 0]
    K = [2, 5, 3, 6, 4, 3, 2, 6, 2, 4, 5, 1]
    batch, probs = build(cuda, cls, K)
    config = [2, 5, 4]  # one CTA per candidate: 8n, 4n (two views per grid), 4n threads
    L = boac.boac_mlem_ragged(batch, config=config).cpu().numpy()
    for b, p in enumerate(probs):
        g = batch.classes[cls[b]]
        S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
        mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
        F1, L1 = one_candidate(g, mu[0], S, K[b], config[cls[b]], cuda)
        torch.testing.assert_close(batch.image(b), F1, rtol=0, atol=0)
        assert L[b] == L1
        F, Lu = boac.boac_mlem(g, mu, S, torch.ones(1, p.n, p.n, device=cuda), K[b])
        assert rel_l2(batch.image(b).cpu().numpy(), F[0].cpu().numpy()) < 1e-5
        assert abs(L[b] - float(Lu[0])) < 1e-6 * abs(L[b])
    for b in (0, 1, 3):  # one per class vs the oracle
        p = probs[b]
        Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu, p.S, K[b])
        assert rel_l2(batch.image(b).cpu().numpy(), Fo[0]) < 1e-4
        assert abs(L[b] - Lo[0]) < 1e-6 * abs(Lo[0])


def test_every_launch_configuration_agrees(cuda):
    cls = [0, 1, 2, 0, 1, 2]
    K = [3, 3, 3, 2, 4, 2]
    batch, _ = build(cuda, cls, K, seed0=200)
    L0 = boac.boac_mlem_ragged(batch).clone()
    F0 = batch.F_pool.clone()
    for cfg in range(boac.N_SINGLE_CTA_CONFIGS):
        config = [cfg if (cfg % 2 == 1 or g.n_views % 4 == 0) else cfg + 1 for g in batch.classes]
        assert all(boac.config_valid(g, c) for g, c in zip(batch.classes, config))
        batch.F_pool.fill_(1.0)
        L = boac.boac_mlem_ragged(batch, config=config)
        assert rel_l2(batch.F_pool.cpu().numpy(), F0.cpu().numpy()) < 1e-5, config
        # float32 projections summed in another order: scores agree to ~1e-7
        torch.testing.assert_close(L, L0, rtol=1e-6, atol=0)


def test_ragged_graph_capture_and_autotuner(cuda):
    cls = [2, 0, 1, 2, 0, 2]
    K = [3, 2, 4, 1, 3, 2]
    batch, _ = build(cuda, cls, K, seed0=300)
    config = autotune.tune_ragged(batch, probe_iters=2, repeats=1)
    assert len(config) == 3 and all(0 <= c < boac.N_CONFIGS for c in config)
    batch.prepare(config)
    batch.F_pool.fill_(1.0)
    L_direct = batch.run().clone()
    F_direct = batch.F_pool.clone()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        batch.F_pool.fill_(1.0)
        batch.run()
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(graph):
        batch.F_pool.fill_(1.0)
        batch.run()
    for _ in range(2):
        batch.L.zero_()
        graph.replay()
        torch.cuda.synchronize()
        torch.testing.assert_close(batch.L, L_direct, rtol=0, atol=0)
        torch.testing.assert_close(batch.F_pool, F_direct, rtol=0, atol=0)


def test_ragged_full_size_sampled(cuda):
    """The ragged workload: 512 candidates in a 1:1:2 mix of 64^2/60 views,
    96^2/90 views and 128^2/120 views, K ~ U{20..80}, own phantom and noise
    per candidate, one call; one candidate per class (the largest K of each)
    checked against the FP64 oracle."""
    wl = synth.RAGGED
    _, _, rng = synth.streams(wl.seed)
    cls, K = synth.ragged_schedule(rng, wl.B, wl.extra["mix"], wl.extra["k_range"])
    batch, probs = build(cuda, [int(c) for c in cls], [int(k) for k in K], seed0=1000)
    L = boac.boac_mlem_ragged(batch).cpu().numpy()
    assert np.all(np.isfinite(L))
    for c in range(3):
        members = [b for b in range(wl.B) if cls[b] == c]
        b = max(members, key=lambda i: K[i])
        p = probs[b]
        Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu, p.S, int(K[b]))
        assert rel_l2(batch.image(b).cpu().numpy(), Fo[0]) < 1e-4, (c, b)
        assert abs(L[b] - Lo[0]) < 1e-6 * abs(Lo[0]), (c, b)


def test_ragged_mixes_one_cta_and_cluster_classes(cuda):
    """A 128 x 128 class (one CTA per candidate) and a 256 x 256 class (a
    cluster of 5 CTAs per candidate) in one call and one workspace: every
    candidate equals its one-candidate call at the same configuration bit for
    bit, boac_mlem to float rounding, and one per class the oracle."""
    classes = [(128, 0.2, 120), (256, 0.1, 16)]
    cls = [1, 0, 1, 0, 0, 1, 1]
    K = [3, 4, 2, 2, 5, 1, 4]
    probs = [make_problem(*classes[c], counts=2e5, B=1, seed=400 + i) for i, c in enumerate(cls)]
    geoms = [Geom.make(n, float(np.float32(dx)), V) for n, dx, V in classes]
    mu = [torch.tensor(p.mu[0], dtype=torch.float32, device=cuda) for p in probs]
    S = [torch.tensor(p.S, dtype=torch.float32, device=cuda) for p in probs]
    batch = boac.RaggedBatch(geoms, cls, K, mu, S, device=cuda)
    config = [4, 6]
    L = boac.boac_mlem_ragged(batch, config=config).cpu().numpy()
    for b, p in enumerate(probs):
        g = geoms[cls[b]]
        F1, L1 = one_candidate(g, mu[b], S[b], K[b], config[cls[b]], cuda)
        torch.testing.assert_close(batch.image(b), F1, rtol=0, atol=0)
        assert L[b] == L1
        F, Lu = boac.boac_mlem(g, torch.tensor(p.mu, dtype=torch.float32, device=cuda),
                               torch.tensor(p.S, dtype=torch.float32, device=cuda),
                               torch.ones(1, p.n, p.n, device=cuda), K[b])
        assert rel_l2(batch.image(b).cpu().numpy(), F[0].cpu().numpy()) < 1e-5
        assert abs(L[b] - float(Lu[0])) < 1e-6 * abs(L[b])
    for b in (1, 0):
        p = probs[b]
        Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu, p.S, K[b])
        assert rel_l2(batch.image(b).cpu().numpy(), Fo[0]) < 1e-4
        assert abs(L[b] - Lo[0]) < 1e-6 * abs(Lo[0])
