"""The device-side cache of scatter schedules: the fused kernels take the
schedule of their geometry from one of a few cached slots (built on the
first call, its tag checked on the device afterwards), or, when every slot
holds another geometry, build it into the workspace on each call.  The
schedule changes the order of the scatter within a class only, so every
route gives the same images and scores: bit-identical across repeated
calls, and within the MLEM tolerance of the FP64 oracle (images 1e-4,
scores 1e-6 relative) for more geometries than the cache has slots."""
import numpy as np
import pytest
import torch

import oracle
from paper_2109_11920_gb300 import Geom
from paper_2109_11920_gb300 import api as boac
from problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu


def run(p, dev, K, config):
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=dev)
    Bn = mu.shape[0]
    S = torch.tensor(p.S, dtype=torch.float32, device=dev)
    batch = boac.RaggedBatch([g], [0] * Bn, [K] * Bn, list(mu), [S] * Bn, device=dev)
    L = boac.boac_mlem_ragged(batch, config=[config])
    return batch.F_pool.view(Bn, p.n, p.n).cpu().numpy(), L.cpu().numpy()


def test_more_geometries_than_slots(cuda):
    """Twelve 64 x 64 geometries (8 to 52 views) with 4 and with 2 views per
    grid: 24 schedules, more than the cache's 8 slots, so the later ones
    are built into the workspace."""
    K = 2
    for V in range(8, 56, 4):
        p = make_problem(64, 0.4, V, 2e5, B=2, seed=100 + V)
        Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu, p.S, K)
        for config in (4, 5):
            if not boac.config_valid(Geom.make(p.n, p.dx, p.V), config):
                continue
            F, L = run(p, cuda, K, config)
            for b in range(2):
                assert rel_l2(F[b], Fo[b]) < 1e-4, (V, config, b)
                assert abs(L[b] - Lo[b]) < 1e-6 * abs(Lo[b]), (V, config, b)


@pytest.mark.parametrize("config", [4, 9])
def test_repeated_calls_bit_identical(cuda, config):
    """The first call of a geometry builds its schedule, the next ones find
    the tag and skip the build: the same images and scores, bit for bit."""
    p = make_problem(128, 0.2, 120, 2e5, B=3, seed=23)
    K = 3
    F1, L1 = run(p, cuda, K, config)
    F2, L2 = run(p, cuda, K, config)
    F3, L3 = run(p, cuda, K, config)
    np.testing.assert_array_equal(F1, F2)
    np.testing.assert_array_equal(F1, F3)
    np.testing.assert_array_equal(L1, L2)
    np.testing.assert_array_equal(L1, L3)


def test_two_streams_same_new_geometry(cuda):
    """A geometry used for the first time on two streams at once: both
    calls may build the slot, writing the same values; both results match
    the one-stream result bit for bit."""
    p = make_problem(96, 25.6 / 96, 92, 2e5, B=4, seed=29)
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    K = 3
    F0 = torch.ones(4, p.n, p.n, device=cuda)
    streams = [torch.cuda.Stream(cuda), torch.cuda.Stream(cuda)]
    out = []
    torch.cuda.synchronize(cuda)
    for s in streams:
        with torch.cuda.stream(s):
            out.append(boac.boac_mlem(g, mu, S, F0.clone(), K, check_status=False))
    torch.cuda.synchronize(cuda)
    Fr, Lr = boac.boac_mlem(g, mu, S, F0.clone(), K)
    for F, L in out:
        np.testing.assert_array_equal(F.cpu().numpy(), Fr.cpu().numpy())
        np.testing.assert_array_equal(L.cpu().numpy(), Lr.cpu().numpy())
    Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu, p.S, K)
    for b in range(4):
        assert rel_l2(Fr[b].cpu().numpy(), Fo[b]) < 1e-4, b
