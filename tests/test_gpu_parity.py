"""CUDA path vs the FP64 oracle, element by element, on seeded inputs built
by the oracle (tests/problems.py).  Tolerances (relative L2 unless stated):
one projection or back-projection 1e-5; MLEM images 1e-4; the float64 score
reduction 1e-9 given the same q.  Marked gpu: run with ``-m gpu``."""
import numpy as np
import pytest
import torch

import oracle
from paper_2109_11920_gb300 import Geom, Tissue, synth
from paper_2109_11920_gb300 import api as boac
from problems import assert_center_classes, make_problem, rel_l2

pytestmark = pytest.mark.gpu

# (n, dx, V): the three image classes of the workloads, plus small odd shapes
SHAPES = [(64, 0.4, 60), (96, 25.6 / 96, 90), (128, 0.2, 120)]
ODD = [(33, 0.7, 7), (20, 1.1, 4)]


def T(x, dev, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=dev)


def geom(p):
    return Geom.make(p.n, p.dx, p.V)


@pytest.fixture(scope="module")
def probs():
    return {s: make_problem(*s, counts=2e5, B=3, seed=11) for s in SHAPES + ODD}


@pytest.mark.parametrize("mode", [oracle.CENTER, oracle.AREA])
def test_rasterize_candidate_groups(cuda, mode):
    """The rasteriser takes a pixel for a group of 8 candidates: 19
    candidates (two full groups and a ragged one) against the oracle, and
    bit for bit against rasterising each candidate alone."""
    p = make_problem(64, 0.4, 60, 1e5, B=19, seed=5, mode=mode)
    g, t = geom(p), Tissue(*p.tissue)
    mu = boac.boac_rasterize_mu(g, t, T(p.coefs, cuda), mode)
    for b in range(19):
        one = boac.boac_rasterize_mu(g, t, T(p.coefs[b:b + 1], cuda), mode)
        assert torch.equal(mu[b], one[0]), b
    mu = mu.cpu().numpy()
    for b in range(19):
        if mode == oracle.CENTER:
            assert_center_classes(mu[b], p.mu[b], p.n, p.dx, p.coefs[b], p.tissue[2])
        else:
            np.testing.assert_allclose(mu[b], p.mu[b], rtol=1e-6, atol=1e-7, err_msg=str(b))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mode", [oracle.CENTER, oracle.AREA])
def test_rasterize(cuda, shape, mode):
    n, dx, V = shape
    p = make_problem(n, dx, V, 1e5, B=8, seed=3, mode=mode)
    mu = boac.boac_rasterize_mu(geom(p), Tissue(*p.tissue), T(p.coefs, cuda), mode).cpu().numpy()
    ref = p.mu
    if mode == oracle.CENTER:
        # identical classes at every pixel whose centre is not within 1e-9 cm
        # of a boundary (checked in float64 on the host, pixel by pixel)
        for b in range(mu.shape[0]):
            assert_center_classes(mu[b], ref[b], n, p.dx, p.coefs[b], p.tissue[2])
        assert np.array_equal(np.unique(mu), np.unique(ref.astype(np.float32)))
    else:
        np.testing.assert_allclose(mu, ref, rtol=1e-6, atol=1e-7)


# Eq. 3-4 edge cases: R(theta) clamped to 0 over part of the circle, a head
# larger than the field of view, no cranium (dR = 0), a negative c_0 (R = 0
# everywhere: only the cranium disk of radius dR around the origin remains),
# and an off-centre lobe whose boundary passes through pixel centres.
EDGE_COEFS = {
    "clamped": [0.5, 3.0, 0.0, 0.0, 0.0, 0.0],
    "beyond_fov": [20.0, 0.3, -0.6, 0.2, -0.1, 0.05],
    "negative_c0": [-2.0, 0.3, -0.6, 0.2, -0.1, 0.05],
    "true_head": list(synth.C_TRUE),
    "lobed": [6.0, 1.5, 2.0, -1.0, 0.8, -0.4],
}


@pytest.mark.parametrize("dR", [0.6, 0.0])
@pytest.mark.parametrize("name", sorted(EDGE_COEFS))
@pytest.mark.parametrize("mode", [oracle.CENTER, oracle.AREA])
def test_rasterize_edge_cases(cuda, name, dR, mode):
    n, dx = 64, float(np.float32(0.4))
    mu_b, mu_c = float(np.float32(0.15)), float(np.float32(0.25))
    dR = float(np.float32(dR))
    coef = np.asarray(EDGE_COEFS[name], dtype=np.float32).astype(np.float64)
    g = Geom.make(n, dx, 60)
    mu = boac.boac_rasterize_mu(g, Tissue(mu_b, mu_c, dR), T(coef[None], cuda), mode).cpu().numpy()[0]
    ref = oracle.rasterize(n, dx, mu_b, mu_c, dR, coef, mode)
    if mode == oracle.CENTER:
        assert_center_classes(mu, ref, n, dx, coef, dR)
    else:
        np.testing.assert_allclose(mu, ref, rtol=1e-6, atol=1e-7)
    if name == "negative_c0":
        # R = 0: nothing is brain; only pixels within dR of the origin are cranium
        assert not np.any(ref == mu_b)
    if name == "beyond_fov" and mode == oracle.CENTER:
        assert np.all(ref == mu_b)


@pytest.mark.parametrize("shape", SHAPES + ODD)
def test_project(cuda, probs, shape):
    p = probs[shape]
    g = p.geom
    rng = np.random.default_rng(1)
    F = np.stack([p.F_true, rng.uniform(0, 2, (p.n, p.n)), np.ones((p.n, p.n))])
    q = boac.boac_project(geom(p), T(p.mu, cuda), T(F, cuda)).cpu().numpy()
    for b in range(3):
        assert rel_l2(q[b], oracle.project(g, p.mu[b], F[b])) < 1e-5


@pytest.mark.parametrize("shape", SHAPES + ODD)
def test_backproject(cuda, probs, shape):
    p = probs[shape]
    g = p.geom
    rng = np.random.default_rng(2)
    y = np.stack([p.S, rng.uniform(0, 3, (p.V, p.n)), np.ones((p.V, p.n))])
    out = boac.boac_backproject(geom(p), T(p.mu, cuda), T(y, cuda)).cpu().numpy()
    sens = boac.boac_backproject(geom(p), T(p.mu, cuda), None).cpu().numpy()
    for b in range(3):
        assert rel_l2(out[b], oracle.backproject(g, p.mu[b], y[b])) < 1e-5
        assert rel_l2(sens[b], oracle.sensitivity(g, p.mu[b])) < 1e-5


@pytest.mark.parametrize("shape", SHAPES)
def test_adjointness_fp32(cuda, probs, shape):
    """<A x, y> = <x, A^T y> for the CUDA pair itself (float32 rounding)."""
    p = probs[shape]
    rng = np.random.default_rng(3)
    x = T(rng.uniform(0, 1, (3, p.n, p.n)), cuda)
    y = T(rng.uniform(0, 1, (3, p.V, p.n)), cuda)
    mu = T(p.mu, cuda)
    lhs = (boac.boac_project(geom(p), mu, x).double() * y.double()).sum()
    rhs = (x.double() * boac.boac_backproject(geom(p), mu, y).double()).sum()
    assert abs(lhs - rhs) / abs(lhs) < 2e-6


def single_cta_config(p):
    """The one-CTA fused kernel's default shape (4n threads, 8n at 64 x 64)."""
    return 2 * (1 if p.n == 64 else 2) + (0 if p.V % 4 == 0 else 1)


def run_mlem(p, dev, K, plain=False, B=None, S=None, path=None):
    """path: None / "default" (boac_mlem's choice), "fused" (the persistent
    fused kernel, pinned through the ragged entry point), "unfused"
    (boac_mlem_unfused), "plain" (one candidate at a time)."""
    path = "plain" if plain else (path or "default")
    mu = T(p.mu if B is None else p.mu[:B], dev)
    Bn = mu.shape[0]
    S = T(p.S if S is None else S, dev)
    if path == "fused":
        batch = boac.RaggedBatch([geom(p)], [0] * Bn, [K] * Bn, list(mu), [S] * Bn, device=dev)
        L = boac.boac_mlem_ragged(batch, config=[single_cta_config(p)])
        return batch.F_pool.view(Bn, p.n, p.n).cpu().numpy(), L.cpu().numpy()
    F = torch.ones(Bn, p.n, p.n, dtype=torch.float32, device=dev)
    F, L = boac.boac_mlem(geom(p), mu, S, F, K, score=True, plain=path == "plain",
                          unfused=path == "unfused")
    return F.cpu().numpy(), L.cpu().numpy()


@pytest.mark.parametrize("path", ["default", "fused", "unfused", "plain"])
@pytest.mark.parametrize("shape", SHAPES)
def test_mlem_small(cuda, probs, shape, path):
    """20 iterations on the 64, 96 and 128 classes through every MLEM path:
    images within 1e-4, scores (float64 reduction of a float32 projection)
    within 1e-6 relative."""
    p = probs[shape]
    K = 20
    F, L = run_mlem(p, cuda, K, path=path)
    Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu, p.S, K)
    for b in range(p.mu.shape[0]):
        assert rel_l2(F[b], Fo[b]) < 1e-4, b
        assert abs(L[b] - Lo[b]) < 1e-6 * abs(Lo[b])


def test_fused_equals_plain(cuda, probs):
    p = probs[SHAPES[2]]
    F1, L1 = run_mlem(p, cuda, 10, path="fused")
    for path in ("plain", "unfused"):
        F2, L2 = run_mlem(p, cuda, 10, path=path)
        assert rel_l2(F1, F2) < 2e-5, path
        np.testing.assert_allclose(L1, L2, rtol=1e-7, err_msg=path)
    # the plain and the unfused path run the same kernels in the same order;
    # the score's ln S! term is summed per bin on the plain path and once for
    # the shared sinogram on the unfused one
    F2, L2 = run_mlem(p, cuda, 10, path="plain")
    F3, L3 = run_mlem(p, cuda, 10, path="unfused")
    np.testing.assert_array_equal(F2, F3)
    np.testing.assert_allclose(L2, L3, rtol=1e-13, atol=0)


def test_loglik_reduction_given_same_q(cuda, probs):
    """The float64 reduction of Eq. 5 matches the oracle's to 1e-9 on the
    same (float32) expected counts."""
    p = probs[SHAPES[2]]
    rng = np.random.default_rng(4)
    q = rng.uniform(0.0, 50.0, (3, p.V, p.n)).astype(np.float32)
    q[0, :, :5] = 0.0  # S = 0 there?  force S = 0 where q = 0 below
    S = np.stack([p.S, rng.poisson(q[1]).astype(float), rng.poisson(q[2]).astype(float)])
    S[0, :, :5] = 0.0
    for lg in (True, False):
        L = boac.boac_loglik(geom(p), T(q, cuda), T(S, cuda), include_lgamma=lg).cpu().numpy()
        for b in range(3):
            ref = oracle.loglik(S[b], q[b].astype(np.float64), lg)
            assert abs(L[b] - ref) <= 1e-9 * abs(ref)
    # q = 0 < S gives -inf
    q[2, 0, 0] = 0.0
    S[2, 0, 0] = 5.0
    L = boac.boac_loglik(geom(p), T(q, cuda), T(S, cuda)).cpu().numpy()
    assert L[2] == -np.inf and np.isfinite(L[1])


def test_score_matches_oracle(cuda, probs):
    p = probs[SHAPES[2]]
    F = np.stack([p.F_true, 0.5 * p.F_true + 0.1, np.ones((p.n, p.n))])
    L = boac.boac_score(geom(p), T(p.mu, cuda), T(p.S, cuda), T(F, cuda)).cpu().numpy()
    for b in range(3):
        ref = oracle.score(p.geom, p.mu[b], p.S, F[b])
        assert abs(L[b] - ref) < 1e-6 * abs(ref)


def test_edge_cases(cuda, probs):
    p = probs[SHAPES[0]]
    g = geom(p)
    mu = T(p.mu, cuda)
    S = T(p.S, cuda)
    # K = 0 leaves F unchanged and scores F^0
    F0 = torch.rand(3, p.n, p.n, device=cuda)
    F, L = boac.boac_mlem(g, mu, S, F0.clone(), 0)
    assert torch.equal(F, F0)
    Lref = boac.boac_score(g, mu, S, F0)
    torch.testing.assert_close(L, Lref, rtol=1e-7, atol=0)
    # all-zero sinogram: r = 0 -> F = 0 after one iteration, L = -sum q = 0
    F, L = boac.boac_mlem(g, mu, torch.zeros_like(S), torch.ones(3, p.n, p.n, device=cuda), 1)
    assert float(F.abs().max()) == 0.0 and float(L.abs().max()) == 0.0
    # mu = 0 (no attenuation correction) runs and matches the oracle
    mu0 = torch.zeros_like(mu)
    F, L = boac.boac_mlem(g, mu0, S, torch.ones(3, p.n, p.n, device=cuda), 5)
    Fo = oracle.mlem(p.geom, np.zeros((p.n, p.n)), p.S, 5)
    assert rel_l2(F[0].cpu().numpy(), Fo) < 1e-4
    # per-candidate sinograms (s_stride != 0)
    S3 = torch.stack([S, 2 * S, S.flip(-1)]).contiguous()
    F, L = boac.boac_mlem(g, mu, S3, torch.ones(3, p.n, p.n, device=cuda), 4)
    Fo1 = oracle.mlem(p.geom, p.mu[1], 2 * p.S, 4)
    assert rel_l2(F[1].cpu().numpy(), Fo1) < 1e-4
    # too small a workspace is refused, nothing launched
    ws = torch.empty(16, dtype=torch.uint8, device=cuda)
    with pytest.raises(Exception, match="workspace"):
        boac.boac_mlem(g, mu, S, torch.ones(3, p.n, p.n, device=cuda), 2, ws=ws)


def test_mlem_batched_full_size_sampled(cuda):
    """The batched workload at full size (128^2, 120 views, 256 candidates,
    50 iterations, one launch as the benchmark times it); the first candidate,
    candidates cut between two CTAs by the work split (1, 152) and the last
    one checked against the oracle."""
    wl = synth.BATCHED
    p = make_problem(wl.n, wl.dx, wl.V, wl.counts, B=wl.B, seed=wl.seed)
    F, L = run_mlem(p, cuda, wl.K, plain=False)
    picks = [0, 1, 152, wl.B - 1]
    Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu[picks], p.S, wl.K)
    for i, b in enumerate(picks):
        assert rel_l2(F[b], Fo[i]) < 1e-4, b
        assert abs(L[b] - Lo[i]) < 1e-6 * abs(Lo[i]), b
    assert np.all(np.isfinite(L)) and np.all(F >= 0)


def test_work_split_status_and_odd_batches(cuda, probs):
    """The fused kernel splits a batch's iterations evenly over its CTAs and
    may cut a candidate between two of them.  At one launch configuration,
    batches of every size give the same images as a one-candidate call, bit
    for bit; boac_mlem's default configuration depends on the batch size, and
    across configurations the results agree to float rounding.  The
    workspace status stays OK."""
    p = probs[SHAPES[0]]
    g = geom(p)
    mu1 = T(p.mu[:1], cuda)
    S = T(p.S, cuda)
    F1 = torch.ones(1, p.n, p.n, device=cuda)
    F1, L1 = boac.boac_mlem(g, mu1, S, F1, 7)
    for B in (2, 5, 151, 152, 153, 457):
        mu = mu1.expand(B, p.n, p.n).contiguous()
        ws = boac.workspace(g, B, boac._lib.OP_MLEM, cuda)
        F = torch.ones(B, p.n, p.n, device=cuda)
        F, L = boac.boac_mlem(g, mu, S, F, 7, ws=ws)
        assert boac.boac_workspace_status(ws) == boac._lib.BOAC_OK
        assert rel_l2(F.cpu().numpy(), F1.expand(B, p.n, p.n).cpu().numpy()) < 1e-5, B
        torch.testing.assert_close(L, L1.expand(B), rtol=1e-6, atol=0)
    for cfg in (2, 4):  # CTAs of 4n and 8n threads
        first = None
        for B in (1, 5, 153, 457):
            batch = boac.RaggedBatch([g], [0] * B, [7] * B, [mu1[0]] * B, [S] * B, device=cuda)
            L = boac.boac_mlem_ragged(batch, config=[cfg])
            F = batch.F_pool.view(B, p.n, p.n)
            if first is None:
                first = (F[0].clone(), L[0].clone())
            torch.testing.assert_close(F, first[0].expand(B, p.n, p.n), rtol=0, atol=0)
            torch.testing.assert_close(L, first[1].expand(B), rtol=0, atol=0)


def test_mlem_invariants_on_gpu(cuda, probs):
    """EM properties of the CUDA path itself (any size): counts preserved,
    sum(A F^{k+1}) = sum(S) over rays with q > 0; images non-negative; the
    likelihood never decreases from one iteration to the next."""
    p = probs[SHAPES[2]]
    g = geom(p)
    mu = T(p.mu, cuda)
    S = T(p.S, cuda)
    prev = None
    for K in range(1, 7):
        F = torch.ones(3, p.n, p.n, device=cuda)
        F, L = boac.boac_mlem(g, mu, S, F, K, include_lgamma=False)
        assert float(F.min()) >= 0.0
        q = boac.boac_project(g, mu, F).double()
        for b in range(3):
            np.testing.assert_allclose(float(q[b].sum()), float(S.double().sum()), rtol=2e-5)
        if prev is not None:
            assert torch.all(L >= prev - 1e-7 * prev.abs())
        prev = L
