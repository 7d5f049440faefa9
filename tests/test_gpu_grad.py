"""d ln P / d c through K MLEM iterations on the GPU (boac_score_grad) against
the FP64 oracle's reverse-mode gradient and central finite differences.
Tolerance: 1e-3 relative to the largest gradient component (the stated bound
for the gradient), score 1e-6 relative."""
import numpy as np
import pytest
import torch

import oracle
from paper_2109_11920_gb300 import Geom, Tissue, synth
from paper_2109_11920_gb300 import api as boac
from problems import make_problem

pytestmark = pytest.mark.gpu


def run_grad(p, dev, K, ckpt, coefs=None, per_cand_S=None, unfused=False):
    c = torch.tensor(p.coefs if coefs is None else coefs, dtype=torch.float32, device=dev)
    S = torch.tensor(p.S if per_cand_S is None else per_cand_S, dtype=torch.float32, device=dev)
    L, grad, F = boac.boac_score_grad(Geom.make(p.n, p.dx, p.V), Tissue(*p.tissue), c, S, K,
                                      ckpt_every=ckpt, want_image=True, unfused=unfused)
    return L.cpu().numpy(), grad.cpu().numpy(), F.cpu().numpy()


def check_against_oracle(p, L, grad, F, K, picks):
    for b in picks:
        Lo, go, Fo = oracle.score_grad(p.geom, p.tissue, p.coefs[b], p.S, K)
        assert abs(L[b] - Lo) < 1e-6 * abs(Lo), (b, L[b], Lo)
        scale = np.abs(go).max()
        np.testing.assert_allclose(grad[b], go, rtol=1e-3, atol=1e-3 * scale, err_msg=f"candidate {b}")
        assert np.linalg.norm(F[b] - Fo) / np.linalg.norm(Fo) < 1e-4


def test_grad_small_against_oracle_and_fd(cuda):
    p = make_problem(32, 0.8, 16, 2e5, B=4, seed=2, mode=oracle.AREA)
    K = 3
    L, grad, F = run_grad(p, cuda, K, ckpt=2)
    check_against_oracle(p, L, grad, F, K, range(4))
    # central differences of the oracle's forward pipeline (h = 1e-4 cm)
    h = 1e-4
    b = 1
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        Lp = oracle.score_grad(p.geom, p.tissue, p.coefs[b] + e, p.S, K)[0]
        Lm = oracle.score_grad(p.geom, p.tissue, p.coefs[b] - e, p.S, K)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(grad[b, k] - fd) <= 1e-3 * np.abs(grad[b]).max(), (k, grad[b, k], fd)


def test_grad_checkpoint_interval_does_not_change_results(cuda):
    p = make_problem(64, 0.4, 60, 2e5, B=3, seed=4, mode=oracle.AREA)
    K = 5
    ref = run_grad(p, cuda, K, ckpt=1)
    for ck in (2, 3, 5, 7):
        out = run_grad(p, cuda, K, ckpt=ck)
        for a, b in zip(ref, out):
            np.testing.assert_array_equal(a, b)


def test_grad_K0_and_per_candidate_sinograms(cuda):
    p = make_problem(64, 0.4, 60, 2e5, B=2, seed=6, mode=oracle.AREA)
    L, grad, F = run_grad(p, cuda, 0, ckpt=2)
    Lo, go, _ = oracle.score_grad(p.geom, p.tissue, p.coefs[0], p.S, 0)
    assert abs(L[0] - Lo) < 1e-6 * abs(Lo)
    np.testing.assert_allclose(grad[0], go, rtol=1e-3, atol=1e-3 * np.abs(go).max())
    S2 = np.stack([p.S, 1.5 * p.S])
    L, grad, F = run_grad(p, cuda, 2, ckpt=1, per_cand_S=S2)
    Lo, go, _ = oracle.score_grad(p.geom, p.tissue, p.coefs[1], 1.5 * p.S, 2)
    np.testing.assert_allclose(grad[1], go, rtol=1e-3, atol=1e-3 * np.abs(go).max())


def test_grad_full_size_sampled(cuda):
    """The differentiable-score workload: 128^2, 120 views, 64 candidates,
    10 iterations, checkpoint every 2; two candidates checked against the
    FP64 oracle adjoint."""
    wl = synth.GRAD
    p = make_problem(wl.n, wl.dx, wl.V, wl.counts, B=wl.B, seed=wl.seed, mode=oracle.AREA)
    L, grad, F = run_grad(p, cuda, wl.K, ckpt=wl.extra["ckpt_every"])
    check_against_oracle(p, L, grad, F, wl.K, [0, wl.B - 1])
    assert np.all(np.isfinite(grad))


def test_autograd_function(cuda):
    p = make_problem(32, 0.8, 16, 2e5, B=3, seed=8, mode=oracle.AREA)
    g, t = Geom.make(p.n, p.dx, p.V), Tissue(*p.tissue)
    c = torch.tensor(p.coefs, dtype=torch.float32, device=cuda, requires_grad=True)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    L = boac.BoacScore.apply(c, g, t, S, 3, 2)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device=cuda)
    (L * w).sum().backward()
    _, grad, _ = boac.boac_score_grad(g, t, c.detach(), S, 3, 2)
    torch.testing.assert_close(c.grad, (w[:, None] * grad).float())


@pytest.mark.parametrize("shape", [(64, 0.4, 60), (96, 25.6 / 96, 90), (128, 0.2, 120)])
def test_fused_gradient_against_oracle_and_unfused(cuda, shape):
    """The fused kernel (boac_score_grad's path at these sizes: one CTA or a
    cluster per candidate) against the FP64 oracle adjoint and against the
    batched launch-per-step kernels, with a checkpoint interval that does
    not divide K (a short last segment)."""
    n, dx, V = shape
    p = make_problem(n, dx, V, 2e5, B=5, seed=44, mode=oracle.AREA)
    K = 5
    L, grad, F = run_grad(p, cuda, K, ckpt=2)
    Lu, gu, Fu = run_grad(p, cuda, K, ckpt=2, unfused=True)
    check_against_oracle(p, L, grad, F, K, [0, 4])
    np.testing.assert_allclose(L, Lu, rtol=1e-7)
    for b in range(5):
        np.testing.assert_allclose(grad[b], gu[b], rtol=2e-4, atol=2e-4 * np.abs(gu[b]).max())
    assert np.linalg.norm(F - Fu) / np.linalg.norm(Fu) < 1e-5
