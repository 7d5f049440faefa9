"""The 9-parameter model p = (c_0..c_5, mu_b, mu_c, dR) on the GPU:
boac_rasterize_mu_params and boac_score_grad_params with tissue values that
differ between candidates, against the FP64 oracle (each candidate with its
own tissue values) and against the 6-coefficient entry points at equal
tissue values.  Gradient tolerance: 1e-3 relative to the largest component
of its group (coefficients and dR in cm, mu_b and mu_c in cm^-1), as for the
6-coefficient gradient; score 1e-6 relative."""
import numpy as np
import pytest
import torch

import oracle
from paper_2109_11920_gb300 import Geom, Tissue, bo, synth
from paper_2109_11920_gb300 import api as boac
from problems import assert_center_classes, make_problem, rel_l2

pytestmark = pytest.mark.gpu

F32 = np.float32
GROUPS = (slice(0, 6), slice(6, 8), slice(8, 9))


def params_of(p, seed, spread=0.2):
    """[B, 9] float32-valued parameters: the problem's coefficients with
    per-candidate tissue values."""
    rng = np.random.default_rng(seed)
    t = synth.tissue_candidates(rng, p.coefs.shape[0], p.tissue, spread)
    return np.concatenate([p.coefs, t], axis=1).astype(F32).astype(np.float64)


def check_grad(grad, go):
    for sl in GROUPS:
        scale = np.abs(go[sl]).max()
        np.testing.assert_allclose(grad[sl], go[sl], rtol=1e-3, atol=1e-3 * scale)


@pytest.mark.parametrize("mode", [oracle.CENTER, oracle.AREA])
def test_rasterize_params_per_candidate(cuda, mode):
    p = make_problem(64, 0.4, 60, 1e5, B=6, seed=71)
    P = params_of(p, 1)
    P[2, 8] = -0.3  # a negative thickness is taken as 0
    g = Geom.make(p.n, p.dx, p.V)
    mu = boac.boac_rasterize_mu_params(g, torch.tensor(P, dtype=torch.float32, device=cuda),
                                       mode).cpu().numpy()
    for b in range(6):
        ref = oracle.rasterize(p.n, p.dx, P[b, 6], P[b, 7], max(P[b, 8], 0.0), P[b, :6], mode)
        if mode == oracle.CENTER:
            assert_center_classes(mu[b], ref, p.n, p.dx, P[b, :6], max(P[b, 8], 0.0))
        else:
            np.testing.assert_allclose(mu[b], ref, rtol=1e-6, atol=1e-7, err_msg=str(b))


def test_rasterize_params_equals_fixed_tissue_entry(cuda):
    p = make_problem(128, 0.2, 120, 1e5, B=5, seed=72)
    g = Geom.make(p.n, p.dx, p.V)
    c = torch.tensor(p.coefs, dtype=torch.float32, device=cuda)
    P = torch.cat([c, torch.tensor(p.tissue, dtype=torch.float32, device=cuda).expand(5, 3)], 1)
    for mode in (oracle.CENTER, oracle.AREA):
        a = boac.boac_rasterize_mu(g, Tissue(*p.tissue), c, mode)
        b = boac.boac_rasterize_mu_params(g, P.contiguous(), mode)
        assert torch.equal(a, b)


def test_grad_params_against_oracle(cuda):
    p = make_problem(32, 0.8, 16, 2e5, B=4, seed=73, mode=oracle.AREA)
    P = params_of(p, 2)
    g = Geom.make(p.n, p.dx, p.V)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    K = 3
    L, grad, F = boac.boac_score_grad_params(g, torch.tensor(P, dtype=torch.float32, device=cuda), S, K,
                                             ckpt_every=2, want_image=True)
    L, grad, F = L.cpu().numpy(), grad.cpu().numpy(), F.cpu().numpy()
    for b in range(4):
        Lo, go, Fo = oracle.score_grad_params(p.geom, P[b], p.S, K)
        assert abs(L[b] - Lo) < 1e-6 * abs(Lo), b
        check_grad(grad[b], go)
        assert rel_l2(F[b], Fo) < 1e-4


def test_grad_params_first_six_are_the_coefficient_gradient(cuda):
    p = make_problem(64, 0.4, 60, 2e5, B=3, seed=74, mode=oracle.AREA)
    g, t = Geom.make(p.n, p.dx, p.V), Tissue(*p.tissue)
    c = torch.tensor(p.coefs, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    P = torch.cat([c, torch.tensor(p.tissue, dtype=torch.float32, device=cuda).expand(3, 3)], 1)
    L6, g6, F6 = boac.boac_score_grad(g, t, c, S, 4, 2, want_image=True)
    L9, g9, F9 = boac.boac_score_grad_params(g, P.contiguous(), S, 4, 2, want_image=True)
    assert torch.equal(L6, L9) and torch.equal(F6, F9)
    torch.testing.assert_close(g9[:, :6], g6, rtol=1e-12, atol=0)


def test_grad_params_zero_iterations_and_nonpositive_thickness(cuda):
    p = make_problem(64, 0.4, 60, 2e5, B=2, seed=75, mode=oracle.AREA)
    P = params_of(p, 3)
    P[1, 8] = -0.2
    g = Geom.make(p.n, p.dx, p.V)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    L, grad, _ = boac.boac_score_grad_params(g, torch.tensor(P, dtype=torch.float32, device=cuda), S, 0, 2)
    L, grad = L.cpu().numpy(), grad.cpu().numpy()
    assert grad[1, 8] == 0.0
    for b in range(2):
        Lo, go, _ = oracle.score_grad_params(p.geom, P[b], p.S, 0)
        assert abs(L[b] - Lo) < 1e-6 * abs(Lo)
        check_grad(grad[b], go)


def test_grad_params_full_size_sampled(cuda):
    """The differentiable-score workload (128^2, 120 views, 64 candidates, 10
    iterations, checkpoint every 2) with per-candidate tissue values; two
    candidates checked against the FP64 oracle adjoint."""
    wl = synth.GRAD
    p = make_problem(wl.n, wl.dx, wl.V, wl.counts, B=wl.B, seed=wl.seed, mode=oracle.AREA)
    P = params_of(p, 4)
    g = Geom.make(p.n, p.dx, p.V)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    L, grad, _ = boac.boac_score_grad_params(g, torch.tensor(P, dtype=torch.float32, device=cuda), S, wl.K,
                                             ckpt_every=wl.extra["ckpt_every"])
    L, grad = L.cpu().numpy(), grad.cpu().numpy()
    assert np.all(np.isfinite(grad))
    for b in (0, wl.B - 1):
        Lo, go, _ = oracle.score_grad_params(p.geom, P[b], p.S, wl.K)
        assert abs(L[b] - Lo) < 1e-6 * abs(Lo), b
        check_grad(grad[b], go)


def test_autograd_and_bo_objective_with_nine_parameters(cuda):
    p = make_problem(32, 0.8, 16, 2e5, B=3, seed=76, mode=oracle.AREA)
    g = Geom.make(p.n, p.dx, p.V)
    P = torch.tensor(params_of(p, 5), dtype=torch.float32, device=cuda, requires_grad=True)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    L = boac.BoacScore.apply(P, g, None, S, 3, 2)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device=cuda)
    (L * w).sum().backward()
    _, grad, _ = boac.boac_score_grad_params(g, P.detach(), S, 3, 2)
    torch.testing.assert_close(P.grad, (w[:, None] * grad).float())
    # the BO objective takes rows of 9 as the 9-parameter model (fused MLEM:
    # a 64 x 64 problem)
    p = make_problem(64, 0.4, 60, 2e5, B=3, seed=77)
    g = Geom.make(p.n, p.dx, p.V)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    Pn = params_of(p, 6)
    evaluate = bo.gpu_objective(g, None, S, 4, include_lgamma=False)
    mu = boac.boac_rasterize_mu_params(g, torch.tensor(Pn, dtype=torch.float32, device=cuda))
    _, Lm = boac.boac_mlem(g, mu, S, torch.ones(3, p.n, p.n, device=cuda), 4, include_lgamma=False)
    np.testing.assert_allclose(evaluate(Pn), -Lm.cpu().numpy(), rtol=0, atol=0)
