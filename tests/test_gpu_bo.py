"""The BO driver on the GPU objective: a few batched cycles on a small
problem pick candidates better than the initial random set, and the
objective equals -L of boac_mlem.  (Where the optimum lies is a property of
the data and of K, not of the optimiser: with 8 iterations and this noise the
likelihood can prefer a head smaller than the true one.)"""
import numpy as np
import pytest
import torch

from paper_2109_11920_gb300 import Geom, Tissue, bo, synth
from paper_2109_11920_gb300 import api as boac
from problems import make_problem

pytestmark = pytest.mark.gpu


def test_bo_driver_on_gpu_objective(cuda):
    p = make_problem(64, 0.4, 60, 2e5, B=1, seed=31)
    g, t = Geom.make(p.n, p.dx, p.V), Tissue(*p.tissue)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    K = 8
    evaluate = bo.gpu_objective(g, t, S, K, include_lgamma=False)
    c_true = np.array(synth.C_TRUE)
    # consistency with the library call
    C = np.stack([c_true, c_true + 0.2])
    mu = boac.boac_rasterize_mu(g, t, torch.tensor(C, dtype=torch.float32, device=cuda))
    _, L = boac.boac_mlem(g, mu, S, torch.ones(2, p.n, p.n, device=cuda), K, include_lgamma=False)
    np.testing.assert_allclose(evaluate(C), -L.cpu().numpy(), rtol=0, atol=0)
    # search c_0 in [6.5, 9.5] cm, the shape terms around their true values
    half = np.array([1.5, 0.15, 0.2, 0.1, 0.05, 0.03])
    lo, hi = c_true - half, c_true + half
    res = bo.BOACOptimizer(evaluate, lo, hi, batch=16, init=32, max_cycles=4, ei_threshold=0.0, seed=7).run()
    init_f = res.history_f[:32]
    assert res.cycles >= 1 and len(res.history_f) > 32
    # the EI-driven picks concentrate where the objective is low
    assert np.median(res.history_f[32:]) < np.median(init_f)
    assert res.best_f <= np.min(init_f)
    assert np.all(res.history_c >= lo - 1e-9) and np.all(res.history_c <= hi + 1e-9)


def test_bo_with_gradient_polish_on_gpu(cuda):
    """The whole search on the AREA objective: batched BO cycles, then the
    incumbent refined by L-BFGS-B on boac_score_grad's exact gradient.  The
    gradient path's objective equals the batched objective's to float
    rounding, and the polish never ends worse than its start."""
    p = make_problem(64, 0.4, 60, 2e5, B=1, seed=33)
    g, t = Geom.make(p.n, p.dx, p.V), Tissue(*p.tissue)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    K = 8
    evaluate = bo.gpu_objective(g, t, S, K, mode=boac._lib.RASTER_AREA)
    fg = bo.gpu_objective_and_grad(g, t, S, K, ckpt_every=2)
    c_true = np.array(synth.C_TRUE)
    C = np.stack([c_true, c_true + 0.1, c_true - 0.05])
    f_grad, grad = fg(C)
    np.testing.assert_allclose(f_grad, evaluate(C), rtol=1e-6)
    assert grad.shape == (3, 6) and np.all(np.isfinite(grad))
    half = np.array([1.5, 0.15, 0.2, 0.1, 0.05, 0.03])
    lo, hi = c_true - half, c_true + half
    res = bo.BOACOptimizer(evaluate, lo, hi, batch=8, init=16, max_cycles=2, ei_threshold=0.0, seed=11,
                           polish=fg, polish_iter=20).run()
    assert res.polish is not None and res.polish["evaluations"] >= 2
    assert res.polish["f"] <= res.polish["start_f"] + 1e-6 * abs(res.polish["start_f"])
    assert res.best_f <= res.polish["start_f"]
    assert np.all(res.best_c >= lo - 1e-9) and np.all(res.best_c <= hi + 1e-9)
