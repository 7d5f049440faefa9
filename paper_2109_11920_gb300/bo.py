"""Bayesian-optimisation driver of BOAC (Sec. III, steps 1-6) on top of the
batched GPU candidate evaluation.

The objective is the negative Poisson log-likelihood -ln P(S | F^K(c), A^mu(c))
(Eq. 5-6) of a candidate head geometry c = (c_0..c_5) (Eq. 3), evaluated on
the GPU by ``boac_rasterize_mu`` + ``boac_mlem`` (K MLEM iterations, Sec. III
step 3) for a whole batch of candidates at once.  Around it:

* a Gaussian-process surrogate of the objective (Eq. 7) with the RBF kernel
  k(c, c') = l exp(-|c - c'|^2 / (2 sigma_0^2)) (Eq. 8; the paper names l a
  length scale but it multiplies the kernel, so here l is the signal variance
  and sigma_0 the length scale), fitted by exact Cholesky regression on
  coefficients scaled to the unit box and standardised objective values;
* Expected Improvement (Eq. 9-10), written for minimisation:
  EI = sigma (gamma Phi(gamma) + phi(gamma)), gamma = (f_best - mu - xi) / sigma
  (the paper's gamma has the opposite sign of mu - f_best, which would reward
  candidates worse than the best one; this is the standard form);
* a chaotic optimisation algorithm for the acquisition function (the paper
  cites one without giving it; this is the two-stage logistic-map search of
  Li & Jiang, "Chaos optimization algorithm", 1997: a global carrier-wave
  search over the box, then a shrinking local search around the best point);
* batches of q candidates per cycle so that every GPU call evaluates many
  candidates: after each pick the surrogate is told a "constant liar" value
  (f_best) at that point and EI is maximised again (Ginsbourger, Le Riche &
  Carraro, "Kriging is well-suited to parallelize optimization", 2010);
* the stopping rule of step 6: stop when the best EI of a cycle falls below a
  threshold (or after a cycle budget);
* optionally, a gradient polish of the incumbent: the library's exact
  gradient of the objective (``boac_score_grad``, through the AREA
  rasterisation) drives L-BFGS-B (Byrd, Lu, Nocedal & Zhu, "A limited memory
  algorithm for bound constrained optimization", 1995; scipy's
  implementation) within the search box, so the optimiser uses the
  gradients alongside its surrogate.

Host-side numpy: the surrogate has at most a few thousand points, so the GPU
work of a cycle (q candidates x K MLEM iterations) dominates by far.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.stats import norm


# ----------------------------------------------------------------- surrogate
def rbf_kernel(X1: np.ndarray, X2: np.ndarray, l: float, sigma0: float) -> np.ndarray:
    """Eq. 8: l * exp(-|x - x'|^2 / (2 sigma0^2)) for all pairs of rows."""
    d2 = (np.sum(X1 * X1, axis=1)[:, None] + np.sum(X2 * X2, axis=1)[None, :] - 2.0 * X1 @ X2.T)
    return l * np.exp(-np.maximum(d2, 0.0) / (2.0 * sigma0 * sigma0))


class GaussianProcess:
    """Exact GP regression with the RBF kernel of Eq. 8 and a noise term."""

    def __init__(self, l: float = 1.0, sigma0: float = 0.3, noise: float = 1e-6):
        self.l, self.sigma0, self.noise = float(l), float(sigma0), float(noise)

    def fit(self, X: np.ndarray, y: np.ndarray) -> "GaussianProcess":
        self.X = np.asarray(X, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        Kxx = rbf_kernel(self.X, self.X, self.l, self.sigma0) + self.noise * np.eye(len(self.X))
        self.Lc = np.linalg.cholesky(Kxx)
        self.alpha = np.linalg.solve(self.Lc.T, np.linalg.solve(self.Lc, y))
        self.y = y
        return self

    def predict(self, Xs: np.ndarray):
        """Posterior mean and standard deviation at the rows of Xs."""
        Xs = np.atleast_2d(np.asarray(Xs, dtype=np.float64))
        Ks = rbf_kernel(Xs, self.X, self.l, self.sigma0)
        mu = Ks @ self.alpha
        v = np.linalg.solve(self.Lc, Ks.T)
        var = self.l - np.sum(v * v, axis=0)
        return mu, np.sqrt(np.maximum(var, 1e-300))

    def log_marginal_likelihood(self) -> float:
        n = len(self.y)
        return float(-0.5 * self.y @ self.alpha - np.sum(np.log(np.diag(self.Lc))) - 0.5 * n * np.log(2 * np.pi))


def fit_gp(X: np.ndarray, y: np.ndarray, noise: float = 1e-6,
           scales=(0.05, 0.1, 0.2, 0.3, 0.5, 0.8, 1.2)) -> GaussianProcess:
    """GP on standardised targets; the length scale sigma_0 maximises the
    log marginal likelihood over a grid (signal variance l = 1 after
    standardisation)."""
    best, best_lml = None, -np.inf
    for s in scales:
        try:
            gp = GaussianProcess(1.0, s, noise).fit(X, y)
        except np.linalg.LinAlgError:
            continue
        lml = gp.log_marginal_likelihood()
        if lml > best_lml:
            best, best_lml = gp, lml
    if best is None:
        raise np.linalg.LinAlgError("no length scale gives a positive-definite kernel matrix")
    return best


# ----------------------------------------------------------------- acquisition
def expected_improvement(mu, sigma, f_best: float, xi: float = 0.0):
    """Eq. 9-10 for minimisation: sigma (gamma Phi(gamma) + phi(gamma)),
    gamma = (f_best - mu - xi) / sigma; 0 where sigma = 0 and mu >= f_best - xi."""
    mu = np.asarray(mu, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    imp = f_best - mu - xi
    with np.errstate(divide="ignore", invalid="ignore"):
        gamma = np.where(sigma > 0, imp / np.where(sigma > 0, sigma, 1.0), 0.0)
        ei = np.where(sigma > 0, sigma * (gamma * norm.cdf(gamma) + norm.pdf(gamma)), np.maximum(imp, 0.0))
    return np.maximum(ei, 0.0)


def logistic_sequence(x0: np.ndarray, n: int) -> np.ndarray:
    """n iterates of the fully chaotic logistic map x <- 4 x (1 - x), per
    component of x0 (each in (0, 1), away from its periodic points)."""
    out = np.empty((n, x0.size))
    x = np.asarray(x0, dtype=np.float64).copy()
    for i in range(n):
        x = 4.0 * x * (1.0 - x)
        out[i] = x
    return out


def chaotic_minimize(fun, dim: int, rng: np.random.Generator, n_global: int = 400,
                     n_local: int = 400, r_start: float = 0.25, r_end: float = 1e-4, block: int = 20,
                     lo=0.0, hi=1.0):
    """Two-stage chaos optimisation (Li & Jiang 1997) of fun over [lo, hi]^dim.

    Stage 1: carrier-wave search -- chaotic variables from independent
    logistic maps, mapped linearly onto the box.  Stage 2: around the best
    point so far, chaotic perturbations whose radius shrinks geometrically
    from r_start to r_end (fractions of the box), re-centred after every
    block of evaluations.  ``fun`` takes an [m, dim] array and returns m
    values (vectorised)."""
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), (dim,))
    hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), (dim,))
    x0 = rng.uniform(0.05, 0.95, dim)
    C = logistic_sequence(x0, n_global)
    P = lo + (hi - lo) * C
    vals = fun(P)
    i = int(np.argmin(vals))
    best_x, best_f = P[i].copy(), float(vals[i])
    # stage 2: local chaotic search with a shrinking radius
    C2 = logistic_sequence(rng.uniform(0.05, 0.95, dim), n_local)
    ratio = (r_end / r_start) ** (1.0 / max(n_local - 1, 1))
    for k0 in range(0, n_local, block):
        k = np.arange(k0, min(k0 + block, n_local))
        radius = (r_start * ratio ** k)[:, None] * (hi - lo)[None, :]
        cand = np.clip(best_x[None, :] + radius * (2.0 * C2[k] - 1.0), lo, hi)
        v = fun(cand)
        j = int(np.argmin(v))
        if v[j] < best_f:
            best_f, best_x = float(v[j]), cand[j].copy()
    return best_x, best_f


# ----------------------------------------------------------------- driver
@dataclass
class BOResult:
    best_c: np.ndarray
    best_f: float
    history_c: np.ndarray
    history_f: np.ndarray
    cycles: int
    ei_trace: list = field(default_factory=list)
    # gradient polish of the incumbent (None if not run): its start and
    # result, and the number of objective-and-gradient evaluations
    polish: dict | None = None


def refine_with_gradient(fg, x0, lo, hi, max_iter: int = 30):
    """Minimise f from x0 within [lo, hi] with L-BFGS-B (scipy), f and its
    gradient from ``fg(X) -> (f[m], grad[m, dim])`` called on one point at a
    time.  The search runs in unit-box coordinates (u = (x - lo) / (hi - lo),
    gradient scaled by hi - lo), so coefficients of different scales weigh
    alike.  Returns (x, f(x), evaluations)."""
    from scipy.optimize import minimize

    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    span = hi - lo
    calls = [0]

    def fun(u):
        calls[0] += 1
        fv, gv = fg(np.asarray(lo + u * span)[None, :])
        fv, gv = float(np.asarray(fv)[0]), np.asarray(gv, dtype=np.float64)[0] * span
        if not np.isfinite(fv):
            return 1e300, np.zeros_like(u)
        return fv, gv

    u0 = np.clip((np.asarray(x0, dtype=np.float64) - lo) / span, 0.0, 1.0)
    res = minimize(fun, u0, jac=True, method="L-BFGS-B", bounds=[(0.0, 1.0)] * u0.size,
                   options={"maxiter": int(max_iter)})
    return lo + res.x * span, float(res.fun), calls[0]


class BOACOptimizer:
    """Bayesian optimisation of the head-geometry coefficients (Sec. III).

    ``evaluate(C)`` maps an [m, 6] array of coefficients to m objective values
    (-ln P, lower is better); on the GPU that is one batched call.  The
    search box is [lo, hi] per coefficient."""

    def __init__(self, evaluate, lo, hi, batch: int = 32, init: int = 64, xi: float = 0.01,
                 ei_threshold: float = 1e-4, max_cycles: int = 20, seed: int = 0,
                 polish=None, polish_iter: int = 30):
        """``polish``: optional ``fg(X) -> (f, grad)`` of the same objective;
        after the cycles the incumbent is refined with it (refine_with_gradient)
        and kept if better."""
        self.evaluate = evaluate
        self.polish, self.polish_iter = polish, int(polish_iter)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)
        self.batch, self.init, self.xi = int(batch), int(init), float(xi)
        self.ei_threshold, self.max_cycles = float(ei_threshold), int(max_cycles)
        self.rng = np.random.default_rng(seed)

    def _to_unit(self, C):
        return (np.asarray(C) - self.lo) / (self.hi - self.lo)

    def _from_unit(self, U):
        return self.lo + np.asarray(U) * (self.hi - self.lo)

    def run(self) -> BOResult:
        dim = self.lo.size
        # step 1: initial random set in the box
        U = self.rng.uniform(0.0, 1.0, (self.init, dim))
        f = np.asarray(self.evaluate(self._from_unit(U)), dtype=np.float64)
        ei_trace = []
        cycles = 0
        for cycles in range(1, self.max_cycles + 1):
            finite = np.isfinite(f)
            m, s = f[finite].mean(), f[finite].std() + 1e-12
            y = (np.where(finite, f, f[finite].max()) - m) / s
            f_best = float(y.min())
            # steps 4-5: surrogate, then a batch of EI maximisers (constant liar)
            Xl, yl = U.copy(), y.copy()
            picks, best_ei = [], 0.0
            for q in range(self.batch):
                gp = fit_gp(Xl, yl)
                neg_ei = lambda P: -expected_improvement(*gp.predict(P), f_best, self.xi)  # noqa: E731
                x, v = chaotic_minimize(neg_ei, dim, self.rng)
                if q == 0:
                    best_ei = -v
                picks.append(x)
                Xl = np.vstack([Xl, x])
                yl = np.append(yl, f_best)
            ei_trace.append(best_ei * s)
            # step 6: stop once the best expected improvement is negligible
            if best_ei * s < self.ei_threshold:
                break
            P = np.array(picks)
            fp = np.asarray(self.evaluate(self._from_unit(P)), dtype=np.float64)
            U = np.vstack([U, P])
            f = np.append(f, fp)
        i = int(np.nanargmin(np.where(np.isfinite(f), f, np.inf)))
        best_c, best_f = self._from_unit(U[i]), float(f[i])
        polish = None
        if self.polish is not None:
            x, fx, calls = refine_with_gradient(self.polish, best_c, self.lo, self.hi, self.polish_iter)
            polish = {"start_c": best_c, "start_f": best_f, "c": x, "f": fx, "evaluations": calls}
            if fx < best_f:
                best_c, best_f = x, fx
        return BOResult(best_c, best_f, self._from_unit(U), f, cycles, ei_trace, polish)


def gpu_objective(g, t, S, K: int, device=None, include_lgamma: bool = False, mode=None):
    """-ln P(S | F^K(c), A^mu(c)) for a batch of coefficient vectors, on the
    GPU: rasterise (Eq. 3-4; CENTER unless ``mode`` says otherwise), K MLEM
    iterations, Eq. 5 score.  Rows of 6 are Legendre coefficients with the
    tissue values t; rows of 9 are the 9-parameter model (c_0..c_5, mu_b,
    mu_c, dR) and t is not used."""
    import torch

    from . import api

    dev = device or S.device

    def evaluate(C: np.ndarray) -> np.ndarray:
        c = torch.tensor(np.asarray(C, dtype=np.float32), device=dev)
        m = api._lib.RASTER_CENTER if mode is None else mode
        if c.shape[1] == 9:
            mu = api.boac_rasterize_mu_params(g, c, m)
        else:
            mu = api.boac_rasterize_mu(g, t, c, m)
        F = torch.ones(c.shape[0], g.n, g.n, device=dev)
        _, L = api.boac_mlem(g, mu, S, F, K, include_lgamma=include_lgamma)
        return (-L).cpu().numpy()

    return evaluate


def gpu_objective_and_grad(g, t, S, K: int, ckpt_every: int = 2, device=None,
                           include_lgamma: bool = False):
    """The objective of ``gpu_objective(..., mode=RASTER_AREA)`` with its
    gradient: fg(C) -> (-ln P [m], -d ln P / dc [m, 6 or 9]) from
    boac_score_grad / boac_score_grad_params (reverse mode through the K MLEM
    iterations and the AREA rasterisation) for a batch of rows."""
    import torch

    from . import api

    dev = device or S.device

    def fg(C: np.ndarray):
        c = torch.tensor(np.asarray(C, dtype=np.float32), device=dev)
        if c.shape[1] == 9:
            L, grad, _ = api.boac_score_grad_params(g, c, S, K, ckpt_every, include_lgamma)
        else:
            L, grad, _ = api.boac_score_grad(g, t, c, S, K, ckpt_every, include_lgamma)
        return -L.cpu().numpy(), -grad.cpu().numpy()

    return fg
