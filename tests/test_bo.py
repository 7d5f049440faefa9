"""Bayesian-optimisation driver (Sec. III steps 1-6) on CPU: the surrogate
against scikit-learn's GP, Expected Improvement against numerical integration
and its limits, the chaotic optimiser on functions with known minima, and the
driver on a synthetic objective."""
import numpy as np
import pytest
from scipy import integrate
from scipy.stats import norm

from paper_2109_11920_gb300 import bo


def test_rbf_kernel_closed_form():
    rng = np.random.default_rng(0)
    X = rng.uniform(size=(5, 6))
    K = bo.rbf_kernel(X, X, 2.0, 0.4)
    for i in range(5):
        for j in range(5):
            assert K[i, j] == pytest.approx(2.0 * np.exp(-np.sum((X[i] - X[j]) ** 2) / (2 * 0.16)), rel=1e-12)


def test_gp_matches_sklearn():
    gp_mod = pytest.importorskip("sklearn.gaussian_process")
    kernels = pytest.importorskip("sklearn.gaussian_process.kernels")
    rng = np.random.default_rng(1)
    X = rng.uniform(size=(30, 6))
    y = np.sin(3 * X[:, 0]) + X[:, 1] ** 2 - X[:, 2] * X[:, 3]
    Xs = rng.uniform(size=(20, 6))
    ours = bo.GaussianProcess(l=1.7, sigma0=0.45, noise=1e-4).fit(X, y)
    mu, sd = ours.predict(Xs)
    ref = gp_mod.GaussianProcessRegressor(
        kernel=kernels.ConstantKernel(1.7, "fixed") * kernels.RBF(0.45, "fixed"), alpha=1e-4, optimizer=None)
    ref.fit(X, y)
    mu_r, sd_r = ref.predict(Xs, return_std=True)
    np.testing.assert_allclose(mu, mu_r, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(sd, sd_r, rtol=1e-6, atol=1e-8)
    assert ours.log_marginal_likelihood() == pytest.approx(ref.log_marginal_likelihood_value_, rel=1e-9)


def test_gp_interpolates_training_points():
    rng = np.random.default_rng(2)
    X = rng.uniform(size=(15, 3))
    y = rng.normal(size=15)
    gp = bo.GaussianProcess(1.0, 0.3, 1e-10).fit(X, y)
    mu, sd = gp.predict(X)
    np.testing.assert_allclose(mu, y, atol=1e-5)
    assert np.all(sd < 1e-3)


@pytest.mark.parametrize("mu,sigma,fb,xi", [(0.3, 0.7, 0.1, 0.0), (-1.0, 0.2, 0.5, 0.05), (2.0, 1.5, -0.5, 0.1)])
def test_expected_improvement_is_the_expectation(mu, sigma, fb, xi):
    """EI = E[max(f_best - xi - Y, 0)], Y ~ N(mu, sigma^2), by quadrature."""
    f = lambda y: max(fb - xi - y, 0.0) * norm.pdf(y, mu, sigma)  # noqa: E731
    ref, _ = integrate.quad(f, mu - 12 * sigma, mu + 12 * sigma, points=[fb - xi], limit=200)
    assert bo.expected_improvement(mu, sigma, fb, xi) == pytest.approx(ref, rel=1e-7, abs=1e-12)


def test_expected_improvement_limits():
    assert bo.expected_improvement(0.2, 0.0, 1.0) == pytest.approx(0.8)  # certain improvement
    assert bo.expected_improvement(2.0, 0.0, 1.0) == 0.0  # certain non-improvement
    s = 0.37
    assert bo.expected_improvement(1.0, s, 1.0) == pytest.approx(s * norm.pdf(0.0))
    mus = np.linspace(-2, 2, 41)
    ei = bo.expected_improvement(mus, 0.5, 0.0)
    assert np.all(np.diff(ei) < 0)  # lower predicted mean, more expected improvement


def test_logistic_map_stays_in_the_unit_interval_and_does_not_cycle():
    seq = bo.logistic_sequence(np.array([0.123, 0.456, 0.789]), 2000)
    assert np.all((seq > 0) & (seq < 1))
    for d in range(3):
        assert len(np.unique(np.round(seq[:, d], 12))) > 1900


def test_chaotic_minimize_finds_known_minima():
    rng = np.random.default_rng(3)
    x_star = np.array([0.31, 0.77, 0.52, 0.18, 0.64, 0.45])
    quad = lambda P: np.sum((P - x_star) ** 2, axis=1)  # noqa: E731
    x, fmin = bo.chaotic_minimize(quad, 6, rng, n_global=2000, n_local=2000)
    assert fmin < 1e-3 and np.max(np.abs(x - x_star)) < 0.03

    def branin(P):  # three global minima, value 0.397887
        x1 = 15 * P[:, 0] - 5
        x2 = 15 * P[:, 1]
        return ((x2 - 5.1 / (4 * np.pi ** 2) * x1 ** 2 + 5 / np.pi * x1 - 6) ** 2
                + 10 * (1 - 1 / (8 * np.pi)) * np.cos(x1) + 10)
    x, fmin = bo.chaotic_minimize(branin, 2, rng, n_global=2000, n_local=1000)
    assert fmin == pytest.approx(0.397887, abs=2e-3)


def test_driver_converges_on_a_synthetic_objective():
    """6-D objective with minimum at c*: the driver gets close in a few
    batched cycles and its EI trace shrinks."""
    c_star = np.array([8.0, 0.3, -0.6, 0.2, -0.1, 0.05])
    lo, hi = c_star - np.array([1.5, 0.3, 0.4, 0.3, 0.2, 0.2]), c_star + np.array([1.0, 0.5, 0.3, 0.2, 0.3, 0.2])
    scale = hi - lo
    calls = []

    def evaluate(C):
        calls.append(len(C))
        return 1e3 * np.sum(((np.asarray(C) - c_star) / scale) ** 2, axis=1)

    opt = bo.BOACOptimizer(evaluate, lo, hi, batch=8, init=32, max_cycles=8, ei_threshold=0.0, seed=4)
    res = opt.run()
    assert calls[0] == 32 and all(c == 8 for c in calls[1:])
    assert res.best_f < 0.1 * np.median(res.history_f[:32])
    assert np.max(np.abs(res.best_c - c_star) / scale) < 0.1
    # a large EI threshold stops after the first cycle without evaluating more
    calls.clear()
    res2 = bo.BOACOptimizer(evaluate, lo, hi, batch=4, init=16, ei_threshold=1e9, seed=5).run()
    assert res2.cycles == 1 and calls == [16]


def test_gradient_polish_known_minima():
    """refine_with_gradient (L-BFGS-B in unit-box coordinates): an
    anisotropic quadratic with its minimum inside the box is found from a
    corner; a minimum outside the box lands on the violated bound with the
    other coordinates at their optimum; Rosenbrock's valley reaches (1, 1)."""
    lo, hi = np.array([5.0, -1.0, -0.5]), np.array([10.0, 1.0, 0.5])
    m = np.array([8.0, 0.3, -0.2])
    w = np.array([1.0, 50.0, 400.0])

    def fg(X, m=m):
        X = np.asarray(X, dtype=np.float64)
        assert np.all(X >= lo - 1e-12) and np.all(X <= hi + 1e-12)
        return np.sum(w * (X - m) ** 2, axis=1), 2 * w * (X - m)

    x, fx, calls = bo.refine_with_gradient(fg, hi, lo, hi, max_iter=100)
    np.testing.assert_allclose(x, m, atol=1e-5)
    assert fx < 1e-8 and calls >= 2
    m_out = np.array([12.0, 0.3, -0.2])  # c_0 beyond its upper bound
    x, _, _ = bo.refine_with_gradient(lambda X: fg(X, m_out), lo, lo, hi, max_iter=100)
    assert x[0] == pytest.approx(hi[0], abs=1e-9)
    np.testing.assert_allclose(x[1:], m_out[1:], atol=1e-5)

    def rosen(X):
        x1, x2 = X[:, 0], X[:, 1]
        f = (1 - x1) ** 2 + 100 * (x2 - x1 ** 2) ** 2
        g = np.stack([-2 * (1 - x1) - 400 * x1 * (x2 - x1 ** 2), 200 * (x2 - x1 ** 2)], axis=1)
        return f, g

    x, fx, _ = bo.refine_with_gradient(rosen, np.array([-1.2, 1.0]), np.array([-2.0, -2.0]),
                                       np.array([2.0, 2.0]), max_iter=500)
    np.testing.assert_allclose(x, [1.0, 1.0], atol=1e-4)


def test_gradient_polish_in_the_driver():
    """The driver's optional polish starts from the BO incumbent, keeps the
    better point, and does not run without a gradient function; non-finite
    values (an infeasible region) do not stop it."""
    c_star = np.array([8.0, 0.3, -0.6, 0.2, -0.1, 0.05])
    lo, hi = c_star - 0.5, c_star + 0.5
    scale = hi - lo

    def evaluate(C):
        C = np.asarray(C)
        f = np.sum(((C - c_star) / scale) ** 2, axis=1)
        return np.where(C[:, 0] > c_star[0] + 0.45, np.inf, f)

    def fg(C):
        C = np.asarray(C)
        f = evaluate(C)
        return f, 2 * (C - c_star) / scale ** 2

    res0 = bo.BOACOptimizer(evaluate, lo, hi, batch=4, init=16, max_cycles=2, ei_threshold=0.0, seed=3).run()
    assert res0.polish is None
    res = bo.BOACOptimizer(evaluate, lo, hi, batch=4, init=16, max_cycles=2, ei_threshold=0.0, seed=3,
                           polish=fg).run()
    assert res.polish is not None
    np.testing.assert_array_equal(res.polish["start_c"], res0.best_c)
    assert res.polish["start_f"] == res0.best_f
    assert res.best_f <= res0.best_f and res.best_f < 1e-10
    np.testing.assert_allclose(res.best_c, c_star, atol=1e-5)
