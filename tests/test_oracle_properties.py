"""Randomised invariants of the FP64 oracle over many small geometries (image
side, view count, pixel size, attenuation and activity drawn at random):
adjointness of the projector pair, the written-out system matrix against
both operators, and MLEM's count preservation and non-negativity.  These are
properties of the method, not of the code, so a wrong index, sign or
transpose anywhere in the operators breaks them for most draws.  Runs on
CPU."""
import numpy as np
import pytest

import oracle

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

geometries = st.tuples(st.integers(8, 20), st.integers(1, 9), st.floats(0.2, 2.0),
                       st.integers(0, 2 ** 31 - 1))


def draw(n, V, dx, seed):
    rng = np.random.default_rng(seed)
    g = oracle.Geometry(n, dx, V)
    mu = rng.uniform(0.0, 0.3, (n, n)) * (rng.uniform(size=(n, n)) < 0.8)
    return g, mu, rng


@settings(max_examples=40, deadline=None)
@given(geometries)
def test_adjoint_pair(params):
    g, mu, rng = draw(*params)
    x = rng.uniform(0.0, 2.0, (g.n, g.n))
    y = rng.uniform(0.0, 2.0, (g.V, g.nb))
    lhs = float((oracle.project(g, mu, x) * y).sum())
    rhs = float((x * oracle.backproject(g, mu, y)).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)


@settings(max_examples=25, deadline=None)
@given(geometries)
def test_system_matrix_matches_both_operators(params):
    g, mu, rng = draw(*params)
    A = oracle.system_matrix(g, mu)
    x = rng.uniform(0.0, 2.0, (g.n, g.n))
    y = rng.uniform(0.0, 2.0, (g.V, g.nb))
    np.testing.assert_allclose(A @ x.ravel(), oracle.project(g, mu, x).ravel(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(A.T @ y.ravel(), oracle.backproject(g, mu, y).ravel(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(A.sum(axis=0), oracle.sensitivity(g, mu).ravel(), rtol=1e-12, atol=1e-13)
    # attenuation only removes counts: A^mu <= A^0 entry by entry
    A0 = oracle.system_matrix(g, np.zeros_like(mu))
    assert np.all(A <= A0 + 1e-15) and A.min() >= 0.0


@settings(max_examples=25, deadline=None)
@given(geometries, st.integers(1, 4))
def test_mlem_counts_and_sign(params, K):
    g, mu, rng = draw(*params)
    F_true = rng.uniform(0.0, 3.0, (g.n, g.n))
    q = oracle.project(g, mu, F_true)
    S = rng.poisson(q * 50.0).astype(np.float64)
    F = np.ones((g.n, g.n))
    for _ in range(K):
        q_prev = oracle.project(g, mu, F)
        F = oracle.mlem(g, mu, S, 1, F)
        assert F.min() >= 0.0
        # sum_i (A F^{k+1})_i = sum_j sens_j F^{k+1}_j = sum_i r_i (A F^k)_i
        #                     = sum of S over the rays with (A F^k)_i > 0
        qn = oracle.project(g, mu, F)
        assert float(qn.sum()) == pytest.approx(float(S[q_prev > 0].sum()), rel=1e-10)


@settings(max_examples=15, deadline=None)
@given(st.integers(12, 20), st.integers(2, 6), st.integers(0, 3), st.integers(0, 2 ** 31 - 1))
def test_tissue_value_derivatives(n, V, K, seed):
    """mu is linear in mu_b and mu_c for a fixed boundary, so L is smooth in
    them: the 9-parameter reverse-mode derivatives match central differences
    tightly over random heads, tissue values and data."""
    rng = np.random.default_rng(seed)
    dx = 24.0 / n
    g = oracle.Geometry(n, dx, V)
    p = np.concatenate([[rng.uniform(5.0, 9.0)], rng.uniform(-0.3, 0.3, 5),
                        [rng.uniform(0.1, 0.2), rng.uniform(0.2, 0.3), rng.uniform(0.4, 0.8)]])
    mu_true = oracle.rasterize(n, dx, p[6], p[7], p[8], p[:6], oracle.AREA)
    S = rng.poisson(oracle.project(g, mu_true, rng.uniform(0.5, 2.0, (n, n))) * 20.0).astype(np.float64)
    L, grad, _ = oracle.score_grad_params(g, p, S, K)

    def L_at(q):
        mu = oracle.rasterize(n, dx, q[6], q[7], q[8], q[:6], oracle.AREA)
        return oracle.score(g, mu, S, oracle.mlem(g, mu, S, K))

    for k in (6, 7):
        h = 1e-5
        e = np.zeros(9)
        e[k] = h
        fd = (L_at(p + e) - L_at(p - e)) / (2 * h)
        assert grad[k] == pytest.approx(fd, rel=1e-5, abs=1e-6 * (abs(L) + 1.0))
