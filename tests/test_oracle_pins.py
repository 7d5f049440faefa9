"""Pins for the FP64 oracle: each test checks it against something other than
itself -- a closed form, a textbook value, a library routine, brute force or
an invariant of the method -- chosen so that a dropped term, a wrong sign or
index, or a transposed operand fails at least one of them.

Runs on CPU (``-m "not gpu"``).
"""
import os
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from scipy import stats

import oracle
from paper_2109_11920_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
MU_B, MU_C, DR = synth.TISSUE


# ----------------------------------------------------------------- helpers
def grid_xy(n, dx):
    c = (n - 1) / 2.0
    x = (np.arange(n) - c) * dx
    X, Y = np.meshgrid(x, x)  # X along columns j, Y along rows i
    return X, Y


def disk_coverage(n, dx, radius, ss=8):
    """Fraction of each pixel inside a centred disk (ss x ss subsamples)."""
    X, Y = grid_xy(n, dx)
    off = ((np.arange(ss) + 0.5) / ss - 0.5) * dx
    cov = np.zeros((n, n))
    for ox in off:
        for oy in off:
            cov += ((X + ox) ** 2 + (Y + oy) ** 2 < radius ** 2)
    return cov / ss ** 2


def bins(g):
    return (np.arange(g.nb) - (g.nb - 1) / 2.0) * g.ds


# ----------------------------------------------------------------- Eq. 3
def test_legendre_textbook_values():
    """P_0..P_5 against exact textbook values (golden fixture)."""
    rows = []
    with open(os.path.join(HERE, "golden", "legendre_p0_p5.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(Fraction(t)) for t in line.split()])
    assert len(rows) == 5
    for row in rows:
        np.testing.assert_allclose(oracle.legendre(row[0]), row[1:], rtol=0, atol=1e-15)


def test_legendre_matches_numpy_and_is_orthogonal():
    rng = np.random.default_rng(1)
    for z in rng.uniform(-1, 1, 25):
        ref = [npleg.legval(z, np.eye(6)[k]) for k in range(6)]
        np.testing.assert_allclose(oracle.legendre(z), ref, rtol=0, atol=1e-14)
    # int_{-1}^{1} P_m P_n dz = 2/(2n+1) delta_mn (Gauss-Legendre, exact here)
    zs, ws = npleg.leggauss(12)
    P = np.array([oracle.legendre(z) for z in zs])
    gram = (P * ws[:, None]).T @ P
    np.testing.assert_allclose(gram, np.diag(2.0 / (2 * np.arange(6) + 1)), atol=1e-14)


# ----------------------------------------------------------------- Eq. 4
def test_rasterize_disk_classes():
    """c = (R0, 0, ...) is a disk: mu_b for r < R0, mu_c up to R0 + dR."""
    n, dx, R0 = 64, 0.4, 8.0
    mu = oracle.rasterize(n, dx, MU_B, MU_C, DR, [R0, 0, 0, 0, 0, 0], oracle.CENTER)
    X, Y = grid_xy(n, dx)
    r = np.hypot(X, Y)
    ref = np.where(r < R0, MU_B, np.where(r < R0 + DR, MU_C, 0.0))
    np.testing.assert_array_equal(mu, ref)


def test_rasterize_legendre_boundary_against_numpy():
    """CENTER mode against R(theta) from numpy's Legendre series at
    cos(theta) = cos(atan2(y, x)); only pixels within 1e-9 cm of a boundary
    may differ (the class there is decided by rounding)."""
    n, dx = 64, 0.4
    c = np.array(synth.C_TRUE)
    mu = oracle.rasterize(n, dx, MU_B, MU_C, DR, c, oracle.CENTER)
    X, Y = grid_xy(n, dx)
    r = np.hypot(X, Y)
    R = np.maximum(npleg.legval(np.cos(np.arctan2(Y, X)), c), 0.0)
    ref = np.where(r < R, MU_B, np.where(r < R + DR, MU_C, 0.0))
    tie = (np.abs(r - R) < 1e-9) | (np.abs(r - R - DR) < 1e-9)
    assert np.all((mu == ref) | tie)
    assert (mu == MU_B).sum() > 100 and (mu == MU_C).sum() > 20



@pytest.mark.parametrize("coef, dR", [(synth.C_TRUE, DR), ([0.5, 3.0, 0, 0, 0, 0], DR),
                                      ([-2.0, 0.3, -0.6, 0.2, -0.1, 0.05], DR),
                                      ([20.0, 0, 0, 0, 0, 0], 0.0)])
def test_center_class_check_is_exact_away_from_ties(coef, dR):
    """The CENTER-mode parity check used against the CUDA rasteriser: the
    oracle's map passes it, few pixels are ties, and one pixel flipped to
    another class away from a boundary -- or a boundary shifted by a tenth of
    a pixel -- fails it."""
    from problems import assert_center_classes, center_tie_mask
    n, dx = 64, 0.4
    c = np.asarray(coef, dtype=np.float64)
    mu = oracle.rasterize(n, dx, MU_B, MU_C, dR, c, oracle.CENTER)
    assert assert_center_classes(mu.astype(np.float32), mu, n, dx, c, dR)[0] == 0
    ties = center_tie_mask(n, dx, c, dR)
    assert ties.sum() <= 2
    bad = mu.astype(np.float32)
    i, j = np.argwhere(~ties)[n * n // 2 + 3]
    bad[i, j] = np.float32(MU_C if mu[i, j] != MU_C else MU_B)
    with pytest.raises(AssertionError):
        assert_center_classes(bad, mu, n, dx, c, dR)
    if c[0] > 0 and c[0] < 10:
        shifted = oracle.rasterize(n, dx, MU_B, MU_C, dR, c + np.array([0.04, 0, 0, 0, 0, 0]),
                                   oracle.CENTER)
        with pytest.raises(AssertionError):
            assert_center_classes(shifted.astype(np.float32), mu, n, dx, c, dR)

def test_rasterize_area_mode():
    """AREA mode: equals CENTER more than a pixel from any boundary, and its
    integral approaches the exact annulus areas (error O(dx^2) per unit
    length of boundary)."""
    n, dx, R0 = 128, 0.2, 8.0
    cen = oracle.rasterize(n, dx, MU_B, MU_C, DR, [R0, 0, 0, 0, 0, 0], oracle.CENTER)
    area = oracle.rasterize(n, dx, MU_B, MU_C, DR, [R0, 0, 0, 0, 0, 0], oracle.AREA)
    X, Y = grid_xy(n, dx)
    r = np.hypot(X, Y)
    far = (np.abs(r - R0) > dx) & (np.abs(r - R0 - DR) > dx)
    np.testing.assert_array_equal(area[far], cen[far])
    exact = MU_B * np.pi * R0 ** 2 + MU_C * np.pi * ((R0 + DR) ** 2 - R0 ** 2)
    assert abs(area.sum() * dx * dx - exact) / exact < 2e-3
    assert area.min() >= 0 and area.max() <= MU_C + 1e-15


# ----------------------------------------------------------------- Eq. 1
def analytic_disk(s, f0, a, mu0, R0):
    """Attenuated Radon transform of a uniform disk (radius a, activity f0)
    centred in a uniform attenuator (radius R0 >= a, mu0): the emission point
    at t sees mu0 over (t, L_R), so S = (2 f0/mu0) e^{-mu0 L_R} sinh(mu0 L_a)."""
    La = np.sqrt(np.maximum(a * a - s * s, 0.0))
    LR = np.sqrt(np.maximum(R0 * R0 - s * s, 0.0))
    if mu0 == 0.0:
        return 2 * f0 * La
    return 2 * f0 / mu0 * np.exp(-mu0 * LR) * np.sinh(mu0 * La)


@pytest.mark.parametrize("mu0", [0.15, 0.0])
def test_analytic_disk_convergence(mu0):
    """P1 (mu0 > 0) and P2 (mu0 = 0, chord length): the discretised operator
    converges to the closed form as the pixel shrinks (fixed 25.6 cm FOV)."""
    a, R0, f0 = 5.0, 9.0, 1.0
    errs = []
    for n in (32, 128, 256):
        dx = 25.6 / n
        g = oracle.Geometry(n, dx, 6)
        F = f0 * disk_coverage(n, dx, a, ss=16)
        mu = mu0 * disk_coverage(n, dx, R0, ss=16)
        q = oracle.project(g, mu, F)
        s = bins(g)
        keep = np.abs(s) < a - 2 * dx
        ref = analytic_disk(s[keep], f0, a, mu0, R0)
        errs.append(np.linalg.norm(q[:, keep] - ref[None]) / np.linalg.norm(np.broadcast_to(ref, q[:, keep].shape)))
    assert errs[0] > errs[1] > errs[2], errs
    # a dropped half-cell term would leave a ~mu0*dx/2 = 0.75% bias at n=256
    assert errs[2] < 2e-3, errs


def test_offcentre_source_attenuation_direction():
    """A small hot disk off-centre inside a uniform attenuating disk: per view,
    the projection summed over bins is sum_pixels (dx^2 f / ds) exp(-mu0 L),
    L the distance from the pixel to the attenuator's edge towards the
    detector, which sits at t -> +inf along (-sin phi, cos phi).  Pins the
    rotation sense and the direction of the attenuation integral (the wrong
    direction is off by exp(+-mu0 * 8 cm) here)."""
    n, V, mu0, R0 = 96, 12, 0.2, 11.0
    dx = 25.6 / n
    g = oracle.Geometry(n, dx, V)
    x0, y0, rad = -4.0, 2.5, 1.2
    X, Y = grid_xy(n, dx)
    F = ((X - x0) ** 2 + (Y - y0) ** 2 < rad ** 2).astype(float)
    mu = mu0 * disk_coverage(n, dx, R0)
    q = oracle.project(g, mu, F)
    P = np.stack([X[F > 0], Y[F > 0]], axis=1)
    for v in range(V):
        cs, sn = oracle.view_cos_sin(v, V)
        d = np.array([-sn, cs])
        pd = P @ d
        L = -pd + np.sqrt(pd * pd - (P * P).sum(1) + R0 * R0)
        expect = (dx * dx / g.ds * np.exp(-mu0 * L)).sum()
        assert abs(q[v].sum() - expect) / expect < 0.02, (v, q[v].sum(), expect)
        # the projection's centre of mass sits at s = x0 cos + y0 sin
        com = (bins(g) * q[v]).sum() / q[v].sum()
        assert abs(com - (x0 * cs + y0 * sn)) < 0.1 * rad


def test_exact_rotations_quarter_turns():
    """P3: at phi = 0, 90, 180, 270 deg every ray sample is a pixel centre, so
    A^mu reduces to exact discrete sums along rows/columns (numpy cumsum)."""
    n, dx = 20, 0.5
    rng = np.random.default_rng(3)
    F = rng.uniform(0, 1, (n, n))
    mu = rng.uniform(0, 0.3, (n, n))
    g = oracle.Geometry(n, dx, 4)
    q = oracle.project(g, mu, F)
    for v in range(4):
        # orient the image so that ray b is column b and the detector is at
        # the last row (k = n-1): phi = 0 is the identity; the other views
        # are quarter turns of the image.
        Fr, mr = np.rot90(F, k=v), np.rot90(mu, k=v)
        # rot90 by +1 maps view 1 (detector towards -x) onto view 0: the
        # sample (k, b) of view v is pixel (k, b) of np.rot90(img, v).
        suffix = np.cumsum(mr[::-1], axis=0)[::-1] - mr  # sum over k' > k
        att = np.exp(-dx * (0.5 * mr + suffix))
        ref = dx * (att * Fr).sum(axis=0)
        np.testing.assert_allclose(q[v], ref, rtol=1e-13, atol=1e-15)



def test_attenuation_table_quarter_turns():
    """The public attenuation-factor table (Eq. 1 inner integral) at
    phi = 0, 90, 180, 270 deg: sample (k, b) of view v is pixel (k, b) of
    the image turned v quarter turns, so every factor is
    exp(-dx (mu_k / 2 + sum_{k' > k} mu_k')) with the sum a numpy cumsum
    along the column towards the detector (k = n - 1)."""
    n, dx = 18, 0.6
    rng = np.random.default_rng(31)
    mu = rng.uniform(0, 0.4, (n, n))
    g = oracle.Geometry(n, dx, 4)
    a = oracle.attenuation(g, mu)
    assert a.shape == (4, n, n)
    for v in range(4):
        mr = np.rot90(mu, k=v)
        suffix = np.cumsum(mr[::-1], axis=0)[::-1] - mr
        np.testing.assert_allclose(a[v], np.exp(-dx * (0.5 * mr + suffix)), rtol=1e-14, atol=0)
    # mu = 0: no attenuation anywhere
    np.testing.assert_array_equal(oracle.attenuation(g, np.zeros((n, n))), np.ones((4, n, n)))

# ----------------------------------------------------------------- Eq. 2
def test_adjointness():
    """P4: <A x, y> = <x, A^T y> to 1e-12 relative."""
    rng = np.random.default_rng(4)
    for n, V in ((24, 7), (33, 10)):
        g = oracle.Geometry(n, 25.6 / n, V)
        mu = oracle.rasterize(n, g.dx, MU_B, MU_C, DR, synth.C_TRUE, oracle.CENTER)
        x = rng.uniform(0, 1, (n, n))
        y = rng.uniform(-1, 1, (V, n))
        lhs = np.sum(oracle.project(g, mu, x) * y)
        rhs = np.sum(x * oracle.backproject(g, mu, y))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def dense_system_matrix(n, dx, V, mu):
    """Independent brute force: every weight from the hat functions over ALL
    pixels (no floor/neighbour logic), attenuation by numpy cumsum, A as a
    dense (V*n) x (n*n) matrix."""
    c = (n - 1) / 2.0
    jj, ii = np.meshgrid(np.arange(n), np.arange(n))
    jj, ii = jj.ravel(), ii.ravel()
    A = np.zeros((V * n, n * n))
    for v in range(V):
        phi = 2 * np.pi * v / V
        cs, sn = np.cos(phi), np.sin(phi)
        for b in range(n):
            s = (b - c) * dx
            W = np.zeros((n, n * n))
            for k in range(n):
                t = (k - c) * dx
                u = c + (s * cs - t * sn) / dx
                w = c + (s * sn + t * cs) / dx
                W[k] = np.maximum(0, 1 - np.abs(u - jj)) * np.maximum(0, 1 - np.abs(w - ii))
            m = W @ mu.ravel()
            after = np.concatenate([np.cumsum(m[::-1])[::-1][1:], [0.0]])
            att = np.exp(-dx * (0.5 * m + after))
            A[v * n + b] = dx * att @ W
    return A


def test_dense_brute_force_16():
    """P5: 16x16, V=8 -- projector and back-projector equal a dense matrix
    built independently, to 1e-13."""
    n, V = 16, 8
    dx = 25.6 / n
    mu = oracle.rasterize(n, dx, MU_B, MU_C, DR, [6.5, 0.4, -0.5, 0.2, -0.1, 0.05], oracle.CENTER)
    A = dense_system_matrix(n, dx, V, mu)
    g = oracle.Geometry(n, dx, V)
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 2, (n, n))
    y = rng.uniform(0, 2, (V, n))
    np.testing.assert_allclose(oracle.project(g, mu, x).ravel(), A @ x.ravel(), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(oracle.backproject(g, mu, y).ravel(), A.T @ y.ravel(), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(oracle.sensitivity(g, mu).ravel(), A.sum(axis=0), rtol=1e-13, atol=1e-14)


def test_system_matrix_written_out():
    """P5b: the oracle's explicit A^mu (the system matrix of Sec. III) equals
    the hat-function brute force above, its products equal the matrix-free
    projector and back-projector, every entry is >= 0 and no row has more
    than 4n nonzeros (four bilinear neighbours per sample)."""
    n, V = 16, 8
    dx = 25.6 / n
    mu = oracle.rasterize(n, dx, MU_B, MU_C, DR, [6.5, 0.4, -0.5, 0.2, -0.1, 0.05], oracle.CENTER)
    g = oracle.Geometry(n, dx, V)
    A = oracle.system_matrix(g, mu)
    np.testing.assert_allclose(A, dense_system_matrix(n, dx, V, mu), rtol=1e-12, atol=1e-14)
    assert A.min() >= 0.0 and (A > 0).sum(axis=1).max() <= 4 * n
    g = oracle.Geometry(24, 0.6, 12)
    mu = oracle.rasterize(24, 0.6, MU_B, MU_C, DR, [6.0, 0.3, -0.4, 0.1, 0.0, 0.05], oracle.AREA)
    A = oracle.system_matrix(g, mu)
    rng = np.random.default_rng(6)
    x = rng.uniform(0, 2, (24, 24))
    y = rng.uniform(0, 2, (12, 24))
    np.testing.assert_allclose(A @ x.ravel(), oracle.project(g, mu, x).ravel(), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(A.T @ y.ravel(), oracle.backproject(g, mu, y).ravel(), rtol=1e-12, atol=1e-14)


def test_mirror_symmetry():
    """P7: with a head symmetric about the x axis (P_k(cos theta) is even in
    theta) and a mirror-symmetric activity, q(v, b) = q((V/2 - v) mod V,
    nb-1-b) up to rounding of cos/sin."""
    n, V = 40, 12
    dx = 25.6 / n
    mu = oracle.rasterize(n, dx, MU_B, MU_C, DR, synth.C_TRUE, oracle.CENTER)
    np.testing.assert_array_equal(mu, mu[::-1])
    rng = np.random.default_rng(6)
    F = rng.uniform(0, 1, (n, n))
    F = F + F[::-1]
    g = oracle.Geometry(n, dx, V)
    q = oracle.project(g, mu, F)
    for v in range(V):
        np.testing.assert_allclose(q[v], q[(V // 2 - v) % V, ::-1], rtol=1e-12, atol=1e-14)


# ----------------------------------------------------------------- MLEM
def small_problem(n=32, V=16, counts=5e4, seed=0):
    dx = 25.6 / n
    g = oracle.Geometry(n, dx, V)
    ph, noise, _ = synth.streams(seed)
    mu = oracle.rasterize(n, dx, MU_B, MU_C, DR, synth.C_TRUE, oracle.CENTER)
    Ftrue = synth.paint_activity(n, dx, mu == MU_B, synth.ellipses(ph, synth.C_TRUE[0]))
    S = synth.poisson_sinogram(noise, oracle.project(g, mu, Ftrue), counts)
    return g, mu, S, Ftrue


def test_mlem_invariants():
    """P6: count preservation sum(A F^{k+1}) = sum(S), F >= 0, EM monotone
    likelihood, and F^1 independent of the scale of F^0."""
    g, mu, S, _ = small_problem()
    F = np.ones((g.n, g.n))
    L_prev = -np.inf
    for it in range(6):
        q = oracle.project(g, mu, F)
        assert np.all(S[q <= 0] == 0)
        L = oracle.loglik(S, q, include_lgamma=False)
        assert L >= L_prev - 1e-12 * abs(L)
        L_prev = L
        F = oracle.mlem(g, mu, S, 1, F)
        assert F.min() >= 0
        np.testing.assert_allclose(oracle.project(g, mu, F).sum(), S.sum(), rtol=1e-12)
    F1a = oracle.mlem(g, mu, S, 1, np.ones((g.n, g.n)))
    F1b = oracle.mlem(g, mu, S, 1, 7.5 * np.ones((g.n, g.n)))
    np.testing.assert_allclose(F1a, F1b, rtol=1e-12, atol=1e-300)


def test_mlem_recovers_noise_free_phantom():
    """With noise-free data MLEM drives A F towards S (likelihood gap to the
    saturated model shrinks monotonically)."""
    g, mu, _, Ftrue = small_problem()
    S = oracle.project(g, mu, Ftrue)
    gaps = []
    for K in (2, 8, 32):
        F = oracle.mlem(g, mu, S, K)
        q = oracle.project(g, mu, F)
        gaps.append(oracle.loglik(S, S, False) - oracle.loglik(S, q, False))
    assert gaps[0] > gaps[1] > gaps[2] >= -1e-9


# ----------------------------------------------------------------- Eq. 5
def test_loglik_is_poisson_logpmf():
    """Eq. 5 with the ln S! term equals scipy's Poisson log-pmf summed."""
    rng = np.random.default_rng(7)
    q = rng.uniform(0.01, 40, 500)
    S = rng.poisson(q).astype(float)
    S[:20] = 0
    np.testing.assert_allclose(oracle.loglik(S, q, True), stats.poisson.logpmf(S, q).sum(), rtol=1e-13)
    # without ln S!: differs by the constant sum(gammaln(S + 1))
    from scipy.special import gammaln
    np.testing.assert_allclose(oracle.loglik(S, q, False), stats.poisson.logpmf(S, q).sum() + gammaln(S + 1).sum(), rtol=1e-13)
    q0 = q.copy(); q0[50] = 0.0; S0 = S.copy(); S0[50] = 3.0
    assert oracle.loglik(S0, q0, True) == -np.inf
    S0[50] = 0.0
    assert np.isfinite(oracle.loglik(S0, q0, True))


def test_score_is_loglik_of_projection():
    g, mu, S, Ftrue = small_problem(n=24, V=8)
    q = oracle.project(g, mu, Ftrue)
    assert oracle.score(g, mu, S, Ftrue) == pytest.approx(oracle.loglik(S, q), rel=1e-15)


# ----------------------------------------------------------------- gradient
def fd_score(g, coef, S, K, h, k):
    def L(cv):
        mu = oracle.rasterize(g.n, g.dx, MU_B, MU_C, DR, cv, oracle.AREA)
        F = oracle.mlem(g, mu, S, K)
        return oracle.score(g, mu, S, F)
    e = np.zeros(6); e[k] = h
    return (L(coef + e) - L(coef - e)) / (2 * h)


def test_gradient_against_central_differences():
    """P8: reverse-mode dL/dc through K MLEM iterations vs central finite
    differences (h = 1e-4 cm) of the forward pipeline, and L itself equals
    rasterize(AREA) -> MLEM -> score."""
    g, mu, S, _ = small_problem(n=32, V=16, counts=2e5, seed=2)
    K = 3
    coef = np.array(synth.C_TRUE) + np.array([0.3, -0.1, 0.15, 0.05, 0.02, -0.03])
    L, grad, FK = oracle.score_grad(g, synth.TISSUE, coef, S, K)
    mu_a = oracle.rasterize(g.n, g.dx, MU_B, MU_C, DR, coef, oracle.AREA)
    np.testing.assert_allclose(FK, oracle.mlem(g, mu_a, S, K), rtol=1e-12, atol=1e-300)
    assert L == pytest.approx(oracle.score(g, mu_a, S, FK), rel=1e-13)
    fd = np.array([fd_score(g, coef, S, K, 1e-4, k) for k in range(6)])
    scale = np.abs(fd).max()
    np.testing.assert_allclose(grad, fd, rtol=1e-3, atol=1e-3 * scale)


def fd_score_params(g, p, S, K, h, k):
    def L(pv):
        dR = max(pv[8], 0.0)
        mu = oracle.rasterize(g.n, g.dx, pv[6], pv[7], dR, pv[:6], oracle.AREA)
        F = oracle.mlem(g, mu, S, K)
        return oracle.score(g, mu, S, F)
    e = np.zeros(9); e[k] = h
    return (L(p + e) - L(p - e)) / (2 * h)


def test_nine_parameter_gradient_against_central_differences():
    """P8b: the 9-parameter form p = (c, mu_b, mu_c, dR) -- reverse-mode dL/dp
    vs central finite differences of rasterize(AREA) -> MLEM -> score with the
    tissue values moved too; its first six entries and L are those of the
    6-coefficient gradient at the same tissue values."""
    g, _, S, _ = small_problem(n=32, V=16, counts=2e5, seed=2)
    K = 3
    coef = np.array(synth.C_TRUE) + np.array([0.3, -0.1, 0.15, 0.05, 0.02, -0.03])
    tissue = (0.13, 0.28, 0.75)
    p = np.concatenate([coef, tissue])
    L, grad, FK = oracle.score_grad_params(g, p, S, K)
    L6, grad6, FK6 = oracle.score_grad(g, tissue, coef, S, K)
    assert L == L6 and np.array_equal(grad[:6], grad6) and np.array_equal(FK, FK6)
    fd = np.array([fd_score_params(g, p, S, K, 1e-4, k) for k in range(9)])
    # each group on its own scale: cm for c and dR, cm^-1 for mu_b and mu_c
    for sl in (slice(0, 6), slice(6, 8), slice(8, 9)):
        scale = np.abs(fd[sl]).max()
        assert scale > 0
        np.testing.assert_allclose(grad[sl], fd[sl], rtol=1e-3, atol=1e-3 * scale)


def test_nine_parameter_gradient_identities():
    """With mu_b = mu_c the map is mu_b f(R + dR): moving c_0 (P_0 = 1) and
    moving dR shift the same outer boundary, so dL/dc_0 = dL/ddR exactly as
    long as R > 0 everywhere (a wrong factor or a dropped mu_c in the dR
    term fails this).  A negative dR is taken as 0: same score as dR = 0 and
    no derivative in dR."""
    g, _, S, _ = small_problem(n=32, V=16, counts=2e5, seed=3)
    K = 2
    coef = np.array(synth.C_TRUE) + np.array([0.2, 0.1, -0.1, 0.0, 0.03, 0.0])
    p = np.concatenate([coef, [0.2, 0.2, 0.5]])
    _, grad, _ = oracle.score_grad_params(g, p, S, K)
    assert grad[8] != 0.0
    assert grad[0] == pytest.approx(grad[8], rel=1e-10)
    # dL/dmu_b + dL/dmu_c is the derivative along mu_b = mu_c (one map value)
    def L_at(m):
        q = p.copy(); q[6] = q[7] = m
        mu = oracle.rasterize(g.n, g.dx, m, m, q[8], q[:6], oracle.AREA)
        return oracle.score(g, mu, S, oracle.mlem(g, mu, S, K))
    h = 1e-4
    fd = (L_at(0.2 + h) - L_at(0.2 - h)) / (2 * h)
    assert grad[6] + grad[7] == pytest.approx(fd, rel=1e-5)
    pneg = p.copy(); pneg[8] = -0.3
    pzero = p.copy(); pzero[8] = 0.0
    Ln, gn, _ = oracle.score_grad_params(g, pneg, S, K)
    Lz, gz, _ = oracle.score_grad_params(g, pzero, S, K)
    assert Ln == Lz and gn[8] == 0.0 and gz[8] == 0.0
    np.testing.assert_array_equal(gn[:8], gz[:8])


def test_batch_driver_equals_single_candidate_calls():
    """The threaded batch driver (the reference of every GPU parity test) is
    the single-candidate code run per candidate: bit-identical images and
    scores for any thread count, per-candidate iteration counts, per-candidate
    sinograms, a given F^0 and with or without the ln S! term."""
    g, mu, S, _ = small_problem(n=24, V=12, counts=5e4, seed=7)
    rng = np.random.default_rng(8)
    B = 5
    mus = np.stack([mu * s for s in (1.0, 0.5, 1.5, 0.0, 1.2)])
    Ss = np.stack([S * (1 + b % 2) for b in range(B)])
    iters = np.array([3, 0, 5, 1, 2])
    F0 = rng.uniform(0.5, 1.5, (B, g.n, g.n))
    for nthreads in (1, 3, 8):
        for lg in (True, False):
            F, L, used = oracle.mlem_batch(g, mus, Ss, iters, F0=F0, include_lgamma=lg, nthreads=nthreads)
            assert 1 <= used <= nthreads
            for b in range(B):
                Fb = oracle.mlem(g, mus[b], Ss[b], int(iters[b]), F0[b])
                np.testing.assert_array_equal(F[b], Fb)
                assert L[b] == oracle.score(g, mus[b], Ss[b], Fb, include_lgamma=lg)
    # shared sinogram, F^0 = 1, no score
    F, L, _ = oracle.mlem_batch(g, mus, S, 2, with_score=False, nthreads=2)
    assert L is None
    np.testing.assert_array_equal(F[2], oracle.mlem(g, mus[2], S, 2))
