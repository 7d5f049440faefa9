"""The system matrix written out (boac_sysmat_*): its CSR pattern and values
against the FP64 oracle's dense A^mu entry by entry, its transposed copy
against A itself, and MLEM on it against the oracle and the matrix-free
fused path (image tolerance 1e-4 relative L2 against the oracle as for the
fused path, score 1e-6 relative)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2109_11920_gb300 import Geom, synth
from paper_2109_11920_gb300 import api as boac
from problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu


def dense_of(m, vals_b):
    """Dense A and A^T of one candidate from the exported pattern."""
    row_ptr, col, colT_ptr, rowT = (t.cpu().numpy() for t in m.pattern())
    v = vals_b.cpu().numpy()
    R, nn = m.rows, m.g.n * m.g.n
    rows = np.repeat(np.arange(R), np.diff(row_ptr))
    A = np.zeros((R, nn), dtype=np.float32)
    A[rows, col] = v[0]
    cols = np.repeat(np.arange(nn), np.diff(colT_ptr))
    AT = np.zeros((nn, R), dtype=np.float32)
    AT[cols, rowT] = v[1]
    return A, AT, row_ptr, col, colT_ptr, rowT


@pytest.mark.parametrize("n,dx,V", [(32, 0.8, 16), (48, 25.6 / 48, 30), (64, 0.4, 60)])
def test_pattern_and_values_against_the_oracle(cuda, n, dx, V):
    p = make_problem(n, dx, V, 1e5, B=3, seed=81, mode=oracle.AREA)
    g = Geom.make(p.n, p.dx, p.V)
    m = boac.SysMat(g, cuda)
    vals = m.values(torch.tensor(p.mu, dtype=torch.float32, device=cuda))
    for b in range(3):
        A, AT, row_ptr, col, colT_ptr, rowT = dense_of(m, boac.SysMat.candidate_values(vals, b))
        Ao = oracle.system_matrix(p.geom, p.mu[b])
        # the library takes sample coordinates in float32: each of the <= 4
        # roundings behind u and w is at most 1.5 n 2^-24, a bilinear weight
        # moves by at most |du| + |dw|, and an entry sums <= 3 weighted samples
        e_w = 2 * 4 * 1.5 * n * 2.0 ** -24
        np.testing.assert_allclose(A, Ao, rtol=1e-5, atol=3 * p.dx * e_w)
        # the pattern holds every nonzero of A^mu, and the transposed copy
        # carries exactly the same values
        assert np.all(A[Ao > 0] > 0)
        np.testing.assert_array_equal(AT, A.T)
    assert row_ptr[0] == 0 and row_ptr[-1] == m.nnz and np.all(np.diff(row_ptr) <= 4 * n)
    for r in range(0, m.rows, 7):
        seg = col[row_ptr[r]:row_ptr[r + 1]]
        assert np.all(np.diff(seg) > 0)
    for pix in range(0, n * n, 5):
        seg = rowT[colT_ptr[pix]:colT_ptr[pix + 1]]
        assert np.all(np.diff(seg) > 0)


def test_project_equals_the_matrix_free_projector(cuda):
    p = make_problem(96, 25.6 / 96, 90, 1e5, B=4, seed=82)
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    F = torch.rand(4, 96, 96, device=cuda, generator=torch.Generator(device=cuda).manual_seed(3))
    m = boac.SysMat(g, cuda)
    q = m.project(m.values(mu), F)
    q_ref = boac.boac_project(g, mu, F)
    for b in range(4):
        assert rel_l2(q[b].cpu().numpy(), q_ref[b].cpu().numpy()) < 2e-6


def test_mlem_against_the_oracle_and_the_fused_path(cuda):
    p = make_problem(64, 0.4, 60, 2e5, B=11, seed=83)  # 11: a partial group of candidates
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    K = 6
    m = boac.SysMat(g, cuda)
    vals = m.values(mu)
    F, L = m.mlem(vals, S, torch.ones(11, 64, 64, device=cuda), K)
    F2, L2 = m.mlem(vals, S, torch.ones(11, 64, 64, device=cuda), K)
    assert torch.equal(F, F2) and torch.equal(L, L2)
    Ff, Lf = boac.boac_mlem(g, mu, S, torch.ones(11, 64, 64, device=cuda), K)
    for b in range(11):
        assert rel_l2(F[b].cpu().numpy(), Ff[b].cpu().numpy()) < 1e-5, b
    np.testing.assert_allclose(L.cpu().numpy(), Lf.cpu().numpy(), rtol=1e-6)
    picks = [0, 7, 10]
    Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu[picks], p.S, K)
    for i, b in enumerate(picks):
        assert rel_l2(F[b].cpu().numpy(), Fo[i]) < 1e-4, b
        assert abs(float(L[b]) - Lo[i]) < 1e-6 * abs(Lo[i]), b


def test_zero_iterations_and_per_candidate_sinograms(cuda):
    p = make_problem(64, 0.4, 60, 2e5, B=2, seed=84)
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    m = boac.SysMat(g, cuda)
    vals = m.values(mu)
    S2 = torch.tensor(np.stack([p.S, 2.0 * p.S]), dtype=torch.float32, device=cuda)
    F0 = torch.full((2, 64, 64), 0.7, device=cuda)
    F, L = m.mlem(vals, S2, F0.clone(), 0)
    assert torch.equal(F, F0)
    Ls = boac.boac_score(g, mu, S2, F0)
    np.testing.assert_allclose(L.cpu().numpy(), Ls.cpu().numpy(), rtol=1e-6)
    F, _ = m.mlem(vals, S2, torch.ones(2, 64, 64, device=cuda), 3)
    Fo = oracle.mlem(p.geom, p.mu[1], 2.0 * p.S, 3)
    assert rel_l2(F[1].cpu().numpy(), Fo) < 1e-4


def test_full_size_batched_workload_sampled(cuda):
    """The batched workload (256 candidates, 128^2, 120 views, K = 50)
    through the explicit matrix: every candidate against the fused path, two
    against the oracle."""
    wl = synth.BATCHED
    p = make_problem(wl.n, wl.dx, wl.V, wl.counts, B=wl.B, seed=wl.seed)
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    m = boac.SysMat(g, cuda)
    F, L = m.mlem(m.values(mu), S, torch.ones(wl.B, 128, 128, device=cuda), wl.K)
    Ff, Lf = boac.boac_mlem(g, mu, S, torch.ones(wl.B, 128, 128, device=cuda), wl.K)
    d = (F - Ff).flatten(1).norm(dim=1) / Ff.flatten(1).norm(dim=1)
    assert float(d.max()) < 1e-4
    np.testing.assert_allclose(L.cpu().numpy(), Lf.cpu().numpy(), rtol=1e-6)
    picks = [0, wl.B - 1]
    Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu[picks], p.S, wl.K)
    for i, b in enumerate(picks):
        assert rel_l2(F[b].cpu().numpy(), Fo[i]) < 1e-4
        assert abs(float(L[b]) - Lo[i]) < 1e-6 * abs(Lo[i])


@pytest.mark.parametrize("n,dx,V", [(256, 0.1, 180), (256, 0.1, 720)])
def test_largest_geometries(cuda, n, dx, V):
    """256 x 256 with 180 and 720 views (the longest pixel segments of A^T):
    the pattern builds, and two MLEM iterations agree with the fused path."""
    p = make_problem(n, dx, V, 1e6, B=2, seed=85)
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    m = boac.SysMat(g, cuda)
    assert 1.5 * n * m.rows < m.nnz < 2.5 * n * m.rows
    F, L = m.mlem(m.values(mu), S, torch.ones(2, n, n, device=cuda), 2)
    Ff, Lf = boac.boac_mlem(g, mu, S, torch.ones(2, n, n, device=cuda), 2)
    for b in range(2):
        assert rel_l2(F[b].cpu().numpy(), Ff[b].cpu().numpy()) < 1e-5
    np.testing.assert_allclose(L.cpu().numpy(), Lf.cpu().numpy(), rtol=1e-6)
