"""The ln S! term of Eq. 5 on every MLEM path.  With one shared sinogram it
is summed once per call (a separate pair of kernels) and subtracted from
every candidate's score; with per-candidate sinograms it stays a term per
bin.  Either way L(with) - L(without) = -sum_i ln Gamma(S_i + 1), checked
against scipy; plus the unfused batched path on image sizes that have no
grouped kernels."""
import numpy as np
import pytest
import torch
from scipy.special import gammaln

import oracle
from paper_2109_11920_gb300 import Geom, Tissue
from paper_2109_11920_gb300 import api as boac
from problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu


def lnfact(S):
    return float(gammaln(np.asarray(S, dtype=np.float64) + 1.0).sum())


def check(L_with, L_without, expected):
    d = (L_with - L_without).cpu().numpy()
    np.testing.assert_allclose(d, -np.asarray(expected), rtol=1e-12, atol=1e-9)


# boac_mlem at 128 x 128 runs 100 candidates on the one-CTA fused kernel, 40 on
# clusters of 4 CTAs and 3 on the unfused kernels; "fused" pins the one-CTA
# kernel through the ragged entry point, whose scores keep the per-bin term.
@pytest.mark.parametrize("path,B", [("default", 100), ("default", 40), ("default", 3), ("unfused", 5), ("fused", 4)])
def test_shared_and_per_candidate_sinograms(cuda, path, B):
    p = make_problem(128, 0.2, 120, 1e6, B=B, seed=91)
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    S_per = torch.stack([S * (1 + (b % 3)) for b in range(B)]).contiguous()
    for sino, exp in ((S, [lnfact(p.S)] * B), (S_per, [lnfact(p.S * (1 + (b % 3))) for b in range(B)])):
        out = []
        for lg in (True, False):
            if path == "fused":
                batch = boac.RaggedBatch([g], [0] * B, [3] * B, list(mu),
                                         list(sino) if sino.dim() == 3 else [sino] * B, device=cuda)
                out.append(boac.boac_mlem_ragged(batch, include_lgamma=lg, config=[4]))
            else:
                _, L = boac.boac_mlem(g, mu, sino, torch.ones(B, 128, 128, device=cuda), 3,
                                      include_lgamma=lg, unfused=path == "unfused")
                out.append(L)
        check(out[0], out[1], exp)


def test_cluster_gradient_and_explicit_matrix_paths(cuda):
    # 256 x 256 on clusters (B = 3 > the unfused bound)
    p = make_problem(256, 0.1, 16, 2e5, B=3, seed=92)
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    Ls = [boac.boac_mlem(g, mu, S, torch.ones(3, 256, 256, device=cuda), 2, include_lgamma=lg)[1] for lg in (True, False)]
    check(Ls[0], Ls[1], [lnfact(p.S)] * 3)
    # the score gradient and the explicit matrix at 64 x 64
    p = make_problem(64, 0.4, 60, 2e5, B=3, seed=93, mode=oracle.AREA)
    g, t = Geom.make(p.n, p.dx, p.V), Tissue(*p.tissue)
    c = torch.tensor(p.coefs, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    Lg = [boac.boac_score_grad(g, t, c, S, 2, 1, include_lgamma=lg)[0] for lg in (True, False)]
    check(Lg[0], Lg[1], [lnfact(p.S)] * 3)
    m = boac.SysMat(g, cuda)
    vals = m.values(torch.tensor(p.mu, dtype=torch.float32, device=cuda))
    Lm = [m.mlem(vals, S, torch.ones(3, 64, 64, device=cuda), 2, include_lgamma=lg)[1] for lg in (True, False)]
    check(Lm[0], Lm[1], [lnfact(p.S)] * 3)


@pytest.mark.parametrize("n,dx,V", [(33, 0.7, 8), (20, 1.1, 4), (33, 0.7, 7)])
def test_unfused_path_without_grouped_kernels(cuda, n, dx, V):
    """Image sizes the grouped projector and back-projection do not cover
    (the per-ray projector and the per-pixel gather run instead), and an odd
    view count, through boac_mlem_unfused, against the oracle."""
    p = make_problem(n, dx, V, 5e4, B=3, seed=94)
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    F, L = boac.boac_mlem(g, mu, S, torch.ones(3, n, n, device=cuda), 6, unfused=True)
    Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu, p.S, 6)
    for b in range(3):
        assert rel_l2(F[b].cpu().numpy(), Fo[b]) < 1e-4, b
        assert abs(float(L[b]) - Lo[b]) < 1e-6 * abs(Lo[b]), b
