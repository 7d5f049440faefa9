"""Device status words of the batched MLEM paths.

1. The fused kernels' bounded hand-over wait, made to run out on purpose.

The work split cuts a candidate between two CTAs (or clusters); the second
part waits for a flag from the first.  boac_test_mlem_handover makes the
first part of one candidate keep that flag to itself, and
boac_set_wait_cycles shortens the wait to about a millisecond, so the wait
gives up: nothing faults or hangs.  Checked: the workspace status word says
BOAC_ETIMEOUT, that candidate's score is NaN, the other candidates are the
same as boac_mlem's, the Python wrapper raises on the status, and the
context stays usable (the next calls succeed)."""
import numpy as np
import pytest
import torch

from paper_2109_11920_gb300 import Geom, _lib
from paper_2109_11920_gb300 import api as boac
from problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu

SHORT_WAIT = 2_000_000  # cycles: about 1 ms at 2 GHz


# (image side, pixel, views, launch configuration): the one-CTA kernel
# (configuration 2: CTAs of 4n threads, four views per grid) and the cluster
# kernel (configuration 6: two CTAs per candidate)
CASES = [(64, 0.4, 60, 2), (64, 0.4, 60, 6), (128, 0.2, 120, 6)]


@pytest.mark.parametrize("n, dx, V, config", CASES)
def test_withheld_handover_times_out_and_reports(cuda, n, dx, V, config):
    p = make_problem(n, dx, V, 2e5, B=3, seed=41)
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    # 3 candidates x 4 iterations on 2 holders: cap = 6 units, so candidate 1
    # (units 4..7) is cut: its first part on holder 0, its second on holder 1
    K, holders = 4, 2
    F_ref, L_ref = boac.boac_mlem(Geom.make(p.n, p.dx, p.V), mu, S, torch.ones(3, n, n, device=cuda), K,
                                  include_lgamma=False)
    old = boac.boac_set_wait_cycles(SHORT_WAIT)
    try:
        # nothing withheld: the short limit is not reached, every score is there
        F, L, st, _ = boac.boac_test_mlem_handover(g, mu, S, K, config, holders, withhold=-1)
        assert st == _lib.BOAC_OK
        assert rel_l2(F.cpu().numpy(), F_ref.cpu().numpy()) < 1e-5
        np.testing.assert_allclose(L.cpu().numpy(), L_ref.cpu().numpy(), rtol=1e-6)
        # candidate 1's flag withheld: its second part gives up
        F, L, st, ws = boac.boac_test_mlem_handover(g, mu, S, K, config, holders, withhold=1)
        assert st == _lib.BOAC_ETIMEOUT
        L, F = L.cpu().numpy(), F.cpu().numpy()
        assert np.isnan(L[1])
        for b in (0, 2):
            assert rel_l2(F[b], F_ref[b].cpu().numpy()) < 1e-5, b
            assert abs(L[b] - L_ref[b].item()) < 1e-6 * abs(L_ref[b].item()), b
        with pytest.raises(_lib.BoacError) as err:
            boac._raise_on_device_status("boac_test_mlem_handover", ws)
        assert err.value.status == _lib.BOAC_ETIMEOUT
    finally:
        assert boac.boac_set_wait_cycles(old) == SHORT_WAIT
    # the context is still usable: a normal call succeeds and checks clean
    F2, L2 = boac.boac_mlem(g, mu, S, torch.ones(3, n, n, device=cuda), K, include_lgamma=False)
    torch.cuda.synchronize()
    np.testing.assert_allclose(L2.cpu().numpy(), L_ref.cpu().numpy(), rtol=1e-12)


def test_wait_limit_setting_round_trips(cuda):
    old = boac.boac_set_wait_cycles(12345)
    try:
        assert boac.boac_set_wait_cycles(0) == 12345   # 0 restores the default
        assert boac.boac_set_wait_cycles(old) == 1 << 32
    finally:
        boac.boac_set_wait_cycles(old)


def test_handover_hook_rejects_bad_arguments(cuda):
    g = Geom.make(64, 0.4, 60)
    assert _lib.load().boac_test_mlem_handover_bytes(g, 3, 4, 2, 4) == 0   # more holders than candidates
    assert _lib.load().boac_test_mlem_handover_bytes(g, 3, 4, 99, 2) == 0  # no such configuration
    assert _lib.load().boac_test_mlem_handover_bytes(g, 3, 4, 2, 2) > 0


@pytest.mark.parametrize("path", ["default", "fused", "cluster"])
def test_minus_inf_score_is_reported_per_candidate(cuda, path):
    """Candidate 1 starts from F = 0: MLEM keeps it at 0 (r = 0 where q = 0),
    so q = 0 on every bin and its score is -inf; the others are finite."""
    p = make_problem(64, 0.4, 60, 2e5, B=3, seed=43)
    g = Geom.make(p.n, p.dx, p.V)
    mu = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    for zero in (False, True):
        F0 = torch.ones(3, 64, 64, device=cuda)
        if zero:
            F0[1] = 0.0
        if path == "default":  # boac_mlem's choice at this batch size: the unfused kernels
            ws = boac.workspace(g, 3, _lib.OP_MLEM, cuda)
            _, L = boac.boac_mlem(g, mu, S, F0, 3, ws=ws)
            st = boac.boac_workspace_status(ws)
        else:
            batch = boac.RaggedBatch([g], [0] * 3, [3] * 3, list(mu), [S] * 3, F0=list(F0), device=cuda)
            L = boac.boac_mlem_ragged(batch, config=[2 if path == "fused" else 6])
            st = batch.status()
        L = L.cpu().numpy()
        if zero:
            assert st == _lib.BOAC_ENONFINITE
            assert L[1] == -np.inf and np.isfinite(L[[0, 2]]).all()
        else:
            assert st == _lib.BOAC_OK and np.isfinite(L).all()
