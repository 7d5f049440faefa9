"""boac_mlem_noalloc -- MLEM for callers that cannot allocate device memory
(for example code running under another framework's allocator or in a
callback where cudaMalloc is not allowed).  It takes its scratch from an
array built into the library instead of a caller workspace.

Called here through the raw C ABI (ctypes, device pointers) and checked
against boac_mlem, the workspace-taking entry point, and against the FP64
oracle on sampled candidates, on two calls in a row with different inputs,
so that leftovers of the first call in the shared scratch would show up in
the second.  This file is named to be collected
last; it passes on its own in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2109_11920_gb300 import Geom, _lib
from paper_2109_11920_gb300 import api as boac
from problems import make_problem, rel_l2

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def call_noalloc(lib, g, mu, S, F, K, L):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.boac_mlem_noalloc(ctypes.byref(g), _p(mu), _p(S), 0, _p(F), K, mu.shape[0], _p(L), 1, stream)


def test_noalloc_matches_workspace_entry_point(cuda):
    from paper_2109_11920_gb300 import build
    build.build()
    lib = _lib.load()
    # 128 x 128, 120 views: one CTA slot's scratch is at least its
    # attenuation exponents, V/2 (n^2 + n) floats, and its sensitivity image,
    # n^2 floats (about 4.0 MB), so the 64 MiB array holds at most 16 slots.
    # 20 candidates are more than that: the work split then cuts candidates
    # between two CTAs (the hand-over path) and slots are reused in a call.
    n, V = 128, 120
    slot_bytes = 4 * ((V // 2) * (n * n + n) + n * n)
    assert (64 << 20) // slot_bytes == 16
    p = make_problem(n, 0.2, V, 1e6, B=20, seed=5)
    g = Geom.make(p.n, p.dx, p.V)
    mu_all = torch.tensor(p.mu, dtype=torch.float32, device=cuda)
    S = torch.tensor(p.S, dtype=torch.float32, device=cuda)
    for call, (order, K) in enumerate([(np.arange(20), 4), (np.arange(20)[::-1].copy(), 3)]):
        mu = mu_all[torch.as_tensor(order, device=cuda)].contiguous()
        F_ref = torch.ones(20, p.n, p.n, device=cuda)
        F_ref, L_ref = boac.boac_mlem(g, mu, S, F_ref, K)
        F = torch.ones(20, p.n, p.n, device=cuda)
        L = torch.empty(20, dtype=torch.float64, device=cuda)
        st = call_noalloc(lib, g, mu, S, F, K, L)
        assert st == _lib.BOAC_OK, _lib.status_string(st)
        torch.cuda.synchronize()
        # boac_mlem may run these 20 candidates on clusters of CTAs (small
        # batch), the no-alloc entry point one CTA per candidate: the same
        # arithmetic summed in another order
        assert rel_l2(F.cpu().numpy(), F_ref.cpu().numpy()) < 1e-5, call
        np.testing.assert_allclose(L.cpu().numpy(), L_ref.cpu().numpy(), rtol=1e-6)
        # and against the FP64 oracle on two sampled candidates (images 1e-4,
        # scores 1e-6 relative, as for boac_mlem)
        for b in (0, 13):
            Fo, Lo, _ = oracle.mlem_batch(p.geom, p.mu[order[b]][None], p.S, K)
            assert rel_l2(F[b].cpu().numpy(), Fo[0]) < 1e-4, (call, b)
            assert abs(L[b].item() - Lo[0]) < 1e-6 * abs(Lo[0]), (call, b)
    # arguments are still checked on the host
    F = torch.ones(20, p.n, p.n, device=cuda)
    L = torch.empty(20, dtype=torch.float64, device=cuda)
    bad = Geom.make(p.n, p.dx, 119)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.boac_mlem_noalloc(ctypes.byref(bad), _p(mu_all), _p(S), 0, _p(F), 2, 20, _p(L), 1,
                                 stream) == _lib.BOAC_EINVAL
    # L is required: a timed-out hand-over shows only as a NaN score here
    assert lib.boac_mlem_noalloc(ctypes.byref(g), _p(mu_all), _p(S), 0, _p(F), 2, 20, None, 1,
                                 stream) == _lib.BOAC_EINVAL


def test_noalloc_rejects_problems_beyond_its_scratch(cuda):
    """At 256 x 256 with 720 views one candidate's scratch (about 95 MB) does
    not fit the built-in 64 MiB: the call fails with BOAC_EWORKSPACE before
    launching anything."""
    lib = _lib.load()
    g = Geom.make(256, 0.1, 720)
    mu = torch.zeros(1, 256, 256, device=cuda)
    S = torch.zeros(720, 256, device=cuda)
    F = torch.ones(1, 256, 256, device=cuda)
    L = torch.empty(1, dtype=torch.float64, device=cuda)
    assert call_noalloc(lib, g, mu, S, F, 2, L) == _lib.BOAC_EWORKSPACE
    assert torch.equal(F, torch.ones_like(F))
