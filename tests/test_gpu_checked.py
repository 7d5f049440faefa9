"""The bounds-checked build, libboac_checked.so (built here on demand with
-DBOAC_CHECKED).  It runs boac_mlem's small-batch path (the unfused grouped
kernels), the fused one-CTA kernel and its cluster mode, and the score
gradient (the fused gradient kernel and the batched reverse mode) on small
cases through the C ABI, and the 256 x 256 band kernel: every checked
shared-memory index and schedule
entry is in range (fault count 0, summed over every translation unit), and
the results equal the normal build's bit for bit (the checks change no
arithmetic)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2109_11920_gb300 import Geom, Tissue, _lib
from paper_2109_11920_gb300 import api as boac
from problems import make_problem

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def run_all(lib, p, dev, K):
    """(F, L) of boac_mlem (3 candidates: the unfused kernels) and of the
    ragged entry point with configurations 4 (one CTA of 8n threads per
    candidate) and 13 (clusters of 8 CTAs), through `lib`."""
    g = Geom.make(p.n, p.dx, p.V)
    B = p.mu.shape[0]
    mu = torch.tensor(p.mu, dtype=torch.float32, device=dev)
    S = torch.tensor(p.S, dtype=torch.float32, device=dev)
    out = []
    F = torch.ones(B, p.n, p.n, device=dev)
    L = torch.empty(B, dtype=torch.float64, device=dev)
    ws = boac.workspace(g, B, _lib.OP_MLEM, dev)
    st = lib.boac_mlem(ctypes.byref(g), _p(mu), _p(S), 0, _p(F), K, B, _p(L), 1, _p(ws), ws.numel(), _stream())
    assert st == _lib.BOAC_OK, _lib.status_string(st)
    out.append((F.cpu().numpy(), L.cpu().numpy()))
    for cfg in (4, 13):
        batch = boac.RaggedBatch([g], [0] * B, [K] * B, list(mu), [S] * B, device=dev)
        c = (ctypes.c_int * 1)(cfg)
        nbytes = lib.boac_mlem_ragged_workspace_bytes(batch.geo, 1, batch.cands, B, c)
        assert nbytes > 0
        wsr = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        st = lib.boac_mlem_ragged(batch.geo, 1, batch.cands, B, _p(batch.mu_pool), _p(batch.S_pool),
                                  _p(batch.F_pool), _p(batch.L), 1, c, _p(wsr), nbytes, _stream())
        assert st == _lib.BOAC_OK, _lib.status_string(st)
        out.append((batch.F_pool.view(B, p.n, p.n).cpu().numpy(), batch.L.cpu().numpy()))
    torch.cuda.synchronize()
    return out


def test_checked_build_runs_clean_and_matches(cuda):
    from paper_2109_11920_gb300 import build
    build.build()
    build.build(checked=True)
    norm, chk = _lib.load(), _lib.load_checked()
    faults = ctypes.c_int(-1)
    assert norm.boac_bounds_faults(ctypes.byref(faults), 0) == _lib.BOAC_EUNSUPPORTED
    assert chk.boac_bounds_faults(ctypes.byref(faults), 1) == _lib.BOAC_OK
    p = make_problem(128, 0.2, 120, 2e5, B=3, seed=29)
    ref = run_all(norm, p, cuda, 4)
    got = run_all(chk, p, cuda, 4)
    assert chk.boac_bounds_faults(ctypes.byref(faults), 0) == _lib.BOAC_OK
    assert faults.value == 0
    for (Fr, Lr), (Fc, Lc) in zip(ref, got):
        np.testing.assert_array_equal(Fc, Fr)
        np.testing.assert_array_equal(Lc, Lr)


def run_grad(lib, p, dev, K, ckpt):
    """(L, dL/dc) of boac_score_grad (the fused gradient kernel) and of
    boac_score_grad_unfused (the batched reverse mode), through `lib`."""
    g = Geom.make(p.n, p.dx, p.V)
    B = p.coefs.shape[0]
    t = Tissue(*p.tissue)
    c = torch.tensor(p.coefs, dtype=torch.float32, device=dev)
    S = torch.tensor(p.S, dtype=torch.float32, device=dev)
    nbytes = lib.boac_score_grad_workspace_bytes(ctypes.byref(g), B, K, ckpt)
    assert nbytes > 0
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = []
    for fn in (lib.boac_score_grad, lib.boac_score_grad_unfused):
        L = torch.empty(B, dtype=torch.float64, device=dev)
        G = torch.empty(B, 6, dtype=torch.float64, device=dev)
        st = fn(ctypes.byref(g), ctypes.byref(t), _p(c), _p(S), 0, K, ckpt, B, 1, _p(L), _p(G), None,
                _p(ws), nbytes, _stream())
        assert st == _lib.BOAC_OK, _lib.status_string(st)
        out.append((L.cpu().numpy(), G.cpu().numpy()))
    torch.cuda.synchronize()
    return out


def test_checked_build_gradient(cuda):
    from paper_2109_11920_gb300 import build
    build.build()
    build.build(checked=True)
    norm, chk = _lib.load(), _lib.load_checked()
    faults = ctypes.c_int(-1)
    assert chk.boac_bounds_faults(ctypes.byref(faults), 1) == _lib.BOAC_OK
    for n, dx, V in ((128, 0.2, 120), (96, 25.6 / 96, 92)):
        p = make_problem(n, dx, V, 2e5, B=3, seed=31, mode=oracle.AREA)
        ref = run_grad(norm, p, cuda, 3, 2)
        got = run_grad(chk, p, cuda, 3, 2)
        for (Lr, Gr), (Lc, Gc) in zip(ref, got):
            np.testing.assert_array_equal(Lc, Lr)
            np.testing.assert_array_equal(Gc, Gr)
    assert chk.boac_bounds_faults(ctypes.byref(faults), 0) == _lib.BOAC_OK
    assert faults.value == 0


def run_band(lib, p, dev, K, cfg=6):
    """Images and scores of the band kernel (clusters of 5 CTAs at 256 x 256)
    through the ragged entry point of `lib`."""
    g = Geom.make(p.n, p.dx, p.V)
    B = p.mu.shape[0]
    mu = torch.tensor(p.mu, dtype=torch.float32, device=dev)
    S = torch.tensor(p.S, dtype=torch.float32, device=dev)
    batch = boac.RaggedBatch([g], [0] * B, [K] * B, list(mu), [S] * B, device=dev)
    c = (ctypes.c_int * 1)(cfg)
    nbytes = lib.boac_mlem_ragged_workspace_bytes(batch.geo, 1, batch.cands, B, c)
    assert nbytes > 0
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    st = lib.boac_mlem_ragged(batch.geo, 1, batch.cands, B, _p(batch.mu_pool), _p(batch.S_pool),
                              _p(batch.F_pool), _p(batch.L), 1, c, _p(ws), nbytes, _stream())
    assert st == _lib.BOAC_OK, _lib.status_string(st)
    torch.cuda.synchronize()
    return batch.F_pool.view(B, p.n, p.n).cpu().numpy(), batch.L.cpu().numpy()


def test_checked_build_band_kernel(cuda):
    from paper_2109_11920_gb300 import build
    build.build()
    build.build(checked=True)
    norm, chk = _lib.load(), _lib.load_checked()
    faults = ctypes.c_int(-1)
    assert chk.boac_bounds_faults(ctypes.byref(faults), 1) == _lib.BOAC_OK
    p = make_problem(256, 0.1, 180, 1e6, B=2, seed=37)
    Fr, Lr = run_band(norm, p, cuda, 2)
    Fc, Lc = run_band(chk, p, cuda, 2)
    assert chk.boac_bounds_faults(ctypes.byref(faults), 0) == _lib.BOAC_OK
    assert faults.value == 0
    np.testing.assert_array_equal(Fc, Fr)
    np.testing.assert_array_equal(Lc, Lr)
