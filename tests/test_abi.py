"""The C-ABI library loads, exports every symbol include/boac.h declares, and
rejects bad arguments on the host before touching the GPU (runs on CPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2109_11920_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "boac.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(boac_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "boac_mlem" in names and "boac_project" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2109_11920_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_status_strings(lib):
    from paper_2109_11920_gb300 import _lib
    assert _lib.status_string(0) == "ok"
    assert "invalid" in _lib.status_string(_lib.BOAC_EINVAL)
    assert "workspace" in _lib.status_string(_lib.BOAC_EWORKSPACE)
    assert "-inf" in _lib.status_string(_lib.BOAC_ENONFINITE)
    assert "wait" in _lib.status_string(_lib.BOAC_ETIMEOUT)
    assert lib.boac_abi_version() >= 1


def test_host_side_argument_checks(lib):
    """Invalid geometry, null pointers and bad sizes fail with BOAC_EINVAL
    before any CUDA call (safe without a GPU)."""
    from paper_2109_11920_gb300 import _lib
    G = _lib.Geom
    good = G.make(64, 0.4, 60)
    bad = [G(4, 4, 60, 0.4, 0.4), G(64, 32, 60, 0.4, 0.4), G(64, 64, 60, 0.4, 0.2),
           G(64, 64, 0, 0.4, 0.4), G(64, 64, 60, -1.0, -1.0), G(512, 512, 60, 0.1, 0.1)]
    t = _lib.Tissue(0.15, 0.25, 0.6)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: checks fail first
    for g in bad:
        assert lib.boac_rasterize_mu(ctypes.byref(g), ctypes.byref(t), fake, 1, 0, fake, None) == _lib.BOAC_EINVAL
        assert lib.boac_project(ctypes.byref(g), fake, fake, 1, fake, None) == _lib.BOAC_EINVAL
        assert lib.boac_workspace_bytes(ctypes.byref(g), 1, _lib.OP_MLEM) == 0
    assert lib.boac_rasterize_mu(ctypes.byref(good), ctypes.byref(t), None, 1, 0, fake, None) == _lib.BOAC_EINVAL
    assert lib.boac_rasterize_mu(ctypes.byref(good), ctypes.byref(t), fake, 0, 0, fake, None) == _lib.BOAC_EINVAL
    assert lib.boac_rasterize_mu(ctypes.byref(good), ctypes.byref(t), fake, 1, 7, fake, None) == _lib.BOAC_EINVAL
    assert lib.boac_project(ctypes.byref(good), fake, None, 1, fake, None) == _lib.BOAC_EINVAL
    assert lib.boac_mlem(ctypes.byref(good), fake, fake, -1, fake, 5, 1, None, 1, fake, 1 << 20, None) == _lib.BOAC_EINVAL
    assert lib.boac_mlem(ctypes.byref(good), fake, fake, 0, fake, -1, 1, None, 1, fake, 1 << 20, None) == _lib.BOAC_EINVAL
    odd = G.make(64, 0.4, 59)
    assert lib.boac_mlem(ctypes.byref(odd), fake, fake, 0, fake, 5, 1, None, 1, fake, 1 << 20, None) == _lib.BOAC_EINVAL
    assert lib.boac_mlem_plain(ctypes.byref(good), fake, fake, 0, fake, 5, 1, None, 1, None, 0, None) == _lib.BOAC_EWORKSPACE
    assert lib.boac_score(ctypes.byref(good), fake, fake, 0, fake, 1, 1, fake, None, 0, None) == _lib.BOAC_EWORKSPACE
    assert lib.boac_backproject(ctypes.byref(good), fake, None, 1, fake, None, 0, None) == _lib.BOAC_EWORKSPACE
    assert lib.boac_workspace_bytes(ctypes.byref(good), 1, _lib.OP_PROJECT) == 0
    # per candidate: its attenuation table (60 views) and 15 per-grid partial images
    assert lib.boac_workspace_bytes(ctypes.byref(good), 3, _lib.OP_BACKPROJECT) == 512 + 3 * (60 + 15) * 64 * 64 * 4


def test_sysmat_host_side_checks(lib):
    """The explicit-matrix entry points reject null handles and bad
    geometries before any CUDA call."""
    from paper_2109_11920_gb300 import _lib
    G = _lib.Geom
    fake = ctypes.c_void_p(0x1000)
    h = ctypes.c_void_p()
    assert lib.boac_sysmat_create(ctypes.byref(G(4, 4, 60, 0.4, 0.4)), ctypes.byref(h), None) == _lib.BOAC_EINVAL
    assert h.value is None
    assert lib.boac_sysmat_create(ctypes.byref(G.make(64, 0.4, 60)), None, None) == _lib.BOAC_EINVAL
    assert lib.boac_sysmat_nnz(None) == -1
    assert lib.boac_sysmat_destroy(None) == _lib.BOAC_EINVAL
    assert lib.boac_sysmat_mlem_workspace_bytes(None, 4) == 0
    assert lib.boac_sysmat_values(None, fake, 1, fake, None) == _lib.BOAC_EINVAL
    assert lib.boac_sysmat_project(None, fake, fake, 1, fake, None) == _lib.BOAC_EINVAL
    assert lib.boac_sysmat_pattern(None, fake, fake, fake, fake, None) == _lib.BOAC_EINVAL
    assert lib.boac_sysmat_mlem(None, fake, fake, 0, fake, 5, 1, None, 1, fake, 1 << 20, None) == _lib.BOAC_EINVAL
