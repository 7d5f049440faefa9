"""FP64 CPU oracle for the BOAC hot path (arXiv 2109.11920) -- ctypes wrapper.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
and its Python binding never touch it.

The arithmetic lives in ``boac_oracle.c`` (plain C, double precision, every
function citing the paper passage it follows).  This module only compiles it
with gcc and marshals numpy arrays.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms of Eq. 1, Eq. 3 and Eq. 5, adjointness, dense brute force,
MLEM invariants, finite differences).  Agreement with the paper's own images
(Table 1) is *parity unpinned*: the paper's phantoms are not published.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "boac_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CENTER = 0
AREA = 1


def build(force: bool = False) -> str:
    """Compile ``boac_oracle.c`` into ``liboracle.so`` (gcc, no fp contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
           "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.c_int
            Dv = ctypes.c_double
            lib.orc_view_cos_sin.argtypes = [I, I, D]
            lib.orc_legendre.argtypes = [Dv, D]
            lib.orc_rasterize.argtypes = [I, Dv, Dv, Dv, Dv, D, I, D]
            geo = [I, I, I, Dv, Dv]
            lib.orc_attenuation.argtypes = geo + [D, D]
            lib.orc_project.argtypes = geo + [D, D, D]
            lib.orc_backproject.argtypes = geo + [D, D, D]
            lib.orc_mlem.argtypes = geo + [D, D, I, D]
            lib.orc_sensitivity.argtypes = geo + [D, D]
            lib.orc_loglik.argtypes = [I, D, D, I]
            lib.orc_loglik.restype = Dv
            lib.orc_score.argtypes = geo + [D, D, D, I]
            lib.orc_score.restype = Dv
            lib.orc_score_grad.argtypes = geo + [Dv, Dv, Dv, D, D, I, I, D, D]
            lib.orc_score_grad.restype = Dv
            lib.orc_system_matrix.argtypes = geo + [D, D]
            lib.orc_score_grad_params.argtypes = geo + [D, D, I, I, D, D]
            lib.orc_score_grad_params.restype = Dv
            lib.orc_mlem_batch.argtypes = geo + [I, D, D, ctypes.c_longlong,
                                                 ctypes.POINTER(ctypes.c_int), D, D, I, I]
            lib.orc_mlem_batch.restype = I
            _lib = lib
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _arr(x, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


class Geometry:
    """n x n pixels of ``dx`` cm; ``V`` views over 360 deg; ``nb`` bins of ``ds`` cm."""

    def __init__(self, n: int, dx: float, V: int, nb: int | None = None, ds: float | None = None):
        self.n = int(n)
        self.dx = float(dx)
        self.V = int(V)
        self.nb = int(nb if nb is not None else n)
        self.ds = float(ds if ds is not None else dx)

    @property
    def args(self):
        return (self.n, self.nb, self.V, self.dx, self.ds)


def view_cos_sin(v: int, V: int):
    out = np.zeros(2)
    _load().orc_view_cos_sin(v, V, _d(out))
    return out[0], out[1]


def legendre(z: float) -> np.ndarray:
    P = np.zeros(6)
    _load().orc_legendre(float(z), _d(P))
    return P


def rasterize(n, dx, mu_b, mu_c, dR, coef, mode=CENTER) -> np.ndarray:
    """Eq. 3 + Eq. 4 on the n x n grid; returns mu[n, n] (cm^-1)."""
    c = _arr(coef, (6,))
    mu = np.zeros((n, n))
    _load().orc_rasterize(n, dx, mu_b, mu_c, dR, _d(c), int(mode), _d(mu))
    return mu


def attenuation(g: Geometry, mu) -> np.ndarray:
    mu = _arr(mu, (g.n, g.n))
    a = np.zeros((g.V, g.n, g.nb))
    _load().orc_attenuation(*g.args, _d(mu), _d(a))
    return a


def project(g: Geometry, mu, F) -> np.ndarray:
    """q = A^mu F (Eq. 1-2); returns q[V, nb]."""
    mu = _arr(mu, (g.n, g.n))
    F = _arr(F, (g.n, g.n))
    q = np.zeros((g.V, g.nb))
    _load().orc_project(*g.args, _d(mu), _d(F), _d(q))
    return q


def backproject(g: Geometry, mu, y) -> np.ndarray:
    """(A^mu)^T y; returns an n x n image."""
    mu = _arr(mu, (g.n, g.n))
    y = _arr(y, (g.V, g.nb))
    out = np.zeros((g.n, g.n))
    _load().orc_backproject(*g.args, _d(mu), _d(y), _d(out))
    return out


def sensitivity(g: Geometry, mu) -> np.ndarray:
    mu = _arr(mu, (g.n, g.n))
    out = np.zeros((g.n, g.n))
    _load().orc_sensitivity(*g.args, _d(mu), _d(out))
    return out


def mlem(g: Geometry, mu, S, K: int, F0=None) -> np.ndarray:
    """K MLEM iterations from F0 (default: ones); returns F^K."""
    mu = _arr(mu, (g.n, g.n))
    S = _arr(S, (g.V, g.nb))
    F = np.ones((g.n, g.n)) if F0 is None else _arr(F0, (g.n, g.n)).copy()
    _load().orc_mlem(*g.args, _d(mu), _d(S), int(K), _d(F))
    return F


def loglik(S, q, include_lgamma: bool = True) -> float:
    S = _arr(S).ravel()
    q = _arr(q).ravel()
    assert S.size == q.size
    return _load().orc_loglik(S.size, _d(S), _d(q), int(include_lgamma))


def score(g: Geometry, mu, S, F, include_lgamma: bool = True) -> float:
    mu = _arr(mu, (g.n, g.n))
    S = _arr(S, (g.V, g.nb))
    F = _arr(F, (g.n, g.n))
    return _load().orc_score(*g.args, _d(mu), _d(S), _d(F), int(include_lgamma))


def score_grad(g: Geometry, tissue, coef, S, K: int, include_lgamma: bool = True):
    """(L, dL/dc[6], F^K) through K MLEM iterations, AREA rasterisation, F^0 = 1."""
    mu_b, mu_c, dR = (float(t) for t in tissue)
    c = _arr(coef, (6,))
    S = _arr(S, (g.V, g.nb))
    grad = np.zeros(6)
    F = np.zeros((g.n, g.n))
    L = _load().orc_score_grad(*g.args, mu_b, mu_c, dR, _d(c), _d(S), int(K),
                               int(include_lgamma), _d(grad), _d(F))
    return L, grad, F


def system_matrix(g: Geometry, mu) -> np.ndarray:
    """Dense A^mu [V * nb, n * n]: row (v, b), column i * n + j."""
    mu = _arr(mu, (g.n, g.n))
    A = np.zeros((g.V * g.nb, g.n * g.n))
    _load().orc_system_matrix(*g.args, _d(mu), _d(A))
    return A


def score_grad_params(g: Geometry, params, S, K: int, include_lgamma: bool = True):
    """(L, dL/dp[9], F^K) for p = (c_0..c_5, mu_b, mu_c, dR): the same pipeline
    as score_grad with the tissue values as variables (dR < 0 taken as 0)."""
    p = _arr(params, (9,))
    S = _arr(S, (g.V, g.nb))
    grad = np.zeros(9)
    F = np.zeros((g.n, g.n))
    L = _load().orc_score_grad_params(*g.args, _d(p), _d(S), int(K), int(include_lgamma),
                                      _d(grad), _d(F))
    return L, grad, F


def mlem_batch(g: Geometry, mu, S, iters, F0=None, with_score=True,
               include_lgamma=True, nthreads: int | None = None):
    """MLEM (+ score) for B candidates on host threads.  ``S`` is [V,nb]
    (shared) or [B,V,nb].  Returns (F[B,n,n], L[B] or None, threads used)."""
    mu = _arr(mu)
    B = mu.shape[0]
    mu = mu.reshape(B, g.n, g.n)
    S = _arr(S)
    s_stride = 0 if S.ndim == 2 else g.V * g.nb
    iters = np.ascontiguousarray(np.broadcast_to(np.asarray(iters, dtype=np.int32), (B,)))
    F = np.ones((B, g.n, g.n)) if F0 is None else _arr(F0, (B, g.n, g.n)).copy()
    L = np.zeros(B) if with_score else None
    nthreads = nthreads or os.cpu_count() or 1
    used = _load().orc_mlem_batch(*g.args, B, _d(mu), _d(S), s_stride,
                                  iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  _d(F), _d(L) if L is not None else None,
                                  int(include_lgamma), int(nthreads))
    return F, L, used
