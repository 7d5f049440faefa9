"""Torch-facing wrappers of the C ABI, one per entry point, same names.

Each function checks that its tensors are contiguous CUDA tensors of the
right dtype and shape, allocates outputs and the workspace the library asks
for with torch, and calls the C entry point on the current stream.  Nothing
here computes any part of the method.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import Geom, RaggedCand, Tissue, check


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _need(t: torch.Tensor, name: str, dtype, shape=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def _sino(S: torch.Tensor, g: Geom, B: int):
    """Shared [V, nb] or per-candidate [B, V, nb] sinogram -> (tensor, stride)."""
    _need(S, "S", torch.float32)
    if tuple(S.shape) == (g.n_views, g.n_bins):
        return S, 0
    if tuple(S.shape) == (B, g.n_views, g.n_bins):
        return S, g.n_views * g.n_bins
    raise ValueError(f"S must be [{g.n_views}, {g.n_bins}] or [{B}, {g.n_views}, {g.n_bins}]")


def boac_workspace_bytes(g: Geom, B: int, op: int) -> int:
    return int(_lib.load().boac_workspace_bytes(ctypes.byref(g), int(B), int(op)))


def workspace(g: Geom, B: int, op: int, device) -> torch.Tensor | None:
    nbytes = boac_workspace_bytes(g, B, op)
    if nbytes == 0:
        return None
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def boac_workspace_status(ws: torch.Tensor) -> int:
    """Device status word of a boac_mlem / ragged workspace (synchronous)."""
    st = ctypes.c_int(0)
    check("boac_workspace_status", _lib.load().boac_workspace_status(_ptr(ws), ws.numel(), ctypes.byref(st)))
    return int(st.value)


def boac_rasterize_mu(g: Geom, t: Tissue, c: torch.Tensor, mode: int = _lib.RASTER_CENTER,
                      out: torch.Tensor | None = None) -> torch.Tensor:
    """Eq. 3-4: mu[B, n, n] (cm^-1) from Legendre coefficients c[B, 6] (cm)."""
    _need(c, "c", torch.float32)
    if c.dim() != 2 or c.shape[1] != 6:
        raise ValueError("c must be [B, 6]")
    B = c.shape[0]
    mu = out if out is not None else torch.empty(B, g.n, g.n, dtype=torch.float32, device=c.device)
    _need(mu, "mu", torch.float32, (B, g.n, g.n))
    check("boac_rasterize_mu", _lib.load().boac_rasterize_mu(
        ctypes.byref(g), ctypes.byref(t), _ptr(c), B, int(mode), _ptr(mu), _stream(c.device)))
    return mu


def boac_rasterize_mu_params(g: Geom, p: torch.Tensor, mode: int = _lib.RASTER_CENTER,
                             out: torch.Tensor | None = None) -> torch.Tensor:
    """Eq. 3-4 with per-candidate tissue values: mu[B, n, n] (cm^-1) from
    p[B, 9] = (c_0..c_5 in cm, mu_b, mu_c in cm^-1, dR in cm)."""
    _need(p, "p", torch.float32)
    if p.dim() != 2 or p.shape[1] != 9:
        raise ValueError("p must be [B, 9]")
    B = p.shape[0]
    mu = out if out is not None else torch.empty(B, g.n, g.n, dtype=torch.float32, device=p.device)
    _need(mu, "mu", torch.float32, (B, g.n, g.n))
    check("boac_rasterize_mu_params", _lib.load().boac_rasterize_mu_params(
        ctypes.byref(g), _ptr(p), B, int(mode), _ptr(mu), _stream(p.device)))
    return mu


def boac_project(g: Geom, mu: torch.Tensor, F: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """Eq. 1-2: q[B, V, nb] = A^mu F."""
    _need(mu, "mu", torch.float32)
    B = mu.shape[0]
    _need(mu, "mu", torch.float32, (B, g.n, g.n))
    _need(F, "F", torch.float32, (B, g.n, g.n))
    q = out if out is not None else torch.empty(B, g.n_views, g.n_bins, dtype=torch.float32, device=mu.device)
    _need(q, "q", torch.float32, (B, g.n_views, g.n_bins))
    check("boac_project", _lib.load().boac_project(
        ctypes.byref(g), _ptr(mu), _ptr(F), B, _ptr(q), _stream(mu.device)))
    return q


def boac_backproject(g: Geom, mu: torch.Tensor, y: torch.Tensor | None,
                     out: torch.Tensor | None = None, ws: torch.Tensor | None = None) -> torch.Tensor:
    """Adjoint of Eq. 2: out[B, n, n] = (A^mu)^T y (y=None: the sensitivity A^T 1)."""
    _need(mu, "mu", torch.float32)
    B = mu.shape[0]
    _need(mu, "mu", torch.float32, (B, g.n, g.n))
    if y is not None:
        _need(y, "y", torch.float32, (B, g.n_views, g.n_bins))
    res = out if out is not None else torch.empty(B, g.n, g.n, dtype=torch.float32, device=mu.device)
    _need(res, "out", torch.float32, (B, g.n, g.n))
    if ws is None:
        ws = workspace(g, B, _lib.OP_BACKPROJECT, mu.device)
    check("boac_backproject", _lib.load().boac_backproject(
        ctypes.byref(g), _ptr(mu), _ptr(y), B, _ptr(res), _ptr(ws), ws.numel(), _stream(mu.device)))
    return res


def boac_set_wait_cycles(cycles: int) -> int:
    """Process-wide limit (GPU cycles) of the fused kernels' bounded hand-over
    wait; ``cycles <= 0`` restores the default.  Returns the previous limit."""
    return int(_lib.load().boac_set_wait_cycles(int(cycles)))


def _raise_on_device_status(fn: str, ws: torch.Tensor | None) -> None:
    """Raise BoacError if the device status word reports a failure
    (BOAC_ENONFINITE, a -inf score, is a result, not a failure)."""
    if ws is not None:
        st = boac_workspace_status(ws)
        if st not in (_lib.BOAC_OK, _lib.BOAC_ENONFINITE):
            raise _lib.BoacError(fn, st)


def boac_mlem(g: Geom, mu: torch.Tensor, S: torch.Tensor, F: torch.Tensor, K: int,
              score: bool = True, include_lgamma: bool = True, plain: bool = False,
              ws: torch.Tensor | None = None, L: torch.Tensor | None = None, unfused: bool = False,
              check_status: bool = True):
    """K MLEM iterations in place on F[B, n, n]; returns (F, L[B] float64 or None).

    By default the library's batched path (the persistent fused kernel, or
    for small batches the unfused batched kernels); ``unfused=True`` pins the
    unfused batched path (boac_mlem_unfused); ``plain=True`` the
    launch-per-step baseline (one candidate at a time).

    ``check_status`` (batched paths): wait for the call to finish and raise
    BoacError if a bounded device wait gave up (BOAC_ETIMEOUT in the
    workspace status word; those candidates' scores are NaN).  Pass False to
    keep the call asynchronous (required inside CUDA-graph capture) and read
    ``boac_workspace_status(ws)`` later."""
    _need(mu, "mu", torch.float32)
    B = mu.shape[0]
    _need(mu, "mu", torch.float32, (B, g.n, g.n))
    _need(F, "F", torch.float32, (B, g.n, g.n))
    S, stride = _sino(S, g, B)
    op = _lib.OP_MLEM_PLAIN if plain else (_lib.OP_MLEM_UNFUSED if unfused else _lib.OP_MLEM)
    if ws is None:
        ws = workspace(g, B, op, mu.device)
    if score and L is None:
        L = torch.empty(B, dtype=torch.float64, device=mu.device)
    if L is not None:
        _need(L, "L", torch.float64, (B,))
    name = "boac_mlem_plain" if plain else ("boac_mlem_unfused" if unfused else "boac_mlem")
    fn = getattr(_lib.load(), name)
    check(name,
          fn(ctypes.byref(g), _ptr(mu), _ptr(S), stride, _ptr(F), int(K), B,
             _ptr(L) if score else None, int(include_lgamma), _ptr(ws),
             ws.numel() if ws is not None else 0, _stream(mu.device)))
    if check_status and not plain:
        _raise_on_device_status(name, ws)
    return F, (L if score else None)


def boac_mlem_plain(g, mu, S, F, K, score=True, include_lgamma=True, ws=None, L=None):
    return boac_mlem(g, mu, S, F, K, score=score, include_lgamma=include_lgamma, plain=True, ws=ws, L=L)


def boac_score(g: Geom, mu: torch.Tensor, S: torch.Tensor, F: torch.Tensor,
               include_lgamma: bool = True, ws: torch.Tensor | None = None) -> torch.Tensor:
    """Eq. 5 at q = A^mu F: L[B] float64."""
    _need(mu, "mu", torch.float32)
    B = mu.shape[0]
    _need(F, "F", torch.float32, (B, g.n, g.n))
    S, stride = _sino(S, g, B)
    if ws is None:
        ws = workspace(g, B, _lib.OP_SCORE, mu.device)
    L = torch.empty(B, dtype=torch.float64, device=mu.device)
    check("boac_score", _lib.load().boac_score(
        ctypes.byref(g), _ptr(mu), _ptr(S), stride, _ptr(F), B, int(include_lgamma), _ptr(L),
        _ptr(ws), ws.numel(), _stream(mu.device)))
    return L


def boac_loglik(g: Geom, q: torch.Tensor, S: torch.Tensor, include_lgamma: bool = True) -> torch.Tensor:
    """Eq. 5 reduction of given expected counts q[B, V, nb]: L[B] float64."""
    _need(q, "q", torch.float32)
    B = q.shape[0]
    _need(q, "q", torch.float32, (B, g.n_views, g.n_bins))
    S, stride = _sino(S, g, B)
    L = torch.empty(B, dtype=torch.float64, device=q.device)
    check("boac_loglik", _lib.load().boac_loglik(
        ctypes.byref(g), _ptr(q), _ptr(S), stride, B, int(include_lgamma), _ptr(L), _stream(q.device)))
    return L


def boac_score_grad(g: Geom, t: Tissue, c: torch.Tensor, S: torch.Tensor, K: int,
                    ckpt_every: int = 2, include_lgamma: bool = True, want_image: bool = False,
                    ws: torch.Tensor | None = None, unfused: bool = False):
    """Score after K MLEM iterations (AREA map, F^0 = 1) and its gradient with
    respect to the Legendre coefficients: returns (L[B], dL/dc[B, 6], F^K or None),
    L and dL/dc in float64.  ``unfused=True`` pins the batched launch-per-step
    kernels (boac_score_grad_unfused) instead of the fused kernel."""
    _need(c, "c", torch.float32)
    if c.dim() != 2 or c.shape[1] != 6:
        raise ValueError("c must be [B, 6]")
    B = c.shape[0]
    S, stride = _sino(S, g, B)
    lib = _lib.load()
    if ws is None:
        nbytes = int(lib.boac_score_grad_workspace_bytes(ctypes.byref(g), B, int(K), int(ckpt_every)))
        if nbytes == 0:
            raise ValueError("invalid arguments for boac_score_grad")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=c.device)
    L = torch.empty(B, dtype=torch.float64, device=c.device)
    grad = torch.empty(B, 6, dtype=torch.float64, device=c.device)
    F = torch.empty(B, g.n, g.n, dtype=torch.float32, device=c.device) if want_image else None
    name = "boac_score_grad_unfused" if unfused else "boac_score_grad"
    check(name, getattr(lib, name)(
        ctypes.byref(g), ctypes.byref(t), _ptr(c), _ptr(S), stride, int(K), int(ckpt_every), B,
        int(include_lgamma), _ptr(L), _ptr(grad), _ptr(F), _ptr(ws), ws.numel(), _stream(c.device)))
    return L, grad, F


def boac_score_grad_params(g: Geom, p: torch.Tensor, S: torch.Tensor, K: int,
                           ckpt_every: int = 2, include_lgamma: bool = True, want_image: bool = False,
                           ws: torch.Tensor | None = None):
    """boac_score_grad in the 9-parameter model p[B, 9] = (c_0..c_5, mu_b, mu_c,
    dR): returns (L[B], dL/dp[B, 9], F^K or None), L and dL/dp in float64."""
    _need(p, "p", torch.float32)
    if p.dim() != 2 or p.shape[1] != 9:
        raise ValueError("p must be [B, 9]")
    B = p.shape[0]
    S, stride = _sino(S, g, B)
    lib = _lib.load()
    if ws is None:
        nbytes = int(lib.boac_score_grad_workspace_bytes(ctypes.byref(g), B, int(K), int(ckpt_every)))
        if nbytes == 0:
            raise ValueError("invalid arguments for boac_score_grad_params")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=p.device)
    L = torch.empty(B, dtype=torch.float64, device=p.device)
    grad = torch.empty(B, 9, dtype=torch.float64, device=p.device)
    F = torch.empty(B, g.n, g.n, dtype=torch.float32, device=p.device) if want_image else None
    check("boac_score_grad_params", lib.boac_score_grad_params(
        ctypes.byref(g), _ptr(p), _ptr(S), stride, int(K), int(ckpt_every), B,
        int(include_lgamma), _ptr(L), _ptr(grad), _ptr(F), _ptr(ws), ws.numel(), _stream(p.device)))
    return L, grad, F


class SysMat:
    """The system matrix A^mu written out (boac_sysmat_*): one sparsity pattern
    per geometry, values per candidate.  ``vals = m.values(mu)`` gives
    [ceil(B/8), 2, nnz, 8] float32 (groups of 8 candidates interleaved; A's
    order, then A^T's; ``SysMat.candidate_values(vals, b)`` extracts one);
    ``m.mlem(vals, S, F, K)`` runs MLEM on it; ``m.project(vals, F)`` is
    q = A F; ``m.pattern()`` returns (row_ptr, col, colT_ptr, rowT) as int32
    device tensors."""

    GROUP = 8

    @staticmethod
    def vals_shape(B: int, nnz: int):
        return ((B + SysMat.GROUP - 1) // SysMat.GROUP, 2, nnz, SysMat.GROUP)

    @staticmethod
    def candidate_values(vals: torch.Tensor, b: int) -> torch.Tensor:
        """[2, nnz] values of candidate b (A's order, then A^T's)."""
        return vals[b // SysMat.GROUP, :, :, b % SysMat.GROUP]

    def __init__(self, g: Geom, device=None):
        self.g = g
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self._lib = _lib.load()
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check("boac_sysmat_create", self._lib.boac_sysmat_create(ctypes.byref(g), ctypes.byref(h),
                                                                     _stream(self.device)))
        self._h = h
        self.nnz = int(self._lib.boac_sysmat_nnz(h))
        self.rows = g.n_views * g.n_bins

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.boac_sysmat_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pattern(self):
        nn = self.g.n * self.g.n
        i32 = dict(dtype=torch.int32, device=self.device)
        row_ptr, col = torch.empty(self.rows + 1, **i32), torch.empty(self.nnz, **i32)
        colT_ptr, rowT = torch.empty(nn + 1, **i32), torch.empty(self.nnz, **i32)
        check("boac_sysmat_pattern", self._lib.boac_sysmat_pattern(
            self._h, _ptr(row_ptr), _ptr(col), _ptr(colT_ptr), _ptr(rowT), _stream(self.device)))
        return row_ptr, col, colT_ptr, rowT

    def values(self, mu: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        _need(mu, "mu", torch.float32)
        B = mu.shape[0]
        shape = self.vals_shape(B, self.nnz)
        vals = out if out is not None else torch.empty(shape, dtype=torch.float32, device=mu.device)
        _need(vals, "vals", torch.float32, shape)
        check("boac_sysmat_values", self._lib.boac_sysmat_values(self._h, _ptr(mu), B, _ptr(vals),
                                                                 _stream(mu.device)))
        return vals

    def project(self, vals: torch.Tensor, F: torch.Tensor) -> torch.Tensor:
        _need(F, "F", torch.float32)
        B = F.shape[0]
        _need(vals, "vals", torch.float32, self.vals_shape(B, self.nnz))
        q = torch.empty(B, self.g.n_views, self.g.n_bins, dtype=torch.float32, device=F.device)
        check("boac_sysmat_project", self._lib.boac_sysmat_project(self._h, _ptr(vals), _ptr(F), B, _ptr(q),
                                                                   _stream(F.device)))
        return q

    def workspace(self, B: int) -> torch.Tensor:
        nbytes = int(self._lib.boac_sysmat_mlem_workspace_bytes(self._h, int(B)))
        return torch.empty(nbytes, dtype=torch.uint8, device=self.device)

    def mlem(self, vals: torch.Tensor, S: torch.Tensor, F: torch.Tensor, K: int, score: bool = True,
             include_lgamma: bool = True, ws: torch.Tensor | None = None):
        """K MLEM iterations on F [B, n, n] in place; returns (F, L or None)."""
        _need(F, "F", torch.float32)
        B = F.shape[0]
        _need(vals, "vals", torch.float32, self.vals_shape(B, self.nnz))
        S, stride = _sino(S, self.g, B)
        ws = ws if ws is not None else self.workspace(B)
        L = torch.empty(B, dtype=torch.float64, device=F.device) if score else None
        check("boac_sysmat_mlem", self._lib.boac_sysmat_mlem(
            self._h, _ptr(vals), _ptr(S), stride, _ptr(F), int(K), B, _ptr(L), int(include_lgamma),
            _ptr(ws), ws.numel(), _stream(F.device)))
        return F, L


class BoacScore(torch.autograd.Function):
    """ln P(S | F^K(c), A^mu(c)) as a differentiable function of the Legendre
    coefficients c[B, 6] (tissue values t), or of the 9-parameter model
    c[B, 9] = (c_0..c_5, mu_b, mu_c, dR) (t unused, may be None): the forward
    runs boac_score_grad / boac_score_grad_params (which return the gradient
    together with the score), the backward scales it by the incoming gradient.
    Usage: ``L = BoacScore.apply(c, geom, tissue, S, K, ckpt_every)``."""

    @staticmethod
    def forward(ctx, c, g, t, S, K, ckpt_every=2, include_lgamma=True):
        cd = c.detach().contiguous()
        if cd.dim() == 2 and cd.shape[1] == 9:
            L, grad, _ = boac_score_grad_params(g, cd, S, K, ckpt_every, include_lgamma)
        else:
            L, grad, _ = boac_score_grad(g, t, cd, S, K, ckpt_every, include_lgamma)
        ctx.save_for_backward(grad)
        ctx.c_dtype = c.dtype
        return L

    @staticmethod
    def backward(ctx, gL):
        (grad,) = ctx.saved_tensors
        return (gL[:, None] * grad).to(ctx.c_dtype), None, None, None, None, None, None


# ---------------------------------------------------------------- ragged
# Launch configurations per size class: ids 0-5 are the one-CTA kernel's
# shapes (2 * shape + 1 for two views per grid); ids 6-8 the cluster kernel
# for V % 4 == 0: 5, 6 or 8 CTAs per candidate for 256 x 256 images, 2, 4 or
# 8 for 128 x 128 and 64 x 64.
N_CONFIGS = 17
N_SINGLE_CTA_CONFIGS = 6
BAND_CLUSTER_SIZES = {256: {6: 5, 7: 6, 8: 8}, 128: {6: 2, 7: 4, 8: 8}, 64: {6: 2, 7: 4, 8: 8}}
# ids 9-16: the fused kernel's cluster mode, 2, 3, 4, 6, 8, 9, 12 or 16 CTAs
# per candidate each on its share of the sample grids (images up to 128 x 128)
SPLIT_CLUSTER_SIZES = {9 + i: g for i, g in enumerate((2, 3, 4, 6, 8, 9, 12, 16))}


def config_valid(g, cfg: int) -> bool:
    """Whether launch configuration ``cfg`` applies to geometry ``g``."""
    if cfg in SPLIT_CLUSTER_SIZES:
        return g.n in (64, 96, 128) and g.n_views % 4 == 0 and g.n_views >= 4 * SPLIT_CLUSTER_SIZES[cfg]
    if cfg >= N_SINGLE_CTA_CONFIGS:
        return cfg in BAND_CLUSTER_SIZES.get(g.n, {}) and g.n_views % 4 == 0
    if not 0 <= cfg < N_SINGLE_CTA_CONFIGS:
        return False
    return g.n_views % 2 == 0 and (cfg % 2 == 1 or g.n_views % 4 == 0)


class RaggedBatch:
    """Candidates of several size classes and iteration counts, packed into
    three flat device pools (mu, sinograms, images) for boac_mlem_ragged.

    ``classes``: list of Geom; ``cls``: class index per candidate; ``K``:
    iterations per candidate; ``mu``/``S``: per-candidate tensors
    ([n, n] and [V, n] of the candidate's class); ``F0``: initial images
    (default ones)."""

    def __init__(self, classes, cls, K, mu, S, F0=None, device=None):
        self.classes = list(classes)
        B = len(cls)
        if not (len(K) == len(mu) == len(S) == B):
            raise ValueError("cls, K, mu and S must have one entry per candidate")
        dev = device or mu[0].device
        geo = (Geom * len(self.classes))(*self.classes)
        cands = (RaggedCand * B)()
        mo = so = fo = 0
        for b in range(B):
            g = self.classes[int(cls[b])]
            if tuple(mu[b].shape) != (g.n, g.n) or tuple(S[b].shape) != (g.n_views, g.n_bins):
                raise ValueError(f"candidate {b}: tensor shapes do not match its class {g}")
            cands[b] = RaggedCand(int(cls[b]), int(K[b]), mo, so, fo)
            mo += g.n * g.n
            so += g.n_views * g.n_bins
            fo += g.n * g.n
        self.geo, self.cands, self.B = geo, cands, B
        self.mu_pool = torch.cat([m.reshape(-1).float() for m in mu]).to(dev).contiguous()
        self.S_pool = torch.cat([x.reshape(-1).float() for x in S]).to(dev).contiguous()
        if F0 is None:
            self.F_pool = torch.ones(fo, dtype=torch.float32, device=dev)
        else:
            self.F_pool = torch.cat([f.reshape(-1).float() for f in F0]).to(dev).contiguous()
        self.L = torch.empty(B, dtype=torch.float64, device=dev)
        self.device = dev

    def image(self, b: int) -> torch.Tensor:
        g = self.classes[self.cands[b].cls]
        o = self.cands[b].F_off
        return self.F_pool[o:o + g.n * g.n].view(g.n, g.n)

    def _config(self, config):
        if config is None:
            return None
        cfg = (ctypes.c_int * len(self.classes))(*[int(c) for c in config])
        return ctypes.cast(cfg, ctypes.c_void_p), cfg

    def workspace_bytes(self, config=None) -> int:
        c = self._config(config)
        n = _lib.load().boac_mlem_ragged_workspace_bytes(self.geo, len(self.classes), self.cands, self.B,
                                                         c[0] if c else None)
        if n == 0:
            raise ValueError("invalid ragged batch or configuration")
        return int(n)

    def prepare(self, config=None, ws=None) -> torch.Tensor:
        """Sort the candidates and copy their records into the workspace."""
        if ws is None:
            ws = torch.empty(self.workspace_bytes(config), dtype=torch.uint8, device=self.device)
        c = self._config(config)
        check("boac_mlem_ragged_prepare", _lib.load().boac_mlem_ragged_prepare(
            self.geo, len(self.classes), self.cands, self.B, c[0] if c else None, _ptr(ws), ws.numel(),
            _stream(self.device)))
        self.ws, self.config = ws, config
        return ws

    def status(self) -> int:
        """Device status word of the last run (synchronous): BOAC_OK, or
        BOAC_ETIMEOUT if a bounded hand-over wait gave up."""
        return boac_workspace_status(self.ws)

    def run(self, include_lgamma: bool = True) -> torch.Tensor:
        """Launch the per-class fused kernels (capturable in a CUDA graph)."""
        c = self._config(self.config)
        check("boac_mlem_ragged_run", _lib.load().boac_mlem_ragged_run(
            self.geo, len(self.classes), self.cands, self.B, _ptr(self.mu_pool), _ptr(self.S_pool),
            _ptr(self.F_pool), _ptr(self.L), int(include_lgamma), c[0] if c else None, _ptr(self.ws),
            self.ws.numel(), _stream(self.device)))
        return self.L


def boac_mlem_ragged(batch: RaggedBatch, include_lgamma: bool = True, config=None) -> torch.Tensor:
    """One-shot ragged MLEM + score: returns L[B] (float64); images in batch.F_pool.
    Waits for the launch and raises BoacError if a bounded device wait gave up."""
    batch.prepare(config)
    L = batch.run(include_lgamma)
    _raise_on_device_status("boac_mlem_ragged", batch.ws)
    return L


# ---------------------------------------------------------------- graphs
class BatchedEvaluator:
    """The batched candidate evaluation -- rasterise mu (Eq. 3-4), K fused MLEM
    iterations, Eq. 5 score -- captured once in a CUDA graph and replayed for
    every new set of coefficients.  ``evaluate(c)`` copies c into the graph's
    static input and replays; results live in ``self.L`` / ``self.F``."""

    def __init__(self, g: Geom, t: Tissue, S: torch.Tensor, B: int, K: int,
                 mode: int = _lib.RASTER_CENTER, include_lgamma: bool = True):
        dev = S.device
        self.g, self.t, self.K, self.mode, self.lg = g, t, int(K), mode, include_lgamma
        self.c = torch.zeros(B, 6, dtype=torch.float32, device=dev)
        self.S = S.contiguous()
        self.mu = torch.empty(B, g.n, g.n, dtype=torch.float32, device=dev)
        self.F = torch.empty(B, g.n, g.n, dtype=torch.float32, device=dev)
        self.L = torch.empty(B, dtype=torch.float64, device=dev)
        self.ws = workspace(g, B, _lib.OP_MLEM, dev)
        self.c.copy_(torch.tensor([[8.0, 0, 0, 0, 0, 0]], device=dev).expand(B, 6))
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):  # warm-up outside capture (sets kernel attributes)
            self._body()
        torch.cuda.current_stream(dev).wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._body()

    def _body(self):
        boac_rasterize_mu(self.g, self.t, self.c, self.mode, out=self.mu)
        self.F.fill_(1.0)
        boac_mlem(self.g, self.mu, self.S, self.F, self.K, score=True, include_lgamma=self.lg,
                  ws=self.ws, L=self.L, check_status=False)

    def status(self) -> int:
        """Device status word of the last replay (synchronous)."""
        return boac_workspace_status(self.ws) if self.ws is not None else _lib.BOAC_OK

    def evaluate(self, c: torch.Tensor) -> torch.Tensor:
        self.c.copy_(c, non_blocking=True)
        self.graph.replay()
        return self.L


def boac_test_mlem_handover(g: Geom, mu: torch.Tensor, S: torch.Tensor, K: int, config: int, holders: int,
                            withhold: int):
    """Test hook of the bounded hand-over wait (boac_test_mlem_handover):
    returns (F[B, n, n], L[B], device status word, workspace)."""
    _need(mu, "mu", torch.float32)
    B = mu.shape[0]
    _need(S, "S", torch.float32, (g.n_views, g.n_bins))
    lib = _lib.load()
    nbytes = int(lib.boac_test_mlem_handover_bytes(ctypes.byref(g), B, int(K), int(config), int(holders)))
    if nbytes == 0:
        raise ValueError("invalid arguments for boac_test_mlem_handover")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=mu.device)
    F = torch.ones(B, g.n, g.n, dtype=torch.float32, device=mu.device)
    L = torch.empty(B, dtype=torch.float64, device=mu.device)
    check("boac_test_mlem_handover", lib.boac_test_mlem_handover(
        ctypes.byref(g), _ptr(mu), _ptr(S), _ptr(F), int(K), B, _ptr(L), int(config), int(holders),
        int(withhold), _ptr(ws), ws.numel(), _stream(mu.device)))
    return F, L, boac_workspace_status(ws), ws
