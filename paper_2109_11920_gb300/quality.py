"""Image-quality study of Sec. IV: reconstructions with attenuation correction
from the BO estimate of the head (MLEM-BOAC) against reconstructions without
attenuation correction (MLEM-NAC), scored against the true emission image by
SSIM, CNR and PSNR (Table 1).

The paper names the three metrics and cites Wang et al. for SSIM without
giving its settings, so the standard forms are used:

* SSIM (Wang, Bovik, Sheikh & Simoncelli, IEEE TIP 2004): local means,
  variances and covariance under an 11 x 11 Gaussian window of standard
  deviation 1.5 pixels (weights normalised to 1), over every window position
  that lies inside the image;
    SSIM = (2 m_x m_y + C1)(2 s_xy + C2) / ((m_x^2 + m_y^2 + C1)(s_x^2 + s_y^2 + C2)),
  C1 = (0.01 L)^2, C2 = (0.03 L)^2, L the value range of the true image; the
  score is the mean over the windows.
* CNR: |mean(ROI) - mean(background)| / std(background), ROI = the hot
  lesions of the true image, background = the rest of the brain.
* PSNR: 10 log10(max(true)^2 / MSE) over the whole image.

The images are compared as reconstructed, without rescaling: the true image
is the phantom in the units in which MLEM reconstructs it (the activity whose
attenuated projection is the expected sinogram).  The paper's phantoms are not
published, so the cases are seeded synthetic heads (Legendre boundaries with
c_0 ~ U(6, 9) cm) and phantoms, 128 x 128 pixels and 72 views as in Sec. IV;
the numbers cannot reproduce Table 1.
"""
from __future__ import annotations

import numpy as np

from . import synth


# ----------------------------------------------------------------- metrics
def gaussian_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    """1-D Gaussian weights, summing to 1 (the 2-D window is their outer product)."""
    x = np.arange(size) - (size - 1) / 2.0
    w = np.exp(-0.5 * (x / sigma) ** 2)
    return w / w.sum()


def _filter_valid(img: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Separable weighted sum over every window position inside the image."""
    k = w.size
    rows = np.lib.stride_tricks.sliding_window_view(img, k, axis=0) @ w   # [n-k+1, m]
    return np.lib.stride_tricks.sliding_window_view(rows, k, axis=1) @ w  # [n-k+1, m-k+1]


def ssim(ref: np.ndarray, img: np.ndarray, data_range: float | None = None,
         size: int = 11, sigma: float = 1.5) -> float:
    """Mean SSIM of ``img`` against ``ref`` (definition in the module docstring)."""
    x = np.asarray(ref, dtype=np.float64)
    y = np.asarray(img, dtype=np.float64)
    if x.shape != y.shape or min(x.shape) < size:
        raise ValueError("images must have the same shape, at least one window wide")
    L = float(x.max() - x.min()) if data_range is None else float(data_range)
    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    w = gaussian_window(size, sigma)
    mx, my = _filter_valid(x, w), _filter_valid(y, w)
    sxx = _filter_valid(x * x, w) - mx * mx
    syy = _filter_valid(y * y, w) - my * my
    sxy = _filter_valid(x * y, w) - mx * my
    s = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return float(s.mean())


def psnr(ref: np.ndarray, img: np.ndarray, peak: float | None = None) -> float:
    """10 log10(peak^2 / MSE), peak = max(ref) unless given."""
    x = np.asarray(ref, dtype=np.float64)
    y = np.asarray(img, dtype=np.float64)
    mse = float(np.mean((x - y) ** 2))
    p = float(x.max()) if peak is None else float(peak)
    return float("inf") if mse == 0.0 else float(10.0 * np.log10(p * p / mse))


def cnr(img: np.ndarray, roi: np.ndarray, background: np.ndarray) -> float:
    """|mean(img[roi]) - mean(img[background])| / std(img[background])."""
    y = np.asarray(img, dtype=np.float64)
    r, b = y[np.asarray(roi, bool)], y[np.asarray(background, bool)]
    if r.size == 0 or b.size < 2:
        raise ValueError("empty region")
    return float(abs(r.mean() - b.mean()) / b.std())


def scores(truth: np.ndarray, img: np.ndarray, roi: np.ndarray, background: np.ndarray) -> dict:
    return {"ssim": ssim(truth, img), "cnr": cnr(img, roi, background), "psnr": psnr(truth, img)}


# ----------------------------------------------------------------- study
QUALITY = synth.Workload("quality128_v72", 128, 0.2, 72, 50, 32, 1e6, seed=500,
                         extra={"cases": 3, "bo_init": 64, "bo_cycles": 4})


def search_box(half_c0: float = 2.0, rel: float = 0.75):
    """Box of the BO search: c_0 in 7.5 +- half_c0 cm, the shape terms within
    +-rel of |C_TRUE_k| around C_TRUE_k (covers every synthetic head)."""
    c = np.asarray(synth.C_TRUE, dtype=np.float64)
    half = rel * np.abs(c)
    lo, hi = c - half, c + half
    lo[0], hi[0] = 7.5 - half_c0, 7.5 + half_c0
    return lo, hi


def run_case(case: int, device, wl=QUALITY, bo_seed: int = 0):
    """One seeded head and phantom: simulate the sinogram with the true map,
    reconstruct without attenuation correction (mu = 0), with the true map,
    and with the map of the BO estimate; return the images, masks and
    scores.  Every step runs through the library (rasterise, project, MLEM)."""
    import torch

    from . import api, bo
    from ._lib import Geom, Tissue

    n, dx, V, K = wl.n, wl.dx, wl.V, wl.K
    g, t = Geom.make(n, dx, V), Tissue(*synth.TISSUE)
    ph, noise, _ = synth.streams(wl.seed + case)
    c_true = synth.slice_coefficients(np.random.default_rng(wl.seed + case), 1)[0]
    c_t = torch.tensor(c_true[None].astype(np.float32), device=device)
    mu_true = api.boac_rasterize_mu(g, t, c_t)
    brain = (mu_true[0] == torch.tensor(t.mu_b, dtype=torch.float32)).cpu().numpy()
    F_true = synth.paint_activity(n, dx, brain, synth.ellipses(ph, c_true[0]))
    q = api.boac_project(g, mu_true, torch.tensor(F_true[None].astype(np.float32), device=device))
    q = q[0].double().cpu().numpy()
    S_np = synth.poisson_sinogram(noise, q, wl.counts)
    truth = F_true * (wl.counts / q.sum())
    S = torch.tensor(S_np.astype(np.float32), device=device)

    def mlem(mu):
        F = torch.ones(1, n, n, device=device)
        F, _ = api.boac_mlem(g, mu, S, F, K)
        return F[0].double().cpu().numpy()

    lo, hi = search_box()
    evaluate = bo.gpu_objective(g, t, S, K)
    res = bo.BOACOptimizer(evaluate, lo, hi, batch=wl.B, init=wl.extra["bo_init"],
                           max_cycles=wl.extra["bo_cycles"], ei_threshold=0.0, seed=bo_seed).run()
    c_bo = torch.tensor(res.best_c[None].astype(np.float32), device=device)
    images = {
        "MLEM-NAC": mlem(torch.zeros(1, n, n, device=device)),
        "MLEM-BOAC": mlem(api.boac_rasterize_mu(g, t, c_bo)),
        "MLEM-AC (true map)": mlem(mu_true),
    }
    roi = F_true == F_true.max()
    background = brain & ~roi
    return {
        "c_true": c_true, "c_bo": res.best_c, "truth": truth, "images": images,
        "scores": {k: scores(truth, v, roi, background) for k, v in images.items()},
        "evaluations": len(res.history_f),
    }
