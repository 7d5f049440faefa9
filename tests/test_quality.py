"""Pins for the image-quality metrics of the NAC / BOAC study (SSIM, CNR,
PSNR): brute force over every window on small images, closed forms and
invariants.  Runs on CPU."""
import numpy as np
import pytest

from paper_2109_11920_gb300 import quality, synth


def ssim_brute(x, y, L, size=11, sigma=1.5):
    """Every window position inside the image, weights written out."""
    t = np.arange(size) - (size - 1) / 2.0
    W = np.exp(-(t[:, None] ** 2 + t[None, :] ** 2) / (2 * sigma ** 2))
    W /= W.sum()
    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    vals = []
    for i in range(x.shape[0] - size + 1):
        for j in range(x.shape[1] - size + 1):
            a, b = x[i:i + size, j:j + size], y[i:i + size, j:j + size]
            ma, mb = (W * a).sum(), (W * b).sum()
            va, vb = (W * (a - ma) ** 2).sum(), (W * (b - mb) ** 2).sum()
            cab = (W * (a - ma) * (b - mb)).sum()
            vals.append((2 * ma * mb + C1) * (2 * cab + C2) / ((ma ** 2 + mb ** 2 + C1) * (va + vb + C2)))
    return np.mean(vals)


def test_gaussian_window():
    w = quality.gaussian_window(11, 1.5)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(w, w[::-1], rtol=0, atol=0)
    assert w[6] / w[5] == pytest.approx(np.exp(-0.5 / 1.5 ** 2), rel=1e-14)


def test_ssim_against_brute_force():
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 4, (17, 14))
    y = x + rng.normal(0, 0.5, x.shape)
    L = x.max() - x.min()
    assert quality.ssim(x, y) == pytest.approx(ssim_brute(x, y, L), rel=1e-12)
    # a different range and an anti-correlated image
    assert quality.ssim(x, -y, 10.0) == pytest.approx(ssim_brute(x, -y, 10.0), rel=1e-12)


def test_ssim_closed_forms():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 4, (20, 20))
    assert quality.ssim(x, x) == pytest.approx(1.0, abs=1e-12)
    # constant images: only the luminance term is left
    a, b, L = 2.0, 3.0, 5.0
    C1 = (0.01 * L) ** 2
    got = quality.ssim(np.full((12, 12), a), np.full((12, 12), b), L)
    assert got == pytest.approx((2 * a * b + C1) / (a * a + b * b + C1), rel=1e-12)
    # symmetric in its arguments for a fixed range
    y = rng.uniform(0, 4, (20, 20))
    assert quality.ssim(x, y, 4.0) == pytest.approx(quality.ssim(y, x, 4.0), rel=1e-13)
    with pytest.raises(ValueError):
        quality.ssim(np.ones((8, 8)), np.ones((8, 8)))


def test_psnr_closed_form():
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 4, (30, 30))
    assert quality.psnr(x, x + 0.1) == pytest.approx(10 * np.log10(x.max() ** 2 / 0.01), rel=1e-12)
    assert quality.psnr(x, x) == float("inf")
    assert quality.psnr(x, 2 * x, peak=1.0) == pytest.approx(-10 * np.log10(np.mean(x ** 2)), rel=1e-12)


def test_cnr_closed_form():
    img = np.zeros((10, 10))
    roi = np.zeros((10, 10), bool)
    roi[:3, :3] = True
    bg = np.zeros((10, 10), bool)
    bg[5:, :] = True
    img[roi] = 7.0
    vals = np.where(np.arange(50) % 2 == 0, 2.5, 1.5)  # mean 2, population std 0.5
    img[bg] = vals
    assert quality.cnr(img, roi, bg) == pytest.approx(abs(7.0 - 2.0) / 0.5, rel=1e-14)
    with pytest.raises(ValueError):
        quality.cnr(img, np.zeros((10, 10), bool), bg)


def test_search_box_covers_the_synthetic_heads():
    lo, hi = quality.search_box()
    C = synth.slice_coefficients(np.random.default_rng(0), 2000)
    assert np.all(C >= lo) and np.all(C <= hi)
    wl = quality.QUALITY
    for case in range(wl.extra["cases"]):
        c = synth.slice_coefficients(np.random.default_rng(wl.seed + case), 1)[0]
        assert np.all(c >= lo) and np.all(c <= hi)
