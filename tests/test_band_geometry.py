"""Geometry the 256 x 256 cluster kernel relies on, checked on the CPU with
float32 arithmetic emulated in numpy: every ray sample inside the image
belongs to exactly one band; within a band the samples of a lattice column
(a ray of the base view) form one run of consecutive k and those of a
lattice row one run of consecutive b; runs and per-thread steps fit the
kernel's buffers (constants restated from boac_band.cu's shapes).  The
kernel's record kernel checks the same at run time and refuses to run
otherwise; this test pins the reasoning behind the buffer sizes."""
import math

import numpy as np
import pytest

N = 256
F32 = np.float32


def band_starts(nb, n=N):
    if n == 256 and nb == 5:
        return [0, 52, 103, 152, 203, 256]
    h = -(-n // nb)
    return [min(r * h, n) for r in range(nb + 1)]


def shape(nb, n=N):
    st = band_starts(nb, n)
    H = max(st[r + 1] - st[r] for r in range(nb))
    LC = ((H + 1) * 141422 + 99999) // 100000 + 2
    TC = 4  # threads per column: the CTA has 4 n threads
    return H, LC, (LC + TC - 1) // TC, (LC + 1) // 2


def cos_sin(v, V):
    """Quadrant exact, in-quadrant angle in float64 rounded once (as the kernels)."""
    quad = (4 * v // V) % 4
    th = 1.5707963267948966192 * ((4 * v) % V) / V
    c, s = F32(math.cos(th)), F32(math.sin(th))
    return [(c, s), (-s, c), (-c, -s), (s, -c)][quad]


def fma32(a, b, c):
    # a * b is exact in float64 for float32 operands; one rounding to float32
    return (a.astype(np.float64) * np.float64(b) + c.astype(np.float64)).astype(F32)


def sample_uw(cs, sn, n=N):
    c = F32(0.5 * (n - 1))
    K, B = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    kc = (K.astype(F32) - c).astype(F32)
    bc = (B.astype(F32) - c).astype(F32)
    u = fma32(-kc, sn, fma32(bc, cs, np.full_like(bc, c)))
    w = fma32(kc, cs, fma32(bc, sn, np.full_like(bc, c)))
    return u, w


def runs(mask, axis):
    """Lengths of the runs along `axis`; asserts each line holds one run."""
    m = np.moveaxis(mask, axis, 0)
    lens = m.sum(0)
    first = np.argmax(m, axis=0)
    last = m.shape[0] - 1 - np.argmax(m[::-1], axis=0)
    nz = lens > 0
    assert np.all(last[nz] - first[nz] + 1 == lens[nz]), "a line's samples are not one run"
    return lens


@pytest.mark.parametrize("n,nb", [(256, 5), (256, 6), (256, 8), (128, 2), (128, 4), (128, 8), (64, 2), (64, 4), (64, 8)])
@pytest.mark.parametrize("V,grids", [(16, None), (120, None), (180, None), (720, range(0, 180, 7))])
def test_band_runs_fit_the_kernel_buffers(n, nb, V, grids):
    NT = 4 * n
    st = band_starts(nb, n)
    H, LC, SC, SR = shape(nb, n)
    for gi in (grids if grids is not None else range(V // 4)):
        base = gi if 8 * gi <= V else gi + 3 * V // 4
        cs, sn = cos_sin(base % V, V)
        assert cs > 0.7  # base angle within (-45, 45] degrees
        u, w = sample_uw(cs, sn, n)
        inside = (u > -1) & (u < n) & (w > -1) & (w < n)
        fi = np.floor(w).astype(int)
        band = np.searchsorted(np.array(st[1:-1]), fi, side="right")
        total = 0
        for r in range(nb):
            m = inside & (band == r)
            total += int(m.sum())
            col = runs(m, 0)  # along k for every b
            row = runs(m, 1)  # along b for every k
            assert col.max() <= LC
            assert int(np.max(-(-col // 4))) <= SC
            active = np.nonzero(row)[0]
            if len(active):
                R = active[-1] - active[0] + 1
                T = NT // R
                assert int(np.max(-(-row // T))) <= SR
        assert total == int(inside.sum())  # each inside sample in exactly one band


def test_band_heights_fill_the_image():
    for n, nb in ((256, 5), (256, 6), (256, 8), (128, 2), (128, 4), (128, 8), (64, 2), (64, 4), (64, 8)):
        st = band_starts(nb, n)
        assert st[0] == 0 and st[-1] == n and all(b > a for a, b in zip(st, st[1:]))


def scatter5_beta(cs, sn):
    """The kernel's choice of 5-class lattice {k + beta b = c (mod 5)} (0: none)."""
    for beta in (3, 2):
        good = True
        for m in range(-2, 3):
            for n in range(-2, 3):
                if (m == 0 and n == 0) or (m + beta * n + 25) % 5:
                    continue
                du = abs(F32(n) * cs - F32(m) * sn)
                dw = abs(F32(n) * sn + F32(m) * cs)
                if max(du, dw) < 2.001:
                    good = False
        if good:
            return beta
    return 0


def footprints_disjoint(u, w, inside, cls):
    """No pixel is touched by two samples of one class (bilinear 2x2 footprints)."""
    fj = np.floor(u).astype(np.int64)
    fi = np.floor(w).astype(np.int64)
    for c in np.unique(cls[inside]):
        sel = inside & (cls == c)
        pix = np.concatenate([((fi[sel] + di) * (N + 2) + fj[sel] + dj) for di in (0, 1) for dj in (0, 1)])
        if len(np.unique(pix)) != len(pix):
            return False
    return True


@pytest.mark.parametrize("V", [16, 120, 180])
def test_scatter_classes_are_race_free(V):
    """Brute force over every grid: the 9-class split (k mod 3, b mod 3) and,
    where the kernel picks one, the 5-class lattice give disjoint footprints
    within each class; the 5-class choice exists away from the axes."""
    K, B = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    for gi in range(V // 4):
        base = gi if 8 * gi <= V else gi + 3 * V // 4
        cs, sn = cos_sin(base % V, V)
        u, w = sample_uw(cs, sn)
        inside = (u > -1) & (u < N) & (w > -1) & (w < N)
        assert footprints_disjoint(u, w, inside, (K % 3) * 3 + (B % 3))
        beta = scatter5_beta(cs, sn)
        if abs(float(sn)) > 1e-3:
            assert beta in (2, 3)
        if beta:
            assert footprints_disjoint(u, w, inside, (K + beta * B) % 5)


def test_a_bad_lattice_is_caught():
    """The brute-force check is not vacuous: 4 classes (k mod 2, b mod 2) let
    footprints overlap at 30 degrees."""
    cs, sn = F32(math.cos(math.radians(30))), F32(math.sin(math.radians(30)))
    K, B = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    u, w = sample_uw(cs, sn)
    inside = (u > -1) & (u < N) & (w > -1) & (w < N)
    assert not footprints_disjoint(u, w, inside, (K % 2) * 2 + (B % 2))
