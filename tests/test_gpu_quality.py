"""The NAC / BOAC image-quality study (Sec. IV, Table 1) on seeded synthetic
heads, 128 x 128 pixels and 72 views: attenuation correction with the map of
the BO estimate scores better than no correction on SSIM, CNR and PSNR in
every case.  (Table 1 itself cannot be reproduced: the paper's phantoms are
not published.)"""
import numpy as np
import pytest

from paper_2109_11920_gb300 import quality

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", range(quality.QUALITY.extra["cases"]))
def test_boac_beats_nac(cuda, case):
    r = quality.run_case(case, cuda)
    s = r["scores"]
    for m in ("ssim", "cnr", "psnr"):
        assert s["MLEM-BOAC"][m] > s["MLEM-NAC"][m], (m, s)
    # the BO estimate's map gives images close to those of the true map
    assert s["MLEM-BOAC"]["psnr"] > s["MLEM-AC (true map)"]["psnr"] - 3.0, s
    assert abs(r["c_bo"][0] - r["c_true"][0]) < 1.0, (r["c_bo"], r["c_true"])
    assert r["evaluations"] == quality.QUALITY.extra["bo_init"] + \
        quality.QUALITY.extra["bo_cycles"] * quality.QUALITY.B
    assert all(np.isfinite(v) for sc in s.values() for v in sc.values())
