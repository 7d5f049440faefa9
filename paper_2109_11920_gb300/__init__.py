"""BOAC hot path on GB300: batched attenuated projection, MLEM and Poisson
score for Bayesian-optimisation attenuation correction in SPECT brain imaging
(Koutsantonis et al., arXiv 2109.11920).

The compute runs in ``libboac.so`` (hand-written sm_103a CUDA behind the C ABI
of ``include/boac.h``); this package is its thin torch binding.  Importing the
package does not load the library; the first call does, and fails loudly if
it is missing.
"""
from ._lib import (BOAC_EINVAL, BOAC_EUNSUPPORTED, BOAC_EWORKSPACE, BOAC_OK, OP_BACKPROJECT,
                   OP_MLEM, OP_MLEM_PLAIN, OP_PROJECT, OP_SCORE, OP_SCORE_GRAD, RASTER_AREA,
                   RASTER_CENTER, BoacError, Geom, Tissue)

__all__ = [
    "Geom", "Tissue", "BoacError", "RASTER_CENTER", "RASTER_AREA",
    "boac_rasterize_mu", "boac_rasterize_mu_params", "boac_project", "boac_backproject",
    "boac_mlem", "boac_mlem_plain", "boac_score", "boac_loglik", "boac_score_grad",
    "boac_score_grad_params", "boac_workspace_bytes",
]


def __getattr__(name):
    # torch-facing wrappers are imported lazily so that the pure-numpy parts
    # (synthetic inputs) do not pull in torch
    if name.startswith("boac_") or name == "workspace":
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
