"""ctypes binding of the C ABI in ``include/boac.h`` (``libboac.so``).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of ``csrc/``.  PyTorch supplies device memory (including the
workspaces the library asks for) and the current stream.  There is no CPU
fallback: if the library is missing or the tensors are not on a CUDA device,
the call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libboac.so")

BOAC_OK = 0
BOAC_EINVAL = -1
BOAC_ECUDA = -2
BOAC_EWORKSPACE = -3
BOAC_EUNSUPPORTED = -4
BOAC_ETIMEOUT = -5
BOAC_ENONFINITE = -6

RASTER_CENTER = 0
RASTER_AREA = 1

OP_PROJECT = 0
OP_BACKPROJECT = 1
OP_MLEM = 2
OP_MLEM_PLAIN = 3
OP_SCORE = 4
OP_SCORE_GRAD = 5
OP_MLEM_UNFUSED = 6


class Geom(ctypes.Structure):
    """``boac_geom``: n x n pixels of pixel_cm, n_views over 360 deg, n_bins = n."""
    _fields_ = [("n", ctypes.c_int), ("n_bins", ctypes.c_int), ("n_views", ctypes.c_int),
                ("pixel_cm", ctypes.c_float), ("bin_cm", ctypes.c_float)]

    @classmethod
    def make(cls, n: int, pixel_cm: float, n_views: int) -> "Geom":
        return cls(int(n), int(n), int(n_views), float(pixel_cm), float(pixel_cm))

    def __repr__(self):
        return f"Geom(n={self.n}, pixel_cm={self.pixel_cm:.6g}, n_views={self.n_views})"


class Tissue(ctypes.Structure):
    """``boac_tissue``: mu_b, mu_c (cm^-1) and cranium thickness dR (cm)."""
    _fields_ = [("mu_b", ctypes.c_float), ("mu_c", ctypes.c_float), ("dR", ctypes.c_float)]


class RaggedCand(ctypes.Structure):
    """``boac_ragged_cand``: size class, iteration count and the float offsets
    of the candidate's mu, sinogram and image in the three device pools."""
    _fields_ = [("cls", ctypes.c_int), ("K", ctypes.c_int), ("mu_off", ctypes.c_longlong),
                ("S_off", ctypes.c_longlong), ("F_off", ctypes.c_longlong)]


class BoacError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} failed: {status_string(status)} ({status})")
        self.status = status


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_SZ = ctypes.c_size_t
_LL = ctypes.c_longlong
_GP = ctypes.POINTER(Geom)
_TP = ctypes.POINTER(Tissue)

# (name, restype, argtypes) of every exported symbol declared in include/boac.h
SIGNATURES = {
    "boac_status_string": (ctypes.c_char_p, [_I]),
    "boac_abi_version": (_I, []),
    "boac_bounds_faults": (_I, [ctypes.POINTER(ctypes.c_int), _I]),
    "boac_workspace_status": (_I, [_P, _SZ, ctypes.POINTER(ctypes.c_int)]),
    "boac_workspace_bytes": (_SZ, [_GP, _I, _I]),
    "boac_set_wait_cycles": (_LL, [_LL]),
    "boac_test_mlem_handover_bytes": (_SZ, [_GP, _I, _I, _I, _I]),
    "boac_test_mlem_handover": (_I, [_GP, _P, _P, _P, _I, _I, _P, _I, _I, _I, _P, _SZ, _P]),
    "boac_rasterize_mu": (_I, [_GP, _TP, _P, _I, _I, _P, _P]),
    "boac_rasterize_mu_params": (_I, [_GP, _P, _I, _I, _P, _P]),
    "boac_project": (_I, [_GP, _P, _P, _I, _P, _P]),
    "boac_backproject": (_I, [_GP, _P, _P, _I, _P, _P, _SZ, _P]),
    "boac_mlem": (_I, [_GP, _P, _P, _LL, _P, _I, _I, _P, _I, _P, _SZ, _P]),
    "boac_mlem_plain": (_I, [_GP, _P, _P, _LL, _P, _I, _I, _P, _I, _P, _SZ, _P]),
    "boac_mlem_unfused": (_I, [_GP, _P, _P, _LL, _P, _I, _I, _P, _I, _P, _SZ, _P]),
    "boac_mlem_noalloc": (_I, [_GP, _P, _P, _LL, _P, _I, _I, _P, _I, _P]),
    "boac_score": (_I, [_GP, _P, _P, _LL, _P, _I, _I, _P, _P, _SZ, _P]),
    "boac_loglik": (_I, [_GP, _P, _P, _LL, _I, _I, _P, _P]),
    "boac_score_grad_workspace_bytes": (_SZ, [_GP, _I, _I, _I]),
    "boac_mlem_ragged_workspace_bytes": (_SZ, [_GP, _I, ctypes.POINTER(RaggedCand), _I, _P]),
    "boac_mlem_ragged_prepare": (_I, [_GP, _I, ctypes.POINTER(RaggedCand), _I, _P, _P, _SZ, _P]),
    "boac_mlem_ragged_run": (_I, [_GP, _I, ctypes.POINTER(RaggedCand), _I, _P, _P, _P, _P, _I, _P, _P,
                                  _SZ, _P]),
    "boac_mlem_ragged": (_I, [_GP, _I, ctypes.POINTER(RaggedCand), _I, _P, _P, _P, _P, _I, _P, _P, _SZ,
                              _P]),
    "boac_score_grad": (_I, [_GP, _TP, _P, _P, _LL, _I, _I, _I, _I, _P, _P, _P, _P, _SZ, _P]),
    "boac_score_grad_params": (_I, [_GP, _P, _P, _LL, _I, _I, _I, _I, _P, _P, _P, _P, _SZ, _P]),
    "boac_score_grad_unfused": (_I, [_GP, _TP, _P, _P, _LL, _I, _I, _I, _I, _P, _P, _P, _P, _SZ, _P]),
    "boac_sysmat_create": (_I, [_GP, ctypes.POINTER(_P), _P]),
    "boac_sysmat_destroy": (_I, [_P]),
    "boac_sysmat_nnz": (_LL, [_P]),
    "boac_sysmat_pattern": (_I, [_P, _P, _P, _P, _P, _P]),
    "boac_sysmat_values": (_I, [_P, _P, _I, _P, _P]),
    "boac_sysmat_project": (_I, [_P, _P, _P, _I, _P, _P]),
    "boac_sysmat_mlem_workspace_bytes": (_SZ, [_P, _I]),
    "boac_sysmat_mlem": (_I, [_P, _P, _P, _LL, _P, _I, _I, _P, _I, _P, _SZ, _P]),
}


CHECKED_LIB_PATH = os.path.join(PKG, "libboac_checked.so")


def _open(path: str):
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -m paper_2109_11920_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(path: str = LIB_PATH):
    """Load libboac.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = _open(path)
    return _lib


def load_checked():
    """A separate handle on the bounds-checked build, libboac_checked.so
    (``build.build(checked=True)``), with the same entry points."""
    return _open(CHECKED_LIB_PATH)


def status_string(status: int) -> str:
    try:
        return load().boac_status_string(int(status)).decode()
    except ImportError:
        return "unknown"


def check(fn: str, status: int) -> None:
    if status != BOAC_OK:
        raise BoacError(fn, status)
