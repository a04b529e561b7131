"""ctypes declarations of the C ABI in include/isrs_gn.h (marshalling only)."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_double_p = ctypes.POINTER(ctypes.c_double)
c_int_p = ctypes.POINTER(ctypes.c_int)

ISRS_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "allocation failed", 4: "timeout",
          5: "numeric error", 6: "unsupported", 7: "debug bounds check failed"}
CELLS_SCI_XCI, CELLS_ALL = 0, 1
PREC_FP32, PREC_FP64 = 0, 1


class Fibre(ctypes.Structure):
    _fields_ = [("L_km", ctypes.c_double), ("f_ref_THz", ctypes.c_double), ("beta2", ctypes.c_double),
                ("beta3", ctypes.c_double), ("beta4", ctypes.c_double), ("Cr", ctypes.c_double),
                ("alpha_R_per_km", ctypes.c_double), ("n_spans", ctypes.c_int), ("profile", ctypes.c_int),
                ("raman_max_THz", ctypes.c_double), ("raman_photon", ctypes.c_int)]


class Channels(ctypes.Structure):
    _fields_ = [("n_ch", ctypes.c_int), ("f_THz", c_double_p), ("B_THz", c_double_p),
                ("alpha_per_km", c_double_p), ("gamma_per_W_km", c_double_p), ("nf_dB", c_double_p),
                ("guard", ctypes.POINTER(ctypes.c_ubyte)), ("raman_scale", c_double_p)]


class Quad(ctypes.Structure):
    _fields_ = [("G", ctypes.c_int), ("n_edges", ctypes.c_int), ("eps_v1", ctypes.c_double),
                ("cell_set", ctypes.c_int), ("precision", ctypes.c_int), ("snr_trx_dB", ctypes.c_double),
                ("ode_h_km", ctypes.c_double), ("G_mci", ctypes.c_int)]


class IsrsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def debug_requested() -> bool:
    """ISRS_GN_DEBUG=1 selects the bounds-checked debug build of the library."""
    return os.environ.get("ISRS_GN_DEBUG", "0") not in ("", "0")


def library_path() -> str:
    return _build.LIB_DEBUG if debug_requested() else _build.LIB


def load(build_if_missing: bool = True):
    """Load the in-tree library (building it when asked; the debug build when
    ISRS_GN_DEBUG=1).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    dbg = debug_requested()
    path = _build.build(debug=dbg) if build_if_missing else library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"ISRS GN CUDA library not built: {path}")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    lib.isrs_create.argtypes = [P(vp), ctypes.c_int]
    lib.isrs_destroy.argtypes = [vp]
    lib.isrs_status_string.argtypes = [ctypes.c_int]
    lib.isrs_status_string.restype = ctypes.c_char_p
    lib.isrs_last_error.argtypes = [vp]
    lib.isrs_last_error.restype = ctypes.c_char_p
    lib.isrs_debug_build.argtypes = []
    lib.isrs_debug_build.restype = ctypes.c_int
    if bool(lib.isrs_debug_build()) != dbg:
        raise RuntimeError(f"{path}: expected the {'debug' if dbg else 'release'} build of the library")
    lib.isrs_beta_from_dispersion.argtypes = [ctypes.c_double] * 4 + [c_double_p]
    lib.isrs_gamma_from_aeff.argtypes = [ctypes.c_double] * 3
    lib.isrs_gamma_from_aeff.restype = ctypes.c_double
    lib.isrs_gn_eta.argtypes = [vp, P(Fibre), P(Channels), vp, P(Quad), c_int_p, ctypes.c_int,
                                vp, vp, vp, vp]
    lib.isrs_gn_snr.argtypes = [vp, P(Fibre), P(Channels), vp, P(Quad), vp, vp, c_double_p, vp]
    lib.isrs_gn_grad.argtypes = [vp, P(Fibre), P(Channels), vp, P(Quad), vp, vp, vp, c_double_p, vp]
    lib.isrs_gn_grad_shard_fwd.argtypes = [vp, P(Fibre), P(Channels), vp, P(Quad), c_int_p, ctypes.c_int, vp, vp]
    lib.isrs_gn_grad_shard_bwd.argtypes = [vp, vp, ctypes.c_int, vp, vp, c_double_p, vp]
    lib.isrs_gn_eta_batched.argtypes = [vp, P(Fibre), ctypes.c_int, P(Channels), ctypes.c_int, c_int_p,
                                        vp, P(Quad), vp, vp]
    lib.isrs_set_tile.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.isrs_debug_inject_fault.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.isrs_debug_inject_fault.restype = ctypes.c_int
    lib.isrs_last_launch_info.argtypes = [vp, P(ctypes.c_int64), P(ctypes.c_int64), c_int_p]
    lib.isrs_last_graph_replay.argtypes = [vp, c_int_p]
    lib.isrs_last_graph_replay.restype = ctypes.c_int
    lib.isrs_last_path_counts.argtypes = [vp, P(ctypes.c_int64)]
    lib.isrs_last_path_counts.restype = ctypes.c_int
    lib.isrs_last_kernel_ms.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]
    lib.isrs_probe_alu_peaks.argtypes = [ctypes.c_int, ctypes.c_int, c_double_p, ctypes.POINTER(ctypes.c_float)]
    lib.isrs_probe_alu_peaks.restype = ctypes.c_int
    for name in ("isrs_last_kernel_ms", "isrs_create", "isrs_destroy", "isrs_beta_from_dispersion", "isrs_gn_eta", "isrs_gn_snr",
                 "isrs_gn_grad", "isrs_gn_grad_shard_fwd", "isrs_gn_grad_shard_bwd", "isrs_gn_eta_batched", "isrs_set_tile", "isrs_last_launch_info"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def check(status: int, handle=None):
    if status != ISRS_OK:
        msg = ""
        if handle is not None:
            raw = load().isrs_last_error(handle)
            msg = raw.decode() if raw else ""
        raise IsrsError(status, msg)
