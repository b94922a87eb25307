"""ctypes declarations of the libhopu C ABI (include/hopu.h, include/hopu_hex.h).

Argument marshalling only: there is no compute here and no fallback.  If the shared
library is missing, loading raises instead of silently doing something else.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, c_char_p, c_double, c_int, c_int64, c_void_p

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libhopu.so")

HOPU_OK, HOPU_EINVAL, HOPU_ENOMEM, HOPU_ECUDA, HOPU_EMESH, HOPU_ETIMEOUT, HOPU_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EMESH", -5: "ETIMEOUT", -6: "ENOTSUP"}
HOPU_FP64, HOPU_FP32, HOPU_FP32_TC, HOPU_TF32 = 0, 1, 2, 3
HOPU_HDIV_TO_L2, HOPU_L2_TO_HDIV, HOPU_L2_TO_HDIV_DUAL = 0, 1, 2
HOPU_WIND_STAGE, HOPU_WIND_FROZEN = 0, 1
KERNEL_FAMILIES = ["v2l", "facet", "volume", "l2v_elem", "l2v_facet", "facet_adj", "volume_adj"]


class MeshDesc(Structure):
    _fields_ = [
        ("dim", c_int),
        ("n_vertices", c_int64),
        ("coords", c_void_p),
        ("n_elems", c_int64),
        ("elem_vertices", c_void_p),
        ("vertex_rep", c_void_p),
    ]


class Options(Structure):
    _fields_ = [("k", c_int), ("l", c_int), ("prec", c_int), ("wind_mode", c_int), ("tile_hint", c_int)]


# name -> (restype, argtypes); the exact set of symbols the headers under include/ declare
SIGNATURES = {
    "hopu_create": (c_int, [POINTER(MeshDesc), POINTER(Options), c_void_p, POINTER(c_void_p)]),
    "hopu_destroy": (c_int, [c_void_p]),
    "hopu_set_stream": (c_int, [c_void_p, c_void_p]),
    "hopu_sizes": (c_int, [c_void_p, POINTER(c_int64), POINTER(c_int64), POINTER(c_int64)]),
    "hopu_project": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "hopu_apply_convection": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "hopu_apply_convection_l2": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "hopu_pack_elements": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    "hopu_unpack_elements": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    "hopu_rk_substep": (c_int, [c_void_p, c_void_p, c_double, c_int]),
    "hopu_set_frozen_wind": (c_int, [c_void_p, c_void_p]),
    "hopu_set_energy_log": (c_int, [c_void_p, c_void_p, c_int64]),
    "hopu_energy": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(c_double)]),
    "hopu_points": (c_int, [c_void_p, c_int, c_void_p, POINTER(c_int64)]),
    "hopu_interpolate": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "hopu_last_error": (c_char_p, [c_void_p]),
    "hopu_hex_create": (c_int, [c_int, c_int, c_int, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p,
                                POINTER(c_void_p)]),
    "hopu_hex_destroy": (c_int, [c_void_p]),
    "hopu_hex_sizes": (c_int, [c_void_p, POINTER(c_int64), POINTER(c_int64)]),
    "hopu_hex_apply": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "hopu_hex_rk_substeps": (c_int, [c_void_p, c_void_p, c_double, c_int, c_int]),
    "hopu_hex_set_inlet": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "hopu_hex_set_facet_l": (c_int, [c_void_p, c_void_p]),
    "hopu_hex_adapt_l": (c_int, [c_void_p, c_void_p, POINTER(c_double), c_void_p, c_void_p]),
    "hopu_hex_energy": (c_int, [c_void_p, c_void_p, c_void_p, c_int, POINTER(c_double)]),
    "hopu_hex_last_error": (c_char_p, [c_void_p]),
    "hopu_clear_error": (c_int, [c_void_p]),
    "hopu_selftest": (c_int, [c_int, c_int, POINTER(c_double)]),
    "hopu_profile": (c_int, [c_void_p, c_int]),
    "hopu_batch_create": (c_int, [c_void_p, c_void_p, c_int, POINTER(Options), c_void_p, POINTER(c_void_p)]),
    "hopu_batch_destroy": (c_int, [c_void_p]),
    "hopu_batch_classes": (c_int, [c_void_p, POINTER(c_int), c_void_p, c_void_p, c_void_p]),
    "hopu_batch_context": (c_int, [c_void_p, c_int, POINTER(c_void_p)]),
    "hopu_batch_layout": (c_int, [c_void_p, c_int, c_void_p]),
    "hopu_batch_rk_substep": (c_int, [c_void_p, c_void_p, c_double, c_int]),
    "hopu_batch_last_error": (c_char_p, [c_void_p]),
    "hopu_apply_convection_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "hopu_profile_read": (c_int, [c_void_p, POINTER(c_double), POINTER(c_int64)]),
    "hopu_measure_alu_peak": (c_int, [c_int, c_int, POINTER(c_double)]),
    "hopu_sync": (c_int, [c_void_p]),
    "hopu_set_wait_limit": (c_int, [c_void_p, c_int64]),
    "hopu_boundary_facets": (c_int, [c_void_p, c_void_p, POINTER(c_int64)]),
    "hopu_set_inlet": (c_int, [c_void_p, c_void_p, c_int64, c_void_p]),
    "hopu_tuning": (c_int, [c_void_p, POINTER(c_int)]),
    "hopu_tuning_volume": (c_int, [c_void_p, POINTER(c_int), POINTER(c_double)]),
    "hopu_set_volume_variant": (c_int, [c_void_p, c_int]),
    "hopu_tuning_l2v": (c_int, [c_void_p, POINTER(c_int), POINTER(c_double)]),
    "hopu_set_l2v_variant": (c_int, [c_void_p, c_int]),
    "hopu_set_facet_l": (c_int, [c_void_p, c_void_p]),
    "hopu_adapt_l": (c_int, [c_void_p, c_void_p, POINTER(c_double), c_void_p, c_void_p]),
    "hopu_vjp_apply": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "hopu_vjp_rollout": (c_int, [c_void_p, c_void_p, c_double, c_int, c_int, c_void_p, POINTER(c_double)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libhopu.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with paper_2408_06698_gb300.build.build() "
            "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class HopuError(RuntimeError):
    def __init__(self, status: int, where: str, text: str = ""):
        super().__init__(f"{where}: HOPU_{STATUS_NAMES.get(status, status)} {text}".rstrip())
        self.status = status
