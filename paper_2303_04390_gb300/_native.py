"""ctypes binding of libphylograd's C ABI (include/phylo_api.h).

Argument marshalling only: every step of an evaluation runs in the CUDA
library.  The functions keep the C names.  Loading fails loudly when the
library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libphylograd.so")

PHYLO_OK = 0
PHYLO_EINVAL = -1
PHYLO_ENOMEM = -2
PHYLO_ECUDA = -3
PHYLO_ESTATE = -4
PHYLO_ENUMERIC = -5
PHYLO_ETIMEOUT = -6
PHYLO_FP64 = 0
PHYLO_FP32 = 1
PHYLO_FLAG_TIP_PARTIALS = 1
PHYLO_FLAG_NO_GRAPH = 2

_c_int = ctypes.c_int
_c_size = ctypes.c_size_t
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)

# name -> (restype, argtypes); the order follows include/phylo_api.h
SIGNATURES = {
    "phylo_workspace_bytes": (_c_int, [_c_int, _c_int, _c_int, _c_int, _c_int,
                                       _c_int, ctypes.POINTER(_c_size)]),
    "phylo_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _c_int, _c_int,
                              _c_int, _c_int, _c_int, _vp, _c_size, _vp]),
    "phylo_set_tree": (_c_int, [_vp, _ip]),
    "phylo_set_tip_states": (_c_int, [_vp, _u8p]),
    "phylo_set_tip_partials": (_c_int, [_vp, _c_int, _dp]),
    "phylo_set_pattern_weights": (_c_int, [_vp, _dp]),
    "phylo_set_eigen": (_c_int, [_vp, _dp, _dp, _dp, _dp]),
    "phylo_set_rate_matrix": (_c_int, [_vp, _dp, _dp]),
    "phylo_eigen_reversible": (_c_int, [_c_int, _dp, _dp, _dp, _dp, _dp]),
    "phylo_set_categories": (_c_int, [_vp, _dp, _dp]),
    "phylo_set_branch_lengths": (_c_int, [_vp, _vp, _c_int]),
    "phylo_evaluate": (_c_int, [_vp, _dp, _dp]),
    "phylo_evaluate_device": (_c_int, [_vp, _vp]),
    "phylo_evaluate_device_timed": (_c_int, [_vp, _vp,
                                             ctypes.POINTER(_vp)]),
    "phylo_forward_device": (_c_int, [_vp, _vp,
                                      ctypes.POINTER(ctypes.c_uint64)]),
    "phylo_backward_device": (_c_int, [_vp, _vp, ctypes.c_uint64]),
    "phylo_gradient_rate_time": (_c_int, [_vp, _vp, _vp, _vp, _vp, _c_int]),
    "phylo_gradient_heights": (_c_int, [_vp, _vp, _vp, _c_int]),
    "phylo_gradient_branch_sum": (_c_int, [_vp, _vp, _vp, _c_int, _vp, _c_int]),
    "phylo_check": (_c_int, [_vp]),
    "phylo_launches_per_evaluation": (_c_int, [_vp]),
    "phylo_level_counts": (_c_int, [_vp, ctypes.POINTER(_c_int),
                                    ctypes.POINTER(_c_int)]),
    "phylo_selftest_bounded_wait": (_c_int, [_c_int, _vp]),
    "phylo_last_error": (ctypes.c_char_p, [_vp]),
    "phylo_destroy": (_c_int, [_vp]),
    "phylo_evaluate_noalloc": (_c_int, [_c_int, _c_int, _c_int, _c_int, _ip,
                                        _u8p, _dp, _dp, _dp, _dp, _dp, _dp,
                                        _dp, _dp, _dp, _dp, _vp,
                                        ctypes.c_char_p, _c_size]),
}

_lib = None


class PhyloError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"[{code}] {message}")
        self.code = code


def load() -> ctypes.CDLL:
    """Load libphylograd.so (built by paper_2303_04390_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: the CUDA library has not been built "
            "(run paper_2303_04390_gb300.build.build()); there is no CPU "
            "fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int, ctx=None) -> None:
    if rc != PHYLO_OK:
        msg = load().phylo_last_error(ctx)
        raise PhyloError(rc, msg.decode() if msg else "")


def __getattr__(name):
    # phylo_* functions are exposed under their C names.
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)
