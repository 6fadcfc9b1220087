"""ctypes binding of the C ABI declared in include/grf.h.

Argument marshalling only: every step of the computation runs inside
libgrf.so.  Importing this module loads the library and fails loudly if it
has not been built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# GRF_LIBRARY=checked selects the build with device-side index checks
# (libgrf_checked.so, same entry points); anything else the release build.
CHECKED = os.environ.get("GRF_LIBRARY", "") == "checked"
LIB_PATH = os.path.join(_HERE, "libgrf_checked.so" if CHECKED else "libgrf.so")

GRF_OK = 0
GRF_EINVAL = -1
GRF_EWORKSPACE = -2
GRF_ECUDA = -3
GRF_ETIMEOUT = -4
GRF_ENOMEM = -5
GRF_EDEVICE = -6

GRF_GAUSSIAN = 0
GRF_EXPONENTIAL = 1
GRF_MATERN = 2

GRF_MAP_Y = 1
GRF_MAP_LOGNORMAL = 2
GRF_MAP_FACIES = 4
GRF_MAP_VALUES = 8
GRF_MAP_POROSITY = 16
GRF_MAX_THRESHOLDS = 15
GRF_MAX_MODES = 1 << 24

c_dp = ctypes.POINTER(ctypes.c_double)
c_fp = ctypes.POINTER(ctypes.c_float)
c_u8p = ctypes.POINTER(ctypes.c_uint8)


class grf_params(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int32), ("dim", ctypes.c_int32), ("nu", ctypes.c_double),
                ("sigma2", ctypes.c_double), ("mean", ctypes.c_double), ("ell", ctypes.c_double * 3),
                ("n_modes", ctypes.c_int64), ("seed", ctypes.c_uint64), ("stream", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("period", ctypes.c_double * 3), ("rot", ctypes.c_double * 9)]


class grf_modes(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("dim", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("kappa", c_dp), ("rho", c_dp), ("psi", c_dp), ("a", c_dp), ("amp", c_dp)]


class grf_map(ctypes.Structure):
    _fields_ = [("bits", ctypes.c_int32), ("n_thresholds", ctypes.c_int32),
                ("thresholds", ctypes.c_float * GRF_MAX_THRESHOLDS),
                ("values", ctypes.c_float * (GRF_MAX_THRESHOLDS + 1)), ("k_ref", ctypes.c_float),
                ("phi0", ctypes.c_float), ("phi1", ctypes.c_float), ("phi_min", ctypes.c_float),
                ("phi_max", ctypes.c_float)]


class grf_outputs(ctypes.Structure):
    _fields_ = [("Y", ctypes.c_void_p), ("K", ctypes.c_void_p), ("facies", ctypes.c_void_p),
                ("prop", ctypes.c_void_p)]


class grf_grads(ctypes.Structure):
    _fields_ = [("dA", ctypes.c_void_p), ("dpsi", ctypes.c_void_p), ("da", ctypes.c_void_p),
                ("dmu", ctypes.c_void_p), ("dsigma", ctypes.c_void_p), ("dell", ctypes.c_void_p),
                ("drot", ctypes.c_void_p), ("dsigma2", ctypes.c_void_p), ("drho", ctypes.c_void_p),
                ("dkappa", ctypes.c_void_p), ("gscale", ctypes.c_void_p)]


class grf_bimap(ctypes.Structure):
    _fields_ = [("n_t", ctypes.c_int32), ("n_s", ctypes.c_int32),
                ("t", ctypes.c_float * GRF_MAX_THRESHOLDS), ("s", ctypes.c_float * GRF_MAX_THRESHOLDS),
                ("rule", (ctypes.c_uint8 * (GRF_MAX_THRESHOLDS + 1)) * (GRF_MAX_THRESHOLDS + 1)),
                ("values", ctypes.c_float * 256)]


class grf_batch_item(ctypes.Structure):
    _fields_ = [("table", ctypes.c_void_p), ("n_modes", ctypes.c_int64), ("dim", ctypes.c_int32),
                ("segment", ctypes.c_int32), ("mean", ctypes.c_double), ("sigma", ctypes.c_double),
                ("map", grf_map), ("out", grf_outputs)]


# name -> (restype, argtypes)
_SIGS = {
    "grf_last_error": (ctypes.c_char_p, []),
    "grf_version": (ctypes.c_char_p, []),
    "grf_gen_modes": (ctypes.c_int, [ctypes.POINTER(grf_params), ctypes.POINTER(grf_modes)]),
    "grf_reparam_modes": (ctypes.c_int, [ctypes.POINTER(grf_params), ctypes.POINTER(grf_modes)]),
    "grf_table_bytes": (ctypes.c_size_t, [ctypes.c_int64]),
    "grf_prefetch_create": (ctypes.c_int, [ctypes.POINTER(grf_params), ctypes.c_int32, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "grf_prefetch_next": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "grf_prefetch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "grf_pack_table": (ctypes.c_int, [ctypes.POINTER(grf_modes), ctypes.c_void_p, ctypes.c_size_t]),
    "grf_upload_table": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "grf_plan_bytes": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int32]),
    "grf_plan_cells": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_size_t, ctypes.c_void_p]),
    "grf_read_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]),
    "grf_synth_field": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(grf_params), ctypes.c_void_p,
                                       ctypes.c_int32, ctypes.POINTER(grf_map),
                                       ctypes.POINTER(grf_outputs), ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.c_void_p]),
    "grf_synth_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64]),
    "grf_synth_grid_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]),
    "grf_plan_grid_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "grf_map_property": (ctypes.c_int, [ctypes.POINTER(grf_map), ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(grf_outputs),
                                        ctypes.c_void_p]),
    "grf_map_bitruncated": (ctypes.c_int, [ctypes.POINTER(grf_bimap), ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "grf_backward_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32]),
    "grf_backward_grid_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]),
    "grf_synth_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(grf_params), ctypes.c_void_p,
                                          ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(grf_grads),
                                          ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "grf_synth_mismatch": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(grf_params), ctypes.c_void_p,
                                          ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_size_t, ctypes.c_void_p]),
    "grf_synth_mismatch_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64]),
    "grf_mismatch_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64]),
    "grf_mismatch_grad": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "grf_mismatch_grad_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p]),
    "grf_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int64]),
    "grf_batch_prepare": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(grf_batch_item), ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "grf_batch_autotune": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(grf_batch_item), ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)]),
    "grf_batch_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "grf_device_info": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "grf_launch_count": (ctypes.c_int64, []),
    "grf_take_path_counts": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "grf_take_adjoint_path_counts": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64),
                                                    ctypes.POINTER(ctypes.c_int64)]),
    "grf_debug_inject_alloc_failures": (ctypes.c_int, [ctypes.c_int32]),
    "grf_release": (ctypes.c_int, [ctypes.c_void_p]),
    "grf_selftest_wait": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "grf_mufu_probe": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "grf_take_grid_tiles": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64)]),
    "grf_take_grid_adjoint_units": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64)]),
    "grf_debug_grid_path": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32]),
    "grf_debug_mma_f16": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "grf_checked_build": (ctypes.c_int, []),
    "grf_take_index_faults": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int64)]),
}

_lib = None


class GRFError(RuntimeError):
    def __init__(self, code, message):
        super().__init__("%s (code %d)" % (message, code))
        self.code = code


def lib():
    """The loaded library (libgrf.so, or libgrf_checked.so under
    GRF_LIBRARY=checked); raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("%s not found: build it with __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc):
    """Raise GRFError with the library's message for a non-zero status."""
    if rc != GRF_OK:
        raise GRFError(rc, lib().grf_last_error().decode())
    return rc


def exported_symbols():
    return sorted(_SIGS)
