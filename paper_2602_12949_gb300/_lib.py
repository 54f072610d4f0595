"""ctypes binding of libniv.so (argument marshalling only; every step runs in the library).

The shared library is built in-tree by ``paper_2602_12949_gb300.build.build()``.
Loading fails loudly when it is missing: there is no fallback implementation.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libniv.so")

NIV_OK = 0
NIV_ERR_ARG = -1
NIV_ERR_ALIGN = -2
NIV_ERR_CUDA = -3
NIV_ERR_UNSUPPORTED = -4
NIV_ERR_DEVICE = -5
NIV_ERR_NOMEM = -6

NIV_FP32, NIV_FP16, NIV_FP8 = 0, 1, 2
NIV_MC_TOTAL, NIV_MC_INDIRECT = 0, 1
NIV_F32, NIV_F16 = 0, 1


class NivError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("niv error %d: %s" % (code, msg))
        self.code = code


class ModelDesc(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int32), ("levels", ctypes.c_int32), ("feat", ctypes.c_int32),
        ("log2_T", ctypes.c_int32), ("base", ctypes.c_double), ("growth", ctypes.c_double),
        ("n_hidden", ctypes.c_int32), ("width", ctypes.c_int32), ("in_extra", ctypes.c_int32),
        ("out_dim", ctypes.c_int32), ("out_act", ctypes.c_int32), ("prime_t", ctypes.c_uint32),
        ("pe_bands", ctypes.c_int32), ("t_bands", ctypes.c_int32),
    ]


class QueryParams(ctypes.Structure):
    _fields_ = [("aabb_min", ctypes.c_float * 3), ("aabb_max", ctypes.c_float * 3), ("t", ctypes.c_float),
                ("image_width", ctypes.c_int32)]


class UpsampleParams(ctypes.Structure):
    _fields_ = [("power", ctypes.c_float), ("sigma", ctypes.c_float), ("eps", ctypes.c_float)]


class FitParams(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("adam_eps", ctypes.c_float), ("loss_eps", ctypes.c_float)]


_lib = None

# (name, restype, argtypes); pointer arguments are passed as integers (c_void_p).
_VP, _I32, _I64, _F, _D, _U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double, ctypes.c_uint64
_U32 = ctypes.c_uint32
_SIGNATURES = [
    ("niv_version", ctypes.c_char_p, []),
    ("niv_last_error", ctypes.c_char_p, []),
    ("niv_sync_status", ctypes.c_int, [_VP]),
    ("niv_create", ctypes.c_int, [ctypes.POINTER(ModelDesc), ctypes.POINTER(_VP)]),
    ("niv_destroy", ctypes.c_int, [_VP]),
    ("niv_level_info", ctypes.c_int, [_VP, _I32, _VP, _VP, _VP, _VP]),
    ("niv_param_count", ctypes.c_int, [_VP, _VP, _VP]),
    ("niv_set_params", ctypes.c_int, [_VP, _VP, _I64, _VP]),
    ("niv_get_params", ctypes.c_int, [_VP, _VP, _I64, _VP]),
    ("niv_save", ctypes.c_int, [_VP, ctypes.c_char_p, _VP]),
    ("niv_load", ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_VP)]),
    ("niv_query", ctypes.c_int, [_VP, _VP, _VP, _I64, _I32, ctypes.POINTER(QueryParams), _VP, _I32, _I32, _VP]),
    ("niv_query_host", ctypes.c_int, [_VP, _VP, _VP, _I64, _I32, ctypes.POINTER(QueryParams), _VP, _I32, _I32, _VP]),
    ("niv_mc_irradiance", ctypes.c_int, [_VP, _I64, _VP, _VP, _VP, _I64, _I32, _U64, _U64, _I32, _VP, _VP, _VP]),
    ("niv_compact_targets", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("niv_probe_bake", ctypes.c_int, [_VP, _I64, _VP, _VP, _VP, _I32, _U64, _U64, _VP, _VP, _VP]),
    ("niv_probe_query", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _I64, _I32, _VP, _I32, _I32, _VP]),
    ("niv_grad", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _I64, ctypes.POINTER(QueryParams), _F, _VP, _VP]),
    ("niv_get_grads", ctypes.c_int, [_VP, _VP, _I64, _VP]),
    ("niv_set_train_forward", ctypes.c_int, [_VP, _I32]),
    ("niv_backward", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _I64, ctypes.POINTER(QueryParams), _VP]),
    ("niv_set_grads", ctypes.c_int, [_VP, _VP, _I64, _VP]),
    ("niv_adam_step", ctypes.c_int, [_VP, _F, _F, _F, _F, _VP]),
    ("niv_fit", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _I64, ctypes.POINTER(QueryParams), ctypes.POINTER(FitParams), _VP, _VP]),
    ("niv_fp8_calibrate", ctypes.c_int, [_VP, _VP, _VP, _I64, _I32, ctypes.POINTER(QueryParams), _VP]),
    ("niv_fp8_get_scales", ctypes.c_int, [_VP, _VP, _VP, _VP, _I32]),
    ("niv_query_shade", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _I64, _I32, ctypes.POINTER(QueryParams), _VP, _I32, _VP]),
    ("niv_query_host_noalloc", ctypes.c_int, [_VP, _VP, _VP, _I64, _I32, ctypes.POINTER(QueryParams), _VP, _I32, _I32, _VP]),
    ("niv_encode", ctypes.c_int, [_VP, _VP, _I64, _I32, ctypes.POINTER(QueryParams), _VP, _VP, _VP]),
    ("niv_selftest_mma", ctypes.c_int, [_I32, _VP, _VP]),
    ("niv_selftest_wait_expiry", ctypes.c_int, [_U32, _VP]),
    ("niv_selftest_philox", ctypes.c_int, [_VP, _I64, _VP, _VP]),
    ("niv_training_samples", ctypes.c_int, [_VP, _I64, _I64, _F, _U64, _U64, _VP, _VP, _VP, _VP, _VP]),
    ("niv_gbuffer_raycast", ctypes.c_int, [_VP, _I64, _I32, _I32, _D, _VP, _F, _VP, _VP, _VP, _I32, _VP, _VP]),
    ("niv_gbuffer_meshes", ctypes.c_int, [_VP, _VP, _I64, _VP, _I32, _I32, _I32, _D, _VP, _VP, _VP, _VP, _I32, _VP,
                                          _VP, _VP, _VP]),
    ("niv_shade", ctypes.c_int, [_VP, _VP, _VP, _I64, _VP, _VP]),
    ("niv_dyn_create", ctypes.c_int, [_VP, _I64, ctypes.POINTER(_VP)]),
    ("niv_dyn_destroy", ctypes.c_int, [_VP]),
    ("niv_dyn_node_count", _I64, [_VP]),
    ("niv_dyn_ao", ctypes.c_int, [_VP, _VP, _VP, _I64, _I32, _I32, _F, _U64, _VP, _VP, _I32, _VP]),
    ("niv_probe_query_rt", ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _I64, _F, _VP, _VP, _I64, _I32, _VP, _I32, _I32,
                                          _VP]),
    ("niv_query_sub", ctypes.c_int, [_VP, _VP, _VP, _I32, _I32, _I32, _I32, ctypes.POINTER(QueryParams), _VP, _I32,
                                     _I32, _VP]),
    ("niv_upsample_shade", ctypes.c_int, [_VP, _VP, _VP, _VP, _I32, _I32, _I32, _VP, _I32, _I32,
                                          ctypes.POINTER(UpsampleParams), _VP, _VP]),
]


def lib():
    """The loaded libniv.so (raises ImportError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libniv.so is not built (run paper_2602_12949_gb300.build.build()); "
                              "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            if hasattr(L, name):
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
        _lib = L
    return _lib


def check(rc):
    """Raise NivError for a failing status code."""
    if rc != NIV_OK:
        raise NivError(rc, lib().niv_last_error().decode())
    return rc
