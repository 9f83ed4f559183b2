"""ctypes loader for libjl.so (argument marshalling only).

The shared library is built in-tree by ``paper_1611_03079_b300.build``.  If it
is missing, loading raises ``RuntimeError`` -- there is no fallback path.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjl.so")

JL_OK, JL_EINVAL, JL_ECUDA, JL_ENOMEM, JL_ETIMEOUT, JL_EUNSUPPORTED = range(6)
JL_FP32, JL_FP64, JL_AUTO = 0, 1, 2
JL_JULIA, JL_MANDELBROT = 0, 1
JL_COUNT_NONE, JL_COUNT_U8, JL_COUNT_U16 = 0, 1, 2

STATUS_NAMES = {0: "JL_OK", 1: "JL_EINVAL", 2: "JL_ECUDA", 3: "JL_ENOMEM", 4: "JL_ETIMEOUT",
                5: "JL_EUNSUPPORTED"}


class JLError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, str(code)), msg))
        self.code = code


class Rect(ctypes.Structure):
    _fields_ = [("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("ymin", ctypes.c_double), ("ymax", ctypes.c_double)]


class Frame(ctypes.Structure):
    """jl_frame (include/jl.h)."""
    _fields_ = [("cr", ctypes.c_double), ("ci", ctypes.c_double), ("rect", Rect),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("precision", ctypes.c_int32), ("count_type", ctypes.c_int32),
                ("counts_offset", ctypes.c_int64), ("rgba_offset", ctypes.c_int64),
                ("hist_offset", ctypes.c_int64)]


class BatchOpts(ctypes.Structure):
    """jl_batch_opts (include/jl.h)."""
    _fields_ = [("chunk_len", ctypes.c_int32), ("fp32_ppt", ctypes.c_int32), ("fp32_unroll", ctypes.c_int32),
                ("fp32_threads", ctypes.c_int32), ("fp64_ppt", ctypes.c_int32), ("fp64_unroll", ctypes.c_int32),
                ("fp64_threads", ctypes.c_int32), ("variant_flags", ctypes.c_int32),
                ("tune", ctypes.c_int32), ("cycle_budget", ctypes.c_int64)]


class Map(ctypes.Structure):
    """jl_map (include/jl.h)."""
    _fields_ = [("kind", ctypes.c_int32), ("degree", ctypes.c_int32), ("num_degree", ctypes.c_int32),
                ("den_degree", ctypes.c_int32), ("num", ctypes.c_double * 18), ("den", ctypes.c_double * 18),
                ("bailout", ctypes.c_double), ("z0r", ctypes.c_double), ("z0i", ctypes.c_double)]


class TuneResult(ctypes.Structure):
    """jl_tune_result (include/jl.h)."""
    _fields_ = [("ppt", ctypes.c_int32), ("unroll", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("ms", ctypes.c_double), ("candidates", ctypes.c_int32)]


_lib = None

# Every entry point declared in include/*.h, with its ctypes signature.
_d, _i32, _vp, _u64 = ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint64
SIGNATURES = {
    "jl_last_error": (ctypes.c_char_p, []),
    "jl_version": (ctypes.c_char_p, []),
    "jl_select_precision": (ctypes.c_int, [Rect, _i32, _i32]),
    "jl_default_palette": (ctypes.c_int, [_vp]),
    "jl_render": (ctypes.c_int, [_d, _d, Rect, _i32, _i32, _i32, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp]),
    "jl_render_frames_to_host": (ctypes.c_int, [ctypes.c_void_p, _i32, _vp, _vp, _vp, _vp, _i32, _vp]),
    "jl_host_plan_create": (ctypes.c_int, [ctypes.c_void_p, _i32, _vp, _vp, _vp, _vp, _i32,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "jl_host_plan_run": (ctypes.c_int, [_vp, _vp]),
    "jl_host_plan_destroy": (None, [_vp]),
    "jl_host_plan_launches": (_i32, [_vp]),
    "jl_render_map": (ctypes.c_int, [ctypes.POINTER(Map), _d, _d, Rect, _i32, _i32, _i32, _i32, _i32, _i32, _vp,
                                     _vp, _vp, _vp, _vp]),
    "jl_render_variant": (ctypes.c_int, [_d, _d, Rect, _i32, _i32, _i32, _i32, _i32, _i32, _vp, _vp, _vp,
                                         _vp, _i32, _i32, _i32, _i32, _vp]),
    "jl_render_static": (ctypes.c_int, [_d, _d, Rect, _i32, _i32, _i32, _i32, _i32, _i32, _vp, _vp, _vp, _vp,
                                        _vp]),
    "jl_variant_list": (ctypes.c_int, [_i32, _vp, _i32]),
    "jl_probe_peak": (ctypes.c_int, [_i32, _i32, _vp, _vp, _vp]),
    "jl_batch_create": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "jl_batch_variant": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "jl_batch_launch": (ctypes.c_int, [_vp, _vp]),
    "jl_batch_status": (ctypes.c_int, [_vp, _vp, _vp]),
    "jl_batch_precisions": (ctypes.c_int, [_vp, _vp, _i32]),
    "jl_batch_pixels": (ctypes.c_int, [_vp, _vp, _vp]),
    "jl_batch_cert_stats": (ctypes.c_int, [_vp, _vp, _vp]),
    "jl_batch_phase_ms": (ctypes.c_int, [_vp, _vp]),
    "jl_batch_destroy": (None, [_vp]),
    "jl_render_batch": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp]),
    "jl_autotune": (ctypes.c_int, [_i32, _i32, _vp, _i32, _i32, _vp]),
    "jl_tune_get": (ctypes.c_int, [_i32, _i32, _vp]),
    "jl_tune_clear": (ctypes.c_int, []),
    "jl_tune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "jl_tune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "jl_model_num_params": (ctypes.c_int, []),
    "jl_model_create": (ctypes.c_int, [_vp, _vp, _vp]),
    "jl_model_destroy": (None, [_vp]),
    "jl_model_get_state": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "jl_model_set_state": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "jl_model_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp, _vp, _vp]),
    "jl_model_forward_layered": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp, _vp, _vp]),
    "jl_model_grads": (ctypes.c_int, [_vp, _vp, _vp, _i32, _vp, _vp, _vp]),
    "jl_train": (ctypes.c_int, [_vp, _vp, _vp, _i32, _vp, _i32, _i32, ctypes.c_float, ctypes.c_float, _vp, _vp]),
    "jl_topk": (ctypes.c_int, [_vp, ctypes.c_int64, _i32, _vp, _vp, _vp]),
    "jl_survey": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _i32, _vp, _vp, _vp, _vp]),
    "jl_hist_l1": (ctypes.c_int, [_vp, _i32, _vp, _i32, _i32, _i32, _vp, _vp]),
    "jl_model_save": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "jl_model_load": (ctypes.c_int, [ctypes.c_char_p, _vp]),
    "jl_gemm_bf16": (ctypes.c_int, [_vp, _i32, _i32, _vp, _i32, _i32, _i32, _i32, _i32, _vp, _i32, _vp, _vp]),
    "jl_selftest_double": (ctypes.c_int, [_vp, _vp, _i32, _vp]),
    "jl_render_to_host": (ctypes.c_int, [_d, _d, Rect, _i32, _i32, _i32, _i32, _i32, _i32, _vp, _vp, _vp,
                                         _vp, _vp]),
}


def lib():
    """Load libjl.so once; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libjl.so not found at %s; run python -m paper_1611_03079_b300.build"
                               % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc):
    if rc != JL_OK:
        msg = lib().jl_last_error()
        raise JLError(rc, msg.decode() if msg else "")
    return rc
