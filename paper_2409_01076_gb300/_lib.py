"""ctypes loader for libsmrt.so (the C ABI of include/smrt.h).

The library is built in-tree by build_lib.py.  There is no fallback: if the
shared library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import threading

from . import build_lib

_lock = threading.Lock()
_lib: ctypes.CDLL | None = None

c_int, c_uint, c_double, c_longlong, c_size_t, c_void_p, c_char_p = (
    ctypes.c_int, ctypes.c_uint, ctypes.c_double, ctypes.c_longlong, ctypes.c_size_t,
    ctypes.c_void_p, ctypes.c_char_p)

# (name, restype, argtypes) for every function declared in include/smrt.h
SIGNATURES = [
    ("smrt_create", c_int, [c_int, c_int, c_double, c_double, c_uint, ctypes.POINTER(c_void_p)]),
    ("smrt_set_option", c_int, [c_void_p, c_int, c_double]),
    ("smrt_get_option", c_int, [c_void_p, c_int, ctypes.POINTER(c_double)]),
    ("smrt_set_stream", c_int, [c_void_p, c_void_p]),
    ("smrt_step", c_int, [c_void_p, c_longlong]),
    ("smrt_sync", c_int, [c_void_p]),
    ("smrt_macros", c_int, [c_void_p, c_void_p, c_void_p]),
    ("smrt_residual", c_int, [c_void_p, c_void_p, c_void_p]),
    ("smrt_residual_noalloc", c_int, [c_void_p, c_int, c_int, c_double, c_double, c_uint, c_int, c_double,
                                      c_void_p, c_void_p]),
    ("smrt_get_f", c_int, [c_void_p, c_void_p]),
    ("smrt_set_f", c_int, [c_void_p, c_void_p]),
    ("smrt_init_macros", c_int, [c_void_p, c_void_p, c_void_p]),
    ("smrt_time", c_longlong, [c_void_p]),
    ("smrt_set_time", c_int, [c_void_p, c_longlong]),
    ("smrt_device_bytes", c_size_t, [c_void_p]),
    ("smrt_last_error", c_char_p, [c_void_p]),
    ("smrt_destroy", None, [c_void_p]),
    ("smrt_batch_create", c_int, [c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_uint, c_int, c_int, c_int,
                                  ctypes.POINTER(c_void_p)]),
    ("smrt_batch_set_stream", c_int, [c_void_p, c_void_p]),
    ("smrt_batch_autotune", c_int, [c_void_p, c_int, ctypes.POINTER(c_int)]),
    ("smrt_batch_set_shape", c_int, [c_void_p, c_int]),
    ("smrt_batch_step", c_int, [c_void_p, c_longlong]),
    ("smrt_batch_run", c_int, [c_void_p, c_double, c_longlong, c_longlong, c_int, ctypes.POINTER(c_int)]),
    ("smrt_batch_status", c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("smrt_batch_get_f", c_int, [c_void_p, c_int, c_void_p]),
    ("smrt_batch_macros", c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    ("smrt_batch_init_macros", c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    ("smrt_batch_nodes", c_longlong, [c_void_p]),
    ("smrt_batch_last_error", c_char_p, [c_void_p]),
    ("smrt_batch_destroy", None, [c_void_p]),
    # include/smrt_nn.h
    ("smrt_nn_gemm", c_int, [c_int, c_int, c_int, c_int, c_int, ctypes.c_float, c_void_p, c_int, c_void_p, c_int,
                             ctypes.c_float, c_void_p, c_int, c_int, c_void_p]),
    ("smrt_nn_gemm_tc", c_int, [c_int, c_int, c_int, c_int, c_int, ctypes.c_float, c_void_p, c_int, c_void_p, c_int,
                                ctypes.c_float, c_void_p, c_int, c_int, c_void_p, c_void_p]),
    ("smrt_nn_conv3_tc", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_int, ctypes.c_float,
                                 ctypes.c_float, c_void_p, c_int, c_void_p, c_void_p]),
    ("smrt_nn_to_half_blocked", c_int, [c_void_p, c_int, c_int, c_int, c_int, ctypes.c_float, c_void_p, c_void_p]),
    ("smrt_nn_to_half_blocked_pad", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, ctypes.c_float, c_void_p,
                                            c_void_p]),
    ("smrt_nn_pad3", c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]),
    ("smrt_nn_unpad3_add", c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]),
    ("smrt_nn_pack3_halves", c_longlong, [c_int, c_int]),
    ("smrt_nn_pack3", c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    ("smrt_nn_conv3_tma", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_int, ctypes.c_float,
                                  ctypes.c_float, c_void_p, c_int, c_void_p, c_void_p]),
    ("smrt_nn_check", c_int, [c_void_p, c_void_p]),
    ("smrt_nn_pack3_many", c_int, [c_int, c_void_p, c_void_p]),
    ("smrt_nn_conv3_tma_act_bwd", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_int, c_void_p, c_int,
                                          c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("smrt_nn_conv3_tma_wait_test", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_int, c_void_p, c_int,
                                            c_void_p, c_double, c_void_p]),
    ("smrt_nn_conv3_tma_bias_act", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_int, c_void_p, c_int,
                                           c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("smrt_nn_conv3_wgrad_tma", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_int, ctypes.c_float,
                                        c_void_p, c_int, c_void_p, c_void_p]),
    ("smrt_nn_im2col3", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_int, c_void_p]),
    ("smrt_nn_col2im3", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p]),
    ("smrt_nn_flip3", c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    ("smrt_nn_to_half", c_int, [c_void_p, c_longlong, ctypes.c_float, c_void_p, c_void_p]),
    ("smrt_nn_to_half_rows", c_int, [c_void_p, c_longlong, c_int, ctypes.c_float, c_void_p, c_int, c_void_p]),
    ("smrt_nn_bias_act", c_int, [c_void_p, c_void_p, c_longlong, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    ("smrt_nn_bias_act_bwd", c_int, [c_void_p, c_void_p, c_longlong, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    ("smrt_nn_bias_act_blocked", c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_int, c_void_p, c_void_p,
                                         c_void_p, c_void_p]),
    ("smrt_nn_bias_act_bwd_blocked", c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_int, c_void_p,
                                             c_void_p, c_void_p, c_void_p]),
    ("smrt_nn_bias_act_bwd_addpool_blocked", c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_int,
                                                     c_void_p, c_void_p, c_void_p, c_void_p]),
    ("smrt_nn_avgpool2_blocked", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    ("smrt_nn_upcat", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    ("smrt_nn_upcat_bwd", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    ("smrt_nn_conv1x1_small", c_int, [c_void_p, c_longlong, c_int, c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    ("smrt_nn_conv1x1_small_bwd", c_int, [c_void_p, c_void_p, c_longlong, c_int, c_void_p, c_int, c_void_p, c_void_p,
                                          c_void_p, c_void_p]),
    ("smrt_nn_avgpool2", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p]),
    ("smrt_nn_avgpool2_bwd", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p]),
    ("smrt_nn_upsample2", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p]),
    ("smrt_nn_upsample2_bwd", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p]),
    ("smrt_nn_concat", c_int, [c_void_p, c_int, c_void_p, c_int, c_longlong, c_void_p, c_void_p]),
    ("smrt_nn_concat_bwd", c_int, [c_void_p, c_int, c_int, c_longlong, c_void_p, c_void_p, c_void_p]),
    ("smrt_nn_add", c_int, [c_void_p, c_void_p, c_longlong, c_void_p, c_void_p]),
    ("smrt_nn_mse", c_int, [c_void_p, c_void_p, c_longlong, ctypes.c_float, c_void_p, c_void_p, c_void_p]),
    ("smrt_nn_adam", c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_longlong, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, ctypes.c_float, c_int, ctypes.c_float, c_void_p, c_void_p]),
    ("smrt_nn_resize_bilinear", c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_int, c_int, c_void_p]),
]


def path() -> str:
    return build_lib.LIB


def load() -> ctypes.CDLL:
    """Build (if stale) and load libsmrt.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            lib_path = build_lib.build()
            L = ctypes.CDLL(lib_path)
            for name, res, args in SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib
