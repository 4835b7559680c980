"""GB300 (sm_103a) D2Q9 SmrtLBM: Python binding of the C ABI in include/smrt.h.

Zhou, "Single MRT-featured Lattice Boltzmann Method (SmrtLBM)", arXiv 2409.01076.

Every function here has the name of the C entry point it calls and does only
argument marshalling: all lattice work runs in the CUDA kernels of libsmrt.so.
A status other than SMRT_OK raises SmrtError carrying the library's message.

Arrays passed in or out are float64, C-contiguous, and either host memory
(numpy arrays, CPU torch tensors -- pinned or not) or CUDA torch tensors on the
current device:  f (9, ny, nx), rho (ny, nx), u (2, ny, nx).
"""
from __future__ import annotations

import ctypes

from . import _lib
from .workloads import ALL_PERIODIC, CAVITY, CHANNEL, COUETTE, MOVING, PERIODIC, WALL, bc_flags

SMRT_OK, SMRT_ERR_ARG, SMRT_ERR_OOM, SMRT_ERR_CUDA = 0, -1, -2, -3
SMRT_ERR_DIVERGED, SMRT_ERR_TIMEOUT, SMRT_ERR_STATE = -4, -5, -6

SMRT_OPT_COLLISION, SMRT_OPT_TAU_S, SMRT_OPT_LAYOUT, SMRT_OPT_PRECISION = 1, 2, 3, 4
SMRT_OPT_CHECK_DIVERGENCE, SMRT_OPT_MEM_LIMIT, SMRT_OPT_TAU = 5, 6, 7
SMRT_COLLISION_SMRT, SMRT_COLLISION_SRT, SMRT_COLLISION_TWO_TAU = 0, 1, 2
SMRT_LAYOUT_AB, SMRT_LAYOUT_AA = 0, 1
SMRT_PREC_F64, SMRT_PREC_F32, SMRT_PREC_F16, SMRT_PREC_BF16 = 0, 1, 2, 3

_STATUS_NAMES = {0: "SMRT_OK", -1: "SMRT_ERR_ARG", -2: "SMRT_ERR_OOM", -3: "SMRT_ERR_CUDA",
                 -4: "SMRT_ERR_DIVERGED", -5: "SMRT_ERR_TIMEOUT", -6: "SMRT_ERR_STATE"}


class SmrtError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (_STATUS_NAMES.get(status, str(status)), message))
        self.status = status


def _check(rc: int, handle) -> None:
    if rc != SMRT_OK:
        raise SmrtError(rc, smrt_last_error(handle))


def _ptr(a, shape, name, writable):
    """Address of a float64 C-contiguous array (numpy or torch) of the given shape."""
    if a is None:
        return None
    mod = type(a).__module__
    if mod.startswith("torch"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("%s must be a contiguous float64 tensor" % name)
        if tuple(a.shape) != tuple(shape):
            raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(a.shape)))
        return ctypes.c_void_p(a.data_ptr())
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("%s must be a C-contiguous float64 numpy array or torch tensor" % name)
    if writable and not a.flags["WRITEABLE"]:
        raise ValueError("%s is read-only" % name)
    if a.shape != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), a.shape))
    return ctypes.c_void_p(a.ctypes.data)


class Handle:
    """An smrt_t* with its lattice size; destroyed when garbage-collected."""

    def __init__(self, ptr: int, nx: int, ny: int):
        self.ptr = ctypes.c_void_p(ptr)
        self.nx, self.ny = nx, ny

    def __del__(self):
        try:
            smrt_destroy(self)
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return self.ptr


def smrt_create(nx: int, ny: int, tau: float, u_lid: float = 0.0, bc: int = CAVITY) -> Handle:
    out = ctypes.c_void_p()
    rc = _lib.load().smrt_create(nx, ny, tau, u_lid, bc, ctypes.byref(out))
    if rc != SMRT_OK:
        raise SmrtError(rc, smrt_last_error(None))
    return Handle(out.value, nx, ny)


def smrt_set_option(h: Handle, key: int, value: float) -> None:
    _check(_lib.load().smrt_set_option(h, key, float(value)), h)


def smrt_get_option(h: Handle, key: int) -> float:
    v = ctypes.c_double()
    _check(_lib.load().smrt_get_option(h, key, ctypes.byref(v)), h)
    return v.value


def smrt_set_stream(h: Handle, stream=None) -> None:
    """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None (legacy default)."""
    raw = 0
    if stream is not None:
        raw = int(getattr(stream, "cuda_stream", stream))
    _check(_lib.load().smrt_set_stream(h, ctypes.c_void_p(raw)), h)


def smrt_step(h: Handle, n: int) -> None:
    _check(_lib.load().smrt_step(h, int(n)), h)


def smrt_sync(h: Handle) -> None:
    _check(_lib.load().smrt_sync(h), h)


def smrt_macros(h: Handle, rho=None, u=None) -> None:
    _check(_lib.load().smrt_macros(h, _ptr(rho, (h.ny, h.nx), "rho", True),
                                   _ptr(u, (2, h.ny, h.nx), "u", True)), h)


def smrt_residual(h: Handle) -> tuple[float, tuple[float, float, float]]:
    """Returns (r, (sum rho, sum rho ux, sum rho uy))."""
    r = ctypes.c_double()
    sums = (ctypes.c_double * 3)()
    _check(_lib.load().smrt_residual(h, ctypes.byref(r), sums), h)
    return r.value, (sums[0], sums[1], sums[2])


def smrt_residual_noalloc(f, tau: float, u_lid: float = 0.0, bc: int = CAVITY,
                          collision: int = SMRT_COLLISION_SMRT, tau_s: float = 1.0, out=None,
                          stream=None):
    """Residual of a caller-held canonical field, allocating nothing on the device.

    For callers that cannot call cudaMalloc (and so cannot create a handle):
    f is a CUDA float64 tensor (9, ny, nx) holding f(t).  `out` may be a CUDA
    float64 tensor of 4 elements (the call then only enqueues work) or None, in
    which case the call waits and returns (r, (sum rho, sum rho ux, sum rho uy)).
    """
    import numpy as np
    _, ny, nx = tuple(f.shape)
    fp = _ptr(f, (9, ny, nx), "f", False)
    raw = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    host = out is None
    res = np.empty(4) if host else out
    rc = _lib.load().smrt_residual_noalloc(fp, nx, ny, tau, u_lid, bc, collision, tau_s,
                                           _ptr(res, (4,), "out", True), ctypes.c_void_p(raw))
    if rc != SMRT_OK:
        raise SmrtError(rc, smrt_last_error(None))
    if host:
        return float(res[0]), (float(res[1]), float(res[2]), float(res[3]))
    return None


def smrt_get_f(h: Handle, f) -> None:
    _check(_lib.load().smrt_get_f(h, _ptr(f, (9, h.ny, h.nx), "f", True)), h)


def smrt_set_f(h: Handle, f) -> None:
    _check(_lib.load().smrt_set_f(h, _ptr(f, (9, h.ny, h.nx), "f", False)), h)


def smrt_init_macros(h: Handle, rho, u) -> None:
    _check(_lib.load().smrt_init_macros(h, _ptr(rho, (h.ny, h.nx), "rho", False),
                                        _ptr(u, (2, h.ny, h.nx), "u", False)), h)


def smrt_time(h: Handle) -> int:
    return int(_lib.load().smrt_time(h))


def smrt_set_time(h: Handle, t: int) -> None:
    _check(_lib.load().smrt_set_time(h, int(t)), h)


def smrt_device_bytes(h: Handle) -> int:
    return int(_lib.load().smrt_device_bytes(h))


def smrt_last_error(h) -> str:
    raw = _lib.load().smrt_last_error(h if h is not None else None)
    return raw.decode() if raw else ""


def smrt_destroy(h: Handle) -> None:
    if h is not None and h.ptr and h.ptr.value:
        _lib.load().smrt_destroy(h.ptr)
        h.ptr = ctypes.c_void_p()
