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
SMRT_OPT_CHECK_DIVERGENCE, SMRT_OPT_MEM_LIMIT, SMRT_OPT_TAU, SMRT_OPT_ROUNDING = 5, 6, 7, 8
SMRT_ROUND_NEAREST, SMRT_ROUND_STOCHASTIC = 0, 1
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
    """An smrt_t* with its lattice size, lid speed and boundary flags; destroyed when garbage-collected."""

    def __init__(self, ptr: int, nx: int, ny: int, u_lid: float = 0.0, bc: int = 0):
        self.ptr = ctypes.c_void_p(ptr)
        self.nx, self.ny = nx, ny
        self.u_lid, self.bc = float(u_lid), int(bc)

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
    return Handle(out.value, nx, ny, u_lid, bc)


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
    stream: a torch.cuda.Stream or raw cudaStream_t; None means torch's current
    stream, the one on which the caller's f was most likely written.
    """
    import numpy as np
    import torch
    if not (isinstance(f, torch.Tensor) and f.is_cuda):
        raise TypeError("f must be a CUDA float64 tensor of shape (9, ny, nx)")
    if out is not None and not (isinstance(out, torch.Tensor) and out.is_cuda):
        raise TypeError("out must be a CUDA float64 tensor of 4 elements (or None for a host result)")
    _, ny, nx = tuple(f.shape)
    fp = _ptr(f, (9, ny, nx), "f", False)
    if stream is None:
        stream = torch.cuda.current_stream(f.device)
    raw = int(getattr(stream, "cuda_stream", stream))
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


# ---- batches of independent lattices ------------------------------------------------

SMRT_BATCH_ACTIVE, SMRT_BATCH_CONVERGED, SMRT_BATCH_CAPPED, SMRT_BATCH_DIVERGED = 0, 1, 2, 3


class BatchHandle:
    """An smrt_batch_t* with the per-lattice sizes; destroyed when garbage-collected."""

    def __init__(self, ptr: int, nx, ny):
        self.ptr = ctypes.c_void_p(ptr)
        self.nx, self.ny = list(nx), list(ny)
        self.count = len(self.nx)

    def __del__(self):
        try:
            smrt_batch_destroy(self)
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return self.ptr


def _bcheck(rc: int, b) -> None:
    if rc != SMRT_OK:
        raise SmrtError(rc, smrt_batch_last_error(b))


def smrt_batch_create(nx, ny, tau, u_lid, bc: int = CAVITY, precision: int = SMRT_PREC_F32,
                      layout: int = SMRT_LAYOUT_AB, collision: int = SMRT_COLLISION_SMRT) -> BatchHandle:
    import numpy as np
    n = len(nx)
    if not (len(ny) == len(tau) == len(u_lid) == n):
        raise ValueError("nx, ny, tau, u_lid must have the same length")
    anx = np.ascontiguousarray(nx, dtype=np.int32)
    any_ = np.ascontiguousarray(ny, dtype=np.int32)
    atau = np.ascontiguousarray(tau, dtype=np.float64)
    au = np.ascontiguousarray(u_lid, dtype=np.float64)
    out = ctypes.c_void_p()
    rc = _lib.load().smrt_batch_create(n, anx.ctypes.data, any_.ctypes.data, atau.ctypes.data, au.ctypes.data,
                                       bc, precision, layout, collision, ctypes.byref(out))
    if rc != SMRT_OK:
        raise SmrtError(rc, smrt_batch_last_error(None))
    return BatchHandle(out.value, anx.tolist(), any_.tolist())


def smrt_batch_set_stream(b: BatchHandle, stream=None) -> None:
    raw = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    _bcheck(_lib.load().smrt_batch_set_stream(b, ctypes.c_void_p(raw)), b)


def smrt_batch_autotune(b: BatchHandle, steps: int = 10) -> int:
    choice = ctypes.c_int(-1)
    _bcheck(_lib.load().smrt_batch_autotune(b, int(steps), ctypes.byref(choice)), b)
    return choice.value


def smrt_batch_set_shape(b: BatchHandle, shape: int) -> None:
    _bcheck(_lib.load().smrt_batch_set_shape(b, int(shape)), b)


def smrt_batch_step(b: BatchHandle, n: int) -> None:
    _bcheck(_lib.load().smrt_batch_step(b, int(n)), b)


SMRT_BATCH_RESIDUAL_STEP, SMRT_BATCH_RESIDUAL_STRIDE = 0, 1


def smrt_batch_run(b: BatchHandle, tol: float, check_every: int, max_steps: int,
                   residual_kind: int = SMRT_BATCH_RESIDUAL_STEP) -> int:
    n_active = ctypes.c_int(-1)
    _bcheck(_lib.load().smrt_batch_run(b, float(tol), int(check_every), int(max_steps), int(residual_kind),
                                       ctypes.byref(n_active)), b)
    return n_active.value


def smrt_batch_status(b: BatchHandle):
    """Returns (steps[count] int64, residual[count] float64, state[count] int32)."""
    import numpy as np
    steps = np.empty(b.count, dtype=np.int64)
    res = np.empty(b.count, dtype=np.float64)
    state = np.empty(b.count, dtype=np.int32)
    _bcheck(_lib.load().smrt_batch_status(b, steps.ctypes.data, res.ctypes.data, state.ctypes.data), b)
    return steps, res, state


def smrt_batch_get_f(b: BatchHandle, k: int, f) -> None:
    _bcheck(_lib.load().smrt_batch_get_f(b, int(k), _ptr(f, (9, b.ny[k], b.nx[k]), "f", True)), b)


def smrt_batch_macros(b: BatchHandle, k: int, rho, u) -> None:
    _bcheck(_lib.load().smrt_batch_macros(b, int(k), _ptr(rho, (b.ny[k], b.nx[k]), "rho", True),
                                          _ptr(u, (2, b.ny[k], b.nx[k]), "u", True)), b)


def smrt_batch_init_macros(b: BatchHandle, k: int, rho, u) -> None:
    _bcheck(_lib.load().smrt_batch_init_macros(b, int(k), _ptr(rho, (b.ny[k], b.nx[k]), "rho", False),
                                               _ptr(u, (2, b.ny[k], b.nx[k]), "u", False)), b)


def smrt_batch_nodes(b: BatchHandle) -> int:
    return int(_lib.load().smrt_batch_nodes(b))


def smrt_batch_last_error(b) -> str:
    raw = _lib.load().smrt_batch_last_error(b if b is not None else None)
    return raw.decode() if raw else ""


def smrt_batch_destroy(b: BatchHandle) -> None:
    if b is not None and b.ptr and b.ptr.value:
        _lib.load().smrt_batch_destroy(b.ptr)
        b.ptr = ctypes.c_void_p()


# ---- neural-network kernels of the learned warm start (include/smrt_nn.h) --------------
from .nn import (smrt_nn_adam, smrt_nn_add, smrt_nn_avgpool2, smrt_nn_avgpool2_bwd, smrt_nn_bias_act,  # noqa: E402
                 smrt_nn_bias_act_bwd, smrt_nn_col2im3, smrt_nn_concat, smrt_nn_concat_bwd, smrt_nn_flip3, smrt_nn_gemm,
                 smrt_nn_gemm_tc, smrt_nn_conv3_tc, smrt_nn_conv3_tma, smrt_nn_conv3_wgrad_tma, smrt_nn_conv3_tma_bias_act,
                 smrt_nn_check, smrt_nn_conv3_tma_wait_test, smrt_nn_conv3_tma_act_bwd, smrt_nn_pack3_many,
                 SMRT_NN_PACK_FORWARD, SMRT_NN_PACK_ADJOINT, smrt_nn_bias_act_bwd_addpool_blocked,
                 smrt_nn_pack3, smrt_nn_pack3_halves, smrt_nn_to_half_blocked, smrt_nn_bias_act_blocked,
                 smrt_nn_to_half_blocked_pad, smrt_nn_pad3, smrt_nn_unpad3_add,
                 smrt_nn_bias_act_bwd_blocked, smrt_nn_avgpool2_blocked, smrt_nn_upcat, smrt_nn_upcat_bwd,
                 smrt_nn_conv1x1_small, smrt_nn_conv1x1_small_bwd,
                 smrt_nn_im2col3, smrt_nn_mse, smrt_nn_resize_bilinear, smrt_nn_to_half, smrt_nn_to_half_rows,
                 smrt_nn_upsample2, smrt_nn_upsample2_bwd)

# ---- checkpoint files of a single lattice ------------------------------------------------
from .checkpoint import load_checkpoint, read_checkpoint, save_checkpoint, write_checkpoint  # noqa: E402,F401
