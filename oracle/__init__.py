"""FP64 CPU oracle for the D2Q9 SmrtLBM update (arXiv 2409.01076).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s ``cpu_baseline`` leg / ``--impl reference`` arm may import this
package.  The product library (``paper_2409_01076_gb300``) never imports it
and shares no code with it.

The arithmetic lives in ``smrt_oracle.c`` (plain C99, FP64, compiled with
``-ffp-contract=off`` so that x86 and Arm hosts give identical bits).  This
module only compiles it on demand and marshals numpy arrays.

Lattice arrays are numpy float64 of shape (9, ny, nx) -- f[a][j][i] -- with the
paper's direction order (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1).
Macro arrays: rho (ny, nx), u (2, ny, nx) = (ux plane, uy plane).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smrt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

SMRT, SRT, TWO_TAU, MRT = 0, 1, 2, 3
PERIODIC, WALL, MOVING = 0, 1, 2
LEFT, RIGHT, BOTTOM, TOP = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def bc_flags(left: int, right: int, bottom: int, top: int) -> int:
    """Pack per-side boundary kinds into the 8-bit flag word."""
    return left | (right << 2) | (bottom << 4) | (top << 6)


CAVITY = bc_flags(WALL, WALL, WALL, MOVING)
ALL_PERIODIC = bc_flags(PERIODIC, PERIODIC, PERIODIC, PERIODIC)


def build(force: bool = False) -> str:
    """Compile smrt_oracle.c into _build/liboracle.so (gcc, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            L.orc_feq.restype = ctypes.c_double
            L.orc_feq.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.orc_weight.restype = ctypes.c_double
            L.orc_weight.argtypes = [ctypes.c_int]
            for name in ("orc_ex", "orc_ey", "orc_opposite"):
                getattr(L, name).restype = ctypes.c_int
                getattr(L, name).argtypes = [ctypes.c_int]
            L.orc_feq_all.argtypes = [ctypes.c_double] * 3 + [dp]
            L.orc_moments.argtypes = [dp, dp, dp, dp]
            L.orc_collide.restype = ctypes.c_int
            L.orc_collide.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp]
            L.orc_collide_mrt.argtypes = [dp, dp, dp]
            L.orc_mrt_M.argtypes = [dp]
            L.orc_mrt_Minv.restype = ctypes.c_int
            L.orc_mrt_Minv.argtypes = [dp]
            L.orc_check_bc.restype = ctypes.c_int
            L.orc_check_bc.argtypes = [ctypes.c_uint]
            L.orc_stream.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint, ctypes.c_double,
                                     ctypes.c_double, dp, dp]
            L.orc_collide_field.restype = ctypes.c_int
            L.orc_collide_field.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]
            L.orc_run.restype = ctypes.c_int
            L.orc_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, dp, ctypes.c_longlong]
            L.orc_init_equilibrium.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
            L.orc_macros.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
            L.orc_residual.restype = ctypes.c_int
            L.orc_residual.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp, dp]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- single-node operations -------------------------------------------------

def velocities() -> np.ndarray:
    L = lib()
    return np.array([[L.orc_ex(a), L.orc_ey(a)] for a in range(9)], dtype=np.int64)


def weights() -> np.ndarray:
    L = lib()
    return np.array([L.orc_weight(a) for a in range(9)])


def opposites() -> np.ndarray:
    L = lib()
    return np.array([L.orc_opposite(a) for a in range(9)], dtype=np.int64)


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    """Eq. (feq-full) at one node."""
    out = np.empty(9)
    lib().orc_feq_all(rho, ux, uy, _p(out))
    return out


def moments(f) -> tuple[float, float, float]:
    """Eq. (fea-0) at one node: (rho, ux, uy)."""
    f = _f64(f)
    r, ux, uy = (ctypes.c_double() for _ in range(3))
    lib().orc_moments(_p(f), ctypes.byref(r), ctypes.byref(ux), ctypes.byref(uy))
    return r.value, ux.value, uy.value


def collide(kind: int, f, tau: float, tau_s: float = 1.0) -> np.ndarray:
    """One node's post-collision populations.

    kind SMRT: Eq. (SmrtLBM-1); SRT: Eq. (lb.srt); TWO_TAU: Eq. (SmrtLBM-lb.1.5);
    MRT: Eq. (lb.1) with S = diag(1/tau_s x7, 1/tau x2).
    """
    f = _f64(f)
    out = np.empty(9)
    rc = lib().orc_collide(kind, _p(f), tau, tau_s, _p(out))
    if rc != 0:
        raise ValueError("bad collision kind %r" % kind)
    return out


def collide_mrt(f, s) -> np.ndarray:
    """Eq. (lb.1) with an arbitrary diagonal S = diag(s)."""
    f, s = _f64(f), _f64(s)
    out = np.empty(9)
    lib().orc_collide_mrt(_p(f), _p(s), _p(out))
    return out


def mrt_M() -> np.ndarray:
    m = np.empty(81)
    lib().orc_mrt_M(_p(m))
    return m.reshape(9, 9)


def mrt_Minv() -> np.ndarray:
    m = np.empty(81)
    if lib().orc_mrt_Minv(_p(m)) != 0:
        raise RuntimeError("M is singular")
    return m.reshape(9, 9)


# ---- lattice operations -------------------------------------------------------

def check_bc(flags: int) -> bool:
    return lib().orc_check_bc(flags) == 0


def stream(post, flags: int, u_lid: float = 0.0, rho_w: float = 1.0) -> np.ndarray:
    """Streaming with halfway / moving-wall bounce-back; post has shape (9, ny, nx)."""
    post = _f64(post)
    _, ny, nx = post.shape
    nxt = np.full_like(post, np.nan)
    lib().orc_stream(nx, ny, flags, u_lid, rho_w, _p(post), _p(nxt))
    return nxt


def collide_field(f, kind: int, tau: float, tau_s: float = 1.0, force=(0.0, 0.0)) -> np.ndarray:
    f = _f64(f)
    _, ny, nx = f.shape
    post = np.empty_like(f)
    rc = lib().orc_collide_field(nx, ny, kind, tau, tau_s, force[0], force[1], _p(f), _p(post))
    if rc != 0:
        raise ValueError("collide_field failed")
    return post


def run(f, steps: int, flags: int, tau: float, u_lid: float = 0.0, kind: int = SMRT,
        tau_s: float = 1.0, force=(0.0, 0.0)) -> np.ndarray:
    """Advance the canonical field f(t) by `steps` updates; returns a new array."""
    g = _f64(f).copy()
    _, ny, nx = g.shape
    rc = lib().orc_run(nx, ny, flags, u_lid, kind, tau, tau_s, force[0], force[1], _p(g), steps)
    if rc != 0:
        raise ValueError("orc_run failed with %d" % rc)
    return g


def init_equilibrium(rho, u) -> np.ndarray:
    """f = f^eq(rho, u) at every node; rho (ny, nx), u (2, ny, nx)."""
    rho, u = _f64(rho), _f64(u)
    ny, nx = rho.shape
    assert u.shape == (2, ny, nx)
    f = np.empty((9, ny, nx))
    lib().orc_init_equilibrium(nx, ny, _p(rho), _p(u), _p(f))
    return f


def macros(f) -> tuple[np.ndarray, np.ndarray]:
    f = _f64(f)
    _, ny, nx = f.shape
    rho = np.empty((ny, nx))
    u = np.empty((2, ny, nx))
    lib().orc_macros(nx, ny, _p(f), _p(rho), _p(u))
    return rho, u


def residual(f, flags: int, tau: float, u_lid: float = 0.0, kind: int = SMRT,
             tau_s: float = 1.0) -> tuple[float, np.ndarray]:
    """r(t) = ||u(t+1)-u(t)|| / ||u(t+1)|| and {sum rho, sum rho ux, sum rho uy} at t."""
    f = _f64(f)
    _, ny, nx = f.shape
    r = ctypes.c_double()
    sums = np.empty(3)
    rc = lib().orc_residual(nx, ny, flags, u_lid, kind, tau, tau_s, _p(f), ctypes.byref(r), _p(sums))
    if rc != 0:
        raise ValueError("orc_residual failed with %d" % rc)
    return r.value, sums


def cavity_initial(nx: int, ny: int) -> np.ndarray:
    """f(0) = f^eq(rho=1, u=0) at every node."""
    return init_equilibrium(np.ones((ny, nx)), np.zeros((2, ny, nx)))
