"""Helpers shared by the GPU tests: run the CUDA path through the C ABI."""
import numpy as np

import paper_2409_01076_gb300 as S

PRECS = {"f64": S.SMRT_PREC_F64, "f32": S.SMRT_PREC_F32, "f16": S.SMRT_PREC_F16, "bf16": S.SMRT_PREC_BF16}
LAYOUTS = {"ab": S.SMRT_LAYOUT_AB, "aa": S.SMRT_LAYOUT_AA}
KINDS = {"smrt": S.SMRT_COLLISION_SMRT, "srt": S.SMRT_COLLISION_SRT, "two_tau": S.SMRT_COLLISION_TWO_TAU}


def make(nx, ny, tau, u_lid, bc, prec="f64", layout="ab", kind="smrt", tau_s=1.0):
    h = S.smrt_create(nx, ny, tau, u_lid, bc)
    S.smrt_set_option(h, S.SMRT_OPT_PRECISION, PRECS[prec])
    S.smrt_set_option(h, S.SMRT_OPT_LAYOUT, LAYOUTS[layout])
    S.smrt_set_option(h, S.SMRT_OPT_COLLISION, KINDS[kind])
    S.smrt_set_option(h, S.SMRT_OPT_TAU_S, tau_s)
    return h


def get_f(h):
    f = np.empty((9, h.ny, h.nx))
    S.smrt_get_f(h, f)
    return f


def get_macros(h):
    rho = np.empty((h.ny, h.nx))
    u = np.empty((2, h.ny, h.nx))
    S.smrt_macros(h, rho, u)
    return rho, u


def run_gpu(f0, steps, bc, tau, u_lid=0.0, prec="f64", layout="ab", kind="smrt", tau_s=1.0, chunks=1):
    _, ny, nx = f0.shape
    h = make(nx, ny, tau, u_lid, bc, prec, layout, kind, tau_s)
    S.smrt_set_f(h, np.ascontiguousarray(f0))
    done = 0
    for c in range(chunks):
        n = steps // chunks + (1 if c < steps % chunks else 0)
        S.smrt_step(h, n)
        done += n
    assert S.smrt_time(h) == steps
    out = get_f(h)
    S.smrt_destroy(h)
    return out


def rel_f(a, b):
    return np.abs(a - b).max() / np.abs(b).max()
