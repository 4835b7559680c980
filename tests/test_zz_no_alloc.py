"""smrt_residual_noalloc: the residual for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc -- a framework's caching allocator owns the
device memory budget, or a latency-critical loop must not let cudaMalloc/cudaFree
synchronize the device -- so they cannot create an smrt_t (its state is allocated
on first use).  smrt_residual_noalloc takes their canonical f(t) in device memory
and computes the residual with its scratch in a fixed file-scope device array.
These tests check it, through the C ABI, against smrt_residual of a handle in
the same state, within the FP64 tolerance of the parity tests, on calls in a row,
and against the FP64 CPU oracle's residual of the same field (the tolerance of
the residual parity test).
This file is collected last so a stop-at-first-failure run has already run the rest.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import paper_2409_01076_gb300 as S
from paper_2409_01076_gb300 import _lib
from paper_2409_01076_gb300 import workloads as W

TOL = 1e-12


def test_noalloc_rejects_bad_sizes_before_touching_the_device():
    lib = _lib.load()
    out = (ctypes.c_double * 4)()
    dummy = ctypes.c_void_p(16)
    for nx, ny in [(1, 8), (8, 1), (1 << 16, 1 << 15)]:
        rc = lib.smrt_residual_noalloc(dummy, nx, ny, 0.7, 0.0, W.CAVITY, 0, 1.0, out, None)
        assert rc == S.SMRT_ERR_ARG
        assert "smrt_residual_noalloc" in S.smrt_last_error(None)
    assert lib.smrt_residual_noalloc(None, 8, 8, 0.7, 0.0, W.CAVITY, 0, 1.0, out, None) == S.SMRT_ERR_ARG
    assert lib.smrt_residual_noalloc(dummy, 8, 8, 0.5, 0.0, W.CAVITY, 0, 1.0, out, None) == S.SMRT_ERR_ARG
    assert lib.smrt_residual_noalloc(dummy, 8, 8, 0.7, 0.0, W.CAVITY, 5, 1.0, out, None) == S.SMRT_ERR_ARG


def test_noalloc_binding_rejects_host_tensors():
    import torch
    f = torch.zeros(9, 8, 8, dtype=torch.float64)
    with pytest.raises(TypeError):
        S.smrt_residual_noalloc(f, 0.7)
    with pytest.raises(TypeError):
        S.smrt_residual_noalloc(np.zeros((9, 8, 8)), 0.7)


def _close(a, b):
    return abs(a - b) <= TOL * max(abs(b), 1e-300)


def _oracle_close(r, sums, f_host, tau, u_lid, bc, kind=O.SMRT):
    r_o, sums_o = O.residual(f_host, bc, tau, u_lid=u_lid, kind=kind)
    n = f_host.shape[1] * f_host.shape[2]
    assert abs(r - r_o) <= 1e-9 * r_o, (r, r_o)
    assert np.abs(np.array(sums) - sums_o).max() <= 1e-12 * n


@pytest.mark.gpu
def test_noalloc_matches_handle_residual_on_calls_in_a_row():
    import torch
    torch.cuda.set_device(0)
    nx, ny, tau, U = 96, 72, 0.62, 0.1
    h = S.smrt_create(nx, ny, tau, U, W.CAVITY)          # FP64, SmrtLBM, two-buffer layout
    f = torch.empty(9, ny, nx, dtype=torch.float64, device="cuda")

    # call 1: host result
    S.smrt_step(h, 150)
    r_ref, sums_ref = S.smrt_residual(h)
    S.smrt_get_f(h, f)
    torch.cuda.synchronize()
    r, sums = S.smrt_residual_noalloc(f, tau, U, W.CAVITY)
    assert r > 0 and _close(r, r_ref), (r, r_ref)
    for a, b in zip(sums, sums_ref):
        assert abs(a - b) <= TOL * nx * ny
    _oracle_close(r, sums, f.cpu().numpy(), tau, U, W.CAVITY)

    # call 2, right after, on a different state: device result on a side stream
    S.smrt_step(h, 77)
    r_ref2, sums_ref2 = S.smrt_residual(h)
    S.smrt_get_f(h, f)
    torch.cuda.synchronize()
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    S.smrt_residual_noalloc(f, tau, U, W.CAVITY, out=out, stream=side)
    side.synchronize()
    got = out.cpu().numpy()
    assert _close(got[0], r_ref2), (got[0], r_ref2)
    assert not _close(got[0], r_ref)                   # nothing stale from call 1
    assert np.abs(got[1:] - np.array(sums_ref2)).max() <= TOL * nx * ny
    _oracle_close(got[0], got[1:], f.cpu().numpy(), tau, U, W.CAVITY)
    S.smrt_destroy(h)


@pytest.mark.gpu
def test_noalloc_periodic_srt_matches_handle():
    import torch
    torch.cuda.set_device(0)
    n, tau = 64, 0.8
    rho, u = W.tgv_fields(n, n, 0.02)
    h = S.smrt_create(n, n, tau, 0.0, W.ALL_PERIODIC)
    S.smrt_set_option(h, S.SMRT_OPT_COLLISION, S.SMRT_COLLISION_SRT)
    S.smrt_init_macros(h, rho, u)
    S.smrt_step(h, 20)
    r_ref, sums_ref = S.smrt_residual(h)
    f = torch.empty(9, n, n, dtype=torch.float64, device="cuda")
    S.smrt_get_f(h, f)
    torch.cuda.synchronize()
    for _ in range(2):
        r, sums = S.smrt_residual_noalloc(f, tau, 0.0, W.ALL_PERIODIC, collision=S.SMRT_COLLISION_SRT)
        assert _close(r, r_ref), (r, r_ref)
        assert np.abs(np.array(sums) - np.array(sums_ref)).max() <= TOL * n * n
        _oracle_close(r, sums, f.cpu().numpy(), tau, 0.0, W.ALL_PERIODIC, kind=O.SRT)
    S.smrt_destroy(h)
