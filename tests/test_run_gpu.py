"""smrt_run: host fields in, n updates, host fields out, with the host link overlapped.

The pipelined path cuts the lattice into row chunks and runs the updates of each chunk as soon as
the chunks it depends on are ready, so every node still sees exactly the arithmetic of smrt_step.
The tests compare it bit for bit with the three separate calls (smrt_init_macros, smrt_step,
smrt_macros) on device arrays: the final f field, rho, u and t, on lattices with ragged chunks,
2 to 32 chunks, every collision, walls, moving walls and periodic sides, 16-bit storage with
stochastic rounding (whose bits depend on t), and the n = 1 and n = 64 ends of the pipelined range.
"""
import numpy as np
import pytest

import paper_2409_01076_gb300 as S
from paper_2409_01076_gb300 import workloads as W

from gpu_util import make

pytestmark = pytest.mark.gpu


def _pinned(a):
    import torch
    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return t


def _fields(nx, ny, seed):
    rho, u = W.random_macros(nx, ny, seed, u_amp=0.03)
    return np.ascontiguousarray(rho), np.ascontiguousarray(u)


def _separate(nx, ny, tau, U, bc, prec, kind, rho, u, n, sr=False):
    import torch
    h = make(nx, ny, tau, U, bc, prec=prec, kind=kind, tau_s=0.9)
    if sr:
        S.smrt_set_option(h, S.SMRT_OPT_ROUNDING, S.SMRT_ROUND_STOCHASTIC)
    S.smrt_init_macros(h, torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    S.smrt_step(h, n)
    ro = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    uo = torch.empty((2, ny, nx), dtype=torch.float64, device="cuda")
    S.smrt_macros(h, ro, uo)
    f = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
    S.smrt_get_f(h, f)
    t = S.smrt_time(h)
    S.smrt_destroy(h)
    return f.cpu().numpy(), ro.cpu().numpy(), uo.cpu().numpy(), t


def _run(nx, ny, tau, U, bc, prec, kind, rho, u, n, sr=False):
    import torch
    h = make(nx, ny, tau, U, bc, prec=prec, kind=kind, tau_s=0.9)
    if sr:
        S.smrt_set_option(h, S.SMRT_OPT_ROUNDING, S.SMRT_ROUND_STOCHASTIC)
    ri, ui = _pinned(rho), _pinned(u)
    ro = torch.zeros((ny, nx), dtype=torch.float64, pin_memory=True)
    uo = torch.zeros((2, ny, nx), dtype=torch.float64, pin_memory=True)
    S.smrt_run(h, ri, ui, n, ro, uo)
    f = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
    S.smrt_get_f(h, f)
    t = S.smrt_time(h)
    S.smrt_destroy(h)
    return f.cpu().numpy(), ro.numpy().copy(), uo.numpy().copy(), t


def _same(a, b):
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y), np.abs(x - y).max()
    assert a[3] == b[3]


@pytest.mark.parametrize("nx,ny", [(37, 1291), (24, 8200)])
@pytest.mark.parametrize("n", [1, 3, 20])
def test_run_equals_the_separate_calls_fp32_cavity(nx, ny, n):
    rho, u = _fields(nx, ny, 11)
    tau, U = 0.6, 0.1
    _same(_run(nx, ny, tau, U, W.CAVITY, "f32", "smrt", rho, u, n),
          _separate(nx, ny, tau, U, W.CAVITY, "f32", "smrt", rho, u, n))


@pytest.mark.parametrize("prec,kind,bc,sr", [
    ("f64", "smrt", W.ALL_PERIODIC, False),
    ("f32", "srt", W.COUETTE, False),
    ("f32", "two_tau", W.bc_flags(W.MOVING, W.MOVING, W.WALL, W.MOVING), False),
    ("f16", "smrt", W.CAVITY, True),
    ("bf16", "smrt", W.ALL_PERIODIC, True),
])
def test_run_equals_the_separate_calls_all_variants(prec, kind, bc, sr):
    nx, ny, n = 45, 777, 7
    rho, u = _fields(nx, ny, 12)
    _same(_run(nx, ny, 0.57, 0.08, bc, prec, kind, rho, u, n, sr),
          _separate(nx, ny, 0.57, 0.08, bc, prec, kind, rho, u, n, sr))


@pytest.mark.parametrize("n", [64, 65])
def test_run_at_the_end_of_the_pipelined_range_and_beyond(n):
    """64 updates is the longest pipelined run; 65 takes the three calls in order."""
    nx, ny = 20, 530
    rho, u = _fields(nx, ny, 13)
    _same(_run(nx, ny, 0.7, 0.1, W.CAVITY, "f32", "smrt", rho, u, n),
          _separate(nx, ny, 0.7, 0.1, W.CAVITY, "f32", "smrt", rho, u, n))


def test_run_from_the_current_state_with_one_output():
    """No input fields: the run starts from the handle's state; only u is written back."""
    import torch
    nx, ny, n = 33, 600, 5
    rho, u = _fields(nx, ny, 14)
    ref = _separate(nx, ny, 0.65, 0.1, W.CAVITY, "f32", "smrt", rho, u, n + 2)
    h = make(nx, ny, 0.65, 0.1, W.CAVITY, prec="f32")
    S.smrt_init_macros(h, torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    S.smrt_step(h, 2)
    uo = torch.zeros((2, ny, nx), dtype=torch.float64, pin_memory=True)
    S.smrt_run(h, None, None, n, None, uo)
    assert S.smrt_time(h) == n + 2
    assert np.array_equal(uo.numpy(), ref[2])
    f = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
    S.smrt_get_f(h, f)
    assert np.array_equal(f.cpu().numpy(), ref[0])
    S.smrt_destroy(h)


def test_run_in_place_layout_takes_the_separate_calls():
    """The in-place layout is not pipelined; smrt_run still gives the separate calls' result."""
    import torch
    nx, ny, n = 30, 520, 4
    rho, u = _fields(nx, ny, 15)
    ref = _separate(nx, ny, 0.6, 0.1, W.CAVITY, "f32", "smrt", rho, u, n)
    h = make(nx, ny, 0.6, 0.1, W.CAVITY, prec="f32", layout="aa")
    ri, ui = _pinned(rho), _pinned(u)
    ro = torch.zeros((ny, nx), dtype=torch.float64, pin_memory=True)
    uo = torch.zeros((2, ny, nx), dtype=torch.float64, pin_memory=True)
    S.smrt_run(h, ri, ui, n, ro, uo)
    assert np.array_equal(ro.numpy(), ref[1]) and np.array_equal(uo.numpy(), ref[2])
    S.smrt_destroy(h)
