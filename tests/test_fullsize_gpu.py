"""Parity at full size, in the launch configuration the benchmark times.

The oracle cannot advance an 8192^2 lattice, but after s steps a node depends
only on the (2s+1)^2 nodes around it.  So the oracle runs a small window of the
same synthetic initial state, (W + 2s)^2 nodes with the window's own sides
where the domain has walls (elsewhere anything: the wrong boundary reaches at
most s nodes in), and its central W x W nodes are compared with the GPU's.
"""
import numpy as np
import pytest

import oracle as O
import paper_2409_01076_gb300 as S
from paper_2409_01076_gb300 import workloads as W

from gpu_util import make

pytestmark = pytest.mark.gpu

F32_UTOL = 2e-5


def _gpu_f_device(h):
    import torch
    f = torch.empty(9, h.ny, h.nx, dtype=torch.float64, device="cuda")
    S.smrt_get_f(h, f)
    torch.cuda.synchronize()
    return f


def _compare_window(fd, ref_window, x0, y0, Wd, U):
    got = fd[:, y0:y0 + Wd, x0:x0 + Wd].cpu().numpy()
    _, ug = O.macros(got)
    _, ur = O.macros(ref_window)
    err = np.abs(ug - ur).max() / U
    assert err <= F32_UTOL, (x0, y0, err)
    assert np.abs(got - ref_window).max() <= 1e-6


@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("kind", ["smrt", "srt"])
def test_tgv_8192_windows(layout, kind):
    import torch
    n, u0, tau, s, Wd = 8192, 0.05, 0.51, 6, 16
    h = make(n, n, tau, 0.0, W.ALL_PERIODIC, prec="f32", layout=layout, kind=kind)
    rho, u = W.tgv_fields(n, n, u0)
    S.smrt_init_macros(h, torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    del rho, u
    S.smrt_step(h, s)
    fd = _gpu_f_device(h)
    okind = O.SMRT if kind == "smrt" else O.SRT
    for x0, y0 in [(0, 0), (n - Wd, n - Wd), (4000, 4100), (1234, 7001), (8100, 17)]:
        r, uu = W.tgv_fields(n, n, u0, x0 - s, y0 - s, Wd + 2 * s, Wd + 2 * s)
        ref = O.run(O.init_equilibrium(r, uu), s, O.ALL_PERIODIC, tau, kind=okind)
        _compare_window(fd, ref[:, s:s + Wd, s:s + Wd], x0, y0, Wd, u0)
    # a property at any size: total mass is conserved
    _, sums = S.smrt_residual(h)
    assert abs(sums[0] / (n * n) - 1.0) < 1e-6
    del fd
    S.smrt_destroy(h)
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec,layout", [("f32", "ab"), ("f16", "aa")])
def test_tgv_16384_windows_past_2_31_elements(prec, layout):
    """A 16384^2 lattice: one buffer holds 9 x 2^28 = 2.4e9 elements, past 2^31, so the plane offsets
    of the upper populations and every pull and push address there need 64-bit arithmetic.  Windows
    at the corners and deep in the plane against the oracle; the residual's mass sum at full size."""
    import torch
    n, u0, tau, s, Wd = 16384, 0.05, 0.51, 6, 16
    h = make(n, n, tau, 0.0, W.ALL_PERIODIC, prec=prec, layout=layout)
    rho, u = W.tgv_fields(n, n, u0)
    S.smrt_init_macros(h, torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
    del rho, u
    S.smrt_step(h, s)
    fd = _gpu_f_device(h)
    for x0, y0 in [(0, 0), (n - Wd, n - Wd), (9000, 15000), (16000, 5)]:
        r, uu = W.tgv_fields(n, n, u0, x0 - s, y0 - s, Wd + 2 * s, Wd + 2 * s)
        ref = O.run(O.init_equilibrium(r, uu), s, O.ALL_PERIODIC, tau)[:, s:s + Wd, s:s + Wd]
        if prec == "f32":
            _compare_window(fd, ref, x0, y0, Wd, u0)
        else:
            # 16-bit offsets: six roundings of each population (~1.5e-5 each); an addressing error
            # would be of the order of the populations themselves
            got = fd[:, y0:y0 + Wd, x0:x0 + Wd].cpu().numpy()
            assert np.abs(got - ref).max() <= 5e-4, (x0, y0)
            assert np.abs(O.macros(got)[1] - O.macros(ref)[1]).max() <= 1e-2 * u0, (x0, y0)
    _, sums = S.smrt_residual(h)
    assert abs(sums[0] / (n * n) - 1.0) < 1e-6
    del fd
    S.smrt_destroy(h)
    torch.cuda.empty_cache()


@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_cavity_4096_re10000_windows(layout):
    import torch
    n, U, re, s, Wd = 4096, 0.1, 1e4, 8, 16
    tau = W.cavity_tau(n, U, re)
    h = make(n, n, tau, U, W.CAVITY, prec="f32", layout=layout)
    S.smrt_step(h, s)
    fd = _gpu_f_device(h)
    m = Wd + s
    # (x0, y0) of the W x W compared block, and the oracle window's origin and sides
    cases = [
        (0, n - Wd, 0, n - m, W.CAVITY),                                   # top-left corner
        (n - Wd, n - Wd, n - m, n - m, W.CAVITY),                          # top-right corner
        (2000, n - Wd, 2000 - s, n - m, W.CAVITY),                         # lid, middle
        (0, 0, 0, 0, W.CAVITY),                                            # bottom-left corner
        (1500, 1500, 1500 - s, 1500 - s, W.ALL_PERIODIC),                  # interior
    ]
    for x0, y0, wx0, wy0, bc in cases:
        size = Wd + 2 * s
        wx0 = min(max(wx0, 0), n - size) if bc == W.CAVITY else wx0
        wy0 = min(max(wy0, 0), n - size) if bc == W.CAVITY else wy0
        f0 = O.cavity_initial(size, size)
        ref = O.run(f0, s, bc, tau, u_lid=U)
        ox, oy = x0 - wx0, y0 - wy0
        _compare_window(fd, ref[:, oy:oy + Wd, ox:ox + Wd], x0, y0, Wd, U)
    del fd
    S.smrt_destroy(h)
    torch.cuda.empty_cache()
