"""Stochastic rounding of the 16-bit storage formats (SMRT_OPT_ROUNDING = SMRT_ROUND_STOCHASTIC).

Each stored offset rounds up or down with the probabilities that make its expected value exact,
from counter-based bits keyed by (node, population, t).  So: the two layouts give the same bits,
a run is reproducible and resumes bit for bit from a checkpoint, the residual pass (which rounds
the next step's post-collision values itself) sees exactly the state the next step stores, the
result still matches the FP64 oracle within the 16-bit bounds of the parity tests, and over a long
cavity run the error against the FP64 path is far below round-to-nearest's coherent error.
"""
import numpy as np
import pytest

import oracle as O
import paper_2409_01076_gb300 as S
from paper_2409_01076_gb300 import workloads as W

from gpu_util import get_f, get_macros, make

pytestmark = pytest.mark.gpu

HALF_UTOL = {"f16": 2e-3, "bf16": 2e-2}


def _sr(h):
    S.smrt_set_option(h, S.SMRT_OPT_ROUNDING, S.SMRT_ROUND_STOCHASTIC)
    return h


def _run(f0, steps, bc, tau, u_lid, prec, layout):
    _, ny, nx = f0.shape
    h = _sr(make(nx, ny, tau, u_lid, bc, prec=prec, layout=layout))
    S.smrt_set_f(h, f0)
    S.smrt_step(h, steps)
    f = get_f(h)
    S.smrt_destroy(h)
    return f


@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("bc,nx", [(W.CAVITY, 64), (W.CAVITY, 70), (W.ALL_PERIODIC, 96),
                                   (W.bc_flags(W.MOVING, W.MOVING, W.WALL, W.MOVING), 130)])
def test_sr_in_place_equals_two_buffer_bitwise(prec, bc, nx):
    rho, u = W.random_macros(nx, 35, seed=12)
    f0 = O.init_equilibrium(rho, u)
    a = _run(f0, 23, bc, 0.57, 0.05, prec, "ab")
    b = _run(f0, 23, bc, 0.57, 0.05, prec, "aa")
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_sr_matches_the_oracle_within_the_16_bit_bounds(prec):
    nx, ny, steps, tau, U = 48, 40, 200, W.cavity_tau(48, 0.1, 100.0), 0.1
    ref = O.run(O.cavity_initial(nx, ny), steps, W.CAVITY, tau, u_lid=U)
    got = _run(O.cavity_initial(nx, ny), steps, W.CAVITY, tau, U, prec, "ab")
    _, ug = O.macros(got)
    _, ur = O.macros(ref)
    assert np.abs(ug - ur).max() / U <= HALF_UTOL[prec]
    # it does round: not the round-to-nearest result
    h = make(nx, ny, tau, U, W.CAVITY, prec=prec)
    S.smrt_step(h, steps)
    assert not np.array_equal(get_f(h), got)
    S.smrt_destroy(h)


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_sr_is_reproducible_and_resumes_from_a_checkpoint(prec, tmp_path):
    nx, ny, tau, U = 66, 50, 0.6, 0.1
    straight = []
    for _ in range(2):
        h = _sr(make(nx, ny, tau, U, W.CAVITY, prec=prec, layout="aa"))
        S.smrt_step(h, 57)
        straight.append(get_f(h))
        S.smrt_destroy(h)
    assert np.array_equal(straight[0], straight[1])
    h = _sr(make(nx, ny, tau, U, W.CAVITY, prec=prec, layout="aa"))
    S.smrt_step(h, 31)
    path = str(tmp_path / "sr.ckp")
    S.save_checkpoint(h, path)
    S.smrt_destroy(h)
    h = S.load_checkpoint(path)
    assert S.smrt_get_option(h, S.SMRT_OPT_ROUNDING) == S.SMRT_ROUND_STOCHASTIC
    S.smrt_step(h, 26)
    assert np.array_equal(get_f(h), straight[0])
    S.smrt_destroy(h)


@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_sr_residual_sees_the_state_the_next_step_stores(prec, layout):
    """smrt_residual rounds u(t+1) itself; with stochastic rounding it must draw the bits the step
    draws.  Recompute r from the moments before and after one real step.  The float formats form the
    change from offset differences in float (1e-5 relative covers its roundings); bits drawn for another
    (node, population, t) would move r by several per cent here."""
    nx, ny, tau, U = 70, 44, 0.58, 0.1
    h = _sr(make(nx, ny, tau, U, W.CAVITY, prec=prec, layout=layout))
    S.smrt_step(h, 41)
    r, _ = S.smrt_residual(h)
    _, u0 = get_macros(h)
    S.smrt_step(h, 1)
    _, u1 = get_macros(h)
    r_ref = np.sqrt(((u1 - u0) ** 2).sum()) / np.sqrt((u1 ** 2).sum())
    assert abs(r - r_ref) <= 1e-5 * r_ref, (r, r_ref)
    S.smrt_destroy(h)


def test_sr_error_after_20000_updates_is_far_below_round_to_nearest():
    """1024^2 cavity at Re 5,000: FP16 and BF16 offsets against the FP64 path after 20,000 updates."""
    import torch
    n, U, steps = 1024, 0.1, 20000
    tau = W.cavity_tau(n, U, 5000.0)

    def run(prec, sr):
        h = make(n, n, tau, U, W.CAVITY, prec=prec)
        if sr:
            _sr(h)
        S.smrt_step(h, steps)
        rho = torch.empty((n, n), dtype=torch.float64, device="cuda")
        u = torch.empty((2, n, n), dtype=torch.float64, device="cuda")
        S.smrt_macros(h, rho, u)
        S.smrt_destroy(h)
        return u

    u64 = run("f64", False)
    err = {}
    for prec in ("f16", "bf16"):
        for sr in (False, True):
            err[(prec, sr)] = float((run(prec, sr) - u64).abs().amax()) / U
    # measured on a GB300: FP16 8.7e-2 -> 2.1e-3, BF16 0.45 -> 1.2e-2
    assert err[("f16", True)] < 0.1 * err[("f16", False)], err
    assert err[("bf16", True)] < 0.1 * err[("bf16", False)], err
    assert err[("f16", True)] < 5e-3 and err[("bf16", True)] < 3e-2, err
