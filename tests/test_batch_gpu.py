"""Batches of independent lattices (smrt_batch_*): parity with the oracle, bit
equality with the single-lattice path, tile-shape autotuning, retirement."""
import math

import numpy as np
import pytest

import oracle as O
import paper_2409_01076_gb300 as S
from paper_2409_01076_gb300 import workloads as W

from gpu_util import get_f, make

SIZES = [(16, 12), (33, 17), (64, 64), (40, 72), (2, 2), (129, 5), (7, 90)]


def _taus(n):
    return [0.55 + 0.09 * k for k in range(n)]


def _ulids(n):
    return [0.02 + 0.013 * k for k in range(n)]


def test_batch_create_rejects_bad_arguments():
    for nx, ny, tau, u in [([1], [8], [0.7], [0.0]), ([8], [8], [0.5], [0.0]), ([8], [8], [0.7], [0.9])]:
        with pytest.raises(S.SmrtError) as ei:
            S.smrt_batch_create(nx, ny, tau, u)
        assert ei.value.status == S.SMRT_ERR_ARG
    with pytest.raises(S.SmrtError):
        S.smrt_batch_create([8], [8], [0.7], [0.0], precision=S.SMRT_PREC_F16)
    with pytest.raises(S.SmrtError):
        S.smrt_batch_create([8], [8], [0.7], [0.0], collision=S.SMRT_COLLISION_TWO_TAU)
    with pytest.raises(S.SmrtError):
        S.smrt_batch_create([8], [8], [0.7], [0.0], bc=W.bc_flags(0, 1, 1, 1))


@pytest.mark.gpu
@pytest.mark.parametrize("layout", [S.SMRT_LAYOUT_AB, S.SMRT_LAYOUT_AA], ids=["ab", "aa"])
@pytest.mark.parametrize("kind", [S.SMRT_COLLISION_SMRT, S.SMRT_COLLISION_SRT], ids=["smrt", "srt"])
def test_batch_f64_matches_oracle(layout, kind):
    nx, ny = [s[0] for s in SIZES], [s[1] for s in SIZES]
    taus, us = _taus(len(SIZES)), _ulids(len(SIZES))
    b = S.smrt_batch_create(nx, ny, taus, us, W.CAVITY, S.SMRT_PREC_F64, layout, kind)
    S.smrt_batch_step(b, 31)
    okind = O.SMRT if kind == S.SMRT_COLLISION_SMRT else O.SRT
    for k, (x, y) in enumerate(SIZES):
        ref = O.run(O.cavity_initial(x, y), 31, W.CAVITY, taus[k], u_lid=us[k], kind=okind)
        f = np.empty((9, y, x))
        S.smrt_batch_get_f(b, k, f)
        assert np.abs(f - ref).max() / np.abs(ref).max() <= 1e-12, k
    steps, res, state = S.smrt_batch_status(b)
    assert (steps == 31).all() and (state == S.SMRT_BATCH_ACTIVE).all()
    S.smrt_batch_destroy(b)


@pytest.mark.gpu
@pytest.mark.parametrize("layout", [S.SMRT_LAYOUT_AB, S.SMRT_LAYOUT_AA], ids=["ab", "aa"])
def test_batch_f32_bitwise_equals_single_lattice_and_autotune_keeps_state(layout):
    sizes = [(300, 70), (64, 64), (1000, 20), (5, 300)]
    nx, ny = [s[0] for s in sizes], [s[1] for s in sizes]
    taus, us = _taus(len(sizes)), _ulids(len(sizes))
    b = S.smrt_batch_create(nx, ny, taus, us, W.CAVITY, S.SMRT_PREC_F32, layout)
    S.smrt_batch_step(b, 13)
    before = []
    for k, (x, y) in enumerate(sizes):
        f = np.empty((9, y, x))
        S.smrt_batch_get_f(b, k, f)
        before.append(f)
    choice = S.smrt_batch_autotune(b, 4)
    assert 0 <= choice < 15
    steps, _, _ = S.smrt_batch_status(b)
    assert (steps == 13).all()
    for k, (x, y) in enumerate(sizes):
        f = np.empty((9, y, x))
        S.smrt_batch_get_f(b, k, f)
        assert np.array_equal(f, before[k]), k          # tuning did not advance or touch the state
    S.smrt_batch_step(b, 8)
    for k, (x, y) in enumerate(sizes):
        h = make(x, y, taus[k], us[k], W.CAVITY, prec="f32", layout="ab" if layout == 0 else "aa")
        S.smrt_step(h, 21)
        f = np.empty((9, y, x))
        S.smrt_batch_get_f(b, k, f)
        assert np.array_equal(f, get_f(h)), k
        S.smrt_destroy(h)
    S.smrt_batch_destroy(b)


@pytest.mark.gpu
@pytest.mark.parametrize("layout", [S.SMRT_LAYOUT_AB, S.SMRT_LAYOUT_AA], ids=["ab", "aa"])
@pytest.mark.parametrize("prec,shapes", [(S.SMRT_PREC_F32, 15), (S.SMRT_PREC_F64, 9)], ids=["f32", "f64"])
def test_every_tile_shape_matches_single_lattice_bitwise(layout, prec, shapes):
    """Each autotuner candidate (with and without the register bound, with and without the edge
    column groups in the vector path, row-segmented or not) computes the same bits as smrt_step,
    on lattices narrower and wider than one tile, with ragged rows; the narrow ones put several
    rows (one to 32 lanes each) into one warp of the row-segmented shapes."""
    sizes = [(300, 70), (64, 64), (1000, 20), (5, 300), (2, 2), (129, 5), (128, 9), (24, 17), (36, 6), (9, 4)]
    nx, ny = [s[0] for s in sizes], [s[1] for s in sizes]
    taus, us = _taus(len(sizes)), _ulids(len(sizes))
    pname = "f32" if prec == S.SMRT_PREC_F32 else "f64"
    ref = []
    for k, (x, y) in enumerate(sizes):
        h = make(x, y, taus[k], us[k], W.CAVITY, prec=pname, layout="ab" if layout == 0 else "aa")
        S.smrt_step(h, 11)
        ref.append(get_f(h))
        S.smrt_destroy(h)
    for shape in range(shapes):
        b = S.smrt_batch_create(nx, ny, taus, us, W.CAVITY, prec, layout)
        S.smrt_batch_set_shape(b, shape)
        S.smrt_batch_step(b, 11)
        for k, (x, y) in enumerate(sizes):
            f = np.empty((9, y, x))
            S.smrt_batch_get_f(b, k, f)
            assert np.array_equal(f, ref[k]), (shape, k)
        with pytest.raises(S.SmrtError) as ei:
            S.smrt_batch_set_shape(b, shapes)
        assert ei.value.status == S.SMRT_ERR_ARG
        S.smrt_batch_destroy(b)


@pytest.mark.gpu
@pytest.mark.parametrize("layout", [S.SMRT_LAYOUT_AB, S.SMRT_LAYOUT_AA], ids=["ab", "aa"])
def test_batch_run_retires_converged_and_capped(layout):
    # low Reynolds number cavities converge quickly; the last one is capped on purpose
    sizes = [(24, 24), (32, 24), (20, 36), (48, 48)]
    re = [5.0, 8.0, 6.0, 50.0]
    taus = [W.cavity_tau(max(x, y), 0.01, r) for (x, y), r in zip(sizes, re)]
    us = [0.01] * 4
    b = S.smrt_batch_create([s[0] for s in sizes], [s[1] for s in sizes], taus, us, W.CAVITY,
                            S.SMRT_PREC_F64, layout)
    left = S.smrt_batch_run(b, 1e-7, 200, 60000)
    assert left == 0
    steps, res, state = S.smrt_batch_status(b)
    assert (steps % 200 == 0).all() and (steps > 0).all()
    assert set(state.tolist()) <= {S.SMRT_BATCH_CONVERGED, S.SMRT_BATCH_CAPPED}
    for k in range(3):
        assert state[k] == S.SMRT_BATCH_CONVERGED and res[k] < 1e-7, (k, res[k], steps[k])
    assert len(set(steps[:3].tolist())) > 1                   # lattices retired at different times
    # a retired lattice is exactly where its own step count says: compare with the oracle,
    # and its residual is the oracle's one-step residual at the step before
    k = 0
    x, y = sizes[k]
    before = O.run(O.cavity_initial(x, y), int(steps[k]) - 1, W.CAVITY, taus[k], u_lid=us[k])
    ref = O.run(before, 1, W.CAVITY, taus[k], u_lid=us[k])
    f = np.empty((9, y, x))
    S.smrt_batch_get_f(b, k, f)
    assert np.abs(f - ref).max() / np.abs(ref).max() <= 1e-12
    r1, _ = O.residual(before, W.CAVITY, taus[k], u_lid=us[k])
    assert abs(res[k] - r1) <= 1e-6 * r1, (res[k], r1)
    S.smrt_batch_destroy(b)

    b = S.smrt_batch_create([32, 32], [32, 32], [0.6, 0.7], [0.05, 0.05], W.CAVITY, S.SMRT_PREC_F32, layout)
    assert S.smrt_batch_run(b, 1e-12, 100, 300) == 0
    steps, res, state = S.smrt_batch_status(b)
    assert (state == S.SMRT_BATCH_CAPPED).all() and (steps == 300).all()
    S.smrt_batch_destroy(b)


@pytest.mark.gpu
@pytest.mark.parametrize("layout", [S.SMRT_LAYOUT_AB, S.SMRT_LAYOUT_AA], ids=["ab", "aa"])
def test_batch_stride_residual_matches_oracle(layout):
    """r = ||u(t) - u(t - K)|| / (K ||u(t)||) after several checks equals the oracle's value."""
    taus, K, T = [0.644, 0.7], 200, 1000
    b = S.smrt_batch_create([24, 32], [24, 24], taus, [0.01, 0.01], W.CAVITY, S.SMRT_PREC_F64, layout)
    assert S.smrt_batch_run(b, 1e-30, K, T, S.SMRT_BATCH_RESIDUAL_STRIDE) == 0
    steps, res, state = S.smrt_batch_status(b)
    assert (steps == T).all() and (state == S.SMRT_BATCH_CAPPED).all()
    for k, nx in enumerate([24, 32]):
        f1 = O.run(O.cavity_initial(nx, 24), T - K, W.CAVITY, taus[k], u_lid=0.01)
        f2 = O.run(f1, K, W.CAVITY, taus[k], u_lid=0.01)
        u1, u2 = O.macros(f1)[1], O.macros(f2)[1]
        expect = np.sqrt(((u2 - u1) ** 2).sum()) / (K * np.sqrt((u2 ** 2).sum()))
        assert abs(res[k] / expect - 1) < 1e-6, (k, res[k], expect)
    S.smrt_batch_destroy(b)


@pytest.mark.gpu
def test_batch_divergence_and_warm_start():
    b = S.smrt_batch_create([16, 20, 24], [16, 20, 24], [0.7, 0.7, 0.7], [0.05] * 3, W.CAVITY, S.SMRT_PREC_F32)
    rho, u = W.rest_fields(20, 20)
    rho[5, 5] = np.nan
    S.smrt_batch_init_macros(b, 1, rho, u)
    rho2, u2 = W.random_macros(24, 24, seed=9, u_amp=0.02)
    S.smrt_batch_init_macros(b, 2, rho2, u2)
    S.smrt_batch_step(b, 3)
    _, _, state = S.smrt_batch_status(b)
    assert state.tolist() == [S.SMRT_BATCH_ACTIVE, S.SMRT_BATCH_DIVERGED, S.SMRT_BATCH_ACTIVE]
    # the warm-started lattice advanced from f^eq(rho2, u2)
    ref = O.run(O.init_equilibrium(rho2, u2), 3, W.CAVITY, 0.7, u_lid=0.05)
    r = np.empty((24, 24))
    uu = np.empty((2, 24, 24))
    S.smrt_batch_macros(b, 2, r, uu)
    assert np.abs(uu - O.macros(ref)[1]).max() < 2e-5 * 0.05
    with pytest.raises(S.SmrtError) as ei:
        S.smrt_batch_init_macros(b, 1, rho, u)               # retired
    assert ei.value.status == S.SMRT_ERR_STATE
    assert S.smrt_batch_run(b, 1e-3, 10, 40) == 0
    _, _, state = S.smrt_batch_status(b)
    assert state[1] == S.SMRT_BATCH_DIVERGED
    S.smrt_batch_destroy(b)
