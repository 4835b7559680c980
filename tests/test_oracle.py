"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formula: each compares it with a
second equation of the paper, a closed form, an invariant, a library routine,
or a hand-derived tiny case, so that a dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2409_01076_gb300 import workloads as W

KINDS = [O.SMRT, O.SRT, O.TWO_TAU, O.MRT]


# ---- lattice constants (listing below Eq. lb.srt, weights below Eq. feq-full) ----

def test_velocity_set_and_weights():
    e = O.velocities()
    assert e.tolist() == [[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1],
                          [1, 1], [-1, 1], [-1, -1], [1, -1]]
    w = O.weights()
    assert w[0] == 4 / 9 and all(w[1:5] == 1 / 9) and all(w[5:] == 1 / 36)
    # lattice isotropy: sum w = 1, sum w e = 0, sum w e_i e_j = delta_ij / 3
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(w @ e).max() < 1e-15
    second = np.einsum("a,ai,aj->ij", w, e, e)
    assert np.abs(second - np.eye(2) / 3).max() < 1e-15
    opp = O.opposites()
    assert opp.tolist() == [0, 3, 4, 1, 2, 7, 8, 5, 6]


# ---- Eq. (feq-full) and Eq. (fea-0) -------------------------------------------

@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.1, 0.05, -0.03), (0.93, -0.12, 0.08)])
def test_equilibrium_moments_closed_form(rho, ux, uy):
    """Moments of the second-order equilibrium: rho, rho u, rho (delta/3 + u u)."""
    f = O.feq(rho, ux, uy)
    e = O.velocities().astype(float)
    u = np.array([ux, uy])
    assert abs(f.sum() - rho) < 1e-15
    assert np.abs(e.T @ f - rho * u).max() < 1e-15
    pi = np.einsum("a,ai,aj->ij", f, e, e)
    assert np.abs(pi - rho * (np.eye(2) / 3 + np.outer(u, u))).max() < 1e-15
    r, vx, vy = O.moments(f)
    assert abs(r - rho) < 1e-15 and abs(vx - ux) < 1e-15 and abs(vy - uy) < 1e-15


# ---- collision identities ------------------------------------------------------

def test_tau_one_returns_equilibrium_exactly():
    """tau = 1 makes 1 - 1/tau vanish in Eq. (SmrtLBM-1): f* = f^eq bit for bit."""
    for f in W.random_node_populations(20, seed=1):
        rho, ux, uy = O.moments(f)
        feq = O.feq(rho, ux, uy)
        assert np.array_equal(O.collide(O.SMRT, f, 1.0), feq)
        for kind in (O.SRT, O.TWO_TAU, O.MRT):
            assert np.abs(O.collide(kind, f, 1.0, 1.0) - feq).max() < 1e-15


@pytest.mark.parametrize("kind", KINDS)
def test_equilibrium_is_fixed_point(kind):
    for rho, ux, uy in [(1.0, 0.0, 0.0), (1.05, 0.08, -0.04), (0.9, -0.1, 0.1)]:
        feq = O.feq(rho, ux, uy)
        out = O.collide(kind, feq, 0.57, 0.8)
        assert np.abs(out - feq).max() <= 1e-15 * np.abs(feq).max() * 4


@pytest.mark.parametrize("kind", KINDS)
def test_collision_conserves_mass_and_momentum(kind):
    e = O.velocities().astype(float)
    for f in W.random_node_populations(50, seed=2):
        out = O.collide(kind, f, 0.53, 1.3)
        assert abs(out.sum() - f.sum()) < 1e-14
        assert np.abs(e.T @ out - e.T @ f).max() < 1e-14


def test_minv_is_inverse_and_orthogonal_form():
    """Gauss-Jordan M^-1 against numpy and against M^T diag(1/|row|^2) (rows of M are orthogonal)."""
    M = O.mrt_M()
    Minv = O.mrt_Minv()
    assert np.abs(M @ Minv - np.eye(9)).max() < 1e-14
    assert np.abs(Minv - np.linalg.inv(M)).max() < 1e-14
    gram = M @ M.T
    assert np.abs(gram - np.diag(np.diag(gram))).max() == 0
    assert np.abs(Minv - M.T @ np.diag(1 / np.diag(gram))).max() < 1e-15
    # rows 7 and 8 are the stress moments p_xx, p_xy; 1/|row|^2 = 1/4 each
    assert np.diag(gram)[7] == 4 and np.diag(gram)[8] == 4


@pytest.mark.parametrize("tau", [0.51, 0.692, 1.7])
def test_smrt_equals_mrt_matrix_form(tau):
    """Eq. (SmrtLBM-1) is Eq. (lb.1) with S = diag(1 x7, 1/tau x2) (Appendix, tau_s = 1)."""
    s = np.array([1.0] * 7 + [1 / tau] * 2)
    for f in W.random_node_populations(50, seed=3):
        lit = O.collide(O.SMRT, f, tau)
        mat = O.collide_mrt(f, s)
        two = O.collide(O.TWO_TAU, f, tau, 1.0)
        assert np.abs(lit - mat).max() < 1e-14
        assert np.abs(lit - two).max() < 1e-14


@pytest.mark.parametrize("tau,tau_s", [(0.51, 0.8), (0.7, 1.9), (1.2, 0.55)])
def test_two_tau_form_equals_mrt_and_reduces_to_srt(tau, tau_s):
    """Eq. (SmrtLBM-lb.1.5) = Eq. (lb.1) with S of Eq. (S-matrix:1); tau_s = tau gives SRT."""
    s = np.array([1 / tau_s] * 7 + [1 / tau] * 2)
    for f in W.random_node_populations(30, seed=4):
        assert np.abs(O.collide(O.TWO_TAU, f, tau, tau_s) - O.collide_mrt(f, s)).max() < 1e-14
        assert np.abs(O.collide(O.TWO_TAU, f, tau, tau) - O.collide(O.SRT, f, tau)).max() < 1e-14
        # MRT with every rate equal is BGK
        assert np.abs(O.collide_mrt(f, np.full(9, 1 / tau)) - O.collide(O.SRT, f, tau)).max() < 1e-14


@pytest.mark.parametrize("tau", [0.6, 2.0])
def test_worked_example_normal_stress(tau):
    """Hand derivation: rest state plus delta on f1 and f3.

    rho = 1 + 2 delta, u = 0, so f^eq_a = w_a (1 + 2 delta) and
    n1 = n3 = 7 delta / 9, n2 = n4 = -2 delta / 9, n5..8 = -delta / 18.
    The indicator sum for a in 1..4 is C1 = (-n1 + n2 - n3 + n4) / 4 = -delta / 2,
    for a in 5..8 it is C2 = (-n5 + n6 - n7 + n8) / 4 = 0.  With A = 1 - 1/tau,
    f*_1 = f*_3 = (1+2d)/9 + A d/2, f*_2 = f*_4 = (1+2d)/9 - A d/2,
    f*_0 = 4(1+2d)/9, f*_5..8 = (1+2d)/36.
    """
    d = 0.09
    f = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f[1] += d
    f[3] += d
    A = 1 - 1 / tau
    r = 1 + 2 * d
    expect = np.array([4 * r / 9, r / 9 + A * d / 2, r / 9 - A * d / 2, r / 9 + A * d / 2,
                       r / 9 - A * d / 2, r / 36, r / 36, r / 36, r / 36])
    assert np.abs(O.collide(O.SMRT, f, tau) - expect).max() < 1e-15


def test_worked_example_shear_stress():
    """Hand derivation: rest state plus delta on f5 and f7 gives Pi_xy = 2 delta.

    n5 = n7 = 17 delta / 18, n6 = n8 = -delta / 18, C2 = -delta / 2, C1 = 0;
    f*_5 = f*_7 = (1+2d)/36 + A d/2, f*_6 = f*_8 = (1+2d)/36 - A d/2.
    """
    d = 0.01
    tau = 0.7
    f = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f[5] += d
    f[7] += d
    A = 1 - 1 / tau
    r = 1 + 2 * d
    expect = np.array([4 * r / 9] + [r / 9] * 4 + [r / 36 + A * d / 2, r / 36 - A * d / 2,
                                                   r / 36 + A * d / 2, r / 36 - A * d / 2])
    assert np.abs(O.collide(O.SMRT, f, tau) - expect).max() < 1e-16


# ---- streaming and bounce-back (left-hand side of Eq. SmrtLBM-1) ----------------

def _distinct_post(nx, ny):
    a, j, i = np.meshgrid(np.arange(9), np.arange(ny), np.arange(nx), indexing="ij")
    return (100.0 * a + 10.0 * j + i).astype(np.float64)


def test_periodic_stream_is_a_roll():
    post = _distinct_post(3, 3)
    nxt = O.stream(post, O.ALL_PERIODIC)
    e = O.velocities()
    for a in range(9):
        assert np.array_equal(nxt[a], np.roll(post[a], shift=(e[a][1], e[a][0]), axis=(0, 1)))


def test_cavity_stream_by_hand_3x3():
    """Hand-checked links of a 3x3 cavity (walls left/right/bottom, lid U on top)."""
    U = 0.1
    post = _distinct_post(3, 3)
    nxt = O.stream(post, O.CAVITY, u_lid=U)
    assert not np.isnan(nxt).any()                    # every entry written once
    # interior link: (1,1) along e5 = (1,1) arrives at (2,2)
    assert nxt[5][2][2] == post[5][1][1]
    # left wall: (0,0) along e3 = (-1,0) returns as f1 at (0,0)
    assert nxt[1][0][0] == post[3][0][0]
    # bottom-left corner: e7 = (-1,-1) leaves through both walls, returns as f5
    assert nxt[5][0][0] == post[7][0][0]
    # lid, straight up: e2 has e.u_w = 0, returns unchanged as f4
    assert nxt[4][2][1] == post[2][2][1]
    # lid, e5 = (1,1): returns as f7 minus 6 (1/36) U
    assert abs(nxt[7][2][1] - (post[5][2][1] - U / 6)) < 1e-13
    # top-left corner, e6 = (-1,1) crosses lid and left wall: lid wins, + U/6
    assert abs(nxt[8][2][0] - (post[6][2][0] + U / 6)) < 1e-13
    # top-right corner, e5 crosses lid and right wall: lid wins, - U/6
    assert abs(nxt[7][2][2] - (post[5][2][2] - U / 6)) < 1e-13
    # right wall mid row: e8 = (1,-1) from (2,1) goes to (3,0): right wall, returns as f6
    assert nxt[6][1][2] == post[8][1][2]


def test_mixed_periodic_wall_corner():
    """x periodic, y walls: a link leaving through the floor is a wall link even where x wraps."""
    post = _distinct_post(4, 3)
    nxt = O.stream(post, W.CHANNEL)
    assert not np.isnan(nxt).any()
    assert nxt[6][0][0] == post[8][0][0]        # e8 = (1,-1) from (0,0) hits the floor
    assert nxt[6][0][3] == post[8][0][3]        # e8 from (3,0): x would wrap, the floor wins
    assert nxt[8][0][0] == post[8][1][3]        # e8 from (3,1) wraps in x to (0,0)
    assert nxt[1][2][0] == post[1][2][3]        # e1 from (3,2) wraps to (0,2)


def test_check_bc():
    assert O.check_bc(O.CAVITY) and O.check_bc(O.ALL_PERIODIC) and O.check_bc(W.COUETTE)
    assert not O.check_bc(W.bc_flags(0, 1, 1, 1))     # left periodic, right wall
    assert not O.check_bc(W.bc_flags(1, 1, 3, 1))     # kind 3 does not exist
