"""smrt_residual on the float formats measured against one real update.

For 32- and 16-bit offsets the residual forms u(t+1) - u(t) in float from the differences of the
stored offsets, (dj - u0 drho) / rho1, instead of subtracting two nearly equal velocities.  Its r
must be the change one real smrt_step makes: r from the moments before and after the step (the
48-bit moments of smrt_macros, differenced in FP64), within 1e-5 relative -- a few float roundings
of the change itself -- early in a run and at the FP32 floor of a converged cavity (r ~ 1e-7, where
u(t+1) and u(t) agree to 7 digits).  The sums rho and rho u match FP64 sums of the same moments
within the bound of float offset sums (per node: mass 1e-8, momentum 1e-7)."""
import numpy as np
import pytest

import paper_2409_01076_gb300 as S
from paper_2409_01076_gb300 import workloads as W

from gpu_util import get_macros, make


def _check_against_one_step(h):
    r, sums = S.smrt_residual(h)
    rho0, u0 = get_macros(h)
    S.smrt_step(h, 1)
    _, u1 = get_macros(h)
    r_ref = np.sqrt(((u1 - u0) ** 2).sum()) / np.sqrt((u1 ** 2).sum())
    assert r > 0 and abs(r - r_ref) <= 1e-5 * r_ref, (r, r_ref)
    n = rho0.size
    assert abs(sums[0] - rho0.sum()) <= 1e-8 * n
    assert abs(sums[1] - (rho0 * u0[0]).sum()) <= 1e-7 * n
    assert abs(sums[2] - (rho0 * u0[1]).sum()) <= 1e-7 * n
    return r


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("kind", ["smrt", "srt"])
def test_float_residual_equals_one_real_step_early(prec, layout, kind):
    h = make(70, 44, 0.58, 0.1, W.CAVITY, prec=prec, layout=layout, kind=kind)
    S.smrt_step(h, 41)
    _check_against_one_step(h)
    S.smrt_destroy(h)


@pytest.mark.gpu
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_float_residual_at_the_fp32_floor_of_a_converged_cavity(layout):
    """64^2 cavity at Re 100, 30,000 updates: FP32 sits at its rounding floor (r ~ 1e-7)."""
    n, U = 64, 0.1
    h = make(n, n, W.cavity_tau(n, U, 100.0), U, W.CAVITY, prec="f32", layout=layout)
    S.smrt_step(h, 30000)
    r = _check_against_one_step(h)
    assert r < 1e-5
    S.smrt_destroy(h)


@pytest.mark.gpu
def test_float_residual_periodic_ragged_tiles():
    """Periodic Taylor-Green on a 97 x 53 lattice: tiles ragged in both directions, wrapped halos."""
    nx, ny, tau = 97, 53, 0.8
    h = make(nx, ny, tau, 0.0, W.ALL_PERIODIC, prec="f32")
    rho, u = W.tgv_fields(nx, ny, 0.03)
    S.smrt_init_macros(h, rho, u)
    S.smrt_step(h, 10)
    _check_against_one_step(h)
    S.smrt_destroy(h)


@pytest.mark.gpu
@pytest.mark.parametrize("layout", ["ab", "aa"])
def test_fp64_residual_with_interior_tiles_matches_the_oracle(layout):
    """FP64, 100 x 76 cavity: tiles whose halo stays inside the lattice (the direct-index path) and
    edge tiles, against oracle.residual on the same state."""
    import oracle as O
    nx, ny, tau, U = 100, 76, 0.6, 0.1
    h = make(nx, ny, tau, U, W.CAVITY, layout=layout)
    S.smrt_step(h, 57)
    f = np.empty((9, ny, nx))
    S.smrt_get_f(h, f)
    r, sums = S.smrt_residual(h)
    r_ref, sums_ref = O.residual(f, W.CAVITY, tau, u_lid=U)
    assert abs(r - r_ref) <= 1e-9 * r_ref, (r, r_ref)
    assert np.abs(np.array(sums) - np.array(sums_ref)).max() <= 1e-12 * nx * ny
    S.smrt_destroy(h)


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny", [(2, 2), (3, 2), (5, 3), (129, 3), (3, 129), (31, 5), (33, 70)])
@pytest.mark.parametrize("bc", [W.CAVITY, W.ALL_PERIODIC, W.COUETTE])
def test_residual_on_tiny_and_thin_lattices(nx, ny, bc):
    """Strips narrower than a warp, segments shorter than the sweep, one-row interiors, wrapped
    halos: FP64 against oracle.residual; FP32 against one real step."""
    import oracle as O
    tau, U = 0.7, (0.0 if bc == W.ALL_PERIODIC else 0.05)
    rho, u = W.random_macros(nx, ny, 21, u_amp=0.02)
    h = make(nx, ny, tau, U, bc)
    S.smrt_init_macros(h, rho, u)
    S.smrt_step(h, 3)
    f = np.empty((9, ny, nx))
    S.smrt_get_f(h, f)
    r, sums = S.smrt_residual(h)
    r_ref, sums_ref = O.residual(f, bc, tau, u_lid=U)
    assert abs(r - r_ref) <= 1e-9 * r_ref, (r, r_ref)
    assert np.abs(np.array(sums) - np.array(sums_ref)).max() <= 1e-12 * nx * ny
    S.smrt_destroy(h)
    h = make(nx, ny, tau, U, bc, prec="f32")
    S.smrt_init_macros(h, rho, u)
    S.smrt_step(h, 3)
    _check_against_one_step(h)
    S.smrt_destroy(h)
