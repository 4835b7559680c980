"""The 64 x 64 Re 100 cavity fixture (tests/golden/cavity64_re100_t2000.txt, written by the oracle):
the oracle must keep reproducing it, and the GPU path must match it at the full 2000 updates."""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_cavity64 as G  # noqa: E402


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def test_fixture_is_a_developed_cavity_flow():
    g = G.read()
    ux, uy = g["ux_column_i32"], g["uy_row_j32"]
    assert ux.shape == (64,) and uy.shape == (64,)
    # the lid (top, +x) drags the top rows forward and the return flow runs backward lower down
    assert ux[-1] > 0.3 * G.U and ux[:40].max() < 0.0
    # a closed cavity with lid precedence conserves mass exactly up to rounding
    assert abs(g["mass"][0] - 64 * 64) < 1e-9


def test_oracle_reproduces_fixture():
    got, ref = G.fields(), G.read()
    for key in ("ux_column_i32", "uy_row_j32", "rho_nodes_j_i", "mass"):
        assert _rel(got[key], ref[key]) <= 1e-13, key
    for key in ("checksum_weighted", "checksum_alternating"):
        assert abs(got[key][0] - ref[key][0]) <= 1e-12 * abs(ref["checksum_weighted"][0]), key


@pytest.mark.gpu
@pytest.mark.parametrize("prec,layout", [("f64", "ab"), ("f64", "aa"), ("f32", "ab"), ("f32", "aa")])
def test_gpu_matches_fixture(prec, layout):
    import paper_2409_01076_gb300 as S
    from gpu_util import get_f, get_macros, make
    ref = G.read()
    h = make(G.N, G.N, G.TAU, G.U, S.CAVITY, prec=prec, layout=layout)
    S.smrt_step(h, G.STEPS)
    rho, u = get_macros(h)
    f = get_f(h)
    S.smrt_destroy(h)
    du = max(np.abs(u[0][:, 32] - ref["ux_column_i32"]).max(), np.abs(u[1][32, :] - ref["uy_row_j32"]).max())
    if prec == "f64":
        assert du <= 1e-12 * G.U
        assert _rel(rho.sum(), ref["mass"]) <= 1e-12       # the FP64 parity bound
        a, j, i = np.meshgrid(np.arange(9), np.arange(G.N), np.arange(G.N), indexing="ij")
        cw = (f * (1.0 + a + j / 64.0 + i / 4096.0)).sum()
        assert abs(cw - ref["checksum_weighted"][0]) <= 1e-12 * abs(ref["checksum_weighted"][0])
    else:
        assert du <= 2e-5 * G.U
