"""Pins of the FP64 U-Net oracle: adjoint identities of its building blocks and
central finite differences of the whole loss (no GPU)."""
import numpy as np
import pytest

from oracle import unet_oracle as U


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_building_blocks_are_adjoint():
    r = _rng(1)
    x = r.normal(size=(2, 6, 4, 3))
    y = r.normal(size=(2 * 6 * 4, 27))
    assert abs((U.im2col3(x) * y).sum() - (x * U.col2im3(y, x.shape)).sum()) < 1e-10
    p = r.normal(size=(2, 3, 2, 3))
    assert abs((U.pool(x) * p).sum() - (x * U.pool_bwd(p)).sum()) < 1e-12
    q = r.normal(size=(2, 12, 8, 3))
    assert abs((U.up(x) * q).sum() - (x * U.up_bwd(q)).sum()) < 1e-12


def test_im2col_taps_by_hand():
    x = np.arange(1 * 3 * 3 * 1, dtype=float).reshape(1, 3, 3, 1) + 1.0   # values 1..9
    col = U.im2col3(x)
    centre = col[4]          # node (1, 1): all nine neighbours
    assert centre.tolist() == [1, 2, 3, 4, 5, 6, 7, 8, 9]
    corner = col[0]          # node (0, 0): only taps (1,1),(1,2),(2,1),(2,2) inside
    assert corner.tolist() == [0, 0, 0, 0, 1, 2, 0, 4, 5]


def test_silu_derivative():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (U.silu(z + h) - U.silu(z - h)) / (2 * h)
    assert np.abs(fd - U.silu_grad(z)).max() < 1e-8


@pytest.mark.parametrize("seed", [0, 1])
def test_gradients_match_finite_differences(seed):
    base, n, h, w = 2, 2, 8, 8
    params = U.init_params(base, seed=seed)
    r = _rng(10 + seed)
    x = r.normal(size=(n, h, w, 3))
    t = r.normal(size=(n, h, w, 3))
    loss, grads, dx = U.loss_and_grads(params, x, t, base)
    eps = 1e-6
    for name in sorted(params):
        p = params[name].reshape(-1)
        for i in r.choice(p.size, size=min(3, p.size), replace=False):
            old = p[i]
            p[i] = old + eps
            lp = U.mse(U.forward(params, x, base)[0], t)
            p[i] = old - eps
            lm = U.mse(U.forward(params, x, base)[0], t)
            p[i] = old
            fd = (lp - lm) / (2 * eps)
            g = grads[name].reshape(-1)[i]
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, i, fd, g)
    # gradient with respect to the input as well
    xi = x.reshape(-1)
    for i in r.choice(xi.size, size=5, replace=False):
        old = xi[i]
        xi[i] = old + eps
        lp = U.mse(U.forward(params, x, base)[0], t)
        xi[i] = old - eps
        lm = U.mse(U.forward(params, x, base)[0], t)
        xi[i] = old
        assert abs((lp - lm) / (2 * eps) - dx.reshape(-1)[i]) < 1e-8
