"""NN kernels of the learned warm start against numpy, and the GPU U-Net's loss
and gradients against the FP64 oracle (oracle/unet_oracle.py) with the same weights."""
import numpy as np
import pytest

import paper_2409_01076_gb300 as S
from oracle import unet_oracle as U

pytestmark = pytest.mark.gpu


def _t(a, dtype=None):
    import torch
    return torch.tensor(np.asarray(a), dtype=dtype or torch.float32, device="cuda")


def _np(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().double().numpy()


def _rng(s):
    return np.random.Generator(np.random.PCG64(s))


@pytest.mark.parametrize("transA", [0, 1])
@pytest.mark.parametrize("transB", [0, 1])
@pytest.mark.parametrize("split", [1, 3])
def test_gemm_all_layouts(transA, transB, split):
    import torch
    r = _rng(transA * 4 + transB * 2 + split)
    M, N, Kd = 70, 45, 137
    a = r.normal(size=(Kd, M) if transA else (M, Kd)).astype(np.float16)
    b = r.normal(size=(N, Kd) if transB else (Kd, N)).astype(np.float16)
    c0 = r.normal(size=(M, N)).astype(np.float32)
    A = _t(a, torch.float16)
    B = _t(b, torch.float16)
    C = _t(c0)
    opa = a.astype(np.float64).T if transA else a.astype(np.float64)
    opb = b.astype(np.float64).T if transB else b.astype(np.float64)
    if split == 1:
        S.smrt_nn_gemm(transA, transB, M, N, Kd, 0.5, A, a.shape[1], B, b.shape[1], 2.0, C, N, 1)
        ref = 0.5 * opa @ opb + 2.0 * c0
    else:
        S.smrt_nn_gemm(transA, transB, M, N, Kd, 0.5, A, a.shape[1], B, b.shape[1], 1.0, C, N, split)
        ref = 0.5 * opa @ opb + c0           # split-K accumulates into C
    assert np.abs(_np(C) - ref).max() <= 1e-4 * np.abs(ref).max()


def test_im2col_col2im_match_oracle():
    import torch
    r = _rng(3)
    x = r.normal(size=(2, 6, 10, 5))
    col = torch.empty((2 * 6 * 10, 45), dtype=torch.float16, device="cuda")
    S.smrt_nn_im2col3(_t(x), col)
    assert np.abs(_np(col) - U.im2col3(x.astype(np.float32).astype(np.float16).astype(np.float64))).max() == 0
    d = r.normal(size=(2 * 6 * 10, 45))
    dx = torch.empty((2, 6, 10, 5), dtype=torch.float32, device="cuda")
    S.smrt_nn_col2im3(_t(d), (2, 6, 10, 5), dx)
    assert np.abs(_np(dx) - U.col2im3(d, (2, 6, 10, 5))).max() < 1e-5


@pytest.mark.parametrize("C,ld", [(5, 48), (8, 72), (16, 144), (3, 32)])
def test_im2col_vector_and_padded_rows(C, ld):
    """The 16-byte path (C % 8 == 0, dense rows) and padded rows (zeroed pad columns), ragged H, W."""
    import torch
    r = _rng(30 + C)
    x = r.normal(size=(3, 7, 11, C))
    col = torch.full((3 * 7 * 11, ld), float("nan"), dtype=torch.float16, device="cuda")
    S.smrt_nn_im2col3(_t(x), col)
    got = _np(col)
    ref = U.im2col3(x.astype(np.float32).astype(np.float16).astype(np.float64))
    assert np.array_equal(got[:, :9 * C], ref)
    assert (got[:, 9 * C:] == 0).all()


def test_to_half_rows_pads_with_zeros():
    import torch
    r = _rng(40)
    a = r.normal(size=(37, 3))
    d = torch.full((37, 8), float("nan"), dtype=torch.float16, device="cuda")
    S.smrt_nn_to_half_rows(_t(a), d, 2.0)
    got = _np(d)
    assert np.array_equal(got[:, :3], (2.0 * a).astype(np.float32).astype(np.float16).astype(np.float64))
    assert (got[:, 3:] == 0).all()


def test_bias_act_forward_backward():
    import torch
    r = _rng(4)
    x = r.normal(size=(300, 7)) * 3
    b = r.normal(size=(7,))
    z = torch.empty((300, 7), device="cuda")
    a = torch.empty((300, 7), device="cuda")
    S.smrt_nn_bias_act(_t(x), _t(b), 1, z, a)
    zr = x + b
    assert np.abs(_np(z) - zr).max() < 1e-5
    assert np.abs(_np(a) - U.silu(zr)).max() < 1e-5
    da = r.normal(size=(300, 7))
    dz = torch.empty((300, 7), device="cuda")
    db = torch.zeros(7, device="cuda")
    S.smrt_nn_bias_act_bwd(_t(da), z, 1, dz, db)
    dzr = da * U.silu_grad(zr)
    assert np.abs(_np(dz) - dzr).max() < 1e-5
    assert np.abs(_np(db) - dzr.sum(axis=0)).max() < 1e-4


def test_pool_upsample_concat_add():
    import torch
    r = _rng(5)
    x = r.normal(size=(2, 8, 6, 3))
    y = torch.empty((2, 4, 3, 3), device="cuda")
    S.smrt_nn_avgpool2(_t(x), y)
    assert np.abs(_np(y) - U.pool(x)).max() < 1e-6
    dx = torch.empty((2, 8, 6, 3), device="cuda")
    S.smrt_nn_avgpool2_bwd(y, (2, 8, 6, 3), dx)
    assert np.abs(_np(dx) - U.pool_bwd(_np(y))).max() < 1e-6
    u = torch.empty((2, 16, 12, 3), device="cuda")
    S.smrt_nn_upsample2(_t(x), u)
    assert np.abs(_np(u) - U.up(x)).max() < 1e-6
    S.smrt_nn_upsample2_bwd(u, (2, 8, 6, 3), dx)
    assert np.abs(_np(dx) - U.up_bwd(_np(u))).max() < 1e-5
    a2 = r.normal(size=(2, 8, 6, 2))
    cat = torch.empty((2, 8, 6, 5), device="cuda")
    S.smrt_nn_concat(_t(x), _t(a2), cat)
    assert np.abs(_np(cat) - np.concatenate([x, a2], axis=3)).max() < 1e-6
    da = torch.empty((2, 8, 6, 3), device="cuda")
    db = torch.empty((2, 8, 6, 2), device="cuda")
    S.smrt_nn_concat_bwd(cat, 3, 2, da, db)
    assert np.abs(_np(da) - x).max() < 1e-6 and np.abs(_np(db) - a2).max() < 1e-6
    s = torch.empty((2, 8, 6, 3), device="cuda")
    S.smrt_nn_add(_t(x), _t(x), s)
    assert np.abs(_np(s) - 2 * x).max() < 1e-5


@pytest.mark.parametrize("C", [12, 16])
def test_vector_elementwise_paths(C):
    """The 16-byte-vector kernels behind the plain entry points (C % 4 == 0) and the fused forms that
    write the blocked half layout, against numpy."""
    import torch
    r = _rng(40 + C)
    n, h, w = 2, 6, 10
    x = r.normal(size=(n, h, w, C)) * 3
    b = r.normal(size=(C,))
    z = torch.empty((n, h, w, C), device="cuda")
    a = torch.empty((n, h, w, C), device="cuda")
    S.smrt_nn_bias_act(_t(x), _t(b), 1, z, a)
    zr = x + b
    assert np.abs(_np(z) - zr).max() < 1e-5 and np.abs(_np(a) - U.silu(zr)).max() < 1e-5
    da = r.normal(size=(n, h, w, C))
    dz = torch.empty((n, h, w, C), device="cuda")
    db = torch.zeros(C, device="cuda")
    S.smrt_nn_bias_act_bwd(_t(da), z, 1, dz, db)
    dzr = da * U.silu_grad(zr)
    assert np.abs(_np(dz) - dzr).max() < 1e-5
    assert np.abs(_np(db) - dzr.reshape(-1, C).sum(axis=0)).max() < 1e-4
    y = torch.empty((n, h // 2, w // 2, C), device="cuda")
    S.smrt_nn_avgpool2(_t(x), y)
    dx = torch.empty((n, h, w, C), device="cuda")
    S.smrt_nn_avgpool2_bwd(y, (n, h, w, C), dx)
    assert np.abs(_np(dx) - U.pool_bwd(U.pool(x))).max() < 1e-5
    s2 = torch.empty((n, h, w, C), device="cuda")
    S.smrt_nn_add(_t(x), _t(da), s2)
    assert np.abs(_np(s2) - (x + da)).max() < 1e-5
    if C % 8:
        return

    def blocked(v):
        return v.reshape(n, v.shape[1], v.shape[2], C // 8, 8).transpose(0, 3, 1, 2, 4).ravel()

    ab = torch.empty(x.size, dtype=torch.float16, device="cuda")
    z2 = torch.empty((n, h, w, C), device="cuda")
    S.smrt_nn_bias_act_blocked(_t(x), _t(b), 1, z2, None, ab)
    assert np.array_equal(_np(z2), _np(z))
    assert np.array_equal(ab.cpu().numpy(), blocked(_np(a).astype(np.float32)).astype(np.float16))
    dzb = torch.empty(x.size, dtype=torch.float16, device="cuda")
    db2 = torch.zeros(C, device="cuda")
    S.smrt_nn_bias_act_bwd_blocked(_t(da), z, 1, None, db2, dzb)
    assert np.array_equal(dzb.cpu().numpy(), blocked(_np(dz).astype(np.float32)).astype(np.float16))
    assert np.abs(_np(db2) - _np(db)).max() < 1e-5
    yb = torch.empty(y.numel(), dtype=torch.float16, device="cuda")
    y2 = torch.empty_like(y)
    S.smrt_nn_avgpool2_blocked(_t(x), y2, yb)
    assert np.abs(_np(y2) - U.pool(x)).max() < 1e-6
    assert np.array_equal(yb.cpu().numpy(), blocked(_np(y2).astype(np.float32)).astype(np.float16))


def test_conv1x1_small_forward_backward():
    """The head's float32 1x1 convolution (32 -> 3) and its backward against numpy."""
    import torch
    r = _rng(42)
    x = r.normal(size=(3, 7, 9, 32))
    w = r.normal(size=(3, 32))
    b = r.normal(size=(3,))
    y = torch.empty((3, 7, 9, 3), device="cuda")
    S.smrt_nn_conv1x1_small(_t(x), _t(w), _t(b), y)
    assert np.abs(_np(y) - (x @ w.T + b)).max() < 1e-4
    dy = r.normal(size=(3, 7, 9, 3))
    dx = torch.empty((3, 7, 9, 32), device="cuda")
    dw = _t(np.ones((3, 32)))
    db = _t(np.ones(3))
    S.smrt_nn_conv1x1_small_bwd(_t(dy), _t(x), _t(w), dx, dw, db)
    assert np.abs(_np(dx) - dy @ w).max() < 1e-4
    assert np.abs(_np(dw) - (1 + dy.reshape(-1, 3).T @ x.reshape(-1, 32))).max() < 1e-3
    assert np.abs(_np(db) - (1 + dy.reshape(-1, 3).sum(axis=0))).max() < 1e-4


def test_upcat_and_its_adjoint():
    import torch
    r = _rng(41)
    n, h, w, ca, cb = 2, 3, 5, 16, 8
    a = r.normal(size=(n, h, w, ca))
    b = r.normal(size=(n, 2 * h, 2 * w, cb))
    ref = np.concatenate([U.up(a), b], axis=3)
    y = torch.empty(ref.shape, device="cuda")
    yb = torch.empty(ref.size, dtype=torch.float16, device="cuda")
    S.smrt_nn_upcat(_t(a), _t(b), y, yb)
    assert np.array_equal(_np(y), ref.astype(np.float32).astype(np.float64))
    blk = ref.reshape(n, 2 * h, 2 * w, (ca + cb) // 8, 8).transpose(0, 3, 1, 2, 4).ravel()
    assert np.array_equal(yb.cpu().numpy(), blk.astype(np.float32).astype(np.float16))
    dy = r.normal(size=ref.shape)
    da = torch.empty((n, h, w, ca), device="cuda")
    db = torch.empty((n, 2 * h, 2 * w, cb), device="cuda")
    S.smrt_nn_upcat_bwd(_t(dy), ca, da, db)
    assert np.abs(_np(da) - U.up_bwd(dy[..., :ca])).max() < 1e-5
    assert np.array_equal(_np(db), dy[..., ca:].astype(np.float32).astype(np.float64))


def test_mse_and_adam():
    import torch
    r = _rng(6)
    y, t = r.normal(size=1000), r.normal(size=1000)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dy = torch.empty(1000, device="cuda")
    S.smrt_nn_mse(_t(y), _t(t), 8.0, loss, dy)
    ya, ta = y.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64)
    assert abs(_np(loss)[0] - np.mean((ya - ta) ** 2)) < 1e-9
    assert np.abs(_np(dy) - 8.0 * 2 * (ya - ta) / 1000).max() < 1e-6
    w0, g = r.normal(size=50), r.normal(size=50)
    w, m, v = _t(w0), torch.zeros(50, device="cuda"), torch.zeros(50, device="cuda")
    inf = torch.zeros(1, dtype=torch.int32, device="cuda")
    wr, mr, vr = w0.copy(), np.zeros(50), np.zeros(50)
    for step in (1, 2, 3):
        S.smrt_nn_adam(w, _t(4.0 * g), m, v, 1e-2, 0.9, 0.999, 1e-8, step, 4.0, inf)
        mr = 0.9 * mr + 0.1 * g
        vr = 0.999 * vr + 0.001 * g * g
        wr = wr - 1e-2 * (mr / (1 - 0.9 ** step)) / (np.sqrt(vr / (1 - 0.999 ** step)) + 1e-8)
    assert np.abs(_np(w) - wr).max() < 1e-5 and int(_np(inf)[0]) == 0
    bad = g.copy()
    bad[3] = np.inf
    S.smrt_nn_adam(w, _t(bad), m, v, 1e-2, 0.9, 0.999, 1e-8, 4, 1.0, inf)
    assert int(_np(inf)[0]) == 1


def test_resize_bilinear_special_cases():
    import torch
    r = _rng(7)
    x = r.normal(size=(1, 8, 8, 2))
    y = torch.empty((1, 8, 8, 2), device="cuda")
    S.smrt_nn_resize_bilinear(_t(x), y)
    assert np.abs(_np(y) - x).max() < 1e-6                       # same size: identity
    # a field linear in the node coordinates is reproduced exactly away from the clamped edges
    h, h2 = 16, 64
    yy, xx = np.meshgrid((np.arange(h) + 0.5) / h, (np.arange(h) + 0.5) / h, indexing="ij")
    lin = np.stack([2 * xx - yy, 0.5 + yy], axis=-1)[None]
    out = torch.empty((1, h2, h2, 2), device="cuda")
    S.smrt_nn_resize_bilinear(_t(lin), out)
    y2, x2 = np.meshgrid((np.arange(h2) + 0.5) / h2, (np.arange(h2) + 0.5) / h2, indexing="ij")
    ref = np.stack([2 * x2 - y2, 0.5 + y2], axis=-1)[None]
    inner = slice(4, h2 - 4)
    assert np.abs(_np(out)[:, inner, inner] - ref[:, inner, inner]).max() < 1e-5


BACKENDS = [("tcgen05", "tma"), ("tcgen05", "gather"), ("wmma", "gather")]
BACKEND_IDS = ["tcgen05-tma", "tcgen05-gather", "wmma"]


@pytest.mark.parametrize("backend,conv", BACKENDS, ids=BACKEND_IDS)
@pytest.mark.parametrize("n,h", [(2, 16), (1, 128)], ids=["2x16", "1x128"])
def test_unet_loss_and_gradients_match_oracle(backend, conv, n, h):
    """Same weights, same batch: loss and every gradient tensor within half-precision operand rounding.
    At 128^2 the weight gradients of the top level run split-K (atomic partial sums)."""
    from paper_2409_01076_gb300.unet import UNet
    base, w = 8, h
    params = U.init_params(base, seed=3)
    r = _rng(8)
    x = r.uniform(0, 1, size=(n, h, w, 3))
    t = 0.3 * r.normal(size=(n, h, w, 3))
    loss_ref, grads_ref, _ = U.loss_and_grads(params, x, t, base)
    net = UNet(base=base, gemm=backend, conv=conv)
    net.load_numpy(params)
    net.grad_scale = 1024.0
    net.loss_and_grad(_t(x), _t(t))
    loss = float(_np(net._loss)[0])
    assert abs(loss / loss_ref - 1) < 5e-3, (loss, loss_ref)
    for key, gr in grads_ref.items():
        g = _np(net.grads[key]) / net.grad_scale
        rel = np.linalg.norm(g - gr) / max(np.linalg.norm(gr), 1e-30)
        cos = (g * gr).sum() / max(np.linalg.norm(g) * np.linalg.norm(gr), 1e-30)
        assert rel < 3e-2 and cos > 0.999, (key, rel, cos)
    if backend == "tcgen05":
        assert net.gemm_timeouts() == 0


@pytest.mark.parametrize("backend,conv", BACKENDS, ids=BACKEND_IDS)
def test_unet_gradients_match_oracle_at_training_size(backend, conv):
    """The warm-start network itself (32 base channels) on a 256^2 input: implicit-GEMM and split-K
    paths at full size.  Every gradient within 5e-3 of the FP64 oracle (half-operand rounding gives
    ~1e-3), cosine > 0.99999."""
    from paper_2409_01076_gb300.unet import UNet
    base, n, h, w = 32, 1, 256, 256
    params = U.init_params(base, seed=3)
    r = _rng(12)
    x = r.uniform(0, 1, size=(n, h, w, 3))
    t = 0.3 * r.normal(size=(n, h, w, 3))
    loss_ref, grads_ref, _ = U.loss_and_grads(params, x, t, base)
    net = UNet(base=base, gemm=backend, conv=conv)
    net.load_numpy(params)
    net.grad_scale = 1024.0
    net.loss_and_grad(_t(x), _t(t))
    assert abs(float(_np(net._loss)[0]) / loss_ref - 1) < 1e-4
    for key, gr in grads_ref.items():
        g = _np(net.grads[key]) / net.grad_scale
        rel = np.linalg.norm(g - gr) / max(np.linalg.norm(gr), 1e-30)
        cos = (g * gr).sum() / max(np.linalg.norm(g) * np.linalg.norm(gr), 1e-30)
        assert rel < 5e-3 and cos > 0.99999, (key, rel, cos)
    if backend == "tcgen05":
        assert net.gemm_timeouts() == 0


def test_fused_silu_backward_gives_the_unfused_gradients():
    """The input gradients that carry the next layer's SiLU backward in their epilogue (the default) give
    the gradients of the separate input-gradient and SiLU-backward kernels, up to the summation order of
    the bias-gradient and weight-gradient atomics."""
    from paper_2409_01076_gb300.unet import UNet
    base, n, h = 32, 2, 64
    params = U.init_params(base, seed=5)
    r = _rng(14)
    x = _t(r.uniform(0, 1, size=(n, h, h, 3)))
    t = _t(0.3 * r.normal(size=(n, h, h, 3)))
    grads = []
    for fused in (True, False):
        net = UNet(base=base)
        net.fuse_act_bwd = fused
        net.load_numpy(params)
        net.grad_scale = 1024.0
        net.loss_and_grad(x, t)
        net.check_timeouts()
        grads.append({k: _np(v).astype(np.float64) for k, v in net.grads.items()})
    for key in grads[0]:
        a, b = grads[0][key], grads[1][key]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert rel < 1e-5, (key, rel)


def test_graph_replay_matches_eager_training():
    """Three Adam steps with the forward and backward pass replayed from one CUDA graph give the
    losses and parameters of three eager steps (up to the order of the weight-gradient atomics)."""
    from paper_2409_01076_gb300.unet import UNet, input_grid
    x = input_grid([150.0, 900.0], 32, 32)
    xs = _np(x)
    t = _t(np.stack([np.sin(3 * xs[..., 1]) * xs[..., 0], np.cos(2 * xs[..., 2]), xs[..., 1] * xs[..., 2]], axis=-1))
    eager, graph = UNet(base=8, seed=4), UNet(base=8, seed=4)
    l_eager = [eager.train_step(x, t, 1e-3) for _ in range(3)]
    xg, tg = x.clone(), t.clone()
    graph.capture(xg, tg)
    l_graph = []
    for _ in range(3):
        graph.replay()
        graph.adam_step(1e-3)
        l_graph.append(float(_np(graph._loss)[0]))
    assert np.allclose(l_graph, l_eager, rtol=1e-4), (l_graph, l_eager)
    for key in eager.params:
        assert np.abs(_np(eager.params[key]) - _np(graph.params[key])).max() < 1e-5, key


def test_unet_training_reduces_the_loss():
    from paper_2409_01076_gb300.unet import UNet, input_grid
    net = UNet(base=8, seed=1)
    x = input_grid([150.0, 900.0], 32, 32)
    r = _rng(9)
    # a smooth synthetic target: a function of the inputs the network must learn
    xs = _np(x)
    t = np.stack([np.sin(3 * xs[..., 1]) * xs[..., 0], np.cos(2 * xs[..., 2]), xs[..., 1] * xs[..., 2]], axis=-1)
    tt = _t(t)
    first = net.train_step(x, tt, 3e-3)
    for _ in range(150):
        last = net.train_step(x, tt, 3e-3)
    assert last < 0.2 * first, (first, last)
