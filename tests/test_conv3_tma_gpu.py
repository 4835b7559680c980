"""TMA-fed 3x3 convolutions (operands by cp.async.bulk.tensor / cp.async.bulk, nine taps as shifted
views of one zero-padded input tile): the blocked half layout and the weight packing element by
element; smrt_nn_conv3_tma and smrt_nn_conv3_wgrad_tma against FP64 products of the same half
operands (numpy), and against the thread-gathered kernel smrt_nn_conv3_tc."""
import numpy as np
import pytest

import paper_2409_01076_gb300 as S
from oracle import unet_oracle as U

pytestmark = pytest.mark.gpu


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _blocked(x):
    """(N, H, W, C) -> flat [N][C/8][H][W][8], the layout the kernels read."""
    n, h, w, c = x.shape
    return np.ascontiguousarray(x.reshape(n, h, w, c // 8, 8).transpose(0, 3, 1, 2, 4)).ravel()


def test_to_half_blocked_layout():
    import torch
    x = _rng(3).normal(size=(2, 5, 7, 24)).astype(np.float32)
    xb = torch.empty(x.size, dtype=torch.float16, device="cuda")
    S.smrt_nn_to_half_blocked(torch.tensor(x, device="cuda"), xb, 0.5)
    torch.cuda.synchronize()
    assert np.array_equal(xb.cpu().numpy(), _blocked((0.5 * x).astype(np.float16)))


def test_padding_kernels_for_a_narrow_input_layer():
    """The 3-channel input as 16 zero-padded channels: blocked halves, padded weights, and the weight
    gradient folded back -- element by element."""
    import torch
    r = _rng(21)
    x = r.normal(size=(2, 5, 7, 3)).astype(np.float32)
    xb = torch.empty(2 * 5 * 7 * 16, dtype=torch.float16, device="cuda")
    S.smrt_nn_to_half_blocked_pad(torch.tensor(x, device="cuda"), 16, xb)
    xp = np.zeros((2, 5, 7, 16), dtype=np.float32)
    xp[..., :3] = x
    w = r.normal(size=(8, 27)).astype(np.float32)
    wh = torch.empty((8, 144), dtype=torch.float16, device="cuda")
    S.smrt_nn_pad3(torch.tensor(w, device="cuda"), 3, 16, wh)
    gp = torch.tensor(r.normal(size=(8, 144)).astype(np.float32), device="cuda")
    gw0 = r.normal(size=(8, 27)).astype(np.float32)
    gw = torch.tensor(gw0, device="cuda")
    S.smrt_nn_unpad3_add(gp, 3, 16, gw)
    torch.cuda.synchronize()
    assert np.array_equal(xb.cpu().numpy(), _blocked(xp.astype(np.float16)))
    whr = np.zeros((8, 9, 16), dtype=np.float16)
    whr[:, :, :3] = w.reshape(8, 9, 3).astype(np.float16)
    assert np.array_equal(wh.cpu().numpy(), whr.reshape(8, 144))
    exp = gw0 + gp.cpu().numpy().reshape(8, 9, 16)[:, :, :3].reshape(8, 27)
    assert np.array_equal(gw.cpu().numpy(), exp)


@pytest.mark.parametrize("cout,C", [(5, 32), (48, 16), (130, 32)])
def test_pack3_layout(cout, C):
    import torch
    w = _rng(1).normal(size=(cout, 9 * C)).astype(np.float16)
    size = S.smrt_nn_pack3_halves(cout, C)
    TN = 32 if cout <= 32 else 64 if cout <= 64 else 128
    ntn = (cout + TN - 1) // TN
    assert size == 9 * C * ntn * TN
    wp = torch.empty(size, dtype=torch.float16, device="cuda")
    S.smrt_nn_pack3(torch.tensor(w, device="cuda"), C, wp)
    torch.cuda.synchronize()
    got = wp.cpu().numpy().reshape(ntn, C // 16, 18, TN, 8)
    for nb in range(ntn):
        for chunk in range(C // 16):
            for tap in range(9):
                for q in range(2):
                    c0 = tap * C + chunk * 16 + q * 8
                    rows = w[nb * TN:(nb + 1) * TN, c0:c0 + 8]
                    blk = got[nb, chunk, tap * 2 + q]
                    assert np.array_equal(blk[:rows.shape[0]], rows), (nb, chunk, tap, q)
                    assert not blk[rows.shape[0]:].any()


def _conv(n, h, w, C, cout, alpha, beta, seed):
    import torch
    r = _rng(seed)
    x = r.normal(size=(n, h, w, C)).astype(np.float16)
    wt = r.normal(size=(cout, 9 * C)).astype(np.float16)
    y0 = r.normal(size=(n * h * w, cout)).astype(np.float32)
    xb = torch.tensor(_blocked(x), device="cuda")
    wd = torch.tensor(wt, device="cuda")
    wp = torch.empty(S.smrt_nn_pack3_halves(cout, C), dtype=torch.float16, device="cuda")
    S.smrt_nn_pack3(wd, C, wp)
    y = torch.tensor(y0, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.smrt_nn_conv3_tma(xb, (n, h, w, C), wp, y, cout, alpha, beta, err)
    torch.cuda.synchronize()
    exp = alpha * U.im2col3(x.astype(np.float64)) @ wt.astype(np.float64).T + beta * y0
    return y.cpu().numpy(), exp, int(err.item()), (x, wd)


@pytest.mark.parametrize("n,h,w,C,cout", [
    (2, 37, 21, 16, 20),      # ragged tiles in both directions, cout < 32
    (1, 32, 40, 32, 32),      # the top U-Net level's shape (2 chunks)
    (2, 18, 10, 48, 64),      # one tile per image, 3 chunks, TN 64
    (1, 16, 8, 80, 48),       # 5 chunks: the 4 stages are reused
    (1, 20, 12, 96, 130),     # two 128-wide output-channel tiles, the second partial
    (1, 24, 16, 384, 128),    # the widest decoder input (24 chunks)
    (10, 70, 40, 32, 136),    # stacked tile pairs (300 CTAs), the last pair partly outside, two N tiles
    (16, 48, 56, 80, 256),    # stacked pairs over 5 chunks (the stages are reused)
    (16, 70, 44, 48, 48),     # a grid where pairs would apply, but 64-wide tiles run single
    (16, 160, 96, 32, 24),    # 1,920 tiles of one 32-wide output block, 2 chunks
])
def test_conv3_tma_matches_fp64_product_of_the_same_halves(n, h, w, C, cout):
    got, exp, err, _ = _conv(n, h, w, C, cout, 0.75, 0.5, seed=C * 1000 + cout)
    assert err == 0
    assert np.abs(got - exp).max() <= 1e-4 * np.abs(exp).max(), np.abs(got - exp).max() / np.abs(exp).max()


def test_conv3_tma_image_smaller_than_the_halo_box():
    """5 x 3 images: the 18 x 10 halo box is larger than the image in both directions."""
    got, exp, err, _ = _conv(3, 5, 3, 16, 32, 1.0, 0.0, seed=77)
    assert err == 0
    assert np.abs(got - exp).max() <= 1e-4 * np.abs(exp).max()


def test_conv3_tma_agrees_with_the_gather_kernel():
    """Same half operands through smrt_nn_conv3_tc (A tiles gathered by threads, tap-major K order):
    equal up to float32 accumulation order."""
    import torch
    n, h, w, C, cout = 2, 64, 48, 64, 96
    got, _, err, (x, wd) = _conv(n, h, w, C, cout, 1.0, 0.0, seed=5)
    ref = torch.zeros((n * h * w, cout), device="cuda")
    e2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.smrt_nn_conv3_tc(torch.tensor(x.astype(np.float32), device="cuda"), wd, ref, 1.0, 0.0, e2)
    torch.cuda.synchronize()
    assert err == 0 and int(e2.item()) == 0
    ref = ref.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("act", [1, 0])
@pytest.mark.parametrize("n,h,w,C,cout", [(2, 21, 13, 32, 136), (2, 37, 21, 32, 24), (3, 40, 18, 48, 64)])
def test_conv3_tma_bias_act_equals_the_unfused_pair_bitwise(act, n, h, w, C, cout):
    """Bias and SiLU in the convolution's epilogue give exactly what smrt_nn_conv3_tma followed by
    smrt_nn_bias_act_blocked gives (z, a and the blocked halves), on ragged tiles: two N tiles of
    128, and one output-channel block of 32 or 64."""
    import torch
    r = _rng(90 + act)
    x = r.normal(size=(n, h, w, C)).astype(np.float16)
    wt = torch.tensor(r.normal(size=(cout, 9 * C)).astype(np.float16), device="cuda")
    bias = torch.tensor(r.normal(size=cout).astype(np.float32), device="cuda")
    xb = torch.tensor(_blocked(x), device="cuda")
    wp = torch.empty(S.smrt_nn_pack3_halves(cout, C), dtype=torch.float16, device="cuda")
    S.smrt_nn_pack3(wt, C, wp)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = torch.empty((n, h, w, cout), device="cuda")
    S.smrt_nn_conv3_tma(xb, (n, h, w, C), wp, y, cout, 1.0, 0.0, err)
    z1, a1 = torch.empty_like(y), torch.empty_like(y)
    ab1 = torch.empty(y.numel(), dtype=torch.float16, device="cuda")
    S.smrt_nn_bias_act_blocked(y, bias, act, z1, a1, ab1)
    z2, a2 = torch.empty_like(y), torch.empty_like(y)
    ab2 = torch.empty(y.numel(), dtype=torch.float16, device="cuda")
    S.smrt_nn_conv3_tma_bias_act(xb, (n, h, w, C), wp, cout, bias, act, z2, a2, ab2, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert torch.equal(z1, z2) and torch.equal(a1, a2) and torch.equal(ab1, ab2)


def _wgrad(n, h, w, C, cout, alpha, seed):
    import torch
    r = _rng(seed)
    x = r.normal(size=(n, h, w, C)).astype(np.float16)
    dz = r.normal(size=(n, h, w, cout)).astype(np.float16)
    g0 = r.normal(size=(cout, 9 * C)).astype(np.float32)
    gw = torch.tensor(g0, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.smrt_nn_conv3_wgrad_tma(torch.tensor(_blocked(x), device="cuda"), (n, h, w, C),
                              torch.tensor(_blocked(dz), device="cuda"), cout, gw, alpha, err)
    torch.cuda.synchronize()
    exp = g0 + alpha * dz.astype(np.float64).reshape(-1, cout).T @ U.im2col3(x.astype(np.float64))
    return gw.cpu().numpy(), exp, int(err.item())


@pytest.mark.parametrize("n,h,w,C,cout", [
    (2, 37, 21, 16, 24),      # ragged tiles, 2 of 16 channel planes (the MMA's other rows unused)
    (1, 32, 40, 32, 32),      # the top U-Net level's shape
    (1, 20, 12, 136, 40),     # two input-channel blocks (the second holds one plane), two output blocks
    (3, 5, 3, 8, 8),          # images smaller than the tile and the halo box
    (4, 64, 64, 96, 32),      # 128 pixel tiles split over the SMs, atomics from many blocks
    (4, 128, 256, 16, 32),    # 1,024 tiles: several per block, every pipeline stage reused
])
def test_conv3_wgrad_tma_matches_fp64_product_of_the_same_halves(n, h, w, C, cout):
    got, exp, err = _wgrad(n, h, w, C, cout, 0.5, seed=C + 7 * cout)
    assert err == 0
    d = np.abs(got - exp).max() / np.abs(exp).max()
    assert d <= 1e-4, d


def test_tma_kernels_reject_unsupported_arguments():
    import torch
    y = torch.zeros((16, 8), device="cuda")
    wp = torch.zeros(9 * 24 * 32, dtype=torch.float16, device="cuda")
    xb = torch.zeros(16 * 24, dtype=torch.float16, device="cuda")
    with pytest.raises(S.SmrtError) as ei:                   # C % 16 != 0
        S.smrt_nn_conv3_tma(xb, (1, 4, 4, 24), wp, y, 8)
    assert ei.value.status == S.SMRT_ERR_ARG
    xm = torch.zeros(16 * 16 + 1, dtype=torch.float16, device="cuda")[1:]       # misaligned
    with pytest.raises(S.SmrtError) as ei:
        S.smrt_nn_conv3_tma(xm, (1, 4, 4, 16), wp, y, 8)
    assert ei.value.status == S.SMRT_ERR_ARG
    with pytest.raises(S.SmrtError) as ei:
        S.smrt_nn_pack3(torch.zeros((8, 9 * 24), dtype=torch.float16, device="cuda"), 24, wp)
    assert ei.value.status == S.SMRT_ERR_ARG
    gw = torch.zeros((12, 9 * 16), device="cuda")
    with pytest.raises(S.SmrtError) as ei:                   # cout % 8 != 0
        S.smrt_nn_conv3_wgrad_tma(xb, (1, 4, 4, 16), xb, 12, gw)
    assert ei.value.status == S.SMRT_ERR_ARG
    assert S.smrt_nn_pack3_halves(8, 24) == -1


def test_wait_timeout_is_reported_and_the_next_call_runs():
    """Failure path of the bounded tensor-core waits: with the TMA producer withholding every copy
    and a 1 ms limit, every block's wait runs out (nothing is ever in flight).  smrt_nn_check then
    returns SMRT_ERR_TIMEOUT and resets the error word, the output is untouched, tensor memory was
    released (the next launch allocates it again), and the next ordinary call is correct -- twice."""
    import torch
    n, h, w, C, cout = 2, 37, 21, 32, 40          # 3 x 3 x 2 x 2 = 36 blocks, two output tiles each
    r = _rng(4242)
    x = r.normal(size=(n, h, w, C)).astype(np.float16)
    wt = r.normal(size=(cout, 9 * C)).astype(np.float16)
    xb = torch.tensor(_blocked(x), device="cuda")
    wp = torch.empty(S.smrt_nn_pack3_halves(cout, C), dtype=torch.float16, device="cuda")
    S.smrt_nn_pack3(torch.tensor(wt, device="cuda"), C, wp)
    exp = U.im2col3(x.astype(np.float64)) @ wt.astype(np.float64).T
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        y = torch.full((n * h * w, cout), float("nan"), device="cuda")
        S.smrt_nn_conv3_tma_wait_test(xb, (n, h, w, C), wp, y, cout, err, wait_ms=1.0)
        with pytest.raises(S.SmrtError) as ei:
            S.smrt_nn_check(err)
        assert ei.value.status == S.SMRT_ERR_TIMEOUT
        assert int(err.item()) == 0                       # the check resets the word
        assert bool(torch.isnan(y).all())                 # blocks that gave up wrote nothing
        S.smrt_nn_conv3_tma(xb, (n, h, w, C), wp, y, cout, 1.0, 0.0, err)
        S.smrt_nn_check(err)                              # no timeout on the ordinary call
        got = y.cpu().numpy()
        assert np.abs(got - exp).max() <= 1e-4 * np.abs(exp).max()
    with pytest.raises(S.SmrtError) as ei:
        S.smrt_nn_conv3_tma_wait_test(xb, (n, h, w, C), wp, y, cout, err, wait_ms=0.0)
    assert ei.value.status == S.SMRT_ERR_ARG


@pytest.mark.parametrize("act", [1, 0])
@pytest.mark.parametrize("n,h,w,C,cout", [(2, 37, 21, 32, 16), (1, 32, 40, 64, 32), (2, 18, 10, 32, 136),
                                         (10, 70, 40, 32, 136), (16, 70, 44, 48, 48)])
def test_conv3_tma_act_bwd_equals_the_unfused_pair(n, h, w, C, cout, act):
    """The input gradient with the SiLU backward of the producing layer in its epilogue gives exactly the
    blocked halves and float32 dz that smrt_nn_conv3_tma followed by smrt_nn_bias_act_bwd_blocked give,
    and the same bias gradient up to summation order."""
    import torch
    r = _rng(700 + C + cout + act)
    dz_b = r.normal(size=(n, h, w, C)).astype(np.float16)
    wt = torch.tensor(r.normal(size=(cout, 9 * C)).astype(np.float16), device="cuda")
    z = torch.tensor(r.normal(size=(n, h, w, cout)).astype(np.float32), device="cuda")
    db0 = r.normal(size=cout).astype(np.float32)
    xb = torch.tensor(_blocked(dz_b), device="cuda")
    wp = torch.empty(S.smrt_nn_pack3_halves(cout, C), dtype=torch.float16, device="cuda")
    S.smrt_nn_pack3(wt, C, wp)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    # unfused
    d = torch.empty((n, h, w, cout), device="cuda")
    S.smrt_nn_conv3_tma(xb, (n, h, w, C), wp, d, cout, 1.0, 0.0, err)
    dz1 = torch.empty_like(d)
    dzb1 = torch.empty(d.numel(), dtype=torch.float16, device="cuda")
    db1 = torch.tensor(db0, device="cuda")
    S.smrt_nn_bias_act_bwd_blocked(d, z, act, dz1, db1, dzb1)
    # fused
    dz2 = torch.empty_like(d)
    dzb2 = torch.empty_like(dzb1)
    db2 = torch.tensor(db0, device="cuda")
    S.smrt_nn_conv3_tma_act_bwd(xb, (n, h, w, C), wp, cout, z, act, dz2, db2, dzb2, err)
    dzb3 = torch.empty_like(dzb1)
    S.smrt_nn_conv3_tma_act_bwd(xb, (n, h, w, C), wp, cout, z, act, None, None, dzb3, err)
    S.smrt_nn_check(err)
    assert torch.equal(dz1, dz2) and torch.equal(dzb1, dzb2) and torch.equal(dzb1, dzb3)
    ref = db1.cpu().numpy().astype(np.float64)
    assert np.abs(db2.cpu().numpy() - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def test_pack3_many_equals_the_separate_calls():
    """One launch for every packed array of a network gives the bits of the separate conversion, padding,
    flip and pack calls: forward operands (one zero-padded input layer), adjoint operands, ragged tiles."""
    import torch
    r = _rng(55)
    layers = [(32, 3, 16), (64, 32, 32), (48, 96, 96), (130, 32, 32), (256, 128, 128)]   # cout, cin, cpad
    descs, expect = [], []
    for cout, cin, cpad in layers:
        w = torch.tensor(r.normal(size=(cout, 9 * cin)).astype(np.float32), device="cuda")
        if cpad != cin:
            wh = torch.empty((cout, 9 * cpad), dtype=torch.float16, device="cuda")
            S.smrt_nn_pad3(w, cin, cpad, wh)
        else:
            wh = w.half()
        ref = torch.empty(S.smrt_nn_pack3_halves(cout, cpad), dtype=torch.float16, device="cuda")
        S.smrt_nn_pack3(wh, cpad, ref)
        dst = torch.full_like(ref, float("nan"))
        descs.append((w, dst, S.SMRT_NN_PACK_FORWARD, cout, cin, cpad))
        expect.append((dst, ref))
        if cout % 16 == 0:
            f = torch.empty((cin, 9 * cout), dtype=torch.float16, device="cuda")
            S.smrt_nn_flip3(w, f)
            ref_a = torch.empty(S.smrt_nn_pack3_halves(cin, cout), dtype=torch.float16, device="cuda")
            S.smrt_nn_pack3(f, cout, ref_a)
            dst_a = torch.full_like(ref_a, float("nan"))
            descs.append((w, dst_a, S.SMRT_NN_PACK_ADJOINT, cout, cin, cin))
            expect.append((dst_a, ref_a))
    S.smrt_nn_pack3_many(descs)
    torch.cuda.synchronize()
    for dst, ref in expect:
        assert torch.equal(dst, ref)


@pytest.mark.parametrize("act", [1, 0])
def test_bias_act_bwd_addpool_equals_pool_add_then_bias_act_bwd(act):
    """The encoder's SiLU backward of (skip part + pooling adjoint of the pooled part) in one pass equals
    avgpool2_bwd, add and bias_act_bwd_blocked in turn (dz and its halves bit for bit, db up to order)."""
    import torch
    n, h, w, c = 2, 20, 14, 48
    r = _rng(31 + act)
    da = torch.tensor(r.normal(size=(n, h, w, c)).astype(np.float32), device="cuda")
    dp = torch.tensor(r.normal(size=(n, h // 2, w // 2, c)).astype(np.float32), device="cuda")
    z = torch.tensor(r.normal(size=(n, h, w, c)).astype(np.float32), device="cuda")
    db0 = r.normal(size=c).astype(np.float32)
    up = torch.empty_like(da)
    S.smrt_nn_avgpool2_bwd(dp, (n, h, w, c), up)
    s = torch.empty_like(da)
    S.smrt_nn_add(da, up, s)
    dz1, dzb1, db1 = torch.empty_like(da), torch.empty(da.numel(), dtype=torch.float16, device="cuda"), \
        torch.tensor(db0, device="cuda")
    S.smrt_nn_bias_act_bwd_blocked(s, z, act, dz1, db1, dzb1)
    dz2, dzb2, db2 = torch.empty_like(da), torch.empty_like(dzb1), torch.tensor(db0, device="cuda")
    S.smrt_nn_bias_act_bwd_addpool_blocked(da, dp, z, act, dz2, db2, dzb2)
    torch.cuda.synchronize()
    assert torch.equal(dz1, dz2) and torch.equal(dzb1, dzb2)
    assert np.abs(db1.cpu().numpy() - db2.cpu().numpy()).max() <= 1e-5 * max(1.0, np.abs(db0).max())
