"""smrt_nn_conv3_tma (TMA-fed operands, nine taps as shifted views of one zero-padded input tile)
against an FP64 product of the same half operands, and against smrt_nn_conv3_tc; smrt_nn_pack3's
layout element by element."""
import numpy as np
import pytest

import paper_2409_01076_gb300 as S
from oracle import unet_oracle as U

pytestmark = pytest.mark.gpu


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_pack3_layout():
    import torch
    cout, C = 5, 32
    w = _rng(1).normal(size=(cout, 9 * C)).astype(np.float16)
    wp = torch.empty(9 * C * cout, dtype=torch.float16, device="cuda")
    S.smrt_nn_pack3(torch.tensor(w, device="cuda"), C, wp)
    torch.cuda.synchronize()
    got = wp.cpu().numpy().reshape(9 * C // 8, cout, 8)
    for chunk in range(C // 16):
        for tap in range(9):
            for q in range(2):
                kg = (chunk * 9 + tap) * 2 + q
                c0 = tap * C + chunk * 16 + q * 8
                assert np.array_equal(got[kg], w[:, c0:c0 + 8]), (chunk, tap, q)


def _conv(n, h, w, C, cout, alpha, beta, seed):
    import torch
    r = _rng(seed)
    x = r.normal(size=(n, h, w, C)).astype(np.float16)
    wt = r.normal(size=(cout, 9 * C)).astype(np.float16)
    y0 = r.normal(size=(n * h * w, cout)).astype(np.float32)
    xd = torch.tensor(x, device="cuda")
    wd = torch.tensor(wt, device="cuda")
    wp = torch.empty(9 * C * cout, dtype=torch.float16, device="cuda")
    S.smrt_nn_pack3(wd, C, wp)
    y = torch.tensor(y0, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.smrt_nn_conv3_tma(xd, wp, y, cout, alpha, beta, err)
    torch.cuda.synchronize()
    exp = alpha * U.im2col3(x.astype(np.float64)) @ wt.astype(np.float64).T + beta * y0
    return y.cpu().numpy(), exp, int(err.item()), (xd, wd, y0)


@pytest.mark.parametrize("n,h,w,C,cout", [
    (2, 37, 21, 16, 20),      # ragged tiles in both directions, cout < 32
    (1, 32, 40, 32, 32),      # the top U-Net level's shape (2 chunks)
    (2, 18, 10, 48, 64),      # one tile per image, 3 chunks, TN 64
    (1, 16, 8, 80, 48),       # 5 chunks: the 4 stages are reused
    (1, 20, 12, 96, 130),     # two 128-wide output-channel tiles, the second partial
    (1, 24, 16, 384, 128),    # the widest decoder input (24 chunks)
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
    got, _, err, (xd, wd, y0) = _conv(n, h, w, C, cout, 1.0, 0.0, seed=5)
    ref = torch.zeros((n * h * w, cout), device="cuda")
    e2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.smrt_nn_conv3_tc(xd.float(), wd, ref, 1.0, 0.0, e2)
    torch.cuda.synchronize()
    assert err == 0 and int(e2.item()) == 0
    ref = ref.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_conv3_tma_rejects_unsupported_arguments():
    import torch
    xh = torch.zeros((1, 4, 4, 24), dtype=torch.float16, device="cuda")     # C % 16 != 0
    wp = torch.zeros(9 * 24 * 8, dtype=torch.float16, device="cuda")
    y = torch.zeros((16, 8), device="cuda")
    with pytest.raises(S.SmrtError) as ei:
        S.smrt_nn_conv3_tma(xh, wp, y, 8)
    assert ei.value.status == S.SMRT_ERR_ARG
    xm = torch.zeros(16 * 16 + 1, dtype=torch.float16, device="cuda")[1:].view(1, 4, 4, 16)   # misaligned
    with pytest.raises(S.SmrtError) as ei:
        S.smrt_nn_conv3_tma(xm, wp, y, 8)
    assert ei.value.status == S.SMRT_ERR_ARG
    with pytest.raises(S.SmrtError) as ei:
        S.smrt_nn_pack3(torch.zeros((8, 9 * 24), dtype=torch.float16, device="cuda"), 24, wp)
    assert ei.value.status == S.SMRT_ERR_ARG
