"""smrt_nn_gemm_tc (tcgen05 tensor cores, accumulator in tensor memory) against numpy on the
same half-rounded operands, and against the WMMA smrt_nn_gemm."""
import numpy as np
import pytest

import paper_2409_01076_gb300 as S

pytestmark = pytest.mark.gpu


def _case(transA, transB, M, N, K, split, seed):
    import torch
    r = np.random.Generator(np.random.PCG64(seed))
    a = r.normal(size=(K, M) if transA else (M, K)).astype(np.float16)
    b = r.normal(size=(N, K) if transB else (K, N)).astype(np.float16)
    c0 = r.normal(size=(M, N)).astype(np.float32)
    A = torch.tensor(a, device="cuda")
    B = torch.tensor(b, device="cuda")
    C = torch.tensor(c0, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    beta = 1.0 if split > 1 else -0.5
    S.smrt_nn_gemm_tc(transA, transB, M, N, K, 1.5, A, a.shape[1], B, b.shape[1], beta, C, N, split, err)
    torch.cuda.synchronize()
    opa = a.astype(np.float64).T if transA else a.astype(np.float64)
    opb = b.astype(np.float64).T if transB else b.astype(np.float64)
    ref = 1.5 * opa @ opb + (1.0 if split > 1 else -0.5) * c0
    return C.cpu().double().numpy(), ref, int(err.item())


@pytest.mark.parametrize("transA", [0, 1])
@pytest.mark.parametrize("transB", [0, 1])
def test_gemm_tc_single_tile(transA, transB):
    got, ref, err = _case(transA, transB, 128, 128, 64, 1, 1)
    assert err == 0
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("transA", [0, 1])
@pytest.mark.parametrize("transB", [0, 1])
@pytest.mark.parametrize("split", [1, 4])
def test_gemm_tc_ragged_multi_tile(transA, transB, split):
    got, ref, err = _case(transA, transB, 300, 200, 520, split, 2 + transA + 2 * transB)
    assert err == 0
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


def test_gemm_tc_matches_wmma_on_a_conv_shape():
    """The weight-gradient shape of the top U-Net level: K is the pixel count."""
    import torch
    r = np.random.Generator(np.random.PCG64(7))
    M, N, K = 32, 288, 8192
    a = torch.tensor(r.normal(size=(K, M)).astype(np.float16), device="cuda")
    b = torch.tensor(r.normal(size=(K, N)).astype(np.float16), device="cuda")
    c1 = torch.zeros((M, N), device="cuda")
    c2 = torch.zeros((M, N), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.smrt_nn_gemm_tc(1, 0, M, N, K, 1.0, a, M, b, N, 1.0, c1, N, 16, err)
    S.smrt_nn_gemm(1, 0, M, N, K, 1.0, a, M, b, N, 1.0, c2, N, 16)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    d = (c1 - c2).abs().max().item()
    assert d <= 1e-4 * c2.abs().max().item()


@pytest.mark.parametrize("N", [20, 50, 200])
@pytest.mark.parametrize("trans_c", [0, 1])
@pytest.mark.parametrize("transA,transB", [(0, 1), (1, 0)])
def test_gemm_tc_tile_widths_and_transposed_store(N, trans_c, transA, transB):
    """32-, 64- and 128-wide tiles; C or C^T stored; odd K (scalar copy path) and even K (vector path)."""
    import torch
    for K in (27, 264):
        r = np.random.Generator(np.random.PCG64(N + K + 7 * trans_c))
        M = 200
        a = r.normal(size=(K, M) if transA else (M, K)).astype(np.float16)
        b = r.normal(size=(N, K) if transB else (K, N)).astype(np.float16)
        opa = a.astype(np.float64).T if transA else a.astype(np.float64)
        opb = b.astype(np.float64).T if transB else b.astype(np.float64)
        ref = opa @ opb
        C = torch.zeros((N, M) if trans_c else (M, N), device="cuda")
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        S.smrt_nn_gemm_tc(transA, transB | (2 * trans_c), M, N, K, 1.0, torch.tensor(a, device="cuda"), a.shape[1],
                          torch.tensor(b, device="cuda"), b.shape[1], 0.0, C, M if trans_c else N, 1, err)
        torch.cuda.synchronize()
        got = C.cpu().double().numpy()
        if trans_c:
            got = got.T
        assert int(err.item()) == 0
        assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max(), (K, N)


def test_flip3_is_the_adjoint_convolution_weight():
    """<conv(x, W), dz> = <x, conv(dz, flip(W))> on a small zero-padded lattice."""
    import torch
    from oracle import unet_oracle as U
    r = np.random.Generator(np.random.PCG64(11))
    cout, cin = 5, 3
    w = r.normal(size=(cout, 9 * cin))
    wf = torch.empty((cin, 9 * cout), dtype=torch.float16, device="cuda")
    S.smrt_nn_flip3(torch.tensor(w, dtype=torch.float32, device="cuda"), wf)
    torch.cuda.synchronize()
    f = wf.cpu().double().numpy()
    for c in range(cin):
        for tap in range(9):
            for o in range(cout):
                assert f[c, tap * cout + o] == np.float16(w[o, (8 - tap) * cin + c])
    x = r.normal(size=(1, 6, 5, cin))
    dz = r.normal(size=(1, 6, 5, cout))
    y = (U.im2col3(x) @ w.T).reshape(1, 6, 5, cout)
    dx = (U.im2col3(dz) @ f.T).reshape(1, 6, 5, cin)
    assert abs((y * dz).sum() - (x * dx).sum()) < 1e-2 * np.abs(y * dz).sum()


@pytest.mark.parametrize("C,cout", [(8, 20), (16, 64), (40, 130), (32, 32)])
def test_conv3_tc_equals_im2col_then_gemm_bitwise(C, cout):
    """The implicit-GEMM convolution gathers the same half A tiles as im2col and runs the same MMAs:
    its output is bit-identical to im2col + smrt_nn_gemm_tc, on ragged images (7 x 11, 3 of them,
    231 pixels: two 128-row tiles, the second partial) and with beta != 0."""
    import torch
    r = np.random.Generator(np.random.PCG64(C * 1000 + cout))
    n, h, w = 3, 7, 11
    x = torch.tensor(r.normal(size=(n, h, w, C)).astype(np.float32), device="cuda")
    wt = torch.tensor(r.normal(size=(cout, 9 * C)).astype(np.float16), device="cuda")
    y0 = torch.tensor(r.normal(size=(n * h * w, cout)).astype(np.float32), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    col = torch.empty((n * h * w, 9 * C), dtype=torch.float16, device="cuda")
    S.smrt_nn_im2col3(x, col)
    ref = y0.clone()
    S.smrt_nn_gemm_tc(0, 1, n * h * w, cout, 9 * C, 0.75, col, 9 * C, wt, 9 * C, 0.5, ref, cout, 1, err)
    got = y0.clone()
    S.smrt_nn_conv3_tc(x, wt, got, 0.75, 0.5, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert torch.equal(got, ref)
    # and against plain arithmetic on the same half operands
    from oracle import unet_oracle as U
    xh = x.cpu().numpy().astype(np.float16).astype(np.float64)
    exp = 0.75 * U.im2col3(xh) @ wt.cpu().numpy().astype(np.float64).T + 0.5 * y0.cpu().numpy()
    assert np.abs(got.cpu().numpy() - exp).max() <= 1e-4 * np.abs(exp).max()


def test_conv3_tc_rejects_unsupported_channels():
    import torch
    x = torch.zeros((1, 4, 4, 12), device="cuda")
    wt = torch.zeros((8, 108), dtype=torch.float16, device="cuda")
    y = torch.zeros((16, 8), device="cuda")
    with pytest.raises(S.SmrtError) as ei:
        S.smrt_nn_conv3_tc(x, wt, y)
    assert ei.value.status == S.SMRT_ERR_ARG
