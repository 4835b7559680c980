"""Bindings of include/smrt_nn.h (same names; argument marshalling only).

Tensors are CUDA torch tensors on the current device; every call runs on the
current torch stream.  A non-OK status raises SmrtError.
"""
from __future__ import annotations

import ctypes

from . import _lib


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _s():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(rc):
    if rc != 0:
        from . import SmrtError, smrt_last_error
        raise SmrtError(rc, smrt_last_error(None))


def smrt_nn_gemm(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, split_k=1):
    _check(_lib.load().smrt_nn_gemm(int(transA), int(transB), int(M), int(N), int(K), float(alpha), _p(A), int(lda),
                                    _p(B), int(ldb), float(beta), _p(C), int(ldc), int(split_k), _s()))


def smrt_nn_gemm_tc(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, split_k=1, err=None):
    _check(_lib.load().smrt_nn_gemm_tc(int(transA), int(transB), int(M), int(N), int(K), float(alpha), _p(A),
                                       int(lda), _p(B), int(ldb), float(beta), _p(C), int(ldc), int(split_k),
                                       _p(err), _s()))


def smrt_nn_conv3_tc(x, w, y, alpha=1.0, beta=0.0, err=None):
    """x: (N, H, W, C) float32; w: (cout, 9C) half; y: N*H*W rows of cout float32 (any view)."""
    n, h, wd, c = x.shape
    cout = w.shape[0]
    _check(_lib.load().smrt_nn_conv3_tc(_p(x), n, h, wd, c, _p(w), int(cout), float(alpha), float(beta), _p(y),
                                        int(y.shape[-1]), _p(err), _s()))


def smrt_nn_to_half_blocked(x, xb, scale=1.0):
    """x: (N, H, W, C) float32; xb: N*C*H*W halves, written as [N][C/8][H][W][8]."""
    n, h, w, c = x.shape
    _check(_lib.load().smrt_nn_to_half_blocked(_p(x), n, h, w, c, float(scale), _p(xb), _s()))


def smrt_nn_to_half_blocked_pad(x, cb, xb, scale=1.0):
    """x: (N, H, W, C) float32; xb: N*cb*H*W halves, blocked, channels C..cb-1 zero."""
    n, h, w, c = x.shape
    _check(_lib.load().smrt_nn_to_half_blocked_pad(_p(x), n, h, w, c, int(cb), float(scale), _p(xb), _s()))


def smrt_nn_pad3(w, C, Cp, wh):
    """w: (cout, 9C) float32; wh: (cout, 9Cp) half."""
    _check(_lib.load().smrt_nn_pad3(_p(w), int(w.shape[0]), int(C), int(Cp), _p(wh), _s()))


def smrt_nn_unpad3_add(gp, C, Cp, gw):
    """gw (cout, 9C) float32 += the C-channel part of gp (cout, 9Cp)."""
    _check(_lib.load().smrt_nn_unpad3_add(_p(gp), int(gw.shape[0]), int(C), int(Cp), _p(gw), _s()))


def smrt_nn_pack3_halves(cout, C):
    return int(_lib.load().smrt_nn_pack3_halves(int(cout), int(C)))


def smrt_nn_pack3(w, C, wp):
    """w: (cout, 9C) half; wp: smrt_nn_pack3_halves(cout, C) halves (any shape)."""
    _check(_lib.load().smrt_nn_pack3(_p(w), int(w.shape[0]), int(C), _p(wp), _s()))


def smrt_nn_conv3_tma(xb, nhwc, wp, y, cout, alpha=1.0, beta=0.0, err=None):
    """xb: blocked half activations of shape nhwc = (N, H, W, C); y: N*H*W rows of cout float32."""
    n, h, w, c = nhwc
    _check(_lib.load().smrt_nn_conv3_tma(_p(xb), int(n), int(h), int(w), int(c), _p(wp), int(cout), float(alpha),
                                         float(beta), _p(y), int(y.shape[-1]), _p(err), _s()))


SMRT_NN_PACK_FORWARD, SMRT_NN_PACK_ADJOINT = 0, 1


class _PackDesc(ctypes.Structure):
    _fields_ = [("w", ctypes.c_void_p), ("dst", ctypes.c_void_p), ("kind", ctypes.c_int), ("cout", ctypes.c_int),
                ("cin", ctypes.c_int), ("cpad", ctypes.c_int)]


def smrt_nn_pack3_many(descs):
    """descs: [(w float32 (cout, 9 cin), dst halves, kind, cout, cin, cpad)] -> every packed array in one launch."""
    arr = (_PackDesc * len(descs))()
    for k, (w, dst, kind, cout, cin, cpad) in enumerate(descs):
        arr[k] = _PackDesc(w.data_ptr(), dst.data_ptr(), int(kind), int(cout), int(cin), int(cpad))
    _check(_lib.load().smrt_nn_pack3_many(len(descs), arr, _s()))


def smrt_nn_conv3_tma_act_bwd(dzb, nhwc, wp, cout, z, act, dz, db, dzb_out, err=None):
    """Input gradient of B (blocked half dz of shape nhwc, flipped packed weights wp) fused with A's SiLU
    backward: dzb_out (blocked halves, cout channels), dz (N*H*W x cout float32 or None), db += column sums."""
    n, h, w, c = nhwc
    _check(_lib.load().smrt_nn_conv3_tma_act_bwd(_p(dzb), int(n), int(h), int(w), int(c), _p(wp), int(cout), _p(z),
                                                 int(act), _p(dz), _p(db), _p(dzb_out), _p(err), _s()))


def smrt_nn_check(err):
    """Raises SmrtError(SMRT_ERR_TIMEOUT) (and resets err) if a tensor-core wait gave up; waits for the stream."""
    _check(_lib.load().smrt_nn_check(_p(err), _s()))


def smrt_nn_conv3_tma_wait_test(xb, nhwc, wp, y, cout, err, wait_ms=1.0):
    """Failure-path test hook: smrt_nn_conv3_tma with a withheld producer and a wait limit of wait_ms."""
    n, h, w, c = nhwc
    _check(_lib.load().smrt_nn_conv3_tma_wait_test(_p(xb), int(n), int(h), int(w), int(c), _p(wp), int(cout), _p(y),
                                                   int(y.shape[-1]), _p(err), float(wait_ms), _s()))


def smrt_nn_conv3_tma_bias_act(xb, nhwc, wp, cout, bias, act, z, a, ab, err=None):
    """Forward convolution with bias and activation in the epilogue; z, a: N*H*W rows of cout float32 or
    None; ab: blocked halves or None."""
    n, h, w, c = nhwc
    _check(_lib.load().smrt_nn_conv3_tma_bias_act(_p(xb), int(n), int(h), int(w), int(c), _p(wp), int(cout),
                                                  _p(bias), int(act), _p(z), _p(a), _p(ab), _p(err), _s()))


def smrt_nn_conv3_wgrad_tma(xb, nhwc, dzb, cout, gw, alpha=1.0, err=None):
    """gw (cout, ldg >= 9C) float32 += alpha * weight gradient from blocked half x and dz."""
    n, h, w, c = nhwc
    _check(_lib.load().smrt_nn_conv3_wgrad_tma(_p(xb), int(n), int(h), int(w), int(c), _p(dzb), int(cout),
                                               float(alpha), _p(gw), int(gw.shape[-1]), _p(err), _s()))


def smrt_nn_im2col3(x, col):
    """col: (N*H*W, ld) half with ld >= 9*C (the row stride is taken from col)."""
    n, h, w, c = x.shape
    _check(_lib.load().smrt_nn_im2col3(_p(x), n, h, w, c, _p(col), int(col.shape[-1]), _s()))


def smrt_nn_col2im3(dcol, shape, dx):
    n, h, w, c = shape
    _check(_lib.load().smrt_nn_col2im3(_p(dcol), n, h, w, c, _p(dx), _s()))


def smrt_nn_flip3(w, wf):
    cout, k9 = w.shape
    _check(_lib.load().smrt_nn_flip3(_p(w), int(cout), int(k9 // 9), _p(wf), _s()))


def smrt_nn_to_half(src, dst, scale=1.0):
    _check(_lib.load().smrt_nn_to_half(_p(src), src.numel(), float(scale), _p(dst), _s()))


def smrt_nn_to_half_rows(src, dst, scale=1.0):
    """src: (rows, cols) float32; dst: (rows, ld) half, ld >= cols, pad columns zeroed."""
    rows, cols = src.shape[0], src.numel() // max(src.shape[0], 1)
    _check(_lib.load().smrt_nn_to_half_rows(_p(src), int(rows), int(cols), float(scale), _p(dst),
                                            int(dst.shape[-1]), _s()))


def smrt_nn_bias_act(x, bias, act, z, a):
    rows = x.numel() // x.shape[-1]
    _check(_lib.load().smrt_nn_bias_act(_p(x), _p(bias), rows, x.shape[-1], int(act), _p(z), _p(a), _s()))


def smrt_nn_bias_act_bwd(da, z, act, dz, db):
    rows = da.numel() // da.shape[-1]
    _check(_lib.load().smrt_nn_bias_act_bwd(_p(da), _p(z), rows, da.shape[-1], int(act), _p(dz), _p(db), _s()))


def smrt_nn_avgpool2(x, y):
    n, h, w, c = x.shape
    _check(_lib.load().smrt_nn_avgpool2(_p(x), n, h, w, c, _p(y), _s()))


def smrt_nn_avgpool2_bwd(dy, shape, dx):
    n, h, w, c = shape
    _check(_lib.load().smrt_nn_avgpool2_bwd(_p(dy), n, h, w, c, _p(dx), _s()))


def smrt_nn_upsample2(x, y):
    n, h, w, c = x.shape
    _check(_lib.load().smrt_nn_upsample2(_p(x), n, h, w, c, _p(y), _s()))


def smrt_nn_upsample2_bwd(dy, shape, dx):
    n, h, w, c = shape
    _check(_lib.load().smrt_nn_upsample2_bwd(_p(dy), n, h, w, c, _p(dx), _s()))


def smrt_nn_concat(a, b, y):
    rows = a.numel() // a.shape[-1]
    _check(_lib.load().smrt_nn_concat(_p(a), a.shape[-1], _p(b), b.shape[-1], rows, _p(y), _s()))


def smrt_nn_concat_bwd(dy, ca, cb, da, db):
    rows = dy.numel() // dy.shape[-1]
    _check(_lib.load().smrt_nn_concat_bwd(_p(dy), int(ca), int(cb), rows, _p(da), _p(db), _s()))


def smrt_nn_add(a, b, y):
    _check(_lib.load().smrt_nn_add(_p(a), _p(b), a.numel(), _p(y), _s()))


def smrt_nn_conv1x1_small(x, w, bias, y):
    """x: (..., C) float32; w: (cout, C) float32, cout <= 3; bias: (cout) or None; y: (..., cout)."""
    c = x.shape[-1]
    _check(_lib.load().smrt_nn_conv1x1_small(_p(x), x.numel() // c, int(c), _p(w), _p(bias), int(w.shape[0]), _p(y),
                                             _s()))


def smrt_nn_conv1x1_small_bwd(dy, x, w, dx, dw, db):
    """Backward of smrt_nn_conv1x1_small: dx (like x) written, dw (cout, C) and db (cout) accumulated."""
    c = x.shape[-1]
    _check(_lib.load().smrt_nn_conv1x1_small_bwd(_p(dy), _p(x), x.numel() // c, int(c), _p(w), int(w.shape[0]),
                                                 _p(dx), _p(dw), _p(db), _s()))


def smrt_nn_bias_act_blocked(x, bias, act, z, a, ab):
    """x: (N, H, W, C) float32 (C % 8 == 0); z, a: like x or None; ab: N*C*H*W halves (blocked) or None."""
    n, h, w, c = x.shape
    _check(_lib.load().smrt_nn_bias_act_blocked(_p(x), _p(bias), n, h, w, c, int(act), _p(z), _p(a), _p(ab), _s()))


def smrt_nn_bias_act_bwd_blocked(da, z, act, dz, db, dzb):
    """da: (N, H, W, C) float32; dz like da or None; db (C) accumulated or None; dzb blocked halves or None."""
    n, h, w, c = da.shape
    _check(_lib.load().smrt_nn_bias_act_bwd_blocked(_p(da), _p(z), n, h, w, c, int(act), _p(dz), _p(db), _p(dzb),
                                                    _s()))


def smrt_nn_bias_act_bwd_addpool_blocked(da, dp, z, act, dz, db, dzb):
    """smrt_nn_bias_act_bwd_blocked of da (N, H, W, C) + the pooling adjoint of dp (N, H/2, W/2, C)."""
    n, h, w, c = da.shape
    _check(_lib.load().smrt_nn_bias_act_bwd_addpool_blocked(_p(da), _p(dp), _p(z), n, h, w, c, int(act), _p(dz),
                                                            _p(db), _p(dzb), _s()))


def smrt_nn_avgpool2_blocked(x, y, yb):
    """x: (N, H, W, C) float32; y: (N, H/2, W/2, C) float32 or None; yb: blocked halves or None."""
    n, h, w, c = x.shape
    _check(_lib.load().smrt_nn_avgpool2_blocked(_p(x), n, h, w, c, _p(y), _p(yb), _s()))


def smrt_nn_upcat(a, b, y, yb):
    """a: (N, H, W, Ca); b: (N, 2H, 2W, Cb); y: (N, 2H, 2W, Ca + Cb) float32 or None; yb: blocked or None."""
    n, h, w, ca = a.shape
    _check(_lib.load().smrt_nn_upcat(_p(a), n, h, w, ca, _p(b), int(b.shape[3]), _p(y), _p(yb), _s()))


def smrt_nn_upcat_bwd(dy, ca, da, db):
    """dy: (N, 2H, 2W, Ca + Cb); da: (N, H, W, Ca) or None; db: (N, 2H, 2W, Cb) or None."""
    n, h2, w2, cy = dy.shape
    _check(_lib.load().smrt_nn_upcat_bwd(_p(dy), n, h2 // 2, w2 // 2, int(ca), int(cy - ca), _p(da), _p(db), _s()))


def smrt_nn_mse(y, t, grad_scale, loss, dy):
    _check(_lib.load().smrt_nn_mse(_p(y), _p(t), y.numel(), float(grad_scale), _p(loss), _p(dy), _s()))


def smrt_nn_adam(w, grad, m, v, lr, b1, b2, eps, step, grad_scale, found_inf):
    _check(_lib.load().smrt_nn_adam(_p(w), _p(grad), _p(m), _p(v), w.numel(), float(lr), float(b1), float(b2),
                                    float(eps), int(step), float(grad_scale), _p(found_inf), _s()))


def smrt_nn_resize_bilinear(x, y):
    n, h, w, c = x.shape
    _, h2, w2, _ = y.shape
    _check(_lib.load().smrt_nn_resize_bilinear(_p(x), n, h, w, c, _p(y), h2, w2, _s()))
