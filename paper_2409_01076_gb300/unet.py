"""U-Net of the learned warm start, trained and run on the GPU by libsmrt's NN kernels.

The network maps three input channels -- the normalised Reynolds number and the
two node coordinates -- to three output channels (u / U, v / U, (rho - 1) / (3 U^2))
of a steady lid-driven cavity.  Every arithmetic step runs in the kernels of
include/smrt_nn.h; PyTorch only allocates the tensors and supplies the stream.

Architecture (4 levels, `base` channels at the top; 32 in use):
    enc1: conv3(3 -> b), conv3(b -> b)                  (H)
    enc2: pool, conv3(b -> 2b), conv3(2b -> 2b)         (H/2)
    enc3: pool, conv3(2b -> 4b), conv3(4b -> 4b)        (H/4)
    mid : pool, conv3(4b -> 8b), conv3(8b -> 8b)        (H/8)
    dec3: up, [. | enc3], conv3(12b -> 4b), conv3(4b -> 4b)
    dec2: up, [. | enc2], conv3(6b -> 2b), conv3(2b -> 2b)
    dec1: up, [. | enc1], conv3(3b -> b), conv3(b -> b)
    head: conv1(b -> 3), linear
3x3 convolutions pad with zeros; activations are SiLU; pooling is 2x2 average;
upsampling is nearest.  A 3x3 weight is stored (cout, 9 cin) with column
(ky * 3 + kx) * cin + c.  Matrix products take half operands with float32
accumulation; master weights, gradients and optimiser state are float32.
"""
from __future__ import annotations

import math

import numpy as np

from . import nn as K

LAYERS = [  # name, cin multiple of b (or the input), cout multiple of b, kernel, activation
    ("enc1a", "in", 1, 3, True), ("enc1b", 1, 1, 3, True),
    ("enc2a", 1, 2, 3, True), ("enc2b", 2, 2, 3, True),
    ("enc3a", 2, 4, 3, True), ("enc3b", 4, 4, 3, True),
    ("mida", 4, 8, 3, True), ("midb", 8, 8, 3, True),
    ("dec3a", 12, 4, 3, True), ("dec3b", 4, 4, 3, True),
    ("dec2a", 6, 2, 3, True), ("dec2b", 2, 2, 3, True),
    ("dec1a", 3, 1, 3, True), ("dec1b", 1, 1, 3, True),
    ("head", 1, "out", 1, False),
]

RE_LO, RE_HI = 100.0, 10000.0


def re_feature(re: float) -> float:
    """log(Re) mapped linearly so that Re = 100 -> 0 and Re = 10^4 -> 1."""
    return (math.log(re) - math.log(RE_LO)) / (math.log(RE_HI) - math.log(RE_LO))


def _pad8(n: int) -> int:
    return (n + 7) // 8 * 8


class _DzPre:
    """dL/dz of a convolution, already through its SiLU backward (and its bias gradient accumulated) by
    the fused epilogue of the next convolution's input gradient: blocked halves, and float32 if needed."""

    def __init__(self, dzf, dzb):
        self.dzf, self.dzb = dzf, dzb


class _DaSum:
    """An activation gradient given as its skip part (full resolution) plus its pooled part (half
    resolution, to go through the 2x2 average-pooling adjoint): summed inside the SiLU backward."""

    def __init__(self, skip, pooled):
        self.skip, self.pooled = skip, pooled


class _Act:
    """An activation (N, H, W, C): its float32 NHWC tensor `f` and/or its blocked half copy `b`
    ([N][C/8][H][W][8], the operand layout of the TMA convolutions); either may be None."""
    __slots__ = ("f", "b", "shape")

    def __init__(self, f, b, shape):
        self.f, self.b, self.shape = f, b, tuple(shape)


class UNet:
    def __init__(self, base: int = 32, cin: int = 3, cout: int = 3, seed: int = 0, device: str = "cuda",
                 gemm: str = "tcgen05", conv: str = "tma"):
        import torch
        self.torch = torch
        self.base, self.cin, self.cout, self.device = base, cin, cout, device
        self.specs = []
        for name, ci, co, k, act in LAYERS:
            ci = cin if ci == "in" else ci * base
            co = cout if co == "out" else co * base
            self.specs.append((name, ci, co, k, act))
        rng = np.random.Generator(np.random.PCG64(seed))
        init = []
        for name, ci, co, k, _ in self.specs:
            fan_in = ci * k * k
            w = rng.normal(0.0, math.sqrt(2.0 / fan_in), size=(co, k * k * ci))
            b = rng.normal(0.0, 0.01, size=(co,))
            init += [(name + ".w", w), (name + ".b", b)]
        # parameters, gradients and Adam moments each live in one flat buffer (one Adam launch, one
        # gradient fill); the per-layer tensors are views into them, 16-byte aligned
        offs, total = {}, 0
        for key, val in init:
            offs[key] = total
            total += (val.size + 3) // 4 * 4
        self._flat = {nm: torch.zeros(total, dtype=torch.float32, device=device) for nm in ("p", "g", "m", "v")}
        self.params, self.grads, self.m, self.v = {}, {}, {}, {}
        for key, val in init:
            o, n = offs[key], val.size
            self.params[key] = self._flat["p"][o:o + n].view(val.shape)
            self.params[key].copy_(torch.tensor(val, dtype=torch.float32))
            self.grads[key] = self._flat["g"][o:o + n].view(val.shape)
            self.m[key] = self._flat["m"][o:o + n].view(val.shape)
            self.v[key] = self._flat["v"][o:o + n].view(val.shape)
        self._graph = None
        self.step_count = 0
        self.grad_scale = 2.0 ** 16
        self._found_inf = torch.zeros(1, dtype=torch.int32, device=device)
        self._loss = torch.zeros(1, dtype=torch.float64, device=device)
        if gemm not in ("tcgen05", "wmma"):
            raise ValueError("gemm must be 'tcgen05' or 'wmma'")
        self.gemm_backend = gemm
        if conv not in ("tma", "gather"):
            raise ValueError("conv must be 'tma' or 'gather'")
        self.conv_path = conv           # tcgen05 3x3 convolutions: TMA halo tiles, or thread-gathered A tiles
        # the input gradient of a convolution that reads another's activation computes that one's SiLU
        # backward and bias gradient in its epilogue (smrt_nn_conv3_tma_act_bwd)
        self.fuse_act_bwd = True
        self._gemm_err = torch.zeros(1, dtype=torch.int32, device=device)   # tensor-core wait timeouts

    def _gemm(self, transA, transB, M, N, Kd, alpha, A, lda, B, ldb, beta, C, ldc, split=1):
        if self.gemm_backend == "tcgen05":
            K.smrt_nn_gemm_tc(transA, transB, M, N, Kd, alpha, A, lda, B, ldb, beta, C, ldc, split, self._gemm_err)
        else:
            K.smrt_nn_gemm(transA, transB, M, N, Kd, alpha, A, lda, B, ldb, beta, C, ldc, split)

    def gemm_timeouts(self) -> int:
        """Tensor-core wait timeouts recorded since the last check (0 unless the hardware stalled)."""
        return int(self._gemm_err.item())

    def check_timeouts(self) -> None:
        """Raises SmrtError(SMRT_ERR_TIMEOUT) if a tensor-core kernel gave up a bounded wait since the
        last check (its blocks skipped their outputs); waits for the current stream."""
        K.smrt_nn_check(self._gemm_err)

    # ---- parameters --------------------------------------------------------------------
    def load_numpy(self, params: dict) -> None:
        for key, val in params.items():
            self.params[key].copy_(self.torch.tensor(val, dtype=self.torch.float32))

    def to_numpy(self) -> dict:
        return {k: v.detach().cpu().numpy().astype(np.float64) for k, v in self.params.items()}

    def n_params(self) -> int:
        return sum(p.numel() for p in self.params.values())

    # ---- one convolution (3x3 via im2col, or 1x1) ----------------------------------------
    def _all_tma(self):
        """Every 3x3 convolution reads packed TMA operands, forward and (but for the input layer) adjoint."""
        return all((self._tma(3, ci) or self._tma_padded(sp)) and (name == "enc1a" or self._tma(3, co))
                   for sp in self.specs for name, ci, co, k, _ in [sp] if k == 3)

    def _half_weights(self):
        if self._all_tma():
            return self._packed_weights()
        t = self.torch
        self._wh, self._wf, self._wp, self._wfp = {}, {}, {}, {}
        for spec in self.specs:
            name, ci, co, k, _ = spec
            w = self.params[name + ".w"]
            h = t.empty(w.shape, dtype=t.float16, device=self.device)
            K.smrt_nn_to_half(w, h)
            self._wh[name] = h
            if self._tma(k, ci):                # packed for the TMA convolution
                self._wp[name] = t.empty(K.smrt_nn_pack3_halves(co, ci), dtype=t.float16, device=self.device)
                K.smrt_nn_pack3(h, ci, self._wp[name])
            elif self._tma_padded(spec):        # the input layer, zero-padded to 16 channels
                hp = t.empty((co, 9 * 16), dtype=t.float16, device=self.device)
                K.smrt_nn_pad3(w, ci, 16, hp)
                self._wp[name] = t.empty(K.smrt_nn_pack3_halves(co, 16), dtype=t.float16, device=self.device)
                K.smrt_nn_pack3(hp, 16, self._wp[name])
            if k == 3 and name != "enc1a":      # weights of the adjoint convolution (input gradient)
                f = t.empty((ci, 9 * co), dtype=t.float16, device=self.device)
                K.smrt_nn_flip3(w, f)
                self._wf[name] = f
                if self._tma(k, co):
                    self._wfp[name] = t.empty(K.smrt_nn_pack3_halves(ci, co), dtype=t.float16, device=self.device)
                    K.smrt_nn_pack3(f, co, self._wfp[name])

    def _packed_weights(self):
        """The TMA path reads only packed halves: every layer's forward and adjoint operand in one launch
        (smrt_nn_pack3_many) into buffers allocated once; the 1x1 head reads its float32 weights."""
        t = self.torch
        if getattr(self, "_pack_descs", None) is None:
            self._wh, self._wf, self._wp, self._wfp = {}, {}, {}, {}
            descs = []
            for spec in self.specs:
                name, ci, co, k, _ = spec
                if k != 3:
                    continue
                w = self.params[name + ".w"]
                cpad = 16 if self._tma_padded(spec) else ci
                self._wp[name] = t.empty(K.smrt_nn_pack3_halves(co, cpad), dtype=t.float16, device=self.device)
                descs.append((w, self._wp[name], K.SMRT_NN_PACK_FORWARD, co, ci, cpad))
                if name != "enc1a" and self._tma(k, co):
                    self._wfp[name] = t.empty(K.smrt_nn_pack3_halves(ci, co), dtype=t.float16, device=self.device)
                    descs.append((w, self._wfp[name], K.SMRT_NN_PACK_ADJOINT, co, ci, ci))
            self._pack_descs = descs
        K.smrt_nn_pack3_many(self._pack_descs)

    def _conv(self, spec, inp, cache, out_f=True, out_b=False):
        """One convolution + bias + activation.  inp: _Act; returns an _Act with the float32 output
        (out_f) and/or its blocked half copy (out_b, for a TMA convolution that reads it next)."""
        t = self.torch
        name, ci, co, k, act = spec
        n, h, w, _ = inp.shape
        rows = n * h * w
        kk = k * k * ci
        y = t.empty((n, h, w, co), dtype=t.float32, device=self.device)
        xb = col = None
        if self._tma_padded(spec):
            # the 3-channel input as a 16-channel TMA convolution whose extra channels (and weights) are zero
            xb = t.empty(rows * 16, dtype=t.float16, device=self.device)
            K.smrt_nn_to_half_blocked_pad(inp.f, 16, xb)
            inp = _Act(inp.f, xb, (n, h, w, 16))
        if self._small_1x1(spec):
            # the head: a few float32 dot products per pixel, bias included
            K.smrt_nn_conv1x1_small(inp.f, self.params[name + ".w"], self.params[name + ".b"], y)
            if cache is not None:
                cache[name] = (None, None, inp.f, None, inp.shape)
            return _Act(y, None, (n, h, w, co))
        if self._tma(k, ci) or self._tma_padded(spec):
            # operands by TMA: blocked half activations, nine taps as shifted views of one haloed tile
            xb = inp.b
            if xb is None:
                xb = t.empty(rows * ci, dtype=t.float16, device=self.device)
                K.smrt_nn_to_half_blocked(inp.f, xb)
            if co % 8 == 0:
                # bias and SiLU in the convolution's epilogue: writes z, a and / or the blocked halves
                want_b = out_b and self._blocked_ok(co)
                z = t.empty_like(y) if (act and cache is not None) else None
                a = y if (out_f or not want_b) else None
                ab = t.empty(rows * co, dtype=t.float16, device=self.device) if want_b else None
                K.smrt_nn_conv3_tma_bias_act(xb, inp.shape, self._wp[name], co, self.params[name + ".b"], act, z, a,
                                             ab, self._gemm_err)
                if cache is not None:
                    cache[name] = (None, z, inp.f, xb, inp.shape)
                return _Act(a, ab, (n, h, w, co))
            K.smrt_nn_conv3_tma(xb, inp.shape, self._wp[name], y, co, 1.0, 0.0, self._gemm_err)
        elif self._implicit(k, ci):
            # implicit GEMM: the A tiles are gathered from x, no im2col matrix is built
            K.smrt_nn_conv3_tc(inp.f, self._wh[name], y, 1.0, 0.0, self._gemm_err)
        else:
            ldk = _pad8(kk)             # whole 16-byte rows for the GEMM's vector loads
            col = t.empty((rows, ldk), dtype=t.float16, device=self.device)
            if k == 3:
                K.smrt_nn_im2col3(inp.f, col)
            else:
                K.smrt_nn_to_half_rows(inp.f.view(rows, ci), col)
            self._gemm(0, 1, rows, co, kk, 1.0, col, ldk, self._wh[name], kk, 0.0, y, co)
        z = t.empty_like(y) if (act and cache is not None) else None
        ab = None
        if out_b and self._blocked_ok(co):
            ab = t.empty(rows * co, dtype=t.float16, device=self.device)
            K.smrt_nn_bias_act_blocked(y, self.params[name + ".b"], act, z, y if out_f else None, ab)
        else:
            out_f = True
            K.smrt_nn_bias_act(y, self.params[name + ".b"], act, z, y)
        if cache is not None:
            cache[name] = (col, z, inp.f, xb, inp.shape)
        return _Act(y if out_f else None, ab, (n, h, w, co))

    def _implicit(self, k, c):
        """3x3 convolutions over C % 8 == 0 channels run as implicit GEMMs on the tcgen05 backend."""
        return self.gemm_backend == "tcgen05" and k == 3 and c % 8 == 0

    def _tma(self, k, c):
        """... and with TMA-fed operands when C % 16 == 0, unless the gather path was chosen."""
        return self.conv_path == "tma" and self._implicit(k, c) and c % 16 == 0

    @staticmethod
    def _small_1x1(spec):
        """A 1x1 convolution without activation and at most 3 outputs: CUDA-core float32 kernels."""
        _, ci, co, k, act = spec
        return k == 1 and not act and co <= 3 and ci % 4 == 0 and ci <= 64

    def _tma_padded(self, spec):
        """The network's input layer (fewer than 16 channels) on the TMA path, zero-padded to 16."""
        name, ci, co, k, _ = spec
        return (name == "enc1a" and k == 3 and ci < 16 and co % 8 == 0 and self.conv_path == "tma"
                and self.gemm_backend == "tcgen05")

    def _blocked_ok(self, c):
        """Whether a c-channel activation may be handed over as blocked halves only."""
        return self.conv_path == "tma" and self.gemm_backend == "tcgen05" and c % 8 == 0

    def _reads_blocked(self, spec):
        """A convolution whose forward and weight gradient read only the blocked half input."""
        _, ci, co, k, _ = spec
        return self._tma(k, ci) and co % 8 == 0

    def _fusable(self, spec_b, spec_a, cache):
        """B's input gradient can carry A's SiLU backward in its epilogue (A's activation is B's input)."""
        _, ci_b, co_b, k_b, _ = spec_b
        name_a, _, co_a, k_a, act_a = spec_a
        _, z_a, _, xb_a, _ = cache[name_a]
        return (self.conv_path == "tma" and self.fuse_act_bwd and k_b == 3 and self._tma(3, co_b)
                and co_a == ci_b and co_a % 8 == 0 and (z_a is not None or not act_a) and k_a == 3
                and not self._small_1x1(spec_a))

    def _conv_bwd(self, spec, da, cache, need_dx=True, then=None):
        """Gradients of one convolution from dL/d(activation) `da` (a float32 tensor, or the _DzPre that the
        consumer's fused input gradient produced).  Returns dL/d(input), or -- when `then` names the
        convolution A whose activation is this one's input and the fusion applies -- A's _DzPre."""
        t = self.torch
        name, ci, co, k, act = spec
        col, z, xf, xb, xshape = cache[name]
        n, h, w, _ = xshape
        rows = n * h * w
        if self._small_1x1(spec):
            dx = t.empty(xshape, dtype=t.float32, device=self.device) if need_dx else None
            K.smrt_nn_conv1x1_small_bwd(da, xf, self.params[name + ".w"], dx, self.grads[name + ".w"],
                                        self.grads[name + ".b"])
            return dx
        kk = k * k * ci
        ldz = _pad8(co)
        gw = self.grads[name + ".w"]
        tma_w = xb is not None and co % 8 == 0              # weight gradient from blocked halves
        tma_dx = need_dx and k == 3 and self._tma(k, co)    # input gradient by the TMA convolution
        if isinstance(da, _DzPre):          # dz and the bias gradient came out of the consumer's epilogue
            dzf, dzb = da.dzf, da.dzb
        elif isinstance(da, _DaSum) and (tma_w or tma_dx) and co % 8 == 0:
            dzf = t.empty_like(da.skip) if (not tma_w or (need_dx and not tma_dx)) else None
            dzb = t.empty(rows * co, dtype=t.float16, device=self.device)
            K.smrt_nn_bias_act_bwd_addpool_blocked(da.skip, da.pooled, z, act, dzf, self.grads[name + ".b"], dzb)
        else:
            if isinstance(da, _DaSum):
                pooled = t.empty_like(da.skip)
                K.smrt_nn_avgpool2_bwd(da.pooled, tuple(da.skip.shape), pooled)
                K.smrt_nn_add(da.skip, pooled, da.skip)
                da = da.skip
            dzf = t.empty_like(da) if (not tma_w or (need_dx and not tma_dx)) else None
            dzb = None
            if tma_w or tma_dx:
                dzb = t.empty(rows * co, dtype=t.float16, device=self.device)
                K.smrt_nn_bias_act_bwd_blocked(da, z, act, dzf, self.grads[name + ".b"], dzb)
            else:
                K.smrt_nn_bias_act_bwd(da, z, act, dzf, self.grads[name + ".b"])
        dzh = None
        if tma_w and xshape[3] != ci:
            # zero-padded input layer: the padded gradient, folded back onto the real channels
            gp = t.zeros((co, 9 * xshape[3]), dtype=t.float32, device=self.device)
            K.smrt_nn_conv3_wgrad_tma(xb, xshape, dzb, co, gp, 1.0, self._gemm_err)
            K.smrt_nn_unpad3_add(gp, ci, xshape[3], gw)
        elif tma_w:
            K.smrt_nn_conv3_wgrad_tma(xb, xshape, dzb, co, gw, 1.0, self._gemm_err)
        else:
            if col is None:         # the forward gathered from x; the weight gradient needs the matrix
                col = t.empty((rows, _pad8(kk)), dtype=t.float16, device=self.device)
                K.smrt_nn_im2col3(xf, col)
            ldk = col.shape[1]
            dzh = t.empty((rows, ldz), dtype=t.float16, device=self.device)
            K.smrt_nn_to_half_rows(dzf.view(rows, co), dzh)
            # many split-K blocks: K is the pixel count, M and N are small
            split = max(1, min(1024, rows // 1024))
            if self.gemm_backend == "tcgen05":
                # dW^T = col^T dz: the 9 cin dimension on the tensor core's M = 128 side, stored transposed
                K.smrt_nn_gemm_tc(1, 2, kk, co, rows, 1.0, col, ldk, dzh, ldz, 1.0, gw, kk, split, self._gemm_err)
            else:
                self._gemm(1, 0, co, kk, rows, 1.0, dzh, ldz, col, ldk, 1.0, gw, kk, split)
        if not need_dx:
            return None
        if tma_dx and then is not None and self._fusable(spec, then, cache):
            name_a, _, co_a, _, act_a = then
            _, z_a, _, _, _ = cache[name_a]
            # A needs float32 dz too unless both its gradients are TMA kernels reading the blocked halves
            tma_a = cache[name_a][3] is not None and self._tma(3, co_a)
            dzf_a = t.empty(xshape, dtype=t.float32, device=self.device) if not tma_a else None
            dzb_a = t.empty(rows * co_a, dtype=t.float16, device=self.device)
            K.smrt_nn_conv3_tma_act_bwd(dzb, (n, h, w, co), self._wfp[name], co_a, z_a, act_a, dzf_a,
                                        self.grads[name_a + ".b"], dzb_a, self._gemm_err)
            return _DzPre(dzf_a, dzb_a)
        dx = t.empty(xshape, dtype=t.float32, device=self.device)
        if k == 1:
            self._gemm(0, 0, rows, ci, co, 1.0, dzh, ldz, self._wh[name], ci, 0.0, dx, ci)
            return dx
        # dx = conv3(dz, flip(W)): the adjoint 3x3 convolution, no col2im
        if tma_dx:
            K.smrt_nn_conv3_tma(dzb, (n, h, w, co), self._wfp[name], dx, ci, 1.0, 0.0, self._gemm_err)
            return dx
        if self._implicit(k, co):
            K.smrt_nn_conv3_tc(dzf.view(n, h, w, co), self._wf[name], dx, 1.0, 0.0, self._gemm_err)
            return dx
        dzcol = t.empty((rows, 9 * co), dtype=t.float16, device=self.device)
        K.smrt_nn_im2col3(dzf.view(n, h, w, co), dzcol)
        self._gemm(0, 1, rows, ci, 9 * co, 1.0, dzcol, 9 * co, self._wf[name], 9 * co, 0.0, dx, ci)
        return dx

    # ---- the network ------------------------------------------------------------------
    def _pool(self, x, blocked):
        """2x2 average pooling of x (_Act with float32); blocked: hand over the blocked halves only."""
        t = self.torch
        n, h, w, c = x.shape
        shape = (n, h // 2, w // 2, c)
        if blocked and self._blocked_ok(c):
            yb = t.empty(n * (h // 2) * (w // 2) * c, dtype=t.float16, device=self.device)
            K.smrt_nn_avgpool2_blocked(x.f, None, yb)
            return _Act(None, yb, shape)
        y = t.empty(shape, dtype=t.float32, device=self.device)
        if c % 8 == 0:
            K.smrt_nn_avgpool2_blocked(x.f, y, None)        # the vectorised kernel, float32 output only
        else:
            K.smrt_nn_avgpool2(x.f, y)
        return _Act(y, None, shape)

    def _upcat(self, a, b, blocked):
        """The decoder input [up2(a) | b] (a, b: _Act with float32)."""
        t = self.torch
        n, h, w, ca = a.shape
        cb = b.shape[3]
        shape = (n, 2 * h, 2 * w, ca + cb)
        if ca % 8 == 0 and cb % 8 == 0:
            yb = None
            if blocked and self._blocked_ok(ca + cb):
                yb = t.empty(n * 4 * h * w * (ca + cb), dtype=t.float16, device=self.device)
                K.smrt_nn_upcat(a.f, b.f, None, yb)
                return _Act(None, yb, shape)
            y = t.empty(shape, dtype=t.float32, device=self.device)
            K.smrt_nn_upcat(a.f, b.f, y, None)
            return _Act(y, None, shape)
        u = t.empty((n, 2 * h, 2 * w, ca), dtype=t.float32, device=self.device)
        K.smrt_nn_upsample2(a.f, u)
        y = t.empty(shape, dtype=t.float32, device=self.device)
        K.smrt_nn_concat(u, b.f, y)
        return _Act(y, None, shape)

    def forward(self, x, cache=None):
        """x: (N, H, W, cin) float32 CUDA, H and W divisible by 8.  Returns (N, H, W, cout).
        Where the next convolution reads TMA tiles, an activation is handed over as blocked halves
        only (no float32 copy is written)."""
        s = {sp[0]: sp for sp in self.specs}
        self._half_weights()
        rb = lambda name: self._reads_blocked(s[name])  # noqa: E731

        def c(name, inp, nxt=None):     # nxt: the convolution that reads the output, if only one does
            b = nxt is not None and rb(nxt)
            return self._conv(s[name], inp, cache, out_f=not b, out_b=b)

        e1 = c("enc1b", c("enc1a", _Act(x, None, tuple(x.shape)), "enc1b"))
        e2 = c("enc2b", c("enc2a", self._pool(e1, rb("enc2a")), "enc2b"))
        e3 = c("enc3b", c("enc3a", self._pool(e2, rb("enc3a")), "enc3b"))
        m = c("midb", c("mida", self._pool(e3, rb("mida")), "midb"))
        d3 = c("dec3b", c("dec3a", self._upcat(m, e3, rb("dec3a")), "dec3b"))
        d2 = c("dec2b", c("dec2a", self._upcat(d3, e2, rb("dec2a")), "dec2b"))
        d1 = c("dec1b", c("dec1a", self._upcat(d2, e1, rb("dec1a")), "dec1b"))
        return c("head", d1).f

    def backward(self, dy, cache):
        """Accumulates scaled gradients of the loss into self.grads from dL/dy (already scaled)."""
        t = self.torch
        s = {sp[0]: sp for sp in self.specs}
        b = self.base
        cb = lambda name, da, need=True: self._conv_bwd(s[name], da, cache, need)  # noqa: E731

        def upcat_bwd(dcat, ca):
            """Gradients of the low-resolution input and of the skip from that of [up2(a) | skip]."""
            n, h2, w2, cc = dcat.shape
            da = t.empty((n, h2 // 2, w2 // 2, ca), dtype=t.float32, device=self.device)
            db = t.empty((n, h2, w2, cc - ca), dtype=t.float32, device=self.device)
            if ca % 4 == 0 and (cc - ca) % 4 == 0:
                K.smrt_nn_upcat_bwd(dcat, ca, da, db)
                return da, db
            du = t.empty((n, h2, w2, ca), dtype=t.float32, device=self.device)
            K.smrt_nn_concat_bwd(dcat, ca, cc - ca, du, db)
            K.smrt_nn_upsample2_bwd(du, (n, h2 // 2, w2 // 2, ca), da)
            return da, db

        def pool_bwd(dyy):
            n, h, w, cc = dyy.shape
            dx = t.empty((n, 2 * h, 2 * w, cc), dtype=t.float32, device=self.device)
            K.smrt_nn_avgpool2_bwd(dyy, (n, 2 * h, 2 * w, cc), dx)
            return dx

        def add_into(acc, other):        # acc += other (skip path + pooled path)
            K.smrt_nn_add(acc, other, acc)
            return acc

        def pair(a, bname, da, need=True):
            """A then B (B reads A's activation): B's input gradient carries A's SiLU backward."""
            return self._conv_bwd(s[a], self._conv_bwd(s[bname], da, cache, True, then=s[a]), cache, need)

        dd1 = cb("head", dy)
        du2, de1 = upcat_bwd(pair("dec1a", "dec1b", dd1), 2 * b)
        du3, de2 = upcat_bwd(pair("dec2a", "dec2b", du2), 4 * b)
        dum, de3 = upcat_bwd(pair("dec3a", "dec3b", du3), 8 * b)
        if self.fuse_act_bwd:
            # each encoder level's activation gradient = its skip part + the pooled level's input
            # gradient through the pooling adjoint, summed inside the SiLU backward
            de3 = _DaSum(de3, pair("mida", "midb", dum))
            de2 = _DaSum(de2, pair("enc3a", "enc3b", de3))
            de1 = _DaSum(de1, pair("enc2a", "enc2b", de2))
        else:
            de3 = add_into(de3, pool_bwd(pair("mida", "midb", dum)))
            de2 = add_into(de2, pool_bwd(pair("enc3a", "enc3b", de3)))
            de1 = add_into(de1, pool_bwd(pair("enc2a", "enc2b", de2)))
        pair("enc1a", "enc1b", de1, need=False)

    def loss_and_grad(self, x, target):
        """MSE loss (float) with scaled gradients accumulated into self.grads (zeroed first)."""
        self._flat["g"].zero_()
        cache = {}
        y = self.forward(x, cache)
        self._loss.zero_()
        dy = self.torch.empty_like(y)
        K.smrt_nn_mse(y, target, self.grad_scale, self._loss, dy)
        self.backward(dy, cache)
        return y

    def adam_step(self, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8) -> bool:
        """Applies the accumulated gradients; returns False (and lowers the loss scale) on overflow.
        Raises SmrtError(SMRT_ERR_TIMEOUT), before touching the parameters, if a tensor-core wait of
        the forward or backward pass gave up."""
        self.check_timeouts()
        self.step_count += 1
        self._found_inf.zero_()
        f = self._flat      # the padding between views holds zeros in all four buffers and stays zero
        K.smrt_nn_adam(f["p"], f["g"], f["m"], f["v"], lr, b1, b2, eps, self.step_count, self.grad_scale,
                       self._found_inf)
        if int(self._found_inf.item()):
            self.grad_scale /= 2.0
            self._graph = None              # the recorded loss gradient carries the old scale
            return False
        return True

    def capture(self, x, target):
        """Records loss_and_grad on the static tensors x and target as one CUDA graph, after an eager
        warm-up on a side stream; replay() re-runs it on their current contents.  The loss scale is
        part of the recording, so adam_step drops the graph when it lowers the scale."""
        t = self.torch
        side = t.cuda.Stream()
        side.wait_stream(t.cuda.current_stream())
        with t.cuda.stream(side):
            self.loss_and_grad(x, target)
        t.cuda.current_stream().wait_stream(side)
        g = t.cuda.CUDAGraph()
        with t.cuda.graph(g):
            self._graph_y = self.loss_and_grad(x, target)
        self._graph = g
        self._graph_in = (x, target)

    def replay(self):
        """loss_and_grad on the tensors given to capture() (their current contents)."""
        if self._graph is None:
            raise RuntimeError("no recorded training step: call capture() first")
        self._graph.replay()
        return self._graph_y

    def train_step(self, x, target, lr: float) -> float:
        self.loss_and_grad(x, target)
        self.adam_step(lr)
        return float(self._loss.item())

    def predict(self, x):
        y = self.forward(x, None)
        self.check_timeouts()
        return y


def input_grid(res, h: int, w: int, device: str = "cuda"):
    """Network input (len(res), h, w, 3): [re_feature, x, y] with node-centred x = (i + 1/2) / w."""
    import torch
    n = len(res)
    x = torch.empty((n, h, w, 3), dtype=torch.float32, device=device)
    xs = (torch.arange(w, dtype=torch.float32, device=device) + 0.5) / w
    ys = (torch.arange(h, dtype=torch.float32, device=device) + 0.5) / h
    x[..., 1] = xs.view(1, 1, w)
    x[..., 2] = ys.view(1, h, 1)
    for k, re in enumerate(res):
        x[k, ..., 0] = re_feature(re)
    return x
