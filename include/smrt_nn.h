/*
 * smrt_nn.h -- C ABI of the small neural-network kernel set used by the learned
 * warm start: a U-Net that predicts a steady cavity field (u, v, rho) from the
 * Reynolds number and the node coordinates, after which the SmrtLBM update of
 * smrt.h iterates to the steady-state tolerance.  The paper has no network;
 * this is the library's own addition, built on the same CUDA library.
 *
 * Conventions
 * - Every pointer is DEVICE memory of the current device; every call enqueues
 *   work on `stream` (a cudaStream_t, NULL = legacy default stream) and returns
 *   SMRT_OK or SMRT_ERR_ARG / SMRT_ERR_CUDA (message in smrt_last_error(NULL)).
 *   Nothing is allocated and nothing is freed.
 * - Activations are float32 NHWC: x[n][y][x][c], row-major, dense.
 * - Matrix operands of smrt_nn_gemm are IEEE half; accumulation is float32.
 */
#ifndef SMRT_NN_H
#define SMRT_NN_H

#include "smrt.h"

#ifdef __cplusplus
extern "C" {
#endif

/* C = alpha * op(A) * op(B) + beta * C, op(A) M x K, op(B) K x N, C M x N float32
 * row-major with leading dimension ldc.  A (half, leading dimension lda) holds
 * op(A) row-major when transA == 0 and op(A)^T (K x M) row-major when transA == 1;
 * B (half, ldb) holds op(B) (K x N) when transB == 0 and op(B)^T (N x K) when 1.
 * split_k > 1 splits the K range over split_k blocks that ATOMICALLY ADD their
 * partial products into C (C must hold the beta * C part already; beta is then
 * ignored).  Tensor-core (WMMA 16x16x16) tiles of 64 x 64 x 32. */
SMRT_API int smrt_nn_gemm(int transA, int transB, int M, int N, int K, float alpha, const void *A, int lda,
                          const void *B, int ldb, float beta, float *C, int ldc, int split_k, void *stream);

/* The same product as smrt_nn_gemm (same arguments and split-K semantics, K >= 1) on the
 * 5th-generation tensor cores.  transB bit 0 is op(B)'s transpose flag as in smrt_nn_gemm;
 * bit 1 set stores C^T instead of C (C is then N x M row-major with leading dimension ldc,
 * and beta / the split-K sums apply to that layout).  Each 128-thread block computes a
 * 128 x TN output tile (TN = 32, 64 or 128, the smallest that covers N), K in steps of 64
 * through two shared-memory stages (no-swizzle K-major core-matrix layout) so that the copy
 * of step k+1 overlaps the tcgen05.mma (half x half -> float32, accumulator in tensor memory)
 * of step k; tcgen05.ld epilogue.  Every wait on the tensor core is bounded: on a timeout the
 * block sets *err = 1 (err: device int, may be NULL), skips its epilogue and still releases
 * its tensor memory.  M == 0 or N == 0 does nothing; SMRT_ERR_ARG for negative M or N, K < 1,
 * split_k < 1, a NULL operand or a leading dimension smaller than its row. */
SMRT_API int smrt_nn_gemm_tc(int transA, int transB, int M, int N, int K, float alpha, const void *A, int lda,
                             const void *B, int ldb, float beta, float *C, int ldc, int split_k, int *err,
                             void *stream);

/* 3x3, stride 1, zero padding 1 convolution as an implicit GEMM on the tensor cores:
 *   y[p][o] = alpha * sum_{tap, c} half(x[n][yy+ky-1][xx+kx-1][c]) * w[o][tap*C + c] + beta * y[p][o]
 * for pixel p = (n*H + yy)*W + xx, tap = ky*3 + kx, outside the image x = 0.  x is NHWC float32
 * (C % 8 == 0, 16-byte aligned), w is cout x 9C half (row-major, the layout of smrt_nn_im2col3's
 * columns), y is N*H*W rows of ldy >= cout float32.  The result is bit-identical to smrt_nn_im2col3
 * followed by smrt_nn_gemm_tc(0, 1, ...): the kernel is that GEMM, with each A tile gathered from x
 * (rounded to half as im2col rounds) instead of read from an im2col matrix, which is never built.
 * err as in smrt_nn_gemm_tc.  SMRT_ERR_ARG for C % 8 != 0, a misaligned x or bad sizes. */
SMRT_API int smrt_nn_conv3_tc(const float *x, int N, int H, int W, int C, const void *w, int cout, float alpha,
                              float beta, float *y, int ldy, int *err, void *stream);

/* ---- TMA-fed 3x3 convolutions ---------------------------------------------------------------
 * These read HALF activations in the channel-group-blocked layout xb[n][c/8][y][x][c%8]
 * ([N][C/8][H][W][8], dense, 16-byte aligned), which smrt_nn_to_half_blocked writes: one image row of
 * one 8-channel group is then W*16 contiguous bytes, so one TMA box brings a whole zero-padded
 * 18 x 10 pixel window as 18 runs of 160 bytes.  Each 128-thread block works on a 16-row x 8-pixel
 * output tile; the nine taps of the filter are nine shifted shared-memory views of that one window
 * (no im2col tile).  A TMA producer lane and a tcgen05.mma issuer lane run an mbarrier pipeline;
 * the float32 accumulator lives in tensor memory.  err as in smrt_nn_gemm_tc: every wait is
 * bounded (here by one second of the GPU's global timer).  SMRT_ERR_ARG for unsupported channel
 * counts, misaligned pointers or sizes the grid cannot cover; SMRT_ERR_CUDA if the driver rejects a
 * tensor map. */

/* xb = half(scale * x) in the blocked layout above; x is NHWC float32 (16-byte aligned), C % 8 == 0. */
SMRT_API int smrt_nn_to_half_blocked(const float *x, int N, int H, int W, int C, float scale, void *xb,
                                     void *stream);

/* Zero-padded forms for a layer with few input channels (C < 16, e.g. the network's 3-channel input),
 * so that it can run as a Cp- (or Cb-) channel TMA convolution whose extra channels are zero:
 * smrt_nn_to_half_blocked_pad: xb (Cb channels, blocked) = half(scale * x) for c < C, 0 above; x is NHWC
 *   float32 with C channels (any C >= 1), Cb >= C, Cb % 8 == 0, xb 16-byte aligned.
 * smrt_nn_pad3: wh (cout x 9 Cp half) from 3x3 weights w (cout x 9 C float32, column tap*C + c):
 *   wh[o][tap*Cp + c] = half(w[o][tap*C + c]) for c < C, 0 for C <= c < Cp.
 * smrt_nn_unpad3_add: gw[o][tap*C + c] += gp[o][tap*Cp + c] for c < C (the weight gradient of the
 *   padded layer folded back; the padded channels' gradient is exactly zero). */
SMRT_API int smrt_nn_to_half_blocked_pad(const float *x, int N, int H, int W, int C, int Cb, float scale, void *xb,
                                         void *stream);
SMRT_API int smrt_nn_pad3(const float *w, int cout, int C, int Cp, void *wh, void *stream);
SMRT_API int smrt_nn_unpad3_add(const float *gp, int cout, int C, int Cp, float *gw, void *stream);

/* Halves that smrt_nn_pack3 writes for (cout, C): 9 * C * cout rounded up to whole output-channel
 * tiles (32 if cout <= 32, 64 if cout <= 64, else multiples of 128); -1 if C % 16 != 0 or cout < 1. */
SMRT_API long long smrt_nn_pack3_halves(int cout, int C);

/* Packs 3x3 weights w (cout x 9C half, column tap*C + c, the layout of smrt_nn_conv3_tc) for
 * smrt_nn_conv3_tma, with TN the output-channel tile above and nb = o / TN, r = o % TN:
 *   wp[(((nb*(C/16) + c/16)*18 + tap*2 + (c%16)/8)*TN + r)*8 + c%8] = w[o][tap*C + c]
 * (zero for o >= cout), so that the operand of one pipeline stage -- all nine taps of 16 input
 * channels for one output-channel tile -- is one contiguous block, copied by one bulk copy.
 * wp: smrt_nn_pack3_halves(cout, C) halves, 16-byte aligned.  C % 16 == 0. */
SMRT_API int smrt_nn_pack3(const void *w, int cout, int C, void *wp, void *stream);

/* Every packed weight array of a network in one launch, straight from the float32 weights
 * w (cout x 9 cin, column tap*cin + c).  Per descriptor:
 *   kind SMRT_NN_PACK_FORWARD: dst = smrt_nn_pack3 of half(w) zero-padded to cpad >= cin input
 *     channels (cpad % 16 == 0; cpad == cin: no padding), the operand of smrt_nn_conv3_tma
 *     (smrt_nn_pack3_halves(cout, cpad) halves);
 *   kind SMRT_NN_PACK_ADJOINT: dst = smrt_nn_pack3 of smrt_nn_flip3(w), the operand of the input
 *     gradient (cin output channels over cout input channels; cout % 16 == 0;
 *     smrt_nn_pack3_halves(cin, cout) halves).
 * The results equal those of the separate conversion, padding, flip and pack calls bit for bit.
 * count <= SMRT_NN_PACK_MAX; dst 16-byte aligned. */
#define SMRT_NN_PACK_MAX 32
enum { SMRT_NN_PACK_FORWARD = 0, SMRT_NN_PACK_ADJOINT = 1 };
typedef struct {
    const float *w;
    void *dst;
    int kind, cout, cin, cpad;
} smrt_nn_pack3_desc;
SMRT_API int smrt_nn_pack3_many(int count, const smrt_nn_pack3_desc *descs, void *stream);

/* 3x3, stride 1, zero padding 1 convolution:
 *   y[p][o] = alpha * sum_{tap, c} x[n][yy+ky-1][xx+kx-1][c] * w[o][tap*C + c] + beta * y[p][o]
 * for p = (n*H + yy)*W + xx, with x given blocked as xb (C % 16 == 0) and w packed as wp.  y: N*H*W
 * rows of ldy >= cout float32.  Output-channel tiles of 32, 64 or 128; K runs over 16-channel chunks
 * (one TMA of two halo planes and one bulk copy of weights per stage, up to four stages).  The sum
 * runs chunk-major (all nine taps of channels 0-15, then of 16-31, ...), so results equal
 * smrt_nn_conv3_tc's up to float32 rounding, not bit for bit.  The input gradient of a convolution
 * is this call on dz with the weights of smrt_nn_flip3. */
SMRT_API int smrt_nn_conv3_tma(const void *xb, int N, int H, int W, int C, const void *wp, int cout, float alpha,
                               float beta, float *y, int ldy, int *err, void *stream);

/* Reads the error word that the tensor-core kernels above set when a bounded wait gives up:
 * waits for `stream`, reads *err (device int) and returns SMRT_OK if it is 0.  Otherwise it
 * resets *err to 0 and returns SMRT_ERR_TIMEOUT: the blocks that gave up skipped their
 * epilogues (their tensor memory was still released), so every output written since the
 * previous check is suspect.  Synchronises the stream. */
SMRT_API int smrt_nn_check(int *err, void *stream);

/* Test hook for the failure path of smrt_nn_conv3_tma (not for computing anything): the same
 * launch, with alpha = 1 and beta = 0, but the TMA producer of every block issues nothing and
 * each wait gives up after wait_ms milliseconds (1e-3 <= wait_ms <= 1000) instead of one second.
 * Every block therefore times out with no copy and no MMA in flight, sets *err = 1 (err is
 * required), leaves y untouched and releases its tensor memory; smrt_nn_check then returns
 * SMRT_ERR_TIMEOUT and the next ordinary call runs normally.  The paper has no counterpart. */
SMRT_API int smrt_nn_conv3_tma_wait_test(const void *xb, int N, int H, int W, int C, const void *wp, int cout,
                                         float *y, int ldy, int *err, double wait_ms, void *stream);

/* smrt_nn_conv3_tma with the bias and the activation in its epilogue (the float32 convolution output
 * never goes to memory): v = conv + bias[o], z = v, a = SiLU(v) (act) or v, ab = half(a) blocked,
 * each written when its pointer is not NULL (z, a: N*H*W rows of cout float32; ab: the blocked layout
 * with cout channels; at least one output).  cout % 8 == 0; outputs 16-byte aligned.  The values
 * equal smrt_nn_conv3_tma followed by smrt_nn_bias_act_blocked bit for bit. */
SMRT_API int smrt_nn_conv3_tma_bias_act(const void *xb, int N, int H, int W, int C, const void *wp, int cout,
                                        const float *bias, int act, float *z, float *a, void *ab, int *err,
                                        void *stream);

/* The input gradient of a convolution B fused with the SiLU backward of the convolution A whose
 * activation B reads (the chain a = SiLU(z_A), z_B = conv3(a)): with d = conv3(dzb, flipped W_B), the
 * smrt_nn_conv3_tma product of B's blocked half dz (C channels) and its flipped packed weights wp,
 *   dz_A = d * SiLU'(z) (act != 0) or d (act == 0),   SiLU'(z) = s (1 + z (1 - s)), s = 1 / (1 + e^-z),
 * written as blocked halves to dzb_out (cout channels, the layout smrt_nn_bias_act_bwd_blocked
 * writes) and, when dz is not NULL, as float32 NHWC rows of cout; db (cout floats, may be NULL)
 * accumulates the column sums of dz_A (A's bias gradient) -- per tile in shared memory, then one
 * float32 atomic per channel and tile, so its last bits vary from run to run.  z: A's pre-activation,
 * N*H*W rows of cout float32.  dzb_out, dz and db equal smrt_nn_conv3_tma followed by
 * smrt_nn_bias_act_bwd_blocked (dzb_out and dz bit for bit, db up to summation order) without the
 * float32 d ever going to memory.  err as in smrt_nn_conv3_tma.  cout % 8 == 0; z, dz, dzb_out
 * 16-byte aligned. */
SMRT_API int smrt_nn_conv3_tma_act_bwd(const void *dzb, int N, int H, int W, int C, const void *wp, int cout,
                                       const float *z, int act, float *dz, float *db, void *dzb_out, int *err,
                                       void *stream);

/* Weight gradient of the same convolution, ACCUMULATED into gw (cout rows of ldg >= 9C float32):
 *   gw[o][tap*C + c] += alpha * sum_p x[n][yy+ky-1][xx+kx-1][c] * dz[p][o]
 * with x and dz both blocked half (xb: C channels, dzb: cout channels, C % 8 == 0, cout % 8 == 0).
 * Blocks of 128 input x 32 output channels; each block sums a run of pixel tiles for all nine taps
 * in tensor memory (both operands MN-major views of the TMA tiles: K is the pixel index) and adds
 * its result with float32 atomics, so the summation order -- and the last bits -- vary from run to
 * run. */
SMRT_API int smrt_nn_conv3_wgrad_tma(const void *xb, int N, int H, int W, int C, const void *dzb, int cout,
                                     float alpha, float *gw, int ldg, int *err, void *stream);

/* 3x3, stride 1, zero padding 1 patches of x (N,H,W,C float32) into col (N*H*W rows of
 * ld >= 9*C halves, row-major): col[p*ld + (ky*3+kx)*C + c] = x[n][y+ky-1][x+kx-1][c].
 * Columns 9*C .. ld-1 are set to zero (a padded ld lets a GEMM read whole 16-byte rows). */
SMRT_API int smrt_nn_im2col3(const float *x, int N, int H, int W, int C, void *col, int ld, void *stream);

/* Adjoint of smrt_nn_im2col3: dx[n][y][x][c] = sum over the 9 patches that read it of dcol (float32). */
SMRT_API int smrt_nn_col2im3(const float *dcol, int N, int H, int W, int C, float *dx, void *stream);

/* The weights of the adjoint 3x3 convolution: for w (cout, 9 cin) float32 with column
 * (ky*3+kx)*cin + c, writes wf (cin, 9 cout) half with wf[c][tap*cout + o] = w[o][(8 - tap)*cin + c].
 * Then dx = im2col3(dz) * wf^T is the input gradient of the convolution (no col2im needed). */
SMRT_API int smrt_nn_flip3(const float *w, int cout, int cin, void *wf, void *stream);

/* dst[i] = (half)(scale * src[i]), n elements. */
SMRT_API int smrt_nn_to_half(const float *src, long long n, float scale, void *dst, void *stream);

/* Row-padded conversion: src is rows x cols float32 (dense), dst rows x ld halves with
 * dst[r*ld + c] = (half)(scale * src[r*cols + c]) for c < cols and 0 for cols <= c < ld. */
SMRT_API int smrt_nn_to_half_rows(const float *src, long long rows, int cols, float scale, void *dst, int ld,
                                  void *stream);

/* z = x + bias[c] (x, z: rows x C), then a = SiLU(z) = z / (1 + exp(-z)) if act, else a = z.
 * z may be NULL (not kept); a may alias x. */
SMRT_API int smrt_nn_bias_act(const float *x, const float *bias, long long rows, int C, int act, float *z, float *a,
                              void *stream);

/* Backward of smrt_nn_bias_act: dz = da * SiLU'(z) (or da), db[c] += sum over rows of dz.
 * dz may alias da; db is accumulated into (zero it first). */
SMRT_API int smrt_nn_bias_act_bwd(const float *da, const float *z, long long rows, int C, int act, float *dz,
                                  float *db, void *stream);

/* Fused forms for the TMA convolutions (blocked half layout [N][C/8][H][W][8] as above); each
 * float32 / half output pointer may be NULL to skip that output.  C % 8 == 0 where blocked output is
 * written; all pointers 16-byte aligned; fewer than 2^31 elements.  The float32 results equal those
 * of the plain kernels element for element.
 *
 * smrt_nn_bias_act_blocked: z = x + bias, a = SiLU(z) (or z), ab = half(a) blocked, for x (N,H,W,C).
 * smrt_nn_bias_act_bwd_blocked: dz = da * SiLU'(z) (or da), db += column sums of dz (db may be NULL),
 *   dzb = half(dz) blocked -- the operand of smrt_nn_conv3_wgrad_tma and of the input-gradient
 *   smrt_nn_conv3_tma, so the float32 dz need not be written at all.
 * smrt_nn_avgpool2_blocked: 2x2 average pooling of x (N,H,W,C) into y (N,H/2,W/2,C) and/or yb.
 * smrt_nn_upcat: the decoder input [up2(a) | b]: a (N,H,W,Ca) upsampled (nearest) to 2H x 2W next
 *   to the skip b (N,2H,2W,Cb), into y (N,2H,2W,Ca+Cb) and/or yb (Ca % 8 == 0, Cb % 8 == 0).
 * smrt_nn_upcat_bwd: its adjoint: da (N,H,W,Ca) = sum over each 2x2 block of dy[..., :Ca], db =
 *   dy[..., Ca:] (Ca % 4 == 0, Cb % 4 == 0; da or db may be NULL). */
SMRT_API int smrt_nn_bias_act_blocked(const float *x, const float *bias, int N, int H, int W, int C, int act,
                                      float *z, float *a, void *ab, void *stream);
SMRT_API int smrt_nn_bias_act_bwd_blocked(const float *da, const float *z, int N, int H, int W, int C, int act,
                                          float *dz, float *db, void *dzb, void *stream);
/* smrt_nn_bias_act_bwd_blocked of da + the 2x2 average-pooling adjoint of dp, in one pass: the encoder's
 * activation gradient is the sum of its skip part da (N,H,W,C) and its pooled part dp (N,H/2,W/2,C), each
 * of whose values goes to its four children times 1/4.  Equals smrt_nn_avgpool2_bwd, smrt_nn_add and
 * smrt_nn_bias_act_bwd_blocked in turn bit for bit (db up to summation order); H and W even. */
SMRT_API int smrt_nn_bias_act_bwd_addpool_blocked(const float *da, const float *dp, const float *z, int N, int H,
                                                  int W, int C, int act, float *dz, float *db, void *dzb,
                                                  void *stream);
SMRT_API int smrt_nn_avgpool2_blocked(const float *x, int N, int H, int W, int C, float *y, void *yb, void *stream);
SMRT_API int smrt_nn_upcat(const float *a, int N, int H, int W, int Ca, const float *b, int Cb, float *y, void *yb,
                           void *stream);
SMRT_API int smrt_nn_upcat_bwd(const float *dy, int N, int H, int W, int Ca, int Cb, float *da, float *db,
                               void *stream);

/* 1x1 convolution with at most 3 outputs (the network's head), float32 on the CUDA cores:
 *   y[p][o] = sum_c x[p][c] w[o][c] + bias[o]      (P pixels, x: P x C, w: cout x C, y: P x cout)
 * and its backward dx[p][c] = sum_o dy[p][o] w[o][c], dw[o][c] += sum_p dy[p][o] x[p][c],
 * db[o] += sum_p dy[p][o] (dx, dw, db may each be NULL; dw, db accumulate with atomics).
 * 4 <= C <= 64, C % 4 == 0, x (and dx) 16-byte aligned; bias may be NULL. */
SMRT_API int smrt_nn_conv1x1_small(const float *x, long long P, int C, const float *w, const float *bias, int cout,
                                   float *y, void *stream);
SMRT_API int smrt_nn_conv1x1_small_bwd(const float *dy, const float *x, long long P, int C, const float *w, int cout,
                                       float *dx, float *dw, float *db, void *stream);

/* 2x2 average pooling (H, W even) and its adjoint. */
SMRT_API int smrt_nn_avgpool2(const float *x, int N, int H, int W, int C, float *y, void *stream);
SMRT_API int smrt_nn_avgpool2_bwd(const float *dy, int N, int H, int W, int C, float *dx, void *stream);

/* Nearest-neighbour 2x upsampling of (N,H,W,C) to (N,2H,2W,C) and its adjoint. */
SMRT_API int smrt_nn_upsample2(const float *x, int N, int H, int W, int C, float *y, void *stream);
SMRT_API int smrt_nn_upsample2_bwd(const float *dy, int N, int H, int W, int C, float *dx, void *stream);

/* Channel concatenation y = [a | b] of (rows, Ca) and (rows, Cb), and its adjoint
 * (da, db may be NULL to skip). */
SMRT_API int smrt_nn_concat(const float *a, int Ca, const float *b, int Cb, long long rows, float *y, void *stream);
SMRT_API int smrt_nn_concat_bwd(const float *dy, int Ca, int Cb, long long rows, float *da, float *db, void *stream);

/* y = a + b, n elements (y may alias a or b). */
SMRT_API int smrt_nn_add(const float *a, const float *b, long long n, float *y, void *stream);

/* Mean squared error L = mean((y - t)^2) over n elements: loss[0] += L (double,
 * zero it first); dy = grad_scale * 2 (y - t) / n (dy may be NULL). */
SMRT_API int smrt_nn_mse(const float *y, const float *t, long long n, float grad_scale, double *loss, float *dy,
                         void *stream);

/* Adam step on n parameters: g = grad / grad_scale, m = b1 m + (1 - b1) g,
 * v = b2 v + (1 - b2) g^2, w -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * Non-finite gradients leave w, m, v unchanged and set found_inf[0] = 1. */
SMRT_API int smrt_nn_adam(float *w, const float *grad, float *m, float *v, long long n, float lr, float b1, float b2,
                          float eps, int step, float grad_scale, int *found_inf, void *stream);

/* Bilinear resampling of (N,H,W,C) to (N,H2,W2,C), node-centred on the unit square:
 * output node (i, j) samples the input at ((i + 1/2) H / H2 - 1/2, ...), clamped at the edges. */
SMRT_API int smrt_nn_resize_bilinear(const float *x, int N, int H, int W, int C, float *y, int H2, int W2,
                                     void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SMRT_NN_H */
