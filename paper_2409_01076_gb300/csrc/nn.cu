// nn.cu -- the neural-network kernels behind include/smrt_nn.h (learned warm start).
//
// GEMM on the tensor cores through WMMA (16x16x16, half operands, float32
// accumulation): 64 x 64 output tiles per 128-thread block, K in steps of 32
// staged in shared memory, optional split-K with atomic accumulation.  The
// convolutions are im2col + GEMM; everything else is elementwise or a
// fixed-order reduction.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <mma.h>

#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include "internal.h"
#include "smrt_nn.h"

namespace {

using namespace nvcuda;

constexpr int GBM = 64, GBN = 64, GBK = 32;
constexpr int APAD = 8, BPAD = 8, CPAD = 4;

__global__ void __launch_bounds__(128)
gemm_kernel(int transA, int transB, int M, int N, int K, float alpha, const __half *__restrict__ A, int lda,
            const __half *__restrict__ B, int ldb, float beta, float *C, int ldc, int k_chunk, int atomic)
{
    __shared__ __align__(32) __half As[GBM][GBK + APAD];
    __shared__ __align__(32) __half Bs[GBK][GBN + BPAD];
    __shared__ __align__(32) float Cs[GBM][GBN + CPAD];
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int kbeg = blockIdx.z * k_chunk;
    const int kend = min(K, kbeg + k_chunk);
    const int warp = threadIdx.x >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][2];
    #pragma unroll
    for (int i = 0; i < 2; ++i)
        #pragma unroll
        for (int j = 0; j < 2; ++j) wmma::fill_fragment(acc[i][j], 0.0f);
    const __half zero = __float2half(0.0f);
    for (int k0 = kbeg; k0 < kend; k0 += GBK) {
        for (int idx = threadIdx.x; idx < GBM * GBK; idx += 128) {
            int i, kk;
            if (!transA) { i = idx / GBK; kk = idx % GBK; }
            else { kk = idx / GBM; i = idx % GBM; }
            const int m = m0 + i, k = k0 + kk;
            __half v = zero;
            if (m < M && k < kend) v = transA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
            As[i][kk] = v;
        }
        for (int idx = threadIdx.x; idx < GBK * GBN; idx += 128) {
            int j, kk;
            if (!transB) { kk = idx / GBN; j = idx % GBN; }
            else { j = idx / GBK; kk = idx % GBK; }
            const int n = n0 + j, k = k0 + kk;
            __half v = zero;
            if (n < N && k < kend) v = transB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
            Bs[kk][j] = v;
        }
        __syncthreads();
        #pragma unroll
        for (int kk = 0; kk < GBK; kk += 16) {
            wmma::fragment<wmma::matrix_a, 16, 16, 16, __half, wmma::row_major> a[2];
            wmma::fragment<wmma::matrix_b, 16, 16, 16, __half, wmma::row_major> b[2];
            #pragma unroll
            for (int i = 0; i < 2; ++i) wmma::load_matrix_sync(a[i], &As[wm + 16 * i][kk], GBK + APAD);
            #pragma unroll
            for (int j = 0; j < 2; ++j) wmma::load_matrix_sync(b[j], &Bs[kk][wn + 16 * j], GBN + BPAD);
            #pragma unroll
            for (int i = 0; i < 2; ++i)
                #pragma unroll
                for (int j = 0; j < 2; ++j) wmma::mma_sync(acc[i][j], a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    #pragma unroll
    for (int i = 0; i < 2; ++i)
        #pragma unroll
        for (int j = 0; j < 2; ++j)
            wmma::store_matrix_sync(&Cs[wm + 16 * i][wn + 16 * j], acc[i][j], GBN + CPAD, wmma::mem_row_major);
    __syncthreads();
    for (int idx = threadIdx.x; idx < GBM * GBN; idx += 128) {
        const int i = idx / GBN, j = idx % GBN;
        const int m = m0 + i, n = n0 + j;
        if (m >= M || n >= N) continue;
        float *c = C + (size_t)m * ldc + n;
        const float v = alpha * Cs[i][j];
        if (atomic) atomicAdd(c, v);
        else *c = (beta != 0.0f) ? v + beta * *c : v;
    }
}

__global__ void im2col3_kernel(const float *__restrict__ x, int N, int H, int W, int C, __half *__restrict__ col,
                               int ld)
{
    const long long total = (long long)N * H * W * ld;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t % ld);
        const long long p = t / ld;
        float v = 0.0f;                 // the pad columns 9C .. ld-1 stay zero
        if (j < 9 * C) {
            const int tap = j / C, c = j % C;
            const int xx = (int)(p % W), yy = (int)((p / W) % H), n = (int)(p / ((long long)W * H));
            const int sy = yy + tap / 3 - 1, sx = xx + tap % 3 - 1;
            if (sy >= 0 && sy < H && sx >= 0 && sx < W) v = x[(((size_t)n * H + sy) * W + sx) * C + c];
        }
        col[t] = __float2half(v);
    }
}

// C % 8 == 0 and ld == 9 C: one thread per (pixel, tap, 8-channel chunk), two float4 loads, one
// 16-byte store.  Requires N*H*W*9*(C/8) < 2^31.
__global__ void im2col3_vec_kernel(const float *__restrict__ x, int N, int H, int W, int C, __half *__restrict__ col,
                                   int ld)
{
    const int cc = C >> 3;
    const int total = N * H * W * 9 * cc;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int chunk = t % cc;
        const int r = t / cc;
        const int tap = r % 9;
        const int p = r / 9;
        const int xx = p % W, rest = p / W;
        const int yy = rest % H, n = rest / H;
        const int sy = yy + tap / 3 - 1, sx = xx + tap % 3 - 1;
        uint4 out = make_uint4(0, 0, 0, 0);
        if (sy >= 0 && sy < H && sx >= 0 && sx < W) {
            const float4 *src = reinterpret_cast<const float4 *>(x + (((size_t)n * H + sy) * W + sx) * C + chunk * 8);
            const float4 a = src[0], b = src[1];
            __half2 h0 = __floats2half2_rn(a.x, a.y), h1 = __floats2half2_rn(a.z, a.w);
            __half2 h2 = __floats2half2_rn(b.x, b.y), h3 = __floats2half2_rn(b.z, b.w);
            out.x = *reinterpret_cast<unsigned *>(&h0);
            out.y = *reinterpret_cast<unsigned *>(&h1);
            out.z = *reinterpret_cast<unsigned *>(&h2);
            out.w = *reinterpret_cast<unsigned *>(&h3);
        }
        reinterpret_cast<uint4 *>(col)[(size_t)p * (ld >> 3) + (size_t)tap * cc + chunk] = out;
    }
}

__global__ void col2im3_kernel(const float *__restrict__ dcol, int N, int H, int W, int C, float *__restrict__ dx)
{
    const long long total = (long long)N * H * W * C;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % C);
        const long long p = t / C;
        const int xx = (int)(p % W), yy = (int)((p / W) % H), n = (int)(p / ((long long)W * H));
        float s = 0.0f;
        #pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            // the patch centred at (yy - dy, xx - dx) read this node through tap (dy+1, dx+1)
            const int py = yy - (tap / 3 - 1), px = xx - (tap % 3 - 1);
            if (py < 0 || py >= H || px < 0 || px >= W) continue;
            s += dcol[((((size_t)n * H + py) * W + px) * 9 + tap) * C + c];
        }
        dx[t] = s;
    }
}

__global__ void flip3_kernel(const float *__restrict__ w, int cout, int cin, __half *__restrict__ wf)
{
    const int total = cout * 9 * cin;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int o = t % cout;
        const int tap = (t / cout) % 9;
        const int c = t / (9 * cout);
        wf[t] = __float2half(w[((size_t)o * 9 + (8 - tap)) * cin + c]);   // t = (c * 9 + tap) * cout + o
    }
}

__global__ void to_half_kernel(const float *__restrict__ s, long long n, float scale, __half *__restrict__ d)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        d[t] = __float2half(scale * s[t]);
}

// Rows of `cols` floats into rows of `ld` halves, the pad columns zeroed.
__global__ void to_half_rows_kernel(const float *__restrict__ s, long long rows, int cols, float scale,
                                    __half *__restrict__ d, int ld)
{
    const long long n = rows * ld;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / ld;
        const int c = (int)(t % ld);
        d[t] = c < cols ? __float2half(scale * s[r * cols + c]) : __float2half(0.0f);
    }
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + expf(-z)); }

__global__ void bias_act_kernel(const float *__restrict__ x, const float *__restrict__ bias, long long rows, int C,
                                int act, float *z, float *a)
{
    const long long total = rows * C;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const float v = x[t] + (bias ? bias[t % C] : 0.0f);
        if (z) z[t] = v;
        a[t] = act ? v * sigmoidf_(v) : v;
    }
}

// dz and the per-block partial column sums of dz; db accumulated with one atomic per block and channel.
__global__ void bias_act_bwd_kernel(const float *__restrict__ da, const float *__restrict__ z, long long rows, int C,
                                    int act, float *dz, float *db)
{
    extern __shared__ float sdb[];            // C floats
    for (int c = threadIdx.x; c < C; c += blockDim.x) sdb[c] = 0.0f;
    __syncthreads();
    const long long total = rows * C;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        float g = da[t];
        if (act) {
            const float s = sigmoidf_(z[t]);
            g *= s * (1.0f + z[t] * (1.0f - s));
        }
        dz[t] = g;
        if (db) atomicAdd(&sdb[t % C], g);
    }
    __syncthreads();
    if (db)
        for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&db[c], sdb[c]);
}

__global__ void avgpool2_kernel(const float *__restrict__ x, int N, int H, int W, int C, float *__restrict__ y)
{
    const int Ho = H / 2, Wo = W / 2;
    const long long total = (long long)N * Ho * Wo * C;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % C);
        const long long p = t / C;
        const int xo = (int)(p % Wo), yo = (int)((p / Wo) % Ho), n = (int)(p / ((long long)Wo * Ho));
        const size_t b = (((size_t)n * H + 2 * yo) * W + 2 * xo) * C + c;
        y[t] = 0.25f * ((x[b] + x[b + C]) + (x[b + (size_t)W * C] + x[b + (size_t)W * C + C]));
    }
}

__global__ void avgpool2_bwd_kernel(const float *__restrict__ dy, int N, int H, int W, int C, float *__restrict__ dx)
{
    const long long total = (long long)N * H * W * C;
    const int Ho = H / 2, Wo = W / 2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % C);
        const long long p = t / C;
        const int xx = (int)(p % W), yy = (int)((p / W) % H), n = (int)(p / ((long long)W * H));
        dx[t] = 0.25f * dy[(((size_t)n * Ho + yy / 2) * Wo + xx / 2) * C + c];
    }
}

__global__ void upsample2_kernel(const float *__restrict__ x, int N, int H, int W, int C, float *__restrict__ y)
{
    const int H2 = 2 * H, W2 = 2 * W;
    const long long total = (long long)N * H2 * W2 * C;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % C);
        const long long p = t / C;
        const int xx = (int)(p % W2), yy = (int)((p / W2) % H2), n = (int)(p / ((long long)W2 * H2));
        y[t] = x[(((size_t)n * H + yy / 2) * W + xx / 2) * C + c];
    }
}

__global__ void upsample2_bwd_kernel(const float *__restrict__ dy, int N, int H, int W, int C, float *__restrict__ dx)
{
    const long long total = (long long)N * H * W * C;
    const int W2 = 2 * W;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % C);
        const long long p = t / C;
        const int xx = (int)(p % W), yy = (int)((p / W) % H), n = (int)(p / ((long long)W * H));
        const size_t b = (((size_t)n * 2 * H + 2 * yy) * W2 + 2 * xx) * C + c;
        dx[t] = (dy[b] + dy[b + C]) + (dy[b + (size_t)W2 * C] + dy[b + (size_t)W2 * C + C]);
    }
}

__global__ void concat_kernel(const float *__restrict__ a, int Ca, const float *__restrict__ b, int Cb, long long rows,
                              float *__restrict__ y)
{
    const int Cy = Ca + Cb;
    const long long total = rows * Cy;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % Cy);
        const long long r = t / Cy;
        y[t] = c < Ca ? a[r * Ca + c] : b[r * Cb + (c - Ca)];
    }
}

__global__ void concat_bwd_kernel(const float *__restrict__ dy, int Ca, int Cb, long long rows, float *da, float *db)
{
    const int Cy = Ca + Cb;
    const long long total = rows * Cy;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % Cy);
        const long long r = t / Cy;
        if (c < Ca) {
            if (da) da[r * Ca + c] = dy[t];
        } else if (db) {
            db[r * Cb + (c - Ca)] = dy[t];
        }
    }
}

__global__ void add_kernel(const float *a, const float *b, long long n, float *y)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        y[t] = a[t] + b[t];
}

__global__ void mse_kernel(const float *__restrict__ y, const float *__restrict__ tt, long long n, float grad_scale,
                           double *loss, float *dy)
{
    __shared__ double red[256 / 32];
    double s = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const float d = y[t] - tt[t];
        s += (double)d * d;
        if (dy) dy[t] = grad_scale * 2.0f * d / (float)n;
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += red[w];
        atomicAdd(loss, b / (double)n);
    }
}

__global__ void adam_kernel(float *w, const float *__restrict__ g, float *m, float *v, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2, float inv_scale, int *found_inf)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const float gi = g[t] * inv_scale;
        if (!isfinite(gi)) {
            *found_inf = 1;
            continue;
        }
        const float mi = b1 * m[t] + (1.0f - b1) * gi;
        const float vi = b2 * v[t] + (1.0f - b2) * gi * gi;
        m[t] = mi;
        v[t] = vi;
        w[t] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void resize_bilinear_kernel(const float *__restrict__ x, int N, int H, int W, int C, float *__restrict__ y,
                                       int H2, int W2)
{
    const long long total = (long long)N * H2 * W2 * C;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % C);
        const long long p = t / C;
        const int xx = (int)(p % W2), yy = (int)((p / W2) % H2), n = (int)(p / ((long long)W2 * H2));
        float sy = ((float)yy + 0.5f) * (float)H / (float)H2 - 0.5f;
        float sx = ((float)xx + 0.5f) * (float)W / (float)W2 - 0.5f;
        sy = fminf(fmaxf(sy, 0.0f), (float)(H - 1));
        sx = fminf(fmaxf(sx, 0.0f), (float)(W - 1));
        const int y0 = min((int)sy, H - 1), x0 = min((int)sx, W - 1);
        const int y1 = min(y0 + 1, H - 1), x1 = min(x0 + 1, W - 1);
        const float fy = sy - (float)y0, fx = sx - (float)x0;
        const float *b = x + (size_t)n * H * W * C + c;
        const float v00 = b[((size_t)y0 * W + x0) * C], v01 = b[((size_t)y0 * W + x1) * C];
        const float v10 = b[((size_t)y1 * W + x0) * C], v11 = b[((size_t)y1 * W + x1) * C];
        y[t] = (1.0f - fy) * ((1.0f - fx) * v00 + fx * v01) + fy * ((1.0f - fx) * v10 + fx * v11);
    }
}

int nn_fail(int code, const char *fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    smrt::set_thread_error(buf);
    return code;
}

// Status of a launch whose error the launcher already fetched.
int vec_done(cudaError_t e, const char *what)
{
    return e == cudaSuccess ? SMRT_OK : nn_fail(SMRT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int launched(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return nn_fail(SMRT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return SMRT_OK;
}

unsigned grid_for(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 152LL * 64) b = 152LL * 64;
    return (unsigned)(b < 1 ? 1 : b);
}

} // namespace

extern "C" {

int smrt_nn_gemm(int transA, int transB, int M, int N, int K, float alpha, const void *A, int lda, const void *B,
                 int ldb, float beta, float *C, int ldc, int split_k, void *stream)
{
    if (M < 0 || N < 0 || K < 0 || !A || !B || !C || split_k < 1 || ldc < N ||
        lda < (transA ? M : K) || ldb < (transB ? K : N))
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_gemm: bad arguments (M %d N %d K %d lda %d ldb %d ldc %d split %d)", M,
                       N, K, lda, ldb, ldc, split_k);
    if (M == 0 || N == 0) return SMRT_OK;
    int chunk = (K + split_k - 1) / split_k;
    chunk = ((chunk + GBK - 1) / GBK) * GBK;
    const int splits = K == 0 ? 1 : (K + chunk - 1) / chunk;
    dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM, splits);
    if (grid.y > 65535 || grid.z > 65535) return nn_fail(SMRT_ERR_ARG, "smrt_nn_gemm: M or split_k too large");
    gemm_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>(transA, transB, M, N, K, alpha, (const __half *)A, lda,
                                                        (const __half *)B, ldb, beta, C, ldc, chunk,
                                                        split_k > 1 ? 1 : 0);
    return launched("smrt_nn_gemm");
}

int smrt_nn_im2col3(const float *x, int N, int H, int W, int C, void *col, int ld, void *stream)
{
    if (!x || !col || N < 1 || H < 1 || W < 1 || C < 1 || ld < 9 * C)
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_im2col3: bad arguments");
    const long long chunks = (long long)N * H * W * 9 * (C / 8);
    if (C % 8 == 0 && ld == 9 * C && chunks < (1LL << 31) &&
        ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(col)) & 15) == 0) {
        im2col3_vec_kernel<<<grid_for(chunks), 256, 0, (cudaStream_t)stream>>>(x, N, H, W, C, (__half *)col, ld);
        return launched("smrt_nn_im2col3");
    }
    im2col3_kernel<<<grid_for((long long)N * H * W * ld), 256, 0, (cudaStream_t)stream>>>(x, N, H, W, C,
                                                                                          (__half *)col, ld);
    return launched("smrt_nn_im2col3");
}

int smrt_nn_col2im3(const float *dcol, int N, int H, int W, int C, float *dx, void *stream)
{
    if (!dcol || !dx || N < 1 || H < 1 || W < 1 || C < 1) return nn_fail(SMRT_ERR_ARG, "smrt_nn_col2im3: bad arguments");
    col2im3_kernel<<<grid_for((long long)N * H * W * C), 256, 0, (cudaStream_t)stream>>>(dcol, N, H, W, C, dx);
    return launched("smrt_nn_col2im3");
}

int smrt_nn_flip3(const float *w, int cout, int cin, void *wf, void *stream)
{
    if (!w || !wf || cout < 1 || cin < 1) return nn_fail(SMRT_ERR_ARG, "smrt_nn_flip3: bad arguments");
    flip3_kernel<<<grid_for((long long)cout * 9 * cin), 256, 0, (cudaStream_t)stream>>>(w, cout, cin, (__half *)wf);
    return launched("smrt_nn_flip3");
}

int smrt_nn_to_half_rows(const float *src, long long rows, int cols, float scale, void *dst, int ld, void *stream)
{
    if (!src || !dst || rows < 0 || cols < 1 || ld < cols) return nn_fail(SMRT_ERR_ARG, "smrt_nn_to_half_rows: bad arguments");
    if (rows == 0) return SMRT_OK;
    to_half_rows_kernel<<<grid_for(rows * ld), 256, 0, (cudaStream_t)stream>>>(src, rows, cols, scale, (__half *)dst, ld);
    return launched("smrt_nn_to_half_rows");
}

int smrt_nn_to_half(const float *src, long long n, float scale, void *dst, void *stream)
{
    if (!src || !dst || n < 0) return nn_fail(SMRT_ERR_ARG, "smrt_nn_to_half: bad arguments");
    if (n == 0) return SMRT_OK;
    to_half_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(src, n, scale, (__half *)dst);
    return launched("smrt_nn_to_half");
}

int smrt_nn_bias_act(const float *x, const float *bias, long long rows, int C, int act, float *z, float *a,
                     void *stream)
{
    if (!x || !a || rows < 0 || C < 1) return nn_fail(SMRT_ERR_ARG, "smrt_nn_bias_act: bad arguments");
    if (rows == 0) return SMRT_OK;
    const cudaError_t e = smrt::vec_bias_act(x, bias, rows, C, act, z, a, nullptr, 1, (cudaStream_t)stream);
    if (e != cudaErrorNotSupported) return vec_done(e, "smrt_nn_bias_act");
    bias_act_kernel<<<grid_for(rows * C), 256, 0, (cudaStream_t)stream>>>(x, bias, rows, C, act, z, a);
    return launched("smrt_nn_bias_act");
}

int smrt_nn_bias_act_bwd(const float *da, const float *z, long long rows, int C, int act, float *dz, float *db,
                         void *stream)
{
    if (!da || !dz || (act && !z) || rows < 0 || C < 1 || C > 4096)
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_bias_act_bwd: bad arguments");
    if (rows == 0) return SMRT_OK;
    const cudaError_t e = smrt::vec_bias_act_bwd(da, z, rows, C, act, dz, db, nullptr, 1, (cudaStream_t)stream);
    if (e != cudaErrorNotSupported) return vec_done(e, "smrt_nn_bias_act_bwd");
    bias_act_bwd_kernel<<<grid_for(rows * C), 256, C * sizeof(float), (cudaStream_t)stream>>>(da, z, rows, C, act, dz,
                                                                                                db);
    return launched("smrt_nn_bias_act_bwd");
}

int smrt_nn_avgpool2(const float *x, int N, int H, int W, int C, float *y, void *stream)
{
    if (!x || !y || N < 1 || H < 2 || W < 2 || C < 1 || (H & 1) || (W & 1))
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_avgpool2: bad arguments");
    avgpool2_kernel<<<grid_for((long long)N * (H / 2) * (W / 2) * C), 256, 0, (cudaStream_t)stream>>>(x, N, H, W, C,
                                                                                                        y);
    return launched("smrt_nn_avgpool2");
}

int smrt_nn_avgpool2_bwd(const float *dy, int N, int H, int W, int C, float *dx, void *stream)
{
    if (!dy || !dx || N < 1 || H < 2 || W < 2 || C < 1 || (H & 1) || (W & 1))
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_avgpool2_bwd: bad arguments");
    const cudaError_t e = smrt::vec_avgpool2_bwd(dy, N, H, W, C, dx, (cudaStream_t)stream);
    if (e != cudaErrorNotSupported) return vec_done(e, "smrt_nn_avgpool2_bwd");
    avgpool2_bwd_kernel<<<grid_for((long long)N * H * W * C), 256, 0, (cudaStream_t)stream>>>(dy, N, H, W, C, dx);
    return launched("smrt_nn_avgpool2_bwd");
}

int smrt_nn_upsample2(const float *x, int N, int H, int W, int C, float *y, void *stream)
{
    if (!x || !y || N < 1 || H < 1 || W < 1 || C < 1) return nn_fail(SMRT_ERR_ARG, "smrt_nn_upsample2: bad arguments");
    upsample2_kernel<<<grid_for((long long)N * 4 * H * W * C), 256, 0, (cudaStream_t)stream>>>(x, N, H, W, C, y);
    return launched("smrt_nn_upsample2");
}

int smrt_nn_upsample2_bwd(const float *dy, int N, int H, int W, int C, float *dx, void *stream)
{
    if (!dy || !dx || N < 1 || H < 1 || W < 1 || C < 1)
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_upsample2_bwd: bad arguments");
    upsample2_bwd_kernel<<<grid_for((long long)N * H * W * C), 256, 0, (cudaStream_t)stream>>>(dy, N, H, W, C, dx);
    return launched("smrt_nn_upsample2_bwd");
}

int smrt_nn_concat(const float *a, int Ca, const float *b, int Cb, long long rows, float *y, void *stream)
{
    if (!a || !b || !y || Ca < 1 || Cb < 1 || rows < 0) return nn_fail(SMRT_ERR_ARG, "smrt_nn_concat: bad arguments");
    if (rows == 0) return SMRT_OK;
    concat_kernel<<<grid_for(rows * (Ca + Cb)), 256, 0, (cudaStream_t)stream>>>(a, Ca, b, Cb, rows, y);
    return launched("smrt_nn_concat");
}

int smrt_nn_concat_bwd(const float *dy, int Ca, int Cb, long long rows, float *da, float *db, void *stream)
{
    if (!dy || Ca < 1 || Cb < 1 || rows < 0) return nn_fail(SMRT_ERR_ARG, "smrt_nn_concat_bwd: bad arguments");
    if (rows == 0) return SMRT_OK;
    concat_bwd_kernel<<<grid_for(rows * (Ca + Cb)), 256, 0, (cudaStream_t)stream>>>(dy, Ca, Cb, rows, da, db);
    return launched("smrt_nn_concat_bwd");
}

int smrt_nn_add(const float *a, const float *b, long long n, float *y, void *stream)
{
    if (!a || !b || !y || n < 0) return nn_fail(SMRT_ERR_ARG, "smrt_nn_add: bad arguments");
    if (n == 0) return SMRT_OK;
    const cudaError_t e = smrt::vec_add(a, b, n, y, (cudaStream_t)stream);
    if (e != cudaErrorNotSupported) return vec_done(e, "smrt_nn_add");
    add_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(a, b, n, y);
    return launched("smrt_nn_add");
}

int smrt_nn_bias_act_blocked(const float *x, const float *bias, int N, int H, int W, int C, int act, float *z,
                             float *a, void *ab, void *stream)
{
    if (!x || N < 1 || H < 1 || W < 1 || C < 8 || C % 8 != 0 || (long long)N * H * W * C >= (1LL << 31))
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_bias_act_blocked: bad arguments (N %d H %d W %d C %d; C %% 8 == 0)", N,
                       H, W, C);
    const cudaError_t e = smrt::vec_bias_act(x, bias, (long long)N * H * W, C, act, z, a, (__half *)ab, H * W,
                                             (cudaStream_t)stream);
    if (e == cudaErrorNotSupported) return nn_fail(SMRT_ERR_ARG, "smrt_nn_bias_act_blocked: misaligned pointer");
    return vec_done(e, "smrt_nn_bias_act_blocked");
}

int smrt_nn_bias_act_bwd_blocked(const float *da, const float *z, int N, int H, int W, int C, int act, float *dz,
                                 float *db, void *dzb, void *stream)
{
    if (!da || (act && !z) || N < 1 || H < 1 || W < 1 || C < 8 || C % 8 != 0 || C > 4096 ||
        (long long)N * H * W * C >= (1LL << 31))
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_bias_act_bwd_blocked: bad arguments (N %d H %d W %d C %d; C %% 8 == 0)",
                       N, H, W, C);
    const cudaError_t e = smrt::vec_bias_act_bwd(da, z, (long long)N * H * W, C, act, dz, db, (__half *)dzb, H * W,
                                                 (cudaStream_t)stream);
    if (e == cudaErrorNotSupported) return nn_fail(SMRT_ERR_ARG, "smrt_nn_bias_act_bwd_blocked: misaligned pointer");
    return vec_done(e, "smrt_nn_bias_act_bwd_blocked");
}

int smrt_nn_bias_act_bwd_addpool_blocked(const float *da, const float *dp, const float *z, int N, int H, int W, int C,
                                         int act, float *dz, float *db, void *dzb, void *stream)
{
    if (!da || !dp || (act && !z) || N < 1 || H < 2 || W < 2 || (H & 1) || (W & 1) || C < 8 || C % 8 != 0 ||
        C > 4096 || (long long)N * H * W * C >= (1LL << 31))
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_bias_act_bwd_addpool_blocked: bad arguments (N %d H %d W %d C %d; even H "
                       "and W, C %% 8 == 0)", N, H, W, C);
    const cudaError_t e = smrt::vec_bias_act_bwd(da, z, (long long)N * H * W, C, act, dz, db, (__half *)dzb, H * W,
                                                 (cudaStream_t)stream, dp, W);
    if (e == cudaErrorNotSupported)
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_bias_act_bwd_addpool_blocked: misaligned pointer");
    return vec_done(e, "smrt_nn_bias_act_bwd_addpool_blocked");
}

int smrt_nn_avgpool2_blocked(const float *x, int N, int H, int W, int C, float *y, void *yb, void *stream)
{
    if (!x || N < 1 || H < 2 || W < 2 || (H & 1) || (W & 1) || C < 8 || C % 8 != 0)
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_avgpool2_blocked: bad arguments (N %d H %d W %d C %d)", N, H, W, C);
    const cudaError_t e = smrt::vec_avgpool2(x, N, H, W, C, y, (__half *)yb, (cudaStream_t)stream);
    if (e == cudaErrorNotSupported)
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_avgpool2_blocked: misaligned pointer or too many elements");
    return vec_done(e, "smrt_nn_avgpool2_blocked");
}

int smrt_nn_upcat(const float *a, int N, int H, int W, int Ca, const float *b, int Cb, float *y, void *yb,
                  void *stream)
{
    const uintptr_t al = reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) |
                         reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(yb);
    if (!a || !b || N < 1 || H < 1 || W < 1 || Ca < 8 || Cb < 8 || Ca % 8 || Cb % 8 || (al & 15) ||
        4LL * N * H * W * (Ca + Cb) >= (1LL << 31))
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_upcat: bad arguments (N %d H %d W %d Ca %d Cb %d)", N, H, W, Ca, Cb);
    return vec_done(smrt::vec_upcat(a, N, H, W, Ca, b, Cb, y, (__half *)yb, (cudaStream_t)stream), "smrt_nn_upcat");
}

int smrt_nn_upcat_bwd(const float *dy, int N, int H, int W, int Ca, int Cb, float *da, float *db, void *stream)
{
    const uintptr_t al = reinterpret_cast<uintptr_t>(dy) | reinterpret_cast<uintptr_t>(da) |
                         reinterpret_cast<uintptr_t>(db);
    if (!dy || N < 1 || H < 1 || W < 1 || Ca < 4 || Cb < 4 || Ca % 4 || Cb % 4 || (al & 15) ||
        4LL * N * H * W * (Ca + Cb) >= (1LL << 31))
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_upcat_bwd: bad arguments (N %d H %d W %d Ca %d Cb %d)", N, H, W, Ca, Cb);
    return vec_done(smrt::vec_upcat_bwd(dy, N, H, W, Ca, Cb, da, db, (cudaStream_t)stream), "smrt_nn_upcat_bwd");
}

int smrt_nn_conv1x1_small(const float *x, long long P, int C, const float *w, const float *bias, int cout, float *y,
                          void *stream)
{
    if (!x || !w || !y || P < 1 || P >= (1LL << 31) || C < 4 || C > 64 || C % 4 || cout < 1 || cout > 3 ||
        (reinterpret_cast<uintptr_t>(x) & 15))
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_conv1x1_small: bad arguments (P %lld C %d cout %d)", P, C, cout);
    return vec_done(smrt::small_conv1x1(x, P, C, w, bias, cout, y, (cudaStream_t)stream), "smrt_nn_conv1x1_small");
}

int smrt_nn_conv1x1_small_bwd(const float *dy, const float *x, long long P, int C, const float *w, int cout, float *dx,
                              float *dw, float *db, void *stream)
{
    if (!dy || !x || !w || P < 1 || P >= (1LL << 31) || C < 4 || C > 64 || C % 4 || cout < 1 || cout > 3 ||
        ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(dx)) & 15))
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_conv1x1_small_bwd: bad arguments (P %lld C %d cout %d)", P, C, cout);
    return vec_done(smrt::small_conv1x1_bwd(dy, x, P, C, w, cout, dx, dw, db, (cudaStream_t)stream),
                    "smrt_nn_conv1x1_small_bwd");
}

int smrt_nn_mse(const float *y, const float *t, long long n, float grad_scale, double *loss, float *dy, void *stream)
{
    if (!y || !t || !loss || n < 1) return nn_fail(SMRT_ERR_ARG, "smrt_nn_mse: bad arguments");
    mse_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(y, t, n, grad_scale, loss, dy);
    return launched("smrt_nn_mse");
}

int smrt_nn_adam(float *w, const float *grad, float *m, float *v, long long n, float lr, float b1, float b2, float eps,
                 int step, float grad_scale, int *found_inf, void *stream)
{
    if (!w || !grad || !m || !v || !found_inf || n < 0 || step < 1 || !(grad_scale > 0.0f))
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_adam: bad arguments");
    if (n == 0) return SMRT_OK;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    adam_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(w, grad, m, v, n, lr, b1, b2, eps, c1, c2,
                                                               1.0f / grad_scale, found_inf);
    return launched("smrt_nn_adam");
}

int smrt_nn_resize_bilinear(const float *x, int N, int H, int W, int C, float *y, int H2, int W2, void *stream)
{
    if (!x || !y || N < 1 || H < 1 || W < 1 || C < 1 || H2 < 1 || W2 < 1)
        return nn_fail(SMRT_ERR_ARG, "smrt_nn_resize_bilinear: bad arguments");
    resize_bilinear_kernel<<<grid_for((long long)N * H2 * W2 * C), 256, 0, (cudaStream_t)stream>>>(x, N, H, W, C, y,
                                                                                                     H2, W2);
    return launched("smrt_nn_resize_bilinear");
}

} // extern "C"
