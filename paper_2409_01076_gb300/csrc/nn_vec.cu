// nn_vec.cu -- vectorised and fused element-wise kernels of the U-Net (include/smrt_nn.h).
//
// Every thread moves V = 4 or 8 consecutive channels of one pixel as 16-byte vectors, with 32-bit
// index arithmetic (element counts below 2^31).  The fused forms write what the next kernel reads:
// the blocked half layout [N][C/8][H][W][8] of the TMA convolutions (so no separate conversion
// pass reads the float32 tensor back), the nearest upsampling together with the skip concatenation
// of the decoder, and its adjoint in one pass.  The plain entry points of nn.cu (bias_act,
// bias_act_bwd, avgpool2_bwd, add) dispatch here when C % 4 == 0 and the pointers are 16-byte
// aligned; each kernel computes exactly what the scalar kernel computes, element for element.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <stdint.h>

#include "internal.h"

namespace {

template <int V>
struct Vec {
    float v[V];
};

template <int V>
__device__ __forceinline__ Vec<V> ldv(const float *p)
{
    Vec<V> r;
    #pragma unroll
    for (int i = 0; i < V; i += 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p + i);
        r.v[i] = q.x; r.v[i + 1] = q.y; r.v[i + 2] = q.z; r.v[i + 3] = q.w;
    }
    return r;
}

template <int V>
__device__ __forceinline__ void stv(float *p, const Vec<V> &r)
{
    #pragma unroll
    for (int i = 0; i < V; i += 4)
        *reinterpret_cast<float4 *>(p + i) = make_float4(r.v[i], r.v[i + 1], r.v[i + 2], r.v[i + 3]);
}

// Eight floats as eight halves (round to nearest), one 16-byte store.
__device__ __forceinline__ void st_half8(__half *p, const Vec<8> &r)
{
    __half2 h[4];
    #pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2half2_rn(r.v[2 * i], r.v[2 * i + 1]);
    *reinterpret_cast<uint4 *>(p) = *reinterpret_cast<uint4 *>(h);
}

// Offset (in halves) of channels [8g, 8g + 8) of pixel p = n * HW + rem in the blocked layout.
__device__ __forceinline__ size_t blocked_off(int p, int g, int G, int HW)
{
    const int n = p / HW, rem = p - n * HW;
    return (((size_t)n * G + g) * HW + rem) * 8;
}

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + expf(-z)); }

// z = x + bias; a = SiLU(z) (or z); ab = half(a) blocked (V == 8 only).  Thread: pixel p, group g.
template <int V>
__global__ void bias_act_vec(const float *__restrict__ x, const float *__restrict__ bias, int P, int C, int act,
                             float *z, float *a, __half *__restrict__ ab, int HW)
{
    const int G = C / V, total = P * G;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int p = t / G, g = t - p * G;
        const size_t off = (size_t)p * C + (size_t)g * V;
        Vec<V> v = ldv<V>(x + off);
        if (bias) {
            const Vec<V> b = ldv<V>(bias + g * V);
            #pragma unroll
            for (int i = 0; i < V; ++i) v.v[i] += b.v[i];
        }
        if (z) stv<V>(z + off, v);
        if (act) {
            #pragma unroll
            for (int i = 0; i < V; ++i) v.v[i] = v.v[i] * sigm(v.v[i]);
        }
        if (a) stv<V>(a + off, v);
        if constexpr (V == 8) {
            if (ab) st_half8(ab + blocked_off(p, g, G, HW), v);
        }
    }
}

// dz = da * SiLU'(z) (or da); db[c] += sum over pixels of dz; dzb = half(dz) blocked (V == 8 only).
// The grid stride is a multiple of G = C / V, so every thread keeps one channel group and sums its
// share of db in registers; a block adds its per-channel sums with one atomic each.
template <int V>
// dp (may be NULL): a gradient at half resolution whose 2x2 average-pooling adjoint (0.25 dp of the
// parent pixel) is added to da first; W is the full-resolution width.
__global__ void bias_act_bwd_vec(const float *__restrict__ da, const float *__restrict__ z, int P, int C, int act,
                                 float *dz, float *db, __half *__restrict__ dzb, int HW,
                                 const float *__restrict__ dp = nullptr, int W = 0)
{
    extern __shared__ float sdb[];          // C floats
    for (int c = threadIdx.x; c < C; c += blockDim.x) sdb[c] = 0.0f;
    __syncthreads();
    const int G = C / V, total = P * G;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int g = t0 % G;
    float acc[V];
    #pragma unroll
    for (int i = 0; i < V; ++i) acc[i] = 0.0f;
    for (int t = t0; t < total; t += gridDim.x * blockDim.x) {
        const int p = t / G;
        const size_t off = (size_t)p * C + (size_t)g * V;
        Vec<V> d = ldv<V>(da + off);
        if (dp) {
            const int n = p / HW, r = p - n * HW, yy = r / W, xx = r - yy * W;
            const Vec<V> q = ldv<V>(dp + (((size_t)n * (HW / W / 2) + yy / 2) * (W / 2) + xx / 2) * C + (size_t)g * V);
            #pragma unroll
            for (int i = 0; i < V; ++i) d.v[i] += 0.25f * q.v[i];
        }
        if (act) {
            const Vec<V> zz = ldv<V>(z + off);
            #pragma unroll
            for (int i = 0; i < V; ++i) {
                const float s = sigm(zz.v[i]);
                d.v[i] *= s * (1.0f + zz.v[i] * (1.0f - s));
            }
        }
        if (dz) stv<V>(dz + off, d);
        #pragma unroll
        for (int i = 0; i < V; ++i) acc[i] += d.v[i];
        if constexpr (V == 8) {
            if (dzb) st_half8(dzb + blocked_off(p, g, G, HW), d);
        }
    }
    if (db) {
        #pragma unroll
        for (int i = 0; i < V; ++i) atomicAdd(&sdb[g * V + i], acc[i]);
        __syncthreads();
        for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&db[c], sdb[c]);
    }
}

// 2x2 average pooling, float32 and/or blocked half output.  Thread: output pixel q, group g of 8.
__global__ void avgpool2_vec(const float *__restrict__ x, int N, int H, int W, int C, float *y, __half *yb)
{
    const int Ho = H / 2, Wo = W / 2, G = C / 8, total = N * Ho * Wo * G;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int q = t / G, g = t - q * G;
        const int n = q / (Ho * Wo), r = q - n * Ho * Wo, yo = r / Wo, xo = r - yo * Wo;
        const float *b = x + (((size_t)n * H + 2 * yo) * W + 2 * xo) * C + 8 * g;
        const Vec<8> a0 = ldv<8>(b), a1 = ldv<8>(b + C), a2 = ldv<8>(b + (size_t)W * C),
                     a3 = ldv<8>(b + (size_t)W * C + C);
        Vec<8> o;
        #pragma unroll
        for (int i = 0; i < 8; ++i) o.v[i] = 0.25f * ((a0.v[i] + a1.v[i]) + (a2.v[i] + a3.v[i]));
        if (y) stv<8>(y + (size_t)q * C + 8 * g, o);
        if (yb) st_half8(yb + blocked_off(q, g, G, Ho * Wo), o);
    }
}

// dx = 0.25 dy of the covering output pixel.  Thread: input pixel p, group of 4.
__global__ void avgpool2_bwd_vec(const float *__restrict__ dy, int N, int H, int W, int C, float *__restrict__ dx)
{
    const int G = C / 4, total = N * H * W * G, Ho = H / 2, Wo = W / 2;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int p = t / G, g = t - p * G;
        const int n = p / (H * W), r = p - n * H * W, yy = r / W, xx = r - yy * W;
        Vec<4> v = ldv<4>(dy + (((size_t)n * Ho + yy / 2) * Wo + xx / 2) * C + 4 * g);
        #pragma unroll
        for (int i = 0; i < 4; ++i) v.v[i] *= 0.25f;
        stv<4>(dx + (size_t)p * C + 4 * g, v);
    }
}

// y = [up2(a) | b] at 2H x 2W, float32 and/or blocked half.  Thread: output pixel q, group g of 8.
__global__ void upcat_vec(const float *__restrict__ a, int N, int H, int W, int Ca, const float *__restrict__ b,
                          int Cb, float *y, __half *yb)
{
    const int H2 = 2 * H, W2 = 2 * W, Cy = Ca + Cb, G = Cy / 8, Ga = Ca / 8, total = N * H2 * W2 * G;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int q = t / G, g = t - q * G;
        Vec<8> v;
        if (g < Ga) {
            const int n = q / (H2 * W2), r = q - n * H2 * W2, yy = r / W2, xx = r - yy * W2;
            v = ldv<8>(a + (((size_t)n * H + yy / 2) * W + xx / 2) * Ca + 8 * g);
        } else {
            v = ldv<8>(b + (size_t)q * Cb + 8 * (g - Ga));
        }
        if (y) stv<8>(y + (size_t)q * Cy + 8 * g, v);
        if (yb) st_half8(yb + blocked_off(q, g, G, H2 * W2), v);
    }
}

// Adjoint of upcat: da (N,H,W,Ca) = sum over each 2x2 block of dy[..., :Ca]; db = dy[..., Ca:].
// Threads [0, n1) make da (low-res pixel, group of 4), threads [n1, n1 + n2) copy db.
__global__ void upcat_bwd_vec(const float *__restrict__ dy, int N, int H, int W, int Ca, int Cb, float *da, float *db)
{
    const int W2 = 2 * W, Cy = Ca + Cb, Ga = Ca / 4, Gb = Cb / 4;
    const int n1 = da ? N * H * W * Ga : 0, n2 = db ? N * 4 * H * W * Gb : 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n1 + n2; t += gridDim.x * blockDim.x) {
        if (t < n1) {
            const int p = t / Ga, g = t - p * Ga;
            const int n = p / (H * W), r = p - n * H * W, yy = r / W, xx = r - yy * W;
            const float *s = dy + (((size_t)n * 2 * H + 2 * yy) * W2 + 2 * xx) * Cy + 4 * g;
            const Vec<4> a0 = ldv<4>(s), a1 = ldv<4>(s + Cy), a2 = ldv<4>(s + (size_t)W2 * Cy),
                         a3 = ldv<4>(s + (size_t)W2 * Cy + Cy);
            Vec<4> o;
            #pragma unroll
            for (int i = 0; i < 4; ++i) o.v[i] = (a0.v[i] + a1.v[i]) + (a2.v[i] + a3.v[i]);
            stv<4>(da + (size_t)p * Ca + 4 * g, o);
        } else {
            const int u = t - n1, q = u / Gb, g = u - q * Gb;
            stv<4>(db + (size_t)q * Cb + 4 * g, ldv<4>(dy + (size_t)q * Cy + Ca + 4 * g));
        }
    }
}

__global__ void add_vec(const float *a, const float *b, int n4, float *y)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += gridDim.x * blockDim.x) {
        Vec<4> u = ldv<4>(a + 4 * (size_t)t);
        const Vec<4> w = ldv<4>(b + 4 * (size_t)t);
        #pragma unroll
        for (int i = 0; i < 4; ++i) u.v[i] += w.v[i];
        stv<4>(y + 4 * (size_t)t, u);
    }
}

__device__ __forceinline__ float warp_sum(float v)
{
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 1x1 convolution with few outputs (the network's head), float32 on the CUDA cores: a product of
// COUT x C per pixel is far too narrow for the tensor cores and is bound by reading x.
// Forward: y[p][o] = sum_c x[p][c] w[o][c] + b[o].  Thread: one pixel.
template <int COUT>
__global__ void conv1x1_small(const float *__restrict__ x, int P, int C, const float *__restrict__ w,
                              const float *__restrict__ bias, float *__restrict__ y)
{
    extern __shared__ float sw[];           // COUT x C weights
    for (int i = threadIdx.x; i < COUT * C; i += blockDim.x) sw[i] = w[i];
    __syncthreads();
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        float acc[COUT];
        #pragma unroll
        for (int o = 0; o < COUT; ++o) acc[o] = bias ? bias[o] : 0.0f;
        const float *xp = x + (size_t)p * C;
        for (int c = 0; c < C; c += 4) {
            const Vec<4> v = ldv<4>(xp + c);
            #pragma unroll
            for (int o = 0; o < COUT; ++o)
                #pragma unroll
                for (int i = 0; i < 4; ++i) acc[o] = fmaf(v.v[i], sw[o * C + c + i], acc[o]);
        }
        #pragma unroll
        for (int o = 0; o < COUT; ++o) y[(size_t)p * COUT + o] = acc[o];
    }
}

// Backward of conv1x1_small: dx[p][c] = sum_o dy[p][o] w[o][c]; dw[o][c] += sum_p dy[p][o] x[p][c];
// db[o] += sum_p dy[p][o].  Thread: one pixel at a time, its share of dw / db in registers; a block
// adds them up in shared memory and then into dw / db with one atomic per entry.  C <= 64.
template <int COUT>
__global__ void __launch_bounds__(128)
conv1x1_small_bwd(const float *__restrict__ dy, const float *__restrict__ x, int P, int C,
                  const float *__restrict__ w, float *__restrict__ dx, float *dw, float *db)
{
    __shared__ float sw[COUT * 64];
    __shared__ float sacc[COUT * 64 + COUT];
    for (int i = threadIdx.x; i < COUT * C; i += blockDim.x) sw[i] = w[i];
    for (int i = threadIdx.x; i < COUT * C + COUT; i += blockDim.x) sacc[i] = 0.0f;
    __syncthreads();
    float gw[COUT][64 / 4][4];
    float gb[COUT];
    #pragma unroll
    for (int o = 0; o < COUT; ++o) {
        gb[o] = 0.0f;
        #pragma unroll
        for (int q = 0; q < 16; ++q)
            #pragma unroll
            for (int i = 0; i < 4; ++i) gw[o][q][i] = 0.0f;
    }
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        float g[COUT];
        #pragma unroll
        for (int o = 0; o < COUT; ++o) {
            g[o] = dy[(size_t)p * COUT + o];
            gb[o] += g[o];
        }
        const float *xp = x + (size_t)p * C;
        float *dxp = dx ? dx + (size_t)p * C : nullptr;
        #pragma unroll
        for (int q = 0; q < 16; ++q) {
            if (4 * q >= C) break;
            const Vec<4> v = ldv<4>(xp + 4 * q);
            Vec<4> d;
            #pragma unroll
            for (int i = 0; i < 4; ++i) {
                float s = 0.0f;
                #pragma unroll
                for (int o = 0; o < COUT; ++o) {
                    gw[o][q][i] = fmaf(g[o], v.v[i], gw[o][q][i]);
                    s = fmaf(g[o], sw[o * C + 4 * q + i], s);
                }
                d.v[i] = s;
            }
            if (dxp) stv<4>(dxp + 4 * q, d);
        }
    }
    // warp sums first (shuffles), then one shared-memory atomic per warp and entry
    const bool lead = (threadIdx.x & 31) == 0;
    #pragma unroll
    for (int o = 0; o < COUT; ++o) {
        const float b = warp_sum(gb[o]);
        if (lead) atomicAdd(&sacc[COUT * C + o], b);
        #pragma unroll
        for (int q = 0; q < 16; ++q) {
            if (4 * q >= C) break;
            #pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float v = warp_sum(gw[o][q][i]);
                if (lead) atomicAdd(&sacc[o * C + 4 * q + i], v);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < COUT * C; i += blockDim.x)
        if (dw) atomicAdd(&dw[i], sacc[i]);
    for (int o = threadIdx.x; o < COUT; o += blockDim.x)
        if (db) atomicAdd(&db[o], sacc[COUT * C + o]);
}

bool al16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

unsigned blocks_for(long long n)
{
    long long b = (n + 255) / 256;
    if (b > 152LL * 16) b = 152LL * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

int gcd(int a, int b) { return b ? gcd(b, a % b) : a; }

// A grid whose stride (blocks x 256) is a multiple of G, so that each thread keeps one channel group.
unsigned blocks_for_groups(long long n, int G)
{
    const int unit = G / gcd(G, 256);
    long long b = blocks_for(n);
    b = (b + unit - 1) / unit * unit;
    return (unsigned)b;
}

} // namespace

namespace smrt {

// The vectorised paths of nn.cu's plain entry points; cudaErrorNotSupported when not applicable.
cudaError_t vec_bias_act(const float *x, const float *bias, long long rows, int C, int act, float *z, float *a,
                         __half *ab, int HW, cudaStream_t s)
{
    const int V = (C % 8 == 0) ? 8 : (C % 4 == 0 ? 4 : 0);
    if (!V || (ab && V != 8) || rows * C >= (1LL << 31) || !al16(x) || (bias && !al16(bias)) || (z && !al16(z)) ||
        (a && !al16(a)) || (ab && !al16(ab)))
        return cudaErrorNotSupported;
    const long long n = rows * (C / V);
    if (V == 8) bias_act_vec<8><<<blocks_for(n), 256, 0, s>>>(x, bias, (int)rows, C, act, z, a, ab, HW);
    else bias_act_vec<4><<<blocks_for(n), 256, 0, s>>>(x, bias, (int)rows, C, act, z, a, nullptr, HW);
    return cudaGetLastError();
}

cudaError_t vec_bias_act_bwd(const float *da, const float *z, long long rows, int C, int act, float *dz, float *db,
                             __half *dzb, int HW, cudaStream_t s, const float *dp, int W)
{
    const int V = (C % 8 == 0) ? 8 : (C % 4 == 0 ? 4 : 0);
    if (!V || (dzb && V != 8) || C > 4096 || rows * C >= (1LL << 31) || !al16(da) || (z && !al16(z)) ||
        (dz && !al16(dz)) || (dzb && !al16(dzb)) || (dp && (!al16(dp) || W < 2 || W % 2 || HW % W || (HW / W) % 2)))
        return cudaErrorNotSupported;
    const int G = C / V;
    const unsigned blocks = blocks_for_groups(rows * G, G);
    if (V == 8)
        bias_act_bwd_vec<8><<<blocks, 256, C * sizeof(float), s>>>(da, z, (int)rows, C, act, dz, db, dzb, HW, dp, W);
    else
        bias_act_bwd_vec<4><<<blocks, 256, C * sizeof(float), s>>>(da, z, (int)rows, C, act, dz, db, nullptr, HW, dp,
                                                                    W);
    return cudaGetLastError();
}

cudaError_t vec_avgpool2(const float *x, int N, int H, int W, int C, float *y, __half *yb, cudaStream_t s)
{
    if (C % 8 || (long long)N * H * W * C >= (1LL << 31) || !al16(x) || (y && !al16(y)) || (yb && !al16(yb)))
        return cudaErrorNotSupported;
    avgpool2_vec<<<blocks_for((long long)N * (H / 2) * (W / 2) * (C / 8)), 256, 0, s>>>(x, N, H, W, C, y, yb);
    return cudaGetLastError();
}

cudaError_t vec_avgpool2_bwd(const float *dy, int N, int H, int W, int C, float *dx, cudaStream_t s)
{
    if (C % 4 || (long long)N * H * W * C >= (1LL << 31) || !al16(dy) || !al16(dx)) return cudaErrorNotSupported;
    avgpool2_bwd_vec<<<blocks_for((long long)N * H * W * (C / 4)), 256, 0, s>>>(dy, N, H, W, C, dx);
    return cudaGetLastError();
}

cudaError_t vec_add(const float *a, const float *b, long long n, float *y, cudaStream_t s)
{
    if (n % 4 || n >= (1LL << 33) || !al16(a) || !al16(b) || !al16(y)) return cudaErrorNotSupported;
    add_vec<<<blocks_for(n / 4), 256, 0, s>>>(a, b, (int)(n / 4), y);
    return cudaGetLastError();
}

cudaError_t vec_upcat(const float *a, int N, int H, int W, int Ca, const float *b, int Cb, float *y, __half *yb,
                      cudaStream_t s)
{
    upcat_vec<<<blocks_for((long long)N * 4 * H * W * ((Ca + Cb) / 8)), 256, 0, s>>>(a, N, H, W, Ca, b, Cb, y, yb);
    return cudaGetLastError();
}

cudaError_t vec_upcat_bwd(const float *dy, int N, int H, int W, int Ca, int Cb, float *da, float *db, cudaStream_t s)
{
    const long long n = (da ? (long long)N * H * W * (Ca / 4) : 0) + (db ? (long long)N * 4 * H * W * (Cb / 4) : 0);
    if (n == 0) return cudaSuccess;
    upcat_bwd_vec<<<blocks_for(n), 256, 0, s>>>(dy, N, H, W, Ca, Cb, da, db);
    return cudaGetLastError();
}

cudaError_t small_conv1x1(const float *x, long long P, int C, const float *w, const float *bias, int cout, float *y,
                          cudaStream_t s)
{
    const unsigned blocks = blocks_for(P);
    const size_t sm = (size_t)cout * C * sizeof(float);
    switch (cout) {
    case 1: conv1x1_small<1><<<blocks, 256, sm, s>>>(x, (int)P, C, w, bias, y); break;
    case 2: conv1x1_small<2><<<blocks, 256, sm, s>>>(x, (int)P, C, w, bias, y); break;
    default: conv1x1_small<3><<<blocks, 256, sm, s>>>(x, (int)P, C, w, bias, y); break;
    }
    return cudaGetLastError();
}

cudaError_t small_conv1x1_bwd(const float *dy, const float *x, long long P, int C, const float *w, int cout, float *dx,
                              float *dw, float *db, cudaStream_t s)
{
    long long b = (P + 127) / 128;
    if (b > 152LL * 2) b = 152LL * 2;      // ~240 registers a thread: two blocks per SM, one wave
    const unsigned blocks = (unsigned)(b < 1 ? 1 : b);
    switch (cout) {
    case 1: conv1x1_small_bwd<1><<<blocks, 128, 0, s>>>(dy, x, (int)P, C, w, dx, dw, db); break;
    case 2: conv1x1_small_bwd<2><<<blocks, 128, 0, s>>>(dy, x, (int)P, C, w, dx, dw, db); break;
    default: conv1x1_small_bwd<3><<<blocks, 128, 0, s>>>(dy, x, (int)P, C, w, dx, dw, db); break;
    }
    return cudaGetLastError();
}

} // namespace smrt
