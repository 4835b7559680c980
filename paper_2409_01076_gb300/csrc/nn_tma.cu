// nn_tma.cu -- smrt_nn_conv3_tma and smrt_nn_pack3: a 3x3 convolution on the 5th-generation
// tensor cores whose operands arrive by TMA (cp.async.bulk.tensor), with the nine taps of the
// filter read as nine shifted views of ONE haloed input tile -- no im2col tile is ever written.
//
// Output tile of a CTA: 16 image rows x 8 pixels of one image (the GEMM's M = 128 rows; row m is
// pixel (y0 + m / 8, x0 + m % 8)) by TN output channels (TN = 32, 64 or 128).
//
// Input tile: the 18 x 10 window around it (one pixel of halo on every side).  Per group of 8
// input channels it is one "plane" [18 rows][10 pixels][8 halves] = 2,880 B in shared memory,
// written by one 4-D TMA load of the NHWC half activations with the box {8, 10, 18, 1} at
// (c, x0 - 1, y0 - 1, n); TMA fills the part outside the image with zeros, which is exactly the
// convolution's zero padding.  Planes are 2,944 B apart (a multiple of 128 B, as TMA wants).
//
// Why no im2col: 8 consecutive pixels of one plane row are 128 contiguous bytes -- one core
// matrix of the no-swizzle K-major operand layout (8 GEMM rows x 8 K halves).  So for tap
// (ky, kx) the GEMM's A operand (rows = the 128 output pixels, K = 16 input channels) is the
// shared-memory descriptor
//     start = plane(q) + (ky * 10 + kx) * 16 B,
//     leading byte offset (next 8 channels, K direction)    = plane stride  = 2,944 B,
//     stride byte offset  (next 8 pixels = next image row)  = 10 * 16 B     =   160 B.
// The weights come pre-packed by smrt_nn_pack3 so that one 3-D TMA load brings all nine taps of a
// 16-channel chunk in the matching K-major layout [9 taps x 2 groups][TN][8 halves].
//
// Pipeline (128 threads, roles in warp 0 and warp 1; the K loop runs over 16-channel chunks):
//   producer (warp 0, one lane): per chunk, wait until the stage is free, arm its "full"
//     mbarrier with the byte count and issue 3 TMA loads (two planes, one weight slab);
//   MMA issuer (warp 1, one lane): per chunk, wait for "full", issue nine tcgen05.mma
//     (M 128, N TN, K 16, half x half -> f32, accumulator in tensor memory), commit to the stage's
//     "empty" mbarrier; after the last chunk commit to "done";
//   epilogue (all 4 warps): wait for "done", tcgen05.ld the accumulator rows, y = alpha acc + beta y.
// Every mbarrier wait is bounded by 1 s of %globaltimer.  A wait that gives up sets *err and the
// CTA's failed flag, waits once more with the same bound (so no copy or MMA is left in flight
// where avoidable), skips the epilogue, and the CTA still releases its tensor memory.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include "internal.h"
#include "smrt_nn.h"

namespace {

constexpr int kTileRows = 16, kTilePx = 8;                 // output tile: 16 rows x 8 pixels
constexpr int kHaloRows = kTileRows + 2, kHaloPx = kTilePx + 2;
constexpr int kChunk = 16;                                 // input channels per pipeline stage
constexpr int kPlaneBytes = kHaloRows * kHaloPx * 16;      // 2,880 B written by one TMA
constexpr int kPlaneStride = 2944;                         // 23 x 128 B
constexpr int kASlab = 2 * kPlaneStride;                   // two planes per 16-channel chunk
constexpr int kMaxStages = 4;
constexpr unsigned long long kWaitNs = 1000000000ull;      // a wait gives up after 1 s (%globaltimer)

static_assert(kPlaneStride >= kPlaneBytes && kPlaneStride % 128 == 0, "plane stride");
static_assert(kTileRows * kTilePx == 128, "M = 128");

template <int TN>
constexpr int stage_bytes()
{
    // A: two planes; B: 18 slabs of TN rows x 16 B; rounded up to 1 KB
    return ((kASlab + 18 * TN * 16) + 1023) / 1024 * 1024;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory matrix descriptor, no swizzle, version 1.
__device__ __forceinline__ unsigned long long desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((saddr & 0x3FFFF) >> 4);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFF) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFF) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor of kind::f16: D f32, A and B half, both K-major, N = TN, M = 128.
template <int TN>
__host__ __device__ constexpr uint32_t idesc()
{
    return (1u << 4) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of parity `parity` of mbarrier `mb`; false after kWaitNs without it.
__device__ __forceinline__ bool wait_parity(uint32_t mb, uint32_t parity)
{
    const unsigned long long t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(mb), "r"(parity) : "memory");
        if (done) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}

// A bounded wait that records a failure and then waits once more (also bounded).
__device__ __forceinline__ bool wait_or_fail(uint32_t mb, uint32_t parity, int *failed, int *err)
{
    if (wait_parity(mb, parity)) return true;
    *failed = 1;
    if (err) atomicExch(err, 1);
    wait_parity(mb, parity);
    return false;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t mbar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3, %4, %5}], [%6];"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint32_t mbar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3, %4}], [%5];"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
                 : "memory");
}

template <int TN>
__global__ void __launch_bounds__(128)
conv3_tma_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmw, int H, int W,
                 int C, int cout, int ntn, int nstages, float alpha, float beta, float *y, int ldy, int vec_y,
                 int *err)
{
    extern __shared__ unsigned char dyn_raw[];
    __shared__ __align__(8) unsigned long long full[kMaxStages], empty[kMaxStages], done;
    __shared__ uint32_t tmem_holder;
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * kTilePx, y0 = blockIdx.y * kTileRows;
    const int img = blockIdx.z / ntn, n0 = (blockIdx.z % ntn) * TN;
    const int nchunks = C / kChunk;
    constexpr int kSB = stage_bytes<TN>();
    constexpr uint32_t kTx = 2 * kPlaneBytes + 18 * TN * 16;      // bytes the 3 loads of a stage bring
    const uint32_t base = (smem_u32(dyn_raw) + 1023u) & ~1023u;   // 1 KB aligned stage 0

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_holder)), "r"((uint32_t)TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 32) {
        for (int s = 0; s < nstages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&done)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;

    if (warp == 0 && lane == 0) {
        // producer
        asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&tmx)) : "memory");
        asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&tmw)) : "memory");
        for (int i = 0; i < nchunks; ++i) {
            const int s = i % nstages;
            if (i >= nstages && !wait_or_fail(smem_u32(&empty[s]), (uint32_t)((i / nstages - 1) & 1), &failed, err))
                break;
            const uint32_t st = base + (uint32_t)(s * kSB), fb = smem_u32(&full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(fb), "r"(kTx) : "memory");
            tma_load_4d(st, &tmx, i * kChunk, x0 - 1, y0 - 1, img, fb);
            tma_load_4d(st + kPlaneStride, &tmx, i * kChunk + 8, x0 - 1, y0 - 1, img, fb);
            tma_load_3d(st + kASlab, &tmw, 0, n0, i * 18, fb);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int i = 0; i < nchunks; ++i) {
            const int s = i % nstages;
            if (!wait_or_fail(smem_u32(&full[s]), (uint32_t)((i / nstages) & 1), &failed, err)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t st = base + (uint32_t)(s * kSB);
            #pragma unroll
            for (int t = 0; t < 9; ++t) {
                const int ky = t / 3, kx = t % 3;
                const unsigned long long ad = desc(st + (uint32_t)((ky * kHaloPx + kx) * 16), kPlaneStride,
                                                   kHaloPx * 16);
                const unsigned long long bd = desc(st + kASlab + (uint32_t)(2 * t * TN * 16), TN * 16, 128);
                const uint32_t acc = (i > 0 || t > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                             :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc<TN>()), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&empty[s])) : "memory");
        }
        // covers every MMA this thread issued, also after a failure
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(smem_u32(&done)) : "memory");
    }
    __syncwarp();
    wait_or_fail(smem_u32(&done), 0u, &failed, err);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");

    if (!failed) {
        const int m = warp * 32 + lane;
        const int yy = y0 + (m >> 3), xx = x0 + (m & 7);
        const bool valid = yy < H && xx < W;
        float *yrow = y + ((size_t)((size_t)img * H + (valid ? yy : 0)) * W + (valid ? xx : 0)) * ldy;
        #pragma unroll 1
        for (int c = 0; c < TN; c += 32) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                         "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                         "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                           "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                           "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (!valid) continue;
            const int col0 = n0 + c;
            if (vec_y && col0 + 32 <= cout) {
                #pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    float4 v = make_float4(alpha * __uint_as_float(r[j]), alpha * __uint_as_float(r[j + 1]),
                                           alpha * __uint_as_float(r[j + 2]), alpha * __uint_as_float(r[j + 3]));
                    float4 *p = reinterpret_cast<float4 *>(yrow + col0 + j);
                    if (beta != 0.0f) {
                        const float4 o = *p;
                        v.x += beta * o.x; v.y += beta * o.y; v.z += beta * o.z; v.w += beta * o.w;
                    }
                    *p = v;
                }
            } else {
                #pragma unroll
                for (int j = 0; j < 32; ++j) {
                    if (col0 + j >= cout) break;
                    float *p = yrow + col0 + j;
                    const float v = alpha * __uint_as_float(r[j]);
                    *p = (beta != 0.0f) ? v + beta * *p : v;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"((uint32_t)TN));
}

// wp[((chunk * 9 + tap) * 2 + q) * cout * 8 + o * 8 + e] = w[o * 9C + tap * C + chunk * 16 + q * 8 + e]
__global__ void pack3_kernel(const __half *__restrict__ w, int cout, int C, __half *__restrict__ wp)
{
    const long long total = 9LL * C * cout;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(i & 7);
        const long long r = i >> 3;
        const int o = (int)(r % cout);
        const int kg = (int)(r / cout);              // (chunk * 9 + tap) * 2 + q
        const int q = kg & 1, ct = kg >> 1, tap = ct % 9, chunk = ct / 9;
        wp[i] = w[(size_t)o * 9 * C + (size_t)tap * C + chunk * kChunk + q * 8 + e];
    }
}

int tma_fail(int code, const char *fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    smrt::set_thread_error(buf);
    return code;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (the library links no libcuda).
EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

template <int TN>
cudaError_t launch_conv3_tma(const CUtensorMap &tmx, const CUtensorMap &tmw, int N, int H, int W, int C, int cout,
                             float alpha, float beta, float *y, int ldy, int *err, cudaStream_t s)
{
    const int ntn = (cout + TN - 1) / TN;
    const int nchunks = C / kChunk;
    const int nstages = nchunks < kMaxStages ? nchunks : kMaxStages;
    // shared memory also caps the CTAs per SM so that their accumulators fit in the 512 TMEM
    // columns: with 128 columns each, at most 4 CTAs may be resident, so reserve >= 2 stages
    const int reserve = (TN == 128 && nstages < 2) ? 2 : nstages;
    const size_t smem = (size_t)reserve * stage_bytes<TN>() + 1024;
    dim3 grid((W + kTilePx - 1) / kTilePx, (H + kTileRows - 1) / kTileRows, N * ntn);
    const int vec_y = (ldy % 4 == 0) && ((reinterpret_cast<uintptr_t>(y) & 15) == 0);
    static bool attr_set = false;       // per instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(conv3_tma_kernel<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(kMaxStages * stage_bytes<TN>() + 1024));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    conv3_tma_kernel<TN><<<grid, 128, smem, s>>>(tmx, tmw, H, W, C, cout, ntn, nstages, alpha, beta, y, ldy, vec_y,
                                                 err);
    return cudaGetLastError();
}

} // namespace

extern "C" int smrt_nn_pack3(const void *w, int cout, int C, void *wp, void *stream)
{
    if (!w || !wp || cout < 1 || C < kChunk || C % kChunk != 0 || 9LL * C * cout > 0x7fffffffLL)
        return tma_fail(SMRT_ERR_ARG, "smrt_nn_pack3: bad arguments (cout %d C %d; C must be a multiple of 16)", cout,
                        C);
    const long long total = 9LL * C * cout;
    const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    pack3_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>((const __half *)w, cout, C, (__half *)wp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_pack3: %s", cudaGetErrorString(e));
    return SMRT_OK;
}

extern "C" int smrt_nn_conv3_tma(const void *xh, int N, int H, int W, int C, const void *wp, int cout, float alpha,
                                 float beta, float *y, int ldy, int *err, void *stream)
{
    if (!xh || !wp || !y || N < 1 || H < 1 || W < 1 || C < kChunk || C % kChunk != 0 || cout < 1 || ldy < cout ||
        (reinterpret_cast<uintptr_t>(xh) & 15) != 0 || (reinterpret_cast<uintptr_t>(wp) & 15) != 0 ||
        (H + kTileRows - 1) / kTileRows > 65535 || (long long)N * H * W * C > (1LL << 40) || 9LL * C > 0x7fffffffLL)
        return tma_fail(SMRT_ERR_ARG,
                        "smrt_nn_conv3_tma: bad arguments (N %d H %d W %d C %d cout %d ldy %d; C must be a multiple "
                        "of 16, xh and wp 16-byte aligned)", N, H, W, C, cout, ldy);
    const int TN = cout <= 32 ? 32 : cout <= 64 ? 64 : 128;
    if ((long long)N * ((cout + TN - 1) / TN) > 65535)
        return tma_fail(SMRT_ERR_ARG, "smrt_nn_conv3_tma: N x output-channel tiles exceeds the grid (N %d cout %d)", N,
                        cout);
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_conv3_tma: cuTensorMapEncodeTiled is not available");

    // activations: (C, W, H, N) halves, box 8 channels x 10 pixels x 18 rows x 1 image
    CUtensorMap tmx, tmw;
    const cuuint64_t xdim[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t xstr[3] = {2ull * C, 2ull * C * W, 2ull * C * W * H};
    const cuuint32_t xbox[4] = {8, (cuuint32_t)kHaloPx, (cuuint32_t)kHaloRows, 1};
    const cuuint32_t ones[4] = {1, 1, 1, 1};
    CUresult r = enc(&tmx, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, const_cast<void *>(xh), xdim, xstr, xbox, ones,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return tma_fail(SMRT_ERR_CUDA, "smrt_nn_conv3_tma: activation tensor map rejected (%d)", (int)r);
    // packed weights: (8, cout, 9C/8) halves, box 8 x TN x 18 (all nine taps of one 16-channel chunk)
    const cuuint64_t wdim[3] = {8, (cuuint64_t)cout, (cuuint64_t)(9 * C / 8)};
    const cuuint64_t wstr[2] = {16, 16ull * cout};
    const cuuint32_t wbox[3] = {8, (cuuint32_t)TN, 18};
    r = enc(&tmw, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void *>(wp), wdim, wstr, wbox, ones,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return tma_fail(SMRT_ERR_CUDA, "smrt_nn_conv3_tma: weight tensor map rejected (%d)", (int)r);

    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (TN == 32) e = launch_conv3_tma<32>(tmx, tmw, N, H, W, C, cout, alpha, beta, y, ldy, err, s);
    else if (TN == 64) e = launch_conv3_tma<64>(tmx, tmw, N, H, W, C, cout, alpha, beta, y, ldy, err, s);
    else e = launch_conv3_tma<128>(tmx, tmw, N, H, W, C, cout, alpha, beta, y, ldy, err, s);
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_conv3_tma: %s", cudaGetErrorString(e));
    return SMRT_OK;
}
