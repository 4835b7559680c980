// nn_tma.cu -- 3x3 convolutions on the 5th-generation tensor cores with operands delivered by TMA
// (cp.async.bulk.tensor / cp.async.bulk), where the nine taps of the filter are nine shifted views
// of ONE haloed input tile in shared memory: no im2col matrix or tile is ever written.
//
//   smrt_nn_to_half_blocked     float32 NHWC -> half, channel-group-blocked [N][C/8][H][W][8]
//   smrt_nn_to_half_blocked_pad the same, zero-padded to more channels (a narrow input layer)
//   smrt_nn_pack3               3x3 weights -> [n-block][16-channel chunk][9 taps x 2 groups][TN][8]
//   smrt_nn_pad3 / _unpad3_add  3x3 weights zero-padded to more input channels / gradient folded back
//   smrt_nn_conv3_tma           y = conv3x3(x, w)  (forward; input gradient with flipped w)
//   smrt_nn_conv3_tma_bias_act  the same with bias + SiLU in the epilogue (z, a, blocked a)
//   smrt_nn_conv3_wgrad_tma     dW += sum_pixels x(shifted) dz  (weight gradient; for 16 or 32 input
//                               channels the taps are grouped along the MMA rows)
//
// Blocked activations.  In [N][C/8][H][W][8] one image row of one 8-channel group is W * 16
// contiguous bytes, so a TMA box over the 4-D view (8W halves, H, C/8, N) brings 18 halo rows of
// 10 pixels x 8 channels as 18 runs of 160 B (an NHWC box would need 180 runs of 16 B).  A box
// starting at x = 8 (x0 - 1) is 16-byte aligned, and TMA fills everything outside the image with
// zeros -- exactly the convolution's zero padding.
//
// Tiles.  An output tile is 16 image rows x 8 pixels (the GEMM's 128 rows; row m is pixel
// (y0 + m / 8, x0 + m % 8)).  Its input window is 18 x 10 pixels, stored per 8-channel group as a
// "plane" [18 rows][10 px][8 halves] of 2,880 B.  Eight consecutive pixels of a plane row are 128
// contiguous bytes: one core matrix of the no-swizzle operand layouts.  Hence, for tap (ky, kx):
//   forward (K = channels, K-major A): start = plane(q) + (ky*10 + kx)*16 B, leading byte offset
//     (next 8 channels) = 2,880 B, stride byte offset (next 8 pixels = next image row) = 160 B;
//   weight gradient (K = pixels, MN-major A with M = channels): start = plane(0) +
//     ((2j + ky)*10 + kx)*16 B for pixel rows 2j, 2j+1, leading byte offset (next 8 pixels = next
//     image row) = 160 B, stride byte offset (next 8 channels) = 2,880 B.
//
// Pipelines.  128 threads; lane 0 of warp 0 is the TMA producer, lane 0 of warp 1 issues the
// tcgen05.mma (half x half -> float32, accumulator in tensor memory), all four warps run the
// tcgen05.ld epilogue.  Stages are tracked by "full" (TMA transaction bytes) and "empty"
// (tcgen05.commit) mbarriers; a final commit to "done" releases the epilogue.  Every wait is
// bounded by 1 s of %globaltimer: a wait that gives up sets *err and the CTA's failed flag, waits
// once more with the same bound (so no copy or MMA is left in flight where avoidable), skips the
// epilogue, and the CTA still releases its tensor memory.
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
constexpr int kChunk = 16;                                 // input channels per forward stage
constexpr int kPlane = kHaloRows * kHaloPx * 16;           // 2,880 B: one halo plane
constexpr int kDzPlane = kTileRows * kTilePx * 16;         // 2,048 B: one 8-channel plane of dz
constexpr int kFwdStages = 4;
constexpr int kWgStages = 6;
constexpr int kWgTN = 32;                                  // output channels per weight-gradient CTA
constexpr int kWgPlanes = 16;                              // input channels per weight-gradient CTA / 8
constexpr unsigned long long kWaitNs = 1000000000ull;      // a wait gives up after 1 s (%globaltimer)

static_assert(kTileRows * kTilePx == 128, "M = 128");

int tile_n(int cout) { return cout <= 32 ? 32 : cout <= 64 ? 64 : 128; }

// Fused epilogues.  on == 1, forward: v = acc + bias[o]; z = v; a = SiLU(v) (or v); ab = half(a) in the
// blocked layout (any of z, a, ab may be null).  on == 2, the input gradient of a convolution B whose
// input is the activation of a convolution A (pre-activation zin, cout channels): d = acc * SiLU'(zin)
// (or acc), z = d (fp32, may be null), ab = half(d) blocked, db[o] += sum over pixels of d (may be null).
// cout % 8 == 0.
struct Epi {
    const float *bias;
    float *z, *a;
    __half *ab;
    int act, on;
    const float *zin;
    float *db;
};

// Warp reduce-scatter of 32 values per lane: afterwards v[0] of lane l is the sum over the warp's lanes
// of their v[l].  Each of the five steps keeps half of a lane's values and adds its partner's matching
// half (31 shuffles).
__device__ __forceinline__ float warp_reduce_scatter32(float v[32], int lane)
{
    #pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool upper = (lane & w) != 0;
        #pragma unroll
        for (int k = 0; k < w; ++k) {
            const float send = upper ? v[k] : v[k + w];
            const float keep = upper ? v[k + w] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return v[0];
}

__device__ __forceinline__ float sigm(float v) { return 1.0f / (1.0f + expf(-v)); }

// MT output tiles stacked along y share one halo window per 8-channel plane: (16 MT + 2) rows x 10
// pixels x 16 B, and every stage's weights.
template <int MT>
constexpr int fwd_plane_bytes() { return (kTileRows * MT + 2) * kHaloPx * 16; }
template <int MT>
constexpr int fwd_a_bytes() { return (2 * fwd_plane_bytes<MT>() + 127) / 128 * 128; }   // 5,760 B for MT = 1
template <int TN, int MT = 1>
constexpr int fwd_stage_bytes()
{
    // A: two planes (rounded up to 128 B); B: 18 slabs of TN rows x 16 B; rounded up to 1 KB
    return (fwd_a_bytes<MT>() + 18 * TN * 16 + 1023) / 1024 * 1024;
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

// Instruction descriptor of kind::f16: D f32, A and B half, M = 128, N = TN; mn: both operands
// MN-major (bits 15 and 16), else both K-major.
template <int TN, bool MN>
__host__ __device__ constexpr uint32_t idesc()
{
    return (1u << 4) | (MN ? (1u << 15) | (1u << 16) : 0u) | ((uint32_t)(TN >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of parity `parity` of mbarrier `mb`; false after limit_ns without it.
__device__ __forceinline__ bool wait_parity(uint32_t mb, uint32_t parity, unsigned long long limit_ns)
{
    const unsigned long long t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(mb), "r"(parity) : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// A bounded wait that records a failure and then waits once more (also bounded).
__device__ __forceinline__ bool wait_or_fail(uint32_t mb, uint32_t parity, int *failed, int *err,
                                             unsigned long long limit_ns = kWaitNs)
{
    if (wait_parity(mb, parity, limit_ns)) return true;
    *failed = 1;
    if (err) atomicExch(err, 1);
    wait_parity(mb, parity, limit_ns);
    return false;
}

__device__ __forceinline__ void expect_tx(uint32_t mb, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mb), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t mbar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3, %4, %5}], [%6];"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
                 : "memory");
}

// Contiguous global -> shared copy (16-byte aligned ends, size a multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(mbar) : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, unsigned long long ad, unsigned long long bd, uint32_t id,
                                        uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(tmem), "l"(ad), "l"(bd), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t mb)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mb)
                 : "memory");
}

// 32 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t r[32])
{
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
}

// Shared prologue: TMEM allocation by warp 0, barrier initialisation by thread 32.
template <uint32_t COLS>
__device__ __forceinline__ uint32_t setup(uint32_t *tmem_holder, unsigned long long *full, unsigned long long *empty,
                                          unsigned long long *done, int nstages, int *failed)
{
    const int tid = threadIdx.x;
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_holder)), "r"(COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 32) {
        for (int s = 0; s < nstages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(done)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *failed = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    return *tmem_holder;
}

template <uint32_t COLS>
__device__ __forceinline__ void teardown(uint32_t tmem)
{
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(COLS));
}

// Epilogue of accumulator columns c .. c + 31 of output-channel block n0 for one pixel (yy, xx) of
// image img (one TMEM lane): plain y = alpha acc + beta y (on == 0), bias + SiLU (on == 1) or the
// SiLU backward with the bias-gradient sums into sdb (on == 2; every lane of the warp takes part).
template <int TN>
__device__ __forceinline__ void epi_store32(const uint32_t r[32], int c, int n0, int cout, bool valid, int img,
                                            int H, int W, int yy, int xx, size_t pix, float alpha, float beta,
                                            float *yrow, int vec_y, const Epi &epi, float *sdb, int lane)
{
    const int col0 = n0 + c;
    if (epi.on == 2) {
        float v[32];
        #pragma unroll
        for (int j = 0; j < 32; j += 8) {
            const bool ok = valid && col0 + j < cout;
            #pragma unroll
            for (int e = 0; e < 8; ++e) v[j + e] = ok ? __uint_as_float(r[j + e]) : 0.0f;
            if (!ok) continue;
            if (epi.act) {
                const float4 *zq = reinterpret_cast<const float4 *>(epi.zin + pix * cout + col0 + j);
                const float4 z0 = zq[0], z1 = zq[1];
                const float zz[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
                #pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float sg = sigm(zz[e]);
                    v[j + e] *= sg * (1.0f + zz[e] * (1.0f - sg));
                }
            }
            if (epi.z) {
                float4 *q = reinterpret_cast<float4 *>(epi.z + pix * cout + col0 + j);
                q[0] = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                q[1] = make_float4(v[j + 4], v[j + 5], v[j + 6], v[j + 7]);
            }
            __half2 h[4];
            #pragma unroll
            for (int e = 0; e < 4; ++e) h[e] = __floats2half2_rn(v[j + 2 * e], v[j + 2 * e + 1]);
            const size_t g = (size_t)(col0 + j) / 8, G = (size_t)cout / 8;
            *reinterpret_cast<uint4 *>(epi.ab + (((size_t)img * G + g) * H * W + (size_t)yy * W + xx) * 8) =
                *reinterpret_cast<uint4 *>(h);
        }
        if (epi.db) {
            const float sum = warp_reduce_scatter32(v, lane);
            atomicAdd(&sdb[c + lane], sum);
        }
        return;
    }
    if (!valid) return;
    if (epi.on) {
        #pragma unroll
        for (int j = 0; j < 32; j += 8) {
            if (col0 + j >= cout) break;
            float v[8];
            #pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(r[j + e]) + epi.bias[col0 + j + e];
            if (epi.z) {
                float4 *q = reinterpret_cast<float4 *>(epi.z + pix * cout + col0 + j);
                q[0] = make_float4(v[0], v[1], v[2], v[3]);
                q[1] = make_float4(v[4], v[5], v[6], v[7]);
            }
            if (epi.act) {
                #pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = v[e] * sigm(v[e]);
            }
            if (epi.a) {
                float4 *q = reinterpret_cast<float4 *>(epi.a + pix * cout + col0 + j);
                q[0] = make_float4(v[0], v[1], v[2], v[3]);
                q[1] = make_float4(v[4], v[5], v[6], v[7]);
            }
            if (epi.ab) {
                __half2 h[4];
                #pragma unroll
                for (int e = 0; e < 4; ++e) h[e] = __floats2half2_rn(v[2 * e], v[2 * e + 1]);
                const size_t g = (size_t)(col0 + j) / 8, G = (size_t)cout / 8;
                *reinterpret_cast<uint4 *>(epi.ab + (((size_t)img * G + g) * H * W + (size_t)yy * W + xx) * 8) =
                    *reinterpret_cast<uint4 *>(h);
            }
        }
        return;
    }
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

// ---- forward -------------------------------------------------------------------------------
// grid (tiles in x, groups of MT tiles in y, N * output-channel blocks); wp points at this launch's
// packed weights: block nb, chunk i is the 18 * TN * 8 halves at ((nb * nchunks + i) * 18 * TN * 8).
// MT = 2: the CTA computes two 16 x 8 tiles stacked along y (accumulators at TMEM columns 0 and TN)
// from one 34-row halo window, so each stage's weights serve twice the pixels.
template <int TN, int MT>
__global__ void __launch_bounds__(128)
conv3_tma_kernel(const __grid_constant__ CUtensorMap tmx, const __half *__restrict__ wp, int H, int W, int C,
                 int cout, int ntn, int nstages, float alpha, float beta, float *y, int ldy, int vec_y, int *err,
                 Epi epi, unsigned long long wait_ns, int withhold)
{
    extern __shared__ unsigned char dyn_raw[];
    __shared__ __align__(8) unsigned long long full[kFwdStages], empty[kFwdStages], done;
    __shared__ uint32_t tmem_holder;
    __shared__ int failed;
    __shared__ float sdb[TN];                                   // on == 2: this tile's bias-gradient sums

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * kTilePx, y0 = blockIdx.y * kTileRows * MT;
    if (epi.on == 2 && threadIdx.x < TN) sdb[threadIdx.x] = 0.0f;
    const int img = blockIdx.z / ntn, nb = blockIdx.z % ntn, n0 = nb * TN;
    const int nchunks = C / kChunk;
    constexpr int kSB = fwd_stage_bytes<TN, MT>();
    constexpr int kPl = fwd_plane_bytes<MT>();
    constexpr int kA = fwd_a_bytes<MT>();
    constexpr uint32_t kTx = 2 * kPl + 18 * TN * 16;          // bytes the two copies of a stage bring
    const uint32_t base = (smem_u32(dyn_raw) + 1023u) & ~1023u;

    const uint32_t tmem = setup<TN * MT>(&tmem_holder, full, empty, &done, nstages, &failed);

    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&tmx)) : "memory");
        const __half *wblk = wp + (size_t)nb * nchunks * 18 * TN * 8;
        // withhold (failure-path test only): the producer issues nothing, so no copy is ever in flight
        for (int i = 0; i < (withhold ? 0 : nchunks); ++i) {
            const int s = i % nstages;
            if (i >= nstages &&
                !wait_or_fail(smem_u32(&empty[s]), (uint32_t)((i / nstages - 1) & 1), &failed, err, wait_ns))
                break;
            const uint32_t st = base + (uint32_t)(s * kSB), fb = smem_u32(&full[s]);
            expect_tx(fb, kTx);
            tma_load_4d(st, &tmx, 8 * (x0 - 1), y0 - 1, 2 * i, img, fb);       // planes 2i, 2i + 1
            bulk_load(st + kA, wblk + (size_t)i * 18 * TN * 8, 18 * TN * 16, fb);
        }
    } else if (warp == 1 && lane == 0) {
        for (int i = 0; i < nchunks; ++i) {
            const int s = i % nstages;
            if (!wait_or_fail(smem_u32(&full[s]), (uint32_t)((i / nstages) & 1), &failed, err, wait_ns)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t st = base + (uint32_t)(s * kSB);
            #pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                #pragma unroll
                for (int t = 0; t < 9; ++t) {
                    const int ky = t / 3 + kTileRows * mt, kx = t % 3;
                    mma_f16(tmem + (uint32_t)(mt * TN), desc(st + (uint32_t)((ky * kHaloPx + kx) * 16), kPl, kHaloPx * 16),
                            desc(st + kA + (uint32_t)(2 * t * TN * 16), TN * 16, 128), idesc<TN, false>(),
                            (i > 0 || t > 0) ? 1u : 0u);
                }
            }
            commit(smem_u32(&empty[s]));
        }
        commit(smem_u32(&done));    // covers every MMA this thread issued, also after a failure
    }
    __syncwarp();
    wait_or_fail(smem_u32(&done), 0u, &failed, err, wait_ns);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");

    #pragma unroll 1
    for (int mt = 0; mt < (failed ? 0 : MT); ++mt) {
        const int m = warp * 32 + lane;
        const int yy = y0 + kTileRows * mt + (m >> 3), xx = x0 + (m & 7);
        const bool valid = yy < H && xx < W;
        const size_t pix = (size_t)((size_t)img * H + (valid ? yy : 0)) * W + (valid ? xx : 0);
        float *yrow = epi.on ? nullptr : y + pix * ldy;
        #pragma unroll 1
        for (int c = 0; c < TN; c += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * TN + c), r);
            epi_store32<TN>(r, c, n0, cout, valid, img, H, W, yy, xx, pix, alpha, beta, yrow, vec_y, epi, sdb, lane);
        }
    }
    if (epi.on == 2 && epi.db && !failed) {
        __syncthreads();                                        // every warp's sums are in sdb
        if (threadIdx.x < TN && n0 + (int)threadIdx.x < cout) atomicAdd(epi.db + n0 + threadIdx.x, sdb[threadIdx.x]);
    }
    teardown<TN * MT>(tmem);
}

// ---- weight gradient -------------------------------------------------------------------------
// grid (input-channel blocks of 128 x output-channel blocks of 32, pixel-tile splits).  A CTA
// accumulates D_t[c][o] = sum over its pixel tiles of x(p + tap t)[c] dz(p)[o] for all nine taps
// (9 x 32 TMEM columns), then adds alpha D_t into gw[o][t*C + c] with float32 atomics.
__global__ void __launch_bounds__(128)
conv3_wgrad_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmz, int H, int W,
                   int C, int cout, int tiles_x, int tiles_y, int ntiles, int nbk, int per, int planes, int nstages,
                   int stage_bytes, float alpha, float *gw, int ldg, int *err)
{
    extern __shared__ unsigned char dyn_raw[];
    __shared__ __align__(8) unsigned long long full[kWgStages], empty[kWgStages], done;
    __shared__ uint32_t tmem_holder;
    __shared__ int failed;
    constexpr uint32_t kCols = 512;         // 9 taps x 32 columns, rounded up to a power of two

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mb = blockIdx.x / nbk, nb = blockIdx.x % nbk;
    const int t_beg = blockIdx.y * per;
    const int t_end = min(ntiles, t_beg + per);
    if (t_beg >= t_end) return;             // uniform over the CTA
    const int a_bytes = (planes * kPlane + 127) / 128 * 128;
    const uint32_t tx = (uint32_t)(planes * kPlane + 4 * kDzPlane);
    const uint32_t base = (smem_u32(dyn_raw) + 1023u) & ~1023u;

    const uint32_t tmem = setup<kCols>(&tmem_holder, full, empty, &done, nstages, &failed);
    const int n_it = t_end - t_beg;

    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&tmx)) : "memory");
        asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&tmz)) : "memory");
        for (int it = 0; it < n_it; ++it) {
            const int s = it % nstages;
            if (it >= nstages && !wait_or_fail(smem_u32(&empty[s]), (uint32_t)((it / nstages - 1) & 1), &failed, err))
                break;
            const int t = t_beg + it, per_img = tiles_x * tiles_y;
            const int img = t / per_img, rem = t - img * per_img;
            const int x0 = (rem % tiles_x) * kTilePx, y0 = (rem / tiles_x) * kTileRows;
            const uint32_t st = base + (uint32_t)(s * stage_bytes), fb = smem_u32(&full[s]);
            expect_tx(fb, tx);
            tma_load_4d(st, &tmx, 8 * (x0 - 1), y0 - 1, kWgPlanes * mb, img, fb);
            tma_load_4d(st + a_bytes, &tmz, 8 * x0, y0, 4 * nb, img, fb);
        }
    } else if (warp == 1 && lane == 0) {
        for (int it = 0; it < n_it; ++it) {
            const int s = it % nstages;
            if (!wait_or_fail(smem_u32(&full[s]), (uint32_t)((it / nstages) & 1), &failed, err)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t st = base + (uint32_t)(s * stage_bytes);
            #pragma unroll 1
            for (int t = 0; t < 9; ++t) {
                const int ky = t / 3, kx = t % 3;
                #pragma unroll
                for (int j = 0; j < kTileRows / 2; ++j) {        // K = 16 pixels: image rows 2j, 2j + 1
                    mma_f16(tmem + (uint32_t)(t * kWgTN),
                            desc(st + (uint32_t)(((2 * j + ky) * kHaloPx + kx) * 16), kHaloPx * 16, kPlane),
                            desc(st + (uint32_t)a_bytes + (uint32_t)(2 * j * 128), 128, kDzPlane),
                            idesc<kWgTN, true>(), (it > 0 || j > 0) ? 1u : 0u);
                }
            }
            commit(smem_u32(&empty[s]));
        }
        commit(smem_u32(&done));
    }
    __syncwarp();
    wait_or_fail(smem_u32(&done), 0u, &failed, err);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");

    if (!failed) {
        const int c = kWgPlanes * 8 * mb + warp * 32 + lane;
        #pragma unroll 1
        for (int t = 0; t < 9; ++t) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * kWgTN), r);
            if (c >= C) continue;
            float *g = gw + (size_t)t * C + c;
            #pragma unroll
            for (int j = 0; j < kWgTN; ++j) {
                const int o = kWgTN * nb + j;
                if (o < cout) atomicAdd(g + (size_t)o * ldg, alpha * __uint_as_float(r[j]));
            }
        }
    }
    teardown<kCols>(tmem);
}

// ---- weight gradient of narrow layers (C = 16 or 32): taps grouped along M --------------------
// With C < 128 most of the 128 MMA rows of conv3_wgrad_kernel would be padding.  Here each tile
// loads its nine tap-shifted 16 x 8 windows (box {64, 16, C/8, 1} at (x0 + kx - 1, y0 + ky - 1)) into
// nine consecutive slots of (C/8) x 2,048 B, so T = 128 / C consecutive taps form one MN-major operand
// of 128 rows = (tap, channel): start = slot(g T) + 2j x 128 B, leading byte offset 128 B (next image
// row), stride byte offset 2,048 B (next 8 channels, continuing into the next tap's slot).  ceil(9 / T)
// groups of eight K = 16 MMAs per tile instead of nine; the rows of a last group's missing taps read
// whatever follows the ninth slot and are never stored.
template <int C>
__global__ void __launch_bounds__(128)
conv3_wgrad_grouped_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmz, int H,
                           int W, int cout, int tiles_x, int tiles_y, int ntiles, int nbk, int per, int nstages,
                           int stage_bytes, float alpha, float *gw, int ldg, int *err)
{
    constexpr int T = 128 / C, NG = (9 + T - 1) / T, SLOT = (C / 8) * kDzPlane;
    constexpr uint32_t kCols = NG * kWgTN <= 64 ? 64 : 128;
    static_assert(NG * kWgTN <= 128 && 128 % C == 0, "narrow channel counts only");
    extern __shared__ unsigned char dyn_raw[];
    __shared__ __align__(8) unsigned long long full[kWgStages], empty[kWgStages], done;
    __shared__ uint32_t tmem_holder;
    __shared__ int failed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = blockIdx.x % nbk;
    const int t_beg = blockIdx.y * per;
    const int t_end = min(ntiles, t_beg + per);
    if (t_beg >= t_end) return;             // uniform over the CTA
    constexpr uint32_t kTx = 9 * SLOT + 4 * kDzPlane;
    const uint32_t base = (smem_u32(dyn_raw) + 1023u) & ~1023u;
    const uint32_t tmem = setup<kCols>(&tmem_holder, full, empty, &done, nstages, &failed);
    const int n_it = t_end - t_beg;

    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&tmx)) : "memory");
        asm volatile("prefetch.tensormap [%0];" :: "l"(reinterpret_cast<uint64_t>(&tmz)) : "memory");
        for (int it = 0; it < n_it; ++it) {
            const int s = it % nstages;
            if (it >= nstages && !wait_or_fail(smem_u32(&empty[s]), (uint32_t)((it / nstages - 1) & 1), &failed, err))
                break;
            const int t = t_beg + it, per_img = tiles_x * tiles_y;
            const int img = t / per_img, rem = t - img * per_img;
            const int x0 = (rem % tiles_x) * kTilePx, y0 = (rem / tiles_x) * kTileRows;
            const uint32_t st = base + (uint32_t)(s * stage_bytes), fb = smem_u32(&full[s]);
            expect_tx(fb, kTx);
            #pragma unroll 1
            for (int tap = 0; tap < 9; ++tap)
                tma_load_4d(st + (uint32_t)(tap * SLOT), &tmx, 8 * (x0 + tap % 3 - 1), y0 + tap / 3 - 1, 0, img, fb);
            tma_load_4d(st + 9u * SLOT, &tmz, 8 * x0, y0, 4 * nb, img, fb);
        }
    } else if (warp == 1 && lane == 0) {
        for (int it = 0; it < n_it; ++it) {
            const int s = it % nstages;
            if (!wait_or_fail(smem_u32(&full[s]), (uint32_t)((it / nstages) & 1), &failed, err)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t st = base + (uint32_t)(s * stage_bytes);
            #pragma unroll
            for (int g = 0; g < NG; ++g) {
                #pragma unroll
                for (int j = 0; j < kTileRows / 2; ++j)        // K = 16 pixels: image rows 2j, 2j + 1
                    mma_f16(tmem + (uint32_t)(g * kWgTN),
                            desc(st + (uint32_t)(g * T * SLOT + 2 * j * 128), 128, kDzPlane),
                            desc(st + 9u * SLOT + (uint32_t)(2 * j * 128), 128, kDzPlane),
                            idesc<kWgTN, true>(), (it > 0 || j > 0) ? 1u : 0u);
            }
            commit(smem_u32(&empty[s]));
        }
        commit(smem_u32(&done));
    }
    __syncwarp();
    wait_or_fail(smem_u32(&done), 0u, &failed, err);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");

    if (!failed) {
        const int m = warp * 32 + lane, u = m / C, c = m % C;
        #pragma unroll 1
        for (int g = 0; g < NG; ++g) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * kWgTN), r);
            const int tap = g * T + u;
            if (tap >= 9) continue;
            float *gp = gw + (size_t)tap * C + c;
            #pragma unroll
            for (int j = 0; j < kWgTN; ++j) {
                const int o = kWgTN * nb + j;
                if (o < cout) atomicAdd(gp + (size_t)o * ldg, alpha * __uint_as_float(r[j]));
            }
        }
    }
    teardown<kCols>(tmem);
}

// ---- layout kernels ------------------------------------------------------------------------
// xb[((n * C/8 + g) * H + y) * W + x][e] = half(scale * x[n][y][x][8 g + e]); one thread per 8 channels.
__global__ void to_half_blocked_kernel(const float *__restrict__ x, int N, int H, int W, int C, float scale,
                                       __half *__restrict__ xb)
{
    const int G = C / 8;
    const long long total = (long long)N * G * H * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int xx = (int)(i % W);
        long long r = i / W;
        const int yy = (int)(r % H);
        r /= H;
        const int g = (int)(r % G);
        const int n = (int)(r / G);
        const float4 *src = reinterpret_cast<const float4 *>(x + (((size_t)n * H + yy) * W + xx) * C + 8 * g);
        const float4 a = src[0], b = src[1];
        __half2 h0 = __floats2half2_rn(scale * a.x, scale * a.y), h1 = __floats2half2_rn(scale * a.z, scale * a.w);
        __half2 h2 = __floats2half2_rn(scale * b.x, scale * b.y), h3 = __floats2half2_rn(scale * b.z, scale * b.w);
        *reinterpret_cast<uint4 *>(xb + (size_t)i * 8) =
            make_uint4(*reinterpret_cast<uint32_t *>(&h0), *reinterpret_cast<uint32_t *>(&h1),
                       *reinterpret_cast<uint32_t *>(&h2), *reinterpret_cast<uint32_t *>(&h3));
    }
}

// xb (Cb channels, blocked) = half(scale * x) for c < C (x NHWC with C channels, any C), zero above.
__global__ void to_half_blocked_pad_kernel(const float *__restrict__ x, int N, int H, int W, int C, int Cb,
                                           float scale, __half *__restrict__ xb)
{
    const int G = Cb / 8;
    const long long total = (long long)N * G * H * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int xx = (int)(i % W);
        long long r = i / W;
        const int yy = (int)(r % H);
        r /= H;
        const int g = (int)(r % G);
        const int n = (int)(r / G);
        const float *src = x + (((size_t)n * H + yy) * W + xx) * C;
        __align__(16) __half h[8];
        #pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int c = 8 * g + e;
            h[e] = __float2half_rn(c < C ? scale * src[c] : 0.0f);
        }
        *reinterpret_cast<uint4 *>(xb + (size_t)i * 8) = *reinterpret_cast<const uint4 *>(h);
    }
}

// wh[o][tap*Cp + c] = half(w[o][tap*C + c]) for c < C, 0 for C <= c < Cp.
__global__ void pad3_kernel(const float *__restrict__ w, int cout, int C, int Cp, __half *__restrict__ wh)
{
    const long long total = 9LL * Cp * cout;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(i / (9 * Cp));
        const int k = (int)(i % (9 * Cp)), tap = k / Cp, c = k % Cp;
        wh[i] = __float2half_rn(c < C ? w[(size_t)o * 9 * C + (size_t)tap * C + c] : 0.0f);
    }
}

// gw[o][tap*C + c] += gp[o][tap*Cp + c] for c < C.
__global__ void unpad3_add_kernel(const float *__restrict__ gp, int cout, int C, int Cp, float *__restrict__ gw)
{
    const long long total = 9LL * C * cout;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(i / (9 * C));
        const int k = (int)(i % (9 * C)), tap = k / C, c = k % C;
        gw[i] += gp[(size_t)o * 9 * Cp + (size_t)tap * Cp + c];
    }
}

// wp[(((nb * nchunks + chunk) * 18 + tap * 2 + q) * TN + r) * 8 + e] = w[nb*TN + r][tap*C + chunk*16 + q*8 + e]
// (zero for output channels nb*TN + r >= cout).
__global__ void pack3_kernel(const __half *__restrict__ w, int cout, int C, int TN, long long total,
                             __half *__restrict__ wp)
{
    const int nchunks = C / kChunk;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(i & 7);
        long long r = i >> 3;
        const int row = (int)(r % TN);
        r /= TN;
        const int kg = (int)(r % 18);
        r /= 18;
        const int chunk = (int)(r % nchunks);
        const int nb = (int)(r / nchunks);
        const int o = nb * TN + row, tap = kg >> 1, q = kg & 1;
        wp[i] = o < cout ? w[(size_t)o * 9 * C + (size_t)tap * C + chunk * kChunk + q * 8 + e] : __float2half(0.0f);
    }
}

// One launch for many packed weight arrays (smrt_nn_pack3_many): the descriptors travel as a kernel
// parameter; thread i of the concatenated index space finds its array and forms that element of
// pack3(src) with src = half(w) padded (forward) or half(flip3(w)) (adjoint), as pack3_kernel does.
struct PackSeg {
    const float *w;
    __half *dst;
    long long start, total;
    int kind, rows, C, TN, cin, cout;
};
struct PackPlan {
    PackSeg seg[SMRT_NN_PACK_MAX];
    int count;
    long long total;
};

__global__ void pack3_many_kernel(const __grid_constant__ PackPlan plan)
{
    // one thread per 8 consecutive halves (one 16-byte store): the eight share every index
    for (long long g8 = blockIdx.x * (long long)blockDim.x + threadIdx.x; g8 < (plan.total >> 3);
         g8 += (long long)gridDim.x * blockDim.x) {
        const long long g = g8 << 3;
        int k = 0;
        while (k + 1 < plan.count && g >= plan.seg[k + 1].start) ++k;
        const PackSeg &S = plan.seg[k];
        const long long i = g - S.start;
        const int nchunks = S.C / kChunk;
        long long r = i >> 3;
        const int row = (int)(r % S.TN);
        r /= S.TN;
        const int kg = (int)(r % 18);
        r /= 18;
        const int chunk = (int)(r % nchunks);
        const int nb = (int)(r / nchunks);
        const int o = nb * S.TN + row, tap = kg >> 1, c0 = chunk * kChunk + (kg & 1) * 8;
        __align__(16) __half v[8];
        #pragma unroll
        for (int e = 0; e < 8; ++e) {
            float x = 0.0f;
            const int c = c0 + e;
            if (o < S.rows) {
                if (S.kind == SMRT_NN_PACK_FORWARD) {
                    if (c < S.cin) x = S.w[(size_t)o * 9 * S.cin + (size_t)tap * S.cin + c];
                } else {                                       // flip3: src[o][tap*cout + c] = w[c][8 - tap][o]
                    x = S.w[((size_t)c * 9 + (8 - tap)) * S.cin + o];
                }
            }
            v[e] = __float2half(x);
        }
        *reinterpret_cast<uint4 *>(S.dst + i) = *reinterpret_cast<const uint4 *>(v);
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

// Tensor map of a blocked half activation [N][C/8][H][W][8] as the 4-D view (8W, H, C/8, N) with
// the box {box_px * 8, box_rows, box_planes, 1}.
CUresult blocked_map(CUtensorMap *map, const void *xb, int N, int H, int W, int C, int box_px, int box_rows,
                     int box_planes)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return CUDA_ERROR_NOT_SUPPORTED;
    const cuuint64_t dim[4] = {8ull * W, (cuuint64_t)H, (cuuint64_t)(C / 8), (cuuint64_t)N};
    const cuuint64_t str[3] = {16ull * W, 16ull * W * H, 2ull * W * H * C};
    const cuuint32_t box[4] = {(cuuint32_t)(8 * box_px), (cuuint32_t)box_rows, (cuuint32_t)box_planes, 1};
    const cuuint32_t ones[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4, const_cast<void *>(xb), dim, str, box, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

bool blocked_args_ok(const void *p, int N, int H, int W, int C)
{
    return p && N >= 1 && H >= 1 && W >= 1 && C >= 8 && C % 8 == 0 && (reinterpret_cast<uintptr_t>(p) & 15) == 0 &&
           (long long)N * H * W * C <= (1LL << 40) && (long long)W * 8 <= 0xffffffffLL;
}

// SMs of the current device (the grid-size heuristics below).
int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 148;
    }
    return n;
}

// Stages a CTA reserves in shared memory: at least what its pipeline uses, and enough that the CTAs
// resident on one SM (228 KB of shared memory, 1 KB of it reserved per CTA, plus the 1 KB alignment
// slack of the dynamic allocation) fit their accumulators in the 512 TMEM columns.
int reserve_stages(int nstages, int stage_bytes, int tmem_cols)
{
    const int max_ctas = 512 / tmem_cols;
    int r = nstages;
    while ((long long)(r * stage_bytes + 2048) * (max_ctas + 1) <= 233472) ++r;
    return r;
}

template <int TN, int MT>
cudaError_t launch_conv3_tma_mt(const void *xb, const __half *wp, int N, int H, int W, int C, int cout, float alpha,
                                float beta, float *y, int ldy, int *err, cudaStream_t s, const Epi &epi,
                                unsigned long long wait_ns, int withhold, CUresult *map_err)
{
    CUtensorMap tmx;
    *map_err = blocked_map(&tmx, xb, N, H, W, C, kHaloPx, kTileRows * MT + 2, 2);
    if (*map_err != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const int ntn = (cout + TN - 1) / TN;
    const int nchunks = C / kChunk;
    // a 32-wide single tile with at most two chunks: one stage (15 KB), so that 14 CTAs share an SM and
    // hide each other's copy latency; otherwise up to four stages per CTA
    const int nstages = (TN == 32 && MT == 1 && nchunks <= 2) ? 1 : (nchunks < kFwdStages ? nchunks : kFwdStages);
    const int reserve = reserve_stages(nstages, fwd_stage_bytes<TN, MT>(), TN * MT);
    const size_t smem = (size_t)reserve * fwd_stage_bytes<TN, MT>() + 1024;
    dim3 grid((W + kTilePx - 1) / kTilePx, (H + kTileRows * MT - 1) / (kTileRows * MT), N * ntn);
    const int vec_y = (ldy % 4 == 0) && ((reinterpret_cast<uintptr_t>(y) & 15) == 0);
    static bool attr_set = false;       // per instantiation
    if (!attr_set) {
        const int most = (kFwdStages > reserve ? kFwdStages : reserve) * fwd_stage_bytes<TN, MT>() + 1024;
        cudaError_t e = cudaFuncSetAttribute(conv3_tma_kernel<TN, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             most > 232448 ? 232448 : most);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    conv3_tma_kernel<TN, MT><<<grid, 128, smem, s>>>(tmx, wp, H, W, C, cout, ntn, nstages, alpha, beta, y, ldy,
                                                     vec_y, err, epi, wait_ns, withhold);
    return cudaGetLastError();
}

// Two stacked tiles per CTA halve the weight traffic per pixel.  They are used for 128-wide output tiles
// (weights are 36 of a stage's 42 KB) unless the coarser grid leaves SMs idle: a pair costs about 1.6
// single tiles (measured on 64 x 64 and 32 x 32 layers at batch 16), so pairs are taken when
// 1.6 ceil(pairs / SMs) <= ceil(tiles / SMs).  Pairs of 64-wide tiles measured 10-20% slower than
// single tiles and are not used.
template <int TN>
cudaError_t launch_conv3_tma(const void *xb, const __half *wp, int N, int H, int W, int C, int cout, float alpha,
                             float beta, float *y, int ldy, int *err, cudaStream_t s, const Epi &epi,
                             CUresult *map_err, unsigned long long wait_ns = kWaitNs, int withhold = 0)
{
    if constexpr (TN == 128) {
        const long long cols = (long long)((W + kTilePx - 1) / kTilePx) * N * ((cout + TN - 1) / TN);
        const long long tiles = cols * ((H + kTileRows - 1) / kTileRows);
        const long long pairs = cols * ((H + 2 * kTileRows - 1) / (2 * kTileRows));
        const int sms = sm_count();
        if (8 * ((pairs + sms - 1) / sms) <= 5 * ((tiles + sms - 1) / sms))
            return launch_conv3_tma_mt<TN, 2>(xb, wp, N, H, W, C, cout, alpha, beta, y, ldy, err, s, epi, wait_ns,
                                              withhold, map_err);
    }
    return launch_conv3_tma_mt<TN, 1>(xb, wp, N, H, W, C, cout, alpha, beta, y, ldy, err, s, epi, wait_ns, withhold,
                                      map_err);
}

} // namespace

extern "C" long long smrt_nn_pack3_halves(int cout, int C)
{
    if (cout < 1 || C < kChunk || C % kChunk != 0) return -1;
    const int TN = tile_n(cout);
    return 9LL * C * ((cout + TN - 1) / TN) * TN;
}

extern "C" int smrt_nn_pack3(const void *w, int cout, int C, void *wp, void *stream)
{
    const long long total = smrt_nn_pack3_halves(cout, C);
    if (!w || !wp || total < 0 || total > 0x7fffffffLL || (reinterpret_cast<uintptr_t>(wp) & 15) != 0)
        return tma_fail(SMRT_ERR_ARG, "smrt_nn_pack3: bad arguments (cout %d C %d; C must be a multiple of 16, wp "
                        "16-byte aligned)", cout, C);
    const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    pack3_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>((const __half *)w, cout, C, tile_n(cout), total,
                                                           (__half *)wp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_pack3: %s", cudaGetErrorString(e));
    return SMRT_OK;
}

extern "C" int smrt_nn_pack3_many(int count, const smrt_nn_pack3_desc *descs, void *stream)
{
    if (count < 1 || count > SMRT_NN_PACK_MAX || !descs)
        return tma_fail(SMRT_ERR_ARG, "smrt_nn_pack3_many: count %d outside 1..%d", count, SMRT_NN_PACK_MAX);
    PackPlan plan;
    plan.count = count;
    long long start = 0;
    for (int k = 0; k < count; ++k) {
        const smrt_nn_pack3_desc &d = descs[k];
        PackSeg &S = plan.seg[k];
        const bool fwd = d.kind == SMRT_NN_PACK_FORWARD;
        if (!d.w || !d.dst || (reinterpret_cast<uintptr_t>(d.dst) & 15) != 0 || d.cout < 1 || d.cin < 1 ||
            (d.kind != SMRT_NN_PACK_FORWARD && d.kind != SMRT_NN_PACK_ADJOINT) ||
            (fwd && (d.cpad < d.cin || d.cpad % kChunk != 0)) || (!fwd && d.cout % kChunk != 0))
            return tma_fail(SMRT_ERR_ARG, "smrt_nn_pack3_many: bad descriptor %d (kind %d cout %d cin %d cpad %d)", k,
                            d.kind, d.cout, d.cin, d.cpad);
        S.w = d.w;
        S.dst = (__half *)d.dst;
        S.kind = d.kind;
        S.rows = fwd ? d.cout : d.cin;                 // output channels of the packed operand
        S.C = fwd ? d.cpad : d.cout;                   // its input channels
        S.TN = tile_n(S.rows);
        S.cin = d.cin;
        S.cout = d.cout;
        S.total = 9LL * S.C * ((S.rows + S.TN - 1) / S.TN) * S.TN;
        S.start = start;
        start += S.total;
    }
    plan.total = start;                                // every segment is a multiple of 8 halves
    const long long groups = start >> 3;
    const int blocks = (int)((groups + 255) / 256 < 8192 ? (groups + 255) / 256 : 8192);
    pack3_many_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(plan);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_pack3_many: %s", cudaGetErrorString(e));
    return SMRT_OK;
}

extern "C" int smrt_nn_to_half_blocked(const float *x, int N, int H, int W, int C, float scale, void *xb,
                                       void *stream)
{
    if (!x || !blocked_args_ok(xb, N, H, W, C) || (reinterpret_cast<uintptr_t>(x) & 15) != 0)
        return tma_fail(SMRT_ERR_ARG, "smrt_nn_to_half_blocked: bad arguments (N %d H %d W %d C %d; C must be a "
                        "multiple of 8, x and xb 16-byte aligned)", N, H, W, C);
    const long long total = (long long)N * (C / 8) * H * W;
    const int blocks = (int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
    to_half_blocked_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, N, H, W, C, scale, (__half *)xb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_to_half_blocked: %s", cudaGetErrorString(e));
    return SMRT_OK;
}

extern "C" int smrt_nn_to_half_blocked_pad(const float *x, int N, int H, int W, int C, int Cb, float scale, void *xb,
                                           void *stream)
{
    if (!x || C < 1 || Cb < C || !blocked_args_ok(xb, N, H, W, Cb))
        return tma_fail(SMRT_ERR_ARG, "smrt_nn_to_half_blocked_pad: bad arguments (N %d H %d W %d C %d Cb %d; Cb >= C, "
                        "Cb %% 8 == 0, xb 16-byte aligned)", N, H, W, C, Cb);
    const long long total = (long long)N * (Cb / 8) * H * W;
    const int blocks = (int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
    to_half_blocked_pad_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, N, H, W, C, Cb, scale, (__half *)xb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_to_half_blocked_pad: %s", cudaGetErrorString(e));
    return SMRT_OK;
}

extern "C" int smrt_nn_pad3(const float *w, int cout, int C, int Cp, void *wh, void *stream)
{
    if (!w || !wh || cout < 1 || C < 1 || Cp < C || 9LL * Cp * cout > 0x7fffffffLL)
        return tma_fail(SMRT_ERR_ARG, "smrt_nn_pad3: bad arguments (cout %d C %d Cp %d)", cout, C, Cp);
    const long long total = 9LL * Cp * cout;
    const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    pad3_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(w, cout, C, Cp, (__half *)wh);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_pad3: %s", cudaGetErrorString(e));
    return SMRT_OK;
}

extern "C" int smrt_nn_unpad3_add(const float *gp, int cout, int C, int Cp, float *gw, void *stream)
{
    if (!gp || !gw || cout < 1 || C < 1 || Cp < C || 9LL * Cp * cout > 0x7fffffffLL)
        return tma_fail(SMRT_ERR_ARG, "smrt_nn_unpad3_add: bad arguments (cout %d C %d Cp %d)", cout, C, Cp);
    const long long total = 9LL * C * cout;
    const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    unpad3_add_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(gp, cout, C, Cp, gw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_unpad3_add: %s", cudaGetErrorString(e));
    return SMRT_OK;
}

namespace {

int conv3_tma_run(const char *name, const void *xb, int N, int H, int W, int C, const void *wp, int cout,
                  float alpha, float beta, float *y, int ldy, int *err, void *stream, unsigned long long wait_ns,
                  int withhold)
{
    if (!blocked_args_ok(xb, N, H, W, C) || C % kChunk != 0 || !wp || !y || cout < 1 || ldy < cout ||
        (reinterpret_cast<uintptr_t>(wp) & 15) != 0 || (H + kTileRows - 1) / kTileRows > 65535 ||
        (long long)N * ((cout + tile_n(cout) - 1) / tile_n(cout)) > 65535)
        return tma_fail(SMRT_ERR_ARG,
                        "%s: bad arguments (N %d H %d W %d C %d cout %d ldy %d; C must be a multiple "
                        "of 16, xb and wp 16-byte aligned)", name, N, H, W, C, cout, ldy);
    cudaStream_t s = (cudaStream_t)stream;
    const __half *w = (const __half *)wp;
    cudaError_t e;
    CUresult r = CUDA_SUCCESS;
    const int TN = tile_n(cout);
    const Epi plain{nullptr, nullptr, nullptr, nullptr, 0, 0, nullptr, nullptr};
    if (TN == 32)
        e = launch_conv3_tma<32>(xb, w, N, H, W, C, cout, alpha, beta, y, ldy, err, s, plain, &r, wait_ns, withhold);
    else if (TN == 64)
        e = launch_conv3_tma<64>(xb, w, N, H, W, C, cout, alpha, beta, y, ldy, err, s, plain, &r, wait_ns, withhold);
    else
        e = launch_conv3_tma<128>(xb, w, N, H, W, C, cout, alpha, beta, y, ldy, err, s, plain, &r, wait_ns, withhold);
    if (r != CUDA_SUCCESS) return tma_fail(SMRT_ERR_CUDA, "%s: tensor map rejected (%d)", name, (int)r);
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "%s: %s", name, cudaGetErrorString(e));
    return SMRT_OK;
}

} // namespace

extern "C" int smrt_nn_conv3_tma(const void *xb, int N, int H, int W, int C, const void *wp, int cout, float alpha,
                                 float beta, float *y, int ldy, int *err, void *stream)
{
    return conv3_tma_run("smrt_nn_conv3_tma", xb, N, H, W, C, wp, cout, alpha, beta, y, ldy, err, stream, kWaitNs,
                         0);
}

extern "C" int smrt_nn_conv3_tma_wait_test(const void *xb, int N, int H, int W, int C, const void *wp, int cout,
                                           float *y, int ldy, int *err, double wait_ms, void *stream)
{
    if (!(wait_ms >= 1e-3 && wait_ms <= 1000.0))
        return tma_fail(SMRT_ERR_ARG, "smrt_nn_conv3_tma_wait_test: wait_ms must lie in [1e-3, 1000] (got %g)",
                        wait_ms);
    if (!err) return tma_fail(SMRT_ERR_ARG, "smrt_nn_conv3_tma_wait_test: err is required");
    return conv3_tma_run("smrt_nn_conv3_tma_wait_test", xb, N, H, W, C, wp, cout, 1.0f, 0.0f, y, ldy, err, stream,
                         (unsigned long long)(wait_ms * 1e6), 1);
}

extern "C" int smrt_nn_check(int *err, void *stream)
{
    if (!err) return tma_fail(SMRT_ERR_ARG, "smrt_nn_check: err is required");
    cudaStream_t s = (cudaStream_t)stream;
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_check: %s", cudaGetErrorString(e));
    if (v == 0) return SMRT_OK;
    e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_check: %s", cudaGetErrorString(e));
    return tma_fail(SMRT_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait (error word %d): the blocks "
                    "concerned skipped their results, so the outputs since the last check are not valid", v);
}

extern "C" int smrt_nn_conv3_tma_bias_act(const void *xb, int N, int H, int W, int C, const void *wp, int cout,
                                          const float *bias, int act, float *z, float *a, void *ab, int *err,
                                          void *stream)
{
    const uintptr_t al = reinterpret_cast<uintptr_t>(z) | reinterpret_cast<uintptr_t>(a) |
                         reinterpret_cast<uintptr_t>(ab);
    if (!blocked_args_ok(xb, N, H, W, C) || C % kChunk != 0 || !wp || !bias || cout < 8 || cout % 8 != 0 ||
        (!z && !a && !ab) || (al & 15) || (reinterpret_cast<uintptr_t>(wp) & 15) != 0 ||
        (H + kTileRows - 1) / kTileRows > 65535 || (long long)N * ((cout + tile_n(cout) - 1) / tile_n(cout)) > 65535)
        return tma_fail(SMRT_ERR_ARG,
                        "smrt_nn_conv3_tma_bias_act: bad arguments (N %d H %d W %d C %d cout %d; C %% 16 == 0, "
                        "cout %% 8 == 0, 16-byte aligned outputs, at least one output)", N, H, W, C, cout);
    cudaStream_t s = (cudaStream_t)stream;
    CUresult r = CUDA_SUCCESS;
    const __half *w = (const __half *)wp;
    const Epi epi{bias, z, a, (__half *)ab, act, 1, nullptr, nullptr};
    cudaError_t e;
    const int TN = tile_n(cout);
    if (TN == 32) e = launch_conv3_tma<32>(xb, w, N, H, W, C, cout, 1.0f, 0.0f, nullptr, cout, err, s, epi, &r);
    else if (TN == 64) e = launch_conv3_tma<64>(xb, w, N, H, W, C, cout, 1.0f, 0.0f, nullptr, cout, err, s, epi, &r);
    else e = launch_conv3_tma<128>(xb, w, N, H, W, C, cout, 1.0f, 0.0f, nullptr, cout, err, s, epi, &r);
    if (r != CUDA_SUCCESS) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_conv3_tma_bias_act: tensor map rejected (%d)", (int)r);
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_conv3_tma_bias_act: %s", cudaGetErrorString(e));
    return SMRT_OK;
}

extern "C" int smrt_nn_conv3_tma_act_bwd(const void *dzb, int N, int H, int W, int C, const void *wp, int cout,
                                         const float *z, int act, float *dz, float *db, void *dzb_out, int *err,
                                         void *stream)
{
    const uintptr_t al = reinterpret_cast<uintptr_t>(z) | reinterpret_cast<uintptr_t>(dz) |
                         reinterpret_cast<uintptr_t>(dzb_out);
    if (!blocked_args_ok(dzb, N, H, W, C) || C % kChunk != 0 || !wp || (act && !z) || !dzb_out || cout < 8 ||
        cout % 8 != 0 || (al & 15) || (reinterpret_cast<uintptr_t>(wp) & 15) != 0 ||
        (H + kTileRows - 1) / kTileRows > 65535 || (long long)N * ((cout + tile_n(cout) - 1) / tile_n(cout)) > 65535)
        return tma_fail(SMRT_ERR_ARG,
                        "smrt_nn_conv3_tma_act_bwd: bad arguments (N %d H %d W %d C %d cout %d; C %% 16 == 0, "
                        "cout %% 8 == 0, 16-byte aligned z, dz, dzb_out)", N, H, W, C, cout);
    cudaStream_t s = (cudaStream_t)stream;
    CUresult r = CUDA_SUCCESS;
    const __half *w = (const __half *)wp;
    const Epi epi{nullptr, dz, nullptr, (__half *)dzb_out, act, 2, z, db};
    cudaError_t e;
    const int TN = tile_n(cout);
    if (TN == 32) e = launch_conv3_tma<32>(dzb, w, N, H, W, C, cout, 1.0f, 0.0f, nullptr, cout, err, s, epi, &r);
    else if (TN == 64) e = launch_conv3_tma<64>(dzb, w, N, H, W, C, cout, 1.0f, 0.0f, nullptr, cout, err, s, epi, &r);
    else e = launch_conv3_tma<128>(dzb, w, N, H, W, C, cout, 1.0f, 0.0f, nullptr, cout, err, s, epi, &r);
    if (r != CUDA_SUCCESS) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_conv3_tma_act_bwd: tensor map rejected (%d)", (int)r);
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_conv3_tma_act_bwd: %s", cudaGetErrorString(e));
    return SMRT_OK;
}

// Launch of conv3_wgrad_grouped_kernel<C> (C = 16 or 32): one CTA per SM over splits of the pixel tiles.
int wgrad_grouped(const void *xb, int N, int H, int W, int C, const void *dzb, int cout, float alpha, float *gw, int ldg,
                  int *err, void *stream, const CUtensorMap &tmz)
{
    const int tiles_x = (W + kTilePx - 1) / kTilePx, tiles_y = (H + kTileRows - 1) / kTileRows;
    const long long ntiles = (long long)N * tiles_x * tiles_y;
    CUtensorMap tmx;
    const CUresult r = blocked_map(&tmx, xb, N, H, W, C, kTilePx, kTileRows, C / 8);
    if (r != CUDA_SUCCESS)
        return tma_fail(SMRT_ERR_CUDA, "smrt_nn_conv3_wgrad_tma: tensor map rejected (%d)", (int)r);
    const int nbk = (cout + kWgTN - 1) / kWgTN;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
    long long splits = sms / nbk;
    if (splits < 1) splits = 1;
    if (splits > ntiles) splits = ntiles;
    const int per = (int)((ntiles + splits - 1) / splits);
    splits = (ntiles + per - 1) / per;
    const int slot = (C / 8) * kDzPlane, T = 128 / C, ng = (9 + T - 1) / T;
    const int stage = (9 * slot + 4 * kDzPlane + 1023) / 1024 * 1024;
    const int reach = ng * T * slot;                 // a stage's last group reads this far
    int nstages = kWgStages;
    auto need = [&](int n) { return (size_t)(n - 1) * stage + (size_t)(stage > reach ? stage : reach); };
    while (nstages > 1 && need(nstages) + 1024 > 220 * 1024) --nstages;
    const size_t smem = need(nstages) + 1024;
    if (smem > 220 * 1024 || nbk > 65535 || splits > 65535)
        return tma_fail(SMRT_ERR_ARG, "smrt_nn_conv3_wgrad_tma: sizes out of range (C %d cout %d)", C, cout);
    cudaStream_t s = (cudaStream_t)stream;
    dim3 grid(nbk, (unsigned)splits);
    cudaError_t e;
    if (C == 16) {
        static bool attr16 = false;
        e = attr16 ? cudaSuccess : cudaFuncSetAttribute(conv3_wgrad_grouped_kernel<16>,
                                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr16 = attr16 || e == cudaSuccess;
        if (e == cudaSuccess)
            conv3_wgrad_grouped_kernel<16><<<grid, 128, smem, s>>>(tmx, tmz, H, W, cout, tiles_x, tiles_y, (int)ntiles,
                                                                   nbk, per, nstages, stage, alpha, gw, ldg, err);
    } else {
        static bool attr32 = false;
        e = attr32 ? cudaSuccess : cudaFuncSetAttribute(conv3_wgrad_grouped_kernel<32>,
                                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr32 = attr32 || e == cudaSuccess;
        if (e == cudaSuccess)
            conv3_wgrad_grouped_kernel<32><<<grid, 128, smem, s>>>(tmx, tmz, H, W, cout, tiles_x, tiles_y, (int)ntiles,
                                                                   nbk, per, nstages, stage, alpha, gw, ldg, err);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_conv3_wgrad_tma: %s", cudaGetErrorString(e));
    return SMRT_OK;
}

extern "C" int smrt_nn_conv3_wgrad_tma(const void *xb, int N, int H, int W, int C, const void *dzb, int cout,
                                       float alpha, float *gw, int ldg, int *err, void *stream)
{
    if (!blocked_args_ok(xb, N, H, W, C) || !blocked_args_ok(dzb, N, H, W, cout) || !gw || ldg < 9 * C)
        return tma_fail(SMRT_ERR_ARG,
                        "smrt_nn_conv3_wgrad_tma: bad arguments (N %d H %d W %d C %d cout %d ldg %d; C and cout must "
                        "be multiples of 8, xb and dzb 16-byte aligned)", N, H, W, C, cout, ldg);
    const int tiles_x = (W + kTilePx - 1) / kTilePx, tiles_y = (H + kTileRows - 1) / kTileRows;
    const long long ntiles = (long long)N * tiles_x * tiles_y;
    if (ntiles > 0x7fffffffLL) return tma_fail(SMRT_ERR_ARG, "smrt_nn_conv3_wgrad_tma: too many pixels");
    const int planes = C / 8 < kWgPlanes ? C / 8 : kWgPlanes;
    CUtensorMap tmx, tmz;
    CUresult r = blocked_map(&tmx, xb, N, H, W, C, kHaloPx, kHaloRows, planes);
    if (r == CUDA_SUCCESS) r = blocked_map(&tmz, dzb, N, H, W, cout, kTilePx, kTileRows, 4);
    if (r != CUDA_SUCCESS)
        return tma_fail(SMRT_ERR_CUDA, "smrt_nn_conv3_wgrad_tma: tensor map rejected (%d)", (int)r);

    if (C == 16 || C == 32) return wgrad_grouped(xb, N, H, W, C, dzb, cout, alpha, gw, ldg, err, stream, tmz);
    const int mbk = (C + 8 * kWgPlanes - 1) / (8 * kWgPlanes), nbk = (cout + kWgTN - 1) / kWgTN;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
    // one CTA per SM (each holds all 512 TMEM columns): split the pixel tiles to fill the SMs
    long long splits = sms / (mbk * nbk);
    if (splits < 1) splits = 1;
    if (splits > ntiles) splits = ntiles;
    const int per = (int)((ntiles + splits - 1) / splits);
    splits = (ntiles + per - 1) / per;
    const int a_bytes = (planes * kPlane + 127) / 128 * 128;
    const int stage = (a_bytes + 4 * kDzPlane + 1023) / 1024 * 1024;
    const int a_reach = kWgPlanes * kPlane;         // the MMA's 128 rows read 16 planes from a stage start
    int nstages = kWgStages;
    auto need = [&](int n) { return (size_t)(n - 1) * stage + (size_t)(stage > a_reach ? stage : a_reach + 128); };
    while (nstages > 2 && need(nstages) + 1024 > 220 * 1024) --nstages;
    size_t smem = need(nstages) + 1024;
    if (smem < 120 * 1024) smem = 120 * 1024;       // keeps a second CTA (and its TMEM request) off the SM
    if (smem > 220 * 1024 || mbk * nbk > 65535 || splits > 65535)
        return tma_fail(SMRT_ERR_ARG, "smrt_nn_conv3_wgrad_tma: sizes out of range (C %d cout %d)", C, cout);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(conv3_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             220 * 1024);
        if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_conv3_wgrad_tma: %s", cudaGetErrorString(e));
        attr_set = true;
    }
    dim3 grid(mbk * nbk, (unsigned)splits);
    conv3_wgrad_kernel<<<grid, 128, smem, (cudaStream_t)stream>>>(tmx, tmz, H, W, C, cout, tiles_x, tiles_y,
                                                                  (int)ntiles, nbk, per, planes, nstages, stage, alpha,
                                                                  gw, ldg, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tma_fail(SMRT_ERR_CUDA, "smrt_nn_conv3_wgrad_tma: %s", cudaGetErrorString(e));
    return SMRT_OK;
}
