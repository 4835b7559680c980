// nn_tc.cu -- smrt_nn_gemm_tc (the GEMM of include/smrt_nn.h) and smrt_nn_conv3_tc (the same
// kernel with its A operand gathered as an implicit im2col of a 3x3 convolution) on the
// 5th-generation tensor cores (tcgen05): operands staged in shared memory, accumulator in TMEM.
//
// One 128-thread CTA computes a 128 x TN tile of C (TN = 32, 64 or 128, picked from N).
// Per K step of 64, double-buffered over two shared-memory stages:
//   1. all threads copy op(A)[128 x 64] and op(B)^T[TN x 64] (both K-major) into one
//      stage in the no-swizzle core-matrix layout: 8 rows x 16 bytes per core matrix
//      (128 contiguous bytes), core matrices adjacent in K 128 B apart (leading byte
//      offset), 8-row groups 1040 B apart (stride byte offset: 1024 plus a 16-byte bank skew).  Rows whose K run is
//      contiguous in global memory move as 16-byte vectors; a transposed operand moves as
//      eight 16-byte vectors along M (or N) per core matrix, transposed in registers into
//      its eight 16-byte rows.  Each thread issues all its loads before its first store;
//   2. fence.proxy.async makes those generic-proxy writes visible to the tensor core;
//   3. thread 0 issues four tcgen05.mma (M 128, N TN, K 16, half x half -> f32) and
//      commits them to that stage's mbarrier;
//   4. before a stage is refilled, every thread waits on its mbarrier (bounded: a
//      timeout sets *err, waits once more with a limit, and the CTA still releases
//      its TMEM), so the copy of one stage overlaps the MMAs of the other.
// Epilogue: warp w reads TMEM lanes 32w..32w+31 (rows of the tile) with tcgen05.ld and
// writes C (16-byte stores, or float4 atomics under split-K, when C is 16-byte aligned with
// ldc % 4 == 0), or C^T when trans_c is set (consecutive lanes write consecutive addresses).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include "internal.h"
#include "smrt_nn.h"

namespace {

constexpr int TM = 128, TK = 64;
constexpr long long kWaitLimit = 1LL << 24;   // try_wait polls before a CTA gives up

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 8-row groups of a tile lie kGroupBytes apart: the 1024 bytes of their eight K-adjacent core
// matrices plus a 16-byte skew, so that the groups' core matrices start in different shared
// memory banks (a warp that writes one core-matrix row per thread into 8 groups is conflict-free).
constexpr int kGroupBytes = (TK / 8) * 128 + 16;
constexpr int kGroupHalves = kGroupBytes / 2;

template <int ROWS>
constexpr int tile_halves() { return (ROWS / 8) * kGroupHalves; }

// Offset (in halves) of element (row, k) of a rows x 64 K-major tile in the core-matrix layout.
__device__ __forceinline__ int core_offset(int row, int k)
{
    return (row >> 3) * kGroupHalves + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

// Shared-memory matrix descriptor: start address, leading byte offset (between core
// matrices adjacent in K), stride byte offset (between 8-row groups), descriptor
// version 1, no swizzle.
__device__ __forceinline__ unsigned long long make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
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
    return (1u << 4) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t phase)
{
    uint32_t done = 0;
    for (long long it = 0; it < kWaitLimit && !done; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(mb), "r"(phase) : "memory");
    }
    return done != 0;
}

// Eight halves X[row * ld + k .. + 7] (K-major source), zero past nrows / kend.
__device__ __forceinline__ uint4 load_k_chunk(const __half *__restrict__ X, int ld, int row, int nrows, int k,
                                              int kend)
{
    if (row >= nrows) return make_uint4(0, 0, 0, 0);
    if (k + 8 <= kend) return *reinterpret_cast<const uint4 *>(X + (size_t)row * ld + k);
    __align__(16) __half h[8];
    #pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = (k + j < kend) ? X[(size_t)row * ld + k + j] : __float2half(0.0f);
    return *reinterpret_cast<const uint4 *>(h);
}

// Eight halves X[k * ld + row .. + 7] (rows contiguous: the source holds op(X)^T), zero past nrows / kend.
__device__ __forceinline__ uint4 load_mn_chunk(const __half *__restrict__ X, int ld, int k, int kend, int row,
                                               int nrows)
{
    if (k >= kend) return make_uint4(0, 0, 0, 0);
    if (row + 8 <= nrows) return *reinterpret_cast<const uint4 *>(X + (size_t)k * ld + row);
    __align__(16) __half h[8];
    #pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = (row + j < nrows) ? X[(size_t)k * ld + row + j] : __float2half(0.0f);
    return *reinterpret_cast<const uint4 *>(h);
}

template <int W>
__device__ __forceinline__ uint32_t word(const uint4 &v)
{
    return W == 0 ? v.x : W == 1 ? v.y : W == 2 ? v.z : v.w;
}

// Row R of the transpose of an 8 x 8 block of halves held as in[k] = 8 halves along rows:
// word w of the result packs (in[2w] half R, in[2w+1] half R).
template <int R>
__device__ __forceinline__ uint4 transpose_row(const uint4 in[8])
{
    constexpr uint32_t sel = (R & 1) ? 0x7632u : 0x5410u;   // high or low halves of both words
    uint4 o;
    o.x = __byte_perm(word<R / 2>(in[0]), word<R / 2>(in[1]), sel);
    o.y = __byte_perm(word<R / 2>(in[2]), word<R / 2>(in[3]), sel);
    o.z = __byte_perm(word<R / 2>(in[4]), word<R / 2>(in[5]), sel);
    o.w = __byte_perm(word<R / 2>(in[6]), word<R / 2>(in[7]), sel);
    return o;
}

// Copy rows [r0, r0 + ROWS) x k [k0, k0 + 64) of op(X) into a K-major core-matrix tile.
// kmajor: X stores each row's K run contiguously (X[row * ld + k]); otherwise X stores
// op(X)^T (X[k * ld + row]).  vec: 16-byte vectors are allowed (ld % 8 == 0, X 16-byte aligned).
// Every thread issues all of its global loads before its first shared-memory store, so a stage
// keeps up to eight 16-byte loads per thread in flight.
template <int ROWS>
__device__ __forceinline__ void load_tile(__half *tile, const __half *__restrict__ X, int ld, bool kmajor, bool vec,
                                          int r0, int nrows, int k0, int kend)
{
    const int tid = threadIdx.x;
    if (vec && kmajor) {
        constexpr int CH = ROWS * (TK / 8) / 128;     // 16-byte chunks per thread
        static_assert(CH >= 1 && ROWS * (TK / 8) % 128 == 0, "tile rows");
        // chunk c: row (c / 64) * 8 + c % 8, K offset ((c / 8) % 8) * 8 -- the rows of one core
        // matrix go to consecutive lanes, so a warp's 16-byte stores cover all banks
        uint4 v[CH];
        #pragma unroll
        for (int i = 0; i < CH; ++i) {
            const int c = tid + i * 128;
            const int r = (c >> 6) * 8 + (c & 7), kc = ((c >> 3) & 7) * 8;
            v[i] = load_k_chunk(X, ld, r0 + r, nrows, k0 + kc, kend);
        }
        #pragma unroll
        for (int i = 0; i < CH; ++i) {
            const int c = tid + i * 128;
            const int r = (c >> 6) * 8 + (c & 7), kc = ((c >> 3) & 7) * 8;
            *reinterpret_cast<uint4 *>(tile + core_offset(r, kc)) = v[i];
        }
        return;
    }
    if (vec) {
        // one 8 x 8 core matrix per thread: eight 16-byte loads along the rows (one per k),
        // transposed in registers into eight 16-byte core-matrix rows
        static_assert(ROWS <= 128, "one core matrix per thread");
        if (tid < ROWS) {
            const int g = tid % (ROWS / 8), kg = tid / (ROWS / 8);
            const int row = r0 + g * 8, kb = k0 + kg * 8;
            uint4 in[8];
            #pragma unroll
            for (int j = 0; j < 8; ++j) in[j] = load_mn_chunk(X, ld, kb + j, kend, row, nrows);
            __half *dst = tile + core_offset(g * 8, kg * 8);   // rows g*8 .. g*8+7 are 8 halves apart
            *reinterpret_cast<uint4 *>(dst + 0 * 8) = transpose_row<0>(in);
            *reinterpret_cast<uint4 *>(dst + 1 * 8) = transpose_row<1>(in);
            *reinterpret_cast<uint4 *>(dst + 2 * 8) = transpose_row<2>(in);
            *reinterpret_cast<uint4 *>(dst + 3 * 8) = transpose_row<3>(in);
            *reinterpret_cast<uint4 *>(dst + 4 * 8) = transpose_row<4>(in);
            *reinterpret_cast<uint4 *>(dst + 5 * 8) = transpose_row<5>(in);
            *reinterpret_cast<uint4 *>(dst + 6 * 8) = transpose_row<6>(in);
            *reinterpret_cast<uint4 *>(dst + 7 * 8) = transpose_row<7>(in);
        }
        return;
    }
    const __half zero = __float2half(0.0f);
    for (int idx = tid; idx < ROWS * TK; idx += 128) {
        int r, kk;
        if (kmajor) { r = idx / TK; kk = idx % TK; }
        else { kk = idx / ROWS; r = idx % ROWS; }
        const int row = r0 + r, k = k0 + kk;
        __half v = zero;
        if (row < nrows && k < kend) v = kmajor ? X[(size_t)row * ld + k] : X[(size_t)k * ld + row];
        tile[core_offset(r, kk)] = v;
    }
}

// Source of the implicit im2col operand of a 3x3, stride-1, zero-padding-1 convolution:
// x is NHWC float32 with C % 8 == 0, 16-byte aligned.
struct ConvSrc {
    const float *x;
    int H, W, C;
};

// Row t of the A tile (t = threadIdx.x, pixel (n, yy, xx)), K positions [k0, k0 + 64) of the
// implicit im2col matrix: K index (ky*3 + kx)*C + c reads x[n][yy+ky-1][xx+kx-1][c], zero outside
// the image, at k >= kend or for a row past the last pixel.  Eight 8-channel chunks, all loads
// issued before the stores; the rows of a core matrix go to consecutive lanes.  The halves are
// rounded exactly as smrt_nn_im2col3 rounds them.
__device__ __forceinline__ void load_conv_tile(__half *tile, const ConvSrc &cs, int n, int yy, int xx, bool valid,
                                               int k0, int kend)
{
    int tap = k0 / cs.C, c = k0 - tap * cs.C;
    uint4 v[TK / 8];
    #pragma unroll
    for (int j = 0; j < TK / 8; ++j) {
        v[j] = make_uint4(0, 0, 0, 0);
        const int sy = yy + tap / 3 - 1, sx = xx + tap % 3 - 1;
        if (valid && k0 + 8 * j < kend && sy >= 0 && sy < cs.H && sx >= 0 && sx < cs.W) {
            const float4 *src = reinterpret_cast<const float4 *>(cs.x + (((size_t)n * cs.H + sy) * cs.W + sx) * cs.C + c);
            const float4 a = src[0], b = src[1];
            __half2 h0 = __floats2half2_rn(a.x, a.y), h1 = __floats2half2_rn(a.z, a.w);
            __half2 h2 = __floats2half2_rn(b.x, b.y), h3 = __floats2half2_rn(b.z, b.w);
            v[j] = make_uint4(*reinterpret_cast<uint32_t *>(&h0), *reinterpret_cast<uint32_t *>(&h1),
                              *reinterpret_cast<uint32_t *>(&h2), *reinterpret_cast<uint32_t *>(&h3));
        }
        c += 8;
        if (c >= cs.C) { c -= cs.C; ++tap; }
    }
    #pragma unroll
    for (int j = 0; j < TK / 8; ++j)
        *reinterpret_cast<uint4 *>(tile + core_offset(threadIdx.x, 8 * j)) = v[j];
}

template <int TN, bool CONV>
__global__ void __launch_bounds__(128)
gemm_tc_kernel(int transA, int transB, int M, int N, int K, float alpha, const __half *__restrict__ A, int lda,
               const __half *__restrict__ B, int ldb, float beta, float *C, int ldc, int trans_c, int k_chunk,
               int atomic, int vec_a, int vec_b, int vec_c, ConvSrc cs, int *err)
{
    constexpr uint32_t kCols = TN;          // TMEM columns: one f32 column per output column
    // dynamic shared memory: two stages of A (128 x 64) then two of B (TN x 64), 1024-byte aligned
    extern __shared__ __align__(1024) unsigned char dyn[];
    __half(*sA)[tile_halves<TM>()] = reinterpret_cast<__half(*)[tile_halves<TM>()]>(dyn);
    __half(*sB)[tile_halves<TN>()] =
        reinterpret_cast<__half(*)[tile_halves<TN>()]>(dyn + 2 * tile_halves<TM>() * sizeof(__half));
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t tmem_holder;
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int kbeg = blockIdx.z * k_chunk;
    const int kend = min(K, kbeg + k_chunk);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(&tmem_holder)), "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mbar[1])));
        failed = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;

    // CONV: this thread's output pixel (row m0 + tid of the implicit im2col matrix)
    int pn = 0, py = 0, px = 0;
    const bool pvalid = m0 + tid < M;
    if (CONV && pvalid) {
        const int p = m0 + tid, hw = cs.H * cs.W;
        pn = p / hw;
        const int rem = p - pn * hw;
        py = rem / cs.W;
        px = rem - py * cs.W;
    }

    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    int step = 0;
    for (int k0 = kbeg; k0 < kend; k0 += TK, ++step) {
        const int s = step & 1;
        if (pending[s]) {           // the MMAs that read this stage two steps ago must be done
            if (!mbar_wait(smem_addr(&mbar[s]), phase[s])) {
                failed = 1;
                if (err) atomicExch(err, 1);
                mbar_wait(smem_addr(&mbar[s]), phase[s]);
            }
            phase[s] ^= 1u;
            pending[s] = false;
        }
        if constexpr (CONV) load_conv_tile(sA[s], cs, pn, py, px, pvalid, k0, kend);
        else load_tile<TM>(sA[s], A, lda, !transA, vec_a, m0, M, k0, kend);
        load_tile<TN>(sB[s], B, ldb, transB, vec_b, n0, N, k0, kend);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (failed) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = smem_addr(sA[s]), sb = smem_addr(sB[s]);
            #pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk) {
                const unsigned long long ad = make_desc(sa + kk * 256, 128, kGroupBytes);
                const unsigned long long bd = make_desc(sb + kk * 256, 128, kGroupBytes);
                const uint32_t acc = (step > 0 || kk > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                             :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc<TN>()), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_addr(&mbar[s])) : "memory");
        }
        pending[s] = true;
    }
    // drain: the last commits cover every MMA issued
    for (int s = 0; s < 2; ++s) {
        if (!pending[s]) continue;
        if (!mbar_wait(smem_addr(&mbar[s]), phase[s])) {
            failed = 1;
            if (err) atomicExch(err, 1);
            mbar_wait(smem_addr(&mbar[s]), phase[s]);
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");

    if (!failed) {
        const int row = m0 + warp * 32 + lane;
        const bool any = kend > kbeg;
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
            if (row < M && !trans_c && vec_c && n0 + c + 32 <= N) {
                // 32 consecutive columns of this thread's row: eight 16-byte stores (or float4 atomics)
                float *crow = C + (size_t)row * ldc + n0 + c;
                #pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    float4 v = any ? make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                 __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]))
                                   : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    v.x *= alpha; v.y *= alpha; v.z *= alpha; v.w *= alpha;
                    float4 *cp = reinterpret_cast<float4 *>(crow + j);
                    if (atomic) {
                        atomicAdd(cp, v);
                    } else {
                        if (beta != 0.0f) {
                            const float4 o = *cp;
                            v.x += beta * o.x; v.y += beta * o.y; v.z += beta * o.z; v.w += beta * o.w;
                        }
                        *cp = v;
                    }
                }
            } else if (row < M) {
                #pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int n = n0 + c + j;
                    if (n >= N) break;
                    const float v = alpha * (any ? __uint_as_float(r[j]) : 0.0f);
                    float *cp = trans_c ? C + (size_t)n * ldc + row : C + (size_t)row * ldc + n;
                    if (atomic) atomicAdd(cp, v);
                    else *cp = (beta != 0.0f) ? v + beta * *cp : v;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kCols));
}

int tc_fail(int code, const char *fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    smrt::set_thread_error(buf);
    return code;
}

template <int TN, bool CONV = false>
cudaError_t launch_tc(int transA, int transB, int M, int N, int K, float alpha, const void *A, int lda, const void *B,
                      int ldb, float beta, float *C, int ldc, int trans_c, int split_k, int *err, cudaStream_t s,
                      ConvSrc cs = ConvSrc{nullptr, 0, 0, 0})
{
    int chunk = (K + split_k - 1) / split_k;
    chunk = ((chunk + TK - 1) / TK) * TK;
    const int splits = (K + chunk - 1) / chunk;
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, splits);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
    const int aligned_a = (lda % 8 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
    const int aligned_b = (ldb % 8 == 0) && ((reinterpret_cast<uintptr_t>(B) & 15) == 0);
    const int aligned_c = (ldc % 4 == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
    const size_t smem = 2 * (size_t)(tile_halves<TM>() + tile_halves<TN>()) * sizeof(__half);
    static bool attr_set = false;       // per instantiation; the attribute is per function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<TN, CONV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    gemm_tc_kernel<TN, CONV><<<grid, 128, smem, s>>>(transA, transB, M, N, K, alpha, (const __half *)A, lda,
                                                  (const __half *)B, ldb, beta, C, ldc, trans_c, chunk,
                                                  split_k > 1 ? 1 : 0, aligned_a, aligned_b, aligned_c, cs, err);
    return cudaGetLastError();
}

} // namespace

extern "C" int smrt_nn_gemm_tc(int transA, int transB, int M, int N, int K, float alpha, const void *A, int lda,
                               const void *B, int ldb, float beta, float *C, int ldc, int split_k, int *err,
                               void *stream)
{
    // transB bit 1 (value 2 | transB) requests the transposed store C^T (N x M, leading dimension ldc)
    const int trans_c = (transB >> 1) & 1;
    transB &= 1;
    if (M < 0 || N < 0 || K < 1 || !A || !B || !C || split_k < 1 || ldc < (trans_c ? M : N) ||
        lda < (transA ? M : K) || ldb < (transB ? K : N))
        return tc_fail(SMRT_ERR_ARG, "smrt_nn_gemm_tc: bad arguments (M %d N %d K %d lda %d ldb %d ldc %d split %d)",
                       M, N, K, lda, ldb, ldc, split_k);
    if (M == 0 || N == 0) return SMRT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (N <= 32) e = launch_tc<32>(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, trans_c, split_k, err, s);
    else if (N <= 64) e = launch_tc<64>(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, trans_c, split_k, err, s);
    else e = launch_tc<128>(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, trans_c, split_k, err, s);
    if (e != cudaSuccess) return tc_fail(SMRT_ERR_CUDA, "smrt_nn_gemm_tc: %s", cudaGetErrorString(e));
    return SMRT_OK;
}

extern "C" int smrt_nn_conv3_tc(const float *x, int N, int H, int W, int C, const void *w, int cout, float alpha,
                                float beta, float *y, int ldy, int *err, void *stream)
{
    const long long rows = (long long)N * H * W;
    if (!x || !w || !y || N < 1 || H < 1 || W < 1 || C < 8 || C % 8 != 0 || cout < 1 || ldy < cout ||
        (reinterpret_cast<uintptr_t>(x) & 15) != 0 || rows > 0x7fffffffLL || 9LL * C > 0x7fffffffLL)
        return tc_fail(SMRT_ERR_ARG, "smrt_nn_conv3_tc: bad arguments (N %d H %d W %d C %d cout %d ldy %d)", N, H, W,
                       C, cout, ldy);
    const int M = (int)rows, K = 9 * C;
    const ConvSrc cs{x, H, W, C};
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (cout <= 32) e = launch_tc<32, true>(0, 1, M, cout, K, alpha, nullptr, K, w, K, beta, y, ldy, 0, 1, err, s, cs);
    else if (cout <= 64) e = launch_tc<64, true>(0, 1, M, cout, K, alpha, nullptr, K, w, K, beta, y, ldy, 0, 1, err, s, cs);
    else e = launch_tc<128, true>(0, 1, M, cout, K, alpha, nullptr, K, w, K, beta, y, ldy, 0, 1, err, s, cs);
    if (e != cudaSuccess) return tc_fail(SMRT_ERR_CUDA, "smrt_nn_conv3_tc: %s", cudaGetErrorString(e));
    return SMRT_OK;
}
