// nn_tc.cu -- smrt_nn_gemm_tc: the GEMM of include/smrt_nn.h on the 5th-generation
// tensor cores (tcgen05): operands staged in shared memory, accumulator in TMEM.
//
// One 128-thread CTA computes a 128 x 128 tile of C.  Per K step of 64:
//   1. all threads copy op(A)[128 x 64] and op(B)^T[128 x 64] (both K-major) into
//      shared memory in the no-swizzle core-matrix layout: 8 rows x 16 bytes per
//      core matrix (128 contiguous bytes), core matrices adjacent in K 128 B apart
//      (leading byte offset), 8-row groups 1024 B apart (stride byte offset);
//   2. fence.proxy.async makes those generic-proxy writes visible to the tensor core;
//   3. thread 0 issues four tcgen05.mma (M 128, N 128, K 16, half x half -> f32)
//      and commits them to an mbarrier;
//   4. every thread waits on the mbarrier (bounded: a timeout sets *err and the CTA
//      stops issuing, still releasing its TMEM) before the buffers are refilled.
// Epilogue: warp w reads TMEM lanes 32w..32w+31 (rows of the tile) with tcgen05.ld.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include "internal.h"
#include "smrt_nn.h"

namespace {

constexpr int TM = 128, TN = 128, TK = 64;
constexpr uint32_t kTmemCols = 128;
constexpr long long kWaitLimit = 1LL << 24;   // try_wait polls before a CTA gives up

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Offset (in halves) of element (row, k) of a 128 x 64 K-major tile in the core-matrix layout.
__device__ __forceinline__ int core_offset(int row, int k)
{
    return ((row >> 3) * (TK / 8) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
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

// Instruction descriptor of kind::f16: D f32, A and B half, both K-major, N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | (0u << 15) | (0u << 16) |
                            ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__global__ void __launch_bounds__(128)
gemm_tc_kernel(int transA, int transB, int M, int N, int K, float alpha, const __half *__restrict__ A, int lda,
               const __half *__restrict__ B, int ldb, float beta, float *C, int ldc, int k_chunk, int atomic,
               int *err)
{
    __shared__ __align__(1024) __half sA[TM * TK];
    __shared__ __align__(1024) __half sB[TN * TK];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_holder;
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int kbeg = blockIdx.z * k_chunk;
    const int kend = min(K, kbeg + k_chunk);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(&tmem_holder)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mbar)));
        failed = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;
    const uint32_t sa = smem_addr(sA), sb = smem_addr(sB), mb = smem_addr(&mbar);
    const __half zero = __float2half(0.0f);

    uint32_t phase = 0;
    bool any = false;
    for (int k0 = kbeg; k0 < kend; k0 += TK) {
        for (int idx = tid; idx < TM * TK; idx += 128) {
            int r, kk;
            if (!transA) { r = idx / TK; kk = idx % TK; }
            else { kk = idx / TM; r = idx % TM; }
            const int m = m0 + r, k = k0 + kk;
            __half v = zero;
            if (m < M && k < kend) v = transA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
            sA[core_offset(r, kk)] = v;
        }
        for (int idx = tid; idx < TN * TK; idx += 128) {
            int r, kk;
            if (transB) { r = idx / TK; kk = idx % TK; }
            else { kk = idx / TN; r = idx % TN; }
            const int n = n0 + r, k = k0 + kk;
            __half v = zero;
            if (n < N && k < kend) v = transB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
            sB[core_offset(r, kk)] = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (failed) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            #pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk) {
                const unsigned long long ad = make_desc(sa + kk * 256, 128, (TK / 8) * 128);
                const unsigned long long bd = make_desc(sb + kk * 256, 128, (TK / 8) * 128);
                const uint32_t acc = (any || kk > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                             :: "r"(tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(mb) : "memory");
        }
        any = true;
        // wait until the MMAs have consumed the tiles (bounded)
        uint32_t done = 0;
        for (long long it = 0; it < kWaitLimit && !done; ++it) {
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(done) : "r"(mb), "r"(phase) : "memory");
        }
        if (!done) {
            failed = 1;
            if (err) atomicExch(err, 1);
            // give the MMAs in flight a second bounded chance to finish before TMEM is released
            for (long long it = 0; it < kWaitLimit && !done; ++it) {
                asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                             "selp.u32 %0, 1, 0, p;\n\t}"
                             : "=r"(done) : "r"(mb), "r"(phase) : "memory");
            }
        }
        phase ^= 1u;
        __syncthreads();
        if (failed) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");

    if (!failed) {
        const int row = m0 + warp * 32 + lane;
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
            if (row < M) {
                #pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int n = n0 + c + j;
                    if (n >= N) break;
                    const float v = alpha * (any ? __uint_as_float(r[j]) : 0.0f);
                    float *cp = C + (size_t)row * ldc + n;
                    if (atomic) atomicAdd(cp, v);
                    else *cp = (beta != 0.0f) ? v + beta * *cp : v;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols));
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

} // namespace

extern "C" int smrt_nn_gemm_tc(int transA, int transB, int M, int N, int K, float alpha, const void *A, int lda,
                               const void *B, int ldb, float beta, float *C, int ldc, int split_k, int *err,
                               void *stream)
{
    if (M < 0 || N < 0 || K < 1 || !A || !B || !C || split_k < 1 || ldc < N || lda < (transA ? M : K) ||
        ldb < (transB ? K : N))
        return tc_fail(SMRT_ERR_ARG, "smrt_nn_gemm_tc: bad arguments (M %d N %d K %d lda %d ldb %d ldc %d split %d)",
                       M, N, K, lda, ldb, ldc, split_k);
    if (M == 0 || N == 0) return SMRT_OK;
    int chunk = (K + split_k - 1) / split_k;
    chunk = ((chunk + TK - 1) / TK) * TK;
    const int splits = (K + chunk - 1) / chunk;
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, splits);
    if (grid.y > 65535 || grid.z > 65535) return tc_fail(SMRT_ERR_ARG, "smrt_nn_gemm_tc: M or split_k too large");
    gemm_tc_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>(transA, transB, M, N, K, alpha, (const __half *)A, lda,
                                                           (const __half *)B, ldb, beta, C, ldc, chunk,
                                                           split_k > 1 ? 1 : 0, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tc_fail(SMRT_ERR_CUDA, "smrt_nn_gemm_tc: %s", cudaGetErrorString(e));
    return SMRT_OK;
}
