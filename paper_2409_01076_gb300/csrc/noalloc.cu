// noalloc.cu -- smrt_residual_noalloc: the steady-state residual of a lattice
// the caller holds, computed without allocating any memory.
//
// It is the residual computation of smrt_residual (tile + halo collision in
// shared memory, per-block partial sums, one deterministic final sum), but its
// per-block partial sums live in a fixed, file-scope device array instead of
// memory obtained from cudaMalloc, and its input is the caller's canonical
// f(t) in device memory rather than a handle's state.
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "kernels.cuh"

namespace {

using smrt::kResidualMaxBlocks;
using smrt::kResidualSums;

// Scratch: kResidualMaxBlocks x kResidualSums partial sums, then 4 result slots.
// 1216 * 5 + 4 doubles = 48,672 bytes on every device that loads the library.
constexpr int kScratchDoubles = kResidualMaxBlocks * kResidualSums + 4;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// The device address of g_noalloc_scratch in the current context.  Host code may
// not use the symbol's name as an address.  The lookup allocates nothing and is
// repeated on every call, so a context that was torn down and created again
// (cudaDeviceReset) never sees a stale address.  The first lookup on a device
// loads this module there, which is why the first call on a device should come
// before any stream capture.
cudaError_t scratch_address(double **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double *>(p);
    return cudaSuccess;
}

// The residual kernel of kernels.cuh, reading the canonical field
// f[a][j][i] (double, already including every wall term) instead of a
// handle's stored offsets.
template <int KIND>
__global__ void __launch_bounds__(256)
residual_canonical_kernel(const double *f, const smrt::Params<double> p, double *partials, int tiles_x,
                          int tiles_y)
{
    using namespace smrt;
    __shared__ double post[9][kRHY][kRHX];
    __shared__ double u0s[3][kRTY][kRTX];
    __shared__ double red[8][kResidualSums];
    const int tid = threadIdx.x;
    const size_t plane = (size_t)p.nx * (size_t)p.ny;
    double acc[kResidualSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const int ntiles = tiles_x * tiles_y;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tx0 = (tile % tiles_x) * kRTX, ty0 = (tile / tiles_x) * kRTY;
        for (int q = tid; q < kRHX * kRHY; q += 256) {
            const int hx = q % kRHX, hy = q / kRHX;
            int i = tx0 - 1 + hx, j = ty0 - 1 + hy;
            const bool tile_node = hx >= 1 && hx <= kRTX && hy >= 1 && hy <= kRTY && i < p.nx && j < p.ny;
            if (i > p.nx || j > p.ny) continue;
            if (resolve(p, i, j) >= 0) continue;
            double g[9];
            #pragma unroll
            for (int a = 0; a < 9; ++a) g[a] = f[(size_t)a * plane + (size_t)j * p.nx + i] - wgt<double>(a);
            if (tile_node) {
                double rr, ux, uy;
                moments_d(g, rr, ux, uy);
                u0s[0][hy - 1][hx - 1] = rr;
                u0s[1][hy - 1][hx - 1] = ux;
                u0s[2][hy - 1][hx - 1] = uy;
            }
            collide<KIND>(p, g);
            #pragma unroll
            for (int a = 0; a < 9; ++a) post[a][hy][hx] = g[a];
        }
        __syncthreads();
        const int lx = tid % kRTX, ly = tid / kRTX;
        const int i = tx0 + lx, j = ty0 + ly;
        if (i < p.nx && j < p.ny) {
            double g1[9];
            #pragma unroll
            for (int a = 0; a < 9; ++a) {
                int si = i - ex(a), sj = j - ey(a);
                int side = resolve(p, si, sj);
                if (side >= 0) g1[a] = post[opp(a)][ly + 1][lx + 1] + p.corr[side][a];
                else g1[a] = post[a][ly + 1 - ey(a)][lx + 1 - ex(a)];
            }
            double r1, ux1, uy1;
            moments_d(g1, r1, ux1, uy1);
            const double r0 = u0s[0][ly][lx], ux0 = u0s[1][ly][lx], uy0 = u0s[2][ly][lx];
            const double dx = ux1 - ux0, dy = uy1 - uy0;
            acc[0] += dx * dx + dy * dy;
            acc[1] += ux1 * ux1 + uy1 * uy1;
            acc[2] += r0;
            acc[3] += r0 * ux0;
            acc[4] += r0 * uy0;
        }
        __syncthreads();
    }
    #pragma unroll
    for (int k = 0; k < kResidualSums; ++k) acc[k] = warp_sum(acc[k]);
    if ((tid & 31) == 0) {
        #pragma unroll
        for (int k = 0; k < kResidualSums; ++k) red[tid >> 5][k] = acc[k];
    }
    __syncthreads();
    if (tid < kResidualSums) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w][tid];
        partials[(size_t)blockIdx.x * kResidualSums + tid] = s;
    }
}

// Fixed-order sum of the partials; out = {r, sum rho, sum rho ux, sum rho uy}.
__global__ void __launch_bounds__(256) finish_kernel(const double *partials, int nblocks, double *out)
{
    __shared__ double sh[kResidualSums][256];
    const int tid = threadIdx.x;
    double acc[kResidualSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = tid; b < nblocks; b += 256) {
        #pragma unroll
        for (int k = 0; k < kResidualSums; ++k) acc[k] += partials[(size_t)b * kResidualSums + k];
    }
    #pragma unroll
    for (int k = 0; k < kResidualSums; ++k) sh[k][tid] = acc[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) {
            #pragma unroll
            for (int k = 0; k < kResidualSums; ++k) sh[k][tid] += sh[k][tid + w];
        }
        __syncthreads();
    }
    if (tid == 0) {
        const double du2 = sh[0][0], u2 = sh[1][0];
        out[0] = (du2 == 0.0 && u2 == 0.0) ? 0.0 : sqrt(du2) / sqrt(u2);
        out[1] = sh[2][0];
        out[2] = sh[3][0];
        out[3] = sh[4][0];
    }
}

int arg_error(const char *fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    smrt::set_thread_error(buf);
    return SMRT_ERR_ARG;
}

int cuda_error(cudaError_t e, const char *what)
{
    char buf[256];
    snprintf(buf, sizeof(buf), "smrt_residual_noalloc: %s: %s", what, cudaGetErrorString(e));
    smrt::set_thread_error(buf);
    return SMRT_ERR_CUDA;
}

bool bc_ok(unsigned bc)
{
    if (bc >> 8) return false;
    for (int s = 0; s < 4; ++s)
        if (((bc >> (2 * s)) & 3u) > SMRT_BC_MOVING) return false;
    return (((bc & 3u) == 0) == (((bc >> 2) & 3u) == 0)) && ((((bc >> 4) & 3u) == 0) == (((bc >> 6) & 3u) == 0));
}

} // namespace

extern "C" SMRT_API int smrt_residual_noalloc(const double *f, int nx, int ny, double tau, double u_lid,
                                              unsigned bc_flags, int collision, double tau_s, double *out,
                                              void *stream)
{
    if (!f || !out) return arg_error("smrt_residual_noalloc: f and out are required");
    if (nx < 2 || ny < 2) return arg_error("smrt_residual_noalloc: need nx, ny >= 2 (got %d x %d)", nx, ny);
    if ((long long)nx * (long long)ny > SMRT_NOALLOC_MAX_NODES)
        return arg_error("smrt_residual_noalloc: %d x %d nodes exceed the maximum of %lld", nx, ny,
                         (long long)SMRT_NOALLOC_MAX_NODES);
    if (!(tau > 0.5) || !isfinite(tau)) return arg_error("smrt_residual_noalloc: tau must be > 0.5 (got %g)", tau);
    if (collision != SMRT_COLLISION_SMRT && collision != SMRT_COLLISION_SRT && collision != SMRT_COLLISION_TWO_TAU)
        return arg_error("smrt_residual_noalloc: unknown collision kind %d", collision);
    if (collision == SMRT_COLLISION_TWO_TAU && (!(tau_s > 0.5) || !isfinite(tau_s)))
        return arg_error("smrt_residual_noalloc: tau_s must be > 0.5 (got %g)", tau_s);
    if (!isfinite(u_lid) || fabs(u_lid) >= 1.0 / sqrt(3.0))
        return arg_error("smrt_residual_noalloc: |u_lid| must be below 1/sqrt(3) (got %g)", u_lid);
    if (!bc_ok(bc_flags)) return arg_error("smrt_residual_noalloc: invalid bc_flags 0x%x", bc_flags);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    cudaPointerAttributes at;
    e = cudaPointerGetAttributes(&at, f);
    if (e != cudaSuccess || (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev) {
        cudaGetLastError();
        return arg_error("smrt_residual_noalloc: f must be device memory of the current device");
    }
    bool out_on_device = false;
    e = cudaPointerGetAttributes(&at, out);
    if (e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
        if (at.device != dev) return arg_error("smrt_residual_noalloc: out is on another device");
        out_on_device = true;
    }
    cudaGetLastError();

    double *scratch = nullptr;
    if ((e = scratch_address(&scratch)) != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress");

    smrt::HostParams hp;
    hp.nx = nx;
    hp.ny = ny;
    hp.pitch = nx;
    hp.plane = (long long)nx * ny;
    hp.bc = bc_flags;
    hp.tau = tau;
    hp.tau_s = (collision == SMRT_COLLISION_TWO_TAU) ? tau_s : 1.0;
    hp.u_lid = u_lid;
    hp.flag = nullptr;
    const smrt::Params<double> p = smrt::make_params<double>(hp);
    const int tiles_x = (nx + smrt::kRTX - 1) / smrt::kRTX, tiles_y = (ny + smrt::kRTY - 1) / smrt::kRTY;
    const long long nt = (long long)tiles_x * tiles_y;
    const int nb = (int)(nt < kResidualMaxBlocks ? nt : kResidualMaxBlocks);
    cudaStream_t s = (cudaStream_t)stream;
    double *partials = scratch;
    double *result = scratch + (size_t)kResidualMaxBlocks * kResidualSums;
    switch (collision) {
    case SMRT_COLLISION_SMRT:
        residual_canonical_kernel<SMRT_COLLISION_SMRT><<<nb, 256, 0, s>>>(f, p, partials, tiles_x, tiles_y);
        break;
    case SMRT_COLLISION_SRT:
        residual_canonical_kernel<SMRT_COLLISION_SRT><<<nb, 256, 0, s>>>(f, p, partials, tiles_x, tiles_y);
        break;
    default:
        residual_canonical_kernel<SMRT_COLLISION_TWO_TAU><<<nb, 256, 0, s>>>(f, p, partials, tiles_x, tiles_y);
        break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "residual launch");
    finish_kernel<<<1, 256, 0, s>>>(partials, nb, out_on_device ? out : result);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "finish launch");
    if (!out_on_device) {
        if ((e = cudaMemcpyAsync(out, result, 4 * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return cuda_error(e, "cudaMemcpyAsync");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    }
    return SMRT_OK;
}
