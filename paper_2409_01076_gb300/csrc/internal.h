// internal.h -- shared between the C-ABI layer (api.cu) and the per-precision
// kernel translation units (prec_*.cu).  Not part of the public interface.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>

#include "smrt.h"

namespace smrt {

// An NVTX range over one entry point (visible in Nsight timelines; header-only NVTX 3, which does
// nothing unless a profiling tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// How the stored arrays map to the canonical f(t): the two-buffer layout, or the
// in-place layout before an even / odd step (t even / t odd).
enum { MODE_AB = 0, MODE_AA_EVEN = 1, MODE_AA_ODD = 2 };

// Plain description of one lattice as the launchers need it.
struct HostParams {
    int nx, ny;
    int pitch;          // stored elements per row
    long long plane;    // stored elements per population plane
    unsigned bc;
    double tau, tau_s, u_lid;
    int *flag;          // device divergence flag
    int rounding = 0;   // SMRT_ROUND_*: how 16-bit storage rounds the stored offsets
    long long t = 0;    // the time of the state a step or residual launch starts from
};

// Device scratch the auxiliary launchers may use (owned by the caller).
struct Scratch {
    double *partials;   // >= kResidualMaxBlocks * kResidualSums doubles
    double *sums;       // >= kResidualSums doubles
};

constexpr int kResidualSums = 5;        // |du|^2, |u1|^2, rho, rho ux, rho uy
constexpr int kResidualMaxBlocks = 1216; // 8 x 152 SMs

// Launchers of one storage precision.  `mode` is MODE_AB / MODE_AA_EVEN /
// MODE_AA_ODD; `kind` an smrt_collision.  Field buffers (double) cover rows
// [row0, row0 + rows) with row-major [plane][rows][nx] layout.
struct KernelTable {
    cudaError_t (*step)(int kind, int mode, const void *src, void *dst, const HostParams &p,
                        cudaStream_t s);
    cudaError_t (*get_f)(int mode, const void *state, double *f, int row0, int rows,
                         const HostParams &p, cudaStream_t s);
    cudaError_t (*set_f)(int mode, void *state, const double *f, int row0, int rows,
                         const HostParams &p, cudaStream_t s);
    cudaError_t (*init_macros)(int mode, void *state, const double *rho, const double *u,
                               int row0, int rows, const HostParams &p, cudaStream_t s);
    cudaError_t (*macros)(int mode, const void *state, double *rho, double *u, int row0,
                          int rows, const HostParams &p, cudaStream_t s);
    cudaError_t (*residual)(int kind, int mode, const void *state, const HostParams &p,
                            const Scratch &scratch, cudaStream_t s);
    size_t elem_bytes;
};

const KernelTable &kernels_f64();
const KernelTable &kernels_f32();
const KernelTable &kernels_f16();
const KernelTable &kernels_bf16();

// Vectorised / fused element-wise kernels of the U-Net (nn_vec.cu).  Each returns
// cudaErrorNotSupported, launching nothing, when the channel count or alignment rules it out.
cudaError_t vec_bias_act(const float *x, const float *bias, long long rows, int C, int act, float *z, float *a,
                         __half *ab, int HW, cudaStream_t s);
cudaError_t vec_bias_act_bwd(const float *da, const float *z, long long rows, int C, int act, float *dz, float *db,
                             __half *dzb, int HW, cudaStream_t s, const float *dp = nullptr, int W = 0);
cudaError_t vec_avgpool2(const float *x, int N, int H, int W, int C, float *y, __half *yb, cudaStream_t s);
cudaError_t vec_avgpool2_bwd(const float *dy, int N, int H, int W, int C, float *dx, cudaStream_t s);
cudaError_t vec_add(const float *a, const float *b, long long n, float *y, cudaStream_t s);
cudaError_t vec_upcat(const float *a, int N, int H, int W, int Ca, const float *b, int Cb, float *y, __half *yb,
                      cudaStream_t s);
cudaError_t vec_upcat_bwd(const float *dy, int N, int H, int W, int Ca, int Cb, float *da, float *db, cudaStream_t s);

cudaError_t small_conv1x1(const float *x, long long P, int C, const float *w, const float *bias, int cout, float *y,
                          cudaStream_t s);
cudaError_t small_conv1x1_bwd(const float *dy, const float *x, long long P, int C, const float *w, int cout, float *dx,
                              float *dw, float *db, cudaStream_t s);

// Records the message smrt_last_error(NULL) returns on the calling thread
// (entry points that take no handle report their errors here).
void set_thread_error(const char *msg);

} // namespace smrt
