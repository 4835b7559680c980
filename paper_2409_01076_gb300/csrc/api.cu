// api.cu -- the C ABI declared in include/smrt.h: argument checking, device
// memory, host/device transfers and dispatch to the per-precision launchers.
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>

#include "internal.h"
#include "smrt.h"

namespace {

using smrt::HostParams;
using smrt::KernelTable;

thread_local std::string g_create_error = "no error";

constexpr size_t kStageBytesMax = 64ull << 20;   // host-transfer staging buffer cap
using smrt::MODE_AB;
using smrt::MODE_AA_EVEN;
using smrt::MODE_AA_ODD;

const KernelTable &table_for(int prec)
{
    switch (prec) {
    case SMRT_PREC_F32: return smrt::kernels_f32();
    case SMRT_PREC_F16: return smrt::kernels_f16();
    case SMRT_PREC_BF16: return smrt::kernels_bf16();
    default: return smrt::kernels_f64();
    }
}

} // namespace

struct smrt_t {
    int nx = 0, ny = 0;
    double tau = 1.0, tau_s = 1.0, u_lid = 0.0;
    unsigned bc = 0;
    int collision = SMRT_COLLISION_SMRT;
    int layout = SMRT_LAYOUT_AB;
    int prec = SMRT_PREC_F64;
    int check_div = 1;
    int rounding = SMRT_ROUND_NEAREST;
    double mem_limit = 0.0;
    cudaStream_t stream = nullptr;

    bool ready = false;
    int device = -1;
    int pitch = 0;
    long long plane = 0;
    size_t buf_bytes = 0;
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;
    int *d_flag = nullptr;
    int *h_flag = nullptr;
    double *d_partials = nullptr;
    double *d_sums = nullptr;
    double *h_sums = nullptr;
    double *d_stage = nullptr;
    size_t stage_bytes = 0;
    size_t dev_bytes = 0;
    long long t = 0;
    std::string err = "no error";
};

namespace {

int fail(smrt_t *h, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_create_error = buf;
    return code;
}

int cuda_fail(smrt_t *h, cudaError_t e, const char *what)
{
    return fail(h, SMRT_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

} // namespace

namespace smrt {
void set_thread_error(const char *msg)
{
    g_create_error = msg;
}
} // namespace smrt

namespace {

#define CUDA_TRY(h, call)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
    } while (0)

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        if (dev < 0) return;
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) {
            err = cudaSetDevice(dev);
            changed = (err == cudaSuccess);
        }
    }
    ~DeviceGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

bool valid_bc(unsigned bc)
{
    if (bc >> 8) return false;
    for (int s = 0; s < 4; ++s)
        if (((bc >> (2 * s)) & 3u) > SMRT_BC_MOVING) return false;
    bool lp = (bc & 3u) == SMRT_BC_PERIODIC, rp = ((bc >> 2) & 3u) == SMRT_BC_PERIODIC;
    bool bp = ((bc >> 4) & 3u) == SMRT_BC_PERIODIC, tp = ((bc >> 6) & 3u) == SMRT_BC_PERIODIC;
    return lp == rp && bp == tp;
}

size_t elem_bytes(int prec)
{
    return (prec == SMRT_PREC_F64) ? 8 : (prec == SMRT_PREC_F32 ? 4 : 2);
}

int pitch_for(int nx, int prec)
{
    long long per = 128 / (long long)elem_bytes(prec);
    return (int)(((long long)nx + per - 1) / per * per);
}

HostParams host_params(const smrt_t *h)
{
    HostParams p;
    p.nx = h->nx;
    p.ny = h->ny;
    p.pitch = h->pitch;
    p.plane = h->plane;
    p.bc = h->bc;
    p.tau = h->tau;
    p.tau_s = h->tau_s;
    p.u_lid = h->u_lid;
    p.flag = h->d_flag;
    p.rounding = h->rounding;
    p.t = h->t;
    return p;
}

int current_mode(const smrt_t *h)
{
    if (h->layout == SMRT_LAYOUT_AB) return MODE_AB;
    return (h->t % 2 == 0) ? MODE_AA_EVEN : MODE_AA_ODD;
}

void release(smrt_t *h)
{
    for (int k = 0; k < 2; ++k)
        if (h->buf[k]) cudaFree(h->buf[k]);
    if (h->d_flag) cudaFree(h->d_flag);
    if (h->d_partials) cudaFree(h->d_partials);
    if (h->d_sums) cudaFree(h->d_sums);
    if (h->d_stage) cudaFree(h->d_stage);
    if (h->h_flag) cudaFreeHost(h->h_flag);
    if (h->h_sums) cudaFreeHost(h->h_sums);
    h->buf[0] = h->buf[1] = nullptr;
    h->d_flag = nullptr;
    h->d_partials = h->d_sums = h->d_stage = h->h_sums = nullptr;
    h->h_flag = nullptr;
    h->stage_bytes = 0;
    h->dev_bytes = 0;
    h->ready = false;
}

int dev_alloc(smrt_t *h, void **p, size_t bytes, const char *what)
{
    if (h->mem_limit > 0.0 && (double)(h->dev_bytes + bytes) > h->mem_limit)
        return fail(h, SMRT_ERR_OOM, "%s: %zu bytes would exceed the memory limit of %.0f bytes (%zu held)",
                    what, bytes, h->mem_limit, h->dev_bytes);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(h, SMRT_ERR_OOM, "%s: cudaMalloc of %zu bytes failed: %s", what, bytes, cudaGetErrorString(e));
    }
    h->dev_bytes += bytes;
    return SMRT_OK;
}

// Allocate the state on first use and set f(0) = f^eq(1, 0), t = 0.
int materialize(smrt_t *h)
{
    if (h->ready) return SMRT_OK;
    CUDA_TRY(h, cudaGetDevice(&h->device));
    h->pitch = pitch_for(h->nx, h->prec);
    h->plane = (long long)h->pitch * h->ny;
    h->buf_bytes = (size_t)9 * (size_t)h->plane * elem_bytes(h->prec);
    const int nbuf = (h->layout == SMRT_LAYOUT_AB) ? 2 : 1;
    int rc;
    for (int k = 0; k < nbuf; ++k)
        if ((rc = dev_alloc(h, &h->buf[k], h->buf_bytes, "population buffer")) != SMRT_OK) {
            release(h);
            return rc;
        }
    if ((rc = dev_alloc(h, (void **)&h->d_flag, sizeof(int), "flag")) != SMRT_OK ||
        (rc = dev_alloc(h, (void **)&h->d_partials,
                        sizeof(double) * smrt::kResidualMaxBlocks * smrt::kResidualSums, "partials")) != SMRT_OK ||
        (rc = dev_alloc(h, (void **)&h->d_sums, sizeof(double) * smrt::kResidualSums, "sums")) != SMRT_OK) {
        release(h);
        return rc;
    }
    cudaError_t e = cudaMallocHost((void **)&h->h_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->h_sums, sizeof(double) * smrt::kResidualSums);
    if (e != cudaSuccess) {
        release(h);
        return cuda_fail(h, e, "cudaMallocHost");
    }
    h->ready = true;
    h->t = 0;
    h->cur = 0;
    *h->h_flag = 0;
    e = cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) {
        HostParams p = host_params(h);
        e = table_for(h->prec).init_macros(current_mode(h), h->buf[0], nullptr, nullptr, 0, h->ny, p, h->stream);
    }
    if (e != cudaSuccess) {
        release(h);
        return cuda_fail(h, e, "initial state");
    }
    return SMRT_OK;
}

// Staging for `planes` double planes: the whole field if it fits in the cap,
// else as many rows as fit, and always at least one full row.
int ensure_stage(smrt_t *h, int planes)
{
    const size_t per_row = (size_t)planes * (size_t)h->nx * sizeof(double);
    size_t want = per_row * (size_t)h->ny;
    if (want > kStageBytesMax) want = kStageBytesMax / per_row * per_row;
    if (want < per_row) want = per_row;
    if (h->stage_bytes >= want) return SMRT_OK;
    if (h->d_stage) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
        cudaFree(h->d_stage);
        h->dev_bytes -= h->stage_bytes;
        h->d_stage = nullptr;
        h->stage_bytes = 0;
    }
    int rc = dev_alloc(h, (void **)&h->d_stage, want, "staging buffer");
    if (rc == SMRT_OK) h->stage_bytes = want;
    return rc;
}

// 0: host memory, 1: device memory of the handle's device, -1: unusable.
// Where a caller's array lives: 1 = memory of the handle's device, 2 = page-locked host memory
// the device addresses directly (its device address goes to *dptr; kernels then read or write
// it over the host link, with no staging copy), 0 = other host memory (staged in chunks),
// -1 = another device's memory.
int classify(smrt_t *h, const void *ptr, const void **dptr = nullptr)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        return (at.device == h->device) ? 1 : -1;
    if (at.type == cudaMemoryTypeHost && at.devicePointer) {
        if (dptr) *dptr = at.devicePointer;
        return 2;
    }
    return 0;
}

// Rows per chunk when `planes` double planes of nx values go through staging.
int chunk_rows(const smrt_t *h, int planes)
{
    size_t per_row = (size_t)planes * (size_t)h->nx * sizeof(double);
    size_t rows = h->stage_bytes / per_row;
    if (rows < 1) rows = 1;
    if (rows > (size_t)h->ny) rows = h->ny;
    return (int)rows;
}

int begin(smrt_t *h)
{
    if (!h) return SMRT_ERR_ARG;
    return materialize(h);
}

} // namespace

extern "C" {

int smrt_create(int nx, int ny, double tau, double u_lid, unsigned bc_flags, smrt_t **out)
{
    if (!out) return fail(nullptr, SMRT_ERR_ARG, "smrt_create: out is NULL");
    *out = nullptr;
    if (nx < 2 || ny < 2) return fail(nullptr, SMRT_ERR_ARG, "smrt_create: need nx, ny >= 2 (got %d x %d)", nx, ny);
    if (!(tau > 0.5) || !isfinite(tau))
        return fail(nullptr, SMRT_ERR_ARG, "smrt_create: tau must be a finite number > 0.5 (got %g)", tau);
    if (!isfinite(u_lid) || fabs(u_lid) >= 1.0 / sqrt(3.0))
        return fail(nullptr, SMRT_ERR_ARG, "smrt_create: |u_lid| must be below 1/sqrt(3) (got %g)", u_lid);
    if (!valid_bc(bc_flags))
        return fail(nullptr, SMRT_ERR_ARG, "smrt_create: invalid bc_flags 0x%x (kinds 0-2, periodic sides paired)",
                    bc_flags);
    // the largest storage (2-byte elements need the widest pitch) must stay addressable per plane
    long long pitch_max = ((long long)nx + 63) / 64 * 64;
    if (pitch_max * (long long)ny >= (1LL << 31) || (long long)ny * nx >= (1LL << 31))
        return fail(nullptr, SMRT_ERR_ARG, "smrt_create: lattice %d x %d too large for one plane", nx, ny);
    smrt_t *h = new (std::nothrow) smrt_t;
    if (!h) return fail(nullptr, SMRT_ERR_OOM, "smrt_create: out of host memory");
    h->nx = nx;
    h->ny = ny;
    h->tau = tau;
    h->tau_s = 1.0;
    h->u_lid = u_lid;
    h->bc = bc_flags;
    *out = h;
    return SMRT_OK;
}

int smrt_set_option(smrt_t *h, int key, double value)
{
    if (!h) return SMRT_ERR_ARG;
    switch (key) {
    case SMRT_OPT_COLLISION:
        if (value != SMRT_COLLISION_SMRT && value != SMRT_COLLISION_SRT && value != SMRT_COLLISION_TWO_TAU)
            return fail(h, SMRT_ERR_ARG, "COLLISION: unknown kind %g", value);
        h->collision = (int)value;
        return SMRT_OK;
    case SMRT_OPT_TAU_S:
        if (!(value > 0.5) || !isfinite(value)) return fail(h, SMRT_ERR_ARG, "TAU_S must be > 0.5 (got %g)", value);
        h->tau_s = value;
        return SMRT_OK;
    case SMRT_OPT_TAU:
        if (!(value > 0.5) || !isfinite(value)) return fail(h, SMRT_ERR_ARG, "TAU must be > 0.5 (got %g)", value);
        h->tau = value;
        return SMRT_OK;
    case SMRT_OPT_LAYOUT:
        if (h->ready) return fail(h, SMRT_ERR_STATE, "LAYOUT can only be set before the state is first touched");
        if (value != SMRT_LAYOUT_AB && value != SMRT_LAYOUT_AA) return fail(h, SMRT_ERR_ARG, "LAYOUT: unknown %g", value);
        h->layout = (int)value;
        return SMRT_OK;
    case SMRT_OPT_PRECISION:
        if (h->ready) return fail(h, SMRT_ERR_STATE, "PRECISION can only be set before the state is first touched");
        if (value != SMRT_PREC_F64 && value != SMRT_PREC_F32 && value != SMRT_PREC_F16 && value != SMRT_PREC_BF16)
            return fail(h, SMRT_ERR_ARG, "PRECISION: unknown %g", value);
        h->prec = (int)value;
        return SMRT_OK;
    case SMRT_OPT_CHECK_DIVERGENCE:
        if (value != 0.0 && value != 1.0) return fail(h, SMRT_ERR_ARG, "CHECK_DIVERGENCE must be 0 or 1");
        h->check_div = (int)value;
        return SMRT_OK;
    case SMRT_OPT_MEM_LIMIT:
        if (h->ready) return fail(h, SMRT_ERR_STATE, "MEM_LIMIT can only be set before the state is first touched");
        if (!(value >= 0.0) || !isfinite(value)) return fail(h, SMRT_ERR_ARG, "MEM_LIMIT must be >= 0");
        h->mem_limit = value;
        return SMRT_OK;
    case SMRT_OPT_ROUNDING:
        if (value != SMRT_ROUND_NEAREST && value != SMRT_ROUND_STOCHASTIC)
            return fail(h, SMRT_ERR_ARG, "ROUNDING: unknown %g", value);
        h->rounding = (int)value;
        return SMRT_OK;
    default:
        return fail(h, SMRT_ERR_ARG, "unknown option key %d", key);
    }
}

int smrt_get_option(const smrt_t *h, int key, double *value)
{
    if (!h || !value) return SMRT_ERR_ARG;
    switch (key) {
    case SMRT_OPT_COLLISION: *value = h->collision; return SMRT_OK;
    case SMRT_OPT_TAU_S: *value = h->tau_s; return SMRT_OK;
    case SMRT_OPT_TAU: *value = h->tau; return SMRT_OK;
    case SMRT_OPT_LAYOUT: *value = h->layout; return SMRT_OK;
    case SMRT_OPT_PRECISION: *value = h->prec; return SMRT_OK;
    case SMRT_OPT_CHECK_DIVERGENCE: *value = h->check_div; return SMRT_OK;
    case SMRT_OPT_MEM_LIMIT: *value = h->mem_limit; return SMRT_OK;
    case SMRT_OPT_ROUNDING: *value = h->rounding; return SMRT_OK;
    default: return fail(const_cast<smrt_t *>(h), SMRT_ERR_ARG, "unknown option key %d", key);
    }
}

int smrt_set_stream(smrt_t *h, void *stream)
{
    if (!h) return SMRT_ERR_ARG;
    h->stream = (cudaStream_t)stream;
    return SMRT_OK;
}

int smrt_sync(smrt_t *h)
{
    int rc = begin(h);
    if (rc != SMRT_OK) return rc;
    DeviceGuard g(h->device);
    CUDA_TRY(h, g.err);
    CUDA_TRY(h, cudaMemcpyAsync(h->h_flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (*h->h_flag) return fail(h, SMRT_ERR_DIVERGED, "diverged: a node had rho <= 0 or non-finite (t <= %lld)", h->t);
    return SMRT_OK;
}

int smrt_step(smrt_t *h, long long n)
{
    smrt::TraceRange trace("smrt_step");
    if (!h) return SMRT_ERR_ARG;
    if (n < 0) return fail(h, SMRT_ERR_ARG, "smrt_step: n must be >= 0 (got %lld)", n);
    int rc = begin(h);
    if (rc != SMRT_OK) return rc;
    DeviceGuard g(h->device);
    CUDA_TRY(h, g.err);
    const KernelTable &T = table_for(h->prec);
    HostParams p = host_params(h);
    for (long long s = 0; s < n; ++s) {
        cudaError_t e;
        p.t = h->t;
        if (h->layout == SMRT_LAYOUT_AB) {
            e = T.step(h->collision, MODE_AB, h->buf[h->cur], h->buf[1 - h->cur], p, h->stream);
            if (e == cudaSuccess) h->cur = 1 - h->cur;
        } else {
            e = T.step(h->collision, current_mode(h), h->buf[0], h->buf[0], p, h->stream);
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
        ++h->t;
    }
    if (h->check_div) return smrt_sync(h);
    return SMRT_OK;
}

int smrt_macros(smrt_t *h, double *rho, double *u)
{
    smrt::TraceRange trace("smrt_macros");
    int rc = begin(h);
    if (rc != SMRT_OK) return rc;
    if (!rho && !u) return SMRT_OK;
    DeviceGuard g(h->device);
    CUDA_TRY(h, g.err);
    const KernelTable &T = table_for(h->prec);
    HostParams p = host_params(h);
    const void *state = h->buf[h->cur];
    const void *drho = rho, *du = u;
    int kr = rho ? classify(h, rho, &drho) : -2, ku = u ? classify(h, u, &du) : -2;
    if (kr == -1 || ku == -1) return fail(h, SMRT_ERR_ARG, "smrt_macros: pointer on another device");
    if (kr != 0 && ku != 0) {            // device memory, or page-locked host memory written directly
        CUDA_TRY(h, T.macros(current_mode(h), state, (double *)drho, (double *)du, 0, h->ny, p, h->stream));
        if (kr == 2 || ku == 2) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        return SMRT_OK;
    }
    // host outputs (or mixed): go through the staging buffer, 3 planes per chunk
    if ((rc = ensure_stage(h, 3)) != SMRT_OK) return rc;
    const int cr = chunk_rows(h, 3);
    const size_t nxb = (size_t)h->nx * sizeof(double);
    for (int r0 = 0; r0 < h->ny; r0 += cr) {
        int rows = (h->ny - r0 < cr) ? h->ny - r0 : cr;
        double *srho = h->d_stage, *su = h->d_stage + (size_t)rows * h->nx;
        CUDA_TRY(h, T.macros(current_mode(h), state, srho, su, r0, rows, p, h->stream));
        if (rho) {
            double *dst = rho + (size_t)r0 * h->nx;
            CUDA_TRY(h, cudaMemcpyAsync(dst, srho, rows * nxb, kr == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                        h->stream));
        }
        if (u) {
            CUDA_TRY(h, cudaMemcpy2DAsync(u + (size_t)r0 * h->nx, (size_t)h->ny * nxb, su, rows * nxb, rows * nxb, 2,
                                          ku == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
        }
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SMRT_OK;
}

int smrt_residual(smrt_t *h, double *r, double *sums)
{
    smrt::TraceRange trace("smrt_residual");
    int rc = begin(h);
    if (rc != SMRT_OK) return rc;
    DeviceGuard g(h->device);
    CUDA_TRY(h, g.err);
    const KernelTable &T = table_for(h->prec);
    HostParams p = host_params(h);
    smrt::Scratch sc;
    sc.partials = h->d_partials;
    sc.sums = h->d_sums;
    CUDA_TRY(h, T.residual(h->collision, current_mode(h), h->buf[h->cur], p, sc, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->h_sums, h->d_sums, sizeof(double) * smrt::kResidualSums, cudaMemcpyDeviceToHost,
                                h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    const double *s = h->h_sums;
    if (r) {
        if (s[0] == 0.0 && s[1] == 0.0) *r = 0.0;
        else *r = sqrt(s[0]) / sqrt(s[1]);
    }
    if (sums) {
        sums[0] = s[2];
        sums[1] = s[3];
        sums[2] = s[4];
    }
    return SMRT_OK;
}

int smrt_get_f(smrt_t *h, double *f)
{
    int rc = begin(h);
    if (rc != SMRT_OK) return rc;
    if (!f) return fail(h, SMRT_ERR_ARG, "smrt_get_f: f is NULL");
    DeviceGuard g(h->device);
    CUDA_TRY(h, g.err);
    const KernelTable &T = table_for(h->prec);
    HostParams p = host_params(h);
    const void *state = h->buf[h->cur];
    const void *df = f;
    int k = classify(h, f, &df);
    if (k == -1) return fail(h, SMRT_ERR_ARG, "smrt_get_f: pointer on another device");
    if (k != 0) {
        CUDA_TRY(h, T.get_f(current_mode(h), state, (double *)df, 0, h->ny, p, h->stream));
        if (k == 2) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        return SMRT_OK;
    }
    if ((rc = ensure_stage(h, 9)) != SMRT_OK) return rc;
    const int cr = chunk_rows(h, 9);
    const size_t nxb = (size_t)h->nx * sizeof(double);
    for (int r0 = 0; r0 < h->ny; r0 += cr) {
        int rows = (h->ny - r0 < cr) ? h->ny - r0 : cr;
        CUDA_TRY(h, T.get_f(current_mode(h), state, h->d_stage, r0, rows, p, h->stream));
        CUDA_TRY(h, cudaMemcpy2DAsync(f + (size_t)r0 * h->nx, (size_t)h->ny * nxb, h->d_stage, rows * nxb, rows * nxb, 9,
                                      cudaMemcpyDeviceToHost, h->stream));
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SMRT_OK;
}

int smrt_set_f(smrt_t *h, const double *f)
{
    int rc = begin(h);
    if (rc != SMRT_OK) return rc;
    if (!f) return fail(h, SMRT_ERR_ARG, "smrt_set_f: f is NULL");
    DeviceGuard g(h->device);
    CUDA_TRY(h, g.err);
    const KernelTable &T = table_for(h->prec);
    HostParams p = host_params(h);
    void *state = h->buf[h->cur];
    const void *df = f;
    int k = classify(h, f, &df);
    if (k == -1) return fail(h, SMRT_ERR_ARG, "smrt_set_f: pointer on another device");
    CUDA_TRY(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
    if (k != 0) {
        CUDA_TRY(h, T.set_f(current_mode(h), state, (const double *)df, 0, h->ny, p, h->stream));
        if (k == 2) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        return SMRT_OK;
    }
    if ((rc = ensure_stage(h, 9)) != SMRT_OK) return rc;
    const int cr = chunk_rows(h, 9);
    const size_t nxb = (size_t)h->nx * sizeof(double);
    for (int r0 = 0; r0 < h->ny; r0 += cr) {
        int rows = (h->ny - r0 < cr) ? h->ny - r0 : cr;
        CUDA_TRY(h, cudaMemcpy2DAsync(h->d_stage, rows * nxb, f + (size_t)r0 * h->nx, (size_t)h->ny * nxb, rows * nxb, 9,
                                      cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(h, T.set_f(current_mode(h), state, h->d_stage, r0, rows, p, h->stream));
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SMRT_OK;
}

int smrt_init_macros(smrt_t *h, const double *rho, const double *u)
{
    int rc = begin(h);
    if (rc != SMRT_OK) return rc;
    if (!rho || !u) return fail(h, SMRT_ERR_ARG, "smrt_init_macros: rho and u are required");
    DeviceGuard g(h->device);
    CUDA_TRY(h, g.err);
    const KernelTable &T = table_for(h->prec);
    HostParams p = host_params(h);
    void *state = h->buf[h->cur];
    const void *drho = rho, *du = u;
    int kr = classify(h, rho, &drho), ku = classify(h, u, &du);
    if (kr == -1 || ku == -1) return fail(h, SMRT_ERR_ARG, "smrt_init_macros: pointer on another device");
    CUDA_TRY(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
    if (kr != 0 && ku != 0) {            // device memory, or page-locked host memory read directly
        CUDA_TRY(h, T.init_macros(current_mode(h), state, (const double *)drho, (const double *)du, 0, h->ny, p,
                                  h->stream));
        if (kr == 2 || ku == 2) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        return SMRT_OK;
    }
    if ((rc = ensure_stage(h, 3)) != SMRT_OK) return rc;
    const int cr = chunk_rows(h, 3);
    const size_t nxb = (size_t)h->nx * sizeof(double);
    for (int r0 = 0; r0 < h->ny; r0 += cr) {
        int rows = (h->ny - r0 < cr) ? h->ny - r0 : cr;
        double *srho = h->d_stage, *su = h->d_stage + (size_t)rows * h->nx;
        CUDA_TRY(h, cudaMemcpyAsync(srho, rho + (size_t)r0 * h->nx, rows * nxb,
                                    kr == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(h, cudaMemcpy2DAsync(su, rows * nxb, u + (size_t)r0 * h->nx, (size_t)h->ny * nxb, rows * nxb, 2,
                                      ku == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(h, T.init_macros(current_mode(h), state, srho, su, r0, rows, p, h->stream));
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return SMRT_OK;
}

long long smrt_time(const smrt_t *h)
{
    return h ? h->t : -1;
}

int smrt_set_time(smrt_t *h, long long t)
{
    if (!h) return SMRT_ERR_ARG;
    if (t < 0) return fail(h, SMRT_ERR_ARG, "smrt_set_time: t must be >= 0");
    if (h->layout == SMRT_LAYOUT_AA && h->ready && (t % 2) != (h->t % 2))
        return fail(h, SMRT_ERR_STATE, "smrt_set_time: the AA layout cannot change the parity of t");
    h->t = t;
    return SMRT_OK;
}

size_t smrt_device_bytes(const smrt_t *h)
{
    return h ? h->dev_bytes : 0;
}

const char *smrt_last_error(const smrt_t *h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

void smrt_destroy(smrt_t *h)
{
    if (!h) return;
    if (h->ready) {
        DeviceGuard g(h->device);
        cudaStreamSynchronize(h->stream);
        release(h);
    }
    delete h;
}

} // extern "C"
