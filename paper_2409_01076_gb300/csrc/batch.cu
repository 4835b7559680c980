// batch.cu -- many independent lattices ("cavities") of uneven size and
// viscosity advanced together (the C ABI smrt_batch_* of include/smrt.h).
//
// Every step is ONE launch of a persistent work-list kernel: a fixed grid
// (SM count x resident blocks) walks the concatenated step-block lists of the
// active lattices; each block runs the single-lattice step_block (the same
// code, hence the same bits, as smrt_step) on its lattice's own slice of one
// shared allocation.  smrt_batch_run captures check_every such launches plus a
// per-lattice residual pass in one CUDA graph and replays it; between replays
// the host retires converged, capped or diverged lattices by rewriting the
// work list in device memory (the graph stays valid: the kernels read the
// list's length from device memory).
#include <cuda_runtime.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <new>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace smrt {
namespace {

template <class C>
struct BatchCav {
    Params<C> p;       // the lattice's own parameters (flag -> its own divergence word)
    StepGeom geo;      // step-block geometry under the current tile shape
    long long offset;  // element offset of the lattice inside each population buffer
    long long uoff;    // node offset of the lattice inside the previous-velocity buffer
    int tiles_per_row; // residual tiles per row (256 nodes each)
};

constexpr int kResTile = 256;

// counts[0] = active lattices, counts[1] = total step blocks, counts[2] = total residual tiles.
// work[t] = (lattice, block of that lattice) for step block t of the concatenated list.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned int d = static_cast<unsigned int>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// CAP bounds the kernel to 64 registers (1024 resident threads per SM); without it the
// compiler takes what the step needs and fewer blocks are resident.
// EDGE: the two-buffer step also runs the edge column groups in the vector path (their geometry
// must say so); without it those columns stay in the band and the vector path carries no edge code.
template <int PREC, int KIND, int MODE, int VEC, int BX, bool CAP, bool EDGE, bool ROWSEG = false, bool CHUNK = false>
__global__ void __launch_bounds__(BX, CAP ? 1024 / BX : 1)
batch_step_kernel(const typename Prec<PREC>::R *src, typename Prec<PREC>::R *dst,
                  const BatchCav<typename Prec<PREC>::C> *__restrict__ cav, const int2 *__restrict__ work,
                  const int *__restrict__ counts)
{
    using Cav = BatchCav<typename Prec<PREC>::C>;
    static_assert(sizeof(Cav) % 8 == 0 && alignof(Cav) >= 8, "lattice record copied in 8-byte words");
    constexpr int kWords = (int)(sizeof(Cav) / 8);
    // A block walks the work list with the grid's stride (concurrent blocks hold neighbouring tiles,
    // whose rows they share in L2), or with CHUNK one contiguous run of ceil(total / grid) tiles (the
    // lattice rarely changes between consecutive tiles: better for many small lattices).  The
    // lattice record of the running tile sits in shared memory (buffer `buf`).  The work list is
    // read two tiles ahead; when the next tile belongs to another lattice its record is copied into
    // the other buffer with cp.async while this tile runs.  So neither the work list nor the record
    // is a dependent load in front of a tile's population loads, and the block synchronises only
    // where its walk crosses from one lattice to another.
    __shared__ __align__(16) unsigned long long rec[2][kWords];
    const int total = counts[1];
    const int G = gridDim.x;
    const int run = CHUNK ? (total + G - 1) / G : 0;
    const int stride = CHUNK ? 1 : G;
    int t = CHUNK ? blockIdx.x * run : blockIdx.x;
    const int tend = CHUNK ? min(t + run, total) : total;
    if (t >= tend) return;
    int2 w = work[t];
    for (int k = threadIdx.x; k < kWords; k += BX)
        rec[0][k] = reinterpret_cast<const unsigned long long *>(cav + w.x)[k];
    __syncthreads();
    int buf = 0;
    int tn = t + stride;
    int2 wn = (tn < tend) ? work[tn] : w;
    for (;;) {
        const int tnn = tn + stride;
        const int2 wnn = (tnn < tend) ? work[tnn] : wn;
        const bool next = tn < tend;
        const bool swap = next && wn.x != w.x;          // block-uniform
        if (swap) {
            const unsigned long long *g = reinterpret_cast<const unsigned long long *>(cav + wn.x);
            for (int k = threadIdx.x; k < kWords; k += BX) cp_async8(&rec[buf ^ 1][k], g + k);
        }
        const Cav &r = *reinterpret_cast<const Cav *>(rec[buf]);
        step_block<PREC, KIND, MODE, VEC, BX, EDGE, ROWSEG>(src + r.offset, dst + r.offset, r.p, r.geo, w.y);
        if (!next) break;
        if (swap) {
            cp_async_wait_all();
            __syncthreads();                           // the new record is visible to every thread
            buf ^= 1;
        }
        t = tn;
        w = wn;
        tn = tnn;
        wn = wnn;
    }
}

// Per-lattice residual pass over u(t) = moments of the canonical f(t): stores u(t)
// as u_prev; with `accumulate` it first sums |u(t) - u_prev|^2, |u(t)|^2 and rho(t)
// over the lattice's nodes.  One 256-node row segment per tile.
template <int PREC, int MODE>
__global__ void __launch_bounds__(kResTile)
batch_residual_kernel(const typename Prec<PREC>::R *state, const BatchCav<typename Prec<PREC>::C> *__restrict__ cav,
                      const int2 *__restrict__ rwork, const int *__restrict__ counts, double2 *uprev,
                      double *partials, int accumulate)
{
    __shared__ double red[kResTile / 32][3];
    const int total = counts[2];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int2 w = rwork[t];
        const BatchCav<typename Prec<PREC>::C> &L = cav[w.x];
        const int lt = w.y;
        const int j = lt / L.tiles_per_row;
        const int i = (lt % L.tiles_per_row) * kResTile + threadIdx.x;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        if (i < L.p.nx) {
            typename Prec<PREC>::C g[9];
            pull_canonical<PREC, MODE>(state + L.offset, L.p, i, j, g);
            double rr, ux, uy;
            moments_any(g, rr, ux, uy);
            double2 *up = uprev + L.uoff + (size_t)j * L.p.nx + i;
            const double2 old = *up;
            const double dx = ux - (double)old.x, dy = uy - (double)old.y;
            s0 = dx * dx + dy * dy;
            s1 = ux * ux + uy * uy;
            s2 = rr;
            *up = make_double2(ux, uy);
        }
        if (!accumulate) continue;
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        if ((threadIdx.x & 31) == 0) {
            red[threadIdx.x >> 5][0] = s0;
            red[threadIdx.x >> 5][1] = s1;
            red[threadIdx.x >> 5][2] = s2;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            double s = 0.0;
            for (int w = 0; w < kResTile / 32; ++w) s += red[w][threadIdx.x];
            partials[(size_t)t * 3 + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// One block per active lattice: fixed-order sum of its tiles' partials into sums[k][3].
__global__ void __launch_bounds__(256)
batch_finish_kernel(const int *__restrict__ act, const int *__restrict__ rpre, const int *__restrict__ counts,
                    const double *__restrict__ partials, double *sums)
{
    __shared__ double sh[3][256];
    const int c = blockIdx.x;
    if (c >= counts[0]) return;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int t = rpre[c] + threadIdx.x; t < rpre[c + 1]; t += 256) {
        a0 += partials[(size_t)t * 3 + 0];
        a1 += partials[(size_t)t * 3 + 1];
        a2 += partials[(size_t)t * 3 + 2];
    }
    sh[0][threadIdx.x] = a0;
    sh[1][threadIdx.x] = a1;
    sh[2][threadIdx.x] = a2;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x < 3) sums[(size_t)act[c] * 3 + threadIdx.x] = sh[threadIdx.x][0];
}

// ---- launch-shape candidates (the autotuner's search space) ----------------------

// A candidate is a base shape (nodes per thread, threads per block, 64-register bound) without
// (index k) or with (index k + nbase) the edge column groups in the vector path.  Measured on one
// GB300: the edge variant is faster on batches of lattices up to ~1024 wide (256^2: +20 %), the
// plain one on batches of 4096^2 lattices (the edge code costs the vector path a few per cent there).
// Row-segmented shapes (index 2 * nbase + m) cut the interior into row segments of the fewest lanes
// that cover a row (step_geom_seg): a warp works on 2 rows of a 128-wide lattice (FP32) or 4 of a
// 64-wide one at once, where a block of the other shapes leaves most of its lanes idle.
struct Shape {
    int vec, bx;
    bool cap;     // 64-register bound
    bool edge;    // edge column groups in the vector path (two-buffer layout)
    bool rowseg;  // row-segmented interior blocks
    bool chunk;   // each block walks one contiguous run of the work list
};
template <int PREC> struct Shapes;
template <> struct Shapes<SMRT_PREC_F32> {
    static constexpr int nbase = 5, nseg = 5, n = 2 * nbase + nseg;
    static Shape at(int k)
    {
        const Shape s[nbase] = {{4, 128, true, false, false}, {4, 64, true, false, false},
                                {4, 256, true, false, false}, {2, 128, true, false, false},
                                {4, 128, false, false, false}};
        const Shape g[nseg] = {{4, 128, true, true, true}, {4, 128, false, true, true}, {4, 256, true, true, true},
                               {4, 128, true, true, true, true}, {4, 256, true, true, true, true}};
        if (k >= 2 * nbase) return g[k - 2 * nbase];
        Shape r = s[k % nbase];
        r.edge = k >= nbase;
        return r;
    }
};
template <> struct Shapes<SMRT_PREC_F64> {
    static constexpr int nbase = 4, nseg = 1, n = 2 * nbase + nseg;
    static Shape at(int k)
    {
        const Shape s[nbase] = {{2, 128, true, false, false}, {2, 64, true, false, false},
                                {1, 128, true, false, false}, {2, 128, false, false, false}};
        const Shape g[nseg] = {{2, 128, true, true, true}};
        if (k >= 2 * nbase) return g[k - 2 * nbase];
        Shape r = s[k % nbase];
        r.edge = k >= nbase;
        return r;
    }
};

template <int PREC, int KIND, int MODE, int VEC, int BX, bool CAP = true, bool EDGE = false, bool ROWSEG = false,
          bool CHUNK = false>
cudaError_t launch_batch_step_shape(const void *src, void *dst, const void *cav, const int2 *work,
                                    const int *counts, int sms, cudaStream_t s)
{
    using P = Prec<PREC>;
    auto kern = batch_step_kernel<PREC, KIND, MODE, VEC, BX, CAP, EDGE, ROWSEG, CHUNK>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BX, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    kern<<<sms * per_sm, BX, 0, s>>>((const typename P::R *)src, (typename P::R *)dst,
                                      (const BatchCav<typename P::C> *)cav, work, counts);
    return cudaGetLastError();
}

template <int PREC, int KIND, int MODE>
cudaError_t launch_batch_step_m(int shape, const void *src, void *dst, const void *cav, const int2 *work,
                                const int *counts, int sms, cudaStream_t s)
{
    // the edge variants exist for the two-buffer step only (the in-place step never takes that path)
    constexpr bool E = MODE == MODE_AB;
    if constexpr (PREC == SMRT_PREC_F32) {
        switch (shape) {
        case 0: return launch_batch_step_shape<PREC, KIND, MODE, 4, 128>(src, dst, cav, work, counts, sms, s);
        case 1: return launch_batch_step_shape<PREC, KIND, MODE, 4, 64>(src, dst, cav, work, counts, sms, s);
        case 2: return launch_batch_step_shape<PREC, KIND, MODE, 4, 256>(src, dst, cav, work, counts, sms, s);
        case 3: return launch_batch_step_shape<PREC, KIND, MODE, 2, 128>(src, dst, cav, work, counts, sms, s);
        case 4: return launch_batch_step_shape<PREC, KIND, MODE, 4, 128, false>(src, dst, cav, work, counts, sms, s);
        case 5: return launch_batch_step_shape<PREC, KIND, MODE, 4, 128, true, E>(src, dst, cav, work, counts, sms, s);
        case 6: return launch_batch_step_shape<PREC, KIND, MODE, 4, 64, true, E>(src, dst, cav, work, counts, sms, s);
        case 7: return launch_batch_step_shape<PREC, KIND, MODE, 4, 256, true, E>(src, dst, cav, work, counts, sms, s);
        case 8: return launch_batch_step_shape<PREC, KIND, MODE, 2, 128, true, E>(src, dst, cav, work, counts, sms, s);
        case 9: return launch_batch_step_shape<PREC, KIND, MODE, 4, 128, false, E>(src, dst, cav, work, counts, sms, s);
        case 10:
            return launch_batch_step_shape<PREC, KIND, MODE, 4, 128, true, E, true>(src, dst, cav, work, counts, sms, s);
        case 11:
            return launch_batch_step_shape<PREC, KIND, MODE, 4, 128, false, E, true>(src, dst, cav, work, counts, sms, s);
        case 12:
            return launch_batch_step_shape<PREC, KIND, MODE, 4, 256, true, E, true>(src, dst, cav, work, counts, sms, s);
        case 13:
            return launch_batch_step_shape<PREC, KIND, MODE, 4, 128, true, E, true, true>(src, dst, cav, work, counts,
                                                                                          sms, s);
        case 14:
            return launch_batch_step_shape<PREC, KIND, MODE, 4, 256, true, E, true, true>(src, dst, cav, work, counts,
                                                                                          sms, s);
        }
    } else {
        switch (shape) {
        case 0: return launch_batch_step_shape<PREC, KIND, MODE, 2, 128>(src, dst, cav, work, counts, sms, s);
        case 1: return launch_batch_step_shape<PREC, KIND, MODE, 2, 64>(src, dst, cav, work, counts, sms, s);
        case 2: return launch_batch_step_shape<PREC, KIND, MODE, 1, 128>(src, dst, cav, work, counts, sms, s);
        case 3: return launch_batch_step_shape<PREC, KIND, MODE, 2, 128, false>(src, dst, cav, work, counts, sms, s);
        case 4: return launch_batch_step_shape<PREC, KIND, MODE, 2, 128, true, E>(src, dst, cav, work, counts, sms, s);
        case 5: return launch_batch_step_shape<PREC, KIND, MODE, 2, 64, true, E>(src, dst, cav, work, counts, sms, s);
        case 6: return launch_batch_step_shape<PREC, KIND, MODE, 1, 128, true, E>(src, dst, cav, work, counts, sms, s);
        case 7: return launch_batch_step_shape<PREC, KIND, MODE, 2, 128, false, E>(src, dst, cav, work, counts, sms, s);
        case 8:
            return launch_batch_step_shape<PREC, KIND, MODE, 2, 128, true, E, true>(src, dst, cav, work, counts, sms, s);
        }
    }
    return cudaErrorInvalidValue;
}

template <int PREC>
cudaError_t launch_batch_step(int kind, int mode, int shape, const void *src, void *dst, const void *cav,
                              const int2 *work, const int *counts, int sms, cudaStream_t s)
{
#define SMRT_BATCH_MODES(K)                                                                                   \
    switch (mode) {                                                                                           \
    case MODE_AB: return launch_batch_step_m<PREC, K, MODE_AB>(shape, src, dst, cav, work, counts, sms, s);    \
    case MODE_AA_EVEN: return launch_batch_step_m<PREC, K, MODE_AA_EVEN>(shape, src, dst, cav, work, counts, sms, s); \
    case MODE_AA_ODD: return launch_batch_step_m<PREC, K, MODE_AA_ODD>(shape, src, dst, cav, work, counts, sms, s); \
    }                                                                                                         \
    return cudaErrorInvalidValue;
    if (kind == SMRT_COLLISION_SMRT) { SMRT_BATCH_MODES(SMRT_COLLISION_SMRT) }
    SMRT_BATCH_MODES(SMRT_COLLISION_SRT)
#undef SMRT_BATCH_MODES
}

// accumulate == 0: snapshot u(t) only; accumulate == 1: also sum against the snapshot
// and reduce the sums per lattice.
template <int PREC>
cudaError_t launch_batch_residual(int mode, int accumulate, const void *state, const void *cav, const int *act,
                                  const int *rpre, const int2 *rwork, const int *counts, double2 *uprev,
                                  double *partials, double *sums, int count, int sms, cudaStream_t s)
{
    using P = Prec<PREC>;
    const int grid = sms * 4;
    switch (mode) {
    case MODE_AB:
        batch_residual_kernel<PREC, MODE_AB><<<grid, kResTile, 0, s>>>(
            (const typename P::R *)state, (const BatchCav<typename P::C> *)cav, rwork, counts, uprev, partials,
            accumulate);
        break;
    case MODE_AA_EVEN:
        batch_residual_kernel<PREC, MODE_AA_EVEN><<<grid, kResTile, 0, s>>>(
            (const typename P::R *)state, (const BatchCav<typename P::C> *)cav, rwork, counts, uprev, partials,
            accumulate);
        break;
    default:
        batch_residual_kernel<PREC, MODE_AA_ODD><<<grid, kResTile, 0, s>>>(
            (const typename P::R *)state, (const BatchCav<typename P::C> *)cav, rwork, counts, uprev, partials,
            accumulate);
        break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !accumulate) return e;
    batch_finish_kernel<<<count, 256, 0, s>>>(act, rpre, counts, partials, sums);
    return cudaGetLastError();
}

template <int PREC>
size_t cav_bytes()
{
    return sizeof(BatchCav<typename Prec<PREC>::C>);
}

template <int PREC>
StepGeom geom_for(int shape, int nx, int ny, bool edge_in)
{
    Shape sh = Shapes<PREC>::at(shape);
    edge_in = edge_in && sh.edge;
    if (sh.rowseg) {
        if (sh.vec == 4 && sh.bx == 256) return step_geom_seg<4, 256>(nx, ny, edge_in);
        if (sh.vec == 4) return step_geom_seg<4, 128>(nx, ny, edge_in);
        return step_geom_seg<2, 128>(nx, ny, edge_in);
    }
    if (sh.vec == 4 && sh.bx == 128) return step_geom<4, 128>(nx, ny, edge_in);
    if (sh.vec == 4 && sh.bx == 64) return step_geom<4, 64>(nx, ny, edge_in);
    if (sh.vec == 4 && sh.bx == 256) return step_geom<4, 256>(nx, ny, edge_in);
    if (sh.vec == 2 && sh.bx == 128) return step_geom<2, 128>(nx, ny, edge_in);
    if (sh.vec == 2 && sh.bx == 64) return step_geom<2, 64>(nx, ny, edge_in);
    return step_geom<1, 128>(nx, ny, edge_in);
}

template <int PREC>
int step_blocks(int shape, const StepGeom &g)
{
    const int bx = Shapes<PREC>::at(shape).bx;
    return g.n_int_blocks + (int)((g.n_edge + bx - 1) / bx);
}

// Fill the device descriptor of one lattice (host side).
template <int PREC>
void fill_cav(void *dst, const HostParams &hp, const StepGeom &geo, long long offset, long long uoff)
{
    using C = typename Prec<PREC>::C;
    BatchCav<C> c;
    c.p = make_params<C>(hp);
    c.geo = geo;
    c.offset = offset;
    c.uoff = uoff;
    c.tiles_per_row = (hp.nx + kResTile - 1) / kResTile;
    memcpy(dst, &c, sizeof(c));
}

} // namespace
} // namespace smrt

// ---------------------------------------------------------------------------------------
// host side

namespace {

using smrt::HostParams;
using smrt::MODE_AA_EVEN;
using smrt::MODE_AA_ODD;
using smrt::MODE_AB;

enum { ST_ACTIVE = 0, ST_CONVERGED = 1, ST_CAPPED = 2, ST_DIVERGED = 3 };

struct Lat {
    int nx, ny, pitch;
    long long plane, offset, nodes, uoff;
    double tau, u_lid;
    long long t = 0;
    int cur = 0;               // AB: buffer holding this lattice's state
    int state = ST_ACTIVE;
    double resid = -1.0;
};

} // namespace

struct smrt_batch_t {
    int count = 0;
    unsigned bc = 0;
    int prec = SMRT_PREC_F32;
    int layout = SMRT_LAYOUT_AB;
    int collision = SMRT_COLLISION_SMRT;
    int shape = 0;
    int sms = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<Lat> lat;
    size_t elem = 4;
    long long total_elems = 0, total_nodes = 0;
    int cur = 0;               // AB: buffer holding the active lattices' state
    void *buf[2] = {nullptr, nullptr};
    void *d_cav = nullptr;
    std::vector<unsigned char> h_cav;
    int *d_act = nullptr, *d_rpre = nullptr, *d_counts = nullptr, *d_flags = nullptr;
    int2 *d_work = nullptr, *d_rwork = nullptr;   // (lattice, block) per step block / residual tile
    int *h_flags = nullptr;
    double2 *d_uprev = nullptr;
    double *d_partials = nullptr, *d_sums = nullptr, *h_sums = nullptr;
    long long max_tiles = 0, max_work = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_k = 0, graph_mode = -1, graph_shape = -1, graph_kind = -1;
    bool list_dirty = true;
    std::string err = "no error";
};

namespace {

int bfail(smrt_batch_t *b, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else smrt::set_thread_error(buf);
    return code;
}

#define BTRY(b, call)                                                                                       \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) return bfail((b), SMRT_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

HostParams lat_params(const smrt_batch_t *b, int k)
{
    const Lat &L = b->lat[k];
    HostParams p;
    p.nx = L.nx;
    p.ny = L.ny;
    p.pitch = L.pitch;
    p.plane = L.plane;
    p.bc = b->bc;
    p.tau = L.tau;
    p.tau_s = 1.0;
    p.u_lid = L.u_lid;
    p.flag = b->d_flags + k;
    return p;
}

int mode_of(const smrt_batch_t *b, long long t)
{
    if (b->layout == SMRT_LAYOUT_AB) return MODE_AB;
    return (t % 2 == 0) ? MODE_AA_EVEN : MODE_AA_ODD;
}

const smrt::KernelTable &table(int prec)
{
    return prec == SMRT_PREC_F64 ? smrt::kernels_f64() : smrt::kernels_f32();
}

int nshapes(int prec)
{
    return prec == SMRT_PREC_F64 ? smrt::Shapes<SMRT_PREC_F64>::n : smrt::Shapes<SMRT_PREC_F32>::n;
}

// Rebuild descriptors (for the current tile shape) and the work lists of the active lattices.
int upload_lists(smrt_batch_t *b)
{
    const size_t cb = b->prec == SMRT_PREC_F64 ? smrt::cav_bytes<SMRT_PREC_F64>() : smrt::cav_bytes<SMRT_PREC_F32>();
    b->h_cav.resize(cb * b->count);
    std::vector<int> act, rpre(1, 0);
    std::vector<int2> work, rwork;
    for (int k = 0; k < b->count; ++k) {
        const Lat &L = b->lat[k];
        HostParams hp = lat_params(b, k);
        smrt::StepGeom g;
        int nb;
        if (b->prec == SMRT_PREC_F64) {
            g = smrt::geom_for<SMRT_PREC_F64>(b->shape, L.nx, L.ny, b->layout == SMRT_LAYOUT_AB);
            nb = smrt::step_blocks<SMRT_PREC_F64>(b->shape, g);
            smrt::fill_cav<SMRT_PREC_F64>(&b->h_cav[cb * k], hp, g, L.offset, L.uoff);
        } else {
            g = smrt::geom_for<SMRT_PREC_F32>(b->shape, L.nx, L.ny, b->layout == SMRT_LAYOUT_AB);
            nb = smrt::step_blocks<SMRT_PREC_F32>(b->shape, g);
            smrt::fill_cav<SMRT_PREC_F32>(&b->h_cav[cb * k], hp, g, L.offset, L.uoff);
        }
        if (L.state != ST_ACTIVE) continue;
        act.push_back(k);
        for (int j = 0; j < nb; ++j) work.push_back(make_int2(k, j));
        const int tiles = L.ny * ((L.nx + smrt::kResTile - 1) / smrt::kResTile);
        for (int j = 0; j < tiles; ++j) rwork.push_back(make_int2(k, j));
        rpre.push_back(rpre.back() + tiles);
    }
    if ((long long)work.size() > b->max_work || (long long)rwork.size() > b->max_tiles)
        return bfail(b, SMRT_ERR_STATE, "work list exceeds its allocation");
    int counts[3] = {(int)act.size(), (int)work.size(), rpre.back()};
    BTRY(b, cudaMemcpyAsync(b->d_cav, b->h_cav.data(), b->h_cav.size(), cudaMemcpyHostToDevice, b->stream));
    if (!act.empty()) {
        BTRY(b, cudaMemcpyAsync(b->d_act, act.data(), act.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
        BTRY(b, cudaMemcpyAsync(b->d_rpre, rpre.data(), rpre.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
        BTRY(b, cudaMemcpyAsync(b->d_work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
        BTRY(b, cudaMemcpyAsync(b->d_rwork, rwork.data(), rwork.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                b->stream));
    }
    BTRY(b, cudaMemcpyAsync(b->d_counts, counts, sizeof(counts), cudaMemcpyHostToDevice, b->stream));
    // the host arrays are stack/vector temporaries: wait until the copies have read them
    BTRY(b, cudaStreamSynchronize(b->stream));
    b->list_dirty = false;
    return SMRT_OK;
}

int active_count(const smrt_batch_t *b)
{
    int n = 0;
    for (const Lat &L : b->lat) n += (L.state == ST_ACTIVE);
    return n;
}

long long active_t(const smrt_batch_t *b)
{
    for (const Lat &L : b->lat)
        if (L.state == ST_ACTIVE) return L.t;
    return 0;
}

// Enqueue one step of every active lattice.
cudaError_t enqueue_step(smrt_batch_t *b, long long t)
{
    const int mode = mode_of(b, t);
    const void *src = b->buf[b->layout == SMRT_LAYOUT_AB ? b->cur : 0];
    void *dst = b->buf[b->layout == SMRT_LAYOUT_AB ? 1 - b->cur : 0];
    if (b->prec == SMRT_PREC_F64)
        return smrt::launch_batch_step<SMRT_PREC_F64>(b->collision, mode, b->shape, src, dst, b->d_cav, b->d_work,
                                                     b->d_counts, b->sms, b->stream);
    return smrt::launch_batch_step<SMRT_PREC_F32>(b->collision, mode, b->shape, src, dst, b->d_cav, b->d_work,
                                                 b->d_counts, b->sms, b->stream);
}

cudaError_t enqueue_residual(smrt_batch_t *b, long long t, int cur, int accumulate)
{
    const int mode = mode_of(b, t);
    const void *state = b->buf[b->layout == SMRT_LAYOUT_AB ? cur : 0];
    if (b->prec == SMRT_PREC_F64)
        return smrt::launch_batch_residual<SMRT_PREC_F64>(mode, accumulate, state, b->d_cav, b->d_act, b->d_rpre,
                                                         b->d_rwork, b->d_counts, b->d_uprev, b->d_partials,
                                                         b->d_sums, b->count, b->sms, b->stream);
    return smrt::launch_batch_residual<SMRT_PREC_F32>(mode, accumulate, state, b->d_cav, b->d_act, b->d_rpre,
                                                     b->d_rwork, b->d_counts, b->d_uprev, b->d_partials, b->d_sums,
                                                     b->count, b->sms, b->stream);
}

void drop_graph(smrt_batch_t *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_k = 0;
}

void* lattice_state(smrt_batch_t *b, int k)
{
    const void *base = b->buf[b->layout == SMRT_LAYOUT_AB ? b->lat[k].cur : 0];
    return (char *)base + (size_t)b->lat[k].offset * b->elem;
}

int check_index(smrt_batch_t *b, int k)
{
    if (!b) return SMRT_ERR_ARG;
    if (k < 0 || k >= b->count) return bfail(b, SMRT_ERR_ARG, "lattice index %d out of range [0, %d)", k, b->count);
    return SMRT_OK;
}

} // namespace

extern "C" {

int smrt_batch_create(int count, const int *nx, const int *ny, const double *tau, const double *u_lid,
                      unsigned bc_flags, int precision, int layout, int collision, smrt_batch_t **out)
{
    if (!out) return bfail(nullptr, SMRT_ERR_ARG, "smrt_batch_create: out is NULL");
    *out = nullptr;
    if (count < 1 || !nx || !ny || !tau || !u_lid)
        return bfail(nullptr, SMRT_ERR_ARG, "smrt_batch_create: need count >= 1 and the four arrays");
    if (precision != SMRT_PREC_F32 && precision != SMRT_PREC_F64)
        return bfail(nullptr, SMRT_ERR_ARG, "smrt_batch_create: precision must be F32 or F64");
    if (layout != SMRT_LAYOUT_AB && layout != SMRT_LAYOUT_AA)
        return bfail(nullptr, SMRT_ERR_ARG, "smrt_batch_create: unknown layout %d", layout);
    if (collision != SMRT_COLLISION_SMRT && collision != SMRT_COLLISION_SRT)
        return bfail(nullptr, SMRT_ERR_ARG, "smrt_batch_create: collision must be SMRT or SRT");
    if (bc_flags >> 8) return bfail(nullptr, SMRT_ERR_ARG, "smrt_batch_create: invalid bc_flags");
    for (int s = 0; s < 4; ++s)
        if (((bc_flags >> (2 * s)) & 3u) > SMRT_BC_MOVING) return bfail(nullptr, SMRT_ERR_ARG, "invalid bc_flags");
    if ((((bc_flags & 3u) == 0) != (((bc_flags >> 2) & 3u) == 0)) ||
        ((((bc_flags >> 4) & 3u) == 0) != (((bc_flags >> 6) & 3u) == 0)))
        return bfail(nullptr, SMRT_ERR_ARG, "smrt_batch_create: periodic sides must be paired");
    smrt_batch_t *b = new (std::nothrow) smrt_batch_t;
    if (!b) return bfail(nullptr, SMRT_ERR_OOM, "smrt_batch_create: out of host memory");
    b->count = count;
    b->bc = bc_flags;
    b->prec = precision;
    b->layout = layout;
    b->collision = collision;
    b->elem = precision == SMRT_PREC_F64 ? 8 : 4;
    const long long per = 128 / (long long)b->elem;
    long long off = 0, uoff = 0, tiles = 0;
    for (int k = 0; k < count; ++k) {
        if (nx[k] < 2 || ny[k] < 2 || !(tau[k] > 0.5) || !isfinite(tau[k]) || !isfinite(u_lid[k]) ||
            fabs(u_lid[k]) >= 1.0 / sqrt(3.0)) {
            delete b;
            return bfail(nullptr, SMRT_ERR_ARG, "smrt_batch_create: lattice %d has invalid size, tau or u_lid", k);
        }
        Lat L;
        L.nx = nx[k];
        L.ny = ny[k];
        L.pitch = (int)((nx[k] + per - 1) / per * per);
        L.plane = (long long)L.pitch * ny[k];
        L.offset = off;
        L.nodes = (long long)nx[k] * ny[k];
        L.uoff = uoff;
        L.tau = tau[k];
        L.u_lid = u_lid[k];
        off += 9 * L.plane;
        uoff += L.nodes;
        tiles += (long long)ny[k] * ((nx[k] + smrt::kResTile - 1) / smrt::kResTile);
        b->lat.push_back(L);
    }
    if (tiles >= (1LL << 31) || off >= (1LL << 40)) {
        delete b;
        return bfail(nullptr, SMRT_ERR_ARG, "smrt_batch_create: batch too large");
    }
    b->total_elems = off;
    b->total_nodes = uoff;
    b->max_tiles = tiles;
    for (int s = 0; s < nshapes(precision); ++s) {        // the largest step-block list of any tile shape
        long long w = 0;
        for (const Lat &L : b->lat)
            w += precision == SMRT_PREC_F64
                     ? smrt::step_blocks<SMRT_PREC_F64>(s, smrt::geom_for<SMRT_PREC_F64>(s, L.nx, L.ny,
                                                                                         layout == SMRT_LAYOUT_AB))
                     : smrt::step_blocks<SMRT_PREC_F32>(s, smrt::geom_for<SMRT_PREC_F32>(s, L.nx, L.ny,
                                                                                         layout == SMRT_LAYOUT_AB));
        if (w > b->max_work) b->max_work = w;
    }
    if (b->max_work >= (1LL << 31)) {
        delete b;
        return bfail(nullptr, SMRT_ERR_ARG, "smrt_batch_create: batch too large");
    }

    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    const int nbuf = layout == SMRT_LAYOUT_AB ? 2 : 1;
    const size_t cb = precision == SMRT_PREC_F64 ? smrt::cav_bytes<SMRT_PREC_F64>() : smrt::cav_bytes<SMRT_PREC_F32>();
    for (int k = 0; k < nbuf && e == cudaSuccess; ++k) e = cudaMalloc(&b->buf[k], (size_t)off * b->elem);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_cav, cb * count);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_act, sizeof(int) * count);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_rpre, sizeof(int) * (count + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_work, sizeof(int2) * (size_t)b->max_work);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_rwork, sizeof(int2) * (size_t)tiles);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_counts, sizeof(int) * 3);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_flags, sizeof(int) * count);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_uprev, sizeof(double2) * (size_t)uoff);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_partials, sizeof(double) * 3 * (size_t)tiles);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_sums, sizeof(double) * 3 * count);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_sums, sizeof(double) * 3 * count);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_flags, sizeof(int) * count);
    if (e == cudaSuccess) e = cudaMemset(b->d_flags, 0, sizeof(int) * count);
    if (e == cudaSuccess) e = cudaMemset(b->d_uprev, 0, sizeof(double2) * (size_t)uoff);
    if (e != cudaSuccess) {
        cudaGetLastError();
        smrt_batch_destroy(b);
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? SMRT_ERR_OOM : SMRT_ERR_CUDA,
                     "smrt_batch_create: %s", cudaGetErrorString(e));
    }
    int rc = upload_lists(b);
    // f(0) = f^eq(1, 0) in every lattice
    for (int k = 0; rc == SMRT_OK && k < count; ++k) {
        HostParams hp = lat_params(b, k);
        e = table(precision).init_macros(mode_of(b, 0), lattice_state(b, k), nullptr, nullptr, 0, b->lat[k].ny, hp,
                                         b->stream);
        if (e != cudaSuccess) rc = bfail(b, SMRT_ERR_CUDA, "initial state: %s", cudaGetErrorString(e));
    }
    if (rc == SMRT_OK && (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
        rc = bfail(b, SMRT_ERR_CUDA, "initial state: %s", cudaGetErrorString(e));
    if (rc != SMRT_OK) {
        smrt::set_thread_error(b->err.c_str());
        smrt_batch_destroy(b);
        return rc;
    }
    *out = b;
    return SMRT_OK;
}

int smrt_batch_set_stream(smrt_batch_t *b, void *stream)
{
    if (!b) return SMRT_ERR_ARG;
    drop_graph(b);
    b->stream = (cudaStream_t)stream;
    return SMRT_OK;
}

int smrt_batch_set_shape(smrt_batch_t *b, int shape)
{
    if (!b) return SMRT_ERR_ARG;
    if (shape < 0 || shape >= nshapes(b->prec))
        return bfail(b, SMRT_ERR_ARG, "smrt_batch_set_shape: shape %d not in [0, %d)", shape, nshapes(b->prec));
    drop_graph(b);
    b->shape = shape;
    b->list_dirty = true;
    return SMRT_OK;
}

int smrt_batch_step(smrt_batch_t *b, long long n)
{
    smrt::TraceRange trace("smrt_batch_step");
    if (!b) return SMRT_ERR_ARG;
    if (n < 0) return bfail(b, SMRT_ERR_ARG, "smrt_batch_step: n must be >= 0");
    if (b->list_dirty) {
        int rc = upload_lists(b);
        if (rc != SMRT_OK) return rc;
    }
    long long t = active_t(b);
    for (long long s = 0; s < n; ++s, ++t) {
        cudaError_t e = enqueue_step(b, t);
        if (e != cudaSuccess) return bfail(b, SMRT_ERR_CUDA, "batch step launch: %s", cudaGetErrorString(e));
        if (b->layout == SMRT_LAYOUT_AB) b->cur = 1 - b->cur;
    }
    for (Lat &L : b->lat)
        if (L.state == ST_ACTIVE) {
            L.t += n;
            L.cur = b->cur;
        }
    BTRY(b, cudaMemcpyAsync(b->h_flags, b->d_flags, sizeof(int) * b->count, cudaMemcpyDeviceToHost, b->stream));
    BTRY(b, cudaStreamSynchronize(b->stream));
    for (int k = 0; k < b->count; ++k)
        if (b->h_flags[k] && b->lat[k].state == ST_ACTIVE) {
            b->lat[k].state = ST_DIVERGED;
            b->list_dirty = true;
        }
    return SMRT_OK;
}

int smrt_batch_autotune(smrt_batch_t *b, int steps, int *choice)
{
    if (!b) return SMRT_ERR_ARG;
    if (steps < 2) return bfail(b, SMRT_ERR_ARG, "smrt_batch_autotune: steps must be >= 2");
    steps += steps % 2;                 // AB: leave the state in its buffer
    drop_graph(b);
    // time each candidate on a scratch copy of the state so the lattices do not advance
    const int nbuf = b->layout == SMRT_LAYOUT_AB ? 2 : 1;
    void *save = nullptr;
    BTRY(b, cudaMalloc(&save, (size_t)b->total_elems * b->elem));
    const void *live = b->buf[b->layout == SMRT_LAYOUT_AB ? b->cur : 0];
    cudaError_t e = cudaMemcpyAsync(save, live, (size_t)b->total_elems * b->elem, cudaMemcpyDeviceToDevice, b->stream);
    float best = 1e30f;
    int best_shape = b->shape;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int orig_cur = b->cur;
    const long long t0 = active_t(b);
    for (int sh = 0; e == cudaSuccess && sh < nshapes(b->prec); ++sh) {
        b->shape = sh;
        int rc = upload_lists(b);
        if (rc != SMRT_OK) { e = cudaErrorUnknown; break; }
        long long t = t0;
        e = enqueue_step(b, t);              // warm-up launch
        if (b->layout == SMRT_LAYOUT_AB) b->cur = 1 - b->cur;
        ++t;
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        for (int s = 0; e == cudaSuccess && s < steps; ++s, ++t) {
            e = enqueue_step(b, t);
            if (b->layout == SMRT_LAYOUT_AB) b->cur = 1 - b->cur;
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) {
            best = ms;
            best_shape = sh;
        }
        // restore the state (and the AA parity / AB buffer) for the next candidate
        b->cur = orig_cur;
        void *dst = b->buf[b->layout == SMRT_LAYOUT_AB ? b->cur : 0];
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dst, save, (size_t)b->total_elems * b->elem, cudaMemcpyDeviceToDevice, b->stream);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaError_t e2 = cudaStreamSynchronize(b->stream);
    cudaFree(save);
    if (e == cudaSuccess) e = e2;
    (void)nbuf;
    // the divergence words may have been set by a candidate run on the copy: clear them
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_flags, 0, sizeof(int) * b->count, b->stream);
    b->shape = best_shape;
    int rc = upload_lists(b);
    if (e != cudaSuccess) return bfail(b, SMRT_ERR_CUDA, "smrt_batch_autotune: %s", cudaGetErrorString(e));
    if (rc != SMRT_OK) return rc;
    if (choice) *choice = best_shape;
    return SMRT_OK;
}

int smrt_batch_run(smrt_batch_t *b, double tol, long long check_every, long long max_steps, int residual_kind,
                   int *n_active)
{
    smrt::TraceRange trace("smrt_batch_run");
    if (!b) return SMRT_ERR_ARG;
    if (!(tol > 0.0) || check_every < 1 || max_steps < 0)
        return bfail(b, SMRT_ERR_ARG, "smrt_batch_run: need tol > 0, check_every >= 1, max_steps >= 0");
    if (residual_kind != SMRT_BATCH_RESIDUAL_STEP && residual_kind != SMRT_BATCH_RESIDUAL_STRIDE)
        return bfail(b, SMRT_ERR_ARG, "smrt_batch_run: unknown residual kind %d", residual_kind);
    check_every += check_every % 2;
    if (b->list_dirty) {
        int rc = upload_lists(b);
        if (rc != SMRT_OK) return rc;
    }
    const bool stride = residual_kind == SMRT_BATCH_RESIDUAL_STRIDE;
    if (stride)   // the first check of this run compares against zero velocity (never converged)
        BTRY(b, cudaMemsetAsync(b->d_uprev, 0, sizeof(double2) * (size_t)b->total_nodes, b->stream));
    long long t = active_t(b);
    // (re)capture: check_every steps + residual pass + copies of the sums and flags
    if (!b->graph || b->graph_k != check_every || b->graph_shape != b->shape || b->graph_mode != mode_of(b, t) ||
        b->graph_kind != residual_kind) {
        drop_graph(b);
        cudaStream_t cap = nullptr;
        BTRY(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaStream_t user = b->stream;
        b->stream = cap;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        int cur0 = b->cur;
        // one-step: check_every - 1 updates, snapshot u, one more update, compare;
        // stride: check_every updates, compare with the previous check's snapshot
        for (long long s = 0; e == cudaSuccess && s < check_every; ++s) {
            if (!stride && s == check_every - 1) e = enqueue_residual(b, t + s, b->cur, 0);
            if (e == cudaSuccess) e = enqueue_step(b, t + s);
            if (b->layout == SMRT_LAYOUT_AB) b->cur = 1 - b->cur;
        }
        if (e == cudaSuccess) e = enqueue_residual(b, t + check_every, b->cur, 1);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->h_sums, b->d_sums, sizeof(double) * 3 * b->count, cudaMemcpyDeviceToHost, cap);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->h_flags, b->d_flags, sizeof(int) * b->count, cudaMemcpyDeviceToHost, cap);
        cudaError_t e_end = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e_end;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        b->stream = user;
        b->cur = cur0;
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            b->graph = nullptr;
            return bfail(b, SMRT_ERR_CUDA, "smrt_batch_run: graph capture: %s", cudaGetErrorString(e));
        }
        b->graph_k = (int)check_every;
        b->graph_shape = b->shape;
        b->graph_mode = mode_of(b, t);
        b->graph_kind = residual_kind;
    }
    const double divisor = stride ? (double)check_every : 1.0;
    while (active_count(b) > 0) {
        BTRY(b, cudaGraphLaunch(b->graph, b->stream));
        BTRY(b, cudaStreamSynchronize(b->stream));
        // check_every is even, so the AB buffer holding the state is unchanged
        bool changed = false;
        for (int k = 0; k < b->count; ++k) {
            Lat &L = b->lat[k];
            if (L.state != ST_ACTIVE) continue;
            L.t += check_every;
            const double d2 = b->h_sums[3 * k], u2 = b->h_sums[3 * k + 1];
            L.resid = (d2 == 0.0 && u2 == 0.0) ? 0.0 : sqrt(d2) / (sqrt(u2) * divisor);
            if (b->h_flags[k] || !isfinite(L.resid)) L.state = ST_DIVERGED;
            else if (L.resid < tol) L.state = ST_CONVERGED;
            else if (L.t >= max_steps) L.state = ST_CAPPED;
            changed |= (L.state != ST_ACTIVE);
        }
        if (changed) {
            int rc = upload_lists(b);
            if (rc != SMRT_OK) return rc;
        }
    }
    if (n_active) *n_active = active_count(b);
    return SMRT_OK;
}

int smrt_batch_status(const smrt_batch_t *b, long long *steps, double *residual, int *state)
{
    if (!b) return SMRT_ERR_ARG;
    for (int k = 0; k < b->count; ++k) {
        if (steps) steps[k] = b->lat[k].t;
        if (residual) residual[k] = b->lat[k].resid;
        if (state) state[k] = b->lat[k].state;
    }
    return SMRT_OK;
}

int smrt_batch_get_f(smrt_batch_t *b, int k, double *f)
{
    int rc = check_index(b, k);
    if (rc != SMRT_OK) return rc;
    if (!f) return bfail(b, SMRT_ERR_ARG, "smrt_batch_get_f: f is NULL");
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, f);
    cudaGetLastError();
    const bool dev = e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    const Lat &L = b->lat[k];
    HostParams hp = lat_params(b, k);
    double *out = f;
    if (!dev) BTRY(b, cudaMalloc((void **)&out, sizeof(double) * 9 * (size_t)L.nodes));
    e = table(b->prec).get_f(mode_of(b, L.t), lattice_state(b, k), out, 0, L.ny, hp, b->stream);
    if (e == cudaSuccess && !dev)
        e = cudaMemcpyAsync(f, out, sizeof(double) * 9 * (size_t)L.nodes, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (!dev) cudaFree(out);
    if (e != cudaSuccess) return bfail(b, SMRT_ERR_CUDA, "smrt_batch_get_f: %s", cudaGetErrorString(e));
    return SMRT_OK;
}

int smrt_batch_macros(smrt_batch_t *b, int k, double *rho, double *u)
{
    int rc = check_index(b, k);
    if (rc != SMRT_OK) return rc;
    if (!rho || !u) return bfail(b, SMRT_ERR_ARG, "smrt_batch_macros: rho and u are required");
    const Lat &L = b->lat[k];
    HostParams hp = lat_params(b, k);
    double *tmp = nullptr;
    BTRY(b, cudaMalloc((void **)&tmp, sizeof(double) * 3 * (size_t)L.nodes));
    cudaError_t e = table(b->prec).macros(mode_of(b, L.t), lattice_state(b, k), tmp, tmp + L.nodes, 0, L.ny, hp,
                                          b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rho, tmp, sizeof(double) * (size_t)L.nodes, cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(u, tmp + L.nodes, sizeof(double) * 2 * (size_t)L.nodes, cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return bfail(b, SMRT_ERR_CUDA, "smrt_batch_macros: %s", cudaGetErrorString(e));
    return SMRT_OK;
}

int smrt_batch_init_macros(smrt_batch_t *b, int k, const double *rho, const double *u)
{
    int rc = check_index(b, k);
    if (rc != SMRT_OK) return rc;
    if (!rho || !u) return bfail(b, SMRT_ERR_ARG, "smrt_batch_init_macros: rho and u are required");
    const Lat &L = b->lat[k];
    if (L.state != ST_ACTIVE || L.t != active_t(b))
        return bfail(b, SMRT_ERR_STATE, "smrt_batch_init_macros: lattice %d is retired", k);
    HostParams hp = lat_params(b, k);
    double *tmp = nullptr;
    BTRY(b, cudaMalloc((void **)&tmp, sizeof(double) * 3 * (size_t)L.nodes));
    cudaError_t e = cudaMemcpyAsync(tmp, rho, sizeof(double) * (size_t)L.nodes, cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tmp + L.nodes, u, sizeof(double) * 2 * (size_t)L.nodes, cudaMemcpyDefault, b->stream);
    if (e == cudaSuccess)
        e = table(b->prec).init_macros(mode_of(b, L.t), lattice_state(b, k), tmp, tmp + L.nodes, 0, L.ny, hp,
                                       b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return bfail(b, SMRT_ERR_CUDA, "smrt_batch_init_macros: %s", cudaGetErrorString(e));
    return SMRT_OK;
}

long long smrt_batch_nodes(const smrt_batch_t *b)
{
    return b ? b->total_nodes : -1;
}

const char *smrt_batch_last_error(const smrt_batch_t *b)
{
    return b ? b->err.c_str() : smrt_last_error(nullptr);
}

void smrt_batch_destroy(smrt_batch_t *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (int k = 0; k < 2; ++k)
        if (b->buf[k]) cudaFree(b->buf[k]);
    void *dev[] = {b->d_cav, b->d_act, b->d_rpre, b->d_work, b->d_rwork, b->d_counts, b->d_flags, b->d_uprev,
                   b->d_partials, b->d_sums};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (b->h_sums) cudaFreeHost(b->h_sums);
    if (b->h_flags) cudaFreeHost(b->h_flags);
    delete b;
}

} // extern "C"
