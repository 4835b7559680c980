// kernels.cuh -- kernel templates and launchers, instantiated once per storage
// precision by prec_*.cu.
//
// Fused step (one launch per time step): every node pulls its nine canonical
// populations f_a(x) (streaming + halfway / moving-wall bounce-back), forms the
// moments and f^eq, applies the collision and stores f*.  Blocks come in two
// kinds inside one grid:
//   - interior blocks: rows 1..ny-2, columns [L, R); each thread owns VEC
//     consecutive nodes, loads each population row with one aligned VEC-wide
//     vector load and gets the +-1 column shift from its warp neighbour with a
//     shuffle (one extra scalar load at each warp edge); no boundary logic;
//   - band blocks: the remaining ring of nodes (rows 0 and ny-1, columns [0, L)
//     and [R, nx)), one node per thread, with the full boundary resolution.
//     In the two-buffer layout L = 0 and R = nx (when nx % VEC == 0): the edge
//     column groups run in the vector path and fix up their boundary pulls.
#pragma once

#include "d2q9.cuh"

namespace smrt {

template <class R, int VEC>
struct alignas(sizeof(R) * VEC) RVec {
    R v[VEC];
};

constexpr unsigned kFull = 0xffffffffu;

struct StepGeom {
    int L, R;            // interior columns [L, R), multiples of VEC
    int bpr;             // interior blocks per row
    int n_int_blocks;    // bpr * (ny - 2), or the row-segment blocks (below)
    long long n_edge;    // band nodes
    // row-segmented blocks only (step_block<..., ROWSEG = true>): a row segment is `seg` lanes
    // (a power of two <= 32) owning seg * VEC consecutive columns; a row holds `spr` segments,
    // the interior `tasks` = (ny - 2) * spr of them, and a block of BX threads takes BX / seg.
    int seg_log2, spr, tasks;
};

// edge_in (the two-buffer layout only): the first and, when nx % VEC == 0, the last VEC-wide
// column group of every interior row run in the vector path too; the one or two populations of
// the edge node that cross the x boundary are then pulled through the full boundary resolution by
// that node's own lane.  (The in-place layout's odd step also stores across the boundary, so it
// keeps those columns in the band.)  A kernel built with step_block<..., EDGE = false> must be
// given edge_in = false geometry.
template <int VEC, int BX>
inline StepGeom step_geom(int nx, int ny, bool edge_in)
{
    StepGeom g;
    int L = VEC < nx ? VEC : nx;
    int R = ((nx - 1) / VEC) * VEC;
    if (edge_in && nx >= 2 * VEC) {
        L = 0;
        R = (nx / VEC) * VEC;
    }
    if (R < L) R = L;
    g.L = L;
    g.R = R;
    int rows = ny - 2 > 0 ? ny - 2 : 0;
    int cols = R;                       // threads must cover [0, R) as loaders
    g.bpr = (R > L) ? (cols + BX * VEC - 1) / (BX * VEC) : 0;
    g.n_int_blocks = g.bpr * rows;
    long long bw = (long long)L + (long long)(nx - R);
    g.n_edge = (ny >= 2 ? 2LL * nx : (long long)nx) + (long long)rows * bw;
    g.seg_log2 = 5;
    g.spr = 0;
    g.tasks = 0;
    return g;
}

// Row-segmented geometry: the same interior and band as step_geom, but the interior is cut into
// row segments of the fewest lanes (a power of two up to a warp) that cover a row, so that a warp
// works on 32 / seg rows of a narrow lattice at once instead of leaving lanes idle.
template <int VEC, int BX>
inline StepGeom step_geom_seg(int nx, int ny, bool edge_in)
{
    StepGeom g = step_geom<VEC, BX>(nx, ny, edge_in);
    const int groups = (g.R + VEC - 1) / VEC;        // VEC-wide column groups covering [0, R)
    int lg = 0;
    while ((1 << lg) < groups && lg < 5) ++lg;
    g.seg_log2 = lg;
    g.spr = (groups + (1 << lg) - 1) >> lg;
    const int rows = ny - 2 > 0 ? ny - 2 : 0;
    g.tasks = (g.R > g.L) ? rows * g.spr : 0;
    const int per_block = BX >> lg;
    g.n_int_blocks = (g.tasks + per_block - 1) / per_block;
    return g;
}

// vals[k] = row[i0 + k + s], s in {-1, 0, +1}, for a thread owning nodes i0..i0+VEC-1.  The lanes
// of one row segment (seg consecutive lanes, a power of two <= 32) own consecutive nodes.
template <int PREC, int VEC>
__device__ __forceinline__ void load_row(const typename Prec<PREC>::R *row, int i0, int s, int lane,
                                         bool loader, int nx, typename Prec<PREC>::C vals[VEC], int seg = 32)
{
    using P = Prec<PREC>;
    using R = typename P::R;
    using C = typename P::C;
    if (VEC == 1) {
        vals[0] = loader ? P::to_c(row[i0 + s]) : C(0);
        return;
    }
    C c[VEC];
    if (loader) {
        RVec<R, VEC> v = *reinterpret_cast<const RVec<R, VEC> *>(row + i0);
        #pragma unroll
        for (int k = 0; k < VEC; ++k) c[k] = P::to_c(v.v[k]);
    } else {
        #pragma unroll
        for (int k = 0; k < VEC; ++k) c[k] = C(0);
    }
    if (s == 0) {
        #pragma unroll
        for (int k = 0; k < VEC; ++k) vals[k] = c[k];
    } else if (s < 0) {
        C left = __shfl_up_sync(kFull, c[VEC - 1], 1, seg);
        if ((lane & (seg - 1)) == 0) left = (loader && i0 >= 1) ? P::to_c(row[i0 - 1]) : C(0);
        vals[0] = left;
        #pragma unroll
        for (int k = 1; k < VEC; ++k) vals[k] = c[k - 1];
    } else {
        C right = __shfl_down_sync(kFull, c[0], 1, seg);
        if ((lane & (seg - 1)) == seg - 1) right = (loader && i0 + VEC < nx) ? P::to_c(row[i0 + VEC]) : C(0);
        #pragma unroll
        for (int k = 0; k < VEC - 1; ++k) vals[k] = c[k + 1];
        vals[VEC - 1] = right;
    }
}

template <class R, int VEC>
__device__ __forceinline__ void store_vec(R *p, const R vals[VEC])
{
    RVec<R, VEC> v;
    #pragma unroll
    for (int k = 0; k < VEC; ++k) v.v[k] = vals[k];
    *reinterpret_cast<RVec<R, VEC> *>(p) = v;
}

// Warp shuffles of stored values (16-bit formats travel in a 32-bit register).
template <class R>
__device__ __forceinline__ R shfl_up_r(R v, int seg)
{
    if constexpr (sizeof(R) == 2) return (R)__shfl_up_sync(kFull, (unsigned)v, 1, seg);
    else return __shfl_up_sync(kFull, v, 1, seg);
}
template <class R>
__device__ __forceinline__ R shfl_down_r(R v, int seg)
{
    if constexpr (sizeof(R) == 2) return (R)__shfl_down_sync(kFull, (unsigned)v, 1, seg);
    else return __shfl_down_sync(kFull, v, 1, seg);
}

// Stores of `cnt` consecutive elements starting at row[c] (cnt <= 7 for 16-bit storage, where an
// unaligned start is served by one 2-, 4- and 8-byte store each instead of cnt scalar stores).
template <class R>
__device__ __forceinline__ void store_run(R *row, int c, const R *v, int cnt)
{
    if constexpr (sizeof(R) == 2) {
        int k = 0;
        if ((c & 1) && k < cnt) { row[c] = v[k]; ++c; ++k; }
        if ((c & 3) && cnt - k >= 2) {
            *reinterpret_cast<unsigned *>(row + c) = (unsigned)v[k] | ((unsigned)v[k + 1] << 16);
            c += 2; k += 2;
        }
        if (cnt - k >= 4) {
            const unsigned lo = (unsigned)v[k] | ((unsigned)v[k + 1] << 16);
            const unsigned hi = (unsigned)v[k + 2] | ((unsigned)v[k + 3] << 16);
            *reinterpret_cast<uint2 *>(row + c) = make_uint2(lo, hi);
            c += 4; k += 4;
        }
        if (cnt - k >= 2) {
            *reinterpret_cast<unsigned *>(row + c) = (unsigned)v[k] | ((unsigned)v[k + 1] << 16);
            c += 2; k += 2;
        }
        if (k < cnt) row[c] = v[k];
    } else {
        for (int k = 0; k < cnt; ++k) row[c + k] = v[k];
    }
}

// row[i0 + k + s] = vals[k] (already in the storage format) for the VEC nodes of every active
// lane, s in {-1, 0, +1}.  Called by all 32 lanes of a warp (the shifted case exchanges values).
// The active lanes of a row segment form one contiguous range.  A shifted store is realigned
// through the neighbour lane so that each lane writes its own aligned vector: element c of that
// vector belongs to node c - s; an element whose node lies in another row segment is written by
// that node's own lane (the segment-edge store), and an element whose node is not active is left
// alone.
template <class R, int VEC>
__device__ __forceinline__ void store_row(R *row, int i0, int s, int lane, bool active, const R vals[VEC],
                                          int seg = 32)
{
    if (VEC == 1 || s == 0) {
        if (!active) return;
        if (VEC == 1) row[i0 + s] = vals[0];
        else store_vec<R, VEC>(row + i0, vals);
        return;
    }
    if (s > 0) {
        const R prev_last = shfl_up_r(vals[VEC - 1], seg);
        const bool prev_active = (__shfl_up_sync(kFull, (int)active, 1, seg) != 0) && (lane & (seg - 1)) != 0;
        if (active && prev_active) {
            R out[VEC];
            out[0] = prev_last;
            #pragma unroll
            for (int k = 1; k < VEC; ++k) out[k] = vals[k - 1];
            store_vec<R, VEC>(row + i0, out);
        } else {
            if (prev_active) row[i0] = prev_last;
            if (active) store_run<R>(row, i0 + 1, vals, VEC - 1);
        }
        if (active && (lane & (seg - 1)) == seg - 1) row[i0 + VEC] = vals[VEC - 1];
    } else {
        const R next_first = shfl_down_r(vals[0], seg);
        const bool next_active =
            (__shfl_down_sync(kFull, (int)active, 1, seg) != 0) && (lane & (seg - 1)) != seg - 1;
        if (active && next_active) {
            R out[VEC];
            #pragma unroll
            for (int k = 0; k < VEC - 1; ++k) out[k] = vals[k + 1];
            out[VEC - 1] = next_first;
            store_vec<R, VEC>(row + i0, out);
        } else {
            if (active) store_run<R>(row, i0, vals + 1, VEC - 1);
            if (next_active) row[i0 + VEC - 1] = next_first;
        }
        if (active && (lane & (seg - 1)) == 0) row[i0 - 1] = vals[0];
    }
}

// f*_a of node `node` in the storage format: rounded to nearest, or stochastically (SR) with the
// bits of (node, a, the launch's step).
template <int PREC, bool SR>
__device__ __forceinline__ typename Prec<PREC>::R round_store(typename Prec<PREC>::C c, uint32_t node_hash, int a)
{
    if constexpr (SR) return Prec<PREC>::to_r_sr(c, sr_pop_bits(node_hash, a));
    else return Prec<PREC>::to_r(c);
}

// One node through the full boundary resolution (band blocks, and the
// reference behaviour every fast path must reproduce bit for bit).
template <int PREC, int KIND, int MODE, bool SR = false>
__device__ __forceinline__ void step_node_generic(const typename Prec<PREC>::R *src,
                                                  typename Prec<PREC>::R *dst,
                                                  const Params<typename Prec<PREC>::C> &p, int i, int j)
{
    using P = Prec<PREC>;
    using C = typename P::C;
    C g[9];
    #pragma unroll
    for (int a = 0; a < 9; ++a) {
        Loc L = pull_loc<MODE>(p, a, i, j);
        C v = P::to_c(src[at(p.plane, p.pitch, L.plane, L.j, L.i)]);
        if (L.side >= 0) v += p.corr[L.side][a];
        g[a] = v;
    }
    if (!collide<KIND, Prec<PREC>::kExactWeights>(p, g)) atomicOr(p.flag, 1);
    const uint32_t nh = SR ? sr_node_hash((uint32_t)j * (uint32_t)p.nx + (uint32_t)i, p.salt) : 0u;
    #pragma unroll
    for (int a = 0; a < 9; ++a) {
        Loc L = push_loc<MODE>(p, a, i, j);
        dst[at(p.plane, p.pitch, L.plane, L.j, L.i)] = round_store<PREC, SR>(g[a], nh, a);
    }
}

// Block b of one lattice's step grid (interior block or band block), executed
// by all BX threads of the calling block.
// ROWSEG: the interior blocks follow the row-segmented geometry of step_geom_seg.
template <int PREC, int KIND, int MODE, int VEC, int BX, bool EDGE = true, bool ROWSEG = false, bool SR = false>
__device__ __forceinline__ void step_block(const typename Prec<PREC>::R *src, typename Prec<PREC>::R *dst,
                                           const Params<typename Prec<PREC>::C> &p, const StepGeom &geo, int b)
{
    using C = typename Prec<PREC>::C;
    const int tid = threadIdx.x;

    if (b >= geo.n_int_blocks) {
        // ---- band: one node per thread, full boundary handling ----
        long long e = (long long)(b - geo.n_int_blocks) * BX + tid;
        if (e >= geo.n_edge) return;
        int i, j;
        if (e < p.nx) {
            i = (int)e; j = 0;
        } else if (e < 2LL * p.nx && p.ny >= 2) {
            i = (int)(e - p.nx); j = p.ny - 1;
        } else {
            long long m = e - 2LL * p.nx;
            int bw = geo.L + (p.nx - geo.R);
            j = 1 + (int)(m / bw);
            int k = (int)(m % bw);
            i = k < geo.L ? k : geo.R + (k - geo.L);
        }
        step_node_generic<PREC, KIND, MODE, SR>(src, dst, p, i, j);
        return;
    }

    // ---- interior: VEC nodes per thread, no boundary logic ----
    const int lane = tid & 31;
    int j, i0, seg = 32;
    bool valid = true;
    if (ROWSEG) {
        seg = 1 << geo.seg_log2;
        const int task = b * (BX >> geo.seg_log2) + (tid >> geo.seg_log2);
        valid = task < geo.tasks;
        const int tk = valid ? task : 0;
        j = 1 + tk / geo.spr;
        i0 = ((tk % geo.spr) << geo.seg_log2) * VEC + (tid & (seg - 1)) * VEC;
    } else {
        j = 1 + b / geo.bpr;
        i0 = (b % geo.bpr) * (BX * VEC) + tid * VEC;
    }
    const bool active = valid && (i0 >= geo.L) && (i0 + VEC <= geo.R);
    const bool loader = (VEC == 1) ? active : (valid && i0 < p.nx);

    C g[VEC][9];
    #pragma unroll
    for (int a = 0; a < 9; ++a) {
        const int plane = (MODE == MODE_AA_ODD) ? opp(a) : a;
        const int row = (MODE == MODE_AA_EVEN) ? j : j - ey(a);
        const int s = (MODE == MODE_AA_EVEN) ? 0 : -ex(a);
        const typename Prec<PREC>::R *rp = src + (size_t)plane * (size_t)p.plane + (size_t)row * (size_t)p.pitch;
        C vals[VEC];
        load_row<PREC, VEC>(rp, i0, s, lane, loader, p.nx, vals, seg);
        #pragma unroll
        for (int k = 0; k < VEC; ++k) g[k][a] = vals[k];
    }
    if (EDGE && MODE == MODE_AB && geo.L == 0 && active) {
        // edge groups: the populations pulled across the left (a = 1, 5, 8) or right (a = 3, 6, 7)
        // boundary, through the full resolution (wall, moving wall or periodic wrap)
        using P = Prec<PREC>;
        if (i0 == 0) {
            #pragma unroll
            for (int a = 1; a < 9; ++a) {
                if (ex(a) != 1) continue;
                const Loc L = pull_loc<MODE>(p, a, 0, j);
                C v = P::to_c(src[at(p.plane, p.pitch, L.plane, L.j, L.i)]);
                if (L.side >= 0) v += p.corr[L.side][a];
                g[0][a] = v;
            }
        }
        if (i0 + VEC == p.nx) {
            #pragma unroll
            for (int a = 1; a < 9; ++a) {
                if (ex(a) != -1) continue;
                const Loc L = pull_loc<MODE>(p, a, p.nx - 1, j);
                C v = P::to_c(src[at(p.plane, p.pitch, L.plane, L.j, L.i)]);
                if (L.side >= 0) v += p.corr[L.side][a];
                g[VEC - 1][a] = v;
            }
        }
    }
    bool ok = true;
    #pragma unroll
    for (int k = 0; k < VEC; ++k) ok &= collide<KIND, Prec<PREC>::kExactWeights>(p, g[k]);
    // only the in-place odd step exchanges values between lanes when storing
    if (!active && !(MODE == MODE_AA_ODD && VEC > 1)) return;
    if (active && !ok) atomicOr(p.flag, 1);
    using R = typename Prec<PREC>::R;
    uint32_t nh[VEC];
    #pragma unroll
    for (int k = 0; k < VEC; ++k)
        nh[k] = SR ? sr_node_hash((uint32_t)j * (uint32_t)p.nx + (uint32_t)(i0 + k), p.salt) : 0u;
    #pragma unroll
    for (int a = 0; a < 9; ++a) {
        const int plane = (MODE == MODE_AA_EVEN) ? opp(a) : a;
        const int row = (MODE == MODE_AA_ODD) ? j + ey(a) : j;
        const int s = (MODE == MODE_AA_ODD) ? ex(a) : 0;
        R *rp = dst + (size_t)plane * (size_t)p.plane + (size_t)row * (size_t)p.pitch;
        R vals[VEC];
        #pragma unroll
        for (int k = 0; k < VEC; ++k) vals[k] = round_store<PREC, SR>(g[k][a], nh[k], a);
        store_row<R, VEC>(rp, i0, s, lane, active, vals, seg);
    }
}

template <int PREC, int KIND, int MODE, int VEC, int BX, bool SR = false>
__global__ void __launch_bounds__(BX)
step_kernel(const typename Prec<PREC>::R *src, typename Prec<PREC>::R *dst,
            const Params<typename Prec<PREC>::C> p, const StepGeom geo)
{
    step_block<PREC, KIND, MODE, VEC, BX, true, false, SR>(src, dst, p, geo, blockIdx.x);
}

// ---- state I/O and macros (one thread per node of a row chunk) -------------------

template <int PREC, int MODE>
__device__ __forceinline__ void pull_canonical(const typename Prec<PREC>::R *state,
                                               const Params<typename Prec<PREC>::C> &p, int i, int j,
                                               typename Prec<PREC>::C g[9])
{
    using P = Prec<PREC>;
    #pragma unroll
    for (int a = 0; a < 9; ++a) {
        Loc L = pull_loc<MODE>(p, a, i, j);
        typename P::C v = P::to_c(state[at(p.plane, p.pitch, L.plane, L.j, L.i)]);
        if (L.side >= 0) v += p.corr[L.side][a];
        g[a] = v;
    }
}

template <int PREC, int MODE>
__global__ void get_f_kernel(const typename Prec<PREC>::R *state, double *f, int row0, int rows,
                             const Params<typename Prec<PREC>::C> p)
{
    long long n = (long long)rows * p.nx;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int r = (int)(t / p.nx), i = (int)(t % p.nx);
    typename Prec<PREC>::C g[9];
    pull_canonical<PREC, MODE>(state, p, i, row0 + r, g);
    #pragma unroll
    for (int a = 0; a < 9; ++a)
        f[((size_t)a * rows + r) * p.nx + i] = (double)g[a] + wgt<double>(a);
}

template <int PREC, int MODE>
__global__ void set_f_kernel(typename Prec<PREC>::R *state, const double *f, int row0, int rows,
                             const Params<typename Prec<PREC>::C> p)
{
    using P = Prec<PREC>;
    long long n = (long long)rows * p.nx;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int r = (int)(t / p.nx), i = (int)(t % p.nx), j = row0 + r;
    #pragma unroll
    for (int a = 0; a < 9; ++a) {
        Loc L = pull_loc<MODE>(p, a, i, j);
        double g = f[((size_t)a * rows + r) * p.nx + i] - wgt<double>(a);
        if (L.side >= 0) g -= (double)p.corr[L.side][a];
        state[at(p.plane, p.pitch, L.plane, L.j, L.i)] = P::to_r((typename P::C)g);
    }
}

// One population of f^eq(rho, u) (Eq. feq-full) as an offset, stored through the pull map.
// Float arithmetic for the 32- and 16-bit formats (their stored value has at most 24
// significant bits); the weight product is rounded as for an exact weight.
template <int PREC, int MODE, int A>
__device__ __forceinline__ void init_store_f(typename Prec<PREC>::R *state, const Params<float> &p, int i, int j,
                                             float drho, float d, float ux, float uy, float uu)
{
    using P = Prec<PREC>;
    const float eu = float(ex(A)) * ux + float(ey(A)) * uy;
    float g = WeightMul<float>::template mul<A>(drho + d * (3.0f * eu + 4.5f * eu * eu - 1.5f * uu));
    const Loc L = pull_loc<MODE>(p, A, i, j);
    if (L.side >= 0) g -= p.corr[L.side][A];
    state[at(p.plane, p.pitch, L.plane, L.j, L.i)] = P::to_r(g);
}

// f = f^eq(rho, u) (Eq. feq-full), written as offsets through the pull map;
// rho == NULL selects rho = 1, u = 0.  rho and u may be device memory or host memory
// the device can address (page-locked and mapped).
template <int PREC, int MODE>
__global__ void init_macros_kernel(typename Prec<PREC>::R *state, const double *rho, const double *u,
                                   int row0, int rows, const Params<typename Prec<PREC>::C> p)
{
    using P = Prec<PREC>;
    long long n = (long long)rows * p.nx;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int r = (int)(t / p.nx), i = (int)(t % p.nx), j = row0 + r;
    size_t q = (size_t)r * p.nx + i;
    double d = 1.0, ux = 0.0, uy = 0.0;           // rho == NULL: the resting state
    if (rho) {
        d = rho[q];
        ux = u[q];
        uy = u[(size_t)rows * p.nx + q];
    }
    if constexpr (PREC == SMRT_PREC_F64) {
        double uu = ux * ux + uy * uy;
        #pragma unroll
        for (int a = 0; a < 9; ++a) {
            double eu = ex(a) * ux + ey(a) * uy;
            double g = wgt<double>(a) * ((d - 1.0) + d * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu));
            Loc L = pull_loc<MODE>(p, a, i, j);
            if (L.side >= 0) g -= (double)p.corr[L.side][a];
            state[at(p.plane, p.pitch, L.plane, L.j, L.i)] = P::to_r((typename P::C)g);
        }
    } else {
        const float drho = (float)(d - 1.0), df = (float)d, fx = (float)ux, fy = (float)uy;
        const float uu = fx * fx + fy * fy;
        init_store_f<PREC, MODE, 0>(state, p, i, j, drho, df, fx, fy, uu);
        init_store_f<PREC, MODE, 1>(state, p, i, j, drho, df, fx, fy, uu);
        init_store_f<PREC, MODE, 2>(state, p, i, j, drho, df, fx, fy, uu);
        init_store_f<PREC, MODE, 3>(state, p, i, j, drho, df, fx, fy, uu);
        init_store_f<PREC, MODE, 4>(state, p, i, j, drho, df, fx, fy, uu);
        init_store_f<PREC, MODE, 5>(state, p, i, j, drho, df, fx, fy, uu);
        init_store_f<PREC, MODE, 6>(state, p, i, j, drho, df, fx, fy, uu);
        init_store_f<PREC, MODE, 7>(state, p, i, j, drho, df, fx, fy, uu);
        init_store_f<PREC, MODE, 8>(state, p, i, j, drho, df, fx, fy, uu);
    }
}

// Moments of Eq. (fea-0) accumulated in double from the canonical offsets.
__device__ __forceinline__ void moments_d(const double g[9], double &rho, double &ux, double &uy)
{
    double drho = 0.0, jx = 0.0, jy = 0.0;
    #pragma unroll
    for (int a = 0; a < 9; ++a) {
        drho += g[a];
        jx += ex(a) * g[a];
        jy += ey(a) * g[a];
    }
    rho = 1.0 + drho;
    ux = jx / rho;
    uy = jy / rho;
}

// s + c += x without rounding error in s + c (Knuth's two-sum; c collects the error terms).
__device__ __forceinline__ void two_sum_acc(float &s, float &c, float x)
{
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}

// The moments of Eq. (fea-0) of nine float offsets, in double, with few double operations:
// each sum is formed in float as an unevaluated pair hi + lo (two-sum), which carries about
// 48 significant bits of it, and 1 / rho is the float reciprocal refined by two Newton steps
// (to double rounding).  The double pipe is the scarce unit of this GPU; this form needs about
// a quarter of the double operations of moments_d, whose results it matches to ~1e-14.
__device__ __forceinline__ void moments_f(const float g[9], double &rho, double &ux, double &uy)
{
    float s0 = g[0], c0 = 0.0f, sx = g[1], cx = 0.0f, sy = g[2], cy = 0.0f;
    two_sum_acc(s0, c0, g[1]);
    two_sum_acc(s0, c0, g[2]);
    two_sum_acc(s0, c0, g[3]);
    two_sum_acc(s0, c0, g[4]);
    two_sum_acc(s0, c0, g[5]);
    two_sum_acc(s0, c0, g[6]);
    two_sum_acc(s0, c0, g[7]);
    two_sum_acc(s0, c0, g[8]);
    two_sum_acc(sx, cx, -g[3]);
    two_sum_acc(sx, cx, g[5]);
    two_sum_acc(sx, cx, -g[6]);
    two_sum_acc(sx, cx, -g[7]);
    two_sum_acc(sx, cx, g[8]);
    two_sum_acc(sy, cy, -g[4]);
    two_sum_acc(sy, cy, g[5]);
    two_sum_acc(sy, cy, g[6]);
    two_sum_acc(sy, cy, -g[7]);
    two_sum_acc(sy, cy, -g[8]);
    rho = 1.0 + ((double)s0 + (double)c0);
    const double r0 = (double)(1.0f / (float)rho);
    const double r1 = r0 * (2.0 - rho * r0);
    const double inv = r1 * (2.0 - rho * r1);
    ux = ((double)sx + (double)cx) * inv;
    uy = ((double)sy + (double)cy) * inv;
}

// moments_d for double offsets, moments_f for float ones.
__device__ __forceinline__ void moments_any(const double g[9], double &rho, double &ux, double &uy)
{
    moments_d(g, rho, ux, uy);
}
__device__ __forceinline__ void moments_any(const float g[9], double &rho, double &ux, double &uy)
{
    moments_f(g, rho, ux, uy);
}

template <int PREC, int MODE>
__global__ void macros_kernel(const typename Prec<PREC>::R *state, double *rho, double *u, int row0,
                              int rows, const Params<typename Prec<PREC>::C> p)
{
    long long n = (long long)rows * p.nx;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int r = (int)(t / p.nx), i = (int)(t % p.nx);
    typename Prec<PREC>::C g[9];
    pull_canonical<PREC, MODE>(state, p, i, row0 + r, g);
    double rr, ux, uy;
    moments_any(g, rr, ux, uy);
    size_t q = (size_t)r * p.nx + i;
    if (rho) rho[q] = rr;
    if (u) {
        u[q] = ux;
        u[(size_t)rows * p.nx + q] = uy;
    }
}

// ---- residual: u(t) and u(t+1) without advancing the state ------------------------
// kRTX x kRTY tiles: the layout of the caller-scratch residual (smrt_residual_noalloc).
constexpr int kRTX = 32, kRTY = 8, kRHX = kRTX + 2, kRHY = kRTY + 2;

// The handle's residual sweeps rows.  A warp owns a strip of kRSW = 30 columns (lanes 1..30; lanes 0
// and 31 are the neighbouring columns, wrapped where the x axis is periodic) and a segment of kRSR
// rows, and walks it from the row below to the row above.  For each row every lane pulls f(t) of its
// node, collides it (the code of the step) and rounds f* to the storage format as the step stores
// it; f(t+1) of a node on the previous row then comes from registers: the populations arriving along
// x from the neighbouring lanes by warp shuffles, those arriving along y from the rows kept before
// and after it, and bounce-back terms from the node's own f*.  Collisions per node: 32/30 x
// (kRSR + 2)/kRSR; no shared memory, no block barrier; f(t) of the next row is loaded while the
// current row collides.  Sums: |u1-u0|^2, |u1|^2, rho0, rho0 ux0, rho0 uy0.
// Double offsets: u0 and u1 by moments_d and their difference.  Float offsets (the 32- and 16-bit
// formats): the change is formed from the offset differences in float,
//   u1 - u0 = (dj - u0 drho) / rho1,  drho = sum_a (g1_a - g0_a),  dj = sum_a c_a (g1_a - g0_a),
// which is u1 - u0 without the cancellation of two nearly equal velocities (relative error ~1e-6 of
// the change itself); rho0 - 1 and j0 = rho0 u0 are float sums of the offsets.  A thread adds its
// nodes' terms into compensated float pairs (value + rounding error, ~48 significant bits); the
// warp, block and grid sums of those are in double.
constexpr int kRSW = 30, kRSR = 64;

__device__ __forceinline__ double warp_sum(double v)
{
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

// pull_canonical for a node whose nine source nodes lie inside the lattice (no wall, no wrap).
template <int PREC, int MODE>
__device__ __forceinline__ void pull_inner(const typename Prec<PREC>::R *state, const Params<typename Prec<PREC>::C> &p,
                                           int i, int j, typename Prec<PREC>::C g[9])
{
    using P = Prec<PREC>;
    const typename P::R *s0 = state + (size_t)j * (size_t)p.pitch + (size_t)i;
    #pragma unroll
    for (int a = 0; a < 9; ++a) {
        const long long off = (MODE == MODE_AA_EVEN) ? (long long)a * p.plane
                              : (long long)(MODE == MODE_AB ? a : opp(a)) * p.plane -
                                    (long long)ey(a) * p.pitch - ex(a);
        g[a] = P::to_c(s0[off]);
    }
}

// f(t) of node (i, j) of the sweep, wrapped onto the lattice; false where (i, j) is behind a wall or
// beyond the lattice (no node).  (i, j) are updated to the wrapped node.
template <int PREC, int MODE>
__device__ __forceinline__ bool sweep_pull(const typename Prec<PREC>::R *state, const Params<typename Prec<PREC>::C> &p,
                                           int &i, int &j, typename Prec<PREC>::C g[9])
{
    if (i > p.nx || j > p.ny) return false;
    if (resolve(p, i, j) >= 0) return false;
    if (i >= 1 && i + 1 < p.nx && j >= 1 && j + 1 < p.ny) pull_inner<PREC, MODE>(state, p, i, j, g);
    else pull_canonical<PREC, MODE>(state, p, i, j, g);
    return true;
}

#ifndef SMRT_RESID_MIN_BLOCKS
#define SMRT_RESID_MIN_BLOCKS 3          // blocks per SM the register budget is set for (sweepable)
#endif


template <int PREC, int KIND, int MODE, bool SR = false>
__global__ void __launch_bounds__(256, SMRT_RESID_MIN_BLOCKS)
residual_kernel(const typename Prec<PREC>::R *__restrict__ state, const Params<typename Prec<PREC>::C> p,
                double *partials, int strips, int segs)
{
    using P = Prec<PREC>;
    using C = typename P::C;
    constexpr bool kFloat = sizeof(C) == 4;
    __shared__ double red[8][kResidualSums];
    const int tid = threadIdx.x, lane = tid & 31;
    double acc[kResidualSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
    float cs[kResidualSums] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, cc[kResidualSums] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    int nodes = 0;
    const long long items = (long long)strips * segs;
    for (long long item = (long long)blockIdx.x * 8 + (tid >> 5); item < items; item += (long long)gridDim.x * 8) {
        const int x0 = (int)(item % strips) * kRSW, r0 = (int)(item / strips) * kRSR;
        const int rows = min(kRSR, p.ny - r0);
        const int i = x0 - 1 + lane;                            // this lane's column
        const bool own_col = lane >= 1 && lane <= kRSW && i < p.nx;
        // row j - 1 (f* of this lane, shuffled arrivals, f(t)) and row j - 2 (the y-arrivals)
        C own1[9], g01[9];
        C in1_1 = 0, in3_1 = 0, in5_1 = 0, in6_1 = 0;          // f*_1, f*_3, f*_5, f*_6 from lanes -1/+1/-1/+1
        C own2_2 = 0, in5_2 = 0, in6_2 = 0;
        #pragma unroll
        for (int a = 0; a < 9; ++a) own1[a] = g01[a] = 0;
        // f(t) of the next row is pulled one iteration ahead, so its loads are in flight during the
        // current row's collision
        int wi_n = i, wj_n = r0 - 1;
        C gn[9];
        #pragma unroll
        for (int a = 0; a < 9; ++a) gn[a] = 0;
        bool has_n = sweep_pull<PREC, MODE>(state, p, wi_n, wj_n, gn);
        #pragma unroll 1
        for (int jj = -1; jj <= rows; ++jj) {
            C g[9], pc[9];
            const int wi = wi_n, wj = wj_n;
            const bool has = has_n;
            #pragma unroll
            for (int a = 0; a < 9; ++a) {
                g[a] = gn[a];
                pc[a] = 0;
            }
            if (jj < rows) {
                wi_n = i;
                wj_n = r0 + jj + 1;
                #pragma unroll
                for (int a = 0; a < 9; ++a) gn[a] = 0;
                has_n = sweep_pull<PREC, MODE>(state, p, wi_n, wj_n, gn);
            }
            if (has) {
                #pragma unroll
                for (int a = 0; a < 9; ++a) pc[a] = g[a];
                collide<KIND, Prec<PREC>::kExactWeights>(p, pc);
                const uint32_t nh = SR ? sr_node_hash((uint32_t)wj * (uint32_t)p.nx + (uint32_t)wi, p.salt) : 0u;
                #pragma unroll
                for (int a = 0; a < 9; ++a) pc[a] = P::to_c(round_store<PREC, SR>(pc[a], nh, a));
            }
            // arrivals along x: ex = +1 populations from lane - 1, ex = -1 from lane + 1
            const C up1 = __shfl_up_sync(kFull, pc[1], 1), up5 = __shfl_up_sync(kFull, pc[5], 1),
                    up8 = __shfl_up_sync(kFull, pc[8], 1);
            const C dn3 = __shfl_down_sync(kFull, pc[3], 1), dn6 = __shfl_down_sync(kFull, pc[6], 1),
                    dn7 = __shfl_down_sync(kFull, pc[7], 1);
            if (jj >= 1 && own_col) {
                // f(t+1) of node (i, r0 + jj - 1)
                const int jn = r0 + jj - 1;
                C g1[9];
                g1[0] = own1[0];
                g1[1] = in1_1;
                g1[3] = in3_1;
                g1[2] = own2_2;
                g1[5] = in5_2;
                g1[6] = in6_2;
                g1[4] = pc[4];
                g1[7] = dn7;
                g1[8] = up8;
                if (i == 0 || i + 1 == p.nx || jn == 0 || jn + 1 == p.ny) {
                    #pragma unroll
                    for (int a = 1; a < 9; ++a) {
                        int si = i - ex(a), sj = jn - ey(a);
                        const int side = resolve(p, si, sj);
                        if (side >= 0) g1[a] = own1[opp(a)] + p.corr[side][a];
                    }
                }
                if constexpr (kFloat) {
                    float d[9];
                    #pragma unroll
                    for (int a = 0; a < 9; ++a) d[a] = g1[a] - g01[a];
                    const float rho0m1 = (((g01[0] + g01[1]) + (g01[2] + g01[3])) +
                                          ((g01[4] + g01[5]) + (g01[6] + g01[7]))) + g01[8];
                    const float jx0 = ((g01[1] - g01[3]) + (g01[5] - g01[6])) + (g01[8] - g01[7]);
                    const float jy0 = ((g01[2] - g01[4]) + (g01[5] - g01[7])) + (g01[6] - g01[8]);
                    const float drho = (((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7]))) + d[8];
                    const float djx = ((d[1] - d[3]) + (d[5] - d[6])) + (d[8] - d[7]);
                    const float djy = ((d[2] - d[4]) + (d[5] - d[7])) + (d[6] - d[8]);
                    const float rho0 = 1.0f + rho0m1;
                    const float inv0 = 1.0f / rho0, inv1 = 1.0f / (rho0 + drho);
                    const float ux0 = jx0 * inv0, uy0 = jy0 * inv0;
                    const float dx = (djx - ux0 * drho) * inv1, dy = (djy - uy0 * drho) * inv1;
                    const float ux1 = ux0 + dx, uy1 = uy0 + dy;
                    two_sum_acc(cs[0], cc[0], dx * dx + dy * dy);
                    two_sum_acc(cs[1], cc[1], ux1 * ux1 + uy1 * uy1);
                    two_sum_acc(cs[2], cc[2], rho0m1);
                    two_sum_acc(cs[3], cc[3], jx0);
                    two_sum_acc(cs[4], cc[4], jy0);
                    ++nodes;
                } else {
                    double r0d, ux0, uy0, r1, ux1, uy1;
                    moments_any(g01, r0d, ux0, uy0);
                    moments_any(g1, r1, ux1, uy1);
                    const double dx = ux1 - ux0, dy = uy1 - uy0;
                    acc[0] += dx * dx + dy * dy;
                    acc[1] += ux1 * ux1 + uy1 * uy1;
                    acc[2] += r0d;
                    acc[3] += r0d * ux0;
                    acc[4] += r0d * uy0;
                }
            }
            // shift: row j - 1 becomes row j - 2, row j becomes row j - 1
            own2_2 = own1[2];
            in5_2 = in5_1;
            in6_2 = in6_1;
            #pragma unroll
            for (int a = 0; a < 9; ++a) {
                own1[a] = pc[a];
                g01[a] = g[a];
            }
            in1_1 = up1;
            in3_1 = dn3;
            in5_1 = up5;
            in6_1 = dn6;
        }
    }
    if constexpr (kFloat) {
        #pragma unroll
        for (int k = 0; k < kResidualSums; ++k) acc[k] = (double)cs[k] + (double)cc[k];
        acc[2] += (double)nodes;
    }
    #pragma unroll
    for (int k = 0; k < kResidualSums; ++k) acc[k] = warp_sum(acc[k]);
    if (lane == 0) {
        #pragma unroll
        for (int k = 0; k < kResidualSums; ++k) red[tid >> 5][k] = acc[k];
    }
    __syncthreads();
    if (tid < kResidualSums) {
        double sum = 0.0;
        for (int w = 0; w < 8; ++w) sum += red[w][tid];
        partials[(size_t)blockIdx.x * kResidualSums + tid] = sum;
    }
}

// Deterministic final sum of the per-block partials (fixed order, one block).
static __global__ void __launch_bounds__(256) reduce_partials_kernel(const double *partials, int nblocks, double *sums)
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
    if (tid < kResidualSums) sums[tid] = sh[tid][0];
}

// ---- launchers ---------------------------------------------------------------------

// Nodes per thread (VEC: one 16-byte vector or less per population row) and
// threads per block of the step kernel; overridable at build time for sweeps.
#ifndef SMRT_VEC_F64
#define SMRT_VEC_F64 2
#endif
#ifndef SMRT_VEC_F32
#define SMRT_VEC_F32 4
#endif
#ifndef SMRT_VEC_F16
#define SMRT_VEC_F16 8
#endif
#ifndef SMRT_BX
#define SMRT_BX 128
#endif
#ifndef SMRT_BX16
#define SMRT_BX16 64     // 16-bit storage: measured +1.4 % (AB) / +2.7 % (AA) over 128 at 8192^2
#endif
template <int PREC> struct Tune;
template <> struct Tune<SMRT_PREC_F64> { static constexpr int VEC = SMRT_VEC_F64, BX = SMRT_BX; };
template <> struct Tune<SMRT_PREC_F32> { static constexpr int VEC = SMRT_VEC_F32, BX = SMRT_BX; };
template <> struct Tune<SMRT_PREC_F16> { static constexpr int VEC = SMRT_VEC_F16, BX = SMRT_BX16; };
template <> struct Tune<SMRT_PREC_BF16> { static constexpr int VEC = SMRT_VEC_F16, BX = SMRT_BX16; };

template <int PREC, int KIND, int MODE>
cudaError_t launch_step_km(const void *src, void *dst, const HostParams &hp, cudaStream_t s)
{
    using P = Prec<PREC>;
    using R = typename P::R;
    constexpr int VEC = Tune<PREC>::VEC, BX = Tune<PREC>::BX;
    const Params<typename P::C> p = make_params<typename P::C>(hp);
    const StepGeom geo = step_geom<VEC, BX>(hp.nx, hp.ny, MODE == MODE_AB);
    const long long edge_blocks = (geo.n_edge + BX - 1) / BX;
    const long long blocks = (long long)geo.n_int_blocks + edge_blocks;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if constexpr (PREC == SMRT_PREC_F16 || PREC == SMRT_PREC_BF16) {
        if (hp.rounding == SMRT_ROUND_STOCHASTIC) {
            step_kernel<PREC, KIND, MODE, VEC, BX, true><<<(unsigned)blocks, BX, 0, s>>>(
                (const R *)src, (R *)dst, p, geo);
            return cudaGetLastError();
        }
    }
    step_kernel<PREC, KIND, MODE, VEC, BX><<<(unsigned)blocks, BX, 0, s>>>(
        (const R *)src, (R *)dst, p, geo);
    return cudaGetLastError();
}

template <int PREC, int KIND>
cudaError_t launch_step_k(int mode, const void *src, void *dst, const HostParams &hp, cudaStream_t s)
{
    switch (mode) {
    case MODE_AB: return launch_step_km<PREC, KIND, MODE_AB>(src, dst, hp, s);
    case MODE_AA_EVEN: return launch_step_km<PREC, KIND, MODE_AA_EVEN>(src, dst, hp, s);
    case MODE_AA_ODD: return launch_step_km<PREC, KIND, MODE_AA_ODD>(src, dst, hp, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int PREC>
cudaError_t launch_step(int kind, int mode, const void *src, void *dst, const HostParams &hp, cudaStream_t s)
{
    switch (kind) {
    case SMRT_COLLISION_SMRT: return launch_step_k<PREC, SMRT_COLLISION_SMRT>(mode, src, dst, hp, s);
    case SMRT_COLLISION_SRT: return launch_step_k<PREC, SMRT_COLLISION_SRT>(mode, src, dst, hp, s);
    case SMRT_COLLISION_TWO_TAU: return launch_step_k<PREC, SMRT_COLLISION_TWO_TAU>(mode, src, dst, hp, s);
    default: return cudaErrorInvalidValue;
    }
}

inline unsigned node_blocks(int rows, int nx, int threads)
{
    long long n = (long long)rows * nx;
    return (unsigned)((n + threads - 1) / threads);
}

#define SMRT_MODE_SWITCH(mode, CALL)                                  \
    switch (mode) {                                                   \
    case MODE_AB: { constexpr int M = MODE_AB; CALL; } break;          \
    case MODE_AA_EVEN: { constexpr int M = MODE_AA_EVEN; CALL; } break;\
    case MODE_AA_ODD: { constexpr int M = MODE_AA_ODD; CALL; } break;  \
    default: return cudaErrorInvalidValue;                            \
    }

template <int PREC>
cudaError_t launch_get_f(int mode, const void *state, double *f, int row0, int rows, const HostParams &hp,
                         cudaStream_t s)
{
    using P = Prec<PREC>;
    const Params<typename P::C> p = make_params<typename P::C>(hp);
    if (rows <= 0) return cudaSuccess;
    const unsigned nb = node_blocks(rows, hp.nx, 256);
    SMRT_MODE_SWITCH(mode, (get_f_kernel<PREC, M><<<nb, 256, 0, s>>>((const typename P::R *)state, f, row0, rows, p)));
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_set_f(int mode, void *state, const double *f, int row0, int rows, const HostParams &hp,
                         cudaStream_t s)
{
    using P = Prec<PREC>;
    const Params<typename P::C> p = make_params<typename P::C>(hp);
    if (rows <= 0) return cudaSuccess;
    const unsigned nb = node_blocks(rows, hp.nx, 256);
    SMRT_MODE_SWITCH(mode, (set_f_kernel<PREC, M><<<nb, 256, 0, s>>>((typename P::R *)state, f, row0, rows, p)));
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_init_macros(int mode, void *state, const double *rho, const double *u, int row0, int rows,
                               const HostParams &hp, cudaStream_t s)
{
    using P = Prec<PREC>;
    const Params<typename P::C> p = make_params<typename P::C>(hp);
    if (rows <= 0) return cudaSuccess;
    const unsigned nb = node_blocks(rows, hp.nx, 256);
    SMRT_MODE_SWITCH(mode, (init_macros_kernel<PREC, M><<<nb, 256, 0, s>>>((typename P::R *)state, rho, u, row0, rows, p)));
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_macros(int mode, const void *state, double *rho, double *u, int row0, int rows,
                          const HostParams &hp, cudaStream_t s)
{
    using P = Prec<PREC>;
    const Params<typename P::C> p = make_params<typename P::C>(hp);
    if (rows <= 0) return cudaSuccess;
    const unsigned nb = node_blocks(rows, hp.nx, 256);
    SMRT_MODE_SWITCH(mode, (macros_kernel<PREC, M><<<nb, 256, 0, s>>>((const typename P::R *)state, rho, u, row0, rows, p)));
    return cudaGetLastError();
}

template <int PREC, int KIND>
cudaError_t launch_residual_k(int mode, const void *state, const HostParams &hp, const Scratch &sc,
                              cudaStream_t s)
{
    using P = Prec<PREC>;
    const Params<typename P::C> p = make_params<typename P::C>(hp);
    const int strips = (hp.nx + kRSW - 1) / kRSW, segs = (hp.ny + kRSR - 1) / kRSR;
    const long long warps = (long long)strips * segs;
    const long long want = (warps + 7) / 8;
    const int nb = (int)(want < kResidualMaxBlocks ? want : kResidualMaxBlocks);
    bool plain = true;
    if constexpr (PREC == SMRT_PREC_F16 || PREC == SMRT_PREC_BF16) {
        if (hp.rounding == SMRT_ROUND_STOCHASTIC) {
            plain = false;
            SMRT_MODE_SWITCH(mode, (residual_kernel<PREC, KIND, M, true><<<nb, 256, 0, s>>>(
                                       (const typename P::R *)state, p, sc.partials, strips, segs)));
        }
    }
    if (plain) {
        SMRT_MODE_SWITCH(mode, (residual_kernel<PREC, KIND, M><<<nb, 256, 0, s>>>((const typename P::R *)state, p,
                                                                                     sc.partials, strips, segs)));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_partials_kernel<<<1, 256, 0, s>>>(sc.partials, nb, sc.sums);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_residual(int kind, int mode, const void *state, const HostParams &hp, const Scratch &sc,
                            cudaStream_t s)
{
    switch (kind) {
    case SMRT_COLLISION_SMRT: return launch_residual_k<PREC, SMRT_COLLISION_SMRT>(mode, state, hp, sc, s);
    case SMRT_COLLISION_SRT: return launch_residual_k<PREC, SMRT_COLLISION_SRT>(mode, state, hp, sc, s);
    case SMRT_COLLISION_TWO_TAU: return launch_residual_k<PREC, SMRT_COLLISION_TWO_TAU>(mode, state, hp, sc, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int PREC>
KernelTable make_table()
{
    KernelTable t;
    t.step = &launch_step<PREC>;
    t.get_f = &launch_get_f<PREC>;
    t.set_f = &launch_set_f<PREC>;
    t.init_macros = &launch_init_macros<PREC>;
    t.macros = &launch_macros<PREC>;
    t.residual = &launch_residual<PREC>;
    t.elem_bytes = sizeof(typename Prec<PREC>::R);
    return t;
}

} // namespace smrt
