// d2q9.cuh -- device-side building blocks of the SmrtLBM kernels (sm_103a).
//
// Lattice constants, storage formats, kernel parameters, the boundary
// resolution of a pulled population and the per-node collision operators.
// Everything here is GPU-side code of this library; it shares nothing with the
// CPU oracle.
//
// Storage: every precision stores the offset g_a = f_a - w_a of each population
// (w_a the D2Q9 weight), which keeps the stored numbers small (|g| ~ |u| w) and
// so gains relative precision in every format; rho = 1 + sum g.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace smrt {

// ---- D2Q9 velocity set in the paper's order (listing below Eq. lb.srt) -------
// a: 0 (0,0), 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1), 5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1)
__host__ __device__ constexpr int ex(int a)
{
    return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int a)
{
    return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}
// reversed link: 1<->3, 2<->4, 5<->7, 6<->8
__host__ __device__ constexpr int opp(int a)
{
    return a == 0 ? 0 : (a <= 4 ? ((a + 1) % 4) + 1 : ((a - 3) % 4) + 5);
}
// weights below Eq. (feq-full)
template <class C>
__host__ __device__ constexpr C wgt(int a)
{
    return a == 0 ? C(4) / C(9) : (a <= 4 ? C(1) / C(9) : C(1) / C(36));
}
static_assert(opp(1) == 3 && opp(3) == 1 && opp(2) == 4 && opp(4) == 2, "opp");
static_assert(opp(5) == 7 && opp(7) == 5 && opp(6) == 8 && opp(8) == 6, "opp");
static_assert(ex(opp(6)) == -ex(6) && ey(opp(6)) == -ey(6), "opp");

// ---- storage formats ----------------------------------------------------------
// R: the raw stored type; C: the arithmetic type.
template <int PREC> struct Prec;
template <> struct Prec<SMRT_PREC_F64> {
    using R = double;
    using C = double;
    static constexpr bool kExactWeights = true;
    static __device__ __forceinline__ C to_c(R r) { return r; }
    static __device__ __forceinline__ R to_r(C c) { return c; }
};
template <> struct Prec<SMRT_PREC_F32> {
    using R = float;
    using C = float;
    static constexpr bool kExactWeights = true;
    static __device__ __forceinline__ C to_c(R r) { return r; }
    static __device__ __forceinline__ R to_r(C c) { return c; }
};
// Stochastic rounding (to_r_sr): c goes to one of its two neighbours in the storage format, the
// farther one with probability equal to the distance from the nearer one (in units of their
// spacing), so that the expected stored value is c itself.  r supplies 16 uniform bits.
// BF16 keeps the upper 16 bits of the float: adding r to the lower 16 and truncating is exactly
// that.  IEEE half keeps 10 of float's 23 mantissa bits where it is normal (|c| >= 2^-14): add 13 of
// the bits below them and truncate; below that its spacing is fixed at 2^-24, so a uniform fraction
// of 2^-24 is added before truncating.  Truncation is toward zero on the magnitude, so the rounding
// is symmetric in the sign.
template <> struct Prec<SMRT_PREC_F16> {
    using R = unsigned short;
    using C = float;
    static constexpr bool kExactWeights = false;
    static __device__ __forceinline__ C to_c(R r) { return __half2float(__ushort_as_half(r)); }
    static __device__ __forceinline__ R to_r(C c) { return __half_as_ushort(__float2half_rn(c)); }
    static __device__ __forceinline__ R to_r_sr(C c, uint32_t r)
    {
        const float yn = __uint_as_float(__float_as_uint(c) + (r & 0x1FFFu));
        const float ys = c + copysignf(__uint_as_float(0x33800000u) * ((float)(r & 0xFFFFu) * (1.0f / 65536.0f)), c);
        return __half_as_ushort(__float2half_rz(fabsf(c) >= 6.103515625e-05f ? yn : ys));
    }
};
template <> struct Prec<SMRT_PREC_BF16> {
    using R = unsigned short;
    using C = float;
    static constexpr bool kExactWeights = false;
    static __device__ __forceinline__ C to_c(R r) { return __bfloat162float(__ushort_as_bfloat16(r)); }
    static __device__ __forceinline__ R to_r(C c) { return __bfloat16_as_ushort(__float2bfloat16_rn(c)); }
    static __device__ __forceinline__ R to_r_sr(C c, uint32_t r)
    {
        return (R)((__float_as_uint(c) + (r & 0xFFFFu)) >> 16);
    }
};

// Counter-based random bits of the stochastic rounding: a 32-bit mix of the node's linear index and
// the step's salt (two multiply-xorshift rounds), and from it 16 bits per population by an odd
// multiplier per population (the upper half of the product).  Keyed by (node, population, time), so
// every layout and every code path that stores f*_a(x, t) draws the same bits.
__device__ __forceinline__ uint32_t sr_node_hash(uint32_t node, uint32_t salt)
{
    uint32_t h = node * 0x9E3779B1u + salt;
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 16;
    return h;
}
__device__ __forceinline__ uint32_t sr_pop_bits(uint32_t h, int a)
{
    const uint32_t m = a == 0 ? 0x9E3779B1u : a == 1 ? 0x85EBCA77u : a == 2 ? 0xC2B2AE3Du : a == 3 ? 0x27D4EB2Fu
                     : a == 4 ? 0x165667B1u : a == 5 ? 0xD3A2646Du : a == 6 ? 0xFD7046C5u : a == 7 ? 0xB55A4F09u
                     : 0x2545F491u;
    return (h * m) >> 16;
}
// The salt of the step that starts from time t (host side).
inline uint32_t sr_salt(long long t)
{
    uint64_t x = (uint64_t)t * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    x ^= x >> 31;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 29;
    return (uint32_t)(x >> 16);
}

// ---- kernel parameters --------------------------------------------------------
enum { SIDE_LEFT = 0, SIDE_RIGHT = 1, SIDE_BOTTOM = 2, SIDE_TOP = 3 };

template <class C>
struct Params {
    int nx, ny;
    int pitch;          // elements per stored row (>= nx, 128-byte multiple)
    long long plane;    // elements per population plane (pitch * ny)
    int periodic_x;     // left/right periodic
    int periodic_y;     // bottom/top periodic
    C omega;            // 1 / tau
    C omega_s;          // 1 / tau_s (two-relaxation-time form)
    C a4;               // (1 - 1/tau) / 4, SmrtLBM
    C trt4;             // (1/tau_s - 1/tau) / 4, two-relaxation-time form
    C corr[4][9];       // moving-wall term 6 w_a (e_a . u_w(side)) added to a wall-pulled offset
    int *flag;          // divergence flag (bit 0)
    uint32_t salt;      // stochastic rounding: the salt of this launch's time step
};

template <class C>
inline Params<C> make_params(const HostParams &h)
{
    Params<C> p;
    p.nx = h.nx;
    p.ny = h.ny;
    p.pitch = h.pitch;
    p.plane = h.plane;
    p.periodic_x = ((h.bc & 3u) == SMRT_BC_PERIODIC);
    p.periodic_y = (((h.bc >> 4) & 3u) == SMRT_BC_PERIODIC);
    p.omega = C(1.0 / h.tau);
    p.omega_s = C(1.0 / h.tau_s);
    p.a4 = C((1.0 - 1.0 / h.tau) / 4.0);
    p.trt4 = C((1.0 / h.tau_s - 1.0 / h.tau) / 4.0);
    for (int s = 0; s < 4; ++s) {
        unsigned kind = (h.bc >> (2 * s)) & 3u;
        double wx = 0.0, wy = 0.0;
        if (kind == SMRT_BC_MOVING) {
            if (s == SIDE_BOTTOM || s == SIDE_TOP) wx = h.u_lid;
            else wy = h.u_lid;
        }
        for (int a = 0; a < 9; ++a)
            p.corr[s][a] = C(6.0 * wgt<double>(a) * (ex(a) * wx + ey(a) * wy));
    }
    p.flag = h.flag;
    p.salt = sr_salt(h.t);
    return p;
}

// ---- boundary resolution --------------------------------------------------------
// Where a canonical population f_a(i, j) is found in storage.  `side` >= 0 marks a
// wall link (the pull source lies behind a wall on that side) whose stored value
// needs the moving-wall term p.corr[side][a] added.
struct Loc {
    int plane, j, i, side;
};

// Resolve the node (i + di, j + dj): wraps periodic axes; returns the wall side
// crossed (bottom/top take precedence over left/right), or -1 if inside.
template <class C>
__device__ __forceinline__ int resolve(const Params<C> &p, int &i, int &j)
{
    int wy = -1, wx = -1;
    if (j < 0) {
        if (p.periodic_y) j += p.ny; else wy = SIDE_BOTTOM;
    } else if (j >= p.ny) {
        if (p.periodic_y) j -= p.ny; else wy = SIDE_TOP;
    }
    if (i < 0) {
        if (p.periodic_x) i += p.nx; else wx = SIDE_LEFT;
    } else if (i >= p.nx) {
        if (p.periodic_x) i -= p.nx; else wx = SIDE_RIGHT;
    }
    return wy >= 0 ? wy : wx;
}

// Location of canonical f_a(i, j) under each storage mode:
//  AB      : f_a(x) = B_a(x - e_a)                    wall: B_{abar}(x) + corr
//  AA even : f_a(x) = F_a(x)                          wall: F_a(x) + corr
//  AA odd  : f_a(x) = F_{abar}(x - e_a)               wall: F_a(x) + corr
template <int MODE, class C>
__device__ __forceinline__ Loc pull_loc(const Params<C> &p, int a, int i, int j)
{
    int si = i - ex(a), sj = j - ey(a);
    int side = resolve(p, si, sj);
    Loc L;
    L.side = side;
    if (side >= 0) {
        L.plane = (MODE == MODE_AB) ? opp(a) : a;
        L.j = j;
        L.i = i;
    } else if (MODE == MODE_AA_EVEN) {
        L.plane = a;
        L.j = j;
        L.i = i;
    } else {
        L.plane = (MODE == MODE_AB) ? a : opp(a);
        L.j = sj;
        L.i = si;
    }
    return L;
}

// Where the post-collision f*_a(i, j) is written by a step of each mode:
//  AB      : B'_a(x)
//  AA even : F_{abar}(x)
//  AA odd  : F_a(x + e_a), or F_{abar}(x) when x + e_a lies behind a wall
template <int MODE, class C>
__device__ __forceinline__ Loc push_loc(const Params<C> &p, int a, int i, int j)
{
    Loc L;
    L.side = -1;
    if (MODE == MODE_AB) {
        L.plane = a; L.j = j; L.i = i;
    } else if (MODE == MODE_AA_EVEN) {
        L.plane = opp(a); L.j = j; L.i = i;
    } else {
        int ti = i + ex(a), tj = j + ey(a);
        int side = resolve(p, ti, tj);
        if (side >= 0) {
            L.plane = opp(a); L.j = j; L.i = i;
        } else {
            L.plane = a; L.j = tj; L.i = ti;
        }
    }
    return L;
}

__device__ __forceinline__ size_t at(long long plane_elems, int pitch, int plane, int j, int i)
{
    return (size_t)plane * (size_t)plane_elems + (size_t)j * (size_t)pitch + (size_t)i;
}

// ---- collision ------------------------------------------------------------------
// x * w for the D2Q9 weight w (4/9, 1/9 or 1/36), with the product rounded as if the
// weight were exact.  In float, w rounds to fl(w) = w (1 + 7.45e-9) for all three
// weights; a plain product would scale the equilibrium's mass and momentum by that
// factor at every collision (sum_a w_a = 1 and sum_a w_a e_a e_a = 1/3 hold for
// fl(w) only up to it).  The update then pushes the flow along itself by 7.45e-9 of
// its momentum per step, a coherent bias that grows linearly in time.  The split
// w = hi + lo (hi = fl(w), lo = fl(w - hi)) and one fused multiply-add remove it.
// Doubles keep the plain product: there the same bias is about 1e-17 per step.  So do the 16-bit
// storage formats (EXACT = false): rounding a stored offset to 11 or 8 significant bits moves it by
// 1e-4 to 1e-3 of itself each step, which buries the 7e-9, while the two extra operations per
// population cost their near-ALU-bound kernels several per cent.
template <class C, bool EXACT = true>
struct WeightMul {
    template <int A>
    static __device__ __forceinline__ C mul(C x) { return wgt<C>(A) * x; }
};
template <>
struct WeightMul<float, true> {
    template <int A>
    static __device__ __forceinline__ float mul(float x)
    {
        constexpr double w = wgt<double>(A);
        constexpr float hi = (float)w;
        constexpr float lo = (float)(w - (double)hi);
        return fmaf(hi, x, lo * x);
    }
};

// In:  g[a] = f_a - w_a (canonical offsets at one node).
// Out: g[a] = f*_a - w_a (post-collision offsets).
// Returns false when rho is not a positive finite number (divergence).
//
// Moments (Eq. fea-0):   rho = 1 + sum g,  j = sum e_a g_a,  u = j / rho.
// Equilibrium offsets (Eq. feq-full), written with rho u = j so that the momentum of
// the equilibrium is j itself rather than rho (j / rho) rounded twice:
//   f^eq_a - w_a = w_a [ (rho - 1) + 3 e.j + 9/2 (e.j)(e.u) - 3/2 j.u ].
// SmrtLBM (Eq. SmrtLBM-1): with n_k = f_k - f^eq_k the indicator sum is
//   C1 = (-n1 + n2 - n3 + n4)/4 for a in 1..4 and C2 = (-n5 + n6 - n7 + n8)/4 for
//   a in 5..8, so with Pxx = n1 - n2 + n3 - n4 = -4 C1 and Pxy = n5 - n6 + n7 - n8 = -4 C2
//   f*_a = f^eq_a + (-1)^a (1 - 1/tau) C = f^eq_a + s_a (1 - 1/tau)/4 P,
//   s = (+,-,+,-) over a = 1..4 (P = Pxx) and over a = 5..8 (P = Pxy), f*_0 = f^eq_0.
// SRT (Eq. lb.srt): f*_a = f_a - (f_a - f^eq_a) / tau.
// Two-tau (Eq. SmrtLBM-lb.1.5): f*_a = f_a - (f_a - f^eq_a)/tau_s + s_a (1/tau_s - 1/tau)/4 P.
template <int KIND, bool EXACT = true, class C>
__device__ __forceinline__ bool collide(const Params<C> &p, C g[9])
{
    using M = WeightMul<C, EXACT>;
    const C drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    const C rho = C(1) + drho;
    const C jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    const C jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
    const C inv = C(1) / rho;
    const C ux = jx * inv, uy = jy * inv;
    const bool ok = (rho > C(0)) && (rho < C(INFINITY));

    const C base = drho - C(1.5) * (jx * ux + jy * uy);
    const C jp = jx + jy, jm = jx - jy;
    const C up = ux + uy, um = ux - uy;
    const C axx = base + C(4.5) * jx * ux, bxx = C(3) * jx;
    const C ayy = base + C(4.5) * jy * uy, byy = C(3) * jy;
    const C app = base + C(4.5) * jp * up, bpp = C(3) * jp;
    const C amm = base + C(4.5) * jm * um, bmm = C(3) * jm;
    C q[9];
    q[0] = M::template mul<0>(base);
    q[1] = M::template mul<1>(axx + bxx);
    q[3] = M::template mul<3>(axx - bxx);
    q[2] = M::template mul<2>(ayy + byy);
    q[4] = M::template mul<4>(ayy - byy);
    q[5] = M::template mul<5>(app + bpp);
    q[7] = M::template mul<7>(app - bpp);
    q[8] = M::template mul<8>(amm + bmm);
    q[6] = M::template mul<6>(amm - bmm);

    if (KIND == SMRT_COLLISION_SRT) {
        #pragma unroll
        for (int a = 0; a < 9; ++a) g[a] = g[a] - p.omega * (g[a] - q[a]);
        return ok;
    }
    const C pxx = ((g[1] - q[1]) + (g[3] - q[3])) - ((g[2] - q[2]) + (g[4] - q[4]));
    const C pxy = ((g[5] - q[5]) + (g[7] - q[7])) - ((g[6] - q[6]) + (g[8] - q[8]));
    if (KIND == SMRT_COLLISION_SMRT) {
        const C txx = p.a4 * pxx, txy = p.a4 * pxy;
        g[0] = q[0];
        g[1] = q[1] + txx;
        g[3] = q[3] + txx;
        g[2] = q[2] - txx;
        g[4] = q[4] - txx;
        g[5] = q[5] + txy;
        g[7] = q[7] + txy;
        g[6] = q[6] - txy;
        g[8] = q[8] - txy;
    } else {
        const C txx = p.trt4 * pxx, txy = p.trt4 * pxy;
        #pragma unroll
        for (int a = 0; a < 9; ++a) g[a] = g[a] - p.omega_s * (g[a] - q[a]);
        g[1] += txx;
        g[3] += txx;
        g[2] -= txx;
        g[4] -= txx;
        g[5] += txy;
        g[7] += txy;
        g[6] -= txy;
        g[8] -= txy;
    }
    return ok;
}

} // namespace smrt
