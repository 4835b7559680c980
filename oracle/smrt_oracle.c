/*
 * smrt_oracle.c -- plain, slow, FP64 CPU oracle for the D2Q9 SmrtLBM update.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm use it.  It shares no code, header, table or
 * constant generator with the CUDA library; the two meet only through the
 * seeded input generators (workloads.py) and the test harness.
 *
 * Every function follows one passage of Zhou, "Single MRT-featured Lattice
 * Boltzmann Method (SmrtLBM)", arXiv 2409.01076, cited by equation label:
 *
 *   Eq. (lb.srt)        SRT-LBM update
 *   Eq. (feq-full)      equilibrium distribution
 *   Eq. (fea-0)         density and velocity moments
 *   Eq. (SmrtLBM-1)     the SmrtLBM update, with the indicator of Eq. (indicator-fn)
 *   Eq. (lb.1)          MRT update, M of Eq. (M-matrix), S of Eq. (S-matrix:1)
 *   Eq. (SmrtLBM-lb.1.5) two-relaxation-time form (tau_s, tau)
 *   Eq. (relation-chapman-viscosity)  nu = (2 tau - 1) e dx / 6
 *
 * The collision operators are written literally (the double sum over k with
 * the indicator function, signs (-1)^alpha and (-1)^k), not in any compacted
 * form.  Streaming is the push form of the left-hand side x + e_alpha dt.
 *
 * Readings where the paper is silent (all shared with the CUDA side by
 * specification only, never by code):
 *   - "standard bounce-back" (Sec. cavity flow) is halfway (link) bounce-back:
 *     a population leaving node x through a wall returns to x reversed one
 *     step later;
 *   - the moving lid u = (u0, 0) is moving-wall bounce-back with wall density
 *     rho_w = 1: the returning population is f*_a - 6 w_a rho_w (e_a . u_w);
 *   - a link that leaves through a bottom/top wall and a left/right side at
 *     once takes the bottom/top wall's velocity ("lid precedence");
 *   - a link that leaves through a wall in one axis is a wall link even when
 *     the other axis is periodic;
 *   - the canonical state f(t) is the post-streaming, pre-collision field (the
 *     left-hand side of Eq. (SmrtLBM-1)); macros at t are its moments.
 *
 * Layout of every lattice array: f[a][j][i] (a = 0..8, j = 0..ny-1 rows with
 * the top at ny-1, i = 0..nx-1), row-major, index (a*ny + j)*nx + i.
 *
 * bc_flags: 2 bits per side, left (bits 0-1), right (2-3), bottom (4-5),
 * top (6-7): 0 periodic, 1 resting wall, 2 wall moving with speed u_lid along
 * the side (along +x for bottom/top, along +y for left/right).
 *
 * Parity pinning status: every function here is pinned by a -m "not gpu"
 * test against a closed form, an identity the paper states, a second paper
 * equation, or a hand-derived tiny case; none is "parity unpinned".
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 velocities in the order the paper lists them below Eq. (lb.srt):
 * (0,0), (e,0), (0,e), (-e,0), (0,-e), (e,e), (-e,e), (-e,-e), (e,-e), e = 1. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

/* Weights below Eq. (feq-full): 4/9 (a = 0), 1/9 (a = 1-4), 1/36 (a = 5-8). */
static double weight(int a)
{
    if (a == 0) return 4.0 / 9.0;
    if (a <= 4) return 1.0 / 9.0;
    return 1.0 / 36.0;
}

/* The reversed link, found by searching for -e_a (not a typed-in table). */
static int opposite(int a)
{
    for (int b = 0; b < 9; ++b)
        if (EX[b] == -EX[a] && EY[b] == -EY[a]) return b;
    return -1;
}

/* (-1)^n for n >= 0. */
static double minus_one_pow(int n) { return (n % 2 == 0) ? 1.0 : -1.0; }

int orc_ex(int a) { return EX[a]; }
int orc_ey(int a) { return EY[a]; }
double orc_weight(int a) { return weight(a); }
int orc_opposite(int a) { return opposite(a); }

/* Eq. (feq-full) with e = 1:
 * f_a^eq = w_a rho (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u). */
double orc_feq(int a, double rho, double ux, double uy)
{
    double eu = EX[a] * ux + EY[a] * uy;
    double uu = ux * ux + uy * uy;
    return weight(a) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
}

void orc_feq_all(double rho, double ux, double uy, double *feq)
{
    for (int a = 0; a < 9; ++a) feq[a] = orc_feq(a, rho, ux, uy);
}

/* Eq. (fea-0): rho = sum_a f_a, u = (1/rho) sum_a e_a f_a. */
void orc_moments(const double *f, double *rho, double *ux, double *uy)
{
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < 9; ++a) {
        r += f[a];
        jx += EX[a] * f[a];
        jy += EY[a] * f[a];
    }
    *rho = r;
    *ux = jx / r;
    *uy = jy / r;
}

/* Eq. (indicator-fn): 1_{S}(m, n) = 1 if m in S and n in S, else 0. */
static int in_set(int x, int s0, int s1, int s2, int s3)
{
    return x == s0 || x == s1 || x == s2 || x == s3;
}
static double indicator(int s0, int s1, int s2, int s3, int m, int n)
{
    return (in_set(m, s0, s1, s2, s3) && in_set(n, s0, s1, s2, s3)) ? 1.0 : 0.0;
}

/* The indicator-weighted signed sum shared by Eqs. (SmrtLBM-1) and
 * (SmrtLBM-lb.1.5):
 *   sum_{k=1}^{8} (-1)^k / 4 [1_{1234}(a,k) + 1_{5678}(a,k)] (f_k - f_k^eq). */
static double indicator_sum(int a, const double *f, const double *feq)
{
    double s = 0.0;
    for (int k = 1; k <= 8; ++k) {
        double ind = indicator(1, 2, 3, 4, a, k) + indicator(5, 6, 7, 8, a, k);
        s += minus_one_pow(k) / 4.0 * ind * (f[k] - feq[k]);
    }
    return s;
}

/* Eq. (SmrtLBM-1), right-hand side at one node:
 *   f*_a = f_a^eq + (-1)^a (1 - 1/tau) * indicator_sum_a. */
void orc_collide_smrt(const double *f, double tau, double *out)
{
    double rho, ux, uy, feq[9];
    orc_moments(f, &rho, &ux, &uy);
    orc_feq_all(rho, ux, uy, feq);
    for (int a = 0; a < 9; ++a)
        out[a] = feq[a] + minus_one_pow(a) * (1.0 - 1.0 / tau) * indicator_sum(a, f, feq);
}

/* Eq. (lb.srt), right-hand side: f*_a = f_a - (f_a - f_a^eq) / tau. */
void orc_collide_srt(const double *f, double tau, double *out)
{
    double rho, ux, uy, feq[9];
    orc_moments(f, &rho, &ux, &uy);
    orc_feq_all(rho, ux, uy, feq);
    for (int a = 0; a < 9; ++a) out[a] = f[a] - (f[a] - feq[a]) / tau;
}

/* Eq. (SmrtLBM-lb.1.5), right-hand side:
 *   f*_a = f_a - (f_a - f_a^eq)/tau_s + (-1)^a (1/tau_s - 1/tau) * indicator_sum_a. */
void orc_collide_two_tau(const double *f, double tau_s, double tau, double *out)
{
    double rho, ux, uy, feq[9];
    orc_moments(f, &rho, &ux, &uy);
    orc_feq_all(rho, ux, uy, feq);
    for (int a = 0; a < 9; ++a)
        out[a] = f[a] - (f[a] - feq[a]) / tau_s
               + minus_one_pow(a) * (1.0 / tau_s - 1.0 / tau) * indicator_sum(a, f, feq);
}

/* Eq. (M-matrix), as printed in the appendix. */
static const double M_PAPER[81] = {
     1,  1,  1,  1,  1,  1,  1,  1,  1,
    -4, -1, -1, -1, -1,  2,  2,  2,  2,
     4, -2, -2, -2, -2,  1,  1,  1,  1,
     0,  1,  0, -1,  0,  1, -1, -1,  1,
     0, -2,  0,  2,  0,  1, -1, -1,  1,
     0,  0,  1,  0, -1,  1,  1, -1, -1,
     0,  0, -2,  0,  2,  1,  1, -1, -1,
     0,  1, -1,  1, -1,  0,  0,  0,  0,
     0,  0,  0,  0,  0,  1, -1,  1, -1,
};

void orc_mrt_M(double *m) { memcpy(m, M_PAPER, sizeof(M_PAPER)); }

/* M^{-1} by Gauss-Jordan elimination with partial pivoting in FP64.
 * Returns 0 on success, -1 if M were singular. */
int orc_mrt_Minv(double *minv)
{
    double a[9][18];
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 18; ++c)
            a[r][c] = (c < 9) ? M_PAPER[r * 9 + c] : (c - 9 == r ? 1.0 : 0.0);
    for (int col = 0; col < 9; ++col) {
        int piv = col;
        for (int r = col + 1; r < 9; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (fabs(a[piv][col]) < 1e-300) return -1;
        if (piv != col)
            for (int c = 0; c < 18; ++c) {
                double t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t;
            }
        double p = a[col][col];
        for (int c = 0; c < 18; ++c) a[col][c] /= p;
        for (int r = 0; r < 9; ++r) {
            if (r == col) continue;
            double fct = a[r][col];
            if (fct == 0.0) continue;
            for (int c = 0; c < 18; ++c) a[r][c] -= fct * a[col][c];
        }
    }
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) minv[r * 9 + c] = a[r][c + 9];
    return 0;
}

/* Eq. (lb.1), right-hand side: f* = f - M^{-1} S M (f - f^eq),
 * S = diag(s[0..8]) (Eq. (S-matrix:1) uses s = 1/tau_s for rows 0-6 and
 * 1/tau for rows 7-8). */
void orc_collide_mrt(const double *f, const double *s, double *out)
{
    double rho, ux, uy, feq[9], n[9], m[9], minv[81];
    orc_moments(f, &rho, &ux, &uy);
    orc_feq_all(rho, ux, uy, feq);
    orc_mrt_Minv(minv);
    for (int a = 0; a < 9; ++a) n[a] = f[a] - feq[a];
    for (int r = 0; r < 9; ++r) {
        double acc = 0.0;
        for (int c = 0; c < 9; ++c) acc += M_PAPER[r * 9 + c] * n[c];
        m[r] = s[r] * acc;
    }
    for (int a = 0; a < 9; ++a) {
        double acc = 0.0;
        for (int r = 0; r < 9; ++r) acc += minv[a * 9 + r] * m[r];
        out[a] = f[a] - acc;
    }
}

enum { ORC_SMRT = 0, ORC_SRT = 1, ORC_TWO_TAU = 2, ORC_MRT = 3 };

/* One node's collision of the chosen kind.  ORC_MRT uses
 * S = diag(1/tau_s x 7, 1/tau x 2), the assumption stated above
 * Eq. (S-matrix:1). */
int orc_collide(int kind, const double *f, double tau, double tau_s, double *out)
{
    switch (kind) {
    case ORC_SMRT: orc_collide_smrt(f, tau, out); return 0;
    case ORC_SRT: orc_collide_srt(f, tau, out); return 0;
    case ORC_TWO_TAU: orc_collide_two_tau(f, tau_s, tau, out); return 0;
    case ORC_MRT: {
        double s[9];
        for (int r = 0; r < 7; ++r) s[r] = 1.0 / tau_s;
        s[7] = s[8] = 1.0 / tau;
        orc_collide_mrt(f, s, out);
        return 0;
    }
    default: return -1;
    }
}

/* ---- lattice-level operations ------------------------------------------ */

enum { SIDE_LEFT = 0, SIDE_RIGHT = 1, SIDE_BOTTOM = 2, SIDE_TOP = 3 };
enum { BC_PERIODIC = 0, BC_WALL = 1, BC_MOVING = 2 };

static int side_kind(unsigned bc_flags, int side) { return (int)((bc_flags >> (2 * side)) & 3u); }

/* Wall velocity of one side: a moving wall slides along its own tangent. */
static void wall_velocity(unsigned bc_flags, int side, double u_lid, double *wx, double *wy)
{
    *wx = 0.0;
    *wy = 0.0;
    if (side_kind(bc_flags, side) != BC_MOVING) return;
    if (side == SIDE_BOTTOM || side == SIDE_TOP) *wx = u_lid;
    else *wy = u_lid;
}

int orc_check_bc(unsigned bc_flags)
{
    for (int s = 0; s < 4; ++s)
        if (side_kind(bc_flags, s) > BC_MOVING) return -1;
    if ((side_kind(bc_flags, SIDE_LEFT) == BC_PERIODIC) != (side_kind(bc_flags, SIDE_RIGHT) == BC_PERIODIC)) return -1;
    if ((side_kind(bc_flags, SIDE_BOTTOM) == BC_PERIODIC) != (side_kind(bc_flags, SIDE_TOP) == BC_PERIODIC)) return -1;
    if (bc_flags >> 8) return -1;
    return 0;
}

static size_t at(int nx, int ny, int a, int j, int i)
{
    return ((size_t)a * (size_t)ny + (size_t)j) * (size_t)nx + (size_t)i;
}

/* Streaming, the left-hand side of Eq. (SmrtLBM-1): the post-collision value
 * f*_a(x) moves to x + e_a.  Periodic sides wrap; a link that leaves through a
 * wall is bounced back halfway: next_{abar}(x) = f*_a(x) - 6 w_a rho_w (e_a . u_w). */
void orc_stream(int nx, int ny, unsigned bc_flags, double u_lid, double rho_w,
                const double *post, double *next)
{
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            for (int a = 0; a < 9; ++a) {
                int ti = i + EX[a], tj = j + EY[a];
                int wall_y = -1, wall_x = -1;
                if (tj < 0) {
                    if (side_kind(bc_flags, SIDE_BOTTOM) == BC_PERIODIC) tj += ny;
                    else wall_y = SIDE_BOTTOM;
                } else if (tj >= ny) {
                    if (side_kind(bc_flags, SIDE_TOP) == BC_PERIODIC) tj -= ny;
                    else wall_y = SIDE_TOP;
                }
                if (ti < 0) {
                    if (side_kind(bc_flags, SIDE_LEFT) == BC_PERIODIC) ti += nx;
                    else wall_x = SIDE_LEFT;
                } else if (ti >= nx) {
                    if (side_kind(bc_flags, SIDE_RIGHT) == BC_PERIODIC) ti -= nx;
                    else wall_x = SIDE_RIGHT;
                }
                double v = post[at(nx, ny, a, j, i)];
                if (wall_y >= 0 || wall_x >= 0) {
                    int side = (wall_y >= 0) ? wall_y : wall_x;
                    double wx, wy;
                    wall_velocity(bc_flags, side, u_lid, &wx, &wy);
                    double eu = EX[a] * wx + EY[a] * wy;
                    next[at(nx, ny, opposite(a), j, i)] = v - 6.0 * weight(a) * rho_w * eu;
                } else {
                    next[at(nx, ny, a, tj, ti)] = v;
                }
            }
}

/* Collision at every node of the canonical field f (in place into post).
 * The body force (fx, fy) is a test-only addition for the Poiseuille check,
 * f*_a += 3 w_a (e_a . F); the paper defines no forcing and the CUDA path has
 * none.  fx = fy = 0 leaves the paper's update untouched. */
int orc_collide_field(int nx, int ny, int kind, double tau, double tau_s,
                      double fx, double fy, const double *f, double *post)
{
    double fn[9], out[9];
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            for (int a = 0; a < 9; ++a) fn[a] = f[at(nx, ny, a, j, i)];
            if (orc_collide(kind, fn, tau, tau_s, out) != 0) return -1;
            for (int a = 0; a < 9; ++a) {
                double force = 3.0 * weight(a) * (EX[a] * fx + EY[a] * fy);
                post[at(nx, ny, a, j, i)] = out[a] + force;
            }
        }
    return 0;
}

/* nsteps applications of the update on the canonical field f (in place). */
int orc_run(int nx, int ny, unsigned bc_flags, double u_lid, int kind,
            double tau, double tau_s, double fx, double fy, double *f, long long nsteps)
{
    if (nx < 1 || ny < 1 || orc_check_bc(bc_flags) != 0) return -1;
    size_t n = (size_t)9 * (size_t)nx * (size_t)ny;
    double *post = (double *)malloc(n * sizeof(double));
    if (!post) return -2;
    for (long long s = 0; s < nsteps; ++s) {
        if (orc_collide_field(nx, ny, kind, tau, tau_s, fx, fy, f, post) != 0) {
            free(post);
            return -1;
        }
        orc_stream(nx, ny, bc_flags, u_lid, 1.0, post, f);
    }
    free(post);
    return 0;
}

/* f = f^eq(rho, u) at every node, Eq. (feq-full).  u holds the ux plane then
 * the uy plane, each [ny][nx]. */
void orc_init_equilibrium(int nx, int ny, const double *rho, const double *u, double *f)
{
    size_t plane = (size_t)nx * (size_t)ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t p = (size_t)j * nx + i;
            for (int a = 0; a < 9; ++a)
                f[at(nx, ny, a, j, i)] = orc_feq(a, rho[p], u[p], u[plane + p]);
        }
}

/* Eq. (fea-0) at every node: rho[ny][nx], u = [ux plane][uy plane]. */
void orc_macros(int nx, int ny, const double *f, double *rho, double *u)
{
    size_t plane = (size_t)nx * (size_t)ny;
    double fn[9];
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t p = (size_t)j * nx + i;
            for (int a = 0; a < 9; ++a) fn[a] = f[at(nx, ny, a, j, i)];
            double r, ux, uy;
            orc_moments(fn, &r, &ux, &uy);
            rho[p] = r;
            u[p] = ux;
            u[plane + p] = uy;
        }
}

/* Steady-state residual (the paper states no criterion; this is the reading
 * used throughout): r(t) = ||u(t+1) - u(t)||_2 / ||u(t+1)||_2 over all nodes,
 * computed by advancing a copy of f one step (f itself is untouched).
 * r = 0 when both norms vanish.  sums (may be NULL) receives
 * {sum rho(t), sum rho ux(t), sum rho uy(t)}. */
int orc_residual(int nx, int ny, unsigned bc_flags, double u_lid, int kind,
                 double tau, double tau_s, const double *f, double *r, double *sums)
{
    size_t plane = (size_t)nx * (size_t)ny;
    double *g = (double *)malloc(9 * plane * sizeof(double));
    double *rho0 = (double *)malloc(plane * sizeof(double));
    double *u0 = (double *)malloc(2 * plane * sizeof(double));
    double *rho1 = (double *)malloc(plane * sizeof(double));
    double *u1 = (double *)malloc(2 * plane * sizeof(double));
    int rc = 0;
    if (!g || !rho0 || !u0 || !rho1 || !u1) { rc = -2; goto done; }
    memcpy(g, f, 9 * plane * sizeof(double));
    orc_macros(nx, ny, f, rho0, u0);
    rc = orc_run(nx, ny, bc_flags, u_lid, kind, tau, tau_s, 0.0, 0.0, g, 1);
    if (rc != 0) goto done;
    orc_macros(nx, ny, g, rho1, u1);
    double num = 0.0, den = 0.0, m = 0.0, px = 0.0, py = 0.0;
    for (size_t p = 0; p < plane; ++p) {
        double dx = u1[p] - u0[p], dy = u1[plane + p] - u0[plane + p];
        num += dx * dx + dy * dy;
        den += u1[p] * u1[p] + u1[plane + p] * u1[plane + p];
        m += rho0[p];
        px += rho0[p] * u0[p];
        py += rho0[p] * u0[plane + p];
    }
    if (r) *r = (num == 0.0 && den == 0.0) ? 0.0 : sqrt(num) / sqrt(den);
    if (sums) { sums[0] = m; sums[1] = px; sums[2] = py; }
done:
    free(g); free(rho0); free(u0); free(rho1); free(u1);
    return rc;
}
