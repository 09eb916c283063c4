/*
 * gcb_oracle_ks.c -- FP64 CPU oracle of the covariant (Kerr-Schild) coupled
 * pusher of Bacchini et al. (2020): GREOM (Sec. 2.3), GRGCA (Sec. 2.4) and
 * their coupling (Sec. 3, 3.2), geometrized units c = G = M = 1.
 *
 * TEST INFRASTRUCTURE ONLY (see gcb_oracle.h).  Metric derivatives are taken
 * with forward-mode dual numbers over the closed-form Kerr-Schild 3+1
 * functions and a numerical 3x3 inverse, so they are derived independently of
 * any hand-written derivative.
 *
 * Parity pins: tests/test_oracle_ks_pins.py (metric identities, Minkowski
 * limit, horizon, dual derivatives vs differences, conserved u_phi and
 * energy of geodesics, circular equatorial orbits, local-frame identities,
 * flat-space cell sizes, GRGCA drift and parallel acceleration).
 */
#define _DEFAULT_SOURCE
#include "gcb_oracle.h"

#include <math.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------------- */
/* dual numbers over (r, theta)                                            */
/* ---------------------------------------------------------------------- */
typedef struct { double v, d[2]; } dual;

static dual dc(double v) { dual x = {v, {0, 0}}; return x; }
static dual dadd(dual a, dual b) { dual x = {a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1]}}; return x; }
static dual dsub(dual a, dual b) { dual x = {a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1]}}; return x; }
static dual dmul(dual a, dual b)
{
    dual x = {a.v * b.v, {a.d[0] * b.v + a.v * b.d[0], a.d[1] * b.v + a.v * b.d[1]}};
    return x;
}
static dual ddiv(dual a, dual b)
{
    double iv = 1.0 / b.v;
    dual x = {a.v * iv, {(a.d[0] - a.v * iv * b.d[0]) * iv, (a.d[1] - a.v * iv * b.d[1]) * iv}};
    return x;
}
static dual dsqrt(dual a)
{
    double s = sqrt(a.v);
    dual x = {s, {0.5 * a.d[0] / s, 0.5 * a.d[1] / s}};
    return x;
}
static dual dsin(dual a) { dual x = {sin(a.v), {cos(a.v) * a.d[0], cos(a.v) * a.d[1]}}; return x; }
static dual dcos(dual a) { dual x = {cos(a.v), {-sin(a.v) * a.d[0], -sin(a.v) * a.d[1]}}; return x; }
static dual dscale(dual a, double s) { dual x = {a.v * s, {a.d[0] * s, a.d[1] * s}}; return x; }

/* Kerr-Schild 3+1 functions (spherical KS coordinates r, theta, phi; M = 1):
 *   rho^2 = r^2 + a^2 cos^2(theta),  z = 2 r / rho^2,
 *   alpha = (1 + z)^{-1/2},  beta^r = z / (1 + z),  beta^theta = beta^phi = 0,
 *   gamma_rr = 1 + z,  gamma_rphi = -a (1 + z) sin^2,  gamma_thth = rho^2,
 *   gamma_phph = (r^2 + a^2 + z a^2 sin^2) sin^2  (others zero),
 * from the Kerr metric in Kerr-Schild form; gamma^{ij} is the numerical
 * inverse of gamma_ij. */
typedef struct {
    dual alpha, beta[3], gdn[3][3], gup[3][3], sqrtg;
} dmetric;

static void ks_metric_dual(double a, double r, double th, dmetric *m)
{
    dual R = {r, {1, 0}}, T = {th, {0, 1}};
    dual s = dsin(T), c = dcos(T);
    dual s2 = dmul(s, s);
    dual rho2 = dadd(dmul(R, R), dscale(dmul(c, c), a * a));
    dual z = ddiv(dscale(R, 2.0), rho2);
    dual onez = dadd(dc(1.0), z);
    m->alpha = ddiv(dc(1.0), dsqrt(onez));
    m->beta[0] = ddiv(z, onez);
    m->beta[1] = dc(0.0);
    m->beta[2] = dc(0.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) m->gdn[i][j] = dc(0.0);
    m->gdn[0][0] = onez;
    m->gdn[0][2] = m->gdn[2][0] = dscale(dmul(onez, s2), -a);
    m->gdn[1][1] = rho2;
    m->gdn[2][2] = dmul(dadd(dadd(dmul(R, R), dc(a * a)), dscale(dmul(z, s2), a * a)), s2);
    /* inverse by cofactors */
    dual (*g)[3] = m->gdn;
    dual c00 = dsub(dmul(g[1][1], g[2][2]), dmul(g[1][2], g[2][1]));
    dual c01 = dsub(dmul(g[1][2], g[2][0]), dmul(g[1][0], g[2][2]));
    dual c02 = dsub(dmul(g[1][0], g[2][1]), dmul(g[1][1], g[2][0]));
    dual det = dadd(dadd(dmul(g[0][0], c00), dmul(g[0][1], c01)), dmul(g[0][2], c02));
    dual inv[3][3];
    inv[0][0] = c00;
    inv[0][1] = dsub(dmul(g[0][2], g[2][1]), dmul(g[0][1], g[2][2]));
    inv[0][2] = dsub(dmul(g[0][1], g[1][2]), dmul(g[0][2], g[1][1]));
    inv[1][0] = c01;
    inv[1][1] = dsub(dmul(g[0][0], g[2][2]), dmul(g[0][2], g[2][0]));
    inv[1][2] = dsub(dmul(g[0][2], g[1][0]), dmul(g[0][0], g[1][2]));
    inv[2][0] = c02;
    inv[2][1] = dsub(dmul(g[0][1], g[2][0]), dmul(g[0][0], g[2][1]));
    inv[2][2] = dsub(dmul(g[0][0], g[1][1]), dmul(g[0][1], g[1][0]));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) m->gup[i][j] = ddiv(inv[i][j], det);
    m->sqrtg = dsqrt(det);
}

/* plain metric values and derivatives at a point */
typedef struct {
    double alpha, beta[3], gdn[3][3], gup[3][3], sqrtg;
    double dalpha[3], dbeta[3][3], dgup[3][3][3];   /* d_i alpha, d_i beta^j, d_i gamma^{jk} */
} metric_t;

static void ks_metric(double a, double r, double th, metric_t *M)
{
    dmetric m;
    ks_metric_dual(a, r, th, &m);
    memset(M, 0, sizeof(*M));
    M->alpha = m.alpha.v;
    M->sqrtg = m.sqrtg.v;
    for (int i = 0; i < 2; ++i) M->dalpha[i] = m.alpha.d[i];
    for (int j = 0; j < 3; ++j) {
        M->beta[j] = m.beta[j].v;
        for (int i = 0; i < 2; ++i) M->dbeta[i][j] = m.beta[j].d[i];
    }
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
            M->gdn[j][k] = m.gdn[j][k].v;
            M->gup[j][k] = m.gup[j][k].v;
            for (int i = 0; i < 2; ++i) M->dgup[i][j][k] = m.gup[j][k].d[i];
        }
}

void orc_ks_metric(double a, double r, double th, double out[64])
{
    metric_t M;
    ks_metric(a, r, th, &M);
    int k = 0;
    out[k++] = M.alpha;
    for (int i = 0; i < 3; ++i) out[k++] = M.beta[i];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) out[k++] = M.gdn[i][j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) out[k++] = M.gup[i][j];
    out[k++] = M.sqrtg;
    for (int i = 0; i < 3; ++i) out[k++] = M.dalpha[i];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) out[k++] = M.dbeta[i][j];
    /* k = 35; the 27 d_i gamma^{jk} follow */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int l = 0; l < 3; ++l) out[k++] = M.dgup[i][j][l];
}

/* ---------------------------------------------------------------------- */
/* fields: linear shape functions on the (log r, theta) node grid (Sec. 4  */
/* intro), not periodic: the cell index is clamped to the grid, so a point  */
/* just outside is extrapolated from the edge cell.                         */
/* ---------------------------------------------------------------------- */
static void ks_cell(const orc_ks_field *f, double r, double th, int *i, int *j, double *tr,
                    double *tt)
{
    double s = (log(r) - f->logr0) / f->dlogr;
    double q = th / f->dth;
    int ci = (int)floor(s), cj = (int)floor(q);
    if (ci < 0) ci = 0;
    if (ci > f->nr - 2) ci = f->nr - 2;
    if (cj < 0) cj = 0;
    if (cj > f->nth - 2) cj = f->nth - 2;
    *i = ci;
    *j = cj;
    *tr = s - ci;
    *tt = q - cj;
}

void orc_ks_gather(const orc_ks_field *f, double r, double th, double D[3], double B[3])
{
    for (int k = 0; k < 3; ++k) D[k] = B[k] = 0.0;
    if (f->kind == ORC_KS_VACUUM) return;
    if (f->kind == ORC_KS_MONOPOLE) {
        /* divergence-free monopole: d_r (sqrt(gamma) B^r) = 0 */
        metric_t M;
        ks_metric(f->par[1], r, th, &M);
        B[0] = f->par[0] * sin(th) / M.sqrtg;
        return;
    }
    int i, j;
    double tr, tt;
    ks_cell(f, r, th, &i, &j, &tr, &tt);
    for (int o = 0; o < 4; ++o) {
        int oi = o & 1, oj = o >> 1;
        double W = (oi ? tr : 1.0 - tr) * (oj ? tt : 1.0 - tt);
        long node = (long)(j + oj) * f->nr + (i + oi);
        for (int k = 0; k < 3; ++k) {
            D[k] += f->D[k][node] * W;
            B[k] += f->B[k][node] * W;
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Effective cell size (Sec. 3, Eq. volint).  Reading: on the axisymmetric */
/* (r, theta) grid the 2D proper element is sqrt(gamma_rr gamma_thth -     */
/* gamma_rth^2) dr dtheta; dl = (its integral over the cell)^(1/2), by 4x4  */
/* Gauss-Legendre quadrature in (r, theta).                                */
/* ---------------------------------------------------------------------- */
static const double GLX[4] = {-0.8611363115940526, -0.3399810435848563, 0.3399810435848563,
                              0.8611363115940526};
static const double GLW[4] = {0.3478548451374538, 0.6521451548625461, 0.6521451548625461,
                              0.3478548451374538};

void orc_ks_cell_sizes(const orc_ks_field *f, double a, double *dl)
{
    for (int j = 0; j < f->nth - 1; ++j) {
        double t0 = j * f->dth, t1 = (j + 1) * f->dth;
        for (int i = 0; i < f->nr - 1; ++i) {
            double r0 = exp(f->logr0 + i * f->dlogr), r1 = exp(f->logr0 + (i + 1) * f->dlogr);
            double area = 0.0;
            for (int p = 0; p < 4; ++p)
                for (int q = 0; q < 4; ++q) {
                    double r = 0.5 * (r0 + r1) + 0.5 * (r1 - r0) * GLX[p];
                    double th = 0.5 * (t0 + t1) + 0.5 * (t1 - t0) * GLX[q];
                    metric_t M;
                    ks_metric(a, r, th, &M);
                    double g2 = M.gdn[0][0] * M.gdn[1][1] - M.gdn[0][1] * M.gdn[0][1];
                    area += GLW[p] * GLW[q] * sqrt(g2);
                }
            area *= 0.25 * (r1 - r0) * (t1 - t0);
            dl[(long)j * (f->nr - 1) + i] = sqrt(area);
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Local frame (Sec. 2.3: orthonormal tetrads, not specified in the paper).*/
/* Reading: the triad e_(a)^i = L^i_a with gamma^{ij} = L L^T (Cholesky), so */
/* covariant u has frame components u^ = L^T u and a contravariant field F  */
/* has F^ = L^{-1} F; then gamma^{ij} u_i u_j = |u^|^2 and the Lorentz force */
/* alpha q/m (gamma_ij D^j + e_ijk gamma^{jl} u_l B^k / Gamma) becomes       */
/* alpha q/m (D^ + u^ x B^ / Gamma).                                        */
/* ---------------------------------------------------------------------- */
static void chol3(const double A[3][3], double L[3][3])
{
    memset(L, 0, 9 * sizeof(double));
    for (int j = 0; j < 3; ++j) {
        double s = A[j][j];
        for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
        L[j][j] = sqrt(s);
        for (int i = j + 1; i < 3; ++i) {
            double t = A[i][j];
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t / L[j][j];
        }
    }
}

static void frame_in(const double L[3][3], const double u[3], double uh[3])
{
    for (int a = 0; a < 3; ++a) {   /* u^_a = sum_i L[i][a] u_i */
        uh[a] = 0.0;
        for (int i = 0; i < 3; ++i) uh[a] += L[i][a] * u[i];
    }
}

static void frame_out(const double L[3][3], const double uh[3], double u[3])
{
    /* solve L^T u = uh (L^T upper triangular) */
    for (int i = 2; i >= 0; --i) {
        double s = uh[i];
        for (int k = i + 1; k < 3; ++k) s -= L[k][i] * u[k];
        u[i] = s / L[i][i];
    }
}

static void field_in(const double L[3][3], const double F[3], double Fh[3])
{
    /* solve L Fh = F (L lower triangular) */
    for (int i = 0; i < 3; ++i) {
        double s = F[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * Fh[k];
        Fh[i] = s / L[i][i];
    }
}

/* Boris push over proper time dtau in the local frame (Sec. 2.3 step 1/3). */
static void boris_local(const double E[3], const double B[3], double qm, double dtau, double u[3])
{
    double h = 0.5 * qm * dtau, um[3], t[3], s[3], up[3], x[3];
    for (int k = 0; k < 3; ++k) um[k] = u[k] + h * E[k];
    double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int k = 0; k < 3; ++k) t[k] = h * B[k] / gm;
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int k = 0; k < 3; ++k) s[k] = 2.0 * t[k] / (1.0 + t2);
    x[0] = um[1] * t[2] - um[2] * t[1];
    x[1] = um[2] * t[0] - um[0] * t[2];
    x[2] = um[0] * t[1] - um[1] * t[0];
    for (int k = 0; k < 3; ++k) up[k] = um[k] + x[k];
    x[0] = up[1] * s[2] - up[2] * s[1];
    x[1] = up[2] * s[0] - up[0] * s[2];
    x[2] = up[0] * s[1] - up[1] * s[0];
    for (int k = 0; k < 3; ++k) u[k] = um[k] + x[k] + h * E[k];
}

/* ---------------------------------------------------------------------- */
/* The same kick in the global coordinate basis (Sec. 2.3 and 2.4 name a    */
/* Boris-like push without tetrads as an option).  Reading: the three Boris */
/* stages with each frame dot product replaced by its metric contraction    */
/* and the frame cross product by the Levi-Civita tensor                    */
/* e_ijk = sqrt(gamma) [ijk] acting on raised vectors (covariant result):   */
/*   u-_i = u_i + h gamma_ij D^j,   Gamma- = (1 + gamma^{ij} u-_i u-_j)^(1/2),  */
/*   t^k = h B^k / Gamma-,          s^k = 2 t^k / (1 + gamma_ij t^i t^j),   */
/*   u'_i = u-_i + e_ijk (gamma^{jl} u-_l) t^k,                              */
/*   u+_i = u-_i + e_ijk (gamma^{jl} u'_l) s^k,   u_i <- u+_i + h gamma_ij D^j. */
/* It reproduces the frame kick because the triad L has det L = 1/sqrt(gamma). */
/* ---------------------------------------------------------------------- */
static double levi_civita(int i, int j, int k)
{
    return 0.5 * (double)((i - j) * (j - k) * (k - i));
}

static void contract(const double G[3][3], const double v[3], double w[3])
{
    for (int i = 0; i < 3; ++i) {
        w[i] = 0.0;
        for (int j = 0; j < 3; ++j) w[i] += G[i][j] * v[j];
    }
}

static void cross_covariant(const metric_t *M, const double a_up[3], const double b_up[3],
                            double c[3])
{
    for (int i = 0; i < 3; ++i) {
        c[i] = 0.0;
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) c[i] += M->sqrtg * levi_civita(i, j, k) * a_up[j] * b_up[k];
    }
}

static void boris_global(const metric_t *M, const double D[3], const double B[3], double qm,
                         double dtau, double u[3])
{
    double h = 0.5 * qm * dtau, Dd[3], um[3], um_up[3], t[3], t_dn[3], s[3], up[3], up_up[3], x[3];
    contract(M->gdn, D, Dd);
    for (int k = 0; k < 3; ++k) um[k] = u[k] + h * Dd[k];
    contract(M->gup, um, um_up);
    double gm = sqrt(1.0 + um[0] * um_up[0] + um[1] * um_up[1] + um[2] * um_up[2]);
    for (int k = 0; k < 3; ++k) t[k] = h * B[k] / gm;
    contract(M->gdn, t, t_dn);
    double t2 = t[0] * t_dn[0] + t[1] * t_dn[1] + t[2] * t_dn[2];
    for (int k = 0; k < 3; ++k) s[k] = 2.0 * t[k] / (1.0 + t2);
    cross_covariant(M, um_up, t, x);
    for (int k = 0; k < 3; ++k) up[k] = um[k] + x[k];
    contract(M->gup, up, up_up);
    cross_covariant(M, up_up, s, x);
    for (int k = 0; k < 3; ++k) u[k] = um[k] + x[k] + h * Dd[k];
}

/* Kick of covariant u by the contravariant fields D, B at (r, theta) over
 * proper time dtau, in the local frame (basis 0) or the global basis (1). */
static void ks_kick(double a, double r, double th, const double D[3], const double B[3],
                    double qm, double dtau, int basis, double u[3])
{
    metric_t M;
    ks_metric(a, r, th, &M);
    if (basis == 1) {
        boris_global(&M, D, B, qm, dtau, u);
        return;
    }
    double L[3][3], uh[3], Dh[3], Bh[3];
    chol3(M.gup, L);
    frame_in(L, u, uh);
    field_in(L, D, Dh);
    field_in(L, B, Bh);
    boris_local(Dh, Bh, qm, dtau, uh);
    frame_out(L, uh, u);
}

void orc_ks_kick(double a, double r, double th, const double D[3], const double B[3], double qm,
                 double dtau, int basis, double u[3])
{
    ks_kick(a, r, th, D, B, qm, dtau, basis, u);
}

/* GREOM half kick (Sec. 2.3 steps 1 and 3): fields and metric at x, proper
 * time alpha dt / 2. */
static void ks_half_kick(const orc_ks_field *f, double a, int basis, double qm, double dt,
                         const double x[3], double u[3])
{
    double D[3], B[3], alpha;
    orc_ks_gather(f, x[0], x[1], D, B);
    {
        metric_t M;
        ks_metric(a, x[0], x[1], &M);
        alpha = M.alpha;
    }
    ks_kick(a, x[0], x[1], D, B, qm, 0.5 * dt * alpha, basis, u);
}

/* 3+1 geodesic terms (Sec. 2.3): V^i = alpha gamma^{ij} u_j / Gamma - beta^i,
 * G_i = -Gamma d_i alpha + u_j d_i beta^j - alpha u_j u_k d_i gamma^{jk} / (2 Gamma). */
static void geodesic_rhs(const metric_t *M, const double u[3], double Gam, double V[3], double G[3])
{
    for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j) s += M->gup[i][j] * u[j];
        V[i] = M->alpha * s / Gam - M->beta[i];
    }
    for (int i = 0; i < 3; ++i) {
        double ub = 0.0, uu = 0.0;
        for (int j = 0; j < 3; ++j) {
            ub += u[j] * M->dbeta[i][j];
            for (int k = 0; k < 3; ++k) uu += u[j] * u[k] * M->dgup[i][j][k];
        }
        G[i] = -Gam * M->dalpha[i] + ub - M->alpha * uu / (2.0 * Gam);
    }
}

static double lorentz(const metric_t *M, const double u[3])
{
    double s = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s += M->gup[i][j] * u[i] * u[j];
    return sqrt(1.0 + s);
}

static int ks_converged(const orc_params *p, int iters, double res, int *nonconv)
{
    if (p->fixed_iters > 0) return iters >= p->fixed_iters;
    if (res < p->tol) return 1;
    if (iters >= p->max_iter) { *nonconv = 1; return 1; }
    return 0;
}

/* GREOM step (Sec. 2.3): half kick at x^n, IMR for (x, u), half kick at x^{n+1}. */
static int greom_step(const orc_ks_field *f, double a, int basis, const orc_params *p, double qm,
                      double x[3], double u[3], int *iters, int *nonconv, double *resid)
{
    double dt = p->dt;
    double up[3] = {u[0], u[1], u[2]};
    ks_half_kick(f, a, basis, qm, dt, x, up);
    double xk[3] = {x[0], x[1], x[2]}, wk[3] = {up[0], up[1], up[2]};
    *iters = 0;
    *nonconv = 0;
    for (;;) {
        double xb[3], ub[3];
        for (int k = 0; k < 3; ++k) { xb[k] = 0.5 * (xk[k] + x[k]); ub[k] = 0.5 * (wk[k] + up[k]); }
        metric_t M;
        ks_metric(a, xb[0], xb[1], &M);
        double Gam = lorentz(&M, ub), V[3], G[3];
        geodesic_rhs(&M, ub, Gam, V, G);
        double res = 0.0, xn[3], wn[3];
        for (int k = 0; k < 3; ++k) {
            xn[k] = x[k] + dt * V[k];
            wn[k] = up[k] + dt * G[k];
            res = fmax(res, fmax(fabs(xn[k] - xk[k]), fabs(wn[k] - wk[k])));
            xk[k] = xn[k];
            wk[k] = wn[k];
        }
        ++*iters;
        *resid = res;
        if (ks_converged(p, *iters, res, nonconv)) break;
    }
    ks_half_kick(f, a, basis, qm, dt, xk, wk);
    for (int k = 0; k < 3; ++k) { x[k] = xk[k]; u[k] = wk[k]; }
    return 1;
}

/* GRGCA frame at a point (Sec. 2.4): B_i = gamma_ij B^j, B = (B_i B^i)^(1/2),
 * b_i = B_i / B, b^i = B^i / B, v_E,i = e_ijk D^j B^k / B^2 with
 * e_ijk = sqrt(gamma) epsilon_ijk, kappa = (1 - gamma^{ij} v_E,i v_E,j)^(-1/2),
 * D_par = D^i b_i. */
typedef struct {
    metric_t M;
    double D[3], B[3], Bmag, bdn[3], bup[3], vE[3], kappa, Dpar;
    int ok;
} gframe_t;

static void gr_frame(const orc_ks_field *f, double a, const double R[3], gframe_t *F)
{
    ks_metric(a, R[0], R[1], &F->M);
    orc_ks_gather(f, R[0], R[1], F->D, F->B);
    double Bd[3];
    for (int i = 0; i < 3; ++i) {
        Bd[i] = 0.0;
        for (int j = 0; j < 3; ++j) Bd[i] += F->M.gdn[i][j] * F->B[j];
    }
    double B2 = Bd[0] * F->B[0] + Bd[1] * F->B[1] + Bd[2] * F->B[2];
    F->ok = B2 > 0.0;
    if (!F->ok) return;
    F->Bmag = sqrt(B2);
    for (int i = 0; i < 3; ++i) { F->bdn[i] = Bd[i] / F->Bmag; F->bup[i] = F->B[i] / F->Bmag; }
    const double *D = F->D, *B = F->B;
    double sg = F->M.sqrtg;
    F->vE[0] = sg * (D[1] * B[2] - D[2] * B[1]) / B2;
    F->vE[1] = sg * (D[2] * B[0] - D[0] * B[2]) / B2;
    F->vE[2] = sg * (D[0] * B[1] - D[1] * B[0]) / B2;
    double v2 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) v2 += F->M.gup[i][j] * F->vE[i] * F->vE[j];
    if (!(v2 < 1.0)) { F->ok = 0; return; }
    F->kappa = 1.0 / sqrt(1.0 - v2);
    F->Dpar = D[0] * F->bdn[0] + D[1] * F->bdn[1] + D[2] * F->bdn[2];
}

static double gr_perp2(const gframe_t *F, const orc_params *p, double mu, double uperp)
{
    return p->mu_mode == ORC_UPERP_CONSERVE ? uperp * uperp : 2.0 * mu * F->Bmag * F->kappa;
}

/* Eq. (grgcalfac): Gamma = kappa (1 + u_par^2 + 2 mu B kappa / m)^(1/2). */
static double gr_gamma(const gframe_t *F, const orc_params *p, double upar, double mu, double uperp)
{
    return F->kappa * sqrt(1.0 + upar * upar + gr_perp2(F, p, mu, uperp));
}

/* GRGCA step (Sec. 2.4 steps 1-3) from R^n = x^n with decomposed u_par, mu, b_perp,g. */
static int grgca_step(const orc_ks_field *f, double a, const orc_params *p, double qm,
                      const gframe_t *F0, double R[3], double *upar, double mu, double uperp,
                      const double bpg[3], int *iters, int *nonconv, double *resid)
{
    double dt = p->dt;
    double u1 = *upar + 0.5 * dt * F0->M.alpha * qm * F0->Dpar;   /* first half push */
    double Rk[3] = {R[0], R[1], R[2]}, wk = u1;
    *iters = 0;
    *nonconv = 0;
    for (;;) {
        double Rb[3];
        for (int k = 0; k < 3; ++k) Rb[k] = 0.5 * (Rk[k] + R[k]);
        double ub = 0.5 * (wk + u1);
        gframe_t Fb;
        gr_frame(f, a, Rb, &Fb);
        if (!Fb.ok) return 0;
        double Gam = gr_gamma(&Fb, p, ub, mu, uperp);
        double ug = sqrt(gr_perp2(&Fb, p, mu, uperp));
        double uful[3], V[3], G[3], tmp[3];
        for (int i = 0; i < 3; ++i) uful[i] = ub * Fb.bdn[i] + Fb.vE[i] * Gam + ug * bpg[i];
        /* Eq. (geoV): V~^i = alpha (u_par gamma^{ij} b_j / Gamma + gamma^{ij} v_E,j) - beta^i */
        for (int i = 0; i < 3; ++i) {
            double s = 0.0;
            for (int j = 0; j < 3; ++j) s += Fb.M.gup[i][j] * (ub * Fb.bdn[j] / Gam + Fb.vE[j]);
            V[i] = Fb.M.alpha * s - Fb.M.beta[i];
        }
        geodesic_rhs(&Fb.M, uful, Gam, tmp, G);
        double Gb = G[0] * Fb.bup[0] + G[1] * Fb.bup[1] + G[2] * Fb.bup[2];
        double res = 0.0;
        for (int k = 0; k < 3; ++k) {
            double rn = R[k] + dt * V[k];
            res = fmax(res, fabs(rn - Rk[k]));
            Rk[k] = rn;
        }
        double wn = u1 + dt * Gb;
        res = fmax(res, fabs(wn - wk));
        wk = wn;
        ++*iters;
        *resid = res;
        if (ks_converged(p, *iters, res, nonconv)) break;
    }
    gframe_t F1;
    gr_frame(f, a, Rk, &F1);
    if (!F1.ok) return 0;
    *upar = wk + 0.5 * dt * F1.M.alpha * qm * F1.Dpar;            /* second half push */
    for (int k = 0; k < 3; ++k) R[k] = Rk[k];
    return 1;
}

static double wrap_phi(double ph)
{
    double w = ph - 2.0 * M_PI * floor(ph / (2.0 * M_PI));
    return w >= 2.0 * M_PI ? w - 2.0 * M_PI : w;
}

/* One coupled GR step (Sec. 3.2) of one particle. */
void orc_ks_step_one(const orc_ks_field *f, const orc_ks_params *kp, const orc_params *p,
                     const double *dl, double x[3], double u[3], unsigned char *flags,
                     orc_detail *d)
{
    orc_detail dd;
    if (!d) d = &dd;
    memset(d, 0, sizeof(*d));
    unsigned char fl = *flags;
    if (fl & (ORC_FLAG_NONFINITE | ORC_FLAG_EXITED)) { d->branch = -1; return; }
    for (int k = 0; k < 3; ++k)
        if (!isfinite(x[k]) || !isfinite(u[k])) {
            *flags = fl | ORC_FLAG_NONFINITE;
            d->branch = -1;
            return;
        }
    double a = kp->a, qm = p->qm[(fl >> 6) & 3], Q = fabs(qm);
    /* switch (Sec. 3, 4.2): rho~_C = Gamma / (|q/m| B) (c = 1) against the
     * cell size of Eq. (volint), E/B = |D^| / |B^| in the local frame */
    gframe_t F0;
    gr_frame(f, a, x, &F0);
    double Gfull = lorentz(&F0.M, u);
    double Dd[3];
    for (int i = 0; i < 3; ++i) {
        Dd[i] = 0.0;
        for (int j = 0; j < 3; ++j) Dd[i] += F0.M.gdn[i][j] * F0.D[j];
    }
    double Emag = sqrt(fmax(0.0, Dd[0] * F0.D[0] + Dd[1] * F0.D[1] + Dd[2] * F0.D[2]));
    int ci, cj;
    double tr, tt;
    ks_cell(f, x[0], x[1], &ci, &cj, &tr, &tt);
    double dlc = dl ? dl[(long)cj * (f->nr - 1) + ci] : 1.0;
    int S;
    if (!F0.ok) {
        S = 1;
        d->margin = -INFINITY;
    } else {
        double rho = Gfull / (Q * F0.Bmag);
        double t1 = 1.0 - rho / (p->f_rho * dlc), t2 = 1.0 - (Emag / F0.Bmag) / p->f_E;
        d->margin = t1 < t2 ? t1 : t2;
        S = (rho / dlc < p->f_rho && Emag / F0.Bmag < p->f_E) ? 0 : 1;
    }
    if (p->force == ORC_FORCE_BORIS) S = 1;
    if (p->force == ORC_FORCE_GCA) S = 0;
    d->S = S;
    d->Gamma_full = Gfull;
    unsigned char out = (fl & 0xC0) | ((fl & ORC_FLAG_S) ? ORC_FLAG_SPREV : 0) | (S ? ORC_FLAG_S : 0);

    double xn[3] = {x[0], x[1], x[2]}, un[3] = {u[0], u[1], u[2]};
    int use_boris = S, iters = 0, nonconv = 0;
    double resid = 0.0;
    if (!S) {
        int ok = F0.ok;
        double upar = 0, mu = 0, uperp = 0, bpg[3] = {0, 0, 0};
        if (ok) {
            /* decomposition at R^n = x^n (variables are not staggered, Sec. 3.2):
             * u_i = u_par b_i + v_E,i Gamma + u_perp,g,i with Gamma of the full u */
            upar = u[0] * F0.bup[0] + u[1] * F0.bup[1] + u[2] * F0.bup[2];
            double ug[3];
            for (int i = 0; i < 3; ++i) ug[i] = u[i] - upar * F0.bdn[i] - F0.vE[i] * Gfull;
            double n2 = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) n2 += F0.M.gup[i][j] * ug[i] * ug[j];
            uperp = sqrt(fmax(n2, 0.0));
            if (uperp < 1e-300) {
                uperp = 0.0;
            } else {
                for (int i = 0; i < 3; ++i) bpg[i] = ug[i] / uperp;
                mu = uperp * uperp / (2.0 * F0.Bmag * F0.kappa);
            }
            d->upar_old = upar;
            d->mu = mu;
            d->uperp = uperp;
            ok = grgca_step(f, a, p, qm, &F0, xn, &upar, mu, uperp, bpg, &iters, &nonconv, &resid);
        }
        if (ok) {
            /* reconstruction at R^{n+1}, gyration direction kept (Sec. 3.2 step 5) */
            gframe_t F1;
            gr_frame(f, a, xn, &F1);
            ok = F1.ok;
            if (ok) {
                double G1 = gr_gamma(&F1, p, upar, mu, uperp);
                double ug = sqrt(gr_perp2(&F1, p, mu, uperp));
                for (int i = 0; i < 3; ++i) un[i] = upar * F1.bdn[i] + F1.vE[i] * G1 + ug * bpg[i];
                d->upar_new = upar;
            }
        }
        if (!ok) {
            use_boris = 1;
            d->gcafail = 1;
            for (int k = 0; k < 3; ++k) { xn[k] = x[k]; un[k] = u[k]; }
        }
    }
    if (use_boris) {
        greom_step(f, a, kp->kick_basis, p, qm, xn, un, &iters, &nonconv, &resid);
        d->branch = 1;
    } else {
        d->branch = 0;
    }
    d->iters = iters;
    d->nonconv = nonconv;
    d->resid = resid;
    /* poles: reflect theta, rotate phi by pi, flip u_theta */
    if (xn[1] < 0.0) { xn[1] = -xn[1]; xn[2] += M_PI; un[1] = -un[1]; }
    if (xn[1] > M_PI) { xn[1] = 2.0 * M_PI - xn[1]; xn[2] += M_PI; un[1] = -un[1]; }
    xn[2] = wrap_phi(xn[2]);
    int fin = 1;
    for (int k = 0; k < 3; ++k) fin = fin && isfinite(xn[k]) && isfinite(un[k]);
    if (!fin) {
        *flags = out | ORC_FLAG_NONFINITE;
        d->branch = -1;
        return;
    }
    for (int k = 0; k < 3; ++k) { x[k] = xn[k]; u[k] = un[k]; }
    if (d->gcafail) out |= ORC_FLAG_GCAFAIL;
    if (nonconv) out |= ORC_FLAG_NONCONV;
    if (x[0] < kp->r_in || x[0] > kp->r_out) out |= ORC_FLAG_EXITED;
    *flags = out;
}

int orc_push_ks(long n, double *const x[3], double *const u[3], unsigned char *flags,
                const orc_ks_field *f, const orc_ks_params *kp, const orc_params *p,
                const double *dl, int n_steps, int nthreads, orc_stats *st)
{
    orc_stats acc;
    memset(&acc, 0, sizeof(acc));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int s = 0; s < n_steps; ++s) {
        long nb = 0, ng = 0, tg = 0, tb = 0, nc = 0, gf = 0, nf = 0, ne = 0, si = 0, mi = 0;
        double ek = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) \
    reduction(+ : nb, ng, tg, tb, nc, gf, nf, ne, si, ek) reduction(max : mi)
#endif
        for (long i = 0; i < n; ++i) {
            double xi[3] = {x[0][i], x[1][i], x[2][i]}, ui[3] = {u[0][i], u[1][i], u[2][i]};
            unsigned char fl = flags[i];
            const unsigned char fl0 = fl;
            orc_detail d;
            orc_ks_step_one(f, kp, p, dl, xi, ui, &fl, &d);
            for (int k = 0; k < 3; ++k) { x[k][i] = xi[k]; u[k][i] = ui[k]; }
            flags[i] = fl;
            if (d.branch < 0) {
                /* already outside [r_in, r_out]: exited; otherwise non-finite */
                if ((fl0 & ORC_FLAG_EXITED) && !(fl0 & ORC_FLAG_NONFINITE)) ++ne; else ++nf;
                continue;
            }
            if (d.branch == 1) ++nb; else ++ng;
            int sp = (fl & ORC_FLAG_SPREV) ? 1 : 0, sn = (fl & ORC_FLAG_S) ? 1 : 0;
            if (sp && !sn) ++tg;
            if (!sp && sn) ++tb;
            if (d.nonconv) ++nc;
            if (d.gcafail) ++gf;
            si += d.iters;
            if (d.iters > mi) mi = d.iters;
            metric_t M;
            ks_metric(kp->a, xi[0], xi[1], &M);
            double u2 = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) u2 += M.gup[a][b] * ui[a] * ui[b];
            ek += u2 / (1.0 + sqrt(1.0 + u2));
        }
        acc.n_boris += nb; acc.n_gca += ng; acc.n_to_gca += tg; acc.n_to_boris += tb;
        acc.n_nonconv += nc; acc.n_gcafail += gf; acc.n_nonfinite += nf;
        acc.n_exited += ne;
        acc.sum_iter += si;
        if (mi > acc.max_iter) acc.max_iter = mi;
        acc.sum_ekin += ek;
    }
    if (st) *st = acc;
    return 0;
}

/* Local-frame components of covariant u and contravariant F at (r, theta),
 * for the tests: out[0..2] = L^T u, out[3..5] = L^{-1} F. */
void orc_ks_frame(double a, double r, double th, const double u[3], const double F[3],
                  double out[6])
{
    metric_t M;
    ks_metric(a, r, th, &M);
    double L[3][3];
    chol3(M.gup, L);
    frame_in(L, u, out);
    field_in(L, F, out + 3);
}
