// gcb_ks.cu -- the covariant coupled step in Kerr-Schild spacetime
// (Sec. 2.3 GREOM, Sec. 2.4 GRGCA, Sec. 3.2 coupling), geometrized units
// c = G = M = 1.  Arithmetic and metric in FP64; field records FP32 or FP64
// (interpolated in their own precision).  Same tile structure as the flat
// push: ballot compaction of each tile into [GCA ..., Boris ..., frozen].
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gcb.h"
#include "gcb_internal.h"

namespace gcb {
namespace ks {

constexpr int TPB = 128;
constexpr int NWARP = TPB / 32;

// Kerr-Schild 3+1 quantities and their (r, theta) derivatives, closed form:
//   rho^2 = r^2 + a^2 cos^2, z = 2r / rho^2, alpha = (1+z)^-1/2, beta^r = z/(1+z),
//   gamma^{rr} = P / ((1+z) rho^2) with P = r^2 + a^2 + z a^2 sin^2,
//   gamma^{r phi} = a / rho^2, gamma^{th th} = 1 / rho^2,
//   gamma^{ph ph} = 1 / (rho^2 sin^2), sqrt(gamma) = rho^2 sin sqrt(1+z),
//   gamma_rr = 1+z, gamma_rph = -a (1+z) sin^2, gamma_thth = rho^2, gamma_phph = P sin^2.
struct Metric {
    double alpha, beta_r, sqrtg;
    double grr, grp, gtt, gpp;          // gamma^{ij}: rr, r-phi, theta-theta, phi-phi
    double drr, drp, dtt, dpp;          // gamma_ij (lower)
    double da[2], dbr[2];               // d_i alpha, d_i beta^r (i = r, theta)
    double dgrr[2], dgrp[2], dgtt[2], dgpp[2];   // d_i gamma^{..}
};

// sin theta, cos theta and log r of a point
struct TrigLog {
    double s, c, lr;
};

__device__ __forceinline__ void trig_log(double r, double th, TrigLog &t)
{
    sincos(th, &t.s, &t.c);
    t.lr = log(r);
}

// The same at (r, th) near a point (r0, th0) whose values t0 are known
// (ir0 = 1/r0): sin and cos by the angle-addition formula with the Maclaurin
// series of sin d and cos d (d = th - th0, through d^7 and d^6), log r =
// log r0 + log(1 + e) (e = r/r0 - 1) by the Mercator series through e^9.  For
// |d| <= 0.02 and |e| <= 0.01 the truncation errors are below 1e-18; farther
// away, or within sin th0 <= 0.05 of a pole (where sin th would lose relative
// precision), the library functions.
__device__ __forceinline__ void trig_log_near(const TrigLog &t0, double r0, double ir0, double th0,
                                              double r, double th, TrigLog &t)
{
    const double d = th - th0;
    const double e = (r - r0) * ir0;
    if (!(fabs(d) <= 0.02 && fabs(e) <= 0.01 && fabs(t0.s) > 0.05)) {
        trig_log(r, th, t);
        return;
    }
    const double d2 = d * d;
    const double sd = d * (1.0 - d2 * (1.0 / 6.0) * (1.0 - d2 * (1.0 / 20.0) * (1.0 - d2 * (1.0 / 42.0))));
    const double cd = 1.0 - d2 * 0.5 * (1.0 - d2 * (1.0 / 12.0) * (1.0 - d2 * (1.0 / 30.0)));
    t.s = fma(t0.s, cd, t0.c * sd);
    t.c = fma(t0.c, cd, -t0.s * sd);
    double q = 1.0 / 9.0;
    q = fma(-e, q, 1.0 / 8.0);
    q = fma(-e, q, 1.0 / 7.0);
    q = fma(-e, q, 1.0 / 6.0);
    q = fma(-e, q, 1.0 / 5.0);
    q = fma(-e, q, 0.25);
    q = fma(-e, q, 1.0 / 3.0);
    q = fma(-e, q, 0.5);
    q = fma(-e, q, 1.0);
    t.lr = fma(e, q, t0.lr);
}

// (t: sin and cos of th)
__device__ __forceinline__ void ks_metric(double a, double r, const TrigLog &t, bool derivs, Metric &m)
{
    const double s = t.s, c = t.c;
    const double s2 = s * s, a2 = a * a;
    const double rho2 = fma(r, r, a2 * c * c);
    const double irho2 = 1.0 / rho2;
    const double z = 2.0 * r * irho2;
    const double onez = 1.0 + z;
    m.alpha = rsqrt(onez);
    const double ionez = m.alpha * m.alpha;
    m.beta_r = z * ionez;
    const double P = fma(z * a2, s2, fma(r, r, a2));
    m.grr = P * ionez * irho2;
    m.grp = a * irho2;
    m.gtt = irho2;
    const double is2 = 1.0 / s2;
    m.gpp = irho2 * is2;
    m.drr = onez;
    m.drp = -a * onez * s2;
    m.dtt = rho2;
    m.dpp = P * s2;
    m.sqrtg = rho2 * s * (onez * m.alpha);
    if (!derivs) return;
    // d rho^2, d z, d P, d sin^2 with respect to (r, theta)
    const double drho2[2] = {2.0 * r, -2.0 * a2 * s * c};
    double dz[2], dP[2];
    const double ds2[2] = {0.0, 2.0 * s * c};
    for (int i = 0; i < 2; ++i) {
        dz[i] = (i == 0 ? 2.0 * irho2 : 0.0) - 2.0 * r * drho2[i] * irho2 * irho2;
        dP[i] = (i == 0 ? 2.0 * r : 0.0) + a2 * (dz[i] * s2 + z * ds2[i]);
    }
    const double a3 = m.alpha * m.alpha * m.alpha;
    for (int i = 0; i < 2; ++i) {
        m.da[i] = -0.5 * a3 * dz[i];
        m.dbr[i] = dz[i] * ionez * ionez;
        const double d_irho2 = -drho2[i] * irho2 * irho2;
        const double d_ionez = -dz[i] * ionez * ionez;
        m.dgrr[i] = dP[i] * ionez * irho2 + P * (d_ionez * irho2 + ionez * d_irho2);
        m.dgrp[i] = a * d_irho2;
        m.dgtt[i] = d_irho2;
        m.dgpp[i] = d_irho2 * is2 - irho2 * is2 * is2 * ds2[i];
    }
}

// gamma^{ij} u_j for covariant u (indices r, theta, phi)
__device__ __forceinline__ void raise(const Metric &m, const double u[3], double v[3])
{
    v[0] = m.grr * u[0] + m.grp * u[2];
    v[1] = m.gtt * u[1];
    v[2] = m.grp * u[0] + m.gpp * u[2];
}
__device__ __forceinline__ void lower(const Metric &m, const double v[3], double u[3])
{
    u[0] = m.drr * v[0] + m.drp * v[2];
    u[1] = m.dtt * v[1];
    u[2] = m.drp * v[0] + m.dpp * v[2];
}

// Local frame of the normal observer: gamma^{ij} = L L^T with L lower
// triangular; for this metric L has L10 = L21 = 0.  Frame components of a
// covariant vector: u^ = L^T u; of a contravariant one: F^ = L^{-1} F.
// (i00, i11, i22: reciprocals of the diagonal, so no conversion divides)
struct Tri {
    double l00, l20, l11, l22, i00, i11, i22;
};
__device__ __forceinline__ void make_tri(const Metric &m, Tri &t)
{
    t.i00 = rsqrt(m.grr);
    t.l00 = m.grr * t.i00;
    t.l20 = m.grp * t.i00;
    t.i11 = rsqrt(m.gtt);
    t.l11 = m.gtt * t.i11;
    const double d22 = fma(-t.l20, t.l20, m.gpp);
    t.i22 = rsqrt(d22);
    t.l22 = d22 * t.i22;
}
__device__ __forceinline__ void cov_to_frame(const Tri &t, const double u[3], double h[3])
{
    h[0] = t.l00 * u[0] + t.l20 * u[2];
    h[1] = t.l11 * u[1];
    h[2] = t.l22 * u[2];
}
__device__ __forceinline__ void frame_to_cov(const Tri &t, const double h[3], double u[3])
{
    u[2] = h[2] * t.i22;
    u[1] = h[1] * t.i11;
    u[0] = (h[0] - t.l20 * u[2]) * t.i00;
}
__device__ __forceinline__ void con_to_frame(const Tri &t, const double F[3], double h[3])
{
    h[0] = F[0] * t.i00;
    h[1] = F[1] * t.i11;
    h[2] = (F[2] - t.l20 * h[0]) * t.i22;
}

struct StepCfg {
    double a, dt, f_rho, f_E, r_in, r_out, tol;
    int max_iter, fixed_iters, force, mu_mode, basis;
};

template <typename FT>
struct KsGrid {
    const FT *rec;
    int stride, nr, nth;
    double logr0, inv_dlogr, inv_dth;
    const double *dl;
};

// cell (clamped to the grid, so points just outside extrapolate the edge cell)
template <typename FT>
__device__ __forceinline__ void ks_cell(const KsGrid<FT> &g, double lr, double th, int &i, int &j,
                                        double &tr, double &tt)
{
    double s = (lr - g.logr0) * g.inv_dlogr;
    double q = th * g.inv_dth;
    double fi = fmin(fmax(floor(s), 0.0), (double)(g.nr - 2));
    double fj = fmin(fmax(floor(q), 0.0), (double)(g.nth - 2));
    i = (int)fi;
    j = (int)fj;
    tr = s - fi;
    tt = q - fj;
}

// linear-shape-function gather of D^i, B^i (Sec. 4 intro) in the record type
// (lr: log r)
template <typename FT>
__device__ __forceinline__ void ks_gather(const KsGrid<FT> &g, double lr, double th, double D[3],
                                          double B[3])
{
    int i, j;
    double tr, tt;
    ks_cell(g, lr, th, i, j, tr, tt);
    FT acc[6] = {FT(0), FT(0), FT(0), FT(0), FT(0), FT(0)};
    const FT ftr = (FT)tr, ftt = (FT)tt;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const int oi = o & 1, oj = o >> 1;
        const FT W = (oi ? ftr : FT(1) - ftr) * (oj ? ftt : FT(1) - ftt);
        const FT *rp = g.rec + ((size_t)(j + oj) * g.nr + (i + oi)) * g.stride;
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[k] = fma(__ldg(rp + k), W, acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) { D[k] = (double)acc[k]; B[k] = (double)acc[3 + k]; }
}

// Boris push in the local frame over proper time dtau (Sec. 2.3 step 1 / 3)
__device__ __forceinline__ void boris_local(const double E[3], const double B[3], double qm,
                                            double dtau, double u[3])
{
    const double h = 0.5 * qm * dtau;
    double um[3], t[3], x[3], up[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) um[k] = fma(h, E[k], u[k]);
    const double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    const double hg = h / gm;
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = hg * B[k];
    const double sf = 2.0 / (1.0 + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    x[0] = um[1] * t[2] - um[2] * t[1];
    x[1] = um[2] * t[0] - um[0] * t[2];
    x[2] = um[0] * t[1] - um[1] * t[0];
#pragma unroll
    for (int k = 0; k < 3; ++k) up[k] = um[k] + x[k];
    x[0] = up[1] * t[2] - up[2] * t[1];
    x[1] = up[2] * t[0] - up[0] * t[2];
    x[2] = up[0] * t[1] - up[1] * t[0];
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = fma(h, E[k], fma(sf, x[k], um[k]));
}

// The same kick in the global coordinate basis (the option of Sec. 2.3 and
// 2.4 that needs no tetrad): covariant u and D_i = gamma_ij D^j, contravariant
// B^k, t^k = h B^k / Gamma-, |t|^2 = gamma_ij t^i t^j and cross products
// (v x t)_i = sqrt(gamma) [ijk] v^j t^k of raised vectors; the frame form
// maps onto this one because det L = 1 / sqrt(gamma).
__device__ __forceinline__ void boris_global(const Metric &m, const double D[3], const double B[3],
                                             double qm, double dtau, double u[3])
{
    const double h = 0.5 * qm * dtau;
    double Dd[3], Bd[3], um[3], v[3], t[3], x[3], w[3];
    lower(m, D, Dd);
    lower(m, B, Bd);
#pragma unroll
    for (int k = 0; k < 3; ++k) um[k] = fma(h, Dd[k], u[k]);
    raise(m, um, v);
    const double gm = sqrt(1.0 + um[0] * v[0] + um[1] * v[1] + um[2] * v[2]);
    const double hg = h / gm;
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = hg * B[k];
    const double t2 = hg * hg * (Bd[0] * B[0] + Bd[1] * B[1] + Bd[2] * B[2]);
    const double sf = 2.0 / (1.0 + t2);
    const double sg = m.sqrtg;
    x[0] = sg * (v[1] * t[2] - v[2] * t[1]);
    x[1] = sg * (v[2] * t[0] - v[0] * t[2]);
    x[2] = sg * (v[0] * t[1] - v[1] * t[0]);
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = um[k] + x[k];
    raise(m, w, v);
    x[0] = sg * (v[1] * t[2] - v[2] * t[1]);
    x[1] = sg * (v[2] * t[0] - v[0] * t[2]);
    x[2] = sg * (v[0] * t[1] - v[1] * t[0]);
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = fma(h, Dd[k], fma(sf, x[k], um[k]));
}

// One GREOM half kick over alpha dt / 2 at x, in the basis c.basis selects
// (t: trigonometry and log r at x; m: the metric at x, returned for reuse)
template <typename FT>
__device__ __forceinline__ void half_kick(const KsGrid<FT> &g, const StepCfg &c, double qm,
                                          const double x[3], const TrigLog &t, double u[3], Metric &m)
{
    ks_metric(c.a, x[0], t, false, m);
    double D[3], B[3];
    ks_gather(g, t.lr, x[1], D, B);
    if (c.basis == GCB_KS_GLOBAL) {
        boris_global(m, D, B, qm, 0.5 * c.dt * m.alpha, u);
        return;
    }
    double Dh[3], Bh[3], uh[3];
    Tri tri;
    make_tri(m, tri);
    cov_to_frame(tri, u, uh);
    con_to_frame(tri, D, Dh);
    con_to_frame(tri, B, Bh);
    boris_local(Dh, Bh, qm, 0.5 * c.dt * m.alpha, uh);
    frame_to_cov(tri, uh, u);
}

// V^i = alpha gamma^{ij} u_j / Gamma - beta^i and
// G_i = -Gamma d_i alpha + u_j d_i beta^j - alpha u_j u_k d_i gamma^{jk} / (2 Gamma)
// (iGam = 1 / Gam)
__device__ __forceinline__ void geodesic_G(const Metric &m, const double u[3], double Gam,
                                           double iGam, double G[3])
{
    const double ha = 0.5 * m.alpha * iGam;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const double uu = m.dgrr[i] * u[0] * u[0] + 2.0 * m.dgrp[i] * u[0] * u[2] +
                          m.dgtt[i] * u[1] * u[1] + m.dgpp[i] * u[2] * u[2];
        G[i] = -Gam * m.da[i] + u[0] * m.dbr[i] - ha * uu;
    }
    G[2] = 0.0;   // axisymmetric: no phi dependence
}

__device__ __forceinline__ bool imr_done(const StepCfg &c, int iters, double res, bool &nonconv)
{
    if (c.fixed_iters > 0) return iters >= c.fixed_iters;
    if (res < c.tol) return true;
    if (iters >= c.max_iter) { nonconv = true; return true; }
    return false;
}

// GREOM: half kick, implicit midpoint for (x, u) (no field inside), half kick.
// (t0: trigonometry and log r at x^n; mfin: the metric at x^{n+1})
template <typename FT>
__device__ void greom_step(const KsGrid<FT> &g, const StepCfg &c, double qm, double x[3],
                           double u[3], const TrigLog &t0, int &iters, bool &nonconv, Metric &mfin)
{
    const double ir0 = 1.0 / x[0];
    double up[3] = {u[0], u[1], u[2]};
    half_kick(g, c, qm, x, t0, up, mfin);
    double xk[3] = {x[0], x[1], x[2]}, wk[3] = {up[0], up[1], up[2]};
    iters = 0;
    nonconv = false;
    for (;;) {
        double xb[3], ub[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) { xb[k] = 0.5 * (xk[k] + x[k]); ub[k] = 0.5 * (wk[k] + up[k]); }
        TrigLog tb;
        trig_log_near(t0, x[0], ir0, x[1], xb[0], xb[1], tb);
        Metric m;
        ks_metric(c.a, xb[0], tb, true, m);
        double v[3];
        raise(m, ub, v);
        const double Gam = sqrt(1.0 + ub[0] * v[0] + ub[1] * v[1] + ub[2] * v[2]);
        const double iGam = 1.0 / Gam;
        double G[3];
        geodesic_G(m, ub, Gam, iGam, G);
        const double f = m.alpha * iGam;
        const double V[3] = {f * v[0] - m.beta_r, f * v[1], f * v[2]};
        double res = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double xn = fma(c.dt, V[k], x[k]);
            const double wn = fma(c.dt, G[k], up[k]);
            res = fmax(res, fmax(fabs(xn - xk[k]), fabs(wn - wk[k])));
            xk[k] = xn;
            wk[k] = wn;
        }
        ++iters;
        if (imr_done(c, iters, res, nonconv)) break;
    }
    TrigLog t1;
    trig_log_near(t0, x[0], ir0, x[1], xk[0], xk[1], t1);
    half_kick(g, c, qm, xk, t1, wk, mfin);
#pragma unroll
    for (int k = 0; k < 3; ++k) { x[k] = xk[k]; u[k] = wk[k]; }
}

// GRGCA frame at a point (Sec. 2.4)
struct GFrame {
    Metric m;
    double D[3], Bmag, bdn[3], bup[3], vE[3], kappa, Dpar;
    bool ok;
};

// (t: trigonometry and log r at R)
template <typename FT>
__device__ __forceinline__ void gr_frame(const KsGrid<FT> &g, double a, const double R[3],
                                         const TrigLog &t, bool derivs, GFrame &F)
{
    ks_metric(a, R[0], t, derivs, F.m);
    double B[3];
    ks_gather(g, t.lr, R[1], F.D, B);
    double Bd[3];
    lower(F.m, B, Bd);
    const double B2 = Bd[0] * B[0] + Bd[1] * B[1] + Bd[2] * B[2];
    F.ok = B2 > 0.0;
    const double B2s = F.ok ? B2 : 1.0;
    const double ib = rsqrt(B2s);
    F.Bmag = B2s * ib;
#pragma unroll
    for (int i = 0; i < 3; ++i) { F.bdn[i] = Bd[i] * ib; F.bup[i] = B[i] * ib; }
    const double sg = F.m.sqrtg * (ib * ib);
    const double *D = F.D;
    F.vE[0] = sg * (D[1] * B[2] - D[2] * B[1]);
    F.vE[1] = sg * (D[2] * B[0] - D[0] * B[2]);
    F.vE[2] = sg * (D[0] * B[1] - D[1] * B[0]);
    double v[3];
    raise(F.m, F.vE, v);
    const double v2 = F.vE[0] * v[0] + F.vE[1] * v[1] + F.vE[2] * v[2];
    F.ok = F.ok && v2 < 1.0;
    F.kappa = rsqrt(F.ok ? 1.0 - v2 : 1.0);
    F.Dpar = D[0] * F.bdn[0] + D[1] * F.bdn[1] + D[2] * F.bdn[2];
}

// The frame at x^n (no metric derivatives) kept between the switch and the
// step: the values a step reads, one shared-memory row each.
constexpr int NFR = 26;

__device__ __forceinline__ void frame_store(double (*s)[TPB], int t, const GFrame &F)
{
    const double v[NFR] = {F.m.alpha, F.m.beta_r, F.m.sqrtg, F.m.grr, F.m.grp, F.m.gtt,
                           F.m.gpp, F.m.drr, F.m.drp, F.m.dtt, F.m.dpp, F.D[0], F.D[1],
                           F.D[2], F.Bmag, F.bdn[0], F.bdn[1], F.bdn[2], F.bup[0], F.bup[1],
                           F.bup[2], F.vE[0], F.vE[1], F.vE[2], F.kappa, F.Dpar};
#pragma unroll
    for (int k = 0; k < NFR; ++k) s[k][t] = v[k];
}

__device__ __forceinline__ void frame_load(const double (*s)[TPB], int t, GFrame &F)
{
    double v[NFR];
#pragma unroll
    for (int k = 0; k < NFR; ++k) v[k] = s[k][t];
    F.m.alpha = v[0]; F.m.beta_r = v[1]; F.m.sqrtg = v[2];
    F.m.grr = v[3]; F.m.grp = v[4]; F.m.gtt = v[5]; F.m.gpp = v[6];
    F.m.drr = v[7]; F.m.drp = v[8]; F.m.dtt = v[9]; F.m.dpp = v[10];
    F.D[0] = v[11]; F.D[1] = v[12]; F.D[2] = v[13];
    F.Bmag = v[14];
    F.bdn[0] = v[15]; F.bdn[1] = v[16]; F.bdn[2] = v[17];
    F.bup[0] = v[18]; F.bup[1] = v[19]; F.bup[2] = v[20];
    F.vE[0] = v[21]; F.vE[1] = v[22]; F.vE[2] = v[23];
    F.kappa = v[24];
    F.Dpar = v[25];
}

__device__ __forceinline__ double gr_perp2(const GFrame &F, const StepCfg &c, double mu, double up)
{
    return c.mu_mode ? up * up : 2.0 * mu * F.Bmag * F.kappa;
}

// GRGCA: half kick of u_par by D_par, implicit midpoint on (R, u_par) with the
// full velocity rebuilt at the midpoint, half kick (Sec. 2.4 steps 1-3).
// (sF, sl: the shared-memory rows and slot holding F0, reloaded for the
// first iterate rather than kept in registers through the iteration)
template <typename FT>
__device__ bool grgca_step(const KsGrid<FT> &g, const StepCfg &c, double qm, const GFrame &F0,
                           const double (*sF)[TPB], int sl, const TrigLog &t0, double R[3],
                           double &upar, double mu, double uperp, const double bpg[3], int &iters,
                           bool &nonconv, GFrame &F1)
{
    const double ir0 = 1.0 / R[0];
    const double u1 = fma(0.5 * c.dt * F0.m.alpha * qm, F0.Dpar, upar);
    double Rk[3] = {R[0], R[1], R[2]}, wk = u1;
    iters = 0;
    nonconv = false;
    // the frame at the current midpoint (Rk + R)/2.  The first iterate's
    // midpoint is R^n itself (Rk = R): its frame is the switch's frame F0,
    // reloaded from its shared-memory slot, with only the metric derivatives
    // added (the same values a fresh gr_frame there would give)
    GFrame Fb;
    frame_load(sF, sl, Fb);
    Fb.ok = F0.ok;
    ks_metric(c.a, R[0], t0, true, Fb.m);
    bool okall = Fb.ok;
    for (;;) {
        const double ub = 0.5 * (wk + u1);
        const double Gam = Fb.kappa * sqrt(1.0 + ub * ub + gr_perp2(Fb, c, mu, uperp));
        const double iGam = 1.0 / Gam;
        const double ug = sqrt(gr_perp2(Fb, c, mu, uperp));
        double uf[3], w[3], vv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            uf[i] = ub * Fb.bdn[i] + Fb.vE[i] * Gam + ug * bpg[i];
            w[i] = ub * iGam * Fb.bdn[i] + Fb.vE[i];
        }
        raise(Fb.m, w, vv);
        const double V[3] = {Fb.m.alpha * vv[0] - Fb.m.beta_r, Fb.m.alpha * vv[1],
                             Fb.m.alpha * vv[2]};
        double G[3];
        geodesic_G(Fb.m, uf, Gam, iGam, G);
        const double Gb = G[0] * Fb.bup[0] + G[1] * Fb.bup[1] + G[2] * Fb.bup[2];
        double res = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double rn = fma(c.dt, V[k], R[k]);
            res = fmax(res, fabs(rn - Rk[k]));
            Rk[k] = rn;
        }
        const double wn = fma(c.dt, Gb, u1);
        res = fmax(res, fabs(wn - wk));
        wk = wn;
        ++iters;
        if (imr_done(c, iters, res, nonconv)) break;
        // the next iterate's midpoint and its frame
        double Rb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) Rb[k] = 0.5 * (Rk[k] + R[k]);
        TrigLog tb;
        trig_log_near(t0, R[0], ir0, R[1], Rb[0], Rb[1], tb);
        gr_frame(g, c.a, Rb, tb, true, Fb);
        okall = okall && Fb.ok;
    }
    if (!okall) return false;
    TrigLog t1;
    trig_log_near(t0, R[0], ir0, R[1], Rk[0], Rk[1], t1);
    gr_frame(g, c.a, Rk, t1, false, F1);   // also the reconstruction's frame
    if (!F1.ok) return false;
    upar = fma(0.5 * c.dt * F1.m.alpha * qm, F1.Dpar, wk);
#pragma unroll
    for (int k = 0; k < 3; ++k) R[k] = Rk[k];
    return true;
}

struct Args {
    int64_t np;
    const double *xin[3], *uin[3];
    const uint8_t *flagsin;
    const int64_t *pidin;
    double *x[3], *u[3];
    uint8_t *flags;
    int64_t *pid;
    double qm[4];
    StepCfg c;
    unsigned long long *stats;
};

// one coupled covariant step of one particle (Sec. 3.2); returns the branch
// taken (0 GCA, 1 GREOM) and fills the flag bits
// (mfin: the metric at the new position, before any pole reflection, which
// leaves it unchanged: it depends on theta through sin^2 and cos^2 only)
template <typename FT>
__device__ int ks_particle(const KsGrid<FT> &g, const StepCfg &c, double qm, int S, const GFrame &F0,
                           const double (*sF)[TPB], int sl, const TrigLog &t0, double x[3],
                           double u[3], int &iters, bool &nonconv, bool &fail, Metric &mfin)
{
    fail = false;
    if (S == 0) {
        bool ok = F0.ok;
        double R[3] = {x[0], x[1], x[2]};
        double upar = 0.0, mu = 0.0, uperp = 0.0, bpg[3] = {0.0, 0.0, 0.0};
        GFrame F1;
        if (ok) {
            // decomposition at R^n = x^n with Gamma of the full u (Sec. 3.2)
            double v[3];
            raise(F0.m, u, v);
            const double Gfull = sqrt(1.0 + u[0] * v[0] + u[1] * v[1] + u[2] * v[2]);
            upar = u[0] * F0.bup[0] + u[1] * F0.bup[1] + u[2] * F0.bup[2];
            double ug[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) ug[i] = u[i] - upar * F0.bdn[i] - F0.vE[i] * Gfull;
            raise(F0.m, ug, v);
            uperp = sqrt(fmax(ug[0] * v[0] + ug[1] * v[1] + ug[2] * v[2], 0.0));
            if (uperp < 1e-300) {
                uperp = 0.0;
            } else {
                const double iu = 1.0 / uperp;
#pragma unroll
                for (int i = 0; i < 3; ++i) bpg[i] = ug[i] * iu;
                mu = uperp * uperp / (2.0 * F0.Bmag * F0.kappa);
            }
            ok = grgca_step(g, c, qm, F0, sF, sl, t0, R, upar, mu, uperp, bpg, iters, nonconv, F1);
        }
        if (ok) {
            // reconstruction at R^{n+1} (frame F1 from the step), gyration
            // direction kept
            ok = F1.ok;
            if (ok) {
                const double G1 = F1.kappa * sqrt(1.0 + upar * upar + gr_perp2(F1, c, mu, uperp));
                const double ugm = sqrt(gr_perp2(F1, c, mu, uperp));
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    u[i] = upar * F1.bdn[i] + F1.vE[i] * G1 + ugm * bpg[i];
                    x[i] = R[i];
                }
                mfin = F1.m;
                return 0;
            }
        }
        fail = true;
    }
    greom_step(g, c, qm, x, u, t0, iters, nonconv, mfin);
    return 1;
}

// Three resident blocks per SM (at most 170 registers a thread, a few bytes of
// spill): faster than two blocks without spills for this FP64-bound kernel.
template <typename FT>
__global__ void __launch_bounds__(TPB, 3) k_push_ks(const KsGrid<FT> g, const Args a)
{
    __shared__ double s_x[3][TPB], s_u[3][TPB];
    __shared__ double s_F[NFR][TPB];
    __shared__ double s_T[3][TPB];   // sin theta, cos theta, log r at x^n
    __shared__ uint8_t s_fl[TPB], s_S[TPB], s_ok[TPB];
    __shared__ unsigned short s_perm[TPB];
    __shared__ int s_wc[2][NWARP];
    __shared__ unsigned long long s_acc[ST_COUNT];
    __shared__ double s_ek;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < ST_COUNT) s_acc[tid] = 0ull;
    if (tid == 0) s_ek = 0.0;
    unsigned nb = 0, ng = 0, tg = 0, tb = 0, nc = 0, gf = 0, nf = 0, si = 0, mi = 0;
    unsigned ne = 0;   // frozen after leaving [r_in, r_out]
    double ek = 0.0;
    const double PI = 3.141592653589793;

    const int64_t ntiles = (a.np + TPB - 1) / TPB;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t i = tile * TPB + tid;
        const bool valid = i < a.np;
        int cls = 2;
        uint8_t fl = 0;
        double xs[3] = {0, 0, 0}, us[3] = {0, 0, 0};
        __syncthreads();  // the previous tile's slots are no longer read
        s_ok[tid] = 0;
        if (valid) {
            fl = a.flagsin[i];
            bool fin = true;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                xs[k] = a.xin[k][i];
                us[k] = a.uin[k][i];
                fin = fin && isfinite(xs[k]) && isfinite(us[k]);
            }
            const uint8_t fl_in = fl;
            if (!fin && !(fl & GCB_FLAG_NONFINITE)) { fl |= GCB_FLAG_NONFINITE; }
            if (fin && !(fl & (GCB_FLAG_NONFINITE | GCB_FLAG_EXITED))) {
                // switch (Sec. 3, 4.2): Gamma/(|q/m| B) against the cell size of
                // Eq. (volint), |D^|/|B^| against f_E; division-free form
                TrigLog t;
                trig_log(xs[0], xs[1], t);
                GFrame F;
                gr_frame(g, a.c.a, xs, t, false, F);
                frame_store(s_F, tid, F);   // the step starts from this frame
                s_T[0][tid] = t.s;
                s_T[1][tid] = t.c;
                s_T[2][tid] = t.lr;
                s_ok[tid] = F.ok ? 1 : 0;
                double v[3], Dd[3];
                raise(F.m, us, v);
                const double G = sqrt(1.0 + us[0] * v[0] + us[1] * v[1] + us[2] * v[2]);
                lower(F.m, F.D, Dd);
                const double Em = sqrt(fmax(Dd[0] * F.D[0] + Dd[1] * F.D[1] + Dd[2] * F.D[2], 0.0));
                int ci, cj;
                double tr, tt;
                ks_cell(g, t.lr, xs[1], ci, cj, tr, tt);
                const double dl = g.dl[(size_t)cj * (g.nr - 1) + ci];
                const double Q = fabs(a.qm[(fl >> GCB_SPECIES_SHIFT) & 3]);
                // B = 0 or v_E >= c: Boris
                int S = (F.ok && G < a.c.f_rho * dl * Q * F.Bmag && Em < a.c.f_E * F.Bmag) ? 0 : 1;
                if (a.c.force == GCB_FORCE_BORIS) S = 1;
                if (a.c.force == GCB_FORCE_GCA) S = 0;
                cls = S;
            } else if ((fl_in & GCB_FLAG_EXITED) && !(fl_in & GCB_FLAG_NONFINITE)) {
                ++ne;
            } else {
                ++nf;
            }
            if (cls == 2) {
#pragma unroll
                for (int k = 0; k < 3; ++k) { a.x[k][i] = xs[k]; a.u[k][i] = us[k]; }
                a.flags[i] = fl;
            }
            if (a.pidin != a.pid) a.pid[i] = a.pidin[i];
        }
        if (valid) {
#pragma unroll
            for (int k = 0; k < 3; ++k) { s_x[k][tid] = xs[k]; s_u[k][tid] = us[k]; }
        }
        s_fl[tid] = fl;
        s_S[tid] = (uint8_t)cls;
        const unsigned bgm = __ballot_sync(0xffffffffu, cls == 0);
        const unsigned bbm = __ballot_sync(0xffffffffu, cls == 1);
        if (lane == 0) { s_wc[0][warp] = __popc(bgm); s_wc[1][warp] = __popc(bbm); }
        __syncthreads();
        int offG = 0, offB = 0, totG = 0, totB = 0;
#pragma unroll
        for (int w = 0; w < NWARP; ++w) {
            const int cg = s_wc[0][w], cb = s_wc[1][w];
            if (w < warp) { offG += cg; offB += cb; }
            totG += cg;
            totB += cb;
        }
        const unsigned lt = (1u << lane) - 1u;
        if (cls == 0) s_perm[offG + __popc(bgm & lt)] = (unsigned short)tid;
        if (cls == 1) s_perm[totG + offB + __popc(bbm & lt)] = (unsigned short)tid;
        __syncthreads();
        if (tid < totG + totB) {
            const int sl = s_perm[tid];
            const uint8_t f0 = s_fl[sl];
            const int S = tid < totG ? 0 : 1;
            const double qm = a.qm[(f0 >> GCB_SPECIES_SHIFT) & 3];
            double x[3], u[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) { x[k] = s_x[k][sl]; u[k] = s_u[k][sl]; }
            GFrame F0;
            frame_load(s_F, sl, F0);
            F0.ok = s_ok[sl] != 0;
            const TrigLog t0 = {s_T[0][sl], s_T[1][sl], s_T[2][sl]};
            int it = 0;
            bool ncv = false, fail = false;
            Metric mfin;
            const int br = ks_particle(g, a.c, qm, S, F0, s_F, sl, t0, x, u, it, ncv, fail, mfin);
            // poles: reflect theta, rotate phi by pi, flip u_theta
            if (x[1] < 0.0) { x[1] = -x[1]; x[2] += PI; u[1] = -u[1]; }
            if (x[1] > PI) { x[1] = 2.0 * PI - x[1]; x[2] += PI; u[1] = -u[1]; }
            x[2] -= 2.0 * PI * floor(x[2] * (0.5 / PI));
            if (x[2] >= 2.0 * PI) x[2] -= 2.0 * PI;
            bool fin = true;
#pragma unroll
            for (int k = 0; k < 3; ++k) fin = fin && isfinite(x[k]) && isfinite(u[k]);
            const int Sprev = f0 & GCB_FLAG_S;
            uint8_t nfl = (uint8_t)((f0 & 0xC0) | (Sprev ? GCB_FLAG_SPREV : 0) | (S ? GCB_FLAG_S : 0));
            const int64_t gi = tile * TPB + sl;
            if (fin) {
                if (fail) nfl |= GCB_FLAG_GCAFAIL;
                if (ncv) nfl |= GCB_FLAG_NONCONV;
                if (x[0] < a.c.r_in || x[0] > a.c.r_out) nfl |= GCB_FLAG_EXITED;
#pragma unroll
                for (int k = 0; k < 3; ++k) { a.x[k][gi] = x[k]; a.u[k][gi] = u[k]; }
                if (br == 0) ++ng; else ++nb;
                if (Sprev && !S) ++tg;
                if (!Sprev && S) ++tb;
                if (ncv) ++nc;
                if (fail) ++gf;
                si += it;
                mi = max(mi, (unsigned)it);
                double v[3];
                raise(mfin, u, v);
                const double u2 = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
                ek += u2 / (1.0 + sqrt(1.0 + u2));
            } else {
                nfl |= GCB_FLAG_NONFINITE;
                ++nf;
#pragma unroll
                for (int k = 0; k < 3; ++k) { a.x[k][gi] = s_x[k][sl]; a.u[k][gi] = s_u[k][sl]; }
            }
            a.flags[gi] = nfl;
        }
    }
    unsigned vals[9] = {nb, ng, tg, tb, nc, gf, nf, si, mi};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        unsigned v = __reduce_add_sync(0xffffffffu, vals[k]);
        if (lane == 0 && v) atomicAdd(&s_acc[k], (unsigned long long)v);
    }
    {
        const unsigned v = __reduce_add_sync(0xffffffffu, ne);
        if (lane == 0 && v) atomicAdd(&a.stats[ST_EXITED], (unsigned long long)v);
    }
    unsigned mx = __reduce_max_sync(0xffffffffu, vals[8]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ek += __shfl_xor_sync(0xffffffffu, ek, o);
    __syncthreads();
    if (lane == 0) {
        if (mx) atomicMax(&s_acc[ST_MAX_ITER], (unsigned long long)mx);
        atomicAdd(&s_ek, ek);
    }
    __syncthreads();
    if (tid < ST_MAX_ITER) {
        if (s_acc[tid]) atomicAdd(&a.stats[tid], s_acc[tid]);
    } else if (tid == ST_MAX_ITER) {
        if (s_acc[tid]) atomicMax(&a.stats[tid], s_acc[tid]);
    } else if (tid == ST_EKIN) {
        atomicAdd(reinterpret_cast<double *>(&a.stats[ST_EKIN]), s_ek);
    }
}

// Effective cell size (Sec. 3, Eq. volint): dl = (integral of
// sqrt(gamma_rr gamma_thth - gamma_rth^2) dr dtheta over the cell)^(1/2),
// 4x4 Gauss-Legendre in (r, theta); for Kerr-Schild gamma_rth = 0.
__global__ void k_cell_size(int nr, int nth, double logr0, double dlogr, double dth, double a,
                            double *dl)
{
    const double gx[4] = {-0.8611363115940526, -0.3399810435848563, 0.3399810435848563,
                          0.8611363115940526};
    const double gw[4] = {0.3478548451374538, 0.6521451548625461, 0.6521451548625461,
                          0.3478548451374538};
    const int ncell = (nr - 1) * (nth - 1);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
        const int i = c % (nr - 1), j = c / (nr - 1);
        const double r0 = exp(logr0 + i * dlogr), r1 = exp(logr0 + (i + 1) * dlogr);
        const double t0 = j * dth, t1 = (j + 1) * dth;
        double area = 0.0;
        for (int p = 0; p < 4; ++p)
            for (int q = 0; q < 4; ++q) {
                const double r = 0.5 * (r0 + r1) + 0.5 * (r1 - r0) * gx[p];
                const double th = 0.5 * (t0 + t1) + 0.5 * (t1 - t0) * gx[q];
                const double c2 = cos(th) * cos(th);
                const double rho2 = r * r + a * a * c2;
                area += gw[p] * gw[q] * sqrt((1.0 + 2.0 * r / rho2) * rho2);
            }
        dl[c] = sqrt(area * 0.25 * (r1 - r0) * (t1 - t0));
    }
}

template <typename FT>
static gcb_status launch(const KsGrid<FT> &g, const Args &a, cudaStream_t st)
{
    static int grid_cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        set_error("cudaGetDevice failed");
        return GCB_ECUDA;
    }
    if (grid_cache[dev] == 0) {
        int nsm = 0, occ = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_push_ks<FT>, TPB, 0) != cudaSuccess) {
            set_error("occupancy query failed");
            return GCB_ECUDA;
        }
        grid_cache[dev] = nsm * (occ > 0 ? occ : 1);
    }
    const int64_t ntiles = (a.np + TPB - 1) / TPB;
    if (ntiles == 0) return GCB_OK;
    const int nb = (int)(ntiles < grid_cache[dev] ? ntiles : grid_cache[dev]);
    k_push_ks<FT><<<nb, TPB, 0, st>>>(g, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("k_push_ks launch: %s", cudaGetErrorString(e));
        return GCB_ECUDA;
    }
    return GCB_OK;
}

template <typename FT>
static gcb_status push_step(const gcb_particles *p, const gcb_particles *in, const gcb_grid_ks *gk,
                            const gcb_ks_params *kp, const gcb_params *prm, cudaStream_t st,
                            unsigned long long *stats)
{
    KsGrid<FT> g;
    g.rec = static_cast<const FT *>(gk->g.rec);
    g.stride = gk->g.stride;
    g.nr = (int)gk->g.n[0];
    g.nth = (int)gk->g.n[1];
    g.logr0 = gk->logr0;
    g.inv_dlogr = 1.0 / gk->g.dx[0];
    g.inv_dth = 1.0 / gk->g.dx[1];
    g.dl = gk->dl;
    Args a;
    a.np = p->n;
    for (int k = 0; k < 3; ++k) {
        a.xin[k] = static_cast<const double *>(in->x[k]);
        a.uin[k] = static_cast<const double *>(in->u[k]);
        a.x[k] = static_cast<double *>(p->x[k]);
        a.u[k] = static_cast<double *>(p->u[k]);
    }
    a.flagsin = in->flags;
    a.flags = p->flags;
    a.pid = p->pid;
    a.pidin = p->pid ? in->pid : nullptr;
    for (int k = 0; k < 4; ++k) a.qm[k] = prm->qm[k];
    a.c.a = kp->a;
    a.c.dt = prm->dt;
    a.c.f_rho = prm->f_rho;
    a.c.f_E = prm->f_E;
    a.c.r_in = kp->r_in;
    a.c.r_out = kp->r_out;
    a.c.tol = prm->gca_tol;
    a.c.max_iter = prm->gca_max_iter;
    a.c.fixed_iters = prm->gca_fixed_iters;
    a.c.force = prm->force;
    a.c.mu_mode = prm->mu_mode;
    a.c.basis = kp->kick_basis;
    a.stats = stats;
    return launch<FT>(g, a, st);
}

}  // namespace ks

gcb_status push_step_ks(const gcb_particles *p, const gcb_particles *in, const gcb_grid_ks *g,
                        const gcb_ks_params *kp, const gcb_params *prm, cudaStream_t st,
                        unsigned long long *stats)
{
    return g->g.dtype == GCB_F32 ? ks::push_step<float>(p, in, g, kp, prm, st, stats)
                                 : ks::push_step<double>(p, in, g, kp, prm, st, stats);
}

gcb_status ks_cell_size(const gcb_grid_ks *g, const gcb_ks_params *kp, double *dl, cudaStream_t st)
{
    const int nr = (int)g->g.n[0], nth = (int)g->g.n[1];
    const int ncell = (nr - 1) * (nth - 1);
    const int nb = (ncell + 255) / 256 < 4096 ? (ncell + 255) / 256 : 4096;
    ks::k_cell_size<<<nb, 256, 0, st>>>(nr, nth, g->logr0, g->g.dx[0], g->g.dx[1], kp->a, dl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("k_cell_size launch: %s", cudaGetErrorString(e));
        return GCB_ECUDA;
    }
    return GCB_OK;
}

}  // namespace gcb
