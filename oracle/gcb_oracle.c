/*
 * gcb_oracle.c -- plain FP64 CPU oracle of the coupled guiding-center / Boris
 * pusher of Bacchini et al. (2020), flat-space (SR) scheme.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the product path.  It shares no code
 * with the CUDA library.  Each function names the passage of the paper it
 * follows; where the paper is silent the reading taken is stated inline.
 *
 * Parity pins: every function here is exercised by tests/test_oracle_pins.py
 * against closed forms, invariants and brute force (no function is unpinned).
 */
#define _DEFAULT_SOURCE
#include "gcb_oracle.h"

#include <math.h>
#include <stdlib.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------- */
/* small vector helpers                                                    */
/* ---------------------------------------------------------------------- */
static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void cross3(const double a[3], const double b[3], double r[3])
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

/* ---------------------------------------------------------------------- */
/* L0: field access (Sec. 4 intro).  F(x) = sum_N F_N W(x - x_N) with the   */
/* linear shape function W(s) = prod_d max(0, 1 - |s_d|/dx_d), and         */
/* grad F(x) = sum_N F_N grad W(x - x_N).  The grid is periodic, so node    */
/* (i + o) of the unwrapped lattice holds the value of node (i + o) mod n.  */
/* The derivative of W is taken inside the cell floor(x/dx) that holds x    */
/* (the almost-everywhere derivative of the shape function).               */
/* ---------------------------------------------------------------------- */
static long wrap_index(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

static void grid_gather(const orc_field *f, int grad_mode, const double x[3],
                        double out[15])
{
    int nd = f->ndim;
    long base[3] = {0, 0, 0};
    double t[3] = {0, 0, 0};
    for (int d = 0; d < nd; ++d) {
        double s = x[d] / f->dx[d];
        double fl = floor(s);
        base[d] = (long)fl;
        t[d] = s - fl;
    }
    for (int c = 0; c < 15; ++c) out[c] = 0.0;
    int ncorner = 1 << nd;
    for (int o = 0; o < ncorner; ++o) {
        long idx[3] = {0, 0, 0};
        double w[3] = {1, 1, 1}, dw[3] = {0, 0, 0};
        for (int d = 0; d < nd; ++d) {
            int od = (o >> d) & 1;
            idx[d] = wrap_index(base[d] + od, f->n[d]);
            /* W along axis d for the node at distance t (left) / 1-t (right) */
            w[d] = od ? t[d] : 1.0 - t[d];
            dw[d] = (od ? 1.0 : -1.0) / f->dx[d];
        }
        long node = (idx[2] * f->n[1] + idx[1]) * f->n[0] + idx[0];
        double W = w[0] * w[1] * w[2];
        double gW[3] = {0, 0, 0};
        for (int d = 0; d < nd; ++d) {
            double g = dw[d];
            for (int e = 0; e < nd; ++e)
                if (e != d) g *= w[e];
            gW[d] = g;
        }
        for (int c = 0; c < 3; ++c) {
            out[c] += f->E[c][node] * W;
            out[3 + c] += f->B[c][node] * W;
        }
        if (grad_mode == ORC_GRAD_GRID) {
            for (int i = 0; i < nd; ++i)
                for (int j = 0; j < 3; ++j)
                    out[6 + 3 * i + j] += f->dB[3 * i + j][node] * W;
        } else {
            for (int i = 0; i < nd; ++i)
                for (int j = 0; j < 3; ++j)
                    out[6 + 3 * i + j] += f->B[j][node] * gW[i];
        }
    }
}

/* Analytic fields used by the closed-form tests.
 *   UNIFORM: par[0..2] E, par[3..5] B.
 *   HARRIS : B = (B0 tanh((y-y0)/delta), 0, Bg), E = (0, 0, Ez) with
 *            par = {B0, delta, Bg, Ez, y0}  (Harris 1962, the sheet of Sec. 4.1).
 *   BOTTLE : B = B0 (-x z/L^2, -y z/L^2, 1 + z^2/L^2), E = par[2..4] uniform,
 *            par = {B0, L, Ex, Ey, Ez}: a divergence-free magnetic mirror.
 *   ROTOR  : B = B0 (sin kx, 0, cos kx), E = (0, E0, 0), par = {B0, k, E0}:
 *            b turns along v_E, so both v_E.(b.grad)b and v_E.(v_E.grad)b
 *            are non-zero (exercises every curvature term).               */
static void analytic_field(const orc_field *f, const double x[3], double out[15])
{
    const double *q = f->par;
    for (int c = 0; c < 15; ++c) out[c] = 0.0;
    if (f->kind == ORC_FIELD_UNIFORM) {
        for (int c = 0; c < 6; ++c) out[c] = q[c];
    } else if (f->kind == ORC_FIELD_HARRIS) {
        double s = (x[1] - q[4]) / q[1];
        double th = tanh(s);
        out[2] = q[3];
        out[3] = q[0] * th;
        out[5] = q[2];
        out[6 + 3 * 1 + 0] = q[0] / q[1] * (1.0 - th * th); /* d_y B_x */
    } else if (f->kind == ORC_FIELD_BOTTLE) {
        double B0 = q[0], L2 = q[1] * q[1];
        out[0] = q[2]; out[1] = q[3]; out[2] = q[4];
        out[3] = -B0 * x[0] * x[2] / L2;
        out[4] = -B0 * x[1] * x[2] / L2;
        out[5] = B0 * (1.0 + x[2] * x[2] / L2);
        out[6 + 0 * 3 + 0] = -B0 * x[2] / L2;        /* d_x B_x */
        out[6 + 2 * 3 + 0] = -B0 * x[0] / L2;        /* d_z B_x */
        out[6 + 1 * 3 + 1] = -B0 * x[2] / L2;        /* d_y B_y */
        out[6 + 2 * 3 + 1] = -B0 * x[1] / L2;        /* d_z B_y */
        out[6 + 2 * 3 + 2] = 2.0 * B0 * x[2] / L2;   /* d_z B_z */
    } else if (f->kind == ORC_FIELD_ROTOR) {
        double B0 = q[0], k = q[1], sn = sin(k * x[0]), cs = cos(k * x[0]);
        out[1] = q[2];
        out[3] = B0 * sn;
        out[5] = B0 * cs;
        out[6 + 0 * 3 + 0] = B0 * k * cs;            /* d_x B_x */
        out[6 + 0 * 3 + 2] = -B0 * k * sn;           /* d_x B_z */
    }
}

void orc_eval_field(const orc_field *f, const orc_params *p, const double x[3],
                    double out[15])
{
    if (f->kind == ORC_FIELD_GRID)
        grid_gather(f, p->grad_mode, x, out);
    else
        analytic_field(f, x, out);
}

/* ---------------------------------------------------------------------- */
/* L1: local field kinematics in the simplified drift frame (Sec. 2.2):     */
/* b = B/B, v_E = c E x B / B^2, kappa = 1/sqrt(1 - v_E^2/c^2),             */
/* E_par = E.b, and the gradients of b that the curvature terms need.       */
/* Reading: d_i b_j = (d_i B_j - b_j b_k d_i B_k) / B (derivative of B/|B|). */
/* ---------------------------------------------------------------------- */
typedef struct {
    double E[3], B[3], dB[3][3];
    double Bmag, b[3], vE[3], kappa, Epar;
    double db[3][3];   /* d_i b_j */
    double bgb[3];     /* (b . grad) b */
    double vgb[3];     /* (v_E . grad) b */
    double gB[3];      /* grad |B|: d_i |B| = b_j d_i B_j (lab-frame b) */
    int ok;            /* B > 0 and v_E < c */
} point_t;

/* Exact drift frame (Sec. 2.2, Beklemishev & Tessarotto 1999): the frame
 * moving with v_E = (w_E / (2 w_E^2/c^2)) (1 - sqrt(1 - 4 w_E^2/c^2)),
 * w_E = c E x B / (E^2 + B^2), sees E and B parallel, with magnitudes
 * B' = sqrt((B^2 - E^2 + (B^2 + E^2) sqrt(1 - 4 w_E^2/c^2)) / 2) and
 * E' = E.B / B'; its field direction is b* = xi E_perp + eta B with
 * E_perp = E - (E.B) B/B^2, Psi = E'(B^2 - B'^2)/(B' E_perp^2),
 * eta = (B sqrt(Psi^2 E_perp^2/B^2 + 1))^{-1}, xi = eta Psi.
 * Written as given, with algebraic rewritings that avoid 0/0:
 * 1 - 4 w_E^2/c^2 = ((B^2 - E^2)^2 + 4 (E.B)^2) / (E^2 + B^2)^2 (from
 * |E x B|^2 = E^2 B^2 - (E.B)^2), and 1 - sqrt(1 - q) = q / (1 + sqrt(1 - q)),
 * so v_E = 2 w_E / (1 + s) with s = sqrt(1 - 4 w_E^2/c^2); then
 * B^2 - B'^2 = (E^2 + B^2)(1 - s)/2 = 2 |E x B|^2 / ((E^2 + B^2)(1 + s)) and
 * |E x B|^2 = B^2 E_perp^2, so E_perp^2 cancels from Psi:
 * Psi = 2 E' B^2 / (B' (E^2 + B^2)(1 + s)), regular as E turns parallel to B
 * (where b* -> b). */
int orc_bt_frame(const double E[3], const double B[3], double c, double out[9])
{
    double E2 = dot3(E, E), B2 = dot3(B, B), EB = dot3(E, B);
    if (!(B2 > 0.0)) return 0;
    double S = E2 + B2;
    double sq = sqrt((B2 - E2) * (B2 - E2) + 4.0 * EB * EB) / S;   /* sqrt(1 - 4 w^2/c^2) */
    double ExB[3];
    cross3(E, B, ExB);
    for (int k = 0; k < 3; ++k) out[k] = 2.0 * c * ExB[k] / (S * (1.0 + sq));
    double vE2 = dot3(out, out) / (c * c);
    out[6] = 1.0 / sqrt(1.0 - vE2);
    double Bp = sqrt(0.5 * (B2 - E2 + S * sq));
    double Ep = EB / Bp;
    out[7] = Ep;
    out[8] = Bp;
    double Bm = sqrt(B2);
    double Ep_[3];
    for (int k = 0; k < 3; ++k) Ep_[k] = E[k] - EB / B2 * B[k];
    double Ep2 = dot3(Ep_, Ep_);
    double Psi = 2.0 * Ep * B2 / (Bp * S * (1.0 + sq));
    double eta = 1.0 / (Bm * sqrt(Psi * Psi * Ep2 / B2 + 1.0));
    double xi = eta * Psi;
    for (int k = 0; k < 3; ++k) out[3 + k] = xi * Ep_[k] + eta * B[k];
    return 1;
}

static void eval_point(const orc_field *f, const orc_params *p, const double R[3],
                       point_t *P)
{
    double raw[15];
    double c = p->c;
    orc_eval_field(f, p, R, raw);
    for (int k = 0; k < 3; ++k) {
        P->E[k] = raw[k];
        P->B[k] = raw[3 + k];
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P->dB[i][j] = raw[6 + 3 * i + j];
    double B2 = dot3(P->B, P->B);
    P->ok = B2 > 0.0;
    P->Bmag = sqrt(B2);
    if (!P->ok) return;
    for (int k = 0; k < 3; ++k) P->b[k] = P->B[k] / P->Bmag;
    double ExB[3];
    cross3(P->E, P->B, ExB);
    for (int k = 0; k < 3; ++k) P->vE[k] = c * ExB[k] / B2;
    double beta2 = dot3(P->vE, P->vE) / (c * c);
    if (!(beta2 < 1.0)) { P->ok = 0; return; }
    P->kappa = 1.0 / sqrt(1.0 - beta2);
    /* d_i b_j of the lab-frame b (the records carry no grad E, so the
     * gradient of b* is taken as that of b in the exact frame too) */
    for (int i = 0; i < 3; ++i) {
        double bdB = P->b[0] * P->dB[i][0] + P->b[1] * P->dB[i][1] +
                     P->b[2] * P->dB[i][2];
        P->gB[i] = bdB;
        for (int j = 0; j < 3; ++j)
            P->db[i][j] = (P->dB[i][j] - P->b[j] * bdB) / P->Bmag;
    }
    if (p->frame == ORC_FRAME_BT) {
        /* Sec. 2.2: the complete b* and v_E in place of the approximated forms */
        double bt[9];
        orc_bt_frame(P->E, P->B, c, bt);
        for (int k = 0; k < 3; ++k) { P->vE[k] = bt[k]; P->b[k] = bt[3 + k]; }
        if (!(dot3(P->vE, P->vE) / (c * c) < 1.0)) { P->ok = 0; return; }
        P->kappa = bt[6];
    }
    P->Epar = dot3(P->E, P->b);
    for (int j = 0; j < 3; ++j) {
        P->bgb[j] = P->b[0] * P->db[0][j] + P->b[1] * P->db[1][j] +
                    P->b[2] * P->db[2][j];
        P->vgb[j] = P->vE[0] * P->db[0][j] + P->vE[1] * P->db[1][j] +
                    P->vE[2] * P->db[2][j];
    }
}

/* Gyro-averaged Lorentz factor, Eq. (lfacgca2):
 * Gamma(R, u_par) = kappa sqrt(1 + (u_par^2 + 2 mu B kappa / m)/c^2).
 * With mu_mode = UPERP_CONSERVE the gyration momentum u_perp,g is held
 * fixed instead of mu (the energy-conserving alternative of Sec. 2.2), so
 * u_perp,g^2 replaces 2 mu B kappa / m. */
static double perp_sq(const point_t *P, const orc_params *p, double mu, double uperp)
{
    return p->mu_mode == ORC_UPERP_CONSERVE ? uperp * uperp
                                            : 2.0 * mu * P->Bmag * P->kappa;
}

static double gamma_gca(const point_t *P, const orc_params *p, double upar,
                        double mu, double uperp)
{
    double c2 = p->c * p->c;
    return P->kappa * sqrt(1.0 + (upar * upar + perp_sq(P, p, mu, uperp)) / c2);
}

/* Curvature drift, Eq. (curvdrift):
 * v_c = (m c kappa^2 / (q B)) b x [ (u_par^2/Gamma)(b.grad)b + u_par (v_E.grad)b ]. */
static void v_curv(const point_t *P, const orc_params *p, double qm, double upar,
                   double Gam, double vc[3])
{
    if (!p->curvature) { vc[0] = vc[1] = vc[2] = 0.0; return; }
    double a[3];
    for (int k = 0; k < 3; ++k)
        a[k] = upar * upar / Gam * P->bgb[k] + upar * P->vgb[k];
    double bxa[3];
    cross3(P->b, a, bxa);
    double pref = p->c * P->kappa * P->kappa / (qm * P->Bmag);
    for (int k = 0; k < 3; ++k) vc[k] = pref * bxa[k];
}

/* ---------------------------------------------------------------------- */
/* Switch (Sec. 3 and Sec. 4.1): S = 0 (GCA) iff rho~_C / dl < f_rho and    */
/* E/B < f_E, with rho~_C = m c^2 Gamma / (|q| B), Gamma from the full u.   */
/* Strict inequalities; B = 0 gives S = 1.  The margin is                   */
/* min(1 - rho~_C/(f_rho dl), 1 - (E/B)/f_E): S = 0 iff margin > 0, and a    */
/* decision with |margin| > 1e-12 is insensitive to rounding.               */
/* ---------------------------------------------------------------------- */
int orc_switch(const double E[3], const double B[3], double Gam, double Q,
               const orc_params *p, double *margin)
{
    double Bmag = sqrt(dot3(B, B));
    double Emag = sqrt(dot3(E, E));
    if (!(Bmag > 0.0)) {
        if (margin) *margin = -INFINITY;
        return 1;
    }
    /* Reading: with c kept general, the length m c^2 Gamma / (|q| B) is the
     * gyro-radius for u_perp,g ~ Gamma c (the paper writes it with c = 1). */
    double rho = p->c * p->c * Gam / (Q * Bmag);
    double t1 = 1.0 - rho / (p->f_rho * p->dl);
    double t2 = 1.0 - (Emag / Bmag) / p->f_E;
    if (margin) *margin = t1 < t2 ? t1 : t2;
    return (rho / p->dl < p->f_rho && Emag / Bmag < p->f_E) ? 0 : 1;
}

/* ---------------------------------------------------------------------- */
/* Boris push (Sec. 2.1; the standard scheme of Boris 1970), fields at x^n: */
/* u- = u + h E;  t = h B/(c gamma-);  s = 2t/(1+t^2);  u' = u- + u- x t;    */
/* u+ = u- + u' x s;  u^{n+1/2} = u+ + h E  (h = q dt / 2m);                 */
/* x^{n+1} = x^n + dt u^{n+1/2} / gamma^{n+1/2}.                            */
/* ---------------------------------------------------------------------- */
static void boris_kick(const double E[3], const double B[3], double qm,
                       const orc_params *p, double h_dt, double u[3])
{
    double c = p->c, h = qm * h_dt;
    double um[3], t[3], s[3], up[3], tmp[3];
    for (int k = 0; k < 3; ++k) um[k] = u[k] + h * E[k];
    double gm = sqrt(1.0 + dot3(um, um) / (c * c));
    for (int k = 0; k < 3; ++k) t[k] = h * B[k] / (c * gm);
    double t2 = dot3(t, t);
    for (int k = 0; k < 3; ++k) s[k] = 2.0 * t[k] / (1.0 + t2);
    cross3(um, t, tmp);
    for (int k = 0; k < 3; ++k) up[k] = um[k] + tmp[k];
    cross3(up, s, tmp);
    for (int k = 0; k < 3; ++k) u[k] = um[k] + tmp[k] + h * E[k];
}

static void boris_step(const double E[3], const double B[3], double qm,
                       const orc_params *p, int nd, double u[3], double disp[3],
                       double v[3])
{
    boris_kick(E, B, qm, p, 0.5 * p->dt, u);
    double g = sqrt(1.0 + dot3(u, u) / (p->c * p->c));
    for (int d = 0; d < 3; ++d) disp[d] = d < nd ? p->dt * u[d] / g : 0.0;
    if (v)
        for (int d = 0; d < 3; ++d) v[d] = u[d] / g;
}

/* ---------------------------------------------------------------------- */
/* Mirror terms (option `mirror`).  Sec. 2.2 names the grad-B ("mirror")    */
/* drift and the mirror force of the guiding-center expansion and discards  */
/* them, giving no formula.  Reading: the standard relativistic forms of    */
/* the expansion the paper cites (Vandervoort 1960, Northrop 1963), in the   */
/* notation of Eq. (curvdrift): the grad-B term (mu/(m Gamma)) grad(B/kappa) */
/* joins the bracket of v_c,                                                */
/*   v_gB = (m c kappa^2/(q B)) b x [ (mu/(m Gamma)) grad(B/kappa) ],         */
/* and the mirror force -(mu/(m Gamma)) b . grad(B/kappa) joins du_par/dt.  */
/* The records carry no grad E, so grad(B/kappa) is taken as grad(B)/kappa  */
/* (grad kappa is second order in E/B); mu is mu/m as stored.  In the       */
/* discrete step the drift is evaluated like v_c (at each fixed-point       */
/* iterate, with its Gamma), and the force explicitly at (x^n,              */
/* u_par^{n-1/2}), with Gamma(R^n, u_par^{n-1/2}).  The conversions at      */
/* R^{n-1/2} and R^{n+1/2} keep the paper's drift set (v_E + v_c).          */
/* ---------------------------------------------------------------------- */
static void v_gradB(const point_t *P, const orc_params *p, double qm, double mu, double Gam,
                    double vg[3])
{
    double a[3], bxa[3];
    for (int k = 0; k < 3; ++k) a[k] = mu / Gam * P->gB[k] / P->kappa;
    cross3(P->b, a, bxa);
    double pref = p->c * P->kappa * P->kappa / (P->Bmag * qm);   /* as in v_c */
    for (int k = 0; k < 3; ++k) vg[k] = pref * bxa[k];
}

static double mirror_force(const point_t *P, const orc_params *p, double upar, double mu,
                           double uperp)
{
    double G0 = gamma_gca(P, p, upar, mu, uperp);
    return -mu / G0 * dot3(P->b, P->gB) / P->kappa;
}

/* ---------------------------------------------------------------------- */
/* Full -> GC conversion (Sec. 3.1): at R^{n-1/2},                         */
/* u = u_par b + (v_E + v_c(R, u_par)) Gamma + u_perp,g, with u_par = u.b   */
/* and Gamma taken equal to the Lorentz factor of the full u.  Then         */
/* mu/m = u_perp,g^2 / (2 B kappa) (Sec. 2.2) and b_perp,g = u_perp,g/|.|.  */
/* Reading: |u_perp,g| < 1e-300 gives b_perp,g = 0 and mu = 0.              */
/* ---------------------------------------------------------------------- */
static int decompose_at(const point_t *P, const orc_params *p, double qm,
                        const double u[3], double *upar, double *mu,
                        double *uperp, double bpg[3])
{
    if (!P->ok) return 0;
    double c = p->c;
    double Gfull = sqrt(1.0 + dot3(u, u) / (c * c));
    double up = dot3(u, P->b);
    double vc[3];
    v_curv(P, p, qm, up, Gfull, vc);
    double ug[3];
    for (int k = 0; k < 3; ++k)
        ug[k] = u[k] - up * P->b[k] - (P->vE[k] + vc[k]) * Gfull;
    double m = sqrt(dot3(ug, ug));
    *upar = up;
    *uperp = m;
    if (m < 1e-300) {
        bpg[0] = bpg[1] = bpg[2] = 0.0;
        *mu = 0.0;
        *uperp = 0.0;
    } else {
        for (int k = 0; k < 3; ++k) bpg[k] = ug[k] / m;
        *mu = m * m / (2.0 * P->Bmag * P->kappa);
    }
    return 1;
}

/* GC -> full reconstruction (Sec. 3.1), at R^{n+1/2}:                     */
/* u = u_par b + (v_E + v_c(R, u_par)) Gamma(R, u_par) + u_perp,g b_perp,g, */
/* u_perp,g = sqrt(2 mu B kappa / m) (or the held u_perp,g), the direction  */
/* b_perp,g kept from the decomposition.                                    */
/* With gyro_phase = 1 the phase is evolved instead (the extra equation     */
/* Sec. 3.1 says could be added): d phi/dt = the gyro-frequency, which in   */
/* the frame drifting with v_E is |q| B'/(m c gamma') with B' = B/kappa and  */
/* gamma' = Gamma/kappa, and in lab time (divided by kappa) |q| B/(m c kappa */
/* Gamma).  A charge gyrates about B in the sense of -q: b_perp,g turns      */
/* about b by phi = -(q/m) B dt/(c kappa Gamma), evaluated at R^{n+1/2} with */
/* Gamma(R^{n+1/2}, u_par^{n+1/2}).                                          */
static void reconstruct_at(const point_t *P, const orc_params *p, double qm,
                           double upar, double mu, double uperp,
                           const double bpg[3], double u[3])
{
    double G = gamma_gca(P, p, upar, mu, uperp);
    double vc[3];
    v_curv(P, p, qm, upar, G, vc);
    double ug = sqrt(perp_sq(P, p, mu, uperp));
    double dir[3] = {bpg[0], bpg[1], bpg[2]};
    if (p->gyro_phase) {
        double phi = -qm * P->Bmag * p->dt / (p->c * P->kappa * G);
        double bxd[3];
        cross3(P->b, bpg, bxd);
        double cs = cos(phi), sn = sin(phi);
        for (int k = 0; k < 3; ++k) dir[k] = cs * bpg[k] + sn * bxd[k];
    }
    for (int k = 0; k < 3; ++k)
        u[k] = upar * P->b[k] + (P->vE[k] + vc[k]) * G + ug * dir[k];
}

int orc_decompose(const orc_field *f, const orc_params *p, double qm,
                  const double R[3], const double u[3], double *upar,
                  double *mu, double *uperp, double bpg[3])
{
    point_t P;
    eval_point(f, p, R, &P);
    return decompose_at(&P, p, qm, u, upar, mu, uperp, bpg);
}

int orc_reconstruct(const orc_field *f, const orc_params *p, double qm,
                    const double R[3], double upar, double mu, double uperp,
                    const double bpg[3], double u[3])
{
    point_t P;
    eval_point(f, p, R, &P);
    if (!P.ok) return 0;
    reconstruct_at(&P, p, qm, upar, mu, uperp, bpg, u);
    return 1;
}

/* ---------------------------------------------------------------------- */
/* u_par update at R^n.                                                     */
/* Zero curvature (Sec. 2.2.1): u_par^{n+1/2} = u_par^{n-1/2} + q dt E_par/m.*/
/* With curvature (Sec. 2.2.2, Eqs. dupardtcase2discsol, duparprime...):    */
/*   a = v_E.(b.grad)b,  g = v_E.(v_E.grad)b,  D = 1 - dt a/2,              */
/*   u' = u_par^{n-1/2}(1 + dt a/2) + q dt E_par/m + (dt/2) Gamma(R^n,      */
/*        u_par^{n-1/2}) g,                                                 */
/*   Gamma1 = Gamma(R^n, u_par^{n+1/2}) is the root >= 1 of                 */
/*   k1 G^2 + k2 G + k3 = 0 with k1 = dt^2 g^2/4 - c^2 D^2/kappa^2,          */
/*   k2 = u' dt g, k3 = u'^2 + (c^2 + 2 mu B kappa/m) D^2,                  */
/*   u_par^{n+1/2} = (u' + (dt/2) Gamma1 g) / D.                            */
/* Reading: the root is taken in the cancellation-free form                 */
/* q = -(k2 + sgn(k2) sqrt(k2^2 - 4 k1 k3))/2, roots q/k1 and k3/q; with    */
/* k1 >= 0, a negative discriminant or no root >= 1 the GCA step fails      */
/* (GCAFAIL) and the particle takes a Boris step instead.                   */
/* ---------------------------------------------------------------------- */
static int upar_kick(const point_t *P, const orc_params *p, double qm,
                     double upar, double mu, double uperp, double *upar_new,
                     orc_detail *d)
{
    double dt = p->dt, c2 = p->c * p->c;
    /* mirror force (option), explicit at (x^n, u_par^{n-1/2}) */
    double fm = p->mirror ? dt * mirror_force(P, p, upar, mu, uperp) : 0.0;
    if (!p->curvature) {
        *upar_new = upar + qm * dt * P->Epar + fm;
        return 1;
    }
    double a = dot3(P->vE, P->bgb);
    double g = dot3(P->vE, P->vgb);
    double D = 1.0 - 0.5 * dt * a;
    double G0 = gamma_gca(P, p, upar, mu, uperp);
    double upr = upar * (1.0 + 0.5 * dt * a) + qm * dt * P->Epar + 0.5 * dt * G0 * g + fm;
    double k1 = 0.25 * dt * dt * g * g - c2 * D * D / (P->kappa * P->kappa);
    double k2 = upr * dt * g;
    double k3 = upr * upr + (c2 + perp_sq(P, p, mu, uperp)) * D * D;
    if (d) { d->k1 = k1; d->k2 = k2; d->k3 = k3; }
    double disc = k2 * k2 - 4.0 * k1 * k3;
    if (!(k1 < 0.0) || !(disc >= 0.0) || D == 0.0) return 0;
    double sq = sqrt(disc);
    double qq = -0.5 * (k2 + (k2 >= 0.0 ? sq : -sq));
    double r1 = qq / k1, r2 = (qq != 0.0) ? k3 / qq : -INFINITY;
    double G1 = r1 >= r2 ? r1 : r2;
    if (!(G1 >= 1.0)) return 0;
    if (d) d->Gamma1 = G1;
    *upar_new = (upr + 0.5 * dt * G1 * g) / D;
    return 1;
}

/* GC velocity dR/dt = u_par b / Gamma + v_E + v_c at a point (Eq. dRdt),   */
/* Gamma and v_c evaluated with the given u_par (Eq. dRdtcase2disc); with   */
/* the mirror option, + v_gB.                                               */
static void gc_velocity(const point_t *P, const orc_params *p, double qm,
                        double upar, double mu, double uperp, double V[3])
{
    double G = gamma_gca(P, p, upar, mu, uperp);
    double vc[3], vg[3] = {0.0, 0.0, 0.0};
    v_curv(P, p, qm, upar, G, vc);
    if (p->mirror) v_gradB(P, p, qm, mu, G, vg);
    for (int k = 0; k < 3; ++k) V[k] = upar * P->b[k] / G + P->vE[k] + vc[k] + vg[k];
}

/* ---------------------------------------------------------------------- */
/* One coupled step (Sec. 3.1): check S at x^n; Boris if S = 1; otherwise   */
/* convert to (R, u_par, mu), advance with the GCA leapfrog of Sec. 2.2.1/2 */
/* and convert back.                                                        */
/* ---------------------------------------------------------------------- */
static double wrap_pos(double x, double L)
{
    double w = x - L * floor(x / L);
    if (w >= L) w -= L;
    return w;
}

static int all_finite(int nd, const double x[3], const double u[3], const double dxp[3])
{
    for (int k = 0; k < 3; ++k)
        if (!isfinite(u[k])) return 0;
    for (int d = 0; d < nd; ++d)
        if (!isfinite(x[d]) || !isfinite(dxp[d])) return 0;
    return 1;
}

void orc_step_one(const orc_field *f, const orc_params *p, double x[3],
                  double u[3], double dxp[3], unsigned char *flags,
                  orc_detail *d)
{
    orc_detail dd;
    if (!d) d = &dd;
    memset(d, 0, sizeof(*d));
    int nd = f->ndim;
    unsigned char fl = *flags;
    int species = (fl >> 6) & 3;
    double qm = p->qm[species], Q = fabs(qm), c = p->c;
    double xn[3] = {0, 0, 0};
    for (int k = 0; k < nd; ++k) xn[k] = x[k];

    unsigned char keep = fl & 0xC0; /* species bits survive */
    if (!all_finite(nd, x, u, dxp)) {
        /* a non-finite particle is frozen: state and flags kept, bit set */
        d->branch = -1;
        *flags = fl | ORC_FLAG_NONFINITE;
        return;
    }

    point_t P0;  /* fields and frame at x^n = R^n */
    eval_point(f, p, xn, &P0);
    double Gfull = sqrt(1.0 + dot3(u, u) / (c * c));
    int S = orc_switch(P0.E, P0.B, Gfull, Q, p, &d->margin);
    if (p->force == ORC_FORCE_BORIS) S = 1;
    if (p->force == ORC_FORCE_GCA) S = 0;
    d->S = S;
    d->Gamma_full = Gfull;
    unsigned char outfl = keep | ((fl & ORC_FLAG_S) ? ORC_FLAG_SPREV : 0) |
                          (S ? ORC_FLAG_S : 0);

    double unew[3] = {u[0], u[1], u[2]};
    double disp[3] = {0, 0, 0};
    int use_boris = S;

    if (!S) {
        int ok = P0.ok;
        /* conversion at R^{n-1/2} = (R^n + R^{n-1})/2 = x^n - dxp/2 */
        double Rh[3] = {0, 0, 0};
        for (int k = 0; k < nd; ++k) Rh[k] = xn[k] - 0.5 * dxp[k];
        point_t Ph;
        eval_point(f, p, Rh, &Ph);
        double upar = 0, mu = 0, uperp = 0, bpg[3] = {0, 0, 0};
        ok = ok && decompose_at(&Ph, p, qm, u, &upar, &mu, &uperp, bpg);
        double upn = 0;
        if (ok) ok = upar_kick(&P0, p, qm, upar, mu, uperp, &upn, d);
        double Rk[3], Rk1[3] = {0, 0, 0}, Vn[3], Vk[3];
        int iters = 0, nonconv = 0;
        if (ok) {
            d->upar_old = upar; d->upar_new = upn; d->mu = mu; d->uperp = uperp;
            for (int k = 0; k < 3; ++k) d->bpg[k] = bpg[k];
            gc_velocity(&P0, p, qm, upn, mu, uperp, Vn);
            for (int k = 0; k < 3; ++k) Rk[k] = xn[k];
            point_t Pk = P0;
            /* fixed point on Eq. (dRdtcase2disc): R^{k+1} = R^n + dt/2 (V^n + V^k) */
            for (;;) {
                if (!Pk.ok) { ok = 0; break; }
                gc_velocity(&Pk, p, qm, upn, mu, uperp, Vk);
                for (int k = 0; k < 3; ++k)
                    Rk1[k] = k < nd ? xn[k] + 0.5 * p->dt * (Vn[k] + Vk[k]) : 0.0;
                /* the step's guiding-center velocity (all three components) */
                for (int k = 0; k < 3; ++k) d->vstep[k] = 0.5 * (Vn[k] + Vk[k]);
                ++iters;
                double res = 0.0;
                for (int k = 0; k < nd; ++k) {
                    double e = fabs(Rk1[k] - Rk[k]);
                    if (e > res) res = e;
                }
                d->resid = res;
                for (int k = 0; k < 3; ++k) Rk[k] = Rk1[k];
                if (p->fixed_iters > 0) {
                    if (iters >= p->fixed_iters) break;
                } else {
                    if (res < p->tol) break;
                    if (iters >= p->max_iter) { nonconv = 1; break; }
                }
                eval_point(f, p, Rk, &Pk);
            }
        }
        if (ok) {
            /* residual H of the final iterate (diagnostic only) */
            point_t Pf;
            eval_point(f, p, Rk, &Pf);
            if (Pf.ok) {
                double Vf[3], h = 0.0;
                gc_velocity(&Pf, p, qm, upn, mu, uperp, Vf);
                for (int k = 0; k < nd; ++k) {
                    double e = fabs(Rk[k] - xn[k] - 0.5 * p->dt * (Vn[k] + Vf[k]));
                    if (e > h) h = e;
                }
                d->H = h;
            }
            /* reconstruction at R^{n+1/2} = (R^{n+1} + R^n)/2 */
            double Rp[3] = {0, 0, 0};
            for (int k = 0; k < nd; ++k) Rp[k] = 0.5 * (Rk[k] + xn[k]);
            point_t Pp;
            eval_point(f, p, Rp, &Pp);
            ok = Pp.ok;
            if (ok) {
                reconstruct_at(&Pp, p, qm, upn, mu, uperp, bpg, unew);
                for (int k = 0; k < nd; ++k) disp[k] = Rk[k] - xn[k];
                d->iters = iters;
                d->nonconv = nonconv;
                for (int k = 0; k < 3; ++k) { d->Rn[k] = xn[k]; d->Rnp1[k] = Rk[k]; }
            }
        }
        if (!ok) {
            use_boris = 1;
            d->gcafail = 1;
            d->iters = 0;
            d->nonconv = 0;
            for (int k = 0; k < 3; ++k) unew[k] = u[k];
        }
    }
    if (use_boris) {
        boris_step(P0.E, P0.B, qm, p, nd, unew, disp, d->vstep);
        d->branch = 1;
    } else {
        d->branch = 0;
    }
    /* store: x^{n+1} = x^n + displacement (wrapped), dxp = displacement */
    double xo[3] = {0, 0, 0}, uo[3], dxo[3] = {0, 0, 0};
    for (int k = 0; k < nd; ++k) {
        double L = (double)f->n[k] * f->dx[k];
        double xnew = xn[k] + disp[k];
        xo[k] = f->kind == ORC_FIELD_GRID ? wrap_pos(xnew, L) : xnew;
        dxo[k] = disp[k];
    }
    for (int k = 0; k < 3; ++k) uo[k] = unew[k];
    if (!all_finite(nd, xo, uo, dxo)) {
        *flags = outfl | ORC_FLAG_NONFINITE;
        d->branch = -1;
        return;
    }
    for (int k = 0; k < nd; ++k) { x[k] = xo[k]; dxp[k] = dxo[k]; }
    for (int k = 0; k < 3; ++k) u[k] = uo[k];
    if (d->gcafail) outfl |= ORC_FLAG_GCAFAIL;
    if (d->nonconv) outfl |= ORC_FLAG_NONCONV;
    *flags = outfl;
}

/* ---------------------------------------------------------------------- */
/* Current deposition (PiC coupling).  The paper's point (Sec. 1, 5) is     */
/* that the coupled scheme hands a PiC code x and u at the usual staggered   */
/* times, so the code deposits the step's current as for any particle; the  */
/* paper gives no deposition of its own.  Reading: the particle is a         */
/* cloud-in-cell cloud moving along the straight path x^n -> x^{n+1} at the  */
/* step's constant velocity, and J is the exact time average of that cloud's */
/* current on the staggered (Yee) points (definition in gcb_oracle.h).  With */
/* the cloud-in-cell charge rho_i = sum Qw S(s - i)/V it satisfies the       */
/* discrete continuity equation.  The time integral is split at every cell   */
/* face the path crosses; inside a piece each factor is linear in t, the     */
/* integrand a polynomial of degree <= 2, which Simpson's rule integrates    */
/* exactly.                                                                 */
/* ---------------------------------------------------------------------- */
static double hat(double s)
{
    double a = fabs(s);
    return a < 1.0 ? 1.0 - a : 0.0;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

int orc_deposit(const orc_field *f, const double x0[3], const double disp[3], double vz,
                double Qw, double dt, double *const J[3], double *const Jabs[3])
{
    int nd = f->ndim;
    double s0[3] = {0, 0, 0}, ds[3] = {0, 0, 0};
    double V = 1.0;
    for (int a = 0; a < nd; ++a) {
        s0[a] = x0[a] / f->dx[a];
        ds[a] = disp[a] / f->dx[a];
        if (!(fabs(ds[a]) <= ORC_DEP_MAX_CELLS)) return 1;
        V *= f->dx[a];
    }
    /* times (in units of dt) at which the path crosses a face s_a = integer */
    double t[2 + 3 * (ORC_DEP_MAX_CELLS + 2)];
    int nt = 0;
    t[nt++] = 0.0;
    t[nt++] = 1.0;
    for (int a = 0; a < nd; ++a) {
        if (ds[a] == 0.0) continue;
        double lo = fmin(s0[a], s0[a] + ds[a]), hi = fmax(s0[a], s0[a] + ds[a]);
        for (double m = floor(lo) + 1.0; m < hi; m += 1.0) t[nt++] = (m - s0[a]) / ds[a];
    }
    qsort(t, (size_t)nt, sizeof(double), cmp_double);
    long nn[3] = {f->n[0], f->n[1], nd == 3 ? f->n[2] : 1};
    for (int k = 0; k + 1 < nt; ++k) {
        double ta = t[k], tb = t[k + 1];
        if (!(tb > ta)) continue;
        double tau = tb - ta;
        /* the piece lies in one cell; positions at its start, middle, end */
        long cell[3] = {0, 0, 0};
        double sq[3][3] = {{0}};
        for (int a = 0; a < nd; ++a) {
            cell[a] = (long)floor(s0[a] + ds[a] * 0.5 * (ta + tb));
            sq[0][a] = s0[a] + ds[a] * ta;
            sq[1][a] = s0[a] + ds[a] * 0.5 * (ta + tb);
            sq[2][a] = s0[a] + ds[a] * tb;
        }
        /* component a (in 2D also the out-of-plane one, a = 2): over the
         * corners o of the cell along the axes other than a, the average
         * over the piece of the product of those axes' hats */
        int ncomp = 3;
        for (int a = 0; a < ncomp; ++a) {
            int oth[2], no = 0;
            for (int b = 0; b < nd; ++b)
                if (b != a) oth[no++] = b;
            double pref = a < nd ? Qw * disp[a] * tau / (dt * V) : Qw * vz * tau / V;
            for (int o = 0; o < (1 << no); ++o) {
                long idx[3] = {cell[0], cell[1], cell[2]};
                for (int r = 0; r < no; ++r) idx[oth[r]] += (o >> r) & 1;
                double g[3];
                for (int q = 0; q < 3; ++q) {
                    g[q] = 1.0;
                    for (int r = 0; r < no; ++r)
                        g[q] *= hat(sq[q][oth[r]] - (double)idx[oth[r]]);
                }
                double avg = (g[0] + 4.0 * g[1] + g[2]) / 6.0;
                double val = pref * avg;
                long ii = wrap_index(idx[0], nn[0]), jj = wrap_index(idx[1], nn[1]),
                     kk = wrap_index(idx[2], nn[2]);
                long lin = (kk * nn[1] + jj) * nn[0] + ii;
                J[a][lin] += val;
                if (Jabs) Jabs[a][lin] += fabs(val);
            }
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Loops over steps and particles.                                          */
/* ---------------------------------------------------------------------- */
static int push_sr_impl(long n, double *const x[3], double *const u[3],
                        double *const dxp[3], unsigned char *flags, const orc_field *f,
                        const orc_params *p, int n_steps, int nthreads, orc_stats *st,
                        orc_deposit_t *dep)
{
    int nd = f->ndim;
    if (nd != 2 && nd != 3) return 1;
    orc_stats acc;
    memset(&acc, 0, sizeof(acc));
    /* per-particle path of the step, deposited after the parallel loop */
    double *path = NULL;
    if (dep) {
        dep->n_skipped = 0;
        path = (double *)malloc(sizeof(double) * 8 * (size_t)(n > 0 ? n : 1));
        if (!path) return 2;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int s = 0; s < n_steps; ++s) {
        long nb = 0, ng = 0, tg = 0, tb = 0, nc = 0, gf = 0, nf = 0, si = 0, mi = 0;
        double ek = 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) \
    reduction(+ : nb, ng, tg, tb, nc, gf, nf, si, ek) reduction(max : mi)
#endif
        for (long i = 0; i < n; ++i) {
            double xi[3] = {0, 0, 0}, ui[3], di[3] = {0, 0, 0};
            for (int k = 0; k < nd; ++k) { xi[k] = x[k][i]; di[k] = dxp[k][i]; }
            for (int k = 0; k < 3; ++k) ui[k] = u[k][i];
            unsigned char fl = flags[i];
            orc_detail d;
            double x0[3] = {xi[0], xi[1], xi[2]};
            orc_step_one(f, p, xi, ui, di, &fl, &d);
            for (int k = 0; k < nd; ++k) { x[k][i] = xi[k]; dxp[k][i] = di[k]; }
            for (int k = 0; k < 3; ++k) u[k][i] = ui[k];
            flags[i] = fl;
            if (path) {
                double *q = path + 8 * i;
                for (int k = 0; k < 3; ++k) { q[k] = x0[k]; q[3 + k] = k < nd ? di[k] : 0.0; }
                q[6] = d.vstep[2];
                q[7] = d.branch;
            }
            if (d.branch < 0) { ++nf; continue; }
            if (d.branch == 1) ++nb; else ++ng;
            int sp = (fl & ORC_FLAG_SPREV) ? 1 : 0, sn = (fl & ORC_FLAG_S) ? 1 : 0;
            if (sp && !sn) ++tg;
            if (!sp && sn) ++tb;
            if (d.nonconv) ++nc;
            if (d.gcafail) ++gf;
            si += d.iters;
            if (d.iters > mi) mi = d.iters;
            double u2 = (ui[0] * ui[0] + ui[1] * ui[1] + ui[2] * ui[2]) / (p->c * p->c);
            ek += u2 / (1.0 + sqrt(1.0 + u2));
        }
        acc.n_boris += nb; acc.n_gca += ng; acc.n_to_gca += tg; acc.n_to_boris += tb;
        acc.n_nonconv += nc; acc.n_gcafail += gf; acc.n_nonfinite += nf;
        acc.sum_iter += si;
        if (mi > acc.max_iter) acc.max_iter = mi;
        acc.sum_ekin += ek;
        if (dep) {
            for (long i = 0; i < n; ++i) {
                const double *q = path + 8 * i;
                if (q[7] < 0.0) continue;   /* frozen: no step, no current */
                double Qw = dep->q[(flags[i] >> 6) & 3] * (dep->w ? dep->w[i] : 1.0);
                if (orc_deposit(f, q, q + 3, q[6], Qw, p->dt, dep->J, dep->Jabs))
                    ++dep->n_skipped;
            }
        }
    }
    free(path);
    if (st) *st = acc;
    return 0;
}

int orc_push_sr(long n, double *const x[3], double *const u[3],
                double *const dxp[3], unsigned char *flags, const orc_field *f,
                const orc_params *p, int n_steps, int nthreads, orc_stats *st)
{
    return push_sr_impl(n, x, u, dxp, flags, f, p, n_steps, nthreads, st, NULL);
}

int orc_push_sr_dep(long n, double *const x[3], double *const u[3],
                    double *const dxp[3], unsigned char *flags,
                    const orc_field *f, const orc_params *p, int n_steps,
                    int nthreads, orc_stats *st, orc_deposit_t *dep)
{
    return push_sr_impl(n, x, u, dxp, flags, f, p, n_steps, nthreads, st, dep);
}

/* Gyro-resolved Boris reference (Sec. 4.1): the step is adapted every       */
/* iteration as dt_k = min(dt_max, 2 pi Omega_C^{-1} / 60), with            */
/* Omega_C = |q| B / (m c Gamma) at the particle.  x and u are advanced as   */
/* a leapfrog with the kick first (fields at x^k), then the drift.          */
int orc_push_resolved(long n, double *const x[3], double *const u[3],
                      unsigned char *flags, const orc_field *f,
                      const orc_params *p, double t_end, double dt_max,
                      int nthreads)
{
    int nd = f->ndim;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#else
    (void)nthreads;
#endif
    for (long i = 0; i < n; ++i) {
        double qm = p->qm[(flags[i] >> 6) & 3], c = p->c;
        double xi[3] = {0, 0, 0}, ui[3];
        for (int k = 0; k < nd; ++k) xi[k] = x[k][i];
        for (int k = 0; k < 3; ++k) ui[k] = u[k][i];
        double t = 0.0;
        orc_params q = *p;
        while (t < t_end) {
            double F[15];
            orc_eval_field(f, p, xi, F);
            double B = sqrt(F[3] * F[3] + F[4] * F[4] + F[5] * F[5]);
            double G = sqrt(1.0 + dot3(ui, ui) / (c * c));
            double dt = dt_max;
            if (B > 0.0) {
                double om = fabs(qm) * B / (c * G);
                double dg = 2.0 * M_PI / (60.0 * om);
                if (dg < dt) dt = dg;
            }
            if (t + dt > t_end) dt = t_end - t;
            q.dt = dt;
            double disp[3];
            boris_step(F, F + 3, qm, &q, nd, ui, disp, NULL);
            for (int k = 0; k < nd; ++k) xi[k] += disp[k];
            t += dt;
        }
        for (int k = 0; k < nd; ++k) x[k][i] = xi[k];
        for (int k = 0; k < 3; ++k) u[k][i] = ui[k];
    }
    return 0;
}
