/*
 * gcb_oracle_grad.cpp -- FP64 forward-mode (dual-number) derivative of the
 * flat-space coupled guiding-center / Boris push of Bacchini et al. (2020),
 * for fields that are linear in a set of mode amplitudes.
 *
 * TEST INFRASTRUCTURE ONLY: the reference that the adjoint of the CUDA
 * library is compared with.  Nothing in the product path includes, links or
 * calls it, and it shares no code with the CUDA library (it uses only the
 * oracle's own header for the parameter struct and the flag bits).
 *
 * What it computes.  The 2D push with gradient grids (grad mode GRID), the
 * field records of every node being base + sum_m a_m pattern_m (the
 * differentiation workload: every component of E, B and the gradient grids
 * is linear in the amplitudes a_m).  Every scalar of one particle's step is
 * a dual number carrying its derivatives with respect to the NM amplitudes
 * and to the particle's three initial momentum components, so one pass over
 * the steps gives d(final state)/d(a, u0) exactly (up to rounding) for the
 * discrete map as the oracle defines it: the branch S, the fixed-point
 * iteration count and the quadratic root are taken on the values (the map
 * is differentiated with them held, as the one-sided derivative at a cell
 * face is the derivative of t = x/dx - floor(x/dx) with floor held).
 *
 * The step follows gcb_oracle.c function by function, in the paper's order:
 * gather (Sec. 4 intro), the simplified drift frame (Sec. 2.2), the switch
 * (Sec. 3, Sec. 4.1), Boris (Sec. 2.1), the conversion at R^{n-1/2} and the
 * reconstruction at R^{n+1/2} (Sec. 3.1), the u_par update and the position
 * fixed point (Sec. 2.2.1 / 2.2.2, Eqs. dupardtcase2discsol,
 * duparprimedtcase2discsol, dRdtcase2disc).  Its values are therefore the
 * oracle's own (tests/test_oracle_grad_pins.py checks that, and pins the
 * derivatives against closed forms and central differences).
 */
#include <cmath>
#include <cstring>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "gcb_oracle.h"

namespace {

constexpr int NM_MAX = 64;         // mode amplitudes
constexpr int ND = NM_MAX + 3;     // + the three initial momentum components
constexpr int DU0 = NM_MAX;        // index of d/du0_x

// A value and its derivatives with respect to the ND directions.
struct Dual {
    double v;
    double d[ND];
    Dual() : v(0.0) { std::memset(d, 0, sizeof(d)); }
    Dual(double x) : v(x) { std::memset(d, 0, sizeof(d)); }   // NOLINT: constants
};

inline Dual operator+(const Dual &a, const Dual &b)
{
    Dual r(a.v + b.v);
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
inline Dual operator-(const Dual &a, const Dual &b)
{
    Dual r(a.v - b.v);
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
inline Dual operator-(const Dual &a)
{
    Dual r(-a.v);
    for (int k = 0; k < ND; ++k) r.d[k] = -a.d[k];
    return r;
}
inline Dual operator*(const Dual &a, const Dual &b)
{
    Dual r(a.v * b.v);
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
inline Dual operator/(const Dual &a, const Dual &b)
{
    const double q = a.v / b.v;
    Dual r(q);
    for (int k = 0; k < ND; ++k) r.d[k] = (a.d[k] - q * b.d[k]) / b.v;
    return r;
}
inline Dual operator+(const Dual &a, double b) { return a + Dual(b); }
inline Dual operator+(double a, const Dual &b) { return Dual(a) + b; }
inline Dual operator-(const Dual &a, double b) { return a - Dual(b); }
inline Dual operator-(double a, const Dual &b) { return Dual(a) - b; }
inline Dual operator*(const Dual &a, double b)
{
    Dual r(a.v * b);
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * b;
    return r;
}
inline Dual operator*(double a, const Dual &b) { return b * a; }
inline Dual operator/(const Dual &a, double b) { return a / Dual(b); }
inline Dual operator/(double a, const Dual &b) { return Dual(a) / b; }
inline Dual sqrt(const Dual &a)
{
    const double s = std::sqrt(a.v);
    Dual r(s);
    for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] / (2.0 * s);
    return r;
}

inline double val(const Dual &a) { return a.v; }

Dual dot3(const Dual a[3], const Dual b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

void cross3(const Dual a[3], const Dual b[3], Dual r[3])
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

struct ModeField {
    long n[2];
    double dx[2];
    const double *base;   // [node][12]: E0 E1 E2 B0 B1 B2 dxB0 dxB1 dxB2 dyB0 dyB1 dyB2
    const double *pat;    // [node][12][nm]
    int nm;
    const double *amps;   // [nm]
};

long wrap_index(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

/* Gather (Sec. 4 intro): F(x) = sum_N F_N W(x - x_N) with the node records
 * F_N = base_N + sum_m a_m pattern_{m,N}, whose derivative with respect to
 * a_m is pattern_{m,N}; the weights carry the position's derivatives. */
void gather(const ModeField &f, const Dual x[2], Dual out[12])
{
    long base[2];
    Dual t[2];
    for (int d = 0; d < 2; ++d) {
        Dual s = x[d] / f.dx[d];
        double fl = std::floor(val(s));
        base[d] = (long)fl;
        t[d] = s - fl;
    }
    for (int c = 0; c < 12; ++c) out[c] = Dual(0.0);
    for (int o = 0; o < 4; ++o) {
        long idx[2];
        Dual w[2];
        for (int d = 0; d < 2; ++d) {
            int od = (o >> d) & 1;
            idx[d] = wrap_index(base[d] + od, f.n[d]);
            w[d] = od ? t[d] : 1.0 - t[d];
        }
        long node = idx[1] * f.n[0] + idx[0];
        Dual W = w[0] * w[1];
        for (int c = 0; c < 12; ++c) {
            const double *pm = f.pat + (node * 12 + c) * f.nm;
            Dual FN(f.base[node * 12 + c]);
            for (int m = 0; m < f.nm; ++m) {
                FN.v += f.amps[m] * pm[m];
                FN.d[m] = pm[m];
            }
            out[c] = out[c] + FN * W;
        }
    }
}

/* Simplified drift frame (Sec. 2.2): b = B/B, v_E = c E x B/B^2,
 * kappa = (1 - v_E^2/c^2)^{-1/2}, E_par = E.b, and
 * d_i b_j = (d_i B_j - b_j b_k d_i B_k)/B for the curvature terms. */
struct Point {
    Dual E[3], B[3], dB[2][3];
    Dual Bmag, b[3], vE[3], kappa, Epar;
    Dual bgb[3], vgb[3];
    bool ok;
};

void eval_point(const ModeField &f, const orc_params *p, const Dual R[2], Point &P)
{
    Dual raw[12];
    gather(f, R, raw);
    const double c = p->c;
    for (int k = 0; k < 3; ++k) {
        P.E[k] = raw[k];
        P.B[k] = raw[3 + k];
    }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) P.dB[i][j] = raw[6 + 3 * i + j];
    Dual B2 = dot3(P.B, P.B);
    P.ok = val(B2) > 0.0;
    if (!P.ok) return;
    P.Bmag = sqrt(B2);
    for (int k = 0; k < 3; ++k) P.b[k] = P.B[k] / P.Bmag;
    Dual ExB[3];
    cross3(P.E, P.B, ExB);
    for (int k = 0; k < 3; ++k) P.vE[k] = c * ExB[k] / B2;
    Dual beta2 = dot3(P.vE, P.vE) / (c * c);
    if (!(val(beta2) < 1.0)) { P.ok = false; return; }
    P.kappa = 1.0 / sqrt(1.0 - beta2);
    P.Epar = dot3(P.E, P.b);
    Dual db[2][3];   // d_i b_j, i over the two grid axes (d_z = 0 in 2D)
    for (int i = 0; i < 2; ++i) {
        Dual bdB = P.b[0] * P.dB[i][0] + P.b[1] * P.dB[i][1] + P.b[2] * P.dB[i][2];
        for (int j = 0; j < 3; ++j) db[i][j] = (P.dB[i][j] - P.b[j] * bdB) / P.Bmag;
    }
    for (int j = 0; j < 3; ++j) {
        P.bgb[j] = P.b[0] * db[0][j] + P.b[1] * db[1][j];
        P.vgb[j] = P.vE[0] * db[0][j] + P.vE[1] * db[1][j];
    }
}

/* Eq. (lfacgca2): Gamma(R, u_par) = kappa sqrt(1 + (u_par^2 + 2 mu B kappa/m)/c^2). */
Dual perp_sq(const Point &P, const orc_params *p, const Dual &mu, const Dual &uperp)
{
    return p->mu_mode == ORC_UPERP_CONSERVE ? uperp * uperp : 2.0 * mu * P.Bmag * P.kappa;
}

Dual gamma_gca(const Point &P, const orc_params *p, const Dual &upar, const Dual &mu,
               const Dual &uperp)
{
    return P.kappa * sqrt(1.0 + (upar * upar + perp_sq(P, p, mu, uperp)) / (p->c * p->c));
}

/* Eq. (curvdrift): v_c = (m c kappa^2/(q B)) b x [(u_par^2/Gamma)(b.grad)b + u_par (v_E.grad)b]. */
void v_curv(const Point &P, const orc_params *p, double qm, const Dual &upar, const Dual &Gam,
            Dual vc[3])
{
    if (!p->curvature) { vc[0] = vc[1] = vc[2] = Dual(0.0); return; }
    Dual a[3];
    for (int k = 0; k < 3; ++k) a[k] = upar * upar / Gam * P.bgb[k] + upar * P.vgb[k];
    Dual bxa[3];
    cross3(P.b, a, bxa);
    Dual pref = p->c * P.kappa * P.kappa / (qm * P.Bmag);
    for (int k = 0; k < 3; ++k) vc[k] = pref * bxa[k];
}

/* Switch (Sec. 3, Sec. 4.1), on values: S = 0 iff m c^2 Gamma/(|q| B dl) < f_rho
 * and E/B < f_E (strict), B = 0 gives S = 1. */
int switch_S(const Point &P, double Gam, double Q, const orc_params *p)
{
    double Bm = std::sqrt(val(P.B[0]) * val(P.B[0]) + val(P.B[1]) * val(P.B[1]) +
                          val(P.B[2]) * val(P.B[2]));
    double Em = std::sqrt(val(P.E[0]) * val(P.E[0]) + val(P.E[1]) * val(P.E[1]) +
                          val(P.E[2]) * val(P.E[2]));
    if (!(Bm > 0.0)) return 1;
    double rho = p->c * p->c * Gam / (Q * Bm);
    return (rho / p->dl < p->f_rho && Em / Bm < p->f_E) ? 0 : 1;
}

/* Boris (Sec. 2.1, Boris 1970): u- = u + hE, t = hB/(c gamma-), s = 2t/(1+t^2),
 * u' = u- + u- x t, u+ = u- + u' x s, u = u+ + hE (h = q dt/2m); disp = dt u/gamma. */
void boris_step(const Dual E[3], const Dual B[3], double qm, const orc_params *p, Dual u[3],
                Dual disp[2])
{
    const double c = p->c, h = qm * 0.5 * p->dt;
    Dual um[3], t[3], s[3], up[3], tmp[3];
    for (int k = 0; k < 3; ++k) um[k] = u[k] + h * E[k];
    Dual gm = sqrt(1.0 + dot3(um, um) / (c * c));
    for (int k = 0; k < 3; ++k) t[k] = h * B[k] / (c * gm);
    Dual t2 = dot3(t, t);
    for (int k = 0; k < 3; ++k) s[k] = 2.0 * t[k] / (1.0 + t2);
    cross3(um, t, tmp);
    for (int k = 0; k < 3; ++k) up[k] = um[k] + tmp[k];
    cross3(up, s, tmp);
    for (int k = 0; k < 3; ++k) u[k] = um[k] + tmp[k] + h * E[k];
    Dual g = sqrt(1.0 + dot3(u, u) / (c * c));
    for (int d = 0; d < 2; ++d) disp[d] = p->dt * u[d] / g;
}

/* Full -> GC conversion at R^{n-1/2} (Sec. 3.1). */
bool decompose_at(const Point &P, const orc_params *p, double qm, const Dual u[3], Dual &upar,
                  Dual &mu, Dual &uperp, Dual bpg[3])
{
    if (!P.ok) return false;
    const double c = p->c;
    Dual Gfull = sqrt(1.0 + dot3(u, u) / (c * c));
    Dual up = dot3(u, P.b);
    Dual vc[3];
    v_curv(P, p, qm, up, Gfull, vc);
    Dual ug[3];
    for (int k = 0; k < 3; ++k) ug[k] = u[k] - up * P.b[k] - (P.vE[k] + vc[k]) * Gfull;
    Dual m = sqrt(dot3(ug, ug));
    upar = up;
    uperp = m;
    if (val(m) < 1e-300) {
        bpg[0] = bpg[1] = bpg[2] = Dual(0.0);
        mu = Dual(0.0);
        uperp = Dual(0.0);
    } else {
        for (int k = 0; k < 3; ++k) bpg[k] = ug[k] / m;
        mu = m * m / (2.0 * P.Bmag * P.kappa);
    }
    return true;
}

/* GC -> full reconstruction at R^{n+1/2} (Sec. 3.1). */
void reconstruct_at(const Point &P, const orc_params *p, double qm, const Dual &upar,
                    const Dual &mu, const Dual &uperp, const Dual bpg[3], Dual u[3])
{
    Dual G = gamma_gca(P, p, upar, mu, uperp);
    Dual vc[3];
    v_curv(P, p, qm, upar, G, vc);
    Dual ug = sqrt(perp_sq(P, p, mu, uperp));
    for (int k = 0; k < 3; ++k) u[k] = upar * P.b[k] + (P.vE[k] + vc[k]) * G + ug * bpg[k];
}

/* u_par update at R^n (Sec. 2.2.1; Sec. 2.2.2 with the quadratic in Gamma). */
bool upar_kick(const Point &P, const orc_params *p, double qm, const Dual &upar, const Dual &mu,
               const Dual &uperp, Dual &upar_new)
{
    const double dt = p->dt, c2 = p->c * p->c;
    if (!p->curvature) {
        upar_new = upar + qm * dt * P.Epar;
        return true;
    }
    Dual a = dot3(P.vE, P.bgb);
    Dual g = dot3(P.vE, P.vgb);
    Dual D = 1.0 - 0.5 * dt * a;
    Dual G0 = gamma_gca(P, p, upar, mu, uperp);
    Dual upr = upar * (1.0 + 0.5 * dt * a) + qm * dt * P.Epar + 0.5 * dt * G0 * g;
    Dual k1 = 0.25 * dt * dt * g * g - c2 * D * D / (P.kappa * P.kappa);
    Dual k2 = upr * dt * g;
    Dual k3 = upr * upr + (c2 + perp_sq(P, p, mu, uperp)) * D * D;
    Dual disc = k2 * k2 - 4.0 * k1 * k3;
    if (!(val(k1) < 0.0) || !(val(disc) >= 0.0) || val(D) == 0.0) return false;
    Dual sq = sqrt(disc);
    Dual qq = -0.5 * (k2 + (val(k2) >= 0.0 ? sq : -sq));
    Dual r1 = qq / k1;
    Dual G1;
    if (val(qq) != 0.0) {
        Dual r2 = k3 / qq;
        G1 = val(r1) >= val(r2) ? r1 : r2;
    } else {
        G1 = r1;
    }
    if (!(val(G1) >= 1.0)) return false;
    upar_new = (upr + 0.5 * dt * G1 * g) / D;
    return true;
}

/* dR/dt = u_par b/Gamma + v_E + v_c (Eq. dRdt). */
void gc_velocity(const Point &P, const orc_params *p, double qm, const Dual &upar, const Dual &mu,
                 const Dual &uperp, Dual V[3])
{
    Dual G = gamma_gca(P, p, upar, mu, uperp);
    Dual vc[3];
    v_curv(P, p, qm, upar, G, vc);
    for (int k = 0; k < 3; ++k) V[k] = upar * P.b[k] / G + P.vE[k] + vc[k];
}

Dual wrap_pos(const Dual &x, double L)
{
    Dual w = x - L * std::floor(val(x) / L);
    if (val(w) >= L) w = w - L;
    return w;
}

bool finite(const Dual &a) { return std::isfinite(a.v); }

/* One coupled step of one particle (Sec. 3.1), as orc_step_one. */
void step_one(const ModeField &f, const orc_params *p, Dual x[2], Dual u[3], Dual dxp[2],
              unsigned char *flags)
{
    unsigned char fl = *flags;
    const double qm = p->qm[(fl >> 6) & 3], Q = std::fabs(qm), c = p->c;
    const unsigned char keep = fl & 0xC0;
    bool fin = true;
    for (int k = 0; k < 3; ++k) fin = fin && finite(u[k]);
    for (int d = 0; d < 2; ++d) fin = fin && finite(x[d]) && finite(dxp[d]);
    if (!fin) { *flags = fl | ORC_FLAG_NONFINITE; return; }

    Point P0;
    eval_point(f, p, x, P0);
    Dual Gfull = sqrt(1.0 + dot3(u, u) / (c * c));
    int S = switch_S(P0, val(Gfull), Q, p);
    if (p->force == ORC_FORCE_BORIS) S = 1;
    if (p->force == ORC_FORCE_GCA) S = 0;
    unsigned char outfl = keep | ((fl & ORC_FLAG_S) ? ORC_FLAG_SPREV : 0) | (S ? ORC_FLAG_S : 0);

    Dual unew[3] = {u[0], u[1], u[2]};
    Dual disp[2];
    bool use_boris = S != 0, gcafail = false, nonconv = false;
    if (!S) {
        bool ok = P0.ok;
        Dual Rh[2];
        for (int k = 0; k < 2; ++k) Rh[k] = x[k] - 0.5 * dxp[k];
        Point Ph;
        eval_point(f, p, Rh, Ph);
        Dual upar, mu, uperp, bpg[3], upn;
        ok = ok && decompose_at(Ph, p, qm, u, upar, mu, uperp, bpg);
        if (ok) ok = upar_kick(P0, p, qm, upar, mu, uperp, upn);
        Dual Rk[2] = {x[0], x[1]}, Rk1[2], Vn[3], Vk[3];
        int iters = 0;
        if (ok) {
            gc_velocity(P0, p, qm, upn, mu, uperp, Vn);
            Point Pk = P0;
            for (;;) {
                if (!Pk.ok) { ok = false; break; }
                gc_velocity(Pk, p, qm, upn, mu, uperp, Vk);
                for (int k = 0; k < 2; ++k) Rk1[k] = x[k] + 0.5 * p->dt * (Vn[k] + Vk[k]);
                ++iters;
                double res = 0.0;
                for (int k = 0; k < 2; ++k) {
                    double e = std::fabs(val(Rk1[k]) - val(Rk[k]));
                    if (e > res) res = e;
                }
                for (int k = 0; k < 2; ++k) Rk[k] = Rk1[k];
                if (p->fixed_iters > 0) {
                    if (iters >= p->fixed_iters) break;
                } else {
                    if (res < p->tol) break;
                    if (iters >= p->max_iter) { nonconv = true; break; }
                }
                eval_point(f, p, Rk, Pk);
            }
        }
        if (ok) {
            Dual Rp[2];
            for (int k = 0; k < 2; ++k) Rp[k] = 0.5 * (Rk[k] + x[k]);
            Point Pp;
            eval_point(f, p, Rp, Pp);
            ok = Pp.ok;
            if (ok) {
                reconstruct_at(Pp, p, qm, upn, mu, uperp, bpg, unew);
                for (int k = 0; k < 2; ++k) disp[k] = Rk[k] - x[k];
            }
        }
        if (!ok) {
            use_boris = true;
            gcafail = true;
            nonconv = false;
            for (int k = 0; k < 3; ++k) unew[k] = u[k];
        }
    }
    if (use_boris) boris_step(P0.E, P0.B, qm, p, unew, disp);

    Dual xo[2], dxo[2];
    for (int k = 0; k < 2; ++k) {
        xo[k] = wrap_pos(x[k] + disp[k], (double)f.n[k] * f.dx[k]);
        dxo[k] = disp[k];
    }
    fin = true;
    for (int k = 0; k < 3; ++k) fin = fin && finite(unew[k]);
    for (int d = 0; d < 2; ++d) fin = fin && finite(xo[d]) && finite(dxo[d]);
    if (!fin) { *flags = outfl | ORC_FLAG_NONFINITE; return; }
    for (int k = 0; k < 2; ++k) { x[k] = xo[k]; dxp[k] = dxo[k]; }
    for (int k = 0; k < 3; ++k) u[k] = unew[k];
    if (gcafail) outfl |= ORC_FLAG_GCAFAIL;
    if (nonconv) outfl |= ORC_FLAG_NONCONV;
    *flags = outfl;
}

}  // namespace

extern "C" {

/*
 * n_steps coupled steps of n particles (2D, grad mode GRID) in the field
 * base + sum_m amps[m] pat[m], carrying derivatives with respect to the nm
 * amplitudes (nm <= 64) and each particle's initial u.
 *   base: [node][12], pat: [node][12][nm], node = j nx + i.
 *   x (2, n), u (3, n), dxp (2, n), flags (n): initial state, overwritten
 *   with the final one (values, as the oracle's push).
 *   jac: (n, 7, nm + 3), row-major: d(final x0, x1, u0, u1, u2, dxp0, dxp1)
 *   / d(a_0 .. a_{nm-1}, u0_x, u0_y, u0_z) of each particle.
 * Returns 0, or 1 for invalid arguments (the exact drift frame and the
 * evolved gyration phase are not differentiated here).
 */
int orcg_push_jac(long n, double *x, double *u, double *dxp, unsigned char *flags,
                  long nx, long ny, double dx, double dy, const double *base, const double *pat,
                  int nm, const double *amps, const orc_params *p, int n_steps, int nthreads,
                  double *jac)
{
    if (nm < 0 || nm > NM_MAX || n < 0 || nx < 1 || ny < 1 || p->frame != ORC_FRAME_SIMPLE ||
        p->gyro_phase != 0 || p->mirror != 0)
        return 1;
    ModeField f{{nx, ny}, {dx, dy}, base, pat, nm, amps};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#else
    (void)nthreads;
#endif
    for (long i = 0; i < n; ++i) {
        Dual xi[2], ui[3], di[2];
        for (int k = 0; k < 2; ++k) { xi[k] = Dual(x[k * n + i]); di[k] = Dual(dxp[k * n + i]); }
        for (int k = 0; k < 3; ++k) {
            ui[k] = Dual(u[k * n + i]);
            ui[k].d[DU0 + k] = 1.0;
        }
        unsigned char fl = flags[i];
        for (int s = 0; s < n_steps; ++s) step_one(f, p, xi, ui, di, &fl);
        const Dual *outs[7] = {&xi[0], &xi[1], &ui[0], &ui[1], &ui[2], &di[0], &di[1]};
        for (int r = 0; r < 7; ++r) {
            double *row = jac + ((size_t)i * 7 + r) * (size_t)(nm + 3);
            for (int m = 0; m < nm; ++m) row[m] = outs[r]->d[m];
            for (int k = 0; k < 3; ++k) row[nm + k] = outs[r]->d[DU0 + k];
        }
        for (int k = 0; k < 2; ++k) { x[k * n + i] = xi[k].v; dxp[k * n + i] = di[k].v; }
        for (int k = 0; k < 3; ++k) u[k * n + i] = ui[k].v;
        flags[i] = fl;
    }
    return 0;
}

}  // extern "C"
