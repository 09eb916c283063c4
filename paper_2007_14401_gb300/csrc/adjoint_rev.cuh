// adjoint_rev.cuh -- transposed derivative (reverse mode) of one flat-space
// particle-step, 2D with gradient records.  Every function *_bwd takes the
// forward inputs and the adjoint of the outputs and ADDS the adjoint of the
// inputs into its accumulators, recomputing the forward intermediates it
// needs.  The step's structure (Sec. 3.1 with Sec. 2.2.2 and Sec. 2.1):
//   F0 = field at x^n;  conversion at R^{n-1/2} = x^n - dxp/2 -> (u_par, mu,
//   u_perp, gyrophase direction);  u_par update at x^n (quadratic in Gamma);
//   K fixed-point iterates d^k = dt/2 (V^n + V^{k-1}) with V^{k-1} the
//   guiding-center velocity at x^n + d^{k-1};  reconstruction of u at
//   R^{n+1/2} = x^n + d^K/2;  outputs x^{n+1} = x^n + d^K, dxp = d^K, u.
#pragma once

#include "gcb_device.cuh"

namespace gcb {
namespace rev {

template <typename T>
struct FrameAdj {
    T Bmag, b[3], vE[3], kappa, Epar, bgb[3], vgb[3];
    __device__ __forceinline__ void zero()
    {
        Bmag = kappa = Epar = T(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) b[k] = vE[k] = bgb[k] = vgb[k] = T(0);
    }
};

// Adjoint of make_frame (with gradients): aF = (d frame / dF)^T af.
template <typename T, int ND>
__device__ __forceinline__ void frame_bwd(const FieldPt<T, ND> &F, T c, T inv_c2,
                                          const FrameAdj<T> &af, FieldPt<T, ND> &aF)
{
    const T B2 = dot3(F.B, F.B);
    const T Bmag = sqrt(B2);
    const T ib = T(1) / Bmag;
    const T ib2 = ib * ib;
    T b[3], x[3], vE[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) b[k] = F.B[k] * ib;
    cross3(F.E, F.B, x);
#pragma unroll
    for (int k = 0; k < 3; ++k) vE[k] = c * x[k] * ib2;
    const T beta2 = dot3(vE, vE) * inv_c2;
    const T om = one_minus_beta2<T>(F.E, F.B, B2, c, beta2);
    const T kappa = T(1) / sqrt(om);
    T w[3], y[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T sw = T(0), sy = T(0);
#pragma unroll
        for (int i = 0; i < ND; ++i) {
            sw = fma(b[i], F.dB[i][j], sw);
            sy = fma(vE[i], F.dB[i][j], sy);
        }
        w[j] = sw;
        y[j] = sy;
    }
    const T bw = dot3(b, w), by = dot3(b, y);

    T ab[3], avE[3], aw[3], ay[3];
    T aib = T(0), abw = T(0), aby = T(0);
    // bgb_j = (w_j - b_j bw) ib,  vgb_j = (y_j - b_j by) ib
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        aw[j] = af.bgb[j] * ib;
        ay[j] = af.vgb[j] * ib;
        ab[j] = af.b[j] - (af.bgb[j] * bw + af.vgb[j] * by) * ib;
        abw -= af.bgb[j] * b[j];
        aby -= af.vgb[j] * b[j];
        aib += af.bgb[j] * (w[j] - b[j] * bw) + af.vgb[j] * (y[j] - b[j] * by);
        avE[j] = af.vE[j];
    }
    abw *= ib;
    aby *= ib;
    // bw = b.w, by = b.y
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        ab[j] += abw * w[j] + aby * y[j];
        aw[j] += abw * b[j];
        ay[j] += aby * b[j];
    }
    // w_j = sum_i b_i dB_ij,  y_j = sum_i vE_i dB_ij
#pragma unroll
    for (int i = 0; i < ND; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            ab[i] += aw[j] * F.dB[i][j];
            avE[i] += ay[j] * F.dB[i][j];
            aF.dB[i][j] = aw[j] * b[i] + ay[j] * vE[i];
        }
    // Epar = E.b
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        aF.E[k] = af.Epar * b[k];
        ab[k] += af.Epar * F.E[k];
    }
    // kappa = (1 - beta2)^(-1/2):  d kappa / d beta2 = kappa^3 / 2
    const T abeta2 = T(0.5) * af.kappa * kappa * kappa * kappa;
#pragma unroll
    for (int k = 0; k < 3; ++k) avE[k] += T(2) * abeta2 * inv_c2 * vE[k];
    // vE = c x ib2,  x = E x B
    T ax[3], aib2 = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ax[k] = c * ib2 * avE[k];
        aib2 += c * avE[k] * x[k];
    }
    T t[3];
    cross3(F.B, ax, t);
#pragma unroll
    for (int k = 0; k < 3; ++k) aF.E[k] += t[k];
    cross3(ax, F.E, t);
    // b = B ib,  ib2 = ib^2,  ib = 1/|B|,  |B| = sqrt(B.B)
#pragma unroll
    for (int k = 0; k < 3; ++k) aib += ab[k] * F.B[k];
    aib += T(2) * ib * aib2;
    const T aBmag = af.Bmag - aib * ib2;
#pragma unroll
    for (int k = 0; k < 3; ++k) aF.B[k] = t[k] + ab[k] * ib + aBmag * b[k];
}

template <typename T>
__device__ __forceinline__ void perp2_bwd(const Frame<T> &f, const StepPar<T> &s, T mu, T uperp,
                                          T aP, FrameAdj<T> &af, T &amu, T &auperp)
{
    if (s.mu_mode) {
        auperp += T(2) * uperp * aP;
    } else {
        amu += T(2) * f.Bmag * f.kappa * aP;
        af.Bmag += T(2) * mu * f.kappa * aP;
        af.kappa += T(2) * mu * f.Bmag * aP;
    }
}

// Gamma = kappa sqrt(1 + (u_par^2 + P)/c^2)
template <typename T>
__device__ __forceinline__ void gamma_gc_bwd(const Frame<T> &f, const StepPar<T> &s, T upar,
                                             T mu, T uperp, T aG, FrameAdj<T> &af, T &aupar,
                                             T &amu, T &auperp)
{
    const T P = perp2(f, s, mu, uperp);
    const T S = sqrt(T(1) + fma(upar, upar, P) * s.inv_c2);
    af.kappa += aG * S;
    const T ain = aG * f.kappa * s.inv_c2 / (T(2) * S);
    aupar += T(2) * upar * ain;
    perp2_bwd(f, s, mu, uperp, ain, af, amu, auperp);
}

// v_c = pref b x (k2 bgb + u_par vgb),  k2 = u_par^2/G,  pref = c kappa^2/(q/m |B|)
template <typename T>
__device__ __forceinline__ void vcurv_bwd(const Frame<T> &f, const StepPar<T> &s, T upar, T G,
                                          const T avc[3], FrameAdj<T> &af, T &aupar, T &aG)
{
    if (!s.curvature) return;
    const T k2 = upar * upar / G;
    T a[3], x[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) a[k] = fma(k2, f.bgb[k], upar * f.vgb[k]);
    cross3(f.b, a, x);
    const T pref = s.c * f.kappa * f.kappa / (s.qm * f.Bmag);
    const T apref = dot3(avc, x);
    T ax[3], t[3], aa[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) ax[k] = pref * avc[k];
    cross3(a, ax, t);
    cross3(ax, f.b, aa);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        af.b[k] += t[k];
        af.bgb[k] += k2 * aa[k];
        af.vgb[k] += upar * aa[k];
    }
    const T ak2 = dot3(aa, f.bgb);
    aupar += dot3(aa, f.vgb) + T(2) * upar / G * ak2;
    aG -= k2 / G * ak2;
    af.kappa += T(2) * pref / f.kappa * apref;
    af.Bmag -= pref / f.Bmag * apref;
}

// V = (u_par/G) b + vE + v_c,  G = Gamma(u_par, mu)
template <typename T>
__device__ __forceinline__ void gc_vel_bwd(const Frame<T> &f, const StepPar<T> &s, T upar, T mu,
                                           T uperp, const T aV[3], FrameAdj<T> &af, T &aupar,
                                           T &amu, T &auperp)
{
    const T G = gamma_gc(f, s, upar, mu, uperp);
    const T ig = upar / G;
    const T aig = dot3(aV, f.b);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        af.b[k] += ig * aV[k];
        af.vE[k] += aV[k];
    }
    T aG = T(0);
    vcurv_bwd(f, s, upar, G, aV, af, aupar, aG);
    aupar += aig / G;
    aG -= ig / G * aig;
    gamma_gc_bwd(f, s, upar, mu, uperp, aG, af, aupar, amu, auperp);
}

// u_par update at x^n (Sec. 2.2.1 without curvature; Sec. 2.2.2 with it: the
// Lorentz factor G1 is the larger root of k1 G^2 + k2 G + k3 = 0, whose
// derivative follows from the quadratic itself: dG1 = -(G1^2 dk1 + G1 dk2 +
// dk3) / (2 k1 G1 + k2)).
template <typename T>
__device__ __forceinline__ void upar_bwd(const Frame<T> &f0, const StepPar<T> &s, T upar, T mu,
                                         T uperp, T aupn, FrameAdj<T> &af, T &aupar, T &amu,
                                         T &auperp)
{
    if (!s.curvature) {
        aupar += aupn;
        af.Epar += s.qm * s.dt * aupn;
        return;
    }
    const T A = dot3(f0.vE, f0.bgb);
    const T gg = dot3(f0.vE, f0.vgb);
    const T D = fma(-s.half_dt, A, T(1));
    const T G0 = gamma_gc(f0, s, upar, mu, uperp);
    const T upr = fma(upar, fma(s.half_dt, A, T(1)), fma(s.qm * s.dt, f0.Epar, s.half_dt * G0 * gg));
    const T c2 = s.c * s.c;
    const T kap2 = f0.kappa * f0.kappa;
    const T P0 = perp2(f0, s, mu, uperp);
    const T k1 = T(0.25) * s.dt * s.dt * gg * gg - c2 * D * D / kap2;
    const T k2 = upr * s.dt * gg;
    const T k3 = fma(upr, upr, (c2 + P0) * D * D);
    const T disc = fma(k2, k2, T(-4) * k1 * k3);
    const T sq = sqrt(disc);
    const T q = T(-0.5) * (k2 + (k2 >= T(0) ? sq : -sq));
    const T r1 = q / k1;
    const T r2 = (q != T(0)) ? k3 / q : T(-1);
    const T G1 = r1 >= r2 ? r1 : r2;
    const T upn = fma(s.half_dt * G1, gg, upr) / D;

    const T iD = T(1) / D;
    const T aG1 = aupn * s.half_dt * gg * iD;
    T agg = aupn * s.half_dt * G1 * iD;
    T aupr = aupn * iD;
    T aD = -aupn * upn * iD;
    const T den = fma(T(2) * k1, G1, k2);
    const T ak1 = -aG1 * G1 * G1 / den;
    const T ak2 = -aG1 * G1 / den;
    const T ak3 = -aG1 / den;
    // k3 = upr^2 + (c^2 + P0) D^2
    aupr += T(2) * upr * ak3;
    const T aP0 = D * D * ak3;
    aD += T(2) * (c2 + P0) * D * ak3;
    // k2 = upr dt gg
    aupr += s.dt * gg * ak2;
    agg += upr * s.dt * ak2;
    // k1 = dt^2 gg^2 / 4 - c^2 D^2 / kappa^2
    agg += T(0.5) * s.dt * s.dt * gg * ak1;
    aD -= T(2) * c2 * D / kap2 * ak1;
    af.kappa += T(2) * c2 * D * D / (kap2 * f0.kappa) * ak1;
    // upr = u_par (1 + dt/2 A) + (q/m) dt Epar + dt/2 G0 gg
    aupar += fma(s.half_dt, A, T(1)) * aupr;
    T aA = upar * s.half_dt * aupr;
    af.Epar += s.qm * s.dt * aupr;
    const T aG0 = s.half_dt * gg * aupr;
    agg += s.half_dt * G0 * aupr;
    // D = 1 - dt/2 A
    aA -= s.half_dt * aD;
    gamma_gc_bwd(f0, s, upar, mu, uperp, aG0, af, aupar, amu, auperp);
    perp2_bwd(f0, s, mu, uperp, aP0, af, amu, auperp);
    // gg = vE.vgb,  A = vE.bgb
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        af.vE[k] += agg * f0.vgb[k] + aA * f0.bgb[k];
        af.vgb[k] += agg * f0.vE[k];
        af.bgb[k] += aA * f0.vE[k];
    }
}

// Conversion at R^{n-1/2}:  G = Gamma(u), u_par = u.b,
// u_g = u - u_par b - (vE + v_c(u_par, G)) G,  u_perp = |u_g|, bpg = u_g/u_perp,
// mu = u_perp^2 / (2 |B| kappa).
template <typename T>
__device__ __forceinline__ void conv_fwd(const Frame<T> &fm, const StepPar<T> &s, const T u[3],
                                         T &Gf, T &upar, T vc[3], T &uperp, T &mu, T bpg[3])
{
    Gf = sqrt(T(1) + dot3(u, u) * s.inv_c2);
    upar = dot3(u, fm.b);
    vcurv(fm, s, upar, Gf, vc);
    T ug[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) ug[k] = u[k] - upar * fm.b[k] - (fm.vE[k] + vc[k]) * Gf;
    uperp = sqrt(dot3(ug, ug));
    if (uperp < Eps<T>::tiny) {
        uperp = T(0);
        mu = T(0);
        bpg[0] = bpg[1] = bpg[2] = T(0);
    } else {
        const T iu = T(1) / uperp;
#pragma unroll
        for (int k = 0; k < 3; ++k) bpg[k] = ug[k] * iu;
        mu = uperp * uperp / (T(2) * fm.Bmag * fm.kappa);
    }
}

template <typename T>
__device__ __forceinline__ void conv_bwd(const Frame<T> &fm, const StepPar<T> &s, const T u[3],
                                         T Gf, T upar, const T vc[3], T uperp, T mu,
                                         const T bpg[3], T aupar, T amu, T auperp,
                                         const T abpg[3], FrameAdj<T> &af, T au[3])
{
    T aug[3] = {T(0), T(0), T(0)};
    if (uperp > T(0)) {
        auperp += amu * uperp / (fm.Bmag * fm.kappa);
        af.Bmag -= amu * mu / fm.Bmag;
        af.kappa -= amu * mu / fm.kappa;
        const T abb = dot3(abpg, bpg);
        const T iu = T(1) / uperp;
#pragma unroll
        for (int k = 0; k < 3; ++k) aug[k] = (abpg[k] - abb * bpg[k]) * iu + auperp * bpg[k];
    }
    T avc[3];
    T aGf = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        au[k] += aug[k];
        af.b[k] -= upar * aug[k];
        af.vE[k] -= Gf * aug[k];
        avc[k] = -Gf * aug[k];
        aGf -= aug[k] * (fm.vE[k] + vc[k]);
    }
    aupar -= dot3(aug, fm.b);
    vcurv_bwd(fm, s, upar, Gf, avc, af, aupar, aGf);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        au[k] += aupar * fm.b[k] + aGf * u[k] * s.inv_c2 / Gf;
        af.b[k] += aupar * u[k];
    }
}

// Reconstruction at R^{n+1/2}:  u = u_par b + (vE + v_c) G + u_n bpg,
// u_n = u_perp (mu_mode) or sqrt(2 mu |B| kappa).
template <typename T>
__device__ __forceinline__ void recon_bwd(const Frame<T> &fp, const StepPar<T> &s, T upn, T mu,
                                          T uperp, const T bpg[3], const T lamu[3],
                                          FrameAdj<T> &af, T &aupn, T &amu, T &auperp, T abpg[3])
{
    const T Gp = gamma_gc(fp, s, upn, mu, uperp);
    T vc[3];
    vcurv(fp, s, upn, Gp, vc);
    const T un = s.mu_mode ? uperp : sqrt(T(2) * mu * fp.Bmag * fp.kappa);
    aupn += dot3(lamu, fp.b);
    T avc[3];
    T aGp = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        af.b[k] += upn * lamu[k];
        af.vE[k] += Gp * lamu[k];
        abpg[k] += un * lamu[k];
        avc[k] = Gp * lamu[k];
        aGp += lamu[k] * (fp.vE[k] + vc[k]);
    }
    const T aun = dot3(lamu, bpg);
    if (s.mu_mode) {
        auperp += aun;
    } else if (un > T(0)) {
        const T iun = T(1) / un;
        amu += aun * fp.Bmag * fp.kappa * iun;
        af.Bmag += aun * mu * fp.kappa * iun;
        af.kappa += aun * mu * fp.Bmag * iun;
    }
    vcurv_bwd(fp, s, upn, Gp, avc, af, aupn, aGp);
    gamma_gc_bwd(fp, s, upn, mu, uperp, aGp, af, aupn, amu, auperp);
}

// Relativistic Boris push (Sec. 2.1) and disp = dt u/gamma: adjoints of u, E, B.
template <typename T, int ND>
__device__ __forceinline__ void boris_bwd(const T E[3], const T B[3], const StepPar<T> &s,
                                          const T u[3], const T lamu[3], const T ldisp[ND],
                                          T au[3], T aE[3], T aB[3])
{
    const T h = s.qm * s.half_dt;
    T um[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) um[k] = fma(h, E[k], u[k]);
    const T gm = sqrt(T(1) + dot3(um, um) * s.inv_c2);
    const T ht = h / (s.c * gm);
    T t[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = ht * B[k];
    const T sf = T(2) / (T(1) + dot3(t, t));
    T x1[3], up[3], x2[3], un[3];
    cross3(um, t, x1);
#pragma unroll
    for (int k = 0; k < 3; ++k) up[k] = um[k] + x1[k];
    cross3(up, t, x2);
#pragma unroll
    for (int k = 0; k < 3; ++k) un[k] = fma(h, E[k], fma(sf, x2[k], um[k]));
    const T g = sqrt(T(1) + dot3(un, un) * s.inv_c2);
    const T f = s.dt / g;

    // disp_d = f un_d (d < ND)
    T aun[3] = {lamu[0], lamu[1], lamu[2]};
    T af = T(0);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        af += ldisp[d] * un[d];
        aun[d] += f * ldisp[d];
    }
    const T ag = -af * s.dt / (g * g);
#pragma unroll
    for (int k = 0; k < 3; ++k) aun[k] += ag * un[k] * s.inv_c2 / g;
    // un = um + sf x2 + h E
    T aum[3], ax2[3], aup[3], ax1[3], at[3], tmp[3];
    const T asf = dot3(aun, x2);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        aum[k] = aun[k];
        ax2[k] = sf * aun[k];
        aE[k] = h * aun[k];
    }
    // x2 = up x t
    cross3(t, ax2, aup);
    cross3(ax2, up, at);
    // up = um + x1
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        aum[k] += aup[k];
        ax1[k] = aup[k];
    }
    // x1 = um x t
    cross3(t, ax1, tmp);
#pragma unroll
    for (int k = 0; k < 3; ++k) aum[k] += tmp[k];
    cross3(ax1, um, tmp);
    // sf = 2/(1 + t.t)
#pragma unroll
    for (int k = 0; k < 3; ++k) at[k] += tmp[k] - sf * sf * asf * t[k];
    // t = ht B,  ht = h/(c gm)
    const T aht = dot3(at, B);
    const T agm = -aht * ht / gm;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        aB[k] = ht * at[k];
        aum[k] += agm * um[k] * s.inv_c2 / gm;
        au[k] = aum[k];
        aE[k] += h * aum[k];
    }
}

}  // namespace rev
}  // namespace gcb
