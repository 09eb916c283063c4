/*
 * gcb_oracle.h -- plain FP64 CPU oracle of the coupled guiding-center / Boris
 * particle pusher of Bacchini, Ripperda, Philippov & Parfrey (2020).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no header, helper, table or kernel
 * with the CUDA library; it is written to be read against the paper, not to
 * be fast (the only concession is an OpenMP loop over particles, which does
 * not change the per-particle arithmetic).
 *
 * Conventions (all FP64):
 *   - flat space, general speed of light c;  alpha_q = q/m is signed,
 *     Q = |q/m|;  mu is stored as mu/m.
 *   - fields live on the nodes of a uniform periodic grid, node (i,j,k) at
 *     position (i dx, j dy, k dz), node index (k*ny + j)*nx + i;  one array
 *     per component.  In 2D runs (ndim = 2) z is ignorable: positions have two
 *     components, momenta three.
 *   - particle state: x^n (ndim comps), u^{n-1/2} (3 comps) and the unwrapped
 *     displacement dxp = x^n - x^{n-1} (ndim comps), staggered as in Sec. 2.1.
 *   - flags byte: bit0 S of the last step, bit1 S of the step before,
 *     bit2 NONCONV, bit3 GCAFAIL, bit4 NONFINITE, bit5 EXITED (covariant
 *     scheme: left [r_in, r_out]), bits 6-7 species index.
 */
#ifndef GCB_ORACLE_H
#define GCB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_FIELD_GRID = 0, ORC_FIELD_UNIFORM = 1, ORC_FIELD_HARRIS = 2,
       ORC_FIELD_BOTTLE = 3, ORC_FIELD_ROTOR = 4 };
enum { ORC_GRAD_DW = 0, ORC_GRAD_GRID = 1 };
enum { ORC_FORCE_NONE = 0, ORC_FORCE_BORIS = 1, ORC_FORCE_GCA = 2 };
enum { ORC_MU_CONSERVE = 0, ORC_UPERP_CONSERVE = 1 };
/* drift frame of the guiding-center decomposition (Sec. 2.2): the simplified
 * one the paper's schemes use, or the exact Beklemishev-Tessarotto one */
enum { ORC_FRAME_SIMPLE = 0, ORC_FRAME_BT = 1 };

enum { ORC_FLAG_S = 1, ORC_FLAG_SPREV = 2, ORC_FLAG_NONCONV = 4,
       ORC_FLAG_GCAFAIL = 8, ORC_FLAG_NONFINITE = 16, ORC_FLAG_EXITED = 32 };

/* Kerr-Schild fields (covariant scheme, geometrized units c = G = M = 1). */
enum { ORC_KS_GRID = 0, ORC_KS_VACUUM = 1, ORC_KS_MONOPOLE = 2 };

typedef struct {
    int kind;            /* ORC_FIELD_* */
    int ndim;            /* 2 or 3 */
    long n[3];           /* nodes per axis (periodic) */
    double dx[3];        /* node spacing */
    const double *E[3];  /* node arrays (kind GRID) */
    const double *B[3];
    const double *dB[9]; /* dB[3*i+j] = d_i B_j at the nodes (grad_mode GRID) */
    double par[16];      /* analytic parameters (see gcb_oracle.c) */
} orc_field;

typedef struct {
    double c, dt;
    double f_rho, f_E;   /* switch thresholds (Sec. 4.1) */
    double dl;           /* effective cell size Delta-ell (Sec. 3) */
    double qm[4];        /* q/m per species */
    int curvature;       /* 1: Sec. 2.2.2 scheme, 0: Sec. 2.2.1 scheme */
    int mu_mode;         /* ORC_MU_CONSERVE or ORC_UPERP_CONSERVE (Sec. 2.2) */
    int grad_mode;       /* ORC_GRAD_DW or ORC_GRAD_GRID */
    int force;           /* ORC_FORCE_*: test aid, bypasses the switch */
    int max_iter;        /* bound of the fixed-point iteration */
    int fixed_iters;     /* > 0: exactly this many iterations, no test */
    double tol;          /* absolute stopping tolerance on |R^{k+1}-R^k|_inf */
    int frame;           /* ORC_FRAME_SIMPLE (b, v_E = cExB/B^2) or ORC_FRAME_BT */
    int gyro_phase;      /* 0: gyration direction kept (Sec. 3.1); 1: advanced by
                            the gyro-frequency over the step */
    int mirror;          /* 0: the paper's reduced GCA; 1: with the grad-B drift
                            and the mirror force it discards (Sec. 2.2) */
} orc_params;

typedef struct {
    long n_boris, n_gca, n_to_gca, n_to_boris;
    long n_nonconv, n_gcafail, n_nonfinite, sum_iter;
    long max_iter;
    double sum_ekin;     /* sum of (Gamma - 1) over particles and steps */
    long n_exited;       /* covariant push: steps not taken after leaving [r_in, r_out] */
} orc_stats;

/* Kerr-Schild field on the axisymmetric node grid (log r, theta):
 * node (i, j) at log r = logr0 + i dlogr, theta = j dth (j = 0 .. nth-1,
 * dth = pi / (nth - 1)); D^i, B^i contravariant KS components, index
 * j * nr + i.  MONOPOLE: B^r = par[0] sin(theta) / sqrt(gamma) with
 * par[1] = spin, D = 0.  VACUUM: no field. */
typedef struct {
    int kind;
    int nr, nth;
    double logr0, dlogr, dth;
    const double *D[3], *B[3];
    double par[8];
} orc_ks_field;

typedef struct {
    double a;            /* black-hole spin */
    double r_in, r_out;  /* particles leaving [r_in, r_out] are flagged EXITED */
    int kick_basis;      /* GREOM half kicks: 0 local frame (tetrad), 1 global coordinate basis */
} orc_ks_params;

/* Everything one particle-step computed, for the closed-form tests. */
typedef struct {
    int S;               /* switch value (after force) */
    double margin;       /* signed criterion margin, see orc_switch */
    int branch;          /* 1 Boris, 0 GCA, -1 frozen */
    int gcafail, nonconv, iters;
    double resid;        /* |R^K - R^{K-1}|_inf of the last iteration */
    double H;            /* |H(R^K)|_inf of the final iterate */
    double upar_old, upar_new, mu, uperp, Gamma_full;
    double Gamma1;       /* Gamma(R^n, u_par^{n+1/2}) from the quadratic */
    double k1, k2, k3;
    double Rn[3], Rnp1[3], bpg[3];
    double vstep[3];     /* velocity of the step's straight path: x^{n+1} - x^n
                            = dt vstep (Boris: u^{n+1/2}/Gamma; GCA: the
                            guiding-center velocity (V^n + V^K)/2); in 2D
                            vstep[2] is its out-of-plane component */
} orc_detail;

/* The exact (Beklemishev-Tessarotto) drift frame of fields E, B (Sec. 2.2):
 * out[0..2] v_E, out[3..5] b*, out[6] kappa, out[7] E', out[8] B'.
 * Returns 0 when B = 0 (out untouched). */
int orc_bt_frame(const double E[3], const double B[3], double c, double out[9]);

/* E, B and d_i B_j (out[0..2] E, out[3..5] B, out[6+3i+j] d_i B_j). */
void orc_eval_field(const orc_field *f, const orc_params *p,
                    const double x[3], double out[15]);

/* Switch S of Sec. 4.1 (0 = GCA, 1 = Boris) at field point (E,B) for a
 * particle of Lorentz factor Gam; *margin receives the criterion margin. */
int orc_switch(const double E[3], const double B[3], double Gam, double Q,
               const orc_params *p, double *margin);

/* One coupled step of one particle (Sec. 3.1). */
void orc_step_one(const orc_field *f, const orc_params *p, double x[3],
                  double u[3], double dxp[3], unsigned char *flags,
                  orc_detail *d);

/* Full -> GC decomposition (Sec. 3.1) at the point R with full u and the
 * Lorentz factor of u; returns 0 on an invalid frame. */
int orc_decompose(const orc_field *f, const orc_params *p, double qm,
                  const double R[3], const double u[3], double *upar,
                  double *mu, double *uperp, double bpg[3]);

/* GC -> full reconstruction (Sec. 3.1) at the point R. */
int orc_reconstruct(const orc_field *f, const orc_params *p, double qm,
                    const double R[3], double upar, double mu, double uperp,
                    const double bpg[3], double u[3]);

/* n_steps coupled steps of n particles (SoA, arrays per component). */
int orc_push_sr(long n, double *const x[3], double *const u[3],
                double *const dxp[3], unsigned char *flags,
                const orc_field *f, const orc_params *p, int n_steps,
                int nthreads, orc_stats *st);

/* Gyro-resolved Boris reference (Sec. 4.1): adaptive step
 * dt_k = min(dt_max, 2 pi / (60 Omega_C)) until time t_end. */
int orc_push_resolved(long n, double *const x[3], double *const u[3],
                      unsigned char *flags, const orc_field *f,
                      const orc_params *p, double t_end, double dt_max,
                      int nthreads);

/* Kerr-Schild metric at (r, theta): out[0] alpha, [1..3] beta^i, [4..12]
 * gamma_ij, [13..21] gamma^{ij}, [22] sqrt(gamma), [23..25] d_i alpha,
 * [26..34] d_i beta^j, [35..61] d_i gamma^{jk} (i = r, theta, phi). */
void orc_ks_metric(double a, double r, double th, double out[64]);

void orc_ks_gather(const orc_ks_field *f, double r, double th, double D[3], double B[3]);

/* Effective cell sizes of Eq. (volint), (nr-1)*(nth-1) values, index j*(nr-1)+i. */
void orc_ks_cell_sizes(const orc_ks_field *f, double a, double *dl);

/* Local-frame components: out[0..2] of covariant u, out[3..5] of contravariant F. */
void orc_ks_frame(double a, double r, double th, const double u[3], const double F[3],
                  double out[6]);

/* Boris kick (Sec. 2.3) of covariant u by contravariant D, B at (r, theta)
 * over proper time dtau: basis 0 in the local frame, 1 in the global basis. */
void orc_ks_kick(double a, double r, double th, const double D[3], const double B[3], double qm,
                 double dtau, int basis, double u[3]);

/* One coupled covariant step (Sec. 3.2) of one particle (x = r, theta, phi;
 * u covariant); dl is the cell-size table (NULL: dl = 1). */
void orc_ks_step_one(const orc_ks_field *f, const orc_ks_params *kp, const orc_params *p,
                     const double *dl, double x[3], double u[3], unsigned char *flags,
                     orc_detail *d);

int orc_push_ks(long n, double *const x[3], double *const u[3], unsigned char *flags,
                const orc_ks_field *f, const orc_ks_params *kp, const orc_params *p,
                const double *dl, int n_steps, int nthreads, orc_stats *st);

/* ---- Current deposition (PiC coupling).  A particle-step is a linear-weight
 * (cloud-in-cell) cloud of charge Qw moving from x^n to x^{n+1} = x^n + disp
 * along a straight line at constant velocity; J is the time average over the
 * step of its current on the staggered points of the node grid:
 *   J_a at (i + e_a/2) = Qw/(dt V) int_0^dt v_a Pi(s_a - i_a - 1/2)
 *                            prod_{b != a} S(s_b - i_b) dt,
 * s = x/dx, S the unit hat, Pi the unit box, V the cell volume; in 2D J_z
 * sits on the nodes, Qw/V int_0^dt v_z S(s_x - i) S(s_y - j) dt / dt.
 * J_a is stored at the index of the point's lower node, node index
 * (k*ny + j)*nx + i, periodic.  Paths longer than ORC_DEP_MAX_CELLS cells
 * along an axis are left out (return 1). */
#define ORC_DEP_MAX_CELLS 64

typedef struct {
    double q[4];         /* charge of one macro-particle per species */
    const double *w;     /* per-particle weight (NULL: 1) */
    double *J[3];        /* current, accumulated */
    double *Jabs[3];     /* optional (NULL): sum of |contribution| per point */
    long n_skipped;      /* out: particle-steps left out (path too long) */
} orc_deposit_t;

int orc_deposit(const orc_field *f, const double x0[3], const double disp[3], double vz,
                double Qw, double dt, double *const J[3], double *const Jabs[3]);

/* orc_push_sr that also deposits every advanced particle-step's current into
 * dep (in particle order after each step's parallel loop). */
int orc_push_sr_dep(long n, double *const x[3], double *const u[3],
                    double *const dxp[3], unsigned char *flags,
                    const orc_field *f, const orc_params *p, int n_steps,
                    int nthreads, orc_stats *st, orc_deposit_t *dep);

#ifdef __cplusplus
}
#endif
#endif
