/*
 * gcb.h -- C ABI of the GB300 coupled guiding-center / Boris particle pusher.
 *
 * Method: Bacchini, Ripperda, Philippov & Parfrey (2020), "A coupled
 * guiding center-Boris particle pusher for magnetized plasmas in
 * compact-object magnetospheres".  For each particle one step
 *   1. gathers E, B (and the gradients of B) at x^n with the linear shape
 *      function of Sec. 4 (intro): F(x) = sum_N F_N W(x - x_N),
 *      grad F(x) = sum_N F_N grad W(x - x_N);
 *   2. evaluates the switch S of Sec. 3 / Sec. 4.1: S = 0 (guiding center)
 *      iff rho~_C / dl < f_rho and E/B < f_E, rho~_C = m c^2 Gamma/(|q| B);
 *   3. advances with the relativistic Boris push (S = 1, Sec. 2.1) or with
 *      the guiding-center leapfrog of Sec. 2.2.1 (no curvature) / Sec. 2.2.2
 *      (with curvature), converting the full state to (R, u_par, mu) at
 *      R^{n-1/2} and back at R^{n+1/2} (Sec. 3.1).
 *
 * All entry points are asynchronous on the caller's CUDA stream unless
 * stated otherwise.  The library never allocates device memory: the caller
 * owns every buffer (including the workspace) and the library keeps no
 * pointer after a call returns.  Errors are returned as gcb_status; nothing
 * is launched when an argument check fails.  gcb_last_error() returns a
 * thread-local message describing the last failure.
 *
 * Units: flat space, general speed of light c (all shipped workloads use
 * c = 1).  u is the spatial part of the 4-velocity (u = gamma v, velocity
 * units); q/m is signed; mu is stored as mu/m.
 */
#ifndef GCB_H
#define GCB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GCB_OK = 0,
    GCB_EINVAL = 1,          /* invalid argument (null pointer, bad size, ...) */
    GCB_ECUDA = 2,           /* a CUDA runtime call failed */
    GCB_EUNSUPPORTED = 3,    /* valid but not implemented combination */
    GCB_ENOMEM = 4           /* caller-provided workspace too small */
} gcb_status;

enum { GCB_F32 = 0, GCB_F64 = 1 };                       /* element types */
enum { GCB_POS_F64 = 0, GCB_POS_F32PAIR = 1 };           /* position storage */
enum { GCB_GRAD_DW = 0, GCB_GRAD_GRID = 1 };             /* source of grad B */
enum { GCB_FORCE_NONE = 0, GCB_FORCE_BORIS = 1, GCB_FORCE_GCA = 2 };
enum { GCB_MU_CONSERVE = 0, GCB_UPERP_CONSERVE = 1 };
enum { GCB_FRAME_SIMPLE = 0, GCB_FRAME_BT = 1 };
enum { GCB_PHASE_KEEP = 0, GCB_PHASE_EVOLVE = 1 };
enum { GCB_MIRROR_OFF = 0, GCB_MIRROR_ON = 1 };

/* Per-particle flag byte. */
enum {
    GCB_FLAG_S = 1,          /* S of the last step (1 = Boris, 0 = GCA) */
    GCB_FLAG_SPREV = 2,      /* S of the step before */
    GCB_FLAG_NONCONV = 4,    /* last GCA fixed point hit gca_max_iter */
    GCB_FLAG_GCAFAIL = 8,    /* last GCA step impossible (quadratic without a
                                root >= 1, B = 0 or v_E >= c on the path):
                                the particle took a Boris step instead */
    GCB_FLAG_NONFINITE = 16, /* state non-finite: particle not advanced */
    GCB_FLAG_EXITED = 32,    /* covariant scheme: left [r_in, r_out]; frozen */
    GCB_SPECIES_SHIFT = 6    /* bits 6-7: species index into gcb_params.qm */
};

/*
 * Field grid in the packed node-record layout.  The grid is uniform and
 * periodic with n[d] nodes along axis d, node (i,j,k) at (i dx0, j dx1, k dx2),
 * node index (k n1 + j) n0 + i.  Each node holds one record of `stride`
 * elements of type `dtype`:
 *     E0 E1 E2 B0 B1 B2 [d_0B_0 d_0B_1 d_0B_2 d_1B_0 ... d_{ndim-1}B_2] pad
 * where the gradient block (3*ndim elements) is present iff has_grad, and
 * the stride (gcb_grid_stride) pads the record to a multiple of 16 bytes.
 * In 2D (ndim = 2) z is ignorable: positions have two components and
 * d_z = 0.  Build records with gcb_grid_pack.
 */
typedef struct {
    int32_t ndim;            /* 2 or 3 */
    int32_t dtype;           /* GCB_F32 or GCB_F64 */
    int64_t n[3];            /* nodes per axis (n[2] = 1 in 2D) */
    double dx[3];            /* node spacing per axis (> 0) */
    int32_t has_grad;        /* records carry d_i B_j (needed by GCB_GRAD_GRID) */
    int32_t stride;          /* elements per record, = gcb_grid_stride(...) */
    const void *rec;         /* device pointer, 16-byte aligned */
} gcb_grid;

/*
 * Particle state, structure of arrays, staggered as in
 * Sec. 2.1: positions x^n at integer steps, u^{n-1/2} at half steps, and the
 * unwrapped displacement dxp = x^n - x^{n-1} of the previous step (the
 * decomposition point R^{n-1/2} = x^n - dxp/2 of Sec. 3.1 needs it).
 *   pos_mode GCB_POS_F64:     x[d] are double arrays; x_lo unused.
 *   pos_mode GCB_POS_F32PAIR: x[d] are float "hi" arrays and x_lo[d] float
 *                             "lo" arrays, position = hi + lo (|lo| <= ulp(hi)/2).
 *   mom_dtype GCB_F64 / GCB_F32: element type of u[0..2] and dxp[0..ndim-1].
 * Positions are kept in [0, L_d) (periodic wrap after every step).
 * Each array must be aligned to its element size and reachable from the
 * current device at its own address: the device's memory, managed memory,
 * or pinned / registered host memory (cudaHostAlloc, cudaHostRegister; with
 * unified addressing the host address itself).  A particle state left in
 * pinned host memory is pushed in place: the kernels read and write it
 * across the host link every step (NVLink-C2C on a Grace host), with no
 * staging copies.  Every entry point that takes particles checks each array
 * with cudaPointerGetAttributes before any launch and returns GCB_EINVAL for
 * one the device cannot reach (plain pageable host memory included).
 */
typedef struct {
    int64_t n;               /* number of particles (>= 0) */
    int32_t ndim;            /* must equal the grid's ndim */
    int32_t pos_mode;
    int32_t mom_dtype;
    int32_t reserved;
    void *x[3];
    void *x_lo[3];
    void *u[3];
    void *dxp[3];
    uint8_t *flags;          /* n bytes, see GCB_FLAG_* */
    int64_t *pid;            /* optional particle ids (NULL = none); sorting
                                permutes them with the particles */
} gcb_particles;

typedef struct {
    double c;                /* speed of light (> 0) */
    double dt;               /* time step (> 0) */
    double f_rho, f_E;       /* switch thresholds (> 0); Sec. 4.1 defaults 0.4, 1 */
    double dl;               /* effective cell size Delta-ell (> 0), Sec. 3 */
    double qm[4];            /* q/m per species (non-zero for used species) */
    int32_t curvature;       /* 1: Sec. 2.2.2 scheme; 0: Sec. 2.2.1 scheme */
    int32_t mu_mode;         /* GCB_MU_CONSERVE (Eq. dmudt) or GCB_UPERP_CONSERVE */
    int32_t grad_mode;       /* GCB_GRAD_DW (differentiate W) or GCB_GRAD_GRID */
    int32_t force;           /* GCB_FORCE_*: bypass the switch (tests, studies) */
    int32_t gca_max_iter;    /* bound of the fixed-point iteration (>= 1) */
    int32_t gca_fixed_iters; /* > 0: exactly this many iterations, no test */
    double gca_tol;          /* absolute tolerance on |R^{k+1}-R^k|_inf (Sec. 2.2) */
    int32_t sort_every;      /* > 0: sort the particles by cell tile before every
                                step whose global index is a multiple of it */
    int32_t sort_tile[3];    /* cells per sort tile along each axis (0 = 8,8,4) */
    int64_t step_index;      /* global index of the first step of this call */
    int32_t fuse_steps;      /* <= 1: one kernel launch per step, the state going
                                through device memory every step (the PiC mode:
                                fields may change between calls of one step);
                                k > 1: up to k steps per launch with each
                                particle tile's state kept on chip between them
                                (the test-particle mode, fields static over the
                                call); a fused launch never spans a sort.  The
                                results are the same bit for bit. */
    int32_t drift_frame;     /* GCB_FRAME_SIMPLE (0): the guiding-center step in
                                the simplified frame b = B/B, v_E = c E x B/B^2
                                that the paper's schemes use (Sec. 2.2);
                                GCB_FRAME_BT: in the exact frame of Sec. 2.2
                                (Beklemishev & Tessarotto): b* and the exact v_E
                                (and kappa from it) in place of b and v_E, and
                                E_par = E.b*, with the gradients of b taken for
                                those of b* (the records carry no grad E).
                                GCB_FRAME_BT: gcb_push_sr and gcb_push_deposit_sr,
                                unfused, FP64 or FP32-pair positions, without the
                                mirror terms; elsewhere GCB_EUNSUPPORTED. */
    int32_t gyro_phase;      /* GCB_PHASE_KEEP (0): the reconstruction keeps the
                                gyration direction of the decomposition (Sec. 3.1);
                                GCB_PHASE_EVOLVE: it turns that direction about b
                                by the step's gyro-phase -(q/m) B dt/(c kappa
                                Gamma) at R^{n+1/2} (the extra equation Sec. 3.1
                                says could be added).  gcb_push_sr only; the
                                covariant push and the adjoint refuse it. */
    int32_t mirror;          /* GCB_MIRROR_OFF (0): the paper's reduced GCA, which
                                drops the grad-B drift and the mirror force
                                (Sec. 2.2); GCB_MIRROR_ON: with them, in the
                                relativistic forms of the expansion the paper cites:
                                (c kappa mu/((q/m) B Gamma)) b x grad B added to
                                the guiding-center velocity and the force
                                -(mu/Gamma) b.grad(B)/kappa to du_par/dt, explicit
                                at (x^n, u_par^{n-1/2}) (mu as mu/m; grad kappa
                                neglected: the records carry no grad E).
                                gcb_push_sr and gcb_push_deposit_sr, unfused,
                                simplified frame; the covariant push and the
                                adjoint refuse it (GCB_EUNSUPPORTED). */
} gcb_params;

/* Counters of one push call (gcb_push_sr, gcb_push_ks, ...), summed over its
 * steps. */
typedef struct {
    int64_t n_boris, n_gca;          /* particle-steps per branch */
    int64_t n_to_gca, n_to_boris;    /* switches S: 1 -> 0 and 0 -> 1 */
    int64_t n_nonconv, n_gcafail;    /* steps with GCB_FLAG_NONCONV / GCB_FLAG_GCAFAIL */
    int64_t n_nonfinite;             /* particle-steps not advanced: non-finite state
                                        (GCB_FLAG_NONFINITE) */
    int64_t sum_iter, max_iter;      /* fixed-point iterations */
    double sum_ekin;                 /* sum of (Gamma - 1) m c^2 / m after each step */
    int64_t n_exited;                /* particle-steps not advanced because the
                                        particle had left [r_in, r_out] before the
                                        step (GCB_FLAG_EXITED; covariant push only) */
} gcb_stats;

/* Library version (major*10000 + minor*100 + patch). */
int gcb_version(void);

/* Human-readable name of a status code (static storage). */
const char *gcb_status_string(gcb_status s);

/* Message of the last failure on the calling thread ("" if none). */
const char *gcb_last_error(void);

/* Elements per node record for a grid of this shape (0 on bad input). */
int32_t gcb_grid_stride(int32_t ndim, int32_t dtype, int32_t has_grad);

/*
 * Pack component arrays into node records (device kernel on `stream`).
 *   g      : destination description; g->rec must point to a device buffer
 *            of n0*n1*n2*stride elements of g->dtype (written here).
 *   comp   : 6 + 3*ndim device pointers to float64 node arrays of n0*n1*n2
 *            values in node order: E0 E1 E2 B0 B1 B2, then d_i B_j (i major)
 *            when g->has_grad.  Values are rounded to g->dtype.
 * Errors: GCB_EINVAL on a null pointer or inconsistent shape/stride.
 */
gcb_status gcb_grid_pack(const gcb_grid *g, const double *const *comp, void *cuda_stream);

/*
 * Split float64 positions into float32 pairs (hi = fl32(x), lo = fl32(x - hi))
 * and back (x = hi + lo in float64): conversion of a GCB_POS_F64 state to
 * GCB_POS_F32PAIR storage.  All pointers are device arrays of n elements.
 */
gcb_status gcb_pos_split(int64_t n, const double *x, float *hi, float *lo, void *cuda_stream);
gcb_status gcb_pos_join(int64_t n, const float *hi, const float *lo, double *x, void *cuda_stream);

/* Workspace bytes gcb_push_sr / gcb_sort_sr need for this problem (a device
 * buffer): 256 bytes of counters, plus, when prm->sort_every > 0 (always for
 * gcb_sort_sr), per-particle keys and one copy of the particle arrays. */
size_t gcb_workspace_bytes(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm);

/*
 * Reorder the particles in place by the tile of cells that holds them (tiles
 * of prm->sort_tile cells, row-major over tiles; non-finite particles last),
 * a counting sort on the device.  Gathers of particles that are close in
 * memory then touch the same few field records, which the L1 cache holds.
 * The order inside a tile is not specified; pid, when given, is permuted
 * with the particles.  ws as for gcb_push_sr with sorting enabled.
 * This is a layout step of the GPU design, not part of the paper's method.
 */
gcb_status gcb_sort_sr(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm,
                       void *cuda_stream, void *ws, size_t ws_bytes);

/*
 * Advance every particle by n_steps coupled steps (Sec. 3.1), in place.
 *   p, g, prm : problem description (host structs, device arrays).
 *   n_steps   : >= 0; each step is one kernel pass over all particles, so
 *               the state round-trips HBM every step as in a PiC code.
 *               With prm->sort_every > 0 the particles are first reordered
 *               (as gcb_sort_sr) before steps whose global index
 *               prm->step_index + j is a multiple of sort_every.
 *   stream    : cudaStream_t (NULL = legacy default stream).
 *   ws        : device workspace of at least gcb_workspace_bytes() bytes,
 *               256-byte aligned; contents on entry are ignored.
 *   out       : host gcb_stats, or NULL.  When non-NULL the call
 *               synchronizes `stream` and fills it; otherwise it returns
 *               without synchronizing.
 * Supported precisions: (mom_dtype F64, pos F64, grid F64) = FP64 path;
 * (mom_dtype F32, pos F64 or F32PAIR, grid F32) = mixed path.
 * Per-particle numerical events are not errors: they set GCB_FLAG_* bits
 * and counters.  No device-side trap or assert exists; every loop is bounded.
 */
gcb_status gcb_push_sr(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm,
                       int n_steps, void *cuda_stream, void *ws, size_t ws_bytes,
                       gcb_stats *out);

/*
 * ---- Push with current deposition (PiC coupling).
 * The paper presents the coupled scheme as usable inside a PiC code (Sec. 1,
 * 5): each step returns x^{n+1} and u^{n+1/2} at the usual staggered times,
 * whichever branch advanced the particle, and the code deposits the step's
 * current.  The paper gives no deposition of its own; this one is the exact
 * current of a linear-weight (cloud-in-cell) particle of charge Q w moving
 * from x^n to x^{n+1} along a straight line at constant velocity, averaged
 * over the step, on the staggered (Yee) points of the field's node grid:
 *
 *   J_a(i + e_a/2) = Q w / (dt V) int_0^dt v_a Pi(s_a(t) - i_a - 1/2)
 *                        prod_{b != a} S(s_b(t) - i_b) dt,
 *
 * s = x/dx in cells, S(s) = max(0, 1 - |s|), Pi the unit box, V the cell
 * volume.  In 2D the out-of-plane component sits on the nodes:
 * J_z(i, j) = Q w v_z / (dt V) int_0^dt S(s_x - i) S(s_y - j) dt, with v_z
 * the step's out-of-plane velocity (Boris: u_z^{n+1/2}/Gamma; guiding
 * center: the z component of (V^n + V^K)/2, the velocity whose in-plane part
 * moved it).  With the cloud-in-cell charge density rho_i = sum Q w S(s - i)/V
 * the deposited J satisfies the discrete continuity equation
 * (rho^{n+1} - rho^n)/dt + sum_a (J_a(i + e_a/2) - J_a(i - e_a/2))/dx_a = 0
 * up to rounding, for paths crossing any number of cells.
 */
#define GCB_DEPOSIT_MAX_CELLS 64  /* longer paths (cells along an axis in one
                                     step) are left out and counted */

typedef struct {
    int32_t dtype;           /* GCB_F32 (mixed path) or GCB_F64 (FP64 path): the
                                type of J and w, equal to mom_dtype */
    int32_t reserved;        /* 0 */
    double q[4];             /* charge of one macro-particle per species */
    const void *w;           /* optional per-particle weights, n elements of dtype
                                (NULL: 1); not permuted by sorting, so a call with
                                w and prm->sort_every > 0 is GCB_EUNSUPPORTED */
    void *J[3];              /* device arrays of n[0] n[1] n[2] elements of dtype,
                                node index (k n[1] + j) n[0] + i, aligned to dtype:
                                J_x at (i+1/2, j, k), J_y at (i, j+1/2, k), J_z at
                                (i, j, k+1/2) (2D: at node (i, j)), each stored at
                                its lower node's index, periodic.  The call ADDS
                                the current of every step (zero them first). */
} gcb_current;

typedef struct {
    int64_t n_skipped;       /* particle-steps whose path was longer than
                                GCB_DEPOSIT_MAX_CELLS cells along an axis
                                (left out of J) */
    int64_t n_pieces;        /* path pieces deposited (one per cell crossed into,
                                plus one per particle-step) */
    int64_t n_atomics;       /* atomic additions into J issued (non-zero values) */
} gcb_deposit_stats;

/*
 * gcb_push_sr that also deposits every advanced particle-step's current into
 * cur->J with atomic additions (the order of the additions is not
 * specified, so J's rounding varies from run to run; FP32 J for the mixed
 * path).  Frozen (non-finite) particles deposit nothing.  The step is that
 * of gcb_push_sr with the same options (drift frame, mirror terms, gyration
 * phase).  Unfused launches only: prm->fuse_steps > 1 or a grid of 2^31
 * nodes or more is GCB_EUNSUPPORTED.  dst (host, optional): when
 * non-NULL the call synchronizes `stream` and fills it (counts over all the
 * call's steps).
 * Other arguments, checks and errors as gcb_push_sr; GCB_EINVAL for a NULL,
 * misaligned or unreachable J or w, a dtype other than the particles'
 * mom_dtype, or a non-finite charge.
 */
gcb_status gcb_push_deposit_sr(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm,
                               const gcb_current *cur, int n_steps, void *cuda_stream, void *ws,
                               size_t ws_bytes, gcb_stats *out, gcb_deposit_stats *dst);

/*
 * ---- Adjoint of the flat-space push (2D, gradient-grid records, no sorting).
 * Gradients of an observable L of the final state with respect to the
 * initial state and to every field-record value.  Not part of the paper: a
 * reverse sweep over the steps (branch and iteration count of every
 * particle-step held fixed), from checkpoints stored every ckpt_every steps
 * with the segment between checkpoints recomputed forward.
 *
 * Workspace bytes for gcb_adjoint_sr (256-byte aligned device buffer).
 */
#define GCB_ADJOINT_MAX_ITER 22   /* gca_max_iter / gca_fixed_iters limit */

/* How the transposed step is formed: REVERSE, the step's derivative written
 * out backwards (the fast default); TANGENT, columns of the step's Jacobian
 * from dual-number replays contracted with the adjoint (a slower second
 * construction of the same quantity, for cross-checks). */
enum { GCB_ADJ_REVERSE = 0, GCB_ADJ_TANGENT = 1 };
/* or-ed into method: the checkpoints are already in ws (gcb_push_sr_ckpt) */
#define GCB_ADJ_HAVE_CKPT 0x100

/* 0 on invalid arguments.  With prm->sort_every > 0 the workspace also holds
 * the sort's scratch, one int32 permutation per checkpoint and scratch copies
 * of the adjoint arrays (see gcb_adjoint_sr). */
size_t gcb_adjoint_workspace_bytes(const gcb_particles *p, const gcb_grid *g,
                                   const gcb_params *prm, int n_steps, int ckpt_every);

/*
 *   p0         : initial state (device arrays, read only; FP64 or mixed
 *                layout as for gcb_push_sr, ndim 2).
 *   method     : GCB_ADJ_REVERSE or GCB_ADJ_TANGENT, optionally or-ed with
 *                GCB_ADJ_HAVE_CKPT (see gcb_push_sr_ckpt).
 *   g, prm     : as for gcb_push_sr; needs g->has_grad and grad_mode GRID.
 *                prm->sort_every > 0: the particles are sorted by cell (tiles
 *                of prm->sort_tile) at every checkpoint, the start included,
 *                so that the segments run on cell-ordered particles; lam and
 *                the state keep the caller's order at the call's boundaries
 *                (the adjoint is permuted with the particles inside).  The
 *                pushes between checkpoints do not sort.  Use
 *                gca_fixed_iters > 0 so every particle-step has the same
 *                iteration count as the forward.
 *   lam[7]     : device arrays of n elements of the momentum type, in the
 *                order x0 x1 u0 u1 u2 dxp0 dxp1: on entry dL/d(final state),
 *                on return dL/d(initial state).
 *   grad_rec   : device array of n0*n1*12 doubles, overwritten with dL/d(record
 *                value) for every node and record component.
 * Errors: GCB_EINVAL / GCB_EUNSUPPORTED / GCB_ENOMEM as for gcb_push_sr.
 */
gcb_status gcb_adjoint_sr(const gcb_particles *p0, const gcb_grid *g, const gcb_params *prm,
                          int n_steps, int ckpt_every, int method, void *const *lam,
                          double *grad_rec, void *cuda_stream, void *ws, size_t ws_bytes);

/*
 * The forward pass for a later gcb_adjoint_sr: n_steps pushes of p in place
 * that also store, in the adjoint workspace ws, the initial state and every
 * ckpt_every-th state (sorted by cell first when prm->sort_every > 0; p then
 * runs in cell order and is returned in its original order).  gcb_adjoint_sr with
 * method | GCB_ADJ_HAVE_CKPT on the same ws, the same n, layout, n_steps and
 * ckpt_every then starts from those checkpoints instead of running its own
 * forward pass (its p0 argument then only describes the layout; the caller
 * keeps ws untouched in between).  out: the forward's statistics, or NULL.
 * Errors as gcb_adjoint_sr.
 */
gcb_status gcb_push_sr_ckpt(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm,
                            int n_steps, int ckpt_every, void *cuda_stream, void *ws,
                            size_t ws_bytes, gcb_stats *out);

/*
 * Fields linear in n_modes amplitudes a_m: rec = base + sum_m a_m pat_m
 * (gcb_grid_combine, writes g->rec) and dL/da_m = <grad_rec, pat_m>
 * (gcb_grad_project, out: n_modes doubles).  base, pat: device records in
 * g's layout, pat holding n_modes consecutive record sets; n_modes <= 64.
 */
gcb_status gcb_grid_combine(const gcb_grid *g, const void *base, const void *pat,
                            const double *amps, int n_modes, void *cuda_stream);
gcb_status gcb_grad_project(const gcb_grid *g, const double *grad_rec, const void *pat,
                            int n_modes, double *out, void *cuda_stream);

/*
 * ---- Covariant (Kerr-Schild) scheme: Sec. 2.3 (GREOM), Sec. 2.4 (GRGCA),
 * Sec. 3.2 (coupling).  Geometrized units c = G = M = 1 (prm->c must be 1).
 *
 * Grid: axisymmetric, uniform in (log r, theta): g.ndim = 2, axis 0 radial
 * with n[0] nodes at log r = logr0 + i dx[0], axis 1 polar with n[1] nodes at
 * theta = j dx[1], dx[1] = pi / (n[1] - 1) (nodes on both poles).  Records
 * (has_grad = 0): D^r D^theta D^phi B^r B^theta B^phi, contravariant
 * Kerr-Schild components (D^i = alpha F^{0i}, B^i = e^{ijk} F_jk / 2).  The
 * linear shape function is used in (log r, theta), not periodic.
 * dl: device array of (n[0]-1)*(n[1]-1) effective cell sizes, index
 * j*(n[0]-1)+i, from gcb_ks_cell_size.
 * Particles: ndim = 3, x = (r, theta, phi), u covariant (u_r, u_theta,
 * u_phi), both FP64 (pos_mode GCB_POS_F64, mom_dtype GCB_F64), not staggered
 * (Sec. 3.2); dxp unused.  Records may be FP32 (FP32 field interpolation) or
 * FP64; all other arithmetic, including the metric, is FP64.
 */
typedef struct {
    gcb_grid g;
    double logr0;
    const double *dl;
} gcb_grid_ks;

/*
 * Basis of the GREOM half kicks (Sec. 2.3 steps 1 and 3).
 *   GCB_KS_TETRAD: the Boris kick in the local frame of the normal observer,
 *     the paper's choice (triad from gamma^{ij} = L L^T, L the Cholesky factor).
 *   GCB_KS_GLOBAL: the same kick written in the global coordinate basis, which
 *     the paper (Sec. 2.3, Sec. 2.4) names as an option for spacetimes where a
 *     tetrad is awkward: D_i = gamma_ij D^j, u-_i = u_i + h D_i,
 *     t^k = h B^k / Gamma-, |t|^2 = gamma_ij t^i t^j, cross products
 *     (a x b)_i = sqrt(gamma) [ijk] a^j b^k of raised vectors, h = (q/m) alpha dt / 4.
 *     Identical to the tetrad kick up to rounding (det L = 1/sqrt(gamma)).
 * The GRGCA kick adds (q/m) alpha dt/2 D_par to the scalar u_par in both bases.
 */
enum { GCB_KS_TETRAD = 0, GCB_KS_GLOBAL = 1 };

typedef struct {
    double a;                /* spin, 0 <= a < 1 */
    double r_in, r_out;      /* particles leaving [r_in, r_out] get GCB_FLAG_EXITED */
    int32_t kick_basis;      /* GCB_KS_TETRAD (0, default) or GCB_KS_GLOBAL; other: GCB_EINVAL */
} gcb_ks_params;

/*
 * Effective cell sizes of Eq. (volint), Sec. 3: on the (r, theta) grid,
 * dl = (integral over the cell of sqrt(gamma_rr gamma_thth - gamma_rth^2)
 * dr dtheta)^(1/2) (the proper meridional area; 4x4 Gauss-Legendre), written
 * to the device array dl_out ((n[0]-1)*(n[1]-1) doubles).  Asynchronous.
 */
gcb_status gcb_ks_cell_size(const gcb_grid_ks *g, const gcb_ks_params *kp, double *dl_out,
                            void *cuda_stream);

/*
 * n_steps coupled covariant steps (Sec. 3.2), in place: the switch of Sec. 3
 * with rho~_C = Gamma/(|q/m| B) and E/B in the local frame of the normal
 * observer; GRGCA (decomposition at x^n, half kick of u_par by D_par,
 * implicit midpoint on (R, u_par), half kick, reconstruction at R^{n+1}) or
 * GREOM (Boris half kicks over alpha dt/2, in the local frame or the global
 * basis as kp->kick_basis selects, around an implicit midpoint geodesic
 * step).  ws/out as gcb_push_sr (sorting unsupported here).
 * Errors: GCB_EINVAL for an invalid grid, spin, radii, kick_basis or
 * parameter; GCB_EUNSUPPORTED for particles that are not ndim 3 with FP64
 * positions and momenta.
 */
gcb_status gcb_push_ks(const gcb_particles *p, const gcb_grid_ks *g, const gcb_ks_params *kp,
                       const gcb_params *prm, int n_steps, void *cuda_stream, void *ws,
                       size_t ws_bytes, gcb_stats *out);

/*
 * Size of the fixed scratch array behind gcb_push_sr_noalloc (per GPU).
 */
#define GCB_NOALLOC_SCRATCH_BYTES (1u << 20)

/*
 * gcb_push_sr without a caller-provided workspace.  The paper has no
 * counterpart: this is a convenience of the library for callers that
 * cannot call cudaMalloc (a host callback or plugin hook that forbids
 * allocation, a device whose memory is held by a pool the caller does not
 * control, a loop that must not allocate after start-up).  The caller still
 * passes the particle arrays and the field records; the scratch comes from a
 * static device array of GCB_NOALLOC_SCRATCH_BYTES (1 MiB) that every GPU
 * loading the library holds until the process exits.
 *   Same arguments, behaviour and results as gcb_push_sr, minus ws/ws_bytes.
 *   Errors: as gcb_push_sr; GCB_ENOMEM (with a message) when the problem
 *   needs more scratch than the array holds -- sorting (prm->sort_every > 0)
 *   needs about 75 bytes per particle, so it fits only small problems;
 *   without sorting the need is 256 bytes.
 *   Each call looks up the array's device address with
 *   cudaGetSymbolAddress on the current device, so an address made stale by
 *   a device reset is never reused.  While its stream is capturing, a call
 *   does not look the address up: it takes the one the last call outside a
 *   capture found on that device, and fails with GCB_EINVAL if there is
 *   none, so make the first call on each device before any stream capture.
 *   All calls share the array: calls whose GPU work overlaps race on it.
 */
gcb_status gcb_push_sr_noalloc(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm,
                               int n_steps, void *cuda_stream, gcb_stats *out);

#ifdef __cplusplus
}
#endif
#endif /* GCB_H */
