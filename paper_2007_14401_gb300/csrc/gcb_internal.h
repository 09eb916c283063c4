// gcb_internal.h -- declarations shared by the host API (gcb_api.cu) and the
// per-precision kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gcb.h"

namespace gcb {

// Device workspace layout of gcb_push_sr (unsigned long long slots).
enum {
    ST_BORIS = 0, ST_GCA, ST_TO_GCA, ST_TO_BORIS, ST_NONCONV, ST_GCAFAIL, ST_NONFINITE,
    ST_SUM_ITER, ST_MAX_ITER, ST_EKIN,
    ST_DEPSKIP,   // particle-steps left out of the current (path too long)
    ST_DEPPIECE,  // path pieces deposited
    ST_DEPATOM,   // atomic additions into the current
    ST_EXITED,    // covariant push: particle-steps frozen after leaving [r_in, r_out]
    ST_COUNT
};
constexpr size_t kStatsBytes = 256;

void set_error(const char *fmt, ...);

// One kernel pass over all particles, reading the arrays of `in` (the
// caller's, or a sorted copy) and writing those of `p`; stats accumulate
// into the device counters `stats` (ST_* layout).  nsteps > 1 takes that many
// steps in the one launch (fused kernel).  Defined per precision.
gcb_status push_step_f64(const gcb_particles *p, const gcb_particles *in, const gcb_grid *g,
                         const gcb_params *prm, cudaStream_t st, unsigned long long *stats,
                         int nsteps = 1);
gcb_status push_step_f32(const gcb_particles *p, const gcb_particles *in, const gcb_grid *g,
                         const gcb_params *prm, cudaStream_t st, unsigned long long *stats,
                         int nsteps = 1);
// One unfused step with the mirror terms (push_mir_*.cu).
gcb_status push_mir_step_f64(const gcb_particles *p, const gcb_particles *in, const gcb_grid *g,
                             const gcb_params *prm, cudaStream_t st, unsigned long long *stats);
gcb_status push_mir_step_f32(const gcb_particles *p, const gcb_particles *in, const gcb_grid *g,
                             const gcb_params *prm, cudaStream_t st, unsigned long long *stats);
// One unfused step that also adds the step's current to cur->J (push_dep_*.cu).
gcb_status push_dep_step_f64(const gcb_particles *p, const gcb_particles *in, const gcb_grid *g,
                             const gcb_params *prm, const gcb_current *cur, cudaStream_t st,
                             unsigned long long *stats);
gcb_status push_dep_step_f32(const gcb_particles *p, const gcb_particles *in, const gcb_grid *g,
                             const gcb_params *prm, const gcb_current *cur, cudaStream_t st,
                             unsigned long long *stats);

// Adjoint (adjoint_sr.cu): one backward step for all particles whose
// pre-step state is `s`; lam[7] (x0 x1 u0 u1 u2 dxp0 dxp1) is updated in
// place, node-record adjoints are added to grad (12 doubles per node).
gcb_status adjoint_step(const gcb_particles *s, const gcb_grid *g, const gcb_params *prm,
                        void *const lam[7], double *grad, int method, cudaStream_t st);
gcb_status grad_project(const gcb_grid *g, const double *grad, const void *pat, int nmodes,
                        double *out, cudaStream_t st);
gcb_status grid_combine(const gcb_grid *g, const void *base, const void *pat, const double *amps,
                        int nmodes, cudaStream_t st);

// Covariant scheme (gcb_ks.cu).
gcb_status push_step_ks(const gcb_particles *p, const gcb_particles *in, const gcb_grid_ks *g,
                        const gcb_ks_params *kp, const gcb_params *prm, cudaStream_t st,
                        unsigned long long *stats);
gcb_status ks_cell_size(const gcb_grid_ks *g, const gcb_ks_params *kp, double *dl, cudaStream_t st);

}  // namespace gcb
