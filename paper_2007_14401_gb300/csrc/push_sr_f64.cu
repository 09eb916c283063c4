// push_sr_f64.cu -- FP64 path: FP64 fields, FP64 positions and momenta.
#include "push_sr.cuh"

namespace gcb {

gcb_status push_step_f64(const gcb_particles *p, const gcb_particles *in, const gcb_grid *g,
                         const gcb_params *prm, cudaStream_t st, unsigned long long *stats,
                         int nsteps)
{
    return dispatch_push<double, 0>(p, in, g, prm, st, stats, nsteps);
}

}  // namespace gcb
