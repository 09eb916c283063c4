// push_mir_f64.cu -- FP64 path with the mirror terms (gcb_params.mirror).
#include "push_sr.cuh"

namespace gcb {

gcb_status push_mir_step_f64(const gcb_particles *p, const gcb_particles *in, const gcb_grid *g,
                             const gcb_params *prm, cudaStream_t st, unsigned long long *stats)
{
    return dispatch_push_mir<double, 0>(p, in, g, prm, st, stats);
}

}  // namespace gcb
