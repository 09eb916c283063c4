// push_dep_f64.cu -- FP64 path with current deposition (FP64 atomics).
#include "push_sr.cuh"

namespace gcb {

gcb_status push_dep_step_f64(const gcb_particles *p, const gcb_particles *in, const gcb_grid *g,
                             const gcb_params *prm, const gcb_current *cur, cudaStream_t st,
                             unsigned long long *stats)
{
    return dispatch_push_dep<double, 0>(p, in, g, prm, cur, st, stats);
}

}  // namespace gcb
