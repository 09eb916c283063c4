// push_sr_f32.cu -- mixed path: FP32 fields, momenta and arithmetic; positions
// stored in FP64 or as FP32 pairs and advanced without loss (see push_sr.cuh).
#include "push_sr.cuh"

namespace gcb {

gcb_status push_step_f32(const gcb_particles *p, const gcb_particles *in, const gcb_grid *g,
                         const gcb_params *prm, cudaStream_t st, unsigned long long *stats,
                         int nsteps)
{
    if (p->pos_mode == GCB_POS_F32PAIR)
        return dispatch_push<float, 1>(p, in, g, prm, st, stats, nsteps);
    return dispatch_push<float, 0>(p, in, g, prm, st, stats, nsteps);
}

}  // namespace gcb
