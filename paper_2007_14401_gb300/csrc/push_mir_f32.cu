// push_mir_f32.cu -- mixed path with the mirror terms (gcb_params.mirror),
// kept in its own translation unit so that it compiles in parallel with the
// plain push kernels.
#include "push_sr.cuh"

namespace gcb {

gcb_status push_mir_step_f32(const gcb_particles *p, const gcb_particles *in, const gcb_grid *g,
                             const gcb_params *prm, cudaStream_t st, unsigned long long *stats)
{
    if (p->pos_mode == GCB_POS_F32PAIR)
        return dispatch_push_mir<float, 1>(p, in, g, prm, st, stats);
    return dispatch_push_mir<float, 0>(p, in, g, prm, st, stats);
}

}  // namespace gcb
