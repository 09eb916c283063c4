// push_dep_f32.cu -- mixed path with current deposition (FP32 atomics into an
// FP32 current), kept in its own translation unit so that it compiles in
// parallel with the plain push kernels.
#include "push_sr.cuh"

namespace gcb {

gcb_status push_dep_step_f32(const gcb_particles *p, const gcb_particles *in, const gcb_grid *g,
                             const gcb_params *prm, const gcb_current *cur, cudaStream_t st,
                             unsigned long long *stats)
{
    if (p->pos_mode == GCB_POS_F32PAIR)
        return dispatch_push_dep<float, 1>(p, in, g, prm, cur, st, stats);
    return dispatch_push_dep<float, 0>(p, in, g, prm, cur, st, stats);
}

}  // namespace gcb
