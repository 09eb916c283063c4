// gcb_api.cu -- host side of the C ABI declared in include/gcb.h: argument
// checks, the step loop, the workspace counters, and the small layout kernels
// (node-record packing, FP32-pair position split/join).
#include <cuda_runtime.h>

#include <vector>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "gcb.h"
#include "gcb_internal.h"
#include "sort_sr.h"

namespace gcb {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Whether the current device can dereference ptr at that address: its own
// device memory, managed memory, or pinned / registered host memory (mapped
// at the same address under unified addressing).  Checked before any launch,
// so that a pointer the GPU cannot reach is refused instead of faulting a
// kernel.  Plain (unregistered) host memory is refused even where the GPU
// could read it coherently.
static bool reachable(const void *ptr)
{
    if (!ptr) return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
    switch (at.type) {
    case cudaMemoryTypeDevice: return at.device == dev;
    case cudaMemoryTypeManaged: return true;
    case cudaMemoryTypeHost: return at.devicePointer == ptr;
    default: return false;
    }
}

// (staggered = false: the covariant state, which has no displacement arrays)
static gcb_status check_reachable(const gcb_particles *p, int nd, bool staggered = true)
{
    if (p->n == 0) return GCB_OK;
    const void *arrs[16];
    int k = 0;
    for (int d = 0; d < nd; ++d) {
        arrs[k++] = p->x[d];
        if (staggered) arrs[k++] = p->dxp[d];
        if (p->pos_mode == GCB_POS_F32PAIR) arrs[k++] = p->x_lo[d];
    }
    for (int c = 0; c < 3; ++c) arrs[k++] = p->u[c];
    arrs[k++] = p->flags;
    if (p->pid) arrs[k++] = p->pid;
    for (int i = 0; i < k; ++i)
        if (!reachable(arrs[i])) {
            set_error("a particle array (pointer %p) is not reachable from the current device "
                      "(device, managed or pinned host memory)", arrs[i]);
            return GCB_EINVAL;
        }
    return GCB_OK;
}

static gcb_status check_grid(const gcb_grid *g)
{
    if (!g) { set_error("grid is NULL"); return GCB_EINVAL; }
    if (g->ndim != 2 && g->ndim != 3) { set_error("grid ndim must be 2 or 3"); return GCB_EINVAL; }
    if (g->dtype != GCB_F32 && g->dtype != GCB_F64) { set_error("grid dtype"); return GCB_EINVAL; }
    int64_t nn = 1;
    for (int d = 0; d < 3; ++d) {
        int64_t n = g->n[d];
        if (d >= g->ndim && n != 1) { set_error("grid n[%d] must be 1 in %dD", d, g->ndim); return GCB_EINVAL; }
        if (d < g->ndim && (n < 2 || !(g->dx[d] > 0.0))) {
            set_error("grid axis %d needs n >= 2 and dx > 0", d);
            return GCB_EINVAL;
        }
        nn *= n;
    }
    if (nn >= (int64_t(1) << 31)) { set_error("grid has too many nodes (>= 2^31)"); return GCB_EUNSUPPORTED; }
    if (g->stride != gcb_grid_stride(g->ndim, g->dtype, g->has_grad)) {
        set_error("grid stride %d does not match gcb_grid_stride", g->stride);
        return GCB_EINVAL;
    }
    if (!g->rec || !aligned(g->rec, 16)) { set_error("grid records NULL or not 16-byte aligned"); return GCB_EINVAL; }
    return GCB_OK;
}

}  // namespace gcb

using namespace gcb;

extern "C" {

int gcb_version(void) { return 100; }

const char *gcb_status_string(gcb_status s)
{
    switch (s) {
    case GCB_OK: return "GCB_OK";
    case GCB_EINVAL: return "GCB_EINVAL";
    case GCB_ECUDA: return "GCB_ECUDA";
    case GCB_EUNSUPPORTED: return "GCB_EUNSUPPORTED";
    case GCB_ENOMEM: return "GCB_ENOMEM";
    }
    return "GCB_UNKNOWN";
}

const char *gcb_last_error(void) { return g_err; }

int32_t gcb_grid_stride(int32_t ndim, int32_t dtype, int32_t has_grad)
{
    if ((ndim != 2 && ndim != 3) || (dtype != GCB_F32 && dtype != GCB_F64)) return 0;
    int need = 6 + (has_grad ? 3 * ndim : 0);
    int chunk = dtype == GCB_F32 ? 4 : 2;  // elements per 16 bytes
    return (need + chunk - 1) / chunk * chunk;
}

size_t gcb_workspace_bytes(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm)
{
    if (!p || !g || !prm || prm->sort_every <= 0 || p->n <= 0) return kStatsBytes;
    SortPlan pl;
    if (!sort_plan(p, g, prm, pl)) return kStatsBytes;
    return pl.total;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// layout kernels
// ---------------------------------------------------------------------------
struct PackSrc {
    const double *c[15];
};

template <typename T>
__global__ void k_pack(T *rec, int stride, int ncomp, int64_t nnodes, PackSrc src)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnodes;
         i += (int64_t)gridDim.x * blockDim.x) {
        T *r = rec + i * stride;
        for (int c = 0; c < stride; ++c) r[c] = c < ncomp ? (T)src.c[c][i] : T(0);
    }
}

__global__ void k_split(int64_t n, const double *x, float *hi, float *lo)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = x[i];
        float h = (float)v;
        hi[i] = h;
        lo[i] = (float)(v - (double)h);
    }
}

__global__ void k_join(int64_t n, const float *hi, const float *lo, double *x)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = (double)hi[i] + (double)lo[i];
}

static int grid_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

static gcb_status launch_check(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: %s", what, cudaGetErrorString(e));
        return GCB_ECUDA;
    }
    return GCB_OK;
}

extern "C" {

gcb_status gcb_grid_pack(const gcb_grid *g, const double *const *comp, void *cuda_stream)
{
    gcb_status s = check_grid(g);
    if (s != GCB_OK) return s;
    if (!comp) { set_error("component list is NULL"); return GCB_EINVAL; }
    int ncomp = 6 + (g->has_grad ? 3 * g->ndim : 0);
    PackSrc src;
    memset(&src, 0, sizeof(src));
    for (int c = 0; c < ncomp; ++c) {
        if (!comp[c] || !aligned(comp[c], 8)) { set_error("component %d NULL or misaligned", c); return GCB_EINVAL; }
        src.c[c] = comp[c];
    }
    int64_t nn = g->n[0] * g->n[1] * g->n[2];
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (g->dtype == GCB_F32)
        k_pack<float><<<grid_for(nn), 256, 0, st>>>((float *)g->rec, g->stride, ncomp, nn, src);
    else
        k_pack<double><<<grid_for(nn), 256, 0, st>>>((double *)g->rec, g->stride, ncomp, nn, src);
    return launch_check("gcb_grid_pack");
}

gcb_status gcb_pos_split(int64_t n, const double *x, float *hi, float *lo, void *cuda_stream)
{
    if (n < 0 || (n > 0 && (!x || !hi || !lo))) { set_error("gcb_pos_split: bad arguments"); return GCB_EINVAL; }
    if (n == 0) return GCB_OK;
    if (!reachable(x) || !reachable(hi) || !reachable(lo)) {
        set_error("gcb_pos_split: an array is not reachable from the current device");
        return GCB_EINVAL;
    }
    k_split<<<grid_for(n), 256, 0, (cudaStream_t)cuda_stream>>>(n, x, hi, lo);
    return launch_check("gcb_pos_split");
}

gcb_status gcb_pos_join(int64_t n, const float *hi, const float *lo, double *x, void *cuda_stream)
{
    if (n < 0 || (n > 0 && (!x || !hi || !lo))) { set_error("gcb_pos_join: bad arguments"); return GCB_EINVAL; }
    if (n == 0) return GCB_OK;
    if (!reachable(x) || !reachable(hi) || !reachable(lo)) {
        set_error("gcb_pos_join: an array is not reachable from the current device");
        return GCB_EINVAL;
    }
    k_join<<<grid_for(n), 256, 0, (cudaStream_t)cuda_stream>>>(n, hi, lo, x);
    return launch_check("gcb_pos_join");
}

// Copy the device counters to `out` and the deposition's to `dst`
// (synchronizing the stream) when either is non-NULL.
static gcb_status read_stats(const unsigned long long *stats, cudaStream_t st, gcb_stats *out,
                             gcb_deposit_stats *dst = nullptr)
{
    if (!out && !dst) return GCB_OK;
    unsigned long long h[ST_COUNT];
    if (cudaMemcpyAsync(h, stats, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("stats readback: %s", cudaGetErrorString(cudaGetLastError()));
        return GCB_ECUDA;
    }
    if (dst) {
        dst->n_skipped = (int64_t)h[ST_DEPSKIP];
        dst->n_pieces = (int64_t)h[ST_DEPPIECE];
        dst->n_atomics = (int64_t)h[ST_DEPATOM];
    }
    if (!out) return GCB_OK;
    out->n_boris = (int64_t)h[ST_BORIS];
    out->n_gca = (int64_t)h[ST_GCA];
    out->n_to_gca = (int64_t)h[ST_TO_GCA];
    out->n_to_boris = (int64_t)h[ST_TO_BORIS];
    out->n_nonconv = (int64_t)h[ST_NONCONV];
    out->n_gcafail = (int64_t)h[ST_GCAFAIL];
    out->n_nonfinite = (int64_t)h[ST_NONFINITE];
    out->sum_iter = (int64_t)h[ST_SUM_ITER];
    out->max_iter = (int64_t)h[ST_MAX_ITER];
    double e;
    memcpy(&e, &h[ST_EKIN], sizeof(e));
    out->sum_ekin = e;
    out->n_exited = (int64_t)h[ST_EXITED];
    return GCB_OK;
}

static gcb_status check_problem(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm)
{
    gcb_status s = check_grid(g);
    if (s != GCB_OK) return s;
    if (!p || !prm) { set_error("particles or params NULL"); return GCB_EINVAL; }
    if (p->n < 0) { set_error("particle count < 0"); return GCB_EINVAL; }
    if (p->ndim != g->ndim) { set_error("particle ndim %d != grid ndim %d", p->ndim, g->ndim); return GCB_EINVAL; }
    if (!(prm->c > 0) || !(prm->dt > 0) || !(prm->f_rho > 0) || !(prm->f_E > 0) || !(prm->dl > 0)) {
        set_error("c, dt, f_rho, f_E and dl must be > 0");
        return GCB_EINVAL;
    }
    if (prm->curvature != 0 && prm->curvature != 1) { set_error("curvature must be 0 or 1"); return GCB_EINVAL; }
    if (prm->mu_mode != GCB_MU_CONSERVE && prm->mu_mode != GCB_UPERP_CONSERVE) { set_error("mu_mode"); return GCB_EINVAL; }
    if (prm->grad_mode != GCB_GRAD_DW && prm->grad_mode != GCB_GRAD_GRID) { set_error("grad_mode"); return GCB_EINVAL; }
    if (prm->grad_mode == GCB_GRAD_GRID && !g->has_grad) { set_error("grad_mode GRID needs gradient records"); return GCB_EINVAL; }
    if (prm->force < GCB_FORCE_NONE || prm->force > GCB_FORCE_GCA) { set_error("force"); return GCB_EINVAL; }
    if (prm->gca_max_iter < 1 || prm->gca_max_iter > 1000 || prm->gca_fixed_iters < 0 ||
        prm->gca_fixed_iters > 1000) {
        set_error("gca_max_iter must be in [1, 1000] and gca_fixed_iters in [0, 1000]");
        return GCB_EINVAL;
    }
    if (!(prm->gca_tol >= 0)) { set_error("gca_tol must be >= 0"); return GCB_EINVAL; }
    if (prm->drift_frame != GCB_FRAME_SIMPLE && prm->drift_frame != GCB_FRAME_BT) {
        set_error("drift_frame must be GCB_FRAME_SIMPLE or GCB_FRAME_BT");
        return GCB_EINVAL;
    }
    if (prm->gyro_phase != GCB_PHASE_KEEP && prm->gyro_phase != GCB_PHASE_EVOLVE) {
        set_error("gyro_phase must be GCB_PHASE_KEEP or GCB_PHASE_EVOLVE");
        return GCB_EINVAL;
    }
    if (prm->drift_frame == GCB_FRAME_BT && prm->fuse_steps > 1) {
        set_error("drift_frame GCB_FRAME_BT runs one step per launch (fuse_steps <= 1)");
        return GCB_EUNSUPPORTED;
    }
    if (prm->mirror != GCB_MIRROR_OFF && prm->mirror != GCB_MIRROR_ON) {
        set_error("mirror must be GCB_MIRROR_OFF or GCB_MIRROR_ON");
        return GCB_EINVAL;
    }
    if (prm->mirror == GCB_MIRROR_ON &&
        (prm->fuse_steps > 1 || prm->drift_frame != GCB_FRAME_SIMPLE)) {
        set_error("the mirror terms run one step per launch (fuse_steps <= 1) in the "
                  "simplified drift frame");
        return GCB_EUNSUPPORTED;
    }
    if (prm->sort_every < 0 || prm->sort_tile[0] < 0 || prm->sort_tile[1] < 0 ||
        prm->sort_tile[2] < 0 || prm->step_index < 0) {
        set_error("sort_every, sort_tile and step_index must be >= 0");
        return GCB_EINVAL;
    }

    bool fp64 = p->mom_dtype == GCB_F64;
    if (fp64) {
        if (p->pos_mode != GCB_POS_F64 || g->dtype != GCB_F64) {
            set_error("FP64 momenta need GCB_POS_F64 positions and an F64 grid");
            return GCB_EUNSUPPORTED;
        }
    } else if (p->mom_dtype == GCB_F32) {
        if (g->dtype != GCB_F32) { set_error("FP32 momenta need an F32 grid"); return GCB_EUNSUPPORTED; }
        if (p->pos_mode != GCB_POS_F64 && p->pos_mode != GCB_POS_F32PAIR) { set_error("pos_mode"); return GCB_EINVAL; }
        if (p->pos_mode == GCB_POS_F32PAIR) {
            for (int d = 0; d < g->ndim; ++d) {
                double L = (double)g->n[d] * g->dx[d];
                if ((double)(float)L != L || (double)(float)g->dx[d] != g->dx[d]) {
                    set_error("FP32-pair positions need n*dx and dx exact in float");
                    return GCB_EUNSUPPORTED;
                }
            }
        }
    } else {
        set_error("mom_dtype");
        return GCB_EINVAL;
    }
    if (p->n > 0) {
        size_t me = fp64 ? 8 : 4;
        size_t pe = p->pos_mode == GCB_POS_F64 ? 8 : 4;
        for (int d = 0; d < p->ndim; ++d) {
            if (!p->x[d] || !aligned(p->x[d], pe) || !p->dxp[d] || !aligned(p->dxp[d], me)) {
                set_error("x[%d] or dxp[%d] NULL or misaligned", d, d);
                return GCB_EINVAL;
            }
            if (p->pos_mode == GCB_POS_F32PAIR && (!p->x_lo[d] || !aligned(p->x_lo[d], 4))) {
                set_error("x_lo[%d] NULL or misaligned", d);
                return GCB_EINVAL;
            }
        }
        for (int k = 0; k < 3; ++k)
            if (!p->u[k] || !aligned(p->u[k], me)) { set_error("u[%d] NULL or misaligned", k); return GCB_EINVAL; }
        if (!p->flags) { set_error("flags NULL"); return GCB_EINVAL; }
        if (p->pid && !aligned(p->pid, 8)) { set_error("pid misaligned"); return GCB_EINVAL; }
        if (!reachable(g->rec)) {
            set_error("the grid records are not reachable from the current device");
            return GCB_EINVAL;
        }
        return check_reachable(p, p->ndim);
    }
    return GCB_OK;
}

// Sort into the workspace; `q` becomes the view of the sorted copy.
static gcb_status sort_step(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm,
                            cudaStream_t st, void *ws, size_t ws_bytes, gcb_particles &q,
                            SortPlan &pl, SortedView &v)
{
    if (p->n >= (int64_t(1) << 31)) { set_error("sorting needs n < 2^31"); return GCB_EUNSUPPORTED; }
    if (!sort_plan(p, g, prm, pl)) { set_error("too many sort tiles"); return GCB_EUNSUPPORTED; }
    if (ws_bytes < pl.total) {
        set_error("workspace too small for sorting (%zu < %zu bytes)", ws_bytes, pl.total);
        return GCB_ENOMEM;
    }
    gcb_status s = sort_into_workspace(p, g, pl, st, (uint8_t *)ws, v);
    if (s != GCB_OK) return s;
    sorted_particles(p, g->ndim, v, q);
    return GCB_OK;
}

gcb_status gcb_sort_sr(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm,
                       void *cuda_stream, void *ws, size_t ws_bytes)
{
    g_err[0] = 0;
    gcb_status s = check_problem(p, g, prm);
    if (s != GCB_OK) return s;
    if (!ws || !aligned(ws, 256)) { set_error("workspace NULL or not 256-byte aligned"); return GCB_EINVAL; }
    if (p->n == 0) return GCB_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    gcb_particles q;
    SortPlan pl;
    SortedView v;
    s = sort_step(p, g, prm, st, ws, ws_bytes, q, pl, v);
    if (s != GCB_OK) return s;
    return copy_back(p, g, pl, v, st);
}

static gcb_status check_ks(const gcb_grid_ks *gk, const gcb_ks_params *kp)
{
    if (!gk || !kp) { set_error("grid or spacetime parameters NULL"); return GCB_EINVAL; }
    gcb_status s = check_grid(&gk->g);
    if (s != GCB_OK) return s;
    const gcb_grid *g = &gk->g;
    if (g->ndim != 2 || g->has_grad) { set_error("Kerr-Schild grid: ndim 2, no gradient records"); return GCB_EINVAL; }
    if (fabs(g->dx[1] * (double)(g->n[1] - 1) - 3.141592653589793) > 1e-9) {
        set_error("Kerr-Schild grid: theta nodes must span [0, pi]");
        return GCB_EINVAL;
    }
    if (!(kp->a >= 0.0 && kp->a < 1.0) || !(kp->r_in > 0.0) || !(kp->r_out > kp->r_in)) {
        set_error("need 0 <= a < 1 and 0 < r_in < r_out");
        return GCB_EINVAL;
    }
    if (kp->kick_basis != GCB_KS_TETRAD && kp->kick_basis != GCB_KS_GLOBAL) {
        set_error("kick_basis must be GCB_KS_TETRAD or GCB_KS_GLOBAL");
        return GCB_EINVAL;
    }
    return GCB_OK;
}

gcb_status gcb_ks_cell_size(const gcb_grid_ks *g, const gcb_ks_params *kp, double *dl_out,
                            void *cuda_stream)
{
    g_err[0] = 0;
    gcb_status s = check_ks(g, kp);
    if (s != GCB_OK) return s;
    if (!dl_out || !aligned(dl_out, 8)) { set_error("dl_out NULL or misaligned"); return GCB_EINVAL; }
    return ks_cell_size(g, kp, dl_out, (cudaStream_t)cuda_stream);
}

gcb_status gcb_push_ks(const gcb_particles *p, const gcb_grid_ks *gk, const gcb_ks_params *kp,
                       const gcb_params *prm, int n_steps, void *cuda_stream, void *ws,
                       size_t ws_bytes, gcb_stats *out)
{
    g_err[0] = 0;
    gcb_status s = check_ks(gk, kp);
    if (s != GCB_OK) return s;
    if (!p || !prm) { set_error("particles or params NULL"); return GCB_EINVAL; }
    if (n_steps < 0 || p->n < 0) { set_error("negative n_steps or particle count"); return GCB_EINVAL; }
    if (p->ndim != 3 || p->pos_mode != GCB_POS_F64 || p->mom_dtype != GCB_F64) {
        set_error("Kerr-Schild particles: ndim 3, FP64 positions and momenta");
        return GCB_EUNSUPPORTED;
    }
    if (prm->c != 1.0) { set_error("the covariant scheme uses c = 1"); return GCB_EINVAL; }
    if (prm->drift_frame != GCB_FRAME_SIMPLE || prm->gyro_phase != GCB_PHASE_KEEP ||
        prm->mirror != GCB_MIRROR_OFF) {
        set_error("the covariant scheme uses the simplified drift frame, keeps the "
                  "gyration direction and has no mirror terms");
        return GCB_EUNSUPPORTED;
    }
    if (!(prm->dt > 0) || !(prm->f_rho > 0) || !(prm->f_E > 0)) { set_error("dt, f_rho, f_E must be > 0"); return GCB_EINVAL; }
    if (prm->mu_mode != GCB_MU_CONSERVE && prm->mu_mode != GCB_UPERP_CONSERVE) { set_error("mu_mode"); return GCB_EINVAL; }
    if (prm->force < GCB_FORCE_NONE || prm->force > GCB_FORCE_GCA) { set_error("force"); return GCB_EINVAL; }
    if (prm->gca_max_iter < 1 || prm->gca_max_iter > 1000 || prm->gca_fixed_iters < 0 ||
        prm->gca_fixed_iters > 1000 || !(prm->gca_tol >= 0)) {
        set_error("iteration bounds");
        return GCB_EINVAL;
    }
    if (prm->sort_every != 0) { set_error("sorting is not supported by the covariant scheme"); return GCB_EUNSUPPORTED; }
    if (!gk->dl || !aligned(gk->dl, 8)) { set_error("cell-size table NULL or misaligned"); return GCB_EINVAL; }
    if (p->n > 0) {
        for (int k = 0; k < 3; ++k)
            if (!p->x[k] || !p->u[k] || !aligned(p->x[k], 8) || !aligned(p->u[k], 8)) {
                set_error("x or u NULL or misaligned");
                return GCB_EINVAL;
            }
        if (!p->flags) { set_error("flags NULL"); return GCB_EINVAL; }
        if (p->pid && !aligned(p->pid, 8)) { set_error("pid misaligned"); return GCB_EINVAL; }
        s = check_reachable(p, 3, false);
        if (s != GCB_OK) return s;
    }
    if (!ws || !aligned(ws, 256)) { set_error("workspace NULL or not 256-byte aligned"); return GCB_EINVAL; }
    if (ws_bytes < kStatsBytes) { set_error("workspace too small"); return GCB_ENOMEM; }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned long long *stats = (unsigned long long *)ws;
    if (cudaMemsetAsync(stats, 0, kStatsBytes, st) != cudaSuccess) {
        set_error("cudaMemsetAsync: %s", cudaGetErrorString(cudaGetLastError()));
        return GCB_ECUDA;
    }
    for (int step = 0; step < n_steps; ++step) {
        s = push_step_ks(p, p, gk, kp, prm, st, stats);
        if (s != GCB_OK) return s;
    }
    return read_stats(stats, st, out);
}

// The current of gcb_push_deposit_sr: types, alignment and reachability of
// its arrays, and the options the deposition supports.
static gcb_status check_current(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm,
                                const gcb_current *cur)
{
    if (!cur) { set_error("current NULL"); return GCB_EINVAL; }
    if (cur->dtype != p->mom_dtype || cur->reserved != 0) {
        set_error("current dtype must equal the particles' mom_dtype (reserved 0)");
        return GCB_EINVAL;
    }
    for (int k = 0; k < 4; ++k)
        if (!isfinite(cur->q[k])) { set_error("non-finite species charge"); return GCB_EINVAL; }
    const size_t es = cur->dtype == GCB_F64 ? 8 : 4;
    for (int k = 0; k < 3; ++k) {
        if (!cur->J[k] || !aligned(cur->J[k], es) || !reachable(cur->J[k])) {
            set_error("current component %d NULL, misaligned or not device-reachable", k);
            return GCB_EINVAL;
        }
    }
    if (cur->w && p->n > 0 && (!aligned(cur->w, es) || !reachable(cur->w))) {
        set_error("weights misaligned or not device-reachable");
        return GCB_EINVAL;
    }
    if (cur->w && prm->sort_every > 0) {
        set_error("per-particle weights are not permuted by sorting: sort_every must be 0");
        return GCB_EUNSUPPORTED;
    }
    if (prm->fuse_steps > 1) {
        set_error("deposition: unfused steps only (fuse_steps <= 1)");
        return GCB_EUNSUPPORTED;
    }
    if (g->n[0] * g->n[1] * g->n[2] >= ((int64_t)1 << 31)) {
        set_error("deposition: the grid must have fewer than 2^31 nodes");
        return GCB_EUNSUPPORTED;
    }
    return GCB_OK;
}

static gcb_status push_sr_impl(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm,
                               const gcb_current *cur, int n_steps, void *cuda_stream, void *ws,
                               size_t ws_bytes, gcb_stats *out, gcb_deposit_stats *dst);

gcb_status gcb_push_sr(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm,
                       int n_steps, void *cuda_stream, void *ws, size_t ws_bytes, gcb_stats *out)
{
    return push_sr_impl(p, g, prm, nullptr, n_steps, cuda_stream, ws, ws_bytes, out, nullptr);
}

gcb_status gcb_push_deposit_sr(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm,
                               const gcb_current *cur, int n_steps, void *cuda_stream, void *ws,
                               size_t ws_bytes, gcb_stats *out, gcb_deposit_stats *dst)
{
    g_err[0] = 0;
    if (!cur) { set_error("current NULL"); return GCB_EINVAL; }
    return push_sr_impl(p, g, prm, cur, n_steps, cuda_stream, ws, ws_bytes, out, dst);
}

static gcb_status push_sr_impl(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm,
                               const gcb_current *cur, int n_steps, void *cuda_stream, void *ws,
                               size_t ws_bytes, gcb_stats *out, gcb_deposit_stats *dst)
{
    g_err[0] = 0;
    gcb_status s = check_problem(p, g, prm);
    if (s != GCB_OK) return s;
    if (cur) {
        s = check_current(p, g, prm, cur);
        if (s != GCB_OK) return s;
    }
    if (n_steps < 0) { set_error("n_steps < 0"); return GCB_EINVAL; }
    if (!ws || !aligned(ws, 256)) { set_error("workspace NULL or not 256-byte aligned"); return GCB_EINVAL; }
    if (ws_bytes < kStatsBytes) { set_error("workspace too small"); return GCB_ENOMEM; }
    const bool fp64 = p->mom_dtype == GCB_F64;

    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned long long *stats = (unsigned long long *)ws;
    if (cudaMemsetAsync(stats, 0, kStatsBytes, st) != cudaSuccess) {
        set_error("cudaMemsetAsync: %s", cudaGetErrorString(cudaGetLastError()));
        return GCB_ECUDA;
    }
    for (int step = 0; step < n_steps;) {
        const gcb_particles *in = p;
        gcb_particles q;
        const int64_t gstep = prm->step_index + step;
        if (prm->sort_every > 0 && p->n > 0 && gstep % prm->sort_every == 0) {
            SortPlan pl;
            SortedView v;
            s = sort_step(p, g, prm, st, ws, ws_bytes, q, pl, v);
            if (s != GCB_OK) return s;
            in = &q;
        }
        // steps fused into this launch: at most fuse_steps, none past the
        // next sort
        int k = 1;
        if (prm->fuse_steps > 1) {
            k = prm->fuse_steps < n_steps - step ? prm->fuse_steps : n_steps - step;
            if (prm->sort_every > 0) {
                const int to_sort = prm->sort_every - (int)(gstep % prm->sort_every);
                k = k < to_sort ? k : to_sort;
            }
        }
        if (cur)
            s = fp64 ? push_dep_step_f64(p, in, g, prm, cur, st, stats)
                     : push_dep_step_f32(p, in, g, prm, cur, st, stats);
        else if (prm->mirror == GCB_MIRROR_ON)
            s = fp64 ? push_mir_step_f64(p, in, g, prm, st, stats)
                     : push_mir_step_f32(p, in, g, prm, st, stats);
        else
            s = fp64 ? push_step_f64(p, in, g, prm, st, stats, k)
                     : push_step_f32(p, in, g, prm, st, stats, k);
        if (s != GCB_OK) return s;
        step += k;
    }
    return read_stats(stats, st, out, dst);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// adjoint driver: checkpoints, segment recomputation, backward sweep
// ---------------------------------------------------------------------------
namespace {

size_t a256(size_t v) { return (v + 255) / 256 * 256; }

// bytes of one state set and the view of a set carved at `base`
size_t state_set_bytes(const gcb_particles *p, int nd)
{
    const size_t n = (size_t)p->n;
    const size_t pe = p->pos_mode == GCB_POS_F64 ? 8 : 4, me = p->mom_dtype == GCB_F64 ? 8 : 4;
    size_t b = nd * a256(n * pe) + 3 * a256(n * me) + nd * a256(n * me) + a256(n);
    if (p->pos_mode == GCB_POS_F32PAIR) b += nd * a256(n * 4);
    return b;
}

gcb_particles state_view(const gcb_particles *p, int nd, uint8_t *base)
{
    gcb_particles q = *p;
    const size_t n = (size_t)p->n;
    const size_t pe = p->pos_mode == GCB_POS_F64 ? 8 : 4, me = p->mom_dtype == GCB_F64 ? 8 : 4;
    size_t off = 0;
    for (int d = 0; d < 3; ++d) { q.x[d] = q.x_lo[d] = q.u[d] = q.dxp[d] = nullptr; }
    for (int d = 0; d < nd; ++d) { q.x[d] = base + off; off += a256(n * pe); }
    if (p->pos_mode == GCB_POS_F32PAIR)
        for (int d = 0; d < nd; ++d) { q.x_lo[d] = base + off; off += a256(n * 4); }
    for (int k = 0; k < 3; ++k) { q.u[k] = base + off; off += a256(n * me); }
    for (int d = 0; d < nd; ++d) { q.dxp[d] = base + off; off += a256(n * me); }
    q.flags = base + off;
    q.pid = nullptr;
    return q;
}

gcb_status copy_state(const gcb_particles *dst, const gcb_particles *src, int nd, cudaStream_t st)
{
    const size_t n = (size_t)src->n;
    const size_t pe = src->pos_mode == GCB_POS_F64 ? 8 : 4, me = src->mom_dtype == GCB_F64 ? 8 : 4;
    bool ok = true;
    for (int d = 0; d < nd; ++d) {
        ok = ok && cudaMemcpyAsync(dst->x[d], src->x[d], n * pe, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
        if (src->pos_mode == GCB_POS_F32PAIR)
            ok = ok && cudaMemcpyAsync(dst->x_lo[d], src->x_lo[d], n * 4, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(dst->dxp[d], src->dxp[d], n * me, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    }
    for (int k = 0; k < 3; ++k)
        ok = ok && cudaMemcpyAsync(dst->u[k], src->u[k], n * me, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(dst->flags, src->flags, n, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    if (!ok) {
        set_error("state copy: %s", cudaGetErrorString(cudaGetLastError()));
        return GCB_ECUDA;
    }
    return GCB_OK;
}

}  // namespace

// Layout of the adjoint workspace (256-byte aligned sections):
//   counters | checkpoint states (nck) | segment states (ckpt_every - 1) |
//   2 scratch states | and with sorting (prm->sort_every > 0): the sort's
//   own workspace | the sort's inverse permutation at each checkpoint |
//   2 composed orders | 7 scratch adjoint arrays | a scratch id array.
struct AdjLayout {
    int nck;
    size_t S;                   // bytes of one state set
    size_t ck, seg, tmp;        // offsets of the state sets
    bool sort;
    size_t sortws, sortws_bytes, inv, ordA, ordB, lamt, pidt;
    size_t total;
};

static bool adj_layout(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm,
                       int n_steps, int ckpt_every, AdjLayout &L)
{
    L.nck = (n_steps + ckpt_every - 1) / ckpt_every;
    L.S = state_set_bytes(p, g->ndim);
    size_t o = kStatsBytes;
    L.ck = o;
    o += (size_t)L.nck * L.S;
    L.seg = o;
    o += (size_t)(ckpt_every - 1) * L.S;
    L.tmp = o;
    o += 2 * L.S;
    L.sort = prm && prm->sort_every > 0 && p->n > 0;
    L.sortws = L.sortws_bytes = L.inv = L.ordA = L.ordB = L.lamt = L.pidt = 0;
    if (L.sort) {
        SortPlan pl;
        if (!sort_plan(p, g, prm, pl)) return false;
        const size_t n = (size_t)p->n, me = p->mom_dtype == GCB_F64 ? 8 : 4;
        L.sortws = o;
        L.sortws_bytes = a256(pl.total);
        o += L.sortws_bytes;
        L.inv = o;
        o += (size_t)L.nck * a256(4 * n);
        L.ordA = o;
        o += a256(4 * n);
        L.ordB = o;
        o += a256(4 * n);
        L.lamt = o;
        o += 7 * a256(me * n);
        L.pidt = o;
        o += a256(8 * n);
    }
    L.total = o;
    return true;
}

// the caller-visible arrays of a particle set (with ids when present)
static int particle_arrays(const gcb_particles *p, int nd, void **arr, int *es)
{
    const int pe = p->pos_mode == GCB_POS_F64 ? 8 : 4, me = p->mom_dtype == GCB_F64 ? 8 : 4;
    int k = 0;
    for (int d = 0; d < nd; ++d) { arr[k] = p->x[d]; es[k++] = pe; }
    if (p->pos_mode == GCB_POS_F32PAIR)
        for (int d = 0; d < nd; ++d) { arr[k] = p->x_lo[d]; es[k++] = 4; }
    for (int c = 0; c < 3; ++c) { arr[k] = p->u[c]; es[k++] = me; }
    for (int d = 0; d < nd; ++d) { arr[k] = p->dxp[d]; es[k++] = me; }
    arr[k] = p->flags;
    es[k++] = 1;
    if (p->pid) { arr[k] = p->pid; es[k++] = 8; }
    return k;
}

// Sort `cur` by cell into the sort workspace, store the sorted state as
// checkpoint c and the sort's inverse permutation (new index -> old index)
// as inv_c; `q` is the sorted copy's view.
static gcb_status sort_checkpoint(const gcb_particles *cur, const gcb_grid *g, const gcb_params *prm,
                                  const AdjLayout &L, uint8_t *w, int c, cudaStream_t st,
                                  gcb_particles &q)
{
    SortPlan pl;
    SortedView v;
    gcb_status s = sort_step(cur, g, prm, st, w + L.sortws, L.sortws_bytes, q, pl, v);
    if (s != GCB_OK) return s;
    const size_t n4 = 4 * (size_t)cur->n;
    if (cudaMemcpyAsync(w + L.inv + (size_t)c * a256(n4), w + L.sortws + pl.off_inv, n4,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        set_error("cudaMemcpyAsync: %s", cudaGetErrorString(cudaGetLastError()));
        return GCB_ECUDA;
    }
    gcb_particles ckv = state_view(cur, g->ndim, w + L.ck + (size_t)c * L.S);
    return copy_state(&ckv, &q, g->ndim, st);
}

// order[j] = original index of the particle at position j of checkpoint c's
// order: inv_0 composed with inv_1 .. inv_c.  Returns the buffer holding it.
static int32_t *compose_order(int64_t n, const AdjLayout &L, uint8_t *w, int c, cudaStream_t st,
                              gcb_status &s)
{
    const size_t n4 = 4 * (size_t)n;
    int32_t *cur = (int32_t *)(w + L.ordA), *nxt = (int32_t *)(w + L.ordB);
    s = GCB_OK;
    if (cudaMemcpyAsync(cur, w + L.inv, n4, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        set_error("cudaMemcpyAsync: %s", cudaGetErrorString(cudaGetLastError()));
        s = GCB_ECUDA;
        return nullptr;
    }
    for (int k = 1; k <= c; ++k) {
        // nxt[j] = cur[inv_k[j]]
        void *dst[1] = {nxt};
        const void *src[1] = {cur};
        const int es[1] = {4};
        s = permute_arrays(n, 1, dst, src, es, (const int32_t *)(w + L.inv + (size_t)k * a256(n4)),
                           false, st);
        if (s != GCB_OK) return nullptr;
        int32_t *t = cur;
        cur = nxt;
        nxt = t;
    }
    return cur;
}

// permute the 7 adjoint arrays through the scratch arrays: lam[j] =
// lam[idx[j]] (gather) or lam[idx[j]] = lam[j] (scatter)
static gcb_status permute_lam(int64_t n, int me, void *const *lam, const AdjLayout &L, uint8_t *w,
                              const int32_t *idx, bool scatter, cudaStream_t st)
{
    void *tmp[7];
    int es[7];
    for (int k = 0; k < 7; ++k) {
        tmp[k] = w + L.lamt + (size_t)k * a256((size_t)me * n);
        es[k] = me;
        if (cudaMemcpyAsync(tmp[k], lam[k], (size_t)me * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
            set_error("cudaMemcpyAsync: %s", cudaGetErrorString(cudaGetLastError()));
            return GCB_ECUDA;
        }
    }
    return permute_arrays(n, 7, (void *const *)lam, (const void *const *)tmp, es, idx, scatter, st);
}

extern "C" {

size_t gcb_adjoint_workspace_bytes(const gcb_particles *p, const gcb_grid *g,
                                   const gcb_params *prm, int n_steps, int ckpt_every)
{
    if (!p || !g || n_steps < 1 || ckpt_every < 1 || p->n < 0) return 0;
    AdjLayout L;
    if (!adj_layout(p, g, prm, n_steps, ckpt_every, L)) return 0;
    return L.total;
}

}  // extern "C"

// checks shared by the adjoint's entry points
static gcb_status check_adjoint(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm,
                                int n_steps, int ckpt_every, const void *ws, size_t ws_bytes)
{
    gcb_status s = check_problem(p, g, prm);
    if (s != GCB_OK) return s;
    if (g->ndim != 2 || !g->has_grad || prm->grad_mode != GCB_GRAD_GRID) {
        set_error("the adjoint supports 2D grids with gradient records (grad_mode GRID)");
        return GCB_EUNSUPPORTED;
    }
    if (prm->drift_frame != GCB_FRAME_SIMPLE || prm->gyro_phase != GCB_PHASE_KEEP ||
        prm->mirror != GCB_MIRROR_OFF) {
        set_error("the adjoint differentiates the simplified drift frame with the gyration "
                  "direction kept and without mirror terms only");
        return GCB_EUNSUPPORTED;
    }
    if (n_steps < 1 || ckpt_every < 1) { set_error("n_steps and ckpt_every must be >= 1"); return GCB_EINVAL; }
    if (prm->gca_max_iter > GCB_ADJOINT_MAX_ITER || prm->gca_fixed_iters > GCB_ADJOINT_MAX_ITER) {
        set_error("the adjoint records at most %d fixed-point iterations per step", GCB_ADJOINT_MAX_ITER);
        return GCB_EUNSUPPORTED;
    }
    if (p->n >= (int64_t(1) << 31)) { set_error("the adjoint needs n < 2^31"); return GCB_EUNSUPPORTED; }
    const size_t need = gcb_adjoint_workspace_bytes(p, g, prm, n_steps, ckpt_every);
    if (need == 0) { set_error("too many sort tiles"); return GCB_EUNSUPPORTED; }
    if (!ws || !aligned(ws, 256)) { set_error("workspace NULL or not 256-byte aligned"); return GCB_EINVAL; }
    if (ws_bytes < need) { set_error("workspace too small (%zu < %zu bytes)", ws_bytes, need); return GCB_ENOMEM; }
    return GCB_OK;
}

extern "C" {

gcb_status gcb_push_sr_ckpt(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm0,
                            int n_steps, int ckpt_every, void *cuda_stream, void *ws,
                            size_t ws_bytes, gcb_stats *out)
{
    g_err[0] = 0;
    gcb_status s = check_adjoint(p, g, prm0, n_steps, ckpt_every, ws, ws_bytes);
    if (s != GCB_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    gcb_params prm = *prm0;
    prm.sort_every = 0;          // the pushes themselves do not sort
    prm.fuse_steps = 0;
    const int nd = g->ndim;
    AdjLayout L;
    adj_layout(p, g, prm0, n_steps, ckpt_every, L);
    uint8_t *w = (uint8_t *)ws;
    unsigned long long *stats = (unsigned long long *)ws;
    if (cudaMemsetAsync(stats, 0, kStatsBytes, st) != cudaSuccess) {
        set_error("cudaMemsetAsync: %s", cudaGetErrorString(cudaGetLastError()));
        return GCB_ECUDA;
    }
    if (p->n > 0) {
        const bool fp64 = p->mom_dtype == GCB_F64;
        auto step = [&](const gcb_particles *in) {
            return fp64 ? push_step_f64(p, in, g, &prm, st, stats) : push_step_f32(p, in, g, &prm, st, stats);
        };
        for (int c = 0; c < L.nck; ++c) {
            const gcb_particles *in = p;
            gcb_particles q;
            if (L.sort) {
                // checkpoint c is the state sorted by cell; the segment starts from it
                if ((s = sort_checkpoint(p, g, prm0, L, w, c, st, q)) != GCB_OK) return s;
                in = &q;
            } else {
                gcb_particles ckv = state_view(p, nd, w + L.ck + (size_t)c * L.S);
                if ((s = copy_state(&ckv, p, nd, st)) != GCB_OK) return s;
            }
            const int len = n_steps - c * ckpt_every < ckpt_every ? n_steps - c * ckpt_every : ckpt_every;
            for (int j = 0; j < len; ++j)
                if ((s = step(j == 0 ? in : p)) != GCB_OK) return s;
        }
        if (L.sort) {
            // back to the caller's order: p[order[j]] = (sorted final state)[j]
            int32_t *order = compose_order(p->n, L, w, L.nck - 1, st, s);
            if (s != GCB_OK) return s;
            gcb_particles t = state_view(p, nd, w + L.tmp);
            if ((s = copy_state(&t, p, nd, st)) != GCB_OK) return s;
            if (p->pid) {
                t.pid = (int64_t *)(w + L.pidt);
                if (cudaMemcpyAsync(t.pid, p->pid, 8 * (size_t)p->n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
                    set_error("cudaMemcpyAsync: %s", cudaGetErrorString(cudaGetLastError()));
                    return GCB_ECUDA;
                }
            }
            void *dst[16], *src[16];
            int es[16];
            const int na = particle_arrays(p, nd, dst, es);
            particle_arrays(&t, nd, src, es);
            if ((s = permute_arrays(p->n, na, dst, (const void *const *)src, es, order, true, st)) != GCB_OK)
                return s;
        }
    }
    return read_stats(stats, st, out);
}

gcb_status gcb_adjoint_sr(const gcb_particles *p0, const gcb_grid *g, const gcb_params *prm0,
                          int n_steps, int ckpt_every, int method, void *const *lam,
                          double *grad_rec, void *cuda_stream, void *ws, size_t ws_bytes)
{
    g_err[0] = 0;
    gcb_status s = check_adjoint(p0, g, prm0, n_steps, ckpt_every, ws, ws_bytes);
    if (s != GCB_OK) return s;
    const bool have_ckpt = (method & GCB_ADJ_HAVE_CKPT) != 0;
    method &= ~GCB_ADJ_HAVE_CKPT;
    if (method != GCB_ADJ_REVERSE && method != GCB_ADJ_TANGENT) { set_error("unknown adjoint method %d", method); return GCB_EINVAL; }
    if (!lam || !grad_rec || !aligned(grad_rec, 8)) { set_error("lam or grad_rec NULL"); return GCB_EINVAL; }
    const int me = p0->mom_dtype == GCB_F64 ? 8 : 4;
    for (int k = 0; k < 7; ++k)
        if (p0->n > 0 && (!lam[k] || !aligned(lam[k], me))) { set_error("lam[%d] NULL or misaligned", k); return GCB_EINVAL; }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    gcb_params prm = *prm0;
    prm.sort_every = 0;
    prm.fuse_steps = 0;
    const int nd = g->ndim;
    AdjLayout L;
    adj_layout(p0, g, prm0, n_steps, ckpt_every, L);
    const size_t S = L.S;
    uint8_t *w = (uint8_t *)ws;
    unsigned long long *stats = (unsigned long long *)w;
    uint8_t *ck = w + L.ck, *seg = w + L.seg, *tmp = w + L.tmp;
    const size_t nrec = (size_t)(g->n[0] * g->n[1] * g->n[2]) * 12;
    if (cudaMemsetAsync(grad_rec, 0, nrec * sizeof(double), st) != cudaSuccess ||
        cudaMemsetAsync(stats, 0, kStatsBytes, st) != cudaSuccess) {
        set_error("cudaMemsetAsync: %s", cudaGetErrorString(cudaGetLastError()));
        return GCB_ECUDA;
    }
    if (p0->n == 0) return GCB_OK;
    const bool fp64 = p0->mom_dtype == GCB_F64;
    auto step = [&](const gcb_particles *out, const gcb_particles *in) {
        return fp64 ? push_step_f64(out, in, g, &prm, st, stats) : push_step_f32(out, in, g, &prm, st, stats);
    };
    gcb_particles tA = state_view(p0, nd, tmp), tB = state_view(p0, nd, tmp + S);
    if (!have_ckpt) {
        // forward: a checkpoint every ckpt_every steps (sorted by cell first
        // when sorting); the last segment needs no forward here
        gcb_particles cur = *p0;
        for (int c = 0; c < L.nck; ++c) {
            gcb_particles ckv = state_view(p0, nd, ck + (size_t)c * S);
            if (L.sort) {
                gcb_particles q;
                if ((s = sort_checkpoint(&cur, g, prm0, L, w, c, st, q)) != GCB_OK) return s;
            } else if ((s = copy_state(&ckv, &cur, nd, st)) != GCB_OK) {
                return s;
            }
            if (c == L.nck - 1) break;
            cur = ckv;
            for (int j = 0; j < ckpt_every; ++j) {
                gcb_particles out = (cur.u[0] == tA.u[0]) ? tB : tA;
                if ((s = step(&out, &cur)) != GCB_OK) return s;
                cur = out;
            }
        }
    }
    // backward over segments, the adjoint kept in the order of the segment's
    // states (and handed from one checkpoint's order to the previous one's)
    if (L.sort) {
        int32_t *order = compose_order(p0->n, L, w, L.nck - 1, st, s);
        if (s != GCB_OK) return s;
        if ((s = permute_lam(p0->n, me, lam, L, w, order, false, st)) != GCB_OK) return s;
    }
    for (int sg = L.nck - 1; sg >= 0; --sg) {
        const int len = (n_steps - sg * ckpt_every) < ckpt_every ? n_steps - sg * ckpt_every : ckpt_every;
        std::vector<gcb_particles> states((size_t)len);
        states[0] = state_view(p0, nd, ck + (size_t)sg * S);
        for (int j = 1; j < len; ++j) {
            states[j] = state_view(p0, nd, seg + (size_t)(j - 1) * S);
            if ((s = step(&states[j], &states[j - 1])) != GCB_OK) return s;
        }
        for (int j = len - 1; j >= 0; --j)
            if ((s = adjoint_step(&states[j], g, &prm, lam, grad_rec, method, st)) != GCB_OK) return s;
        if (L.sort) {
            const int32_t *inv = (const int32_t *)(w + L.inv + (size_t)sg * a256(4 * (size_t)p0->n));
            if ((s = permute_lam(p0->n, me, lam, L, w, inv, true, st)) != GCB_OK) return s;
        }
    }
    return GCB_OK;
}

gcb_status gcb_grid_combine(const gcb_grid *g, const void *base, const void *pat,
                            const double *amps, int n_modes, void *cuda_stream)
{
    g_err[0] = 0;
    gcb_status s = check_grid(g);
    if (s != GCB_OK) return s;
    if (!base || !pat || !amps || n_modes < 0 || n_modes > 64) { set_error("gcb_grid_combine: bad arguments"); return GCB_EINVAL; }
    return grid_combine(g, base, pat, amps, n_modes, (cudaStream_t)cuda_stream);
}

gcb_status gcb_grad_project(const gcb_grid *g, const double *grad_rec, const void *pat,
                            int n_modes, double *out, void *cuda_stream)
{
    g_err[0] = 0;
    gcb_status s = check_grid(g);
    if (s != GCB_OK) return s;
    if (g->stride != 12 || !grad_rec || !pat || !out || n_modes < 1 || n_modes > 64) {
        set_error("gcb_grad_project: needs 12-element records and 1..64 modes");
        return GCB_EINVAL;
    }
    return grad_project(g, grad_rec, pat, n_modes, out, (cudaStream_t)cuda_stream);
}

}  // extern "C"
