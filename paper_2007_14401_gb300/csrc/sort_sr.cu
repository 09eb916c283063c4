// sort_sr.cu -- counting sort of the particle arrays by tile of cells.
//
// keys    : tile index of every particle (row-major over tiles, non-finite
//           particles in an extra last bucket); the rank inside the bucket
//           comes from one atomicAdd per group of equal keys in a warp
//           (__match_any_sync), so runs of already-sorted particles cost one
//           atomic per warp.
// scan    : exclusive prefix sum of the bucket counts (multi-block).
// inverse : inv[offset[key] + rank] = i, the one scattered store per particle;
// gather  : position j of the sorted copy (held in the workspace) takes
//           element inv[j] of every array -- scattered reads, coalesced writes.
// gcb_push_sr then runs its next step from that copy into the caller's
// arrays, so a sort costs no separate copy back; gcb_sort_sr copies back.
#include <cuda_runtime.h>

#include "gcb_internal.h"
#include "sort_sr.h"

namespace gcb {

static size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// multi-block scan: each block of kScanThreads threads owns kScanChunk counts
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int64_t kScanChunk = (int64_t)kScanThreads * kScanItems;

bool sort_plan(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm, SortPlan &pl)
{
    static const int def_tile[3] = {8, 8, 4};
    int64_t nt = 1;
    for (int d = 0; d < 3; ++d) {
        int t = prm && prm->sort_tile[d] > 0 ? prm->sort_tile[d] : def_tile[d];
        if (d >= g->ndim) t = 1;
        pl.tile[d] = t;
        pl.ntile[d] = (int)((g->n[d] + t - 1) / t);
        nt *= pl.ntile[d];
    }
    pl.nbuckets = nt + 1;
    if (pl.nbuckets >= (int64_t(1) << 31)) return false;
    size_t n = (size_t)p->n;
    size_t off = kStatsBytes;
    pl.off_keys = off;
    off += align256(n * 4);
    pl.off_ranks = off;
    off += align256(n * 4);
    pl.off_hist = off;
    off += align256((size_t)pl.nbuckets * 4);
    pl.nscan_blocks = (pl.nbuckets + kScanChunk - 1) / kScanChunk;
    pl.off_bsum = off;
    off += align256((size_t)pl.nscan_blocks * 4);
    pl.off_inv = off;
    off += align256(n * 4);
    // the permuted copy: x[nd], x_lo[nd] (pair), u[3], dxp[nd], flags, pid
    size_t pe = p->pos_mode == GCB_POS_F64 ? 8 : 4;
    size_t me = p->mom_dtype == GCB_F64 ? 8 : 4;
    int na = 0;
    auto add = [&](size_t es) {
        pl.off_arr[na] = off;
        pl.es[na] = (int)es;
        off += align256(n * es);
        ++na;
    };
    for (int d = 0; d < g->ndim; ++d) add(pe);
    if (p->pos_mode == GCB_POS_F32PAIR)
        for (int d = 0; d < g->ndim; ++d) add(4);
    for (int k = 0; k < 3; ++k) add(me);
    for (int d = 0; d < g->ndim; ++d) add(me);
    add(1);
    add(8);  // pid slot (used when p->pid != NULL)
    pl.narr = na;
    pl.total = off;
    return true;
}

// the caller's arrays in the order sort_plan lays them out
static int caller_arrays(const gcb_particles *p, int ndim, void **a)
{
    int na = 0;
    for (int d = 0; d < ndim; ++d) a[na++] = p->x[d];
    if (p->pos_mode == GCB_POS_F32PAIR)
        for (int d = 0; d < ndim; ++d) a[na++] = p->x_lo[d];
    for (int k = 0; k < 3; ++k) a[na++] = p->u[k];
    for (int d = 0; d < ndim; ++d) a[na++] = p->dxp[d];
    a[na++] = p->flags;
    a[na++] = p->pid;
    return na;
}

struct KeyArgs {
    int64_t n;
    int ndim, pair;
    const void *x[3];
    const float *xlo[3];
    float inv_dx[3];
    int ncell[3], tile[3], ntile[3];
    int32_t *keys, *ranks, *hist;
    int frozen_key;
};

__global__ void k_sort_keys(const KeyArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool v = i < a.n;
        const unsigned act = __ballot_sync(0xffffffffu, v);
        if (!v) continue;
        int key = 0, mul = 1;
        bool fin = true;
        for (int d = 0; d < a.ndim; ++d) {
            // the cell in FP32: a particle within rounding of a cell face may
            // be filed in the neighbouring cell, which does not matter here
            float xf;
            if (a.pair) {
                float lo = a.xlo[d][i];
                xf = ((const float *)a.x[d])[i];
                fin = fin && isfinite(xf) && isfinite(lo);
            } else {
                double xd = ((const double *)a.x[d])[i];
                fin = fin && isfinite(xd);
                xf = (float)xd;
            }
            float c = floorf(xf * a.inv_dx[d]);
            int ci = fin ? (int)fminf(fmaxf(c, 0.0f), (float)(a.ncell[d] - 1)) : 0;
            key += (ci / a.tile[d]) * mul;
            mul *= a.ntile[d];
        }
        if (!fin) key = a.frozen_key;
        const unsigned peers = __match_any_sync(act, key);
        const int leader = __ffs(peers) - 1;
        const int before = __popc(peers & ((1u << lane) - 1u));
        int b = 0;
        if (lane == leader) b = atomicAdd(&a.hist[key], __popc(peers));
        b = __shfl_sync(peers, b, leader);
        a.keys[i] = key;
        a.ranks[i] = b + before;
    }
}

// Exclusive scan of hist[0..m) in place, three passes: per-chunk sums,
// a scan of the chunk sums (one block), and the per-chunk scan with its
// offset.  Thread t of a block owns items [t*I, t*I + I) of the chunk.
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *sh, int32_t &total)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int32_t s = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    total = sh[nw - 1];
    int32_t excl = x - v + (w > 0 ? sh[w - 1] : 0);
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const int32_t *hist, int64_t m,
                                                            int32_t *bsum)
{
    __shared__ int32_t sh[32];
    const int64_t base = blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < m) s += hist[base + k];
    int32_t tot;
    block_excl_scan(s, sh, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(int32_t *hist, int64_t m,
                                                            const int32_t *boff)
{
    __shared__ int32_t sh[32];
    const int64_t base = blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < m ? hist[base + k] : 0;
        s += v[k];
    }
    int32_t tot;
    int32_t run = block_excl_scan(s, sh, tot) + boff[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < m) hist[base + k] = run;
        run += v[k];
    }
}

// In-place exclusive scan of a short array (the chunk sums) by one block.
__global__ void k_scan(int32_t *hist, int64_t m)
{
    __shared__ int32_t part[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (m + blockDim.x - 1) / blockDim.x;
    const int64_t lo = t * chunk, hi = lo + chunk < m ? lo + chunk : m;
    int32_t s = 0;
    for (int64_t k = lo; k < hi; ++k) s += hist[k];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        int32_t v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int32_t run = part[t] - s;
    for (int64_t k = lo; k < hi; ++k) {
        int32_t c = hist[k];
        hist[k] = run;
        run += c;
    }
}

__global__ void k_inverse(int64_t n, const int32_t *keys, const int32_t *ranks,
                          const int32_t *off, int32_t *inv)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        inv[(int64_t)off[keys[i]] + ranks[i]] = (int32_t)i;
}

struct GatherArgs {
    int64_t n;
    int na;
    const void *src[14];
    void *dst[14];
    int es[14];
    const int32_t *inv;
};

__global__ void k_gather_copy(const GatherArgs a)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = a.inv[j];
#pragma unroll 1
        for (int k = 0; k < a.na; ++k) {
            if (!a.src[k]) continue;
            switch (a.es[k]) {
            case 1: ((uint8_t *)a.dst[k])[j] = ((const uint8_t *)a.src[k])[i]; break;
            case 4: ((uint32_t *)a.dst[k])[j] = ((const uint32_t *)a.src[k])[i]; break;
            default: ((uint64_t *)a.dst[k])[j] = ((const uint64_t *)a.src[k])[i]; break;
            }
        }
    }
}

// The same gather for a layout fixed at compile time: N4 arrays of 4-byte
// elements, N8 of 8-byte elements, the flags and optionally the ids, with no
// per-element branch on the element size (the read-only loads of one
// particle are free to be in flight together).
struct GatherFixedArgs {
    int64_t n;
    const uint32_t *s4[12];
    uint32_t *d4[12];
    const unsigned long long *s8[9];
    unsigned long long *d8[9];
    const uint8_t *sf;
    uint8_t *df;
    const unsigned long long *sp;   // ids or NULL
    unsigned long long *dp;
    const int32_t *inv;
};

template <int N4, int N8>
__global__ void k_gather_fixed(const GatherFixedArgs a)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = a.inv[j];
#pragma unroll
        for (int k = 0; k < N4; ++k) a.d4[k][j] = __ldg(a.s4[k] + i);
#pragma unroll
        for (int k = 0; k < N8; ++k) a.d8[k][j] = __ldg(a.s8[k] + i);
        a.df[j] = __ldg(a.sf + i);
        if (a.sp) a.dp[j] = __ldg(a.sp + i);
    }
}

// Element-wise permutation of up to 16 arrays: dst[j] = src[idx[j]]
// (gather) or dst[idx[j]] = src[j] (scatter).
struct PermArgs {
    int64_t n;
    int na;
    const void *src[16];
    void *dst[16];
    int es[16];
    const int32_t *idx;
    int scatter;
};

__global__ void k_permute(const PermArgs a)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = a.idx[j];
        const int64_t from = a.scatter ? j : i, to = a.scatter ? i : j;
#pragma unroll 1
        for (int k = 0; k < a.na; ++k) {
            switch (a.es[k]) {
            case 1: ((uint8_t *)a.dst[k])[to] = ((const uint8_t *)a.src[k])[from]; break;
            case 4: ((uint32_t *)a.dst[k])[to] = ((const uint32_t *)a.src[k])[from]; break;
            default: ((uint64_t *)a.dst[k])[to] = ((const uint64_t *)a.src[k])[from]; break;
            }
        }
    }
}

static int blocks_for(int64_t n, int tpb)
{
    int64_t b = (n + tpb - 1) / tpb;
    const int64_t cap = 152 * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

gcb_status sort_into_workspace(const gcb_particles *p, const gcb_grid *g, const SortPlan &pl,
                               cudaStream_t st, uint8_t *ws, SortedView &out)
{
    if (p->n == 0) return GCB_OK;
    int32_t *keys = (int32_t *)(ws + pl.off_keys);
    int32_t *ranks = (int32_t *)(ws + pl.off_ranks);
    int32_t *hist = (int32_t *)(ws + pl.off_hist);
    if (cudaMemsetAsync(hist, 0, (size_t)pl.nbuckets * 4, st) != cudaSuccess) {
        set_error("cudaMemsetAsync: %s", cudaGetErrorString(cudaGetLastError()));
        return GCB_ECUDA;
    }
    KeyArgs ka;
    ka.n = p->n;
    ka.ndim = g->ndim;
    ka.pair = p->pos_mode == GCB_POS_F32PAIR;
    for (int d = 0; d < 3; ++d) {
        ka.x[d] = p->x[d];
        ka.xlo[d] = (const float *)p->x_lo[d];
        ka.inv_dx[d] = (float)(1.0 / g->dx[d]);
        ka.ncell[d] = (int)g->n[d];
        ka.tile[d] = pl.tile[d];
        ka.ntile[d] = pl.ntile[d];
    }
    ka.keys = keys;
    ka.ranks = ranks;
    ka.hist = hist;
    ka.frozen_key = (int)(pl.nbuckets - 1);
    k_sort_keys<<<blocks_for(p->n, 256), 256, 0, st>>>(ka);
    int32_t *bsum = (int32_t *)(ws + pl.off_bsum);
    k_scan_sums<<<(unsigned)pl.nscan_blocks, kScanThreads, 0, st>>>(hist, pl.nbuckets, bsum);
    k_scan<<<1, 1024, 0, st>>>(bsum, pl.nscan_blocks);
    k_scan_down<<<(unsigned)pl.nscan_blocks, kScanThreads, 0, st>>>(hist, pl.nbuckets, bsum);
    int32_t *inv = (int32_t *)(ws + pl.off_inv);
    k_inverse<<<blocks_for(p->n, 256), 256, 0, st>>>(p->n, keys, ranks, hist, inv);
    GatherArgs ga;
    ga.n = p->n;
    void *src[14];
    ga.na = caller_arrays(p, g->ndim, src);
    for (int k = 0; k < ga.na; ++k) {
        ga.src[k] = src[k];
        ga.dst[k] = src[k] ? (void *)(ws + pl.off_arr[k]) : nullptr;
        ga.es[k] = pl.es[k];
        out.arr[k] = ga.dst[k];
    }
    out.narr = ga.na;
    ga.inv = inv;
    // the layouts of the pushes' states get a gather without size branches
    GatherFixedArgs fa;
    int n4 = 0, n8 = 0;
    bool fixed = true;
    fa.n = p->n;
    fa.inv = inv;
    fa.sf = nullptr;
    fa.df = nullptr;
    fa.sp = nullptr;
    fa.dp = nullptr;
    for (int k = 0; k < ga.na && fixed; ++k) {
        if (!ga.src[k]) continue;
        if (ga.es[k] == 4 && n4 < 12) {
            fa.s4[n4] = (const uint32_t *)ga.src[k];
            fa.d4[n4++] = (uint32_t *)ga.dst[k];
        } else if (ga.es[k] == 8 && k == ga.na - 1) {   // the ids (last array)
            fa.sp = (const unsigned long long *)ga.src[k];
            fa.dp = (unsigned long long *)ga.dst[k];
        } else if (ga.es[k] == 8 && n8 < 9) {
            fa.s8[n8] = (const unsigned long long *)ga.src[k];
            fa.d8[n8++] = (unsigned long long *)ga.dst[k];
        } else if (ga.es[k] == 1 && !fa.sf) {
            fa.sf = (const uint8_t *)ga.src[k];
            fa.df = (uint8_t *)ga.dst[k];
        } else {
            fixed = false;
        }
    }
    fixed = fixed && fa.sf;
    // (the 2D mixed state with FP32-pair positions: a step with a sort measured
    // 1.57 against 1.71 ms at 2^24 particles; the 3D one, 12 arrays, measured
    // slower than the generic gather, its registers halving the resident
    // threads)
    const int nb = blocks_for(p->n, 256);
    if (fixed && n4 == 9 && n8 == 0) k_gather_fixed<9, 0><<<nb, 256, 0, st>>>(fa);
    else k_gather_copy<<<nb, 256, 0, st>>>(ga);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("sort kernels: %s", cudaGetErrorString(e));
        return GCB_ECUDA;
    }
    return GCB_OK;
}

gcb_status copy_back(const gcb_particles *p, const gcb_grid *g, const SortPlan &pl,
                     const SortedView &v, cudaStream_t st)
{
    void *dst[14];
    int na = caller_arrays(p, g->ndim, dst);
    for (int k = 0; k < na; ++k) {
        if (!dst[k]) continue;
        if (cudaMemcpyAsync(dst[k], v.arr[k], (size_t)p->n * pl.es[k], cudaMemcpyDeviceToDevice,
                            st) != cudaSuccess) {
            set_error("cudaMemcpyAsync: %s", cudaGetErrorString(cudaGetLastError()));
            return GCB_ECUDA;
        }
    }
    return GCB_OK;
}

// The view of a particle set whose arrays are the sorted copy.
void sorted_particles(const gcb_particles *p, int ndim, const SortedView &v, gcb_particles &q)
{
    q = *p;
    int k = 0;
    for (int d = 0; d < ndim; ++d) q.x[d] = v.arr[k++];
    if (p->pos_mode == GCB_POS_F32PAIR)
        for (int d = 0; d < ndim; ++d) q.x_lo[d] = v.arr[k++];
    for (int c = 0; c < 3; ++c) q.u[c] = v.arr[k++];
    for (int d = 0; d < ndim; ++d) q.dxp[d] = v.arr[k++];
    q.flags = (uint8_t *)v.arr[k++];
    q.pid = (int64_t *)v.arr[k++];
}

gcb_status permute_arrays(int64_t n, int na, void *const *dst, const void *const *src,
                          const int *es, const int32_t *idx, bool scatter, cudaStream_t st)
{
    if (n == 0 || na == 0) return GCB_OK;
    if (na > 16) { set_error("permute_arrays: at most 16 arrays"); return GCB_EINVAL; }
    PermArgs a;
    a.n = n;
    a.na = na;
    for (int k = 0; k < na; ++k) {
        a.src[k] = src[k];
        a.dst[k] = dst[k];
        a.es[k] = es[k];
    }
    a.idx = idx;
    a.scatter = scatter ? 1 : 0;
    k_permute<<<blocks_for(n, 256), 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("k_permute: %s", cudaGetErrorString(e));
        return GCB_ECUDA;
    }
    return GCB_OK;
}

}  // namespace gcb
