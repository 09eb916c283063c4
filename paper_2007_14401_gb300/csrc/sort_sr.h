// sort_sr.h -- the cell-tile sort of the particle arrays (internal).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "gcb.h"

namespace gcb {

// Workspace layout of a sort: counters | keys | ranks | bucket offsets |
// chunk sums | inverse permutation | one permuted copy of every particle
// array (256-byte aligned sections).
struct SortPlan {
    int tile[3], ntile[3];
    int64_t nbuckets;
    int64_t nscan_blocks;    // blocks of the multi-block scan of the counts
    size_t off_keys, off_ranks, off_hist, off_bsum, off_inv;
    size_t off_arr[14];
    int es[14];
    int narr;
    size_t total;
};

struct SortedView {
    void *arr[14];
    int narr;
};

bool sort_plan(const gcb_particles *p, const gcb_grid *g, const gcb_params *prm, SortPlan &pl);
gcb_status sort_into_workspace(const gcb_particles *p, const gcb_grid *g, const SortPlan &pl,
                               cudaStream_t st, uint8_t *ws, SortedView &out);
gcb_status copy_back(const gcb_particles *p, const gcb_grid *g, const SortPlan &pl,
                     const SortedView &v, cudaStream_t st);
void sorted_particles(const gcb_particles *p, int ndim, const SortedView &v, gcb_particles &q);
// dst[k][j] = src[k][idx[j]] (gather) or dst[k][idx[j]] = src[k][j] (scatter)
// for na arrays of element sizes es[k] (1, 4 or 8 bytes); n elements each.
gcb_status permute_arrays(int64_t n, int na, void *const *dst, const void *const *src,
                          const int *es, const int32_t *idx, bool scatter, cudaStream_t st);

}  // namespace gcb
