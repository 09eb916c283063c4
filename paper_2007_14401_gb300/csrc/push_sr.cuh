// push_sr.cuh -- one coupled step (Sec. 3.1) over all particles, one kernel.
//
// Each block walks tiles of TPB consecutive particles (persistent grid):
//   phase 1  every thread loads one particle (coalesced SoA loads; the
//            unfused FP32 2D kernels take it from shared memory, where
//            asynchronous copies issued during the previous tile put it),
//            gathers E, B at x^n, evaluates the switch S and stages the
//            particle in shared memory;
//   compact  a warp ballot per branch plus a block prefix over the per-warp
//            counts orders the tile's slots as [GCA ..., Boris ..., frozen],
//            so all warps but one run a single branch and GCA lanes run the
//            same loop (the queues of the GCA and Boris branches);
//   phase 2  thread t advances the particle in slot perm[t] and stores it
//            back at that particle's own index.
// Counters are reduced per block and added atomically to the workspace.
#pragma once

#include "gcb_device.cuh"
#include "gcb_internal.h"

namespace gcb {

// Particles per tile (= threads per block).  FP32 2D: one warp, so a
// tile's vote and compaction stay within the warp and no block barrier
// holds warps back (the GCA-dominated 2D push measured 4% faster than with
// 128; GB300, 2^24 particles); FP32 3D and FP64: 128 (4 warps), so the
// compaction of mixed tiles (both branches) leaves at most one mixed warp
// (the 3D sheet measured 7% faster than with 32).
#ifndef GCB_TILE_F32_2D
#define GCB_TILE_F32_2D 32
#endif
#ifndef GCB_TILE_F32_3D
#define GCB_TILE_F32_3D 128
#endif
template <typename R, int ND>
struct Tile {
    static constexpr int n = sizeof(R) == 8 ? 128 : (ND == 2 ? GCB_TILE_F32_2D : GCB_TILE_F32_3D);
};

// 1: tiles whose particles all take one branch skip the staging (see k_push_sr)
#ifndef GCB_UNIFORM_TILES
#define GCB_UNIFORM_TILES 1
#endif
// minimum resident threads per SM requested from the register allocator:
// FP32 2D 512 (at most 128 registers a thread); FP32 3D 384 (at most 170
// registers: 184 unconstrained leaves 256 threads, which measured 16% slower,
// and 512 spills)
#ifndef GCB_MIN_THREADS_F32_2D
#define GCB_MIN_THREADS_F32_2D 512
#endif
#ifndef GCB_MIN_THREADS_F32_3D
#define GCB_MIN_THREADS_F32_3D 384
#endif
#ifndef GCB_SEED_CACHE
#define GCB_SEED_CACHE 1
#endif
#ifndef GCB_REG2D
#define GCB_REG2D 1
#endif
// 1: phase 1 gathers at R^{n-1/2} = x^n - dxp/2 together with x^n (2D), so
// that the two gathers' loads are in flight at once
#ifndef GCB_HOIST_HALF
#define GCB_HOIST_HALF 1
#endif
// FP32 3D with current deposition and gradient records: 256 (the 3D walk
// spills 684 B at 384); with gradients from W, 384 as without deposition
// (measured 14% faster than 256 on the 3D sheet)
#ifndef GCB_MIN_THREADS_F32_3D_DEP_GRID
#define GCB_MIN_THREADS_F32_3D_DEP_GRID 256
#endif
template <typename R, int ND, int GM = 1, bool DEP = false>
struct MinBlocks {
    static constexpr int n = sizeof(R) == 8
        ? 1
        : (ND == 3 ? ((DEP && GM == 2) ? GCB_MIN_THREADS_F32_3D_DEP_GRID : GCB_MIN_THREADS_F32_3D)
                   : GCB_MIN_THREADS_F32_2D) / Tile<R, ND>::n;
};

template <typename R>
struct PushArgs {
    DevGrid<R> g;
    double L[3];              // box length per axis
    double dxd[3], inv_dxd[3];
    float Lf[3];              // box length in float (pair positions)
    int64_t np;
    // input arrays (the caller's, or the sorted copy in the workspace)
    const void *xin[3];
    const float *xloin[3];
    const R *uin[3];
    const R *dxpin[3];
    const uint8_t *flagsin;
    const int64_t *pidin;
    // output arrays (always the caller's)
    void *x[3];               // double (PM 0) or float hi (PM 1)
    float *xlo[3];
    R *u[3];
    R *dxp[3];
    uint8_t *flags;
    int64_t *pid;             // written only when pidin differs
    StepPar<R> sp;            // sp.qm is set per particle
    R qm[4];
    R rho_thr;                // f_rho * dl
    R f_E;
    R c2;
    int force;
    int nsteps;               // steps of this launch (> 1 only for the fused kernel)
    unsigned long long *stats;
    // current deposition (kernels with DEP)
    R *J[3];
    const R *w;               // per-particle weights or NULL
    R dq[4];                  // charge per species
    R jc[3];                  // dx_a / (dt V): J_a per cell of displacement along a
    R jz;                     // 1 / V: 2D J_z per unit v_z and step fraction
    int pf;                   // the input state is in device memory (GCB_PREFETCH_STATE)
};

// Particle state is read and written once per step and the field records
// many times: the state's loads and stores are marked streaming (evict
// first), so that they do not push the records out of L1 and L2.
#ifndef GCB_STREAM_STATE
#define GCB_STREAM_STATE 1
#endif
template <typename T>
__device__ __forceinline__ T ld_state(const T *p)
{
    if constexpr (GCB_STREAM_STATE) return __ldcs(p);
    else return *p;
}
template <typename T>
__device__ __forceinline__ void st_state(T *p, T v)
{
    if constexpr (GCB_STREAM_STATE) __stcs(p, v);
    else *p = v;
}

// 1: unfused FP32 2D kernels copy the state of the block's next tile into
// shared memory with asynchronous copies (cp.async) while the current tile
// is advanced, so that the state's DRAM latency overlaps a tile of
// arithmetic instead of stalling the tile's first gather (state in device
// memory only; host-resident state is read directly).  Measured 1.3% faster
// on the 2D push (2^24 particles); no effect on the 3D push, whose
// deposition kernels it made spill.
#ifndef GCB_PREFETCH_STATE
#define GCB_PREFETCH_STATE 1
#endif
template <int B>
__device__ __forceinline__ void cp_async(void *dst, const void *src)
{
    static_assert(B == 4 || B == 8, "4- or 8-byte elements");
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(B)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int PM>
struct PosType;
template <>
struct PosType<0> { using T = double; };
template <>
struct PosType<1> { using T = float; };

// x (stored) -> base cell index in [0, n) and offset from that cell's origin
// (positions are kept in [0, L); the clamp only matters for positions that
// rounding put on an edge or for invalid input).
template <typename R>
__device__ __forceinline__ void split_pos_f64(double x, double dxd, double inv_dxd, double nmax,
                                              int &ib, R &l)
{
    double fl = fmin(fmax(floor(x * inv_dxd), 0.0), nmax);
    ib = (int)fl;
    l = (R)fma(-fl, dxd, x);
}
__device__ __forceinline__ void split_pos_pair(float h, float lo, float dx, float inv_dx,
                                               float nmax, int &ib, float &l)
{
    float fl = fminf(fmaxf(floorf(h * inv_dx), 0.0f), nmax);
    ib = (int)fl;
    l = fmaf(-fl, dx, h) + lo;
}

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (h, lo) += d for an FP32-pair position, then wrap into [0, L).
__device__ __forceinline__ void pair_add_wrap(float &h, float &lo, float d, float L)
{
    float s, e;
    two_sum(h, d, s, e);
    e += lo;
    h = s + e;
    lo = e - (h - s);
    if (h < 0.0f) {
        two_sum(h, L, s, e);
        e += lo;
        h = s + e;
        lo = e - (h - s);
    }
    if (h >= L) {
        h -= L;  // exact: L <= h < 2L
        float t = h + lo;
        lo = lo - (t - h);
        h = t;
    }
    if (h < 0.0f || h >= L) {  // lo pushed the sum across an edge
        h = 0.0f;
        lo = 0.0f;
    }
}

__device__ __forceinline__ double wrap_f64(double x, double L)
{
    if (x < 0.0) x += L;
    if (x >= L) x -= L;
    return x;
}

template <typename R>
__device__ __forceinline__ bool finite_r(R v) { return isfinite(v); }

// ---------------------------------------------------------------------------
// Current deposition (gcb_push_deposit_sr): the current of a cloud-in-cell
// particle moving along the straight path x^n -> x^{n+1}, averaged over the
// step, on the staggered points.  The path is walked cell by cell (the face
// each axis crosses next, the nearest first).  Inside one cell every hat is
// linear in time, so a piece's average of one hat is its value at the
// piece's midpoint, and the average of the product of two hats adds the
// product of the piece's extents (in cells) along those axes over 12.
// ---------------------------------------------------------------------------
// Per particle-step: the current's arrays and grid sizes, and the factors
// Q w dx_a/(dt V) (per cell of displacement along a) and, in 2D,
// Q w v_z/V (per unit step fraction), formed once for all the pieces.
template <typename R>
struct DepCtx {
    R *J[3];
    R f[3];
    int n[3];
};

// returns the number of atomic additions issued
template <typename R, int ND>
__device__ __forceinline__ int dep_piece(const DepCtx<R> &q, const int cell[ND], const R p0[ND],
                                         const R p1[ND], R tau)
{
    int nat = 0;
    const int nx = q.n[0], ny = q.n[1];
    int I[2], Jn[2];
    I[0] = cell[0];
    I[1] = cell[0] + 1 == nx ? 0 : cell[0] + 1;
    Jn[0] = cell[1];
    Jn[1] = cell[1] + 1 == ny ? 0 : cell[1] + 1;
    R d[ND], m[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) {
        d[k] = p1[k] - p0[k];
        m[k] = R(0.5) * (p0[k] + p1[k]);
    }
    if constexpr (ND == 2) {
        // 32-bit indices (the deposition is limited to grids of < 2^31 nodes)
        const int r0 = Jn[0] * nx, r1 = Jn[1] * nx;
        const int i00 = r0 + I[0], i10 = r0 + I[1], i01 = r1 + I[0], i11 = r1 + I[1];
        if (d[0] != R(0)) {   // J_x at (i+1/2, j) and (i+1/2, j+1)
            const R f = q.f[0] * d[0];
            atomicAdd(q.J[0] + i00, f * (R(1) - m[1]));
            atomicAdd(q.J[0] + i01, f * m[1]);
            nat += 2;
        }
        if (d[1] != R(0)) {   // J_y at (i, j+1/2) and (i+1, j+1/2)
            const R f = q.f[1] * d[1];
            atomicAdd(q.J[1] + i00, f * (R(1) - m[0]));
            atomicAdd(q.J[1] + i10, f * m[0]);
            nat += 2;
        }
        if (q.f[2] != R(0) && tau > R(0)) {   // J_z at the cell's four nodes
            const R f = q.f[2] * tau;
            const R cr = d[0] * d[1] * R(1.0 / 12.0);
            const R w0 = R(1) - m[0], w1 = R(1) - m[1];
            atomicAdd(q.J[2] + i00, f * fma(w0, w1, cr));
            atomicAdd(q.J[2] + i10, f * fma(m[0], w1, -cr));
            atomicAdd(q.J[2] + i01, f * fma(w0, m[1], -cr));
            atomicAdd(q.J[2] + i11, f * fma(m[0], m[1], cr));
            nat += 4;
        }
    } else {
        const int nz = q.n[2];
        int K[2];
        K[0] = cell[2];
        K[1] = cell[2] + 1 == nz ? 0 : cell[2] + 1;
        auto lin = [&](int i, int j, int k) { return (k * ny + j) * nx + i; };
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (d[c] == R(0)) continue;
            // the other two axes in cyclic order, b then e
            const int b = c == 2 ? 0 : c + 1, e = c == 0 ? 2 : c - 1;
            const R f = q.f[c] * d[c];
            const R cr = d[b] * d[e] * R(1.0 / 12.0);
#pragma unroll
            for (int oe = 0; oe < 2; ++oe)
#pragma unroll
                for (int ob = 0; ob < 2; ++ob) {
                    const R wb = ob ? m[b] : R(1) - m[b];
                    const R we = oe ? m[e] : R(1) - m[e];
                    const R v = f * fma(wb, we, (ob == oe) ? cr : -cr);
                    int idx;
                    if (c == 0) idx = lin(I[0], Jn[ob], K[oe]);
                    else if (c == 1) idx = lin(I[oe], Jn[0], K[ob]);
                    else idx = lin(I[ob], Jn[oe], K[0]);
                    atomicAdd(q.J[c] + idx, v);
                }
            nat += 4;
        }
    }
    return nat;
}

// false: the path is longer than GCB_DEPOSIT_MAX_CELLS cells along an axis
// and nothing is deposited.  ib, l: cell and offset of x^n; disp = x^{n+1} - x^n.
template <typename R, int ND>
__device__ __forceinline__ bool deposit_path(const PushArgs<R> &a, const int ib[ND], const R l[ND],
                                             const R disp[ND], R Qw, R vz, unsigned &npc,
                                             unsigned &nat)
{
    DepCtx<R> q;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        q.J[k] = a.J[k];
        q.n[k] = a.g.n[k];
    }
    q.f[0] = Qw * a.jc[0];
    q.f[1] = Qw * a.jc[1];
    q.f[2] = ND == 2 ? Qw * a.jz * vz : Qw * a.jc[2];
    // off: the current cell's offset from the cell of x^n (held in R)
    R s0[ND], ds[ND], p0[ND], tn[ND], td[ND], off[ND];
    int cell[ND], stp[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) {
        ds[k] = disp[k] * a.g.inv_dx[k];
        if (!(fabs(ds[k]) <= R(GCB_DEPOSIT_MAX_CELLS))) return false;
        s0[k] = fmin(fmax(l[k] * a.g.inv_dx[k], R(0)), R(1));
        p0[k] = s0[k];
        cell[k] = ib[k];
        off[k] = R(0);
        if (ds[k] > R(0)) {
            stp[k] = 1;
            td[k] = R(1) / ds[k];
            tn[k] = (R(1) - s0[k]) * td[k];
        } else if (ds[k] < R(0)) {
            stp[k] = -1;
            td[k] = R(-1) / ds[k];
            tn[k] = s0[k] * td[k];
        } else {
            stp[k] = 0;
            td[k] = R(0);
            tn[k] = R(2);
        }
    }
    R t = R(0);
    // every piece but the last ends on a face; each axis crosses at most
    // GCB_DEPOSIT_MAX_CELLS + 1 faces
    constexpr int kMaxPieces = ND * (GCB_DEPOSIT_MAX_CELLS + 2) + 1;
    for (int it = 0; it < kMaxPieces; ++it) {
        R te = R(1);
#pragma unroll
        for (int k = 0; k < ND; ++k) te = fmin(te, tn[k]);
        R p1[ND];
#pragma unroll
        for (int k = 0; k < ND; ++k)
            p1[k] = fmin(fmax(fma(ds[k], te, s0[k]) - off[k], R(0)), R(1));
        nat += dep_piece<R, ND>(q, cell, p0, p1, te - t);
        ++npc;
        if (te >= R(1)) break;
#pragma unroll
        for (int k = 0; k < ND; ++k) {
            if (stp[k] != 0 && tn[k] <= te) {   // enters the next cell along k
                int c = cell[k] + stp[k];
                cell[k] = c < 0 ? q.n[k] - 1 : (c == q.n[k] ? 0 : c);
                off[k] += R(stp[k]);
                tn[k] += td[k];
                p1[k] = stp[k] > 0 ? R(0) : R(1);
            }
            p0[k] = p1[k];
        }
        t = te;
    }
    return true;
}

// FUSE = false: one step per launch (the PiC mode: state through HBM every
// step).  FUSE = true: a.nsteps steps per launch, each tile's state kept in
// its shared-memory slots between the steps and written once at the end (the
// test-particle mode); every step's arithmetic is the unfused step's.
// DEP (unfused only): each advanced particle-step also adds its current to a.J.
// MIR (unfused only): the guiding-center step with the mirror terms.
template <typename R, int ND, int PM, int GM, bool FUSE, bool BT = false, bool DEP = false,
          bool MIR = false>
__global__ void __launch_bounds__(Tile<R, ND>::n, MinBlocks<R, ND, GM, DEP>::n) k_push_sr(const PushArgs<R> a)
{
    static_assert(!(DEP && FUSE), "deposition runs in unfused launches");
    constexpr int TPB = Tile<R, ND>::n;
    constexpr int NWARP = TPB / 32;
    constexpr int NF = (GM != 0) ? 6 + 3 * ND : 6;   // staged field values at x^n
    using PosT = typename PosType<PM>::T;
    __shared__ PosT s_x[ND][TPB];
    __shared__ float s_xl[PM ? ND : 1][TPB];
    __shared__ R s_l[ND][TPB];
    __shared__ int s_ib[ND][TPB];
    __shared__ R s_u[3][TPB];
    __shared__ R s_d[ND][TPB];
    __shared__ R s_F[NF][TPB];
    __shared__ uint8_t s_fl[TPB];
    __shared__ unsigned short s_perm[TPB];
    __shared__ int s_wc[2][NWARP];
    __shared__ unsigned long long s_acc[ST_COUNT];
    __shared__ double s_ek;
    // the state of this block's next tile, copied while the current one is
    // advanced (two buffers: the copies into one overlap the reads of the other)
    constexpr bool PF = GCB_PREFETCH_STATE && !FUSE && sizeof(R) == 4 && ND == 2;
    constexpr int PFN = PF ? TPB : 1;
    __shared__ PosT s_px[2][ND][PFN];
    __shared__ float s_pxl[2][PM ? ND : 1][PFN];
    __shared__ R s_pd[2][ND][PFN];
    __shared__ R s_pu[2][3][PFN];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < ST_COUNT) s_acc[tid] = 0ull;
    if (tid == 0) s_ek = 0.0;

    unsigned nb = 0, ng = 0, tg = 0, tb = 0, nc = 0, gf = 0, nf = 0, si = 0, mi = 0;
    unsigned nds = 0, npc = 0, nat = 0;   // DEP: skipped paths, pieces, atomics
    double ek = 0.0;

    const int64_t ntiles = (a.np + TPB - 1) / TPB;
    const bool pf = PF && a.pf;
    int pb = 0;              // buffer holding the current tile's state
    uint8_t fl_next = 0;     // the next tile's flag (a plain load, one tile ahead)
    // copies of particle j's state into buffer b (one commit group per tile)
    auto prefetch = [&](int b, int64_t j) {
        if (j < a.np) {
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                cp_async<sizeof(PosT)>(&s_px[b][d][tid], reinterpret_cast<const PosT *>(a.xin[d]) + j);
                if (PM) cp_async<4>(&s_pxl[b][d][tid], a.xloin[d] + j);
                cp_async<sizeof(R)>(&s_pd[b][d][tid], a.dxpin[d] + j);
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) cp_async<sizeof(R)>(&s_pu[b][k][tid], a.uin[k] + j);
            fl_next = ld_state(a.flagsin + j);
        }
        cp_async_commit();
    };
    // tiles strided over the grid: at any moment the blocks of all SMs work
    // on neighbouring tiles, so the field records in use stay few and hot
    // in L2 (one contiguous run of tiles per block measured 48% slower)
    if (pf) prefetch(0, (int64_t)blockIdx.x * TPB + tid);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const int64_t i = tile * TPB + tid;
      const bool valid = i < a.np;
      // the next tile's copies go out before this tile's are awaited
      uint8_t fl_cur = 0;
      if (pf) {
          fl_cur = fl_next;
          prefetch(pb ^ 1, i + (int64_t)gridDim.x * TPB);
          cp_async_wait<1>();
      }
      for (int stp = 0; stp < (FUSE ? a.nsteps : 1); ++stp) {
        int cls = 2;
        uint8_t fl = 0;
        int64_t pid = 0;
        PosT xs[ND];
        float xl[ND];
        R l[ND], uu[3], dd[ND];
        FieldPt<R, ND> F;
        constexpr bool HOIST = GCB_HOIST_HALF && ND == 2;
        FieldPt<R, ND> Fh;          // fields at R^{n-1/2} (HOIST)
        int ib[ND];
        using Gth = PlainGather<R, ND, GM>;
        StepRecs<Gth, ND, GM> cr;
        cr.clear();
        if (valid) {
            const bool from_smem = FUSE && stp > 0;   // the slot holds the previous step's output
            if (!from_smem && a.pidin != a.pid) pid = ld_state(a.pidin + i);
            bool fin = true;
            if (pf) {
                fl = fl_cur;
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    xs[d] = s_px[pb][d][tid];
                    xl[d] = PM ? s_pxl[pb][d][tid] : 0.0f;
                    dd[d] = s_pd[pb][d][tid];
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) uu[k] = s_pu[pb][k][tid];
            } else {
                fl = from_smem ? s_fl[tid] : ld_state(a.flagsin + i);
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    xs[d] = from_smem ? s_x[d][tid] : ld_state(reinterpret_cast<const PosT *>(a.xin[d]) + i);
                    xl[d] = PM ? (from_smem ? s_xl[d][tid] : ld_state(a.xloin[d] + i)) : 0.0f;
                    dd[d] = from_smem ? s_d[d][tid] : ld_state(a.dxpin[d] + i);
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) uu[k] = from_smem ? s_u[k][tid] : ld_state(a.uin[k] + i);
            }
#pragma unroll
            for (int d = 0; d < ND; ++d)
                fin = fin && finite_r(xs[d]) && finite_r(xl[d]) && finite_r(dd[d]);
#pragma unroll
            for (int k = 0; k < 3; ++k) fin = fin && finite_r(uu[k]);
            if (fin) {
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    if (PM == 0)
                        split_pos_f64<R>((double)xs[d], a.dxd[d], a.inv_dxd[d],
                                         (double)(a.g.n[d] - 1), ib[d], l[d]);
                    else {
                        float lf;
                        split_pos_pair((float)xs[d], xl[d], (float)a.g.dx[d], (float)a.g.inv_dx[d],
                                       (float)(a.g.n[d] - 1), ib[d], lf);
                        l[d] = (R)lf;
                    }
                }
                if constexpr (GCB_SEED_CACHE && Gth::kCellCache) gather_cached<ND, GM>(a.g, ib, l, F, cr);
                else gather_any<R, ND, GM>(a.g, ib, l, F);
                if constexpr (HOIST) {
                    R ph[ND];
#pragma unroll
                    for (int d = 0; d < ND; ++d) ph[d] = fma(R(-0.5), dd[d], l[d]);
                    gather_any<R, ND, GM>(a.g, ib, ph, Fh);
                }
                // switch S (Sec. 3, Sec. 4.1) in division-free form:
                // S = 0 iff c^2 Gamma < f_rho dl |q/m| B and |E| < f_E B.
                R Q = fabs(a.qm[(fl >> GCB_SPECIES_SHIFT) & 3]);
                R G = sqrt(R(1) + dot3(uu, uu) * a.sp.inv_c2);
                R Bm = sqrt(dot3(F.B, F.B));
                R Em = sqrt(dot3(F.E, F.E));
                int S = (a.c2 * G < a.rho_thr * Q * Bm && Em < a.f_E * Bm) ? 0 : 1;
                if (a.force == GCB_FORCE_BORIS) S = 1;
                if (a.force == GCB_FORCE_GCA) S = 0;
                cls = S;
            } else {
                // frozen: written back unchanged (with its flag) right here;
                // fused, it stays in its slot for the final store
                fl |= GCB_FLAG_NONFINITE;
                ++nf;
                if (!FUSE) {
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        st_state(reinterpret_cast<PosT *>(a.x[d]) + i, xs[d]);
                        if (PM) st_state(a.xlo[d] + i, xl[d]);
                        st_state(a.dxp[d] + i, dd[d]);
                    }
#pragma unroll
                    for (int k = 0; k < 3; ++k) st_state(a.u[k] + i, uu[k]);
                    st_state(a.flags + i, fl);
                }
            }
            if (a.pidin != a.pid && (!FUSE || stp == 0)) st_state(a.pid + i, pid);
        }
        // Tiles whose valid particles all take one branch (the common case in
        // strongly magnetized runs) skip the compaction and the staging of
        // the field: each thread advances its own particle.  The rest of the
        // state is held in registers through phase 2 (REG: 2D, measured
        // faster) or kept in the thread's slot and read where used (3D,
        // whose kernels hold more live values and whose tiles are more often
        // mixed, measured faster that way).
        constexpr bool REG = (ND == 2) && GCB_REG2D;
        int uni = 0;
        if (GCB_UNIFORM_TILES) {
            if (__syncthreads_and(!valid || cls == 0)) uni = 1;
            else if (__syncthreads_and(!valid || cls == 1)) uni = 2;
        }
        bool work, isg;
        int sl = tid;
        if (uni) {
            // the barrier of the vote has ended every read of the slots
            if (!REG && valid) {
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    s_x[d][tid] = xs[d];
                    if (PM) s_xl[d][tid] = xl[d];
                    s_d[d][tid] = dd[d];
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) s_u[k][tid] = uu[k];
            }
            if (!REG) s_fl[tid] = fl;
            work = valid && cls != 2;
            isg = uni == 1;
        } else {
            __syncthreads();  // the previous tile's slots are no longer read
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                if (valid) {
                    s_x[d][tid] = xs[d];
                    if (PM) s_xl[d][tid] = xl[d];
                    s_d[d][tid] = dd[d];
                    s_l[d][tid] = l[d];
                    s_ib[d][tid] = ib[d];
                }
            }
            if (valid && cls != 2) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    s_F[k][tid] = F.E[k];
                    s_F[3 + k][tid] = F.B[k];
                }
                if (GM != 0) {
#pragma unroll
                    for (int ii = 0; ii < ND; ++ii)
#pragma unroll
                        for (int j = 0; j < 3; ++j) s_F[6 + 3 * ii + j][tid] = F.dB[ii][j];
                }
            }
            if (valid) {
#pragma unroll
                for (int k = 0; k < 3; ++k) s_u[k][tid] = uu[k];
            }
            s_fl[tid] = fl;
            const unsigned bgm = __ballot_sync(0xffffffffu, cls == 0);
            const unsigned bbm = __ballot_sync(0xffffffffu, cls == 1);
            if (lane == 0) {
                s_wc[0][warp] = __popc(bgm);
                s_wc[1][warp] = __popc(bbm);
            }
            __syncthreads();
            int offG = 0, offB = 0, totG = 0, totB = 0;
#pragma unroll
            for (int w = 0; w < NWARP; ++w) {
                int cg = s_wc[0][w], cb = s_wc[1][w];
                if (w < warp) { offG += cg; offB += cb; }
                totG += cg;
                totB += cb;
            }
            const unsigned lt = (1u << lane) - 1u;
            if (cls == 0) s_perm[offG + __popc(bgm & lt)] = (unsigned short)tid;
            if (cls == 1) s_perm[totG + offB + __popc(bbm & lt)] = (unsigned short)tid;
            __syncthreads();
            // this thread advances slot perm[tid]: [GCA ..., Boris ...]
            cr.clear();   // the records loaded were those of the thread's own particle
            work = tid < totG + totB;
            isg = tid < totG;
            if (work) {
                sl = s_perm[tid];
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    ib[d] = s_ib[d][sl];
                    l[d] = s_l[d][sl];
                    if (REG) {
                        xs[d] = s_x[d][sl];
                        xl[d] = PM ? s_xl[d][sl] : 0.0f;
                        dd[d] = s_d[d][sl];
                    }
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    F.E[k] = s_F[k][sl];
                    F.B[k] = s_F[3 + k][sl];
                    if (REG) uu[k] = s_u[k][sl];
                }
                if (REG) fl = s_fl[sl];
                if (isg && GM != 0) {
#pragma unroll
                    for (int ii = 0; ii < ND; ++ii)
#pragma unroll
                        for (int j = 0; j < 3; ++j) F.dB[ii][j] = s_F[6 + 3 * ii + j][sl];
                }
            }
        }

        // phase 2: advance the particle of slot sl (field, cell and offset in
        // F, ib, l; the rest of its state in registers (REG) or in the slot)
        if (work) {
            const uint8_t f0 = REG ? fl : s_fl[sl];
            StepPar<R> sp = a.sp;
            sp.qm = a.qm[(f0 >> GCB_SPECIES_SHIFT) & 3];
            R ds[ND], us[3], disp[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d) ds[d] = REG ? dd[d] : s_d[d][sl];
#pragma unroll
            for (int k = 0; k < 3; ++k) us[k] = REG ? uu[k] : s_u[k][sl];
            int it = 0;
            bool ncv = false, fail = false;
            bool done = false;
            R vzg = R(0);   // out-of-plane guiding-center velocity of the step (2D DEP)
            if (isg) {
                done = gca_step_c<R, ND, GM, Gth, BT, MIR>(Gth{a.g}, sp, ib, l, ds, F, us, disp, it,
                                                      ncv, cr, (HOIST && uni) ? &Fh : nullptr,
                                                      (DEP && ND == 2) ? &vzg : nullptr);
                if (!done) {
                    fail = true;
                    it = 0;
                    ncv = false;
#pragma unroll
                    for (int k = 0; k < 3; ++k) us[k] = REG ? uu[k] : s_u[k][sl];
                }
            }
            if (!done) boris<R, ND>(F.E, F.B, sp, us, disp);
            // store: x^{n+1} = x^n + disp (wrapped), dxp = disp
            PosT xn[ND];
            float xln[ND];
            bool fin = true;
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const PosT x0 = REG ? xs[d] : s_x[d][sl];
                if (PM == 0) {
                    xn[d] = (PosT)wrap_f64((double)x0 + (double)disp[d], a.L[d]);
                    xln[d] = 0.0f;
                } else {
                    float h = (float)x0, lo = REG ? xl[d] : s_xl[d][sl];
                    pair_add_wrap(h, lo, (float)disp[d], a.Lf[d]);
                    xn[d] = (PosT)h;
                    xln[d] = lo;
                }
                fin = fin && finite_r(disp[d]);
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) fin = fin && finite_r(us[k]);
            const int Sprev = f0 & GCB_FLAG_S;
            const int Snew = isg ? 0 : 1;
            uint8_t nfl = (uint8_t)((f0 & 0xC0) | (Sprev ? GCB_FLAG_SPREV : 0) | (Snew ? GCB_FLAG_S : 0));
            // the particle goes straight back to its own index in the output
            // arrays (for a uniform tile, or an all-GCA or all-Boris one,
            // slot == thread and these stores are coalesced)
            const int64_t gi = tile * TPB + sl;
            if (fin) {
                if (fail) nfl |= GCB_FLAG_GCAFAIL;
                if (ncv) nfl |= GCB_FLAG_NONCONV;
                if (FUSE) {
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        s_x[d][sl] = xn[d];
                        if (PM) s_xl[d][sl] = xln[d];
                        s_d[d][sl] = disp[d];
                    }
#pragma unroll
                    for (int k = 0; k < 3; ++k) s_u[k][sl] = us[k];
                } else {
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        st_state(reinterpret_cast<PosT *>(a.x[d]) + gi, xn[d]);
                        if (PM) st_state(a.xlo[d] + gi, xln[d]);
                        st_state(a.dxp[d] + gi, disp[d]);
                    }
#pragma unroll
                    for (int k = 0; k < 3; ++k) st_state(a.u[k] + gi, us[k]);
                }
                if constexpr (DEP) {
                    // the step's out-of-plane velocity (2D): the guiding
                    // center's, or u_z^{n+1/2}/Gamma after a Boris step
                    R vz = R(0);
                    if constexpr (ND == 2)
                        vz = done ? vzg : us[2] / sqrt(R(1) + dot3(us, us) * sp.inv_c2);
                    R Qw = a.dq[(f0 >> GCB_SPECIES_SHIFT) & 3];
                    if (a.w) Qw *= ld_state(a.w + gi);
                    if (!deposit_path<R, ND>(a, ib, l, disp, Qw, vz, npc, nat)) ++nds;
                }
                if (done) ++ng; else ++nb;
                if (Sprev && !Snew) ++tg;
                if (!Sprev && Snew) ++tb;
                if (ncv) ++nc;
                if (fail) ++gf;
                si += it;
                mi = max(mi, (unsigned)it);
                R u2 = dot3(us, us) * sp.inv_c2;
                ek += (double)(u2 / (R(1) + sqrt(R(1) + u2)));
            } else {
                // not advanced: the input state is kept (copied when the input
                // is a sorted copy rather than the output arrays themselves;
                // fused, written to the slot, which a uniform 2D tile's first
                // step has not staged)
                nfl |= GCB_FLAG_NONFINITE;
                ++nf;
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const PosT x0 = REG ? xs[d] : s_x[d][sl];
                    const float l0 = PM ? (REG ? xl[d] : s_xl[d][sl]) : 0.0f;
                    const R d0 = REG ? dd[d] : s_d[d][sl];
                    if (FUSE) {
                        s_x[d][sl] = x0;
                        if (PM) s_xl[d][sl] = l0;
                        s_d[d][sl] = d0;
                    } else {
                        st_state(reinterpret_cast<PosT *>(a.x[d]) + gi, x0);
                        if (PM) st_state(a.xlo[d] + gi, l0);
                        st_state(a.dxp[d] + gi, d0);
                    }
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const R u0 = REG ? uu[k] : s_u[k][sl];
                    if (FUSE) s_u[k][sl] = u0; else st_state(a.u[k] + gi, u0);
                }
            }
            if (FUSE) s_fl[sl] = nfl; else st_state(a.flags + gi, nfl);
        }
        if (FUSE) __syncthreads();   // the slots hold this step's output
      }
      if (FUSE && valid) {
          // the tile's state after its nsteps steps, coalesced
#pragma unroll
          for (int d = 0; d < ND; ++d) {
              st_state(reinterpret_cast<PosT *>(a.x[d]) + i, s_x[d][tid]);
              if (PM) st_state(a.xlo[d] + i, s_xl[d][tid]);
              st_state(a.dxp[d] + i, s_d[d][tid]);
          }
#pragma unroll
          for (int k = 0; k < 3; ++k) st_state(a.u[k] + i, s_u[k][tid]);
          st_state(a.flags + i, s_fl[tid]);
      }
      pb ^= 1;
    }
    if (pf) cp_async_wait<0>();   // the last (empty) group

    // block reduction of the counters
    unsigned vals[9] = {nb, ng, tg, tb, nc, gf, nf, si, mi};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        unsigned v = __reduce_add_sync(0xffffffffu, vals[k]);
        if (lane == 0 && v) atomicAdd(&s_acc[k], (unsigned long long)v);
    }
    if constexpr (DEP) {
        const unsigned dv[3] = {nds, npc, nat};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const unsigned v = __reduce_add_sync(0xffffffffu, dv[k]);
            if (lane == 0 && v) atomicAdd(&a.stats[ST_DEPSKIP + k], (unsigned long long)v);
        }
    }
    unsigned m = __reduce_max_sync(0xffffffffu, vals[8]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ek += __shfl_xor_sync(0xffffffffu, ek, o);
    __syncthreads();
    if (lane == 0) {
        if (m) atomicMax(&s_acc[ST_MAX_ITER], (unsigned long long)m);
        atomicAdd(&s_ek, ek);
    }
    __syncthreads();
    if (tid < ST_MAX_ITER) {
        if (s_acc[tid]) atomicAdd(&a.stats[tid], s_acc[tid]);
    } else if (tid == ST_MAX_ITER) {
        if (s_acc[tid]) atomicMax(&a.stats[tid], s_acc[tid]);
    } else if (tid == ST_EKIN) {
        atomicAdd(reinterpret_cast<double *>(&a.stats[ST_EKIN]), s_ek);
    }
}

// ---------------------------------------------------------------------------
// host side: argument packing and launch
// ---------------------------------------------------------------------------
static bool device_memory(const void *ptr)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice;
}

template <typename R>
static void fill_args(PushArgs<R> &a, const gcb_particles *p, const gcb_particles *in,
                      const gcb_grid *g, const gcb_params *prm, unsigned long long *stats)
{
    a.g.rec = static_cast<const R *>(g->rec);
    a.g.stride = g->stride;
    for (int d = 0; d < 3; ++d) {
        a.g.n[d] = (int)g->n[d];
        a.g.nR[d] = (R)g->n[d];
        a.g.dx[d] = (R)g->dx[d];
        a.g.inv_dx[d] = (R)(1.0 / g->dx[d]);
        a.L[d] = (double)g->n[d] * g->dx[d];
        a.Lf[d] = (float)a.L[d];
        a.dxd[d] = g->dx[d];
        a.inv_dxd[d] = 1.0 / g->dx[d];
        a.x[d] = p->x[d];
        a.xlo[d] = static_cast<float *>(p->x_lo[d]);
        a.u[d] = static_cast<R *>(p->u[d]);
        a.dxp[d] = static_cast<R *>(p->dxp[d]);
        a.xin[d] = in->x[d];
        a.xloin[d] = static_cast<const float *>(in->x_lo[d]);
        a.uin[d] = static_cast<const R *>(in->u[d]);
        a.dxpin[d] = static_cast<const R *>(in->dxp[d]);
    }
    a.np = p->n;
    a.flags = p->flags;
    a.flagsin = in->flags;
    a.pid = p->pid;
    a.pidin = p->pid ? in->pid : nullptr;
    a.sp.c = (R)prm->c;
    a.sp.inv_c2 = (R)(1.0 / (prm->c * prm->c));
    a.sp.dt = (R)prm->dt;
    a.sp.half_dt = (R)(0.5 * prm->dt);
    a.sp.qm = R(0);
    a.sp.curvature = prm->curvature;
    a.sp.mu_mode = prm->mu_mode;
    a.sp.phase = prm->gyro_phase;
    a.sp.max_iter = prm->gca_max_iter;
    a.sp.fixed_iters = prm->gca_fixed_iters;
    a.sp.tol = (R)prm->gca_tol;
    for (int k = 0; k < 4; ++k) a.qm[k] = (R)prm->qm[k];
    a.rho_thr = (R)(prm->f_rho * prm->dl);
    a.f_E = (R)prm->f_E;
    a.c2 = (R)(prm->c * prm->c);
    a.force = prm->force;
    a.nsteps = 1;
    a.stats = stats;
    // the asynchronous copies of the state's next tile read device memory
    // only; a state in host (or managed) memory is read with plain loads
    a.pf = 1;
    for (int d = 0; d < g->ndim; ++d) {
        const void *arrs[3] = {in->x[d], in->dxp[d], in->pos_mode == GCB_POS_F32PAIR ? in->x_lo[d] : nullptr};
        for (const void *q : arrs)
            if (q && !device_memory(q)) a.pf = 0;
    }
    for (int k = 0; k < 3; ++k)
        if (!device_memory(in->u[k])) a.pf = 0;
}

template <typename R, int ND, int PM, int GM, bool FUSE, bool BT = false, bool DEP = false,
          bool MIR = false>
static gcb_status launch_push(const PushArgs<R> &a, cudaStream_t st)
{
    static int grid_cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        set_error("cudaGetDevice failed");
        return GCB_ECUDA;
    }
    int grid = grid_cache[dev];
    if (grid == 0) {
        int nsm = 0, occ = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_push_sr<R, ND, PM, GM, FUSE, BT, DEP, MIR>,
                                                          Tile<R, ND>::n, 0) !=
                cudaSuccess) {
            set_error("occupancy query failed: %s", cudaGetErrorString(cudaGetLastError()));
            return GCB_ECUDA;
        }
        grid = nsm * (occ > 0 ? occ : 1);
        grid_cache[dev] = grid;
    }
    constexpr int TPB = Tile<R, ND>::n;
    int64_t ntiles = (a.np + TPB - 1) / TPB;
    if (ntiles == 0) return GCB_OK;
    int nb = (int)(ntiles < grid ? ntiles : grid);
    k_push_sr<R, ND, PM, GM, FUSE, BT, DEP, MIR><<<nb, TPB, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("kernel launch failed: %s", cudaGetErrorString(e));
        return GCB_ECUDA;
    }
    return GCB_OK;
}

template <typename R, int PM, bool FUSE, bool BT = false, bool DEP = false, bool MIR = false>
static gcb_status dispatch_dims(const PushArgs<R> &a, const gcb_grid *g, const gcb_params *prm,
                                cudaStream_t st)
{
    const bool grid_grad = prm->grad_mode == GCB_GRAD_GRID;
    if (g->ndim == 2)
        return grid_grad ? launch_push<R, 2, PM, 2, FUSE, BT, DEP, MIR>(a, st)
                         : launch_push<R, 2, PM, 1, FUSE, BT, DEP, MIR>(a, st);
    return grid_grad ? launch_push<R, 3, PM, 2, FUSE, BT, DEP, MIR>(a, st)
                     : launch_push<R, 3, PM, 1, FUSE, BT, DEP, MIR>(a, st);
}

// Which (arithmetic, position) pairs carry kernels of the exact drift frame:
// FP64 and the FP32-pair positions of the mixed path.
template <typename R, int PM>
struct BtInstantiated : std::integral_constant<bool, sizeof(R) == 8 || PM == 1> {};

// nsteps > 1: that many steps in one launch (test-particle mode)
template <typename R, int PM>
static gcb_status dispatch_push(const gcb_particles *p, const gcb_particles *in, const gcb_grid *g,
                                const gcb_params *prm, cudaStream_t st, unsigned long long *stats,
                                int nsteps)
{
    PushArgs<R> a;
    fill_args<R>(a, p, in, g, prm, stats);
    if (prm->drift_frame == GCB_FRAME_BT) {
        // the exact drift frame: unfused launches only (checked by the caller)
        if constexpr (BtInstantiated<R, PM>::value) return dispatch_dims<R, PM, false, true>(a, g, prm, st);
        set_error("drift_frame GCB_FRAME_BT needs FP64 or FP32-pair positions");
        return GCB_EUNSUPPORTED;
    }
    if (nsteps <= 1) return dispatch_dims<R, PM, false>(a, g, prm, st);
    a.nsteps = nsteps;
    return dispatch_dims<R, PM, true>(a, g, prm, st);
}

// One unfused step with the mirror terms (simplified drift frame, no
// deposition; checked by the caller).
template <typename R, int PM>
static gcb_status dispatch_push_mir(const gcb_particles *p, const gcb_particles *in,
                                    const gcb_grid *g, const gcb_params *prm, cudaStream_t st,
                                    unsigned long long *stats)
{
    PushArgs<R> a;
    fill_args<R>(a, p, in, g, prm, stats);
    return dispatch_dims<R, PM, false, false, false, true>(a, g, prm, st);
}

// One unfused step with current deposition into cur, in the simplified or
// the exact drift frame, with or without the mirror terms (not both; checked
// by the caller).
template <typename R, int PM>
static gcb_status dispatch_push_dep(const gcb_particles *p, const gcb_particles *in,
                                    const gcb_grid *g, const gcb_params *prm,
                                    const gcb_current *cur, cudaStream_t st,
                                    unsigned long long *stats)
{
    PushArgs<R> a;
    fill_args<R>(a, p, in, g, prm, stats);
    double V = 1.0;
    for (int d = 0; d < g->ndim; ++d) V *= g->dx[d];
    for (int k = 0; k < 3; ++k) {
        a.J[k] = static_cast<R *>(cur->J[k]);
        a.jc[k] = k < g->ndim ? (R)(g->dx[k] / (prm->dt * V)) : R(0);
    }
    a.jz = (R)(1.0 / V);
    a.w = static_cast<const R *>(cur->w);
    for (int k = 0; k < 4; ++k) a.dq[k] = (R)cur->q[k];
    if (prm->mirror == GCB_MIRROR_ON) return dispatch_dims<R, PM, false, false, true, true>(a, g, prm, st);
    if (prm->drift_frame == GCB_FRAME_BT) {
        if constexpr (BtInstantiated<R, PM>::value) return dispatch_dims<R, PM, false, true, true>(a, g, prm, st);
        set_error("drift_frame GCB_FRAME_BT needs FP64 or FP32-pair positions");
        return GCB_EUNSUPPORTED;
    }
    return dispatch_dims<R, PM, false, false, true>(a, g, prm, st);
}

}  // namespace gcb
