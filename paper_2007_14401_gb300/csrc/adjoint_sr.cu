// adjoint_sr.cu -- reverse-mode adjoint of the flat-space coupled push
// (2D, gradient-grid records), for gradients of trajectory observables with
// respect to the initial state and the field records.
//
// One particle-step maps s = (x, u, dxp) and the fields interpolated at the
// step's gather points F_g (12 components each) to s'.  Given the adjoint
// lambda' = dL/ds', the kernel forms
//     dL/ds   = (ds'/ds)^T lambda'                     (kept per particle)
//     dL/dF_g = (ds'/dF_g)^T lambda'                   (scattered to nodes)
// and a node record value f_N receives W_g(N) dL/dF_g, the linear shape
// function being the only way it enters the step.  The columns of the step's
// Jacobian come from replaying the step on dual numbers (value + N tangents)
// in registers, N directions per pass; the branch taken and the fixed-point
// iteration count are those of the plain replay (held fixed, not
// differentiated).  The sweep over steps runs backwards from checkpoints
// stored every `ckpt_every` steps, recomputing each segment forward.
#include <cuda_runtime.h>
#include <string.h>

#include "dual.cuh"
#include "gcb_internal.h"
#include "adjoint_rev.cuh"
#include "push_sr.cuh"

// Code size of the reverse kernel: its per-point pieces (gather + frame,
// frame transpose + scatter, and at level 2 the guiding-center velocity
// transpose and the replay's gather) are called out of line instead of being
// inlined at every gather point, which keeps the kernel's instruction
// footprint within the instruction caches.
#ifndef GCB_ADJ_OUTLINE
#define GCB_ADJ_OUTLINE 0
#endif
// GCB_ADJ_CACHE: cells (0, 1 or 2) whose node adjoints a thread accumulates
// in shared memory over a particle-step before adding them to the FP64 node
// accumulators (0: every gather's contributions are added directly).
#ifndef GCB_ADJ_CACHE
#define GCB_ADJ_CACHE 1
#endif
// GCB_ADJ_FCACHE: gather points (x^n first, then the step's gathers in order)
// whose interpolated field the replay keeps in shared memory for the reverse
// loop, which otherwise gathers again; points past it are re-gathered.
#ifndef GCB_ADJ_FCACHE
#define GCB_ADJ_FCACHE 6
#endif
#ifndef GCB_ADJ_BLOCKS_F32
#define GCB_ADJ_BLOCKS_F32 4
#endif
#if GCB_ADJ_OUTLINE >= 1
#define GCB_ADJ_FN1 __device__ __noinline__
#else
#define GCB_ADJ_FN1 __device__ __forceinline__
#endif
#if GCB_ADJ_OUTLINE >= 2
#define GCB_ADJ_FN2 __device__ __noinline__
#else
#define GCB_ADJ_FN2 __device__ __forceinline__
#endif

namespace gcb {
namespace adj {

constexpr int TPB = 128;
constexpr int NDIR = 4;          // tangent directions per pass
constexpr int MAXG = GCB_ADJOINT_MAX_ITER + 2;   // gathers per step: x^n, R^{n-1/2},
                                                // iterates 1..iters-1, R^{n+1/2}
constexpr int NF = 12;           // interpolated components per gather (2D, gradient grids)
constexpr int NS = 7;            // state directions: x(2), u(3), dxp(2)

// Gather on dual positions from plain records: the weights carry the
// position tangents; this pass's field directions are seeded on the result;
// nodes and weights of every gather are recorded for the scatter.
template <typename T, int N>
struct DualGather {
    DevGrid<T> g;
    int *count;
    int base;
    int *nodes;
    T *wts;
    __device__ __forceinline__ void operator()(const int ib[2], const Dual<T, N> l[2],
                                               FieldPt<Dual<T, N>, 2> &F) const
    {
        using D = Dual<T, N>;
        const int k = (*count)++;
        int i0[2], i1[2];
        D t[2];
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            T tv;
            cell_of(g, d, ib[d], l[d].v, tv, i0[d], i1[d]);
            const T c = floor(l[d].v * g.inv_dx[d]);
            t[d] = l[d] * g.inv_dx[d] - c;   // = tv, with the position's tangent
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) { F.E[c] = D(T(0)); F.B[c] = D(T(0)); }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) F.dB[i][j] = D(T(0));
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int ix = (o & 1) ? i1[0] : i0[0];
            const int iy = (o & 2) ? i1[1] : i0[1];
            const int node = iy * g.n[0] + ix;
            const D wx = (o & 1) ? t[0] : T(1) - t[0];
            const D wy = (o & 2) ? t[1] : T(1) - t[1];
            const D W = wx * wy;
            if (k < MAXG) {
                nodes[k * 4 + o] = node;
                wts[k * 4 + o] = W.v;
            }
            const T *rp = g.rec + (size_t)node * g.stride;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                F.E[c] = fma(W, D(__ldg(rp + c)), F.E[c]);
                F.B[c] = fma(W, D(__ldg(rp + 3 + c)), F.B[c]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) F.dB[i][j] = fma(W, D(__ldg(rp + 6 + 3 * i + j)), F.dB[i][j]);
        }
        // seed d(output)/d(F_k,c) for the directions of this pass
        const int d0 = NS + NF * k - base;
#pragma unroll
        for (int c = 0; c < NF; ++c) {
            const int j = d0 + c;
            if (j >= 0 && j < N) {
                D &f = c < 3 ? F.E[c] : (c < 6 ? F.B[c - 3] : F.dB[(c - 6) / 3][(c - 6) % 3]);
                f.d[j] += T(1);
            }
        }
    }
};

template <typename T>
struct AdjArgs {
    DevGrid<T> g;
    int64_t np;
    int pair;                    // positions as FP32 pairs
    const void *x[2];
    const float *xlo[2];
    const T *u[3];
    const T *dxp[2];
    const uint8_t *flags;
    T *lam[NS];                  // in: dL/d(state after the step); out: before it
    double *grad;                // node records' adjoint, stride 12 per node
    StepPar<T> sp;
    T qm[4];
    T rho_thr, f_E, c2;
    int force;
};

template <typename T>
__device__ __forceinline__ void load_pos(const AdjArgs<T> &a, int64_t i, int d, int &ib, T &l,
                                         bool &fin)
{
    if (a.pair) {
        const float h = ((const float *)a.x[d])[i], lo = a.xlo[d][i];
        fin = fin && isfinite(h) && isfinite(lo);
        float lf;
        split_pos_pair(h, lo, (float)a.g.dx[d], (float)a.g.inv_dx[d], (float)(a.g.n[d] - 1), ib, lf);
        l = (T)lf;
    } else {
        const double x = ((const double *)a.x[d])[i];
        fin = fin && isfinite(x);
        split_pos_f64<T>(x, (double)a.g.dx[d], 1.0 / (double)a.g.dx[d], (double)(a.g.n[d] - 1), ib, l);
    }
}

template <typename T, int N>
__global__ void __launch_bounds__(TPB) k_adjoint_sr(const AdjArgs<T> a)
{
    using D = Dual<T, N>;
    int nodes[MAXG * 4];
    T wts[MAXG * 4];
    for (int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x; i < a.np;
         i += (int64_t)gridDim.x * TPB) {
        const uint8_t fl = a.flags[i];
        bool fin = true;
        int ib[2];
        T l[2], u[3], dxp[2], lo[NS];
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            load_pos(a, i, d, ib[d], l[d], fin);
            dxp[d] = a.dxp[d][i];
            fin = fin && isfinite(dxp[d]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) { u[k] = a.u[k][i]; fin = fin && isfinite(u[k]); }
#pragma unroll
        for (int k = 0; k < NS; ++k) lo[k] = a.lam[k][i];
        if (!fin) continue;          // a frozen particle's step is the identity

        // plain replay: the switch, the branch and the iteration count
        StepPar<T> sp = a.sp;
        sp.qm = a.qm[(fl >> GCB_SPECIES_SHIFT) & 3];
        FieldPt<T, 2> F0;
        gather<T, 2, 2>(a.g, ib, l, F0);
        const T Q = fabs(sp.qm);
        const T G = sqrt(T(1) + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * sp.inv_c2);
        const T Bm = sqrt(F0.B[0] * F0.B[0] + F0.B[1] * F0.B[1] + F0.B[2] * F0.B[2]);
        const T Em = sqrt(F0.E[0] * F0.E[0] + F0.E[1] * F0.E[1] + F0.E[2] * F0.E[2]);
        int S = (a.c2 * G < a.rho_thr * Q * Bm && Em < a.f_E * Bm) ? 0 : 1;
        if (a.force == GCB_FORCE_BORIS) S = 1;
        if (a.force == GCB_FORCE_GCA) S = 0;
        int iters = 0;
        bool gca = false;
        if (S == 0) {
            T uu[3] = {u[0], u[1], u[2]}, disp[2];
            bool ncv;
            gca = gca_step<T, 2, 2>(PlainGather<T, 2, 2>{a.g}, sp, ib, l, dxp, F0, uu, disp, iters, ncv);
        }
        const int ngather = gca ? iters + 2 : 1;
        if (ngather > MAXG) continue;    // excluded by the host's iteration-cap check
        const int ndir = NS + NF * ngather;

        StepPar<D> sd;
        sd.c = D(sp.c);
        sd.inv_c2 = D(sp.inv_c2);
        sd.dt = D(sp.dt);
        sd.half_dt = D(sp.half_dt);
        sd.qm = D(sp.qm);
        sd.curvature = sp.curvature;
        sd.mu_mode = sp.mu_mode;
        sd.phase = 0;
        sd.max_iter = sp.max_iter;
        sd.fixed_iters = gca ? iters : sp.fixed_iters;   // replay exactly this many
        sd.tol = D(T(-1));
        T li[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) li[k] = T(0);
        for (int base = 0; base < ndir; base += N) {
            D ld[2], ud[3], dd[2];
#pragma unroll
            for (int d = 0; d < 2; ++d) { ld[d] = D(l[d]); dd[d] = D(dxp[d]); }
#pragma unroll
            for (int k = 0; k < 3; ++k) ud[k] = D(u[k]);
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const int dir = base + j;
                if (dir < 2) ld[dir].d[j] = T(1);
                else if (dir < 5) ud[dir - 2].d[j] = T(1);
                else if (dir < 7) dd[dir - 5].d[j] = T(1);
            }
            int count = 0;
            DualGather<T, N> gth{a.g, &count, base, nodes, wts};
            FieldPt<D, 2> Fd;
            gth(ib, ld, Fd);
            D disp[2];
            bool ok = false;
            if (gca) {
                int it2;
                bool ncv2;
                ok = gca_step<D, 2, 2>(gth, sd, ib, ld, dd, Fd, ud, disp, it2, ncv2);
            }
            if (!ok) boris<D, 2>(Fd.E, Fd.B, sd, ud, disp);
            // columns of this pass, contracted with the output adjoint
#pragma unroll
            for (int j = 0; j < N; ++j) {
                const int dir = base + j;
                if (dir >= ndir) break;
                T c = lo[2] * ud[0].d[j] + lo[3] * ud[1].d[j] + lo[4] * ud[2].d[j];
#pragma unroll
                for (int d = 0; d < 2; ++d)
                    c += lo[d] * (ld[d].d[j] + disp[d].d[j]) + lo[5 + d] * disp[d].d[j];
                if (dir < NS) {
                    li[dir] = c;
                } else if (c != T(0)) {
                    const int gk = (dir - NS) / NF, comp = (dir - NS) % NF;
#pragma unroll
                    for (int o = 0; o < 4; ++o)
                        atomicAdd(&a.grad[(size_t)nodes[gk * 4 + o] * 12 + comp],
                                  (double)(wts[gk * 4 + o] * c));
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NS; ++k) a.lam[k][i] = li[k];
    }
}

// ---------------------------------------------------------------------------
// reverse mode: replay the step recording its gather points, then run the
// transposed step backwards (adjoint_rev.cuh), re-gathering at each point.
// ---------------------------------------------------------------------------

template <typename T>
GCB_ADJ_FN2 void plain_gather2(const DevGrid<T> &g, const int ib[2], const T l[2], FieldPt<T, 2> &F)
{
    gather<T, 2, 2>(g, ib, l, F);
}

// Interpolated fields of the step's gather points, kept per thread in shared
// memory (thread-fastest: element (point, component) at [(point*NF+c)*TPB]).
// Point 0 is x^n, point 1 + k the step's k-th gather.
template <typename T>
struct FCache {
    T *base;
    __device__ __forceinline__ void store(int pt, const FieldPt<T, 2> &F) const
    {
        if (pt >= GCB_ADJ_FCACHE) return;
        T *q = base + pt * NF * TPB;
#pragma unroll
        for (int c = 0; c < 3; ++c) { q[c * TPB] = F.E[c]; q[(3 + c) * TPB] = F.B[c]; }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) q[(6 + 3 * i + j) * TPB] = F.dB[i][j];
    }
    __device__ __forceinline__ void load(int pt, FieldPt<T, 2> &F) const
    {
        const T *q = base + pt * NF * TPB;
#pragma unroll
        for (int c = 0; c < 3; ++c) { F.E[c] = q[c * TPB]; F.B[c] = q[(3 + c) * TPB]; }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) F.dB[i][j] = q[(6 + 3 * i + j) * TPB];
    }
};

// Plain gather that records where it was called (R^{n-1/2}, the iterates,
// R^{n+1/2}, in that order) and keeps what it interpolated.
template <typename T>
struct RecGather {
    DevGrid<T> g;
    T (*pts)[2];
    int *count;
    FCache<T> fc;
    __device__ __forceinline__ void operator()(const int ib[2], const T l[2], FieldPt<T, 2> &F) const
    {
        const int k = (*count)++;
        if (k < MAXG) {
            pts[k][0] = l[0];
            pts[k][1] = l[1];
        }
        plain_gather2(g, ib, l, F);
        fc.store(1 + k, F);
    }
};

// Node-record adjoints of one particle-step, accumulated per thread for up
// to GCB_ADJ_CACHE cells (4 nodes x 12 components each) in shared memory laid
// out thread-fastest, and added to the FP64 node accumulators when a cell is
// evicted and at the end of the step: the step's gathers (x^n, R^{n-1/2},
// the iterates, R^{n+1/2}) mostly share one cell, so this replaces most of
// the per-gather atomics.  (One cell measured faster than two: the second
// costs shared memory that the field cache uses better.)
template <typename T>
struct NodeCache {
    T *acc;          // this thread's slot 0 element; element (s, o, c) at acc[((s*4+o)*NF+c)*TPB]
    double *grad;
    int nx, ny;
    int key[2];      // lower-left node of the cached cell, -1 when empty
    int mru;         // most recently used slot

    __device__ __forceinline__ T &at(int sl, int o, int c) const
    {
        return acc[((sl * 4 + o) * NF + c) * TPB];
    }
    __device__ __forceinline__ void flush(int sl)
    {
        const int k = sl ? key[1] : key[0];
        if (k < 0) return;
        const int ix = k % nx, iy = k / nx;
        const int jx = ix + 1 == nx ? 0 : ix + 1, jy = iy + 1 == ny ? 0 : iy + 1;
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int node = ((o & 2) ? jy : iy) * nx + ((o & 1) ? jx : ix);
            double *gp = grad + (size_t)node * NF;
#pragma unroll
            for (int c = 0; c < NF; ++c) {
                const T v = at(sl, o, c);
                if (v != T(0)) atomicAdd(gp + c, (double)v);
            }
        }
    }
    // slot holding cell `k` (evicting the least recently used one if needed)
    __device__ __forceinline__ int slot(int k)
    {
        int sl;
        if (k == key[0]) {
            sl = 0;
        } else if (GCB_ADJ_CACHE > 1 && k == key[1]) {
            sl = 1;
        } else {
            sl = GCB_ADJ_CACHE > 1 ? 1 - mru : 0;
            flush(sl);
            if (sl) key[1] = k; else key[0] = k;
#pragma unroll
            for (int o = 0; o < 4; ++o)
#pragma unroll
                for (int c = 0; c < NF; ++c) at(sl, o, c) = T(0);
        }
        mru = sl;
        return sl;
    }
    __device__ __forceinline__ void finish()
    {
        flush(0);
        if (GCB_ADJ_CACHE > 1) flush(1);
        key[0] = key[1] = -1;
    }
};

// Transpose of F = sum_o W_o(p) rec_o: the node records receive W_o aF (via
// the cache) and the position adjoint sum_o grad W_o (rec_o . aF) is returned.
template <typename T>
__device__ __forceinline__ void gather_bwd(const DevGrid<T> &g, NodeCache<T> &nc, const int ib[2],
                                           const T p[2], const FieldPt<T, 2> &aF, T ap[2])
{
    int i0[2], i1[2];
    T t[2];
#pragma unroll
    for (int d = 0; d < 2; ++d) cell_of(g, d, ib[d], p[d], t[d], i0[d], i1[d]);
    T av[NF];
#pragma unroll
    for (int c = 0; c < 3; ++c) { av[c] = aF.E[c]; av[3 + c] = aF.B[c]; }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) av[6 + 3 * i + j] = aF.dB[i][j];
#if GCB_ADJ_CACHE
    const int sl = nc.slot(i0[1] * g.n[0] + i0[0]);
#endif
    ap[0] = ap[1] = T(0);
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const int ix = (o & 1) ? i1[0] : i0[0];
        const int iy = (o & 2) ? i1[1] : i0[1];
        const int node = iy * g.n[0] + ix;
        const T wx = (o & 1) ? t[0] : T(1) - t[0];
        const T wy = (o & 2) ? t[1] : T(1) - t[1];
        const T dwx = (o & 1) ? g.inv_dx[0] : -g.inv_dx[0];
        const T dwy = (o & 2) ? g.inv_dx[1] : -g.inv_dx[1];
        const T *rp = g.rec + (size_t)node * g.stride;
        // rec_o . aF, the record read in 16-byte chunks
        constexpr int CH = Chunk<T>::n;
        T dv = T(0);
#pragma unroll
        for (int q = 0; q < NF / CH; ++q) {
            T v[CH];
            load_chunk(rp + q * CH, v);
#pragma unroll
            for (int j = 0; j < CH; ++j) dv = fma(v[j], av[q * CH + j], dv);
        }
        ap[0] = fma(dwx * wy, dv, ap[0]);
        ap[1] = fma(wx * dwy, dv, ap[1]);
        const T W = wx * wy;
#if GCB_ADJ_CACHE
#pragma unroll
        for (int c = 0; c < NF; ++c) nc.at(sl, o, c) = fma(W, av[c], nc.at(sl, o, c));
#else
        double *gp = nc.grad + (size_t)node * NF;
#pragma unroll
        for (int c = 0; c < NF; ++c)
            if (av[c] != T(0)) atomicAdd(gp + c, (double)(W * av[c]));
#endif
    }
}

template <typename T>
GCB_ADJ_FN1 void gather_frame(const DevGrid<T> &g, const int ib[2], const T p[2],
                                             const StepPar<T> &s, FieldPt<T, 2> &F, Frame<T> &f)
{
    gather<T, 2, 2>(g, ib, p, F);
    make_frame<T, 2, true>(F, s.c, s.inv_c2, f);
}

// frame adjoint at gather point p -> node records and position adjoint
template <typename T>
GCB_ADJ_FN1 void frame_gather_bwd(const DevGrid<T> &g, NodeCache<T> &grad, const int ib[2],
                                                 const T p[2], const FieldPt<T, 2> &F,
                                                 const StepPar<T> &s, const rev::FrameAdj<T> &af,
                                                 T ap[2])
{
    FieldPt<T, 2> aF;
    rev::frame_bwd<T, 2>(F, s.c, s.inv_c2, af, aF);
    gather_bwd(g, grad, ib, p, aF, ap);
}

// Reverse sweep of a guiding-center step taken with K iterations whose gather
// points (R^{n-1/2}, x^n + d^1 .. x^n + d^{K-1}, R^{n+1/2}) are pts[0..K].
template <typename T>
GCB_ADJ_FN2 void vel_bwd(const Frame<T> &f, const StepPar<T> &s, T upn, T mu, T uperp,
                         const T aV[3], rev::FrameAdj<T> &af, T &aupn, T &amu, T &auperp)
{
    rev::gc_vel_bwd(f, s, upn, mu, uperp, aV, af, aupn, amu, auperp);
}

// u_par^{n+1/2} from the frame at x^n (the forward update of Sec. 2.2.1 / 2.2.2)
template <typename T>
__device__ __forceinline__ T upar_new(const Frame<T> &f0, const StepPar<T> &s, T upar, T mu, T uperp)
{
    if (!s.curvature) return fma(s.qm * s.dt, f0.Epar, upar);
    const T A = dot3(f0.vE, f0.bgb);
    const T gg = dot3(f0.vE, f0.vgb);
    const T D = fma(-s.half_dt, A, T(1));
    const T G0 = gamma_gc(f0, s, upar, mu, uperp);
    const T upr = fma(upar, fma(s.half_dt, A, T(1)), fma(s.qm * s.dt, f0.Epar, s.half_dt * G0 * gg));
    const T c2 = s.c * s.c;
    const T kap2 = f0.kappa * f0.kappa;
    const T k1 = T(0.25) * s.dt * s.dt * gg * gg - c2 * D * D / kap2;
    const T k2 = upr * s.dt * gg;
    const T k3 = fma(upr, upr, (c2 + perp2(f0, s, mu, uperp)) * D * D);
    const T disc = fma(k2, k2, T(-4) * k1 * k3);
    const T sq = sqrt(disc);
    const T q = T(-0.5) * (k2 + (k2 >= T(0) ? sq : -sq));
    const T r1 = q / k1;
    const T r2 = (q != T(0)) ? k3 / q : T(-1);
    const T G1 = r1 >= r2 ? r1 : r2;
    return fma(s.half_dt * G1, gg, upr) / D;
}

// Reverse sweep of a guiding-center step taken with K iterations whose gather
// points (R^{n-1/2}, x^n + d^1 .. x^n + d^{K-1}, R^{n+1/2}) are pts[0..K].
// One loop over the step's gather points in reverse order of their use:
//   stage 0        R^{n+1/2}: reconstruction of u
//   stage 1..K-1   x^n + d^{K-stage}: the iterate's velocity V^{K-stage}
//   stage K        x^n: V^n and the u_par update
//   stage K+1      R^{n-1/2}: conversion of u
// so that the gather, frame and scatter code is present once.
// field and frame at gather point `pt` (FCache numbering) located at p
template <typename T>
__device__ __forceinline__ void frame_at(const DevGrid<T> &g, const FCache<T> &fc, int pt,
                                         const int ib[2], const T p[2], const StepPar<T> &s,
                                         FieldPt<T, 2> &F, Frame<T> &f)
{
    if (pt < GCB_ADJ_FCACHE) {
        fc.load(pt, F);
        make_frame<T, 2, true>(F, s.c, s.inv_c2, f);
    } else {
        gather_frame(g, ib, p, s, F, f);
    }
}

template <typename T>
__device__ __forceinline__ void gca_rev(const DevGrid<T> &g, NodeCache<T> &grad, const FCache<T> &fc,
                                        const StepPar<T> &s, const int ib[2], const T l[2],
                                        const T u[3], int K, const T (*pts)[2], const T lo[NS],
                                        T li[NS])
{
    using rev::FrameAdj;
    FieldPt<T, 2> F;
    Frame<T> f;
    // forward quantities of the conversion (at R^{n-1/2}) and of the u_par update (at x^n)
    T Gf, upar, vcm[3], uperp, mu, bpg[3], upn;
    for (int j = 0; j < 2; ++j) {
        frame_at(g, fc, j == 0 ? 1 : 0, ib, j == 0 ? pts[0] : l, s, F, f);
        if (j == 0) rev::conv_fwd(f, s, u, Gf, upar, vcm, uperp, mu, bpg);
        else upn = upar_new(f, s, upar, mu, uperp);
    }
    T aupn = T(0), amu = T(0), auperp = T(0), aupar = T(0);
    T abpg[3] = {T(0), T(0), T(0)}, au[3] = {T(0), T(0), T(0)};
    T al[2] = {lo[0], lo[1]};
    T ad[2] = {lo[0] + lo[5], lo[1] + lo[6]};      // x^{n+1} = x^n + d^K, dxp = d^K
    T aVn[3] = {T(0), T(0), T(0)};
    for (int st = 0; st <= K + 1; ++st) {
        const T *p = st == 0 ? pts[K] : (st < K ? pts[K - st] : (st == K ? l : pts[0]));
        const int pt = st == 0 ? K + 1 : (st < K ? K - st + 1 : (st == K ? 0 : 1));
        frame_at(g, fc, pt, ib, p, s, F, f);
        FrameAdj<T> af;
        af.zero();
        if (st == 0) {
            const T lu[3] = {lo[2], lo[3], lo[4]};
            rev::recon_bwd(f, s, upn, mu, uperp, bpg, lu, af, aupn, amu, auperp, abpg);
        } else if (st <= K) {
            // d^k = dt/2 (V^n + V^{k-1}) with V^0 = V^n: stage st < K carries
            // V^{K-st}; stage K carries V^n with every term collected
            T aV[3];
            if (st < K) {
                aV[0] = s.half_dt * ad[0];
                aV[1] = s.half_dt * ad[1];
                aVn[0] += aV[0];
                aVn[1] += aV[1];
            } else {
                aV[0] = aVn[0] + s.dt * ad[0];
                aV[1] = aVn[1] + s.dt * ad[1];
            }
            aV[2] = T(0);
            vel_bwd(f, s, upn, mu, uperp, aV, af, aupn, amu, auperp);
            if (st == K) rev::upar_bwd(f, s, upar, mu, uperp, aupn, af, aupar, amu, auperp);
        } else {
            rev::conv_bwd(f, s, u, Gf, upar, vcm, uperp, mu, bpg, aupar, amu, auperp, abpg, af, au);
        }
        T ap[2];
        frame_gather_bwd(g, grad, ib, p, F, s, af, ap);
        al[0] += ap[0];
        al[1] += ap[1];
        if (st == 0) {                 // R^{n+1/2} = x^n + d^K / 2
            ad[0] += T(0.5) * ap[0];
            ad[1] += T(0.5) * ap[1];
        } else if (st < K) {           // x^n + d^{K-st}
            ad[0] = ap[0];
            ad[1] = ap[1];
        } else if (st == K + 1) {      // R^{n-1/2} = x^n - dxp / 2
            li[5] = T(-0.5) * ap[0];
            li[6] = T(-0.5) * ap[1];
        }
    }
    li[0] = al[0];
    li[1] = al[1];
    li[2] = au[0];
    li[3] = au[1];
    li[4] = au[2];
}

// resident blocks per SM the reverse kernel is compiled for (FP32: 4, i.e.
// at most 128 registers; FP64 kernels need more registers than that allows)
template <typename T> struct RevBlocks { static constexpr int n = GCB_ADJ_BLOCKS_F32; };
template <> struct RevBlocks<double> { static constexpr int n = 1; };

template <typename T>
__global__ void __launch_bounds__(TPB, RevBlocks<T>::n) k_adjoint_rev(const AdjArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char s_raw[];
    T pts[MAXG][2];
    NodeCache<T> nc;
    nc.acc = reinterpret_cast<T *>(s_raw) + threadIdx.x;
    const FCache<T> fc{reinterpret_cast<T *>(s_raw) + GCB_ADJ_CACHE * 4 * NF * TPB + threadIdx.x};
    nc.grad = a.grad;
    nc.nx = a.g.n[0];
    nc.ny = a.g.n[1];
    nc.key[0] = nc.key[1] = -1;
    nc.mru = 1;
    for (int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x; i < a.np;
         i += (int64_t)gridDim.x * TPB) {
        const uint8_t fl = a.flags[i];
        bool fin = true;
        int ib[2];
        T l[2], u[3], dxp[2], lo[NS];
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            load_pos(a, i, d, ib[d], l[d], fin);
            dxp[d] = a.dxp[d][i];
            fin = fin && isfinite(dxp[d]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) { u[k] = a.u[k][i]; fin = fin && isfinite(u[k]); }
#pragma unroll
        for (int k = 0; k < NS; ++k) lo[k] = a.lam[k][i];
        if (!fin) continue;          // a frozen particle's step is the identity

        StepPar<T> sp = a.sp;
        sp.qm = a.qm[(fl >> GCB_SPECIES_SHIFT) & 3];
        FieldPt<T, 2> F0;
        gather<T, 2, 2>(a.g, ib, l, F0);
        fc.store(0, F0);
        const T Q = fabs(sp.qm);
        const T G = sqrt(T(1) + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * sp.inv_c2);
        const T Bm = sqrt(F0.B[0] * F0.B[0] + F0.B[1] * F0.B[1] + F0.B[2] * F0.B[2]);
        const T Em = sqrt(F0.E[0] * F0.E[0] + F0.E[1] * F0.E[1] + F0.E[2] * F0.E[2]);
        int S = (a.c2 * G < a.rho_thr * Q * Bm && Em < a.f_E * Bm) ? 0 : 1;
        if (a.force == GCB_FORCE_BORIS) S = 1;
        if (a.force == GCB_FORCE_GCA) S = 0;
        int K = 0;
        bool gca = false;
        if (S == 0) {
            T uu[3] = {u[0], u[1], u[2]}, disp[2];
            bool ncv;
            int cnt = 0;
            gca = gca_step<T, 2, 2>(RecGather<T>{a.g, pts, &cnt, fc}, sp, ib, l, dxp, F0, uu, disp, K, ncv);
            gca = gca && cnt == K + 1 && cnt <= MAXG;
        }
        T li[NS];
        if (gca) {
            gca_rev(a.g, nc, fc, sp, ib, l, u, K, pts, lo, li);
        } else {
            T lu[3] = {lo[2], lo[3], lo[4]};
            T ldisp[2] = {lo[0] + lo[5], lo[1] + lo[6]};
            T au[3], aE[3], aB[3];
            rev::boris_bwd<T, 2>(F0.E, F0.B, sp, u, lu, ldisp, au, aE, aB);
            FieldPt<T, 2> aF;
#pragma unroll
            for (int c = 0; c < 3; ++c) { aF.E[c] = aE[c]; aF.B[c] = aB[c]; }
#pragma unroll
            for (int ii = 0; ii < 2; ++ii)
#pragma unroll
                for (int j = 0; j < 3; ++j) aF.dB[ii][j] = T(0);
            T ap[2];
            gather_bwd(a.g, nc, ib, l, aF, ap);
            li[0] = lo[0] + ap[0];
            li[1] = lo[1] + ap[1];
            li[2] = au[0];
            li[3] = au[1];
            li[4] = au[2];
            li[5] = T(0);
            li[6] = T(0);
        }
#if GCB_ADJ_CACHE
        nc.finish();
#endif
#pragma unroll
        for (int k = 0; k < NS; ++k) a.lam[k][i] = li[k];
    }
}

template <typename T>
constexpr int rev_smem()
{
    return (GCB_ADJ_CACHE * 4 + GCB_ADJ_FCACHE) * NF * TPB * (int)sizeof(T);
}

template <typename T>
static gcb_status launch(const AdjArgs<T> &a, int method, cudaStream_t st)
{
    if (a.np == 0) return GCB_OK;
    int64_t nb = (a.np + TPB - 1) / TPB;
    if (nb > 152 * 64) nb = 152 * 64;
    if (method == GCB_ADJ_REVERSE) {
        cudaError_t e = cudaFuncSetAttribute(k_adjoint_rev<T>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             rev_smem<T>());
        if (e != cudaSuccess) {
            set_error("k_adjoint_rev smem attribute: %s", cudaGetErrorString(e));
            return GCB_ECUDA;
        }
        k_adjoint_rev<T><<<(int)nb, TPB, rev_smem<T>(), st>>>(a);
    }
    else
        k_adjoint_sr<T, NDIR><<<(int)nb, TPB, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("k_adjoint_sr launch: %s", cudaGetErrorString(e));
        return GCB_ECUDA;
    }
    return GCB_OK;
}

}  // namespace adj

// The adjoint of one step for all particles whose pre-step state is `s`.
gcb_status adjoint_step(const gcb_particles *s, const gcb_grid *g, const gcb_params *prm,
                        void *const lam[7], double *grad, int method, cudaStream_t st)
{
    auto fill = [&](auto &a, auto tag) {
        using T = decltype(tag);
        a.g.rec = static_cast<const T *>(g->rec);
        a.g.stride = g->stride;
        for (int d = 0; d < 3; ++d) {
            a.g.n[d] = (int)g->n[d];
            a.g.nR[d] = (T)g->n[d];
            a.g.dx[d] = (T)g->dx[d];
            a.g.inv_dx[d] = (T)(1.0 / g->dx[d]);
        }
        a.np = s->n;
        a.pair = s->pos_mode == GCB_POS_F32PAIR;
        for (int d = 0; d < 2; ++d) {
            a.x[d] = s->x[d];
            a.xlo[d] = static_cast<const float *>(s->x_lo[d]);
            a.dxp[d] = static_cast<const T *>(s->dxp[d]);
        }
        for (int k = 0; k < 3; ++k) a.u[k] = static_cast<const T *>(s->u[k]);
        a.flags = s->flags;
        for (int k = 0; k < 7; ++k) a.lam[k] = static_cast<T *>(lam[k]);
        a.grad = grad;
        a.sp.c = (T)prm->c;
        a.sp.inv_c2 = (T)(1.0 / (prm->c * prm->c));
        a.sp.dt = (T)prm->dt;
        a.sp.half_dt = (T)(0.5 * prm->dt);
        a.sp.qm = T(0);
        a.sp.curvature = prm->curvature;
        a.sp.mu_mode = prm->mu_mode;
        a.sp.phase = 0;   // the adjoint differentiates the step with the direction kept
        a.sp.max_iter = prm->gca_max_iter;
        a.sp.fixed_iters = prm->gca_fixed_iters;
        a.sp.tol = (T)prm->gca_tol;
        for (int k = 0; k < 4; ++k) a.qm[k] = (T)prm->qm[k];
        a.rho_thr = (T)(prm->f_rho * prm->dl);
        a.f_E = (T)prm->f_E;
        a.c2 = (T)(prm->c * prm->c);
        a.force = prm->force;
    };
    if (s->mom_dtype == GCB_F64) {
        adj::AdjArgs<double> a;
        fill(a, 0.0);
        return adj::launch(a, method, st);
    }
    adj::AdjArgs<float> a;
    fill(a, 0.0f);
    return adj::launch(a, method, st);
}

}  // namespace gcb

// ---------------------------------------------------------------------------
// mode projection and field combination (fields linear in mode amplitudes)
// ---------------------------------------------------------------------------
namespace gcb {
namespace adj {

// dL/da_m = sum_e grad[e] pat_m[e]; grid row m = blockIdx.y.
template <typename PT>
__global__ void __launch_bounds__(256) k_project(const double *grad, const PT *pat, int64_t nelem,
                                                 double *out)
{
    __shared__ double s_w[8];
    const int m = blockIdx.y;
    const PT *pm = pat + (size_t)m * nelem;
    double acc = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nelem;
         e += (int64_t)gridDim.x * blockDim.x)
        acc = fma(grad[e], (double)pm[e], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w];
        atomicAdd(&out[m], t);
    }
}

template <typename PT>
__global__ void k_combine(PT *rec, const PT *base, const PT *pat, const double *amps, int64_t nelem,
                          int nmodes)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nelem;
         e += (int64_t)gridDim.x * blockDim.x) {
        double v = (double)base[e];
        for (int m = 0; m < nmodes; ++m) v = fma(amps[m], (double)pat[(size_t)m * nelem + e], v);
        rec[e] = (PT)v;
    }
}

}  // namespace adj

gcb_status grad_project(const gcb_grid *g, const double *grad, const void *pat, int nmodes,
                        double *out, cudaStream_t st)
{
    const int64_t nelem = g->n[0] * g->n[1] * g->n[2] * (int64_t)g->stride;
    if (cudaMemsetAsync(out, 0, sizeof(double) * nmodes, st) != cudaSuccess) {
        set_error("cudaMemsetAsync: %s", cudaGetErrorString(cudaGetLastError()));
        return GCB_ECUDA;
    }
    int64_t nb = (nelem + 255) / 256;
    if (nb > 152 * 4) nb = 152 * 4;
    const dim3 grid((unsigned)nb, (unsigned)nmodes);
    if (g->dtype == GCB_F32)
        adj::k_project<float><<<grid, 256, 0, st>>>(grad, (const float *)pat, nelem, out);
    else
        adj::k_project<double><<<grid, 256, 0, st>>>(grad, (const double *)pat, nelem, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_error("k_project: %s", cudaGetErrorString(e)); return GCB_ECUDA; }
    return GCB_OK;
}

gcb_status grid_combine(const gcb_grid *g, const void *base, const void *pat, const double *amps,
                        int nmodes, cudaStream_t st)
{
    const int64_t nelem = g->n[0] * g->n[1] * g->n[2] * (int64_t)g->stride;
    int64_t nb = (nelem + 255) / 256;
    if (nb > 152 * 32) nb = 152 * 32;
    if (g->dtype == GCB_F32)
        adj::k_combine<float><<<(int)nb, 256, 0, st>>>((float *)g->rec, (const float *)base,
                                                       (const float *)pat, amps, nelem, nmodes);
    else
        adj::k_combine<double><<<(int)nb, 256, 0, st>>>((double *)g->rec, (const double *)base,
                                                        (const double *)pat, amps, nelem, nmodes);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_error("k_combine: %s", cudaGetErrorString(e)); return GCB_ECUDA; }
    return GCB_OK;
}

}  // namespace gcb
