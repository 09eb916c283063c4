// gcb_device.cuh -- per-particle arithmetic of the coupled guiding-center /
// Boris pusher (Bacchini et al. 2020), templated on the arithmetic type R
// (double for the FP64 path, float for the mixed path).
//
// Positions inside a step are "local": every point the step visits is held as
// an offset l (type R, physical units) from the origin of the particle's base
// cell ib (the cell of x^n).  Offsets stay within a few cells, so in FP32 they
// keep ~1e-7 cell resolution however large the box is; the absolute position
// is only touched at load and store (FP64 or an FP32 pair).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>
#include <type_traits>

namespace gcb {

template <typename R>
struct Eps;
template <>
struct Eps<float> {
    static constexpr float value = 1.1920929e-07f;
    static constexpr float tiny = 1e-30f;
};
template <>
struct Eps<double> {
    static constexpr double value = 2.220446049250313e-16;
    static constexpr double tiny = 1e-300;
};

// Grid as the kernels see it.
template <typename R>
struct DevGrid {
    const R *rec;       // node records, `stride` elements each
    int stride;
    int n[3];           // nodes per axis
    R nR[3];            // n as R
    R dx[3], inv_dx[3];
};

// Field point: E, B and d_i B_j (i < ND).
template <typename R, int ND>
struct FieldPt {
    R E[3], B[3];
    R dB[ND][3];
};

// Vector loads of one node record.  Records are 16-byte aligned and padded to
// whole 16-byte chunks.
__device__ __forceinline__ void load_chunk(const float *p, float *v)
{
    float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load_chunk(const double *p, double *v)
{
    double2 q = __ldg(reinterpret_cast<const double2 *>(p));
    v[0] = q.x; v[1] = q.y;
}
template <typename R>
struct Chunk { static constexpr int n = 16 / sizeof(R); };

// Cell of local offset l along axis d: fractional position t in the cell and
// the periodic node indices i0 (left) and i1 (right).  ib is in [0, n); the
// cell offset is clamped to [-n, n] (NaN to -n), so one conditional add or
// subtract of n always lands in [0, n): every access stays inside the grid
// whatever the offset (an offset of more than one box length, possible only
// for a broken step, is clamped rather than wrapped).
template <typename R>
__device__ __forceinline__ void cell_of(const DevGrid<R> &g, int d, int ib, R l, R &t, int &i0,
                                        int &i1)
{
    const int n = g.n[d];
    R s = l * g.inv_dx[d];
    R c = floor(s);
    t = s - c;
    c = fmin(fmax(c, -g.nR[d]), g.nR[d]);
    int i = ib + (int)c;
    i += i < 0 ? n : 0;
    i -= i >= n ? n : 0;
    int j = i + 1;
    j -= j >= n ? n : 0;
    i0 = i;
    i1 = j;
}

// Linear-shape-function gather (Sec. 4 intro): F(x) = sum_N F_N W(x - x_N),
// grad F(x) = sum_N F_N grad W(x - x_N), W the product of 1D hat functions.
// GM = 0: E and B only;  1: gradients of B from grad W (differentiate the
// interpolant inside the cell floor(x/dx));  2: gradients interpolated from
// the gradient block of the records.
template <typename R, int ND, int GM>
__device__ __forceinline__ void gather(const DevGrid<R> &g, const int ib[ND], const R l[ND],
                                       FieldPt<R, ND> &F)
{
    int i0[ND], i1[ND];
    R t[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) cell_of(g, d, ib[d], l[d], t[d], i0[d], i1[d]);
#pragma unroll
    for (int k = 0; k < 3; ++k) { F.E[k] = R(0); F.B[k] = R(0); }
    if (GM != 0) {
#pragma unroll
        for (int i = 0; i < ND; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) F.dB[i][j] = R(0);
    }
    constexpr int NC = 1 << ND;
    constexpr int CH = Chunk<R>::n;
    // elements needed from each record
    constexpr int NEED = (GM == 2) ? 6 + 3 * ND : 6;
    constexpr int NCHUNK = (NEED + CH - 1) / CH;
#pragma unroll
    for (int o = 0; o < NC; ++o) {
        int node;
        R w[ND];
        if (ND == 2) {
            int ix = (o & 1) ? i1[0] : i0[0];
            int iy = (o & 2) ? i1[1] : i0[1];
            node = iy * g.n[0] + ix;
        } else {
            int ix = (o & 1) ? i1[0] : i0[0];
            int iy = (o & 2) ? i1[1] : i0[1];
            int iz = (o & 4) ? i1[ND - 1] : i0[ND - 1];
            node = (iz * g.n[1] + iy) * g.n[0] + ix;
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) w[d] = ((o >> d) & 1) ? t[d] : R(1) - t[d];
        R W = w[0];
#pragma unroll
        for (int d = 1; d < ND; ++d) W *= w[d];
        R v[NCHUNK * CH];
        const R *rp = g.rec + (size_t)node * g.stride;
#pragma unroll
        for (int c = 0; c < NCHUNK; ++c) load_chunk(rp + c * CH, v + c * CH);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            F.E[k] = fma(v[k], W, F.E[k]);
            F.B[k] = fma(v[3 + k], W, F.B[k]);
        }
        if (GM == 1) {
#pragma unroll
            for (int i = 0; i < ND; ++i) {
                R gw = (((o >> i) & 1) ? g.inv_dx[i] : -g.inv_dx[i]);
#pragma unroll
                for (int e = 0; e < ND; ++e)
                    if (e != i) gw *= w[e];
#pragma unroll
                for (int j = 0; j < 3; ++j) F.dB[i][j] = fma(v[3 + j], gw, F.dB[i][j]);
            }
        } else if (GM == 2) {
#pragma unroll
            for (int i = 0; i < ND; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) F.dB[i][j] = fma(v[6 + 3 * i + j], W, F.dB[i][j]);
        }
    }
}

// FP32 gather with Blackwell's packed FP32x2 FMA: the record is consumed as
// float pairs, each node adds W * pair to a pair accumulator.  Same sums as
// gather<float> (one rounding per FMA), half the FMA instructions.
//
// It is split in three steps -- locate the cell, load its nodes' records,
// interpolate -- so that a particle whose next evaluation point lies in the
// cell it already loaded (the fixed-point iterates of one step almost
// always do) can interpolate again from the records it holds in registers:
// CellRecs below.  Both routes run the same interpolation on the same
// record values, so their results are bitwise equal.
template <int ND, int GM>
struct CellRecs {
    // float pairs per node: E0E1 E2B0 B1B2, then the gradient block's 3 ND
    // values (3D: the last pair's second half is the record's padding)
    static constexpr int NP = (GM == 2) ? (6 + 3 * ND + 1) / 2 : 3;
    static constexpr int NC = 1 << ND;
    float2 pr[NC][NP];
    int cell[ND];          // cell offsets from the base cell; INT_MIN: empty
    __device__ __forceinline__ void clear() { cell[0] = INT_MIN; }
};

// Cell of local offset l (as cell_of, split): fractional position t and the
// clamped cell offset c from the base cell.
__device__ __forceinline__ void cell_split(const DevGrid<float> &g, int d, float l, float &t, int &c)
{
    const float s = l * g.inv_dx[d];
    const float f = floorf(s);
    t = s - f;
    c = (int)fminf(fmaxf(f, -g.nR[d]), g.nR[d]);
}

// One 16-byte chunk of a node record.  The records are read many times per
// step (every particle of a cell, every gather of a step) while the particle
// state streams past once; with GCB_FIELD_L2_LAST the chunk is read under an
// L2 evict-last policy, so the state does not push the records out of L2.
// Off: the state's evict-first loads and stores already keep the records in
// L2, and the policy's instructions made the 2D push 0.6% slower (GB300,
// 2^24 particles).
#ifndef GCB_FIELD_L2_LAST
#define GCB_FIELD_L2_LAST 0
#endif
__device__ __forceinline__ float4 ld_record(const float4 *p)
{
    if constexpr (GCB_FIELD_L2_LAST) {
        uint64_t pol;
        asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
        float4 v;
        asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
            : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
            : "l"(__cvta_generic_to_global(p)), "l"(pol));
        return v;
    } else {
        return __ldg(p);
    }
}

// Load the records of the nodes of cell ib + c (periodic).
template <int ND, int GM>
__device__ __forceinline__ void load_cell(const DevGrid<float> &g, const int ib[ND], const int c[ND],
                                          CellRecs<ND, GM> &cr)
{
    int i0[ND], i1[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const int n = g.n[d];
        int i = ib[d] + c[d];
        i += i < 0 ? n : 0;
        i -= i >= n ? n : 0;
        int j = i + 1;
        j -= j >= n ? n : 0;
        i0[d] = i;
        i1[d] = j;
        cr.cell[d] = c[d];
    }
    constexpr int NQ = (2 * CellRecs<ND, GM>::NP + 3) / 4;   // float4 chunks read per record
#pragma unroll
    for (int o = 0; o < CellRecs<ND, GM>::NC; ++o) {
        int node;
        if (ND == 2) {
            int ix = (o & 1) ? i1[0] : i0[0];
            int iy = (o & 2) ? i1[1] : i0[1];
            node = iy * g.n[0] + ix;
        } else {
            int ix = (o & 1) ? i1[0] : i0[0];
            int iy = (o & 2) ? i1[1] : i0[1];
            int iz = (o & 4) ? i1[ND - 1] : i0[ND - 1];
            node = (iz * g.n[1] + iy) * g.n[0] + ix;
        }
        const float4 *rp = reinterpret_cast<const float4 *>(g.rec + (size_t)node * g.stride);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float4 v = ld_record(rp + q);
            if (2 * q < CellRecs<ND, GM>::NP) cr.pr[o][2 * q] = make_float2(v.x, v.y);
            if (2 * q + 1 < CellRecs<ND, GM>::NP) cr.pr[o][2 * q + 1] = make_float2(v.z, v.w);
        }
    }
}

// Interpolate at fractional position t in the loaded cell.
template <int ND, int GM>
__device__ __forceinline__ void interp_cell(const DevGrid<float> &g, const CellRecs<ND, GM> &cr,
                                            const float t[ND], FieldPt<float, ND> &F)
{
    constexpr int NP = CellRecs<ND, GM>::NP;
    float2 acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = make_float2(0.f, 0.f);
    float2 dacc[ND][2];                          // grad-W mode: d_i (B0,B1), d_i (B2,-)
    if (GM == 1) {
#pragma unroll
        for (int i = 0; i < ND; ++i) dacc[i][0] = dacc[i][1] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int o = 0; o < CellRecs<ND, GM>::NC; ++o) {
        float w[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) w[d] = ((o >> d) & 1) ? t[d] : 1.f - t[d];
        float W = w[0];
#pragma unroll
        for (int d = 1; d < ND; ++d) W *= w[d];
        const float2 W2 = make_float2(W, W);
#pragma unroll
        for (int k = 0; k < NP; ++k) acc[k] = __ffma2_rn(cr.pr[o][k], W2, acc[k]);
        if (GM == 1) {
            // pairs 1 and 2 hold (E2, B0) and (B1, B2)
            const float2 b01 = make_float2(cr.pr[o][1].y, cr.pr[o][2].x);
            const float2 b2 = make_float2(cr.pr[o][2].y, 0.f);
#pragma unroll
            for (int i = 0; i < ND; ++i) {
                float gw = ((o >> i) & 1) ? g.inv_dx[i] : -g.inv_dx[i];
#pragma unroll
                for (int e = 0; e < ND; ++e)
                    if (e != i) gw *= w[e];
                const float2 G2 = make_float2(gw, gw);
                dacc[i][0] = __ffma2_rn(b01, G2, dacc[i][0]);
                dacc[i][1] = __ffma2_rn(b2, G2, dacc[i][1]);
            }
        }
    }
    float v[2 * NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) { v[2 * k] = acc[k].x; v[2 * k + 1] = acc[k].y; }
#pragma unroll
    for (int k = 0; k < 3; ++k) { F.E[k] = v[k]; F.B[k] = v[3 + k]; }
    if (GM == 2) {
#pragma unroll
        for (int i = 0; i < ND; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) F.dB[i][j] = v[6 + 3 * i + j];
    } else if (GM == 1) {
#pragma unroll
        for (int i = 0; i < ND; ++i) {
            F.dB[i][0] = dacc[i][0].x;
            F.dB[i][1] = dacc[i][0].y;
            F.dB[i][2] = dacc[i][1].x;
        }
    }
}

template <int ND, int GM>
__device__ __forceinline__ void gather_x2(const DevGrid<float> &g, const int ib[ND],
                                          const float l[ND], FieldPt<float, ND> &F)
{
    float t[ND];
    int c[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) cell_split(g, d, l[d], t[d], c[d]);
    CellRecs<ND, GM> cr;
    load_cell<ND, GM>(g, ib, c, cr);
    interp_cell<ND, GM>(g, cr, t, F);
}

// Gather through the records held in cr: loaded again only when the point
// lies in another cell than the one cr holds.
template <int ND, int GM>
__device__ __forceinline__ void gather_cached(const DevGrid<float> &g, const int ib[ND],
                                              const float l[ND], FieldPt<float, ND> &F,
                                              CellRecs<ND, GM> &cr)
{
    float t[ND];
    int c[ND];
    bool hit = true;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        cell_split(g, d, l[d], t[d], c[d]);
        hit = hit && c[d] == cr.cell[d];
    }
    if (!hit) load_cell<ND, GM>(g, ib, c, cr);
    interp_cell<ND, GM>(g, cr, t, F);
}

// The gather used by the kernels: packed FP32x2 for float, scalar for double.
template <typename R, int ND, int GM>
__device__ __forceinline__ void gather_any(const DevGrid<R> &g, const int ib[ND], const R l[ND],
                                           FieldPt<R, ND> &F)
{
    if constexpr (sizeof(R) == 4)
        gather_x2<ND, GM>(g, ib, l, F);
    else
        gather<R, ND, GM>(g, ib, l, F);
}

template <typename R>
__device__ __forceinline__ R dot3(const R a[3], const R b[3])
{
    return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
}
template <typename R>
__device__ __forceinline__ void cross3(const R a[3], const R b[3], R r[3])
{
    r[0] = fma(a[1], b[2], -a[2] * b[1]);
    r[1] = fma(a[2], b[0], -a[0] * b[2]);
    r[2] = fma(a[0], b[1], -a[1] * b[0]);
}

// Kinematics of the simplified drift frame (Sec. 2.2): b = B/B,
// v_E = c E x B / B^2, kappa = (1 - v_E^2/c^2)^{-1/2}, E_par = E.b and the
// directional derivatives (b.grad)b, (v_E.grad)b, with
// d_i b_j = (d_i B_j - b_j (b . d_i B)) / B.
template <typename R>
struct Frame {
    R Bmag, ib, b[3], vE[3], kappa, Epar;
    R bgb[3], vgb[3];
    R gB[3];      // grad |B| (mirror terms only)
    bool ok;
};

// 1/sqrt(x): one reciprocal square root instruction in the arithmetic types
// of the kernels, the quotient for other types (dual numbers).
template <typename R>
__device__ __forceinline__ R inv_sqrt(R x) { return R(1) / sqrt(x); }
template <>
__device__ __forceinline__ float inv_sqrt<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double inv_sqrt<double>(double x) { return rsqrt(x); }

template <typename R>
__device__ __forceinline__ R one_minus_beta2(const R E[3], const R B[3], R B2, R c, R beta2)
{
    return R(1) - beta2;
}
// FP32: near |E| -> |B| the difference 1 - v_E^2/c^2 cancels; redo it in FP64.
template <>
__device__ __forceinline__ float one_minus_beta2<float>(const float E[3], const float B[3],
                                                        float B2, float c, float beta2)
{
    if (beta2 < 0.99f) return 1.0f - beta2;
    double e[3] = {E[0], E[1], E[2]}, b[3] = {B[0], B[1], B[2]};
    double x0 = e[1] * b[2] - e[2] * b[1];
    double x1 = e[2] * b[0] - e[0] * b[2];
    double x2 = e[0] * b[1] - e[1] * b[0];
    double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    // v_E^2 / c^2 = |E x B|^2 / B^4 (c cancels)
    double v2 = (x0 * x0 + x1 * x1 + x2 * x2) / (bb * bb);
    return (float)(1.0 - v2);
}

// Exact drift frame of Sec. 2.2 (Beklemishev & Tessarotto): the frame moving
// with v_E = (w_E/(2 w_E^2/c^2)) (1 - sqrt(1 - 4 w_E^2/c^2)), w_E = c E x B /
// (E^2 + B^2), sees E and B parallel along b* = xi E_perp + eta B, with
// E_perp = E - (E.B) B/B^2, B' = sqrt((B^2 - E^2 + (B^2 + E^2) s)/2),
// E' = E.B/B', Psi = E'(B^2 - B'^2)/(B' E_perp^2), eta = (B sqrt(Psi^2
// E_perp^2/B^2 + 1))^{-1}, xi = eta Psi.  Evaluated as
// s = sqrt((B^2 - E^2)^2 + 4 (E.B)^2)/(E^2 + B^2) (= sqrt(1 - 4 w_E^2/c^2)),
// v_E = 2 c E x B / ((E^2 + B^2)(1 + s)) and Psi = 2 E' B^2/(B' (E^2 + B^2)
// (1 + s)): the same quantities, free of the 0/0 of the printed forms at
// E x B = 0 and E_perp = 0.  om = 1 - v_E^2/c^2.
template <typename T>
__device__ __forceinline__ void bt_frame(const T E[3], const T B[3], T B2, T c, T vE[3], T bs[3],
                                         T &om)
{
    const T E2 = dot3(E, E), EB = dot3(E, B);
    const T S = E2 + B2, d = B2 - E2;
    const T sq = sqrt(fma(d, d, T(4) * EB * EB)) / S;
    T x[3];
    cross3(E, B, x);
    const T f = T(2) * c / (S * (T(1) + sq));
#pragma unroll
    for (int k = 0; k < 3; ++k) vE[k] = f * x[k];
    const T Bp = sqrt(T(0.5) * fma(S, sq, d));
    const T Ep = EB / Bp;
    const T ebb = EB / B2;
    T ep[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) ep[k] = fma(-ebb, B[k], E[k]);
    const T Ep2 = dot3(ep, ep);
    const T Psi = T(2) * Ep * B2 / (Bp * S * (T(1) + sq));
    const T eta = T(1) / (sqrt(B2) * sqrt(Psi * Psi * Ep2 / B2 + T(1)));
    const T xi = eta * Psi;
#pragma unroll
    for (int k = 0; k < 3; ++k) bs[k] = fma(xi, ep[k], eta * B[k]);
    om = T(1) - dot3(vE, vE) / (c * c);
}

// PROJ = false leaves out the projection of (b.grad)B and (v_E.grad)B onto
// the plane normal to b: every use of (b.grad)b and (v_E.grad)b in the step
// is b x (.) or v_E . (.), which annihilates the component along b (v_E is
// normal to B), so the step's results are the same up to rounding.
// BT = true builds the exact frame (bt_frame) in place of the simplified
// one: b*, the exact v_E and kappa from it, E_par = E.b*; the gradient terms
// are (b*.grad)b and (v_E.grad)b with grad b that of the lab-frame b = B/B
// (projected), the records carrying no grad E.
// MIR = true also forms grad |B|: d_i |B| = b_j d_i B_j (the mirror terms).
template <typename R, int ND, bool GRADS, bool PROJ = true, bool BT = false, bool MIR = false>
__device__ __forceinline__ void make_frame(const FieldPt<R, ND> &F, R c, R inv_c2, Frame<R> &f)
{
    if constexpr (BT) {
        R B2 = dot3(F.B, F.B);
        f.ok = B2 > R(0);
        if (!f.ok) B2 = R(1);
        f.Bmag = sqrt(B2);
        const R ib = R(1) / f.Bmag;
        f.ib = ib;
        R bl[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) bl[k] = F.B[k] * ib;
        R om;
        bt_frame<R>(F.E, F.B, B2, c, f.vE, f.b, om);
        if constexpr (sizeof(R) == 4) {
            if (!(om > R(0.01))) {   // near |v_E| -> c: 1 - v_E^2/c^2 again in FP64
                double e[3] = {F.E[0], F.E[1], F.E[2]}, bb[3] = {F.B[0], F.B[1], F.B[2]};
                double v[3], s_[3], o;
                bt_frame<double>(e, bb, (double)B2, (double)c, v, s_, o);
                om = (R)o;
            }
        }
        f.ok = f.ok && (om > R(0));
        f.kappa = R(1) / sqrt(f.ok ? om : R(1));
        f.Epar = dot3(F.E, f.b);
        if (GRADS) {
            R w[3], y[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                R sw = R(0), sy = R(0);
#pragma unroll
                for (int i = 0; i < ND; ++i) {
                    sw = fma(f.b[i], F.dB[i][j], sw);
                    sy = fma(f.vE[i], F.dB[i][j], sy);
                }
                w[j] = sw;
                y[j] = sy;
            }
            const R bw = dot3(bl, w), by = dot3(bl, y);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                f.bgb[j] = fma(-bl[j], bw, w[j]) * ib;
                f.vgb[j] = fma(-bl[j], by, y[j]) * ib;
            }
        }
        return;
    }
    R B2 = dot3(F.B, F.B);
    f.ok = B2 > R(0);
    if (!f.ok) B2 = R(1);
    R ib = PROJ ? R(1) / sqrt(B2) : inv_sqrt(B2);
    f.Bmag = PROJ ? sqrt(B2) : B2 * ib;
    if (PROJ) ib = R(1) / f.Bmag;
    f.ib = ib;
    R ib2 = ib * ib;
#pragma unroll
    for (int k = 0; k < 3; ++k) f.b[k] = F.B[k] * ib;
    R x[3];
    cross3(F.E, F.B, x);
#pragma unroll
    for (int k = 0; k < 3; ++k) f.vE[k] = c * x[k] * ib2;
    R beta2 = dot3(f.vE, f.vE) * inv_c2;
    R om = one_minus_beta2<R>(F.E, F.B, B2, c, beta2);
    f.ok = f.ok && (om > R(0));
    f.kappa = PROJ ? R(1) / sqrt(f.ok ? om : R(1)) : inv_sqrt(f.ok ? om : R(1));
    f.Epar = dot3(F.E, f.b);
    if (GRADS) {
        // w = (b.grad)B, y = (v_E.grad)B; then (b.grad)b = (w - b (b.w))/B etc.
        R w[3], y[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            R sw = R(0), sy = R(0);
#pragma unroll
            for (int i = 0; i < ND; ++i) {
                sw = fma(f.b[i], F.dB[i][j], sw);
                sy = fma(f.vE[i], F.dB[i][j], sy);
            }
            w[j] = sw;
            y[j] = sy;
        }
        if (PROJ) {
            R bw = dot3(f.b, w), by = dot3(f.b, y);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                f.bgb[j] = fma(-f.b[j], bw, w[j]) * ib;
                f.vgb[j] = fma(-f.b[j], by, y[j]) * ib;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                f.bgb[j] = w[j] * ib;
                f.vgb[j] = y[j] * ib;
            }
        }
        if constexpr (MIR) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
                f.gB[i] = i < ND ? dot3(f.b, F.dB[i]) : R(0);
        }
    }
}

// Parameters of one particle-step, in the arithmetic type.
template <typename R>
struct StepPar {
    R c, inv_c2, dt, half_dt, qm;
    int curvature, mu_mode, max_iter, fixed_iters;
    R tol;
    int phase;   // 1: the gyration phase advances over the step (GCB_PHASE_EVOLVE)
};

// Gyration energy term of Eq. (lfacgca2): 2 mu B kappa / m, or u_perp,g^2
// when u_perp,g is held instead of mu (energy-conserving alternative, Sec. 2.2).
template <typename R>
__device__ __forceinline__ R perp2(const Frame<R> &f, const StepPar<R> &s, R mu, R uperp)
{
    return s.mu_mode ? uperp * uperp : R(2) * mu * f.Bmag * f.kappa;
}

// Eq. (lfacgca2): Gamma(R, u_par) = kappa sqrt(1 + (u_par^2 + 2 mu B kappa/m)/c^2).
template <typename R>
__device__ __forceinline__ R gamma_gc(const Frame<R> &f, const StepPar<R> &s, R upar, R mu, R uperp)
{
    return f.kappa * sqrt(R(1) + fma(upar, upar, perp2(f, s, mu, uperp)) * s.inv_c2);
}

// Eq. (curvdrift): v_c = (m c kappa^2/(q B)) b x [(u_par^2/Gamma)(b.grad)b + u_par (v_E.grad)b].
template <typename R>
__device__ __forceinline__ void vcurv(const Frame<R> &f, const StepPar<R> &s, R upar, R G, R vc[3])
{
    if (!s.curvature) { vc[0] = vc[1] = vc[2] = R(0); return; }
    R a[3];
    R k2 = upar * upar / G;
#pragma unroll
    for (int k = 0; k < 3; ++k) a[k] = fma(k2, f.bgb[k], upar * f.vgb[k]);
    R x[3];
    cross3(f.b, a, x);
    R pref = s.c * f.kappa * f.kappa / (s.qm * f.Bmag);
#pragma unroll
    for (int k = 0; k < 3; ++k) vc[k] = pref * x[k];
}

// Guiding-center velocity, Eq. (dRdt): u_par b / Gamma + v_E + v_c.
template <typename R>
__device__ __forceinline__ void gc_vel(const Frame<R> &f, const StepPar<R> &s, R upar, R mu, R uperp,
                                       R V[3])
{
    R G = gamma_gc(f, s, upar, mu, uperp);
    R vc[3];
    vcurv(f, s, upar, G, vc);
    R ig = upar / G;
#pragma unroll
    for (int k = 0; k < 3; ++k) V[k] = fma(ig, f.b[k], f.vE[k] + vc[k]);
}

// The same two quantities from 1/Gamma and cq = c/(q/m), as the push
// evaluates them: v_c with prefactor cq kappa^2/B, and u_par b/Gamma + v_E +
// v_c with the one reciprocal of Gamma.
template <typename R>
__device__ __forceinline__ void vcurv_ig(const Frame<R> &f, const StepPar<R> &s, R cq, R upar, R iG,
                                         R vc[3])
{
    if (!s.curvature) { vc[0] = vc[1] = vc[2] = R(0); return; }
    R a[3];
    R k2 = upar * upar * iG;
#pragma unroll
    for (int k = 0; k < 3; ++k) a[k] = fma(k2, f.bgb[k], upar * f.vgb[k]);
    R x[3];
    cross3(f.b, a, x);
    R pref = cq * f.kappa * f.kappa * f.ib;
#pragma unroll
    for (int k = 0; k < 3; ++k) vc[k] = pref * x[k];
}

// MIR = true adds the grad-B drift (the mirror option): the term
// (mu/(m Gamma)) grad(B)/kappa in the bracket of v_c, i.e.
// v_gB = cq kappa mu/(Gamma B) b x grad B (mu as mu/m).
template <typename R, bool MIR = false>
__device__ __forceinline__ void gc_vel_ig(const Frame<R> &f, const StepPar<R> &s, R cq, R upar, R mu,
                                          R uperp, R V[3])
{
    R iG = R(1) / gamma_gc(f, s, upar, mu, uperp);
    R vc[3];
    vcurv_ig(f, s, cq, upar, iG, vc);
    if constexpr (MIR) {
        R x[3];
        cross3(f.b, f.gB, x);
        const R pg = cq * f.kappa * mu * iG * f.ib;
#pragma unroll
        for (int k = 0; k < 3; ++k) vc[k] = fma(pg, x[k], vc[k]);
    }
    R ig = upar * iG;
#pragma unroll
    for (int k = 0; k < 3; ++k) V[k] = fma(ig, f.b[k], f.vE[k] + vc[k]);
}

// Relativistic Boris push (Sec. 2.1, Boris 1970) with E, B at x^n:
// u- = u + hE, t = hB/(c gamma-), s = 2t/(1+t^2), u' = u- + u- x t,
// u+ = u- + u' x s, u^{n+1/2} = u+ + hE (h = q dt/2m); disp = dt u/gamma.
template <typename R, int ND>
__device__ __forceinline__ void boris(const R E[3], const R B[3], const StepPar<R> &s, R u[3],
                                      R disp[ND])
{
    R h = s.qm * s.half_dt;
    R um[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) um[k] = fma(h, E[k], u[k]);
    R gm = sqrt(R(1) + dot3(um, um) * s.inv_c2);
    R ht = h / (s.c * gm);
    R t[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = ht * B[k];
    R sf = R(2) / (R(1) + dot3(t, t));
    R x[3], up[3];
    cross3(um, t, x);
#pragma unroll
    for (int k = 0; k < 3; ++k) up[k] = um[k] + x[k];
    cross3(up, t, x);
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = fma(h, E[k], fma(sf, x[k], um[k]));
    R g = sqrt(R(1) + dot3(u, u) * s.inv_c2);
    R f = s.dt / g;
#pragma unroll
    for (int d = 0; d < ND; ++d) disp[d] = f * u[d];
}

// Guiding-center step (Sec. 3.1 with Sec. 2.2.1 / 2.2.2) from local x^n = ln
// in base cell ib (fields there: F0), previous displacement dxp and full
// u^{n-1/2}.  Returns
// false when the step cannot be taken (B = 0 or v_E >= c on the path, or no
// Lorentz factor >= 1 solves the quadratic); u and disp are then untouched.
// The gather the step uses: any callable gth(ib, l, F).  PlainGather is the
// kernels' (the grid's records in the arithmetic type); the adjoint kernel
// passes one that also records weights and seeds tangents.  A gatherer with
// kCellCache = true also offers gth.cached(ib, l, F, cr), which keeps the
// records of the last cell it loaded in cr (FP32: CellRecs); the step then
// passes every gather after the one at x^n through it.
// Which FP32 kernels keep the cell's records between gathers: measured on
// GB300, the 3D push (8 nodes of 2 record chunks per gather) gains 9%, the
// 2D push with gradient records (4 nodes of 3 chunks) loses 2-4% to the
// registers the records take.
#ifndef GCB_CELL_CACHE_2D
#define GCB_CELL_CACHE_2D 0
#endif
#ifndef GCB_CELL_CACHE_3D
#define GCB_CELL_CACHE_3D 1
#endif
template <typename R, int ND, int GM>
struct PlainGather {
    static constexpr bool kCellCache =
        sizeof(R) == 4 && (ND == 2 ? GCB_CELL_CACHE_2D : GCB_CELL_CACHE_3D);
    DevGrid<R> g;
    __device__ __forceinline__ void operator()(const int ib[ND], const R l[ND],
                                               FieldPt<R, ND> &F) const
    {
        gather_any<R, ND, GM>(g, ib, l, F);
    }
    template <typename C>
    __device__ __forceinline__ void cached(const int ib[ND], const R l[ND], FieldPt<R, ND> &F,
                                           C &cr) const
    {
        if constexpr (kCellCache) gather_cached<ND, GM>(g, ib, l, F, cr);
        else gather_any<R, ND, GM>(g, ib, l, F);
    }
};

template <typename G, typename = void>
struct HasCellCache : std::false_type {};
template <typename G>
struct HasCellCache<G, std::void_t<decltype(G::kCellCache)>>
    : std::integral_constant<bool, G::kCellCache> {};

struct NoCellRecs {
    __device__ __forceinline__ void clear() {}
};

// The records a gatherer keeps between the gathers of one step.
template <typename Gth, int ND, int GM>
using StepRecs = std::conditional_t<HasCellCache<Gth>::value, CellRecs<ND, GM>, NoCellRecs>;

// cr: the records the step's cached gathers start from (cleared, or those of
// the cell of x^n when the caller gathered there through them).  Fh: the
// fields at R^{n-1/2} = x^n - dxp/2 when the caller has gathered them already
// (the same gather the step would make), else null.
// MIR = true: with the mirror terms (grad-B drift in the guiding-center
// velocity, mirror force -(mu/Gamma) b.grad(B)/kappa explicit at
// (x^n, u_par^{n-1/2}) in the u_par update).
template <typename R, int ND, int GM, typename Gth, bool BT = false, bool MIR = false>
__device__ __forceinline__ bool gca_step_c(const Gth &gth, const StepPar<R> &s, const int ib[ND],
                                           const R ln[ND], const R dxp[ND],
                                           const FieldPt<R, ND> &F0, R u[3], R disp[ND],
                                           int &iters, bool &nonconv, StepRecs<Gth, ND, GM> &cr,
                                           const FieldPt<R, ND> *Fh = nullptr, R *vz = nullptr)
{
    constexpr bool CACHE = HasCellCache<Gth>::value;
    constexpr bool GR = (GM != 0);
    auto gat = [&](const R p[ND], FieldPt<R, ND> &Fo) {
        if constexpr (CACHE) gth.cached(ib, p, Fo, cr);
        else gth(ib, p, Fo);
    };
    const R cq = s.c / s.qm;
    FieldPt<R, ND> F;
    Frame<R> f0, f;
    make_frame<R, ND, GR, false, BT, MIR>(F0, s.c, s.inv_c2, f0);

    // conversion at R^{n-1/2} = x^n - dxp/2 (Sec. 3.1)
    R pt[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) pt[d] = fma(R(-0.5), dxp[d], ln[d]);
    if (Fh) F = *Fh;
    else gat(pt, F);
    make_frame<R, ND, GR, false, BT>(F, s.c, s.inv_c2, f);
    if (!(f0.ok && f.ok)) return false;
    R Gfull = sqrt(R(1) + dot3(u, u) * s.inv_c2);
    R upar = dot3(u, f.b);
    R vc[3];
    vcurv_ig(f, s, cq, upar, R(1) / Gfull, vc);
    R ug[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) ug[k] = u[k] - upar * f.b[k] - (f.vE[k] + vc[k]) * Gfull;
    R uperp = sqrt(dot3(ug, ug));
    R mu, bpg[3];
    if (uperp < Eps<R>::tiny) {
        uperp = R(0);
        mu = R(0);
        bpg[0] = bpg[1] = bpg[2] = R(0);
    } else {
        R iu = R(1) / uperp;
#pragma unroll
        for (int k = 0; k < 3; ++k) bpg[k] = ug[k] * iu;
        mu = uperp * uperp / (R(2) * f.Bmag * f.kappa);
    }

    // u_par update at R^n (Sec. 2.2.1 / Eqs. dupardtcase2discsol, duparprimedtcase2discsol)
    R upn;
    R fm = R(0);   // dt times the mirror force (MIR)
    if constexpr (MIR)
        fm = -s.dt * mu * dot3(f0.b, f0.gB) / (gamma_gc(f0, s, upar, mu, uperp) * f0.kappa);
    if (!s.curvature) {
        upn = fma(s.qm * s.dt, f0.Epar, upar) + fm;
    } else {
        R a = dot3(f0.vE, f0.bgb);
        R gg = dot3(f0.vE, f0.vgb);
        R D = fma(-s.half_dt, a, R(1));
        R G0 = gamma_gc(f0, s, upar, mu, uperp);
        R upr = fma(upar, fma(s.half_dt, a, R(1)), fma(s.qm * s.dt, f0.Epar, s.half_dt * G0 * gg));
        if constexpr (MIR) upr += fm;
        R c2 = s.c * s.c;
        R kap2 = f0.kappa * f0.kappa;
        R k1 = R(0.25) * s.dt * s.dt * gg * gg - c2 * D * D / kap2;
        R k2 = upr * s.dt * gg;
        R k3 = fma(upr, upr, (c2 + perp2(f0, s, mu, uperp)) * D * D);
        R disc = fma(k2, k2, R(-4) * k1 * k3);
        if (!(k1 < R(0)) || !(disc >= R(0)) || D == R(0)) return false;
        R sq = sqrt(disc);
        R q = R(-0.5) * (k2 + (k2 >= R(0) ? sq : -sq));
        R r1 = q / k1;
        R r2 = (q != R(0)) ? k3 / q : R(-1);
        R G1 = r1 >= r2 ? r1 : r2;
        if (!(G1 >= R(1))) return false;
        upn = fma(s.half_dt * G1, gg, upr) / D;
    }

    // fixed point on Eq. (dRdtcase2disc): R^{k+1} = R^n + dt/2 (V^n + V^k),
    // iterated on the displacement R^{k+1} - R^n from R^0 = R^n.
    R Vn[3];
    gc_vel_ig<R, MIR>(f0, s, cq, upn, mu, uperp, Vn);
    R dk[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) dk[d] = R(0);
    R V[3] = {Vn[0], Vn[1], Vn[2]};
    iters = 0;
    nonconv = false;
    bool okall = true;
    for (;;) {
        R res = R(0), big = R(0);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            R nd = s.half_dt * (Vn[d] + V[d]);
            R e = fabs(nd - dk[d]);
            res = fmax(res, e);
            big = fmax(big, fabs(nd));
            dk[d] = nd;
        }
        ++iters;
        if (s.fixed_iters > 0) {
            if (iters >= s.fixed_iters) break;
        } else {
            // FP32 floor: stop once the change is within 8 ulp of the displacement.
            if (res < s.tol || res <= R(8) * Eps<R>::value * big) break;
            if (iters >= s.max_iter) { nonconv = true; break; }
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) pt[d] = ln[d] + dk[d];
        gat(pt, F);
        make_frame<R, ND, GR, false, BT, MIR>(F, s.c, s.inv_c2, f);
        okall = okall && f.ok;   // a bad frame fails the step after the loop
        gc_vel_ig<R, MIR>(f, s, cq, upn, mu, uperp, V);
    }
    if (!okall) return false;

    // reconstruction at R^{n+1/2} = (R^{n+1} + R^n)/2 (Sec. 3.1)
#pragma unroll
    for (int d = 0; d < ND; ++d) pt[d] = fma(R(0.5), dk[d], ln[d]);
    gat(pt, F);
    make_frame<R, ND, GR, false, BT>(F, s.c, s.inv_c2, f);
    if (!f.ok) return false;
    R Gp = gamma_gc(f, s, upn, mu, uperp);
    vcurv_ig(f, s, cq, upn, R(1) / Gp, vc);
    R un = s.mu_mode ? uperp : sqrt(R(2) * mu * f.Bmag * f.kappa);
    if constexpr (std::is_floating_point<R>::value) {
        if (s.phase) {
            // evolved gyration phase: b_perp,g turns about b by the step's
            // gyro-phase phi = -(q/m) B dt/(c kappa Gamma) (the lab-time rate of
            // the gyration in the frame drifting with v_E), taken in FP64 (the
            // angle reaches Omega_C dt ~ 1e5 rad in strongly magnetized runs)
            const double phi = -(double)s.qm * (double)f.Bmag * (double)s.dt /
                               ((double)s.c * (double)f.kappa * (double)Gp);
            // the angle in half turns, wrapped into [-1, 1] (exact for the
            // multiples of 2 removed), then sin and cos of pi times it
            const double t = phi * 0.31830988618379067;   // 1/pi
            const double r = fma(-2.0, rint(0.5 * t), t);
            R sn, cs;
            if constexpr (sizeof(R) == 4) sincospif((float)r, &sn, &cs);
            else sincospi(r, &sn, &cs);
            R bxd[3];
            cross3(f.b, bpg, bxd);
#pragma unroll
            for (int k = 0; k < 3; ++k) bpg[k] = fma(cs, bpg[k], sn * bxd[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = fma(upn, f.b[k], fma(f.vE[k] + vc[k], Gp, un * bpg[k]));
#pragma unroll
    for (int d = 0; d < ND; ++d) disp[d] = dk[d];
    // out-of-plane component of the step's guiding-center velocity (V^n + V^K)/2
    // (2D current deposition); the in-plane ones are disp/dt
    if (vz) *vz = R(0.5) * (Vn[2] + V[2]);
    return true;
}

template <typename R, int ND, int GM, typename Gth>
__device__ __forceinline__ bool gca_step(const Gth &gth, const StepPar<R> &s, const int ib[ND],
                                         const R ln[ND], const R dxp[ND], const FieldPt<R, ND> &F0,
                                         R u[3], R disp[ND], int &iters, bool &nonconv)
{
    StepRecs<Gth, ND, GM> cr;
    cr.clear();
    return gca_step_c<R, ND, GM>(gth, s, ib, ln, dxp, F0, u, disp, iters, nonconv, cr);
}

}  // namespace gcb
