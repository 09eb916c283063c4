// dual.cuh -- forward-mode dual numbers for the adjoint kernel: a value and N
// tangent components.  The per-step arithmetic of gcb_device.cuh, instantiated
// on Dual<T, N>, carries N directional derivatives alongside every value;
// comparisons and rounding act on the value only, so control flow (branch,
// iteration count, cell index) is that of the plain evaluation.
#pragma once

#include <cuda_runtime.h>

#include "gcb_device.cuh"

namespace gcb {

// The overloads below would hide the global math functions from unqualified
// calls inside this namespace; keep those visible alongside.
using ::fabs;
using ::floor;
using ::fma;
using ::fmax;
using ::fmin;
using ::sqrt;

template <typename T, int N>
struct Dual {
    T v;
    T d[N];
    __device__ __forceinline__ Dual() {}
    __device__ __forceinline__ Dual(T x) : v(x)
    {
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = T(0);
    }
    __device__ __forceinline__ explicit operator int() const { return (int)v; }
    __device__ __forceinline__ Dual &operator+=(const Dual &b)
    {
        v += b.v;
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] += b.d[k];
        return *this;
    }
    __device__ __forceinline__ Dual &operator*=(const Dual &b)
    {
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = d[k] * b.v + v * b.d[k];
        v *= b.v;
        return *this;
    }
};

#define GCB_DUAL template <typename T, int N> __device__ __forceinline__

GCB_DUAL Dual<T, N> operator-(const Dual<T, N> &a)
{
    Dual<T, N> r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
    return r;
}
GCB_DUAL Dual<T, N> operator+(const Dual<T, N> &a, const Dual<T, N> &b)
{
    Dual<T, N> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
GCB_DUAL Dual<T, N> operator-(const Dual<T, N> &a, const Dual<T, N> &b)
{
    Dual<T, N> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
GCB_DUAL Dual<T, N> operator*(const Dual<T, N> &a, const Dual<T, N> &b)
{
    Dual<T, N> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = fma(a.d[k], b.v, a.v * b.d[k]);
    return r;
}
GCB_DUAL Dual<T, N> operator/(const Dual<T, N> &a, const Dual<T, N> &b)
{
    Dual<T, N> r;
    const T ib = T(1) / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}
GCB_DUAL Dual<T, N> operator+(const Dual<T, N> &a, T b) { return a + Dual<T, N>(b); }
GCB_DUAL Dual<T, N> operator+(T a, const Dual<T, N> &b) { return Dual<T, N>(a) + b; }
GCB_DUAL Dual<T, N> operator-(const Dual<T, N> &a, T b) { return a - Dual<T, N>(b); }
GCB_DUAL Dual<T, N> operator-(T a, const Dual<T, N> &b) { return Dual<T, N>(a) - b; }
GCB_DUAL Dual<T, N> operator*(const Dual<T, N> &a, T b)
{
    Dual<T, N> r;
    r.v = a.v * b;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b;
    return r;
}
GCB_DUAL Dual<T, N> operator*(T a, const Dual<T, N> &b) { return b * a; }
GCB_DUAL Dual<T, N> operator/(const Dual<T, N> &a, T b) { return a * (T(1) / b); }
GCB_DUAL Dual<T, N> operator/(T a, const Dual<T, N> &b) { return Dual<T, N>(a) / b; }

GCB_DUAL bool operator<(const Dual<T, N> &a, const Dual<T, N> &b) { return a.v < b.v; }
GCB_DUAL bool operator<=(const Dual<T, N> &a, const Dual<T, N> &b) { return a.v <= b.v; }
GCB_DUAL bool operator>(const Dual<T, N> &a, const Dual<T, N> &b) { return a.v > b.v; }
GCB_DUAL bool operator>=(const Dual<T, N> &a, const Dual<T, N> &b) { return a.v >= b.v; }
GCB_DUAL bool operator==(const Dual<T, N> &a, const Dual<T, N> &b) { return a.v == b.v; }
GCB_DUAL bool operator!=(const Dual<T, N> &a, const Dual<T, N> &b) { return a.v != b.v; }
GCB_DUAL bool operator<(const Dual<T, N> &a, T b) { return a.v < b; }
GCB_DUAL bool operator>(const Dual<T, N> &a, T b) { return a.v > b; }

GCB_DUAL Dual<T, N> fma(const Dual<T, N> &a, const Dual<T, N> &b, const Dual<T, N> &c)
{
    Dual<T, N> r;
    r.v = fma(a.v, b.v, c.v);
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = fma(a.d[k], b.v, fma(a.v, b.d[k], c.d[k]));
    return r;
}
GCB_DUAL Dual<T, N> sqrt(const Dual<T, N> &a)
{
    Dual<T, N> r;
    r.v = sqrt(a.v);
    const T h = r.v > T(0) ? T(0.5) / r.v : T(0);
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * h;
    return r;
}
GCB_DUAL Dual<T, N> fabs(const Dual<T, N> &a) { return a.v < T(0) ? -a : a; }
GCB_DUAL Dual<T, N> floor(const Dual<T, N> &a) { return Dual<T, N>(floor(a.v)); }
GCB_DUAL Dual<T, N> fmax(const Dual<T, N> &a, const Dual<T, N> &b) { return a.v >= b.v ? a : b; }
GCB_DUAL Dual<T, N> fmin(const Dual<T, N> &a, const Dual<T, N> &b) { return a.v <= b.v ? a : b; }

#undef GCB_DUAL

template <typename T, int N>
struct Eps<Dual<T, N>> {
    static constexpr T value = Eps<T>::value;
    static constexpr T tiny = Eps<T>::tiny;
};

}  // namespace gcb
