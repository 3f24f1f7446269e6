// lbfd_dual.cuh -- forward-mode (tangent-linear) numbers for the step kernel.
//
// Dual<T, N> carries a value and N directional derivatives.  Every
// arithmetic operation of the step propagates the derivatives by the chain
// rule, so the unchanged step kernel instantiated with this type computes,
// alongside the state, its exact derivative with respect to N parameters
// (the derivative of the discrete scheme, branch decisions such as the
// WENO upwind side or max(Y, 0) taken on the values).
#pragma once
#include <cmath>

namespace lbfd {

template <typename T, int N>
struct Dual {
    T v;
    T d[N];

    __host__ __device__ Dual() {}
    // constants and converted plain values carry no derivative
    __host__ __device__ Dual(double x) : v(T(x))
    {
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = T(0);
    }
    __host__ __device__ Dual(int x) : Dual(double(x)) {}

    __host__ __device__ Dual& operator+=(const Dual& b)
    {
        v += b.v;
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] += b.d[k];
        return *this;
    }
    __host__ __device__ Dual& operator-=(const Dual& b)
    {
        v -= b.v;
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] -= b.d[k];
        return *this;
    }
    __host__ __device__ Dual& operator*=(const Dual& b)
    {
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = d[k] * b.v + v * b.d[k];
        v *= b.v;
        return *this;
    }
};

template <typename T, int N>
__host__ __device__ inline Dual<T, N> operator+(Dual<T, N> a, const Dual<T, N>& b) { return a += b; }
template <typename T, int N>
__host__ __device__ inline Dual<T, N> operator-(Dual<T, N> a, const Dual<T, N>& b) { return a -= b; }
template <typename T, int N>
__host__ __device__ inline Dual<T, N> operator*(Dual<T, N> a, const Dual<T, N>& b) { return a *= b; }
template <typename T, int N>
__host__ __device__ inline Dual<T, N> operator-(const Dual<T, N>& a)
{
    Dual<T, N> r;
    r.v = -a.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
    return r;
}
template <typename T, int N>
__host__ __device__ inline Dual<T, N> operator/(const Dual<T, N>& a, const Dual<T, N>& b)
{
    Dual<T, N> r;
    const T inv = T(1) / b.v;
    r.v = a.v * inv;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * inv;
    return r;
}
template <typename T, int N>
__host__ __device__ inline Dual<T, N>& operator/=(Dual<T, N>& a, const Dual<T, N>& b)
{
    a = a / b;
    return a;
}

// comparisons act on the values
template <typename T, int N>
__host__ __device__ inline bool operator<(const Dual<T, N>& a, const Dual<T, N>& b) { return a.v < b.v; }
template <typename T, int N>
__host__ __device__ inline bool operator>(const Dual<T, N>& a, const Dual<T, N>& b) { return a.v > b.v; }
template <typename T, int N>
__host__ __device__ inline bool operator<=(const Dual<T, N>& a, const Dual<T, N>& b) { return a.v <= b.v; }
template <typename T, int N>
__host__ __device__ inline bool operator>=(const Dual<T, N>& a, const Dual<T, N>& b) { return a.v >= b.v; }

template <typename T, int N>
__host__ __device__ inline Dual<T, N> exp(const Dual<T, N>& a)
{
    Dual<T, N> r;
    if constexpr (sizeof(T) == 4) r.v = expf(a.v);
    else r.v = ::exp(a.v);
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = r.v * a.d[k];
    return r;
}

template <typename T, int N>
__device__ __forceinline__ Dual<T, N> fdiv(const Dual<T, N>& a, const Dual<T, N>& b) { return a / b; }

// value part of a stored number
__host__ __device__ inline double val(double x) { return x; }
__host__ __device__ inline double val(float x) { return (double)x; }
template <typename T, int N>
__host__ __device__ inline double val(const Dual<T, N>& x) { return (double)x.v; }

// FP64 copy of an FP32 dual number and back (round to nearest)
template <int N>
__host__ __device__ inline Dual<double, N> widen(const Dual<float, N>& a)
{
    Dual<double, N> r;
    r.v = a.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = a.d[k];
    return r;
}
template <int N>
__host__ __device__ inline Dual<float, N> narrow(const Dual<double, N>& a)
{
    Dual<float, N> r;
    r.v = (float)a.v;
#pragma unroll
    for (int k = 0; k < N; ++k) r.d[k] = (float)a.d[k];
    return r;
}

// tangents with respect to (ln A, Ta, T_wall, u_in): FP64, and FP32 (the
// mixed tangent form: FP32 state and arithmetic, FP64 Arrhenius above
// T_fp64 and FP64 accumulation of the objectives)
constexpr int NTAN = 4;
using Tan = Dual<double, NTAN>;
using Tanf = Dual<float, NTAN>;

}  // namespace lbfd
