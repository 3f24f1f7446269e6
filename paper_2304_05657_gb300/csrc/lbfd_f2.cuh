// lbfd_f2.cuh -- a pair of FP32 values computed with the packed FP32
// instructions of sm_100-class GPUs (fma/add/mul.rn.f32x2): one instruction
// updates two cells.  The tile kernel that computes two neighbouring cells
// per thread instantiates the step's arithmetic with R = F2.
//
// A product is kept unevaluated (F2M) until it meets an addition, so that
// a * b + c issues one packed FMA, as the scalar compiler would contract
// it; a product used on its own is evaluated with one packed multiply.
#pragma once
#include <cuda_runtime.h>

namespace lbfd {

struct F2M;

struct F2 {
    float2 v;
    F2() = default;
    __host__ __device__ constexpr F2(float a) : v{a, a} {}
    __host__ __device__ constexpr F2(double a) : v{(float)a, (float)a} {}
    __host__ __device__ constexpr F2(int a) : v{(float)a, (float)a} {}
    __host__ __device__ constexpr F2(float a, float b) : v{a, b} {}
    __device__ __forceinline__ F2(float2 a) : v(a) {}
    __device__ __forceinline__ F2(const F2M& m);
    __device__ __forceinline__ F2& operator+=(const F2& b);
    __device__ __forceinline__ F2& operator-=(const F2& b);
    __device__ __forceinline__ F2& operator*=(const F2& b);
    __device__ __forceinline__ F2& operator+=(const F2M& b);
    __device__ __forceinline__ F2& operator-=(const F2M& b);
};

// a * b, not yet rounded
struct F2M {
    float2 a, b;
};

__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
// a - b in one packed instruction: b * (-1) + a, exact like a subtraction
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

__device__ __forceinline__ F2::F2(const F2M& m) : v(__fmul2_rn(m.a, m.b)) {}

__device__ __forceinline__ F2M operator*(const F2& a, const F2& b) { return F2M{a.v, b.v}; }
__device__ __forceinline__ F2M operator*(const F2M& m, const F2& c) { return F2M{f2mul(m.a, m.b), c.v}; }
__device__ __forceinline__ F2M operator*(const F2& c, const F2M& m) { return F2M{c.v, f2mul(m.a, m.b)}; }
__device__ __forceinline__ F2M operator*(const F2M& m, const F2M& n) { return F2M{f2mul(m.a, m.b), f2mul(n.a, n.b)}; }

__device__ __forceinline__ F2 operator+(const F2& a, const F2& b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(const F2& a, const F2& b) { return F2(f2sub(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(const F2& a) { return F2(f2neg(a.v)); }
__device__ __forceinline__ F2M operator-(const F2M& m) { return F2M{f2neg(m.a), m.b}; }

__device__ __forceinline__ F2 operator+(const F2M& m, const F2& c) { return F2(__ffma2_rn(m.a, m.b, c.v)); }
__device__ __forceinline__ F2 operator+(const F2& c, const F2M& m) { return F2(__ffma2_rn(m.a, m.b, c.v)); }
__device__ __forceinline__ F2 operator-(const F2M& m, const F2& c) { return F2(__ffma2_rn(m.a, m.b, f2neg(c.v))); }
__device__ __forceinline__ F2 operator-(const F2& c, const F2M& m) { return F2(__ffma2_rn(f2neg(m.a), m.b, c.v)); }
__device__ __forceinline__ F2 operator+(const F2M& m, const F2M& n) { return F2(__ffma2_rn(m.a, m.b, f2mul(n.a, n.b))); }
__device__ __forceinline__ F2 operator-(const F2M& m, const F2M& n)
{
    return F2(__ffma2_rn(f2neg(n.a), n.b, f2mul(m.a, m.b)));
}

// exact (IEEE) division; the hot paths use fdiv
__device__ __forceinline__ F2 operator/(const F2& a, const F2& b) { return F2(a.v.x / b.v.x, a.v.y / b.v.y); }

__device__ __forceinline__ F2& F2::operator+=(const F2& b) { return *this = *this + b; }
__device__ __forceinline__ F2& F2::operator-=(const F2& b) { return *this = *this - b; }
__device__ __forceinline__ F2& F2::operator*=(const F2& b) { return *this = F2(*this * b); }
__device__ __forceinline__ F2& F2::operator+=(const F2M& b) { return *this = *this + b; }
__device__ __forceinline__ F2& F2::operator-=(const F2M& b) { return *this = *this - b; }

// per-lane fast division (hardware reciprocal), as fdiv(float, float)
__device__ __forceinline__ F2 fdiv(const F2& a, const F2& b)
{
    return F2(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y));
}

// per-lane select
__device__ __forceinline__ F2 f2sel(bool p0, bool p1, const F2& a, const F2& b)
{
    return F2(p0 ? a.v.x : b.v.x, p1 ? a.v.y : b.v.y);
}

// the scalar type behind a compute type: constants are formed in it
template <typename R>
struct ScalarOf {
    using type = R;
};
template <>
struct ScalarOf<F2> {
    using type = float;
};
template <typename R>
using scalar_t = typename ScalarOf<R>::type;

// WENO3 derivative of two cells (the per-lane form of weno3_deriv_fast)
__device__ __forceinline__ F2 weno3_deriv_fast(const F2* v, const F2& u, const F2& eps)
{
    const bool n0 = u.v.x < 0.f, n1 = u.v.y < 0.f;
    const F2 a = f2sel(n0, n1, v[4], v[0]);
    const F2 b = f2sel(n0, n1, v[3], v[1]);
    const F2 c = v[2];
    const F2 d = f2sel(n0, n1, v[1], v[3]);
    const F2 dab = b - a, dbc = c - b, dcd = d - c;
    const F2 e_ab = eps + dab * dab, e_bc = eps + dbc * dbc, e_cd = eps + dcd * dcd;
    const F2 w0p = e_cd * e_cd, w1p = F2(2.f) * e_bc * e_bc;
    const F2 fp = c + F2(0.5f) * fdiv(w0p * dbc + w1p * dcd, w0p + w1p);
    const F2 w0m = e_bc * e_bc, w1m = F2(2.f) * e_ab * e_ab;
    const F2 fm = b + F2(0.5f) * fdiv(w0m * dab + w1m * dbc, w0m + w1m);
    const F2 r = fp - fm;
    return f2sel(n0, n1, -r, r);
}

}  // namespace lbfd
