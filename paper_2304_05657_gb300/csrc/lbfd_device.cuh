// lbfd_device.cuh -- device-side building blocks of the fused coupled step:
// lattice constants, boundary classification, pull streaming with boundary
// rules, FD line gathering with ghost nodes, FD operators, and the cumulant
// collision.  Written for sm_103a; templated on the compute type R (double
// for the FP64 form, float for the mixed form, F2 for two cells in packed
// FP32, dual numbers for the tangent forms, Rev for the adjoint).
//
// Method: Hosseini & Thevenin, arXiv 2304.05657, Sec. II-III.
#pragma once
#include <cstdint>
#include <type_traits>

#include "lbfd_dual.cuh"
#include "lbfd_f2.cuh"
#include "lbfd_params.h"

namespace lbfd {

// Fast division: the hardware reciprocal path in FP32 (about 2 ulp, for
// divisors of normal magnitude), IEEE division in FP64.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

enum { BC_PERIODIC = 0, BC_WALL_ADIABATIC = 1, BC_WALL_ISOTHERMAL = 2, BC_INLET = 3, BC_OUTLET = 4,
       BC_OUTLET_PRESSURE = 5 };
enum { PT_FLUID = 0, PT_SOLID = 16 };
// ghost modes of an FD line point
enum { G_DIRECT = 0, G_NEUMANN = 1, G_DIRICHLET_T = 2, G_INLET = 3, G_CURVED = 4 };

// ---------------------------------------------------------------------------
// lattice: D1Q3 tensor products, i = (cx+1) + 3(cy+1) + 9(cz+1)
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cx_of(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy_of(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz_of(int i) { return i / 9 - 1; }
template <typename R>
__host__ __device__ constexpr R w1(int c) { return c == 0 ? R(2) / R(3) : R(1) / R(6); }
template <int DIM, typename R>
__host__ __device__ constexpr R weight(int i)
{
    return DIM == 2 ? w1<R>(cx_of(i)) * w1<R>(cy_of(i))
                    : w1<R>(cx_of(i)) * w1<R>(cy_of(i)) * w1<R>(cz_of(i));
}
template <int DIM>
__host__ __device__ constexpr int ccomp(int i, int a)
{
    return a == 0 ? cx_of(i) : (a == 1 ? cy_of(i) : (DIM == 3 ? cz_of(i) : 0));
}
template <int DIM>
__host__ __device__ constexpr int opposite(int i) { return (DIM == 2 ? 8 : 26) - i; }

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ int extent(const StepParams<R>& P, int a)
{
    return a == 0 ? P.nx : (a == 1 ? P.ny : P.nz);
}

template <typename R>
__device__ __forceinline__ long long cell_of(const StepParams<R>& P, int x, int y, int z)
{
    return (long long)x + (long long)P.nx * ((long long)y + (long long)P.ny * z);
}

// Classify a point that differs from a fluid cell along one or more axes.
// Periodic axes wrap; a crossed non-periodic face returns its bc type.
// FACES == false: the caller guarantees that no non-periodic face is
// crossed (cells whose stencils stay inside the domain up to periodic wrap).
template <int DIM, typename R, bool FACES = true>
__device__ __forceinline__ int classify(const StepParams<R>& P, int q[3], const uint8_t* LBFD_RESTRICT solid,
                                        long long* idx, int* face)
{
    int wall = -1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int n = extent(P, a);
        int f = -1;
        if (q[a] < 0) f = 2 * a;
        else if (q[a] >= n) f = 2 * a + 1;
        if (f < 0) continue;
        if (!FACES || P.bc[f] == BC_PERIODIC) q[a] = ((q[a] % n) + n) % n;  // extents may be < 3
        else if (wall < 0) wall = f;
    }
    if (FACES && wall >= 0) {
        *face = wall;
        return P.bc[wall];
    }
    *idx = cell_of(P, q[0], q[1], DIM == 3 ? q[2] : 0);
    return solid[*idx] ? PT_SOLID : PT_FLUID;
}

// ---------------------------------------------------------------------------
// thermochemistry
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R inv_molar_mass(const StepParams<R>& P, const R* Y)
{
    R s = R(0);
#pragma unroll
    for (int k = 0; k < NSP; ++k) s += Y[k] * P.inv_Wk[k];
    return s;
}

// Y[k] for a species index known only at run time, without indexing a
// register array
template <typename R>
__device__ __forceinline__ R pick_species(const R* Y, int k)
{
    R r = Y[0];
#pragma unroll
    for (int j = 1; j < NSP; ++j) r = k == j ? Y[j] : r;
    return r;
}

// EOS at constant P_0 (Sec. II.A) with rho(T_in, Y_in) = 1
template <typename R>
__device__ __forceinline__ R eos(const StepParams<R>& P, R T, R invW)
{
    return fdiv(P.T_in * P.invW_in, T * invW);
}

// Single-step rate per unit mass of fuel, per step.  The mixed form
// evaluates it in FP64 where T > T_fp64.
template <typename R>
__device__ __forceinline__ R arrhenius(const StepParams<R>& P, R T, R yf, R yo)
{
    yf = yf > R(0) ? yf : R(0);
    yo = yo > R(0) ? yo : R(0);
    if constexpr (std::is_same<R, float>::value) {
        if (T > P.T_fp64) {
            const double q = P.A_lat_d * (double)yf * (double)yo * ::exp(-P.Ta_d / (double)T);
            return (float)q;
        }
        return P.A_lat * yf * yo * expf(-(P.Ta / T));
    } else if constexpr (std::is_same<R, double>::value) {
        return P.A_lat * yf * yo * ::exp(-(P.Ta / T));
    } else if constexpr (std::is_same<R, Tanf>::value) {
        if (T > P.T_fp64) {  // FP64 rate and derivatives, as the mixed form
            Tan A = widen(P.A_lat), Ta = widen(P.Ta);
            A.v = P.A_lat_d;
            A.d[0] = P.A_lat_d;  // d(A dt)/d(ln A)
            Ta.v = P.Ta_d;
            return narrow(A * widen(yf) * widen(yo) * exp(-(Ta / widen(T))));
        }
        return P.A_lat * yf * yo * exp(-(P.Ta / T));
    } else {
        return P.A_lat * yf * yo * exp(-(P.Ta / T));  // the Dual overload
    }
}

// ---------------------------------------------------------------------------
// FD operators (Sec. II.D), unit spacing, v[0..4] = phi_{i-2..i+2}
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R fd_d1(const R* v)  // 4th-order central first derivative
{
    return (v[0] - v[4] + R(8) * (v[3] - v[1])) * R(scalar_t<R>(1) / scalar_t<R>(12));
}
template <typename R>
__device__ __forceinline__ R fd_d2(const R* v)  // 4th-order central second derivative
{
    return (R(16) * (v[1] + v[3]) - (v[0] + v[4]) - R(30) * v[2]) * R(scalar_t<R>(1) / scalar_t<R>(12));
}
// the same stencils times 12 (the tiles fold 1/12 into their coefficients)
template <typename R>
__device__ __forceinline__ R fd_D1(const R* v)
{
    return v[0] - v[4] + R(8) * (v[3] - v[1]);
}
template <typename R>
__device__ __forceinline__ R fd_D2(const R* v)
{
    return R(16) * (v[1] + v[3]) - (v[0] + v[4]) - R(30) * v[2];
}
template <typename R>
__device__ __forceinline__ R fd_c2(const R* v)  // centred 2nd order
{
    return R(0.5) * (v[3] - v[1]);
}

// WENO3 face value: a far upwind, b upwind cell, c downwind cell
template <typename R>
__device__ __forceinline__ R weno3_face(R a, R b, R c, R eps)
{
    R q0 = R(1.5) * b - R(0.5) * a;
    R q1 = R(0.5) * (b + c);
    R e0 = eps + (b - a) * (b - a);
    R e1 = eps + (c - b) * (c - b);
    // alpha_0 = (1/3)/e0^2, alpha_1 = (2/3)/e1^2; the common factor is dropped
    R a0 = e1 * e1;
    R a1 = R(2) * e0 * e0;
    return (a0 * q0 + a1 * q1) / (a0 + a1);
}
template <typename R>
__device__ __forceinline__ R weno3_deriv(const R* v, R u, R eps)
{
    if (u >= R(0)) return weno3_face(v[1], v[2], v[3], eps) - weno3_face(v[0], v[1], v[2], eps);
    return weno3_face(v[4], v[3], v[2], eps) - weno3_face(v[3], v[2], v[1], eps);
}


// WENO3 derivative without a branch on the sign of u: for u < 0 the line is
// mirrored and the result negated (the two upwind formulas are mirror
// images).  The squared difference across the centre is shared by both
// faces.  Same reconstruction as weno3_deriv, rounding aside.
template <typename R>
__device__ __forceinline__ R weno3_deriv_fast(const R* v, R u, R eps)
{
    const bool neg = u < R(0);
    const R a = neg ? v[4] : v[0];
    const R b = neg ? v[3] : v[1];
    const R c = v[2];
    const R d = neg ? v[1] : v[3];
    const R dab = b - a, dbc = c - b, dcd = d - c;
    const R e_ab = eps + dab * dab, e_bc = eps + dbc * dbc, e_cd = eps + dcd * dcd;
    // face c+1/2 from (b, c, d): q0 = c + dbc/2, q1 = c + dcd/2, weights e_cd^2 : 2 e_bc^2
    const R w0p = e_cd * e_cd, w1p = R(2) * e_bc * e_bc;
    const R fp = c + R(0.5) * fdiv(w0p * dbc + w1p * dcd, w0p + w1p);
    // face c-1/2 from (a, b, c): q0 = b + dab/2, q1 = b + dbc/2, weights e_bc^2 : 2 e_ab^2
    const R w0m = e_bc * e_bc, w1m = R(2) * e_ab * e_ab;
    const R fm = b + R(0.5) * fdiv(w0m * dab + w1m * dbc, w0m + w1m);
    const R r = fp - fm;
    return neg ? -r : r;
}

// ---------------------------------------------------------------------------
// central moments (Eq. 21) by axis-wise D1Q3 transforms, and cumulants
// (Eq. 22) with their exact inverse.  Moment index p + 3q + 9r.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void cm3_forward(R& f0, R& f1, R& f2, R u)
{
    R r0 = f0 + f1 + f2;
    R r1 = f2 - f0;
    R r2 = f2 + f0;
    f0 = r0;
    f1 = r1 - u * r0;
    f2 = r2 - R(2) * u * r1 + u * u * r0;
}
template <typename R>
__device__ __forceinline__ void cm3_inverse(R& m0, R& m1, R& m2, R u)
{
    R r0 = m0;
    R r1 = m1 + u * m0;
    R r2 = m2 + R(2) * u * m1 + u * u * m0;
    m0 = R(0.5) * (r2 - r1);
    m1 = r0 - r2;
    m2 = R(0.5) * (r2 + r1);
}

template <int DIM, typename R>
__device__ __forceinline__ void central_forward(R* f, const R* u)
{
    constexpr int NZ = DIM == 3 ? 3 : 1;
#pragma unroll
    for (int c = 0; c < NZ; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) cm3_forward(f[3 * b + 9 * c], f[1 + 3 * b + 9 * c], f[2 + 3 * b + 9 * c], u[0]);
#pragma unroll
    for (int c = 0; c < NZ; ++c)
#pragma unroll
        for (int p = 0; p < 3; ++p) cm3_forward(f[p + 9 * c], f[p + 3 + 9 * c], f[p + 6 + 9 * c], u[1]);
    if (DIM == 3) {
#pragma unroll
        for (int j = 0; j < 9; ++j) cm3_forward(f[j], f[j + 9], f[j + 18], u[2]);
    }
}

// The central moments of orders 0-2 only (the others are left partly
// transformed): the collision with omega_hi = 1 needs no more, since it
// sets every cumulant of order >= 3 to its equilibrium.  The same
// expressions as central_forward for the moments it forms.
template <typename R>
__device__ __forceinline__ void cm3_forward01(R& f0, R& f1, R f2, R u)
{
    R r0 = f0 + f1 + f2;
    R r1 = f2 - f0;
    f0 = r0;
    f1 = r1 - u * r0;
}
template <int DIM, typename R>
__device__ __forceinline__ void central_forward_lo(R* f, const R* u)
{
    constexpr int NZ = DIM == 3 ? 3 : 1;
#pragma unroll
    for (int c = 0; c < NZ; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) cm3_forward(f[3 * b + 9 * c], f[1 + 3 * b + 9 * c], f[2 + 3 * b + 9 * c], u[0]);
#pragma unroll
    for (int c = 0; c < NZ; ++c) {  // y lines of x order p: y orders up to 2 - p
        cm3_forward(f[9 * c], f[3 + 9 * c], f[6 + 9 * c], u[1]);
        cm3_forward01(f[1 + 9 * c], f[4 + 9 * c], f[7 + 9 * c], u[1]);
        f[2 + 9 * c] = f[2 + 9 * c] + f[5 + 9 * c] + f[8 + 9 * c];
    }
    if (DIM == 3) {  // z lines of x-y order s: z orders up to 2 - s
        cm3_forward(f[0], f[9], f[18], u[2]);
        cm3_forward01(f[1], f[10], f[19], u[2]);
        cm3_forward01(f[3], f[12], f[21], u[2]);
        f[2] = f[2] + f[11] + f[20];
        f[4] = f[4] + f[13] + f[22];
        f[6] = f[6] + f[15] + f[24];
    }
}

template <int DIM, typename R>
__device__ __forceinline__ void central_inverse(R* m, const R* u)
{
    constexpr int NZ = DIM == 3 ? 3 : 1;
    if (DIM == 3) {
#pragma unroll
        for (int j = 0; j < 9; ++j) cm3_inverse(m[j], m[j + 9], m[j + 18], u[2]);
    }
#pragma unroll
    for (int c = 0; c < NZ; ++c)
#pragma unroll
        for (int p = 0; p < 3; ++p) cm3_inverse(m[p + 9 * c], m[p + 3 + 9 * c], m[p + 6 + 9 * c], u[1]);
#pragma unroll
    for (int c = 0; c < NZ; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) cm3_inverse(m[3 * b + 9 * c], m[1 + 3 * b + 9 * c], m[2 + 3 * b + 9 * c], u[0]);
}

#define LBFD_M(p, q, r) ((p) + 3 * (q) + 9 * (r))

// In place: central moments -> cumulants (orders >= 4 change).
template <int DIM, typename R>
__device__ __forceinline__ void to_cumulants(R* m)
{
#define C_(p, q, r) m[LBFD_M(p, q, r)]
    if (DIM == 2) {
        C_(2, 2, 0) -= C_(2, 0, 0) * C_(0, 2, 0) + R(2) * C_(1, 1, 0) * C_(1, 1, 0);
        return;
    }
    // sixth order first: it reads the order-4 central moments
    R k222 = C_(2, 2, 2)
        - (C_(2, 0, 0) * C_(0, 2, 2) + C_(0, 2, 0) * C_(2, 0, 2) + C_(0, 0, 2) * C_(2, 2, 0))
        - R(4) * (C_(1, 1, 0) * C_(1, 1, 2) + C_(1, 0, 1) * C_(1, 2, 1) + C_(0, 1, 1) * C_(2, 1, 1))
        - R(4) * C_(1, 1, 1) * C_(1, 1, 1)
        - R(2) * (C_(2, 1, 0) * C_(0, 1, 2) + C_(2, 0, 1) * C_(0, 2, 1) + C_(1, 2, 0) * C_(1, 0, 2))
        + R(2) * C_(2, 0, 0) * C_(0, 2, 0) * C_(0, 0, 2)
        + R(4) * (C_(2, 0, 0) * C_(0, 1, 1) * C_(0, 1, 1) + C_(0, 2, 0) * C_(1, 0, 1) * C_(1, 0, 1)
                  + C_(0, 0, 2) * C_(1, 1, 0) * C_(1, 1, 0))
        + R(16) * C_(1, 1, 0) * C_(1, 0, 1) * C_(0, 1, 1);
    R k122 = C_(1, 2, 2) - C_(0, 0, 2) * C_(1, 2, 0) - C_(0, 2, 0) * C_(1, 0, 2)
        - R(4) * C_(0, 1, 1) * C_(1, 1, 1) - R(2) * (C_(1, 0, 1) * C_(0, 2, 1) + C_(1, 1, 0) * C_(0, 1, 2));
    R k212 = C_(2, 1, 2) - C_(0, 0, 2) * C_(2, 1, 0) - C_(2, 0, 0) * C_(0, 1, 2)
        - R(4) * C_(1, 0, 1) * C_(1, 1, 1) - R(2) * (C_(0, 1, 1) * C_(2, 0, 1) + C_(1, 1, 0) * C_(1, 0, 2));
    R k221 = C_(2, 2, 1) - C_(2, 0, 0) * C_(0, 2, 1) - C_(0, 2, 0) * C_(2, 0, 1)
        - R(4) * C_(1, 1, 0) * C_(1, 1, 1) - R(2) * (C_(1, 0, 1) * C_(1, 2, 0) + C_(0, 1, 1) * C_(2, 1, 0));
    C_(2, 2, 2) = k222;
    C_(1, 2, 2) = k122;
    C_(2, 1, 2) = k212;
    C_(2, 2, 1) = k221;
    C_(2, 2, 0) -= C_(2, 0, 0) * C_(0, 2, 0) + R(2) * C_(1, 1, 0) * C_(1, 1, 0);
    C_(2, 0, 2) -= C_(2, 0, 0) * C_(0, 0, 2) + R(2) * C_(1, 0, 1) * C_(1, 0, 1);
    C_(0, 2, 2) -= C_(0, 2, 0) * C_(0, 0, 2) + R(2) * C_(0, 1, 1) * C_(0, 1, 1);
    C_(2, 1, 1) -= C_(2, 0, 0) * C_(0, 1, 1) + R(2) * C_(1, 1, 0) * C_(1, 0, 1);
    C_(1, 2, 1) -= C_(0, 2, 0) * C_(1, 0, 1) + R(2) * C_(1, 1, 0) * C_(0, 1, 1);
    C_(1, 1, 2) -= C_(0, 0, 2) * C_(1, 1, 0) + R(2) * C_(1, 0, 1) * C_(0, 1, 1);
#undef C_
}

// In place: cumulants -> central moments (exact inverse of to_cumulants).
template <int DIM, typename R>
__device__ __forceinline__ void from_cumulants(R* m)
{
#define C_(p, q, r) m[LBFD_M(p, q, r)]
    if (DIM == 2) {
        C_(2, 2, 0) += C_(2, 0, 0) * C_(0, 2, 0) + R(2) * C_(1, 1, 0) * C_(1, 1, 0);
        return;
    }
    C_(2, 2, 0) += C_(2, 0, 0) * C_(0, 2, 0) + R(2) * C_(1, 1, 0) * C_(1, 1, 0);
    C_(2, 0, 2) += C_(2, 0, 0) * C_(0, 0, 2) + R(2) * C_(1, 0, 1) * C_(1, 0, 1);
    C_(0, 2, 2) += C_(0, 2, 0) * C_(0, 0, 2) + R(2) * C_(0, 1, 1) * C_(0, 1, 1);
    C_(2, 1, 1) += C_(2, 0, 0) * C_(0, 1, 1) + R(2) * C_(1, 1, 0) * C_(1, 0, 1);
    C_(1, 2, 1) += C_(0, 2, 0) * C_(1, 0, 1) + R(2) * C_(1, 1, 0) * C_(0, 1, 1);
    C_(1, 1, 2) += C_(0, 0, 2) * C_(1, 1, 0) + R(2) * C_(1, 0, 1) * C_(0, 1, 1);
    C_(1, 2, 2) += C_(0, 0, 2) * C_(1, 2, 0) + C_(0, 2, 0) * C_(1, 0, 2)
        + R(4) * C_(0, 1, 1) * C_(1, 1, 1) + R(2) * (C_(1, 0, 1) * C_(0, 2, 1) + C_(1, 1, 0) * C_(0, 1, 2));
    C_(2, 1, 2) += C_(0, 0, 2) * C_(2, 1, 0) + C_(2, 0, 0) * C_(0, 1, 2)
        + R(4) * C_(1, 0, 1) * C_(1, 1, 1) + R(2) * (C_(0, 1, 1) * C_(2, 0, 1) + C_(1, 1, 0) * C_(1, 0, 2));
    C_(2, 2, 1) += C_(2, 0, 0) * C_(0, 2, 1) + C_(0, 2, 0) * C_(2, 0, 1)
        + R(4) * C_(1, 1, 0) * C_(1, 1, 1) + R(2) * (C_(1, 0, 1) * C_(1, 2, 0) + C_(0, 1, 1) * C_(2, 1, 0));
    C_(2, 2, 2) += (C_(2, 0, 0) * C_(0, 2, 2) + C_(0, 2, 0) * C_(2, 0, 2) + C_(0, 0, 2) * C_(2, 2, 0))
        + R(4) * (C_(1, 1, 0) * C_(1, 1, 2) + C_(1, 0, 1) * C_(1, 2, 1) + C_(0, 1, 1) * C_(2, 1, 1))
        + R(4) * C_(1, 1, 1) * C_(1, 1, 1)
        + R(2) * (C_(2, 1, 0) * C_(0, 1, 2) + C_(2, 0, 1) * C_(0, 2, 1) + C_(1, 2, 0) * C_(1, 0, 2))
        - R(2) * C_(2, 0, 0) * C_(0, 2, 0) * C_(0, 0, 2)
        - R(4) * (C_(2, 0, 0) * C_(0, 1, 1) * C_(0, 1, 1) + C_(0, 2, 0) * C_(1, 0, 1) * C_(1, 0, 1)
                  + C_(0, 0, 2) * C_(1, 1, 0) * C_(1, 1, 0))
        - R(16) * C_(1, 1, 0) * C_(1, 0, 1) * C_(0, 1, 1);
#undef C_
}

__host__ __device__ constexpr int moment_order(int j) { return j % 3 + (j / 3) % 3 + j / 9; }

// Cumulants of orders >= 2 of g^eq / (rho cs^2) (Eq. 10, 12, 21, 22) in
// closed form.  On the product-weight lattices (D2Q9, D3Q27) the central
// moments of the discrete second-order equilibrium are polynomials in
// e = P_h / (rho cs^2) - 1 and the velocity; taking them through Eq. 22
// gives the expressions below (a, b, c = u_x^2, u_y^2, u_z^2), the same
// numbers as transforming the Q values, up to rounding.  Orders 0 and 1 are
// not relaxed and are left unset.
template <int DIM, typename R>
__device__ __forceinline__ void eq_cumulants(R* fe, R e, const R* u)
{
    using Sc = scalar_t<R>;
    const R third = R(Sc(1) / Sc(3)), ninth = R(Sc(1) / Sc(9));
    const R ux = u[0], uy = u[1];
    const R a = ux * ux, b = uy * uy;
    const R Ph = e + R(1), Ph3 = Ph * third, e3 = e * third, E2 = e * e;
    const R s1 = R(3) + e - R(3) * E2, s2 = E2 * third, s3 = (E2 + e) * ninth;
    // second order: kappa_aa = e u_a^2 + Ph/3, kappa_ab = e u_a u_b
    // third: kappa_aab = -u_b (Ph u_a^2 + e/3); fourth: c_aabb = u_a^2 u_b^2 s1 - s2 (u_a^2 + u_b^2) - s3
    fe[LBFD_M(2, 0, 0)] = e * a + Ph3;
    fe[LBFD_M(0, 2, 0)] = e * b + Ph3;
    fe[LBFD_M(1, 1, 0)] = e * ux * uy;
    fe[LBFD_M(2, 1, 0)] = -(uy * (Ph * a + e3));
    fe[LBFD_M(1, 2, 0)] = -(ux * (Ph * b + e3));
    fe[LBFD_M(2, 2, 0)] = a * b * s1 - s2 * (a + b) - s3;
    if constexpr (DIM == 3) {
        const R uz = u[2];
        const R c = uz * uz;
        fe[LBFD_M(0, 0, 2)] = e * c + Ph3;
        fe[LBFD_M(1, 0, 1)] = e * ux * uz;
        fe[LBFD_M(0, 1, 1)] = e * uy * uz;
        fe[LBFD_M(2, 0, 1)] = -(uz * (Ph * a + e3));
        fe[LBFD_M(0, 2, 1)] = -(uz * (Ph * b + e3));
        fe[LBFD_M(1, 0, 2)] = -(ux * (Ph * c + e3));
        fe[LBFD_M(0, 1, 2)] = -(uy * (Ph * c + e3));
        fe[LBFD_M(1, 1, 1)] = -(Ph * ux * uy * uz);
        fe[LBFD_M(2, 0, 2)] = a * c * s1 - s2 * (a + c) - s3;
        fe[LBFD_M(0, 2, 2)] = b * c * s1 - s2 * (b + c) - s3;
        // fourth, c_aabc = u_b u_c (u_a^2 s1 - s2)
        fe[LBFD_M(2, 1, 1)] = uy * uz * (a * s1 - s2);
        fe[LBFD_M(1, 2, 1)] = ux * uz * (b * s1 - s2);
        fe[LBFD_M(1, 1, 2)] = ux * uy * (c * s1 - s2);
        // fifth, c_abbcc = u_a (u_b^2 u_c^2 t1 + (u_b^2 + u_c^2) t2 + t3)
        const R t1 = R(-6) + R(9) * e + R(10) * E2;
        const R t2 = (e + R(4) * E2) * third, t3 = (e + R(2) * E2) * ninth;
        fe[LBFD_M(1, 2, 2)] = ux * (b * c * t1 + (b + c) * t2 + t3);
        fe[LBFD_M(2, 1, 2)] = uy * (a * c * t1 + (a + c) * t2 + t3);
        fe[LBFD_M(2, 2, 1)] = uz * (a * b * t1 + (a + b) * t2 + t3);
        // sixth, in the elementary symmetric polynomials of a, b, c
        const R E3 = E2 * e;
        const R sg1 = a + b + c, sg2 = a * b + a * c + b * c, sg3 = a * b * c;
        fe[LBFD_M(2, 2, 2)] = sg3 * (R(30) * E3 - R(25) * E2 - R(64) * e)
            + sg2 * (R(2) * E3 - (R(5) * E2 + R(7) * e) * third) + sg1 * (R(2) * E3 - E2) * ninth
            + (R(2) * E3 * third + E2 + e * third) * ninth;
    }
}

// ---------------------------------------------------------------------------
// Collision of one cell (Eq. 9, 10, 12-15, 19, 21-24): g (post-streaming)
// is replaced by g*.  Relaxation toward the cumulants of g^eq/(rho cs^2);
// orders 0-1 carried, second order split into trace (omega_b) and
// deviatoric/off-diagonal (omega_s), orders >= 3 at omega_hi.
// ---------------------------------------------------------------------------
// HI1: omega_hi == 1 (the caller checks), so the pre-collision cumulants of
// order >= 3 are not formed: the relaxation sets them to equilibrium, as
// fe + (1 - omega_hi) (g - fe) does for omega_hi = 1.
template <int DIM, typename R, typename PR, bool HI1 = false>
__device__ __forceinline__ void collide(const StepParams<PR>& P, R* g, R rho, const R* u, const R* grad_rho,
                                        R Lam)
{
    using Sc = scalar_t<R>;
    constexpr int Q = DIM == 2 ? 9 : 27;
    const R cs2 = R(Sc(1) / Sc(3));
    R sum_g = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) sum_g += g[i];
    const R rcs2 = rho * cs2;
    const R P_h = sum_g + R(0.5) * rcs2 * Lam;  // Eq. 13a
    const R uu = u[0] * u[0] + u[1] * u[1] + (DIM == 3 ? u[2] * u[2] : R(0));
    const R inv_rcs2 = fdiv(R(1), rcs2);
    R xi[Q], fe[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R wi = R(weight<DIM, Sc>(i));
        R cu = R(0), cg = R(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const int c = ccomp<DIM>(i, a);
            cu += R(c) * u[a];
            cg += (R(c) - u[a]) * grad_rho[a];
        }
        // f^eq / rho, Eq. 10
        const R feq_r = wi * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
        xi[i] = cs2 * (feq_r - wi) * cg + wi * rcs2 * Lam;  // Eq. 9
        g[i] = (g[i] + R(0.5) * xi[i]) * inv_rcs2;  // Eq. 19
    }
    if constexpr (HI1) {
        central_forward_lo<DIM>(g, u);  // orders 0-2: cumulants = central moments
    } else {
        central_forward<DIM>(g, u);
        to_cumulants<DIM>(g);
    }
    // the target: cumulants of g^eq / (rho cs2) = w (P_h/(rho cs2) - 1) + f^eq/rho (Eq. 12)
    eq_cumulants<DIM>(fe, P_h * inv_rcs2 - R(1), u);
    // relaxation
    const R ws = R(P.omega_s), wb = R(P.omega_b), wh = R(P.omega_hi);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int o = moment_order(j);
        if (o >= 3) g[j] = HI1 ? fe[j] : fe[j] + (R(1) - wh) * (g[j] - fe[j]);
    }
    if (DIM == 2) {
        const int ixx = LBFD_M(2, 0, 0), iyy = LBFD_M(0, 2, 0), ixy = LBFD_M(1, 1, 0);
        const R tr = g[ixx] + g[iyy], tre = fe[ixx] + fe[iyy];
        const R dv = g[ixx] - g[iyy], dve = fe[ixx] - fe[iyy];
        const R trs = tre + (R(1) - wb) * (tr - tre);
        const R dvs = dve + (R(1) - ws) * (dv - dve);
        g[ixx] = R(0.5) * (trs + dvs);
        g[iyy] = R(0.5) * (trs - dvs);
        g[ixy] = fe[ixy] + (R(1) - ws) * (g[ixy] - fe[ixy]);
    } else {
        const int ixx = LBFD_M(2, 0, 0), iyy = LBFD_M(0, 2, 0), izz = LBFD_M(0, 0, 2);
        const R tr = g[ixx] + g[iyy] + g[izz], tre = fe[ixx] + fe[iyy] + fe[izz];
        const R d1 = g[ixx] - g[iyy], d1e = fe[ixx] - fe[iyy];
        const R d2 = g[ixx] - g[izz], d2e = fe[ixx] - fe[izz];
        const R trs = tre + (R(1) - wb) * (tr - tre);
        const R d1s = d1e + (R(1) - ws) * (d1 - d1e);
        const R d2s = d2e + (R(1) - ws) * (d2 - d2e);
        const R xx = (trs + d1s + d2s) * R(Sc(1) / Sc(3));
        g[ixx] = xx;
        g[iyy] = xx - d1s;
        g[izz] = xx - d2s;
        const int o1 = LBFD_M(1, 1, 0), o2 = LBFD_M(1, 0, 1), o3 = LBFD_M(0, 1, 1);
        g[o1] = fe[o1] + (R(1) - ws) * (g[o1] - fe[o1]);
        g[o2] = fe[o2] + (R(1) - ws) * (g[o2] - fe[o2]);
        g[o3] = fe[o3] + (R(1) - ws) * (g[o3] - fe[o3]);
    }
    from_cumulants<DIM>(g);
    central_inverse<DIM>(g, u);
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = rcs2 * g[i] + R(0.5) * xi[i];  // Eq. 14
}

}  // namespace lbfd
