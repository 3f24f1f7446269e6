// lbfd_rev.cuh -- reverse-mode numbers for the discrete adjoint of one step.
//
// The adjoint kernel runs the general-form step of one cell with R = Rev:
// every arithmetic operation appends a node to the thread's tape (its value's
// partial derivatives with respect to at most two operands), every read of
// the input state appends a leaf naming the state element, and the step's
// outputs carry the node that produced them.  A reverse sweep over the tape
// then turns the adjoints of the outputs into adjoints of the input state
// (scattered with atomic adds, since neighbouring cells read the same
// elements) and of the parameters theta = (ln A, Ta, T_wall, u_in).
// Branches (WENO upwind side, ghost modes, max(Y, 0)) are taken on the
// values, as in the forward step, so this is the exact transpose of the
// derivative of the discrete step.
//
// The tape lives in global memory, node k of thread t at k * NT + t (NT
// threads in the launch: the sweeps of a warp touch consecutive addresses);
// the tape pointers are in constant memory, so one adjoint launch runs at a
// time per device.
#pragma once
#include <cmath>
#include <cstdint>

namespace lbfd {

// node parents: >= 0 an earlier node, -1 none, -2 a state leaf (a0 holds the
// element index), -3 a parameter leaf (a0 holds the parameter, a1 the
// derivative of the value with respect to it)
constexpr int REV_NONE = -1, REV_STATE = -2, REV_THETA = -3;

struct RevTape {
    double* a0;  // [maxn][nt] partial with respect to parent 0
    double* a1;  // [maxn][nt] partial with respect to parent 1
    int16_t* p0;
    int16_t* p1;
    double* adj;                // [maxn][nt] adjoints during the sweep
    const void* in_base;        // the input state (RevStore elements)
    int maxn;                   // nodes per thread
    int* overflow;              // set when a thread runs out of nodes
};

// the tape pointers of the running adjoint launch (lbfd_adjoint.cu is the
// only translation unit that includes this header)
__constant__ RevTape rev_tape;
// nodes used by each thread of a block (dynamic shared memory, one int per
// thread)
extern __shared__ int rev_count_dyn[];

// i = node + 1, 0 for a constant (so that zero-filled memory is constant)
struct Rev {
    double v;
    int i;
    __host__ __device__ Rev() : v(0.0), i(0) {}
    __host__ __device__ Rev(double x) : v(x), i(0) {}
    __host__ __device__ Rev(int x) : v((double)x), i(0) {}
    __host__ __device__ Rev(double x, int node) : v(x), i(node + 1) {}
    __device__ inline Rev(const struct RevStore& s);
};

// a state element as the adjoint kernel stores it: the value and, for an
// output, the node that produced it (node + 1, 0 if none)
struct RevStore {
    double v;
    int i;
    int pad;
    __host__ __device__ RevStore() : v(0.0), i(0), pad(0) {}
    __host__ __device__ RevStore(const Rev& r) : v(r.v), i(r.i), pad(0) {}
};

__device__ __forceinline__ long long rev_thread() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long rev_threads() { return (long long)gridDim.x * blockDim.x; }

__device__ __forceinline__ int rev_push(double a0, int p0, double a1, int p1)
{
    int& n = rev_count_dyn[threadIdx.x];
    const int k = n;
    if (k >= rev_tape.maxn) {
        *rev_tape.overflow = 1;
        return -1;
    }
    n = k + 1;
    const long long at = (long long)k * rev_threads() + rev_thread();
    rev_tape.a0[at] = a0;
    rev_tape.a1[at] = a1;
    rev_tape.p0[at] = (int16_t)p0;
    rev_tape.p1[at] = (int16_t)p1;
    return k;
}

// a read of the input state: a leaf naming the element
__device__ inline Rev::Rev(const RevStore& s) : v(s.v)
{
    const long long e = &s - reinterpret_cast<const RevStore*>(rev_tape.in_base);
    i = rev_push(__longlong_as_double(e), REV_STATE, 0.0, REV_NONE) + 1;
}

// a parameter leaf: value x, d x / d theta_k = dxdt
__device__ inline Rev rev_theta(double x, int k, double dxdt)
{
    return Rev(x, rev_push((double)k, REV_THETA, dxdt, REV_NONE));
}

// (a node index of -1 from a full tape makes the result a constant; the
// overflow flag tells the host)
__device__ inline Rev rev_unary(double v, const Rev& a, double da)
{
    if (a.i == 0) return Rev(v);
    return Rev(v, rev_push(da, a.i - 1, 0.0, REV_NONE));
}
__device__ inline Rev rev_binary(double v, const Rev& a, double da, const Rev& b, double db)
{
    if (a.i == 0 && b.i == 0) return Rev(v);
    if (a.i == 0) return Rev(v, rev_push(db, b.i - 1, 0.0, REV_NONE));
    if (b.i == 0) return Rev(v, rev_push(da, a.i - 1, 0.0, REV_NONE));
    return Rev(v, rev_push(da, a.i - 1, db, b.i - 1));
}

__device__ inline Rev operator+(const Rev& a, const Rev& b) { return rev_binary(a.v + b.v, a, 1.0, b, 1.0); }
__device__ inline Rev operator-(const Rev& a, const Rev& b) { return rev_binary(a.v - b.v, a, 1.0, b, -1.0); }
__device__ inline Rev operator*(const Rev& a, const Rev& b) { return rev_binary(a.v * b.v, a, b.v, b, a.v); }
__device__ inline Rev operator/(const Rev& a, const Rev& b)
{
    const double q = a.v / b.v;
    return rev_binary(q, a, 1.0 / b.v, b, -q / b.v);
}
__device__ inline Rev operator-(const Rev& a) { return rev_unary(-a.v, a, -1.0); }
__device__ inline Rev& operator+=(Rev& a, const Rev& b) { return a = a + b; }
__device__ inline Rev& operator-=(Rev& a, const Rev& b) { return a = a - b; }
__device__ inline Rev& operator*=(Rev& a, const Rev& b) { return a = a * b; }
__device__ inline Rev& operator/=(Rev& a, const Rev& b) { return a = a / b; }
__device__ inline bool operator<(const Rev& a, const Rev& b) { return a.v < b.v; }
__device__ inline bool operator>(const Rev& a, const Rev& b) { return a.v > b.v; }
__device__ inline bool operator<=(const Rev& a, const Rev& b) { return a.v <= b.v; }
__device__ inline bool operator>=(const Rev& a, const Rev& b) { return a.v >= b.v; }
__device__ inline Rev exp(const Rev& a)
{
    const double e = ::exp(a.v);
    return rev_unary(e, a, e);
}
__device__ inline Rev fdiv(const Rev& a, const Rev& b) { return a / b; }
__host__ __device__ inline double val(const Rev& x) { return x.v; }

template <typename R>
struct ScalarOf;
template <>
struct ScalarOf<Rev> {
    using type = double;
};

}  // namespace lbfd
