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
    int32_t* par;  // [maxn][nt] parent 0 in the low 16 bits, parent 1 in the high
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

// A value and its derivative with respect to one tape node: d v / d node =
// s, i = node + 1, 0 for a constant (so that zero-filled memory is
// constant).  Operations on one node (unary functions, constant factors and
// terms) only change s: nodes are pushed only where two nodes meet (and for
// reads of the state), which keeps the tape short.
struct Rev {
    double v;
    double s;
    int i;
    __host__ __device__ Rev() : v(0.0), s(0.0), i(0) {}
    __host__ __device__ Rev(double x) : v(x), s(0.0), i(0) {}
    __host__ __device__ Rev(int x) : v((double)x), s(0.0), i(0) {}
    __host__ __device__ Rev(double x, int node) : v(x), s(1.0), i(node + 1) {}
    __device__ inline Rev(const struct RevStore& st);
};

// a state element as the adjoint kernel stores it: the value and, for an
// output, the node that produced it (node + 1, 0 if none) with unit
// derivative
struct RevStore {
    double v;
    int i;
    int pad;
    __host__ __device__ RevStore() : v(0.0), i(0), pad(0) {}
    __device__ inline RevStore(const Rev& r);
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
    if (p1 >= 0 || p0 == REV_THETA) rev_tape.a1[at] = a1;  // read only then
    rev_tape.par[at] = (int32_t)(((uint32_t)p1 << 16) | ((uint32_t)p0 & 0xffffu));
    return k;
}

// a read of the input state: a leaf naming the element (not inlined, as
// rev_link below)
__device__ __noinline__ int rev_leaf(long long e) { return rev_push(__longlong_as_double(e), REV_STATE, 0.0, REV_NONE) + 1; }
__device__ inline Rev::Rev(const RevStore& st) : v(st.v), s(1.0)
{
    i = rev_leaf(&st - reinterpret_cast<const RevStore*>(rev_tape.in_base));
}

// the node and derivative of a value with partials da, db with respect to
// operands (as, ai), (bs, bi).  A node is pushed only for two distinct
// nodes; a full tape makes the result a constant (the overflow flag tells
// the host).  Not inlined: the recorded step is one long straight-line
// body, and a call per operation keeps it small enough for the instruction
// caches.
struct RevLink {
    double s;
    int i;
};
// x * s, without an FP64 multiply when either factor is 1 (most derivatives
// and partials).  FP64 arithmetic is the scarce resource of the recording:
// the multiply sits in a branch of its own so that it is not executed
// speculatively.
__device__ __forceinline__ double rev_scale(double x, double s)
{
    constexpr long long ONE = 0x3FF0000000000000ll;
    double r;
    if (__double_as_longlong(s) == ONE)
        r = x;
    else if (__double_as_longlong(x) == ONE)
        r = s;
    else
        asm volatile("mul.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(x), "d"(s));
    return r;
}
__device__ __noinline__ RevLink rev_link(double da, double as, int ai, double db, double bs, int bi)
{
    RevLink r;
    if (ai == bi) {  // one node, or constants
        r.i = ai;
        r.s = ai == 0 ? 0.0 : rev_scale(da, as) + rev_scale(db, bs);
    } else if (bi == 0) {
        r.i = ai;
        r.s = rev_scale(da, as);
    } else if (ai == 0) {
        r.i = bi;
        r.s = rev_scale(db, bs);
    } else {
        r.i = rev_push(rev_scale(da, as), ai - 1, rev_scale(db, bs), bi - 1) + 1;
        r.s = 1.0;
    }
    return r;
}
__device__ inline Rev rev_unary(double v, const Rev& a, double da)
{
    Rev r(v);
    if (a.i != 0) {
        r.i = a.i;
        r.s = rev_scale(da, a.s);
    }
    return r;
}
__device__ inline Rev rev_binary(double v, const Rev& a, double da, const Rev& b, double db)
{
    Rev r(v);
    const RevLink l = rev_link(da, a.s, a.i, db, b.s, b.i);
    r.s = l.s;
    r.i = l.i;
    return r;
}

// an output: a node of unit derivative (pushed when the value's derivative
// with respect to its node is not 1)
__device__ inline RevStore::RevStore(const Rev& r) : v(r.v), i(r.i), pad(0)
{
    if (r.i != 0 && r.s != 1.0) i = rev_push(r.s, r.i - 1, 0.0, REV_NONE) + 1;
}

__device__ inline Rev operator+(const Rev& a, const Rev& b) { return rev_binary(a.v + b.v, a, 1.0, b, 1.0); }
__device__ inline Rev operator-(const Rev& a, const Rev& b) { return rev_binary(a.v - b.v, a, 1.0, b, -1.0); }
__device__ inline Rev operator*(const Rev& a, const Rev& b) { return rev_binary(a.v * b.v, a, b.v, b, a.v); }
__device__ inline Rev operator/(const Rev& a, const Rev& b)
{
    const double q = a.v / b.v;
    if (b.i == 0) return rev_unary(q, a, 1.0 / b.v);
    const double r = 1.0 / b.v;
    return rev_binary(q, a, r, b, -q * r);
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
