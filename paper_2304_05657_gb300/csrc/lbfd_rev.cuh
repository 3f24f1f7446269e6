// lbfd_rev.cuh -- reverse-mode numbers for the discrete adjoint of one step.
//
// The adjoint kernel runs the general-form step of one cell with R = RevT<V>:
// every arithmetic operation that joins two recorded values appends a node
// to the thread's tape (its value's partial derivatives with respect to the
// two operands), every read of the input state appends a leaf naming the
// state element, and the step's outputs carry the node that produced them.
// A reverse sweep over the tape then turns the adjoints of the outputs into
// adjoints of the input state (scattered with atomic adds, since
// neighbouring cells read the same elements) and of the parameters
// theta = (ln A, Ta, T_wall, u_in).  Branches (WENO upwind side, ghost
// modes, max(Y, 0)) are taken on the values, as in the forward step, so this
// is the exact transpose of the derivative of the discrete step.
//
// V is the type of the recorded values and partials: double for the FP64
// adjoint, float for the adjoint of the FP32 forward pass (the adjoints
// themselves are accumulated in FP64 by the sweep either way).
//
// The tape lives in global memory, node k of thread t at k * NT + t (NT
// threads in the launch: the sweeps of a warp touch consecutive addresses);
// the tape pointers are in constant memory, so one record launch runs at a
// time per device.
#pragma once
#include <cmath>
#include <cstdint>

namespace lbfd {

// node parents: >= 0 an earlier node, -1 none, -2 a state leaf (a0 holds the
// element index in its bits), -3 a parameter leaf (a0 holds the parameter,
// a1 the derivative of the value with respect to it)
constexpr int REV_NONE = -1, REV_STATE = -2, REV_THETA = -3;

struct RevTape {
    void* a0;       // [maxn][nt] partial with respect to parent 0 (V)
    void* a1;       // [maxn][nt] partial with respect to parent 1 (V)
    int32_t* par;   // [maxn][nt] parent 0 in the low 16 bits, parent 1 in the high
    const void* in_base;  // the input state (RevStoreT<V> elements)
    int maxn;             // nodes per thread
    int* overflow;        // set when a thread runs out of nodes
};

// the tape pointers of the running record launch (lbfd_adjoint.cu is the
// only translation unit that includes this header)
__constant__ RevTape rev_tape;
// nodes used by each thread of a block (dynamic shared memory, one int per
// thread)
extern __shared__ int rev_count_dyn[];

template <typename V>
struct RevStoreT;

// A value and its derivative with respect to one tape node: d v / d node =
// s, i = node + 1, 0 for a constant (so that zero-filled memory is
// constant).  Operations on one node (unary functions, constant factors and
// terms) only change s: nodes are pushed only where two nodes meet (and for
// reads of the state), which keeps the tape short.
template <typename V>
struct RevT {
    V v;
    V s;
    int i;
    __host__ __device__ RevT() : v(V(0)), s(V(0)), i(0) {}
    __host__ __device__ RevT(double x) : v(V(x)), s(V(0)), i(0) {}
    __host__ __device__ RevT(int x) : v(V(x)), s(V(0)), i(0) {}
    __host__ __device__ RevT(double x, int node) : v(V(x)), s(V(1)), i(node + 1) {}
    __device__ inline RevT(const RevStoreT<V>& st);
};
using Rev = RevT<double>;
using RevF = RevT<float>;

// a state element as the record kernel stores it: the value and, for an
// output, the node that produced it (node + 1, 0 if none) with unit
// derivative
template <typename V>
struct RevStoreT {
    V v;
    int i;
    __host__ __device__ RevStoreT() : v(V(0)), i(0) {}
    __device__ inline RevStoreT(const RevT<V>& r);
};

__device__ __forceinline__ long long rev_thread() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long rev_threads() { return (long long)gridDim.x * blockDim.x; }

template <typename V>
__device__ __forceinline__ int rev_push(V a0, int p0, V a1, int p1)
{
    int& n = rev_count_dyn[threadIdx.x];
    const int k = n;
    if (k >= rev_tape.maxn) {
        *rev_tape.overflow = 1;
        return -1;
    }
    n = k + 1;
    const long long at = (long long)k * rev_threads() + rev_thread();
    static_cast<V*>(rev_tape.a0)[at] = a0;
    if (p1 >= 0 || p0 == REV_THETA) static_cast<V*>(rev_tape.a1)[at] = a1;  // read only then
    rev_tape.par[at] = (int32_t)(((uint32_t)p1 << 16) | ((uint32_t)p0 & 0xffffu));
    return k;
}

// the element index of a state leaf in the bits of a partial (float: the
// host keeps the indices below 2^31)
__device__ __forceinline__ double rev_index_bits(double, long long e) { return __longlong_as_double(e); }
__device__ __forceinline__ float rev_index_bits(float, long long e) { return __int_as_float((int)e); }
__device__ __forceinline__ long long rev_index_of(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ long long rev_index_of(float x) { return (long long)__float_as_int(x); }

// a read of the input state: a leaf naming the element (not inlined, as
// rev_link below)
template <typename V>
__device__ __noinline__ int rev_leaf(long long e)
{
    return rev_push<V>(rev_index_bits(V(0), e), REV_STATE, V(0), REV_NONE) + 1;
}
template <typename V>
__device__ inline RevT<V>::RevT(const RevStoreT<V>& st) : v(st.v), s(V(1))
{
    i = rev_leaf<V>(&st - reinterpret_cast<const RevStoreT<V>*>(rev_tape.in_base));
}

// x * s.  In FP64 without a multiply when either factor is 1 (most
// derivatives and partials): FP64 arithmetic is the scarce resource of the
// recording, and the multiply sits in a branch of its own so that it is not
// executed speculatively.  FP32 multiplies are cheap.
__device__ __forceinline__ float rev_scale(float x, float s) { return x * s; }
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

// the node and derivative of a value with partials da, db with respect to
// operands (as, ai), (bs, bi).  A node is pushed only for two distinct
// nodes; a full tape makes the result a constant (the overflow flag tells
// the host).  Not inlined: the recorded step is one long straight-line
// body, and a call per operation keeps it small enough for the instruction
// caches.
template <typename V>
struct RevLink {
    V s;
    int i;
};
template <typename V>
__device__ __noinline__ RevLink<V> rev_link(V da, V as, int ai, V db, V bs, int bi)
{
    RevLink<V> r;
    if (ai == bi) {  // one node, or constants
        r.i = ai;
        r.s = ai == 0 ? V(0) : rev_scale(da, as) + rev_scale(db, bs);
    } else if (bi == 0) {
        r.i = ai;
        r.s = rev_scale(da, as);
    } else if (ai == 0) {
        r.i = bi;
        r.s = rev_scale(db, bs);
    } else {
        r.i = rev_push<V>(rev_scale(da, as), ai - 1, rev_scale(db, bs), bi - 1) + 1;
        r.s = V(1);
    }
    return r;
}
template <typename V>
__device__ inline RevT<V> rev_unary(V v, const RevT<V>& a, V da)
{
    RevT<V> r;
    r.v = v;
    if (a.i != 0) {
        r.i = a.i;
        r.s = rev_scale(da, a.s);
    }
    return r;
}
template <typename V>
__device__ inline RevT<V> rev_binary(V v, const RevT<V>& a, V da, const RevT<V>& b, V db)
{
    RevT<V> r;
    r.v = v;
    const RevLink<V> l = rev_link<V>(da, a.s, a.i, db, b.s, b.i);
    r.s = l.s;
    r.i = l.i;
    return r;
}

// an output: a node of unit derivative (pushed when the value's derivative
// with respect to its node is not 1)
template <typename V>
__device__ inline RevStoreT<V>::RevStoreT(const RevT<V>& r) : v(r.v), i(r.i)
{
    if (r.i != 0 && r.s != V(1)) i = rev_push<V>(r.s, r.i - 1, V(0), REV_NONE) + 1;
}

template <typename V>
__device__ inline RevT<V> operator+(const RevT<V>& a, const RevT<V>& b)
{
    return rev_binary<V>(a.v + b.v, a, V(1), b, V(1));
}
template <typename V>
__device__ inline RevT<V> operator-(const RevT<V>& a, const RevT<V>& b)
{
    return rev_binary<V>(a.v - b.v, a, V(1), b, V(-1));
}
template <typename V>
__device__ inline RevT<V> operator*(const RevT<V>& a, const RevT<V>& b)
{
    return rev_binary<V>(a.v * b.v, a, b.v, b, a.v);
}
template <typename V>
__device__ inline RevT<V> operator/(const RevT<V>& a, const RevT<V>& b)
{
    const V q = a.v / b.v;
    if (b.i == 0) return rev_unary<V>(q, a, V(1) / b.v);
    const V r = V(1) / b.v;
    return rev_binary<V>(q, a, r, b, -q * r);
}
template <typename V>
__device__ inline RevT<V> operator-(const RevT<V>& a)
{
    return rev_unary<V>(-a.v, a, V(-1));
}
template <typename V>
__device__ inline RevT<V>& operator+=(RevT<V>& a, const RevT<V>& b) { return a = a + b; }
template <typename V>
__device__ inline RevT<V>& operator-=(RevT<V>& a, const RevT<V>& b) { return a = a - b; }
template <typename V>
__device__ inline RevT<V>& operator*=(RevT<V>& a, const RevT<V>& b) { return a = a * b; }
template <typename V>
__device__ inline RevT<V>& operator/=(RevT<V>& a, const RevT<V>& b) { return a = a / b; }
template <typename V>
__device__ inline bool operator<(const RevT<V>& a, const RevT<V>& b) { return a.v < b.v; }
template <typename V>
__device__ inline bool operator>(const RevT<V>& a, const RevT<V>& b) { return a.v > b.v; }
template <typename V>
__device__ inline bool operator<=(const RevT<V>& a, const RevT<V>& b) { return a.v <= b.v; }
template <typename V>
__device__ inline bool operator>=(const RevT<V>& a, const RevT<V>& b) { return a.v >= b.v; }
__device__ __forceinline__ double rev_exp(double x) { return ::exp(x); }
__device__ __forceinline__ float rev_exp(float x) { return expf(x); }
template <typename V>
__device__ inline RevT<V> exp(const RevT<V>& a)
{
    const V e = rev_exp(a.v);
    return rev_unary<V>(e, a, e);
}
template <typename V>
__device__ inline RevT<V> fdiv(const RevT<V>& a, const RevT<V>& b) { return a / b; }
template <typename V>
__host__ __device__ inline V val(const RevT<V>& x) { return x.v; }

template <typename R>
struct ScalarOf;
template <typename V>
struct ScalarOf<RevT<V>> {
    using type = V;
};

}  // namespace lbfd
