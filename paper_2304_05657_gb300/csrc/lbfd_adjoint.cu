// lbfd_adjoint.cu -- reverse-mode (discrete adjoint) step: given the adjoint
// lambda^{n+1} of the state after a step, the adjoint lambda^n of the state
// before it and the contribution to dJ/dtheta, theta = (ln A, Ta, T_wall,
// u_in).  One thread per fluid cell records the general-form step of its
// cell on a tape (lbfd_rev.cuh), several steps per launch, and one thread per
// cell sweeps a step's tape backwards.
#include <type_traits>

#include "lbfd_internal.h"
#include "lbfd_step_general.cuh"
#include "lbfd_rev.cuh"

namespace lbfd {

constexpr int REV_BLOCK = 64;
// the adjoints of this many recent tape nodes per thread stay in shared
// memory during the reverse sweep; the loads of tape entries and of farther
// adjoints run this many sweeps ahead
constexpr int REV_WIN = 32, REV_LAG = 8;

// the state as tape input (values only): FP64, or the FP32 state of the
// mixed form (V = float records its step in FP32)
template <typename S, typename V>
__global__ void __launch_bounds__(256) to_rev_kernel(long long n, const S* __restrict__ in,
                                                     RevStoreT<V>* __restrict__ out)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = RevStoreT<V>(RevT<V>((double)in[e]));
}

// Record: thread t of the launch takes cell c0 + u, u = t % chunk, of the
// step from the state of slot t / chunk (several steps' tapes are recorded
// in one launch), and leaves its node count in count[t].
template <int DIM, typename V>
__global__ void __launch_bounds__(REV_BLOCK, 8)
    adjoint_record_kernel(StepParams<RevT<V>> P, const RevStoreT<V>* __restrict__ rin, RevStoreT<V>* __restrict__ rout,
                          const uint8_t* __restrict__ solid, long long c0, long long n, long long chunk,
                          long long nel, int* __restrict__ count)
{
    constexpr int Q = DIM == 2 ? 9 : 27;
    rev_count_dyn[threadIdx.x] = 0;
    const long long t = rev_thread();
    const long long slot = t / chunk, u = t - slot * chunk, c = c0 + u;
    if (u < n && c < P.ncell && !solid[c]) {
        // theta = (ln A, Ta, T_wall, u_in) are the tape's first four nodes
        // (parameter leaves), and P names them as the nodes of A dt, Ta, the
        // isothermal wall and solid temperatures and u_in (rev_params)
        rev_push<V>(V(0), REV_THETA, P.A_lat.v, REV_NONE);  // d(A dt)/d(ln A) = A dt
        rev_push<V>(V(1), REV_THETA, V(1), REV_NONE);
        rev_push<V>(V(2), REV_THETA, V(1), REV_NONE);
        rev_push<V>(V(3), REV_THETA, V(1), REV_NONE);
        const long long N = P.N;
        const RevStoreT<V>* in = rin + slot * nel;
        RevStoreT<V>* out = rout + slot * nel;
        int p[3];
        p[0] = (int)(c % P.nx);
        const long long r = c / P.nx;
        p[1] = (int)(r % P.ny);
        p[2] = (int)(r / P.ny);
        cell_step_general<DIM, RevStoreT<V>, RevT<V>>(P, p, c, in, out, in + (long long)Q * N, out + (long long)Q * N,
                                              in + (long long)(Q + 1) * N, out + (long long)(Q + 1) * N, solid);
    }
    count[t] = rev_count_dyn[threadIdx.x];
}

// Reverse sweep of the tapes of slot `slot` (threads slot * chunk + u of the
// record launch, NT threads in all): lam += (dF/dx)^T lam_next, dtheta +=
// (dF/dtheta)^T lam_next.  The adjoints of the REV_WIN most recent nodes not
// yet swept live in shared memory (slot k % REV_WIN of this thread), older
// ones in adj (node k of thread u at k * chunk + u), which the farther
// children update with atomic adds that nothing waits for (the thread's own
// later read of the same element sees them).  When node k is swept its slot
// passes to node k - REV_WIN, whose value in adj is final then: it is loaded
// at once and added REV_LAG sweeps later.  The tape entries of node
// k - REV_LAG are loaded when node k is swept, so no sweep waits on a load;
// theta contributions accumulate in registers.  The partials (V) enter FP64
// products: the adjoints are FP64 whatever V is.
template <typename V>
__global__ void __launch_bounds__(REV_BLOCK)
    adjoint_sweep_kernel(const RevStoreT<V>* __restrict__ out, const uint8_t* __restrict__ solid, long long c0,
                         long long n, long long ncell, long long N, int planes, long long slot, long long NT,
                         long long ebase, const int* __restrict__ count, const double* __restrict__ lam_next,
                         double* __restrict__ lam, double* __restrict__ dtheta, double* __restrict__ adj_buf,
                         const V* __restrict__ tape_a0, const V* __restrict__ tape_a1,
                         const int32_t* __restrict__ tape_par, int* __restrict__ max_nodes)
{
    extern __shared__ double win_dyn[];
    const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned chunk = gridDim.x * blockDim.x;
    const long long c = c0 + u;
    if (u >= n || c >= ncell || solid[c]) return;
    const long long t = slot * chunk + u;
    const int nn = count[t];
    atomicMax(max_nodes, nn);
    // node offsets in the tape (k * NT) and in adj (k * chunk) fit 32 bits
    // (the host keeps maxn * NT below 2^32)
    double* adj = adj_buf + u;
    double* win = win_dyn + threadIdx.x;
    constexpr unsigned WM = REV_WIN - 1;
    for (int k = 0; k < nn - REV_WIN; ++k) adj[(unsigned)k * chunk] = 0.0;
#pragma unroll
    for (int j = 0; j < REV_WIN; ++j) win[j * REV_BLOCK] = 0.0;
    for (int j = 0; j < planes; ++j) {  // seed the outputs of the cell with lambda^{n+1}
        const long long e = (long long)j * N + c;
        const int node = out[e].i - 1;
        if (node < 0) continue;
        if (node >= nn - REV_WIN) win[((unsigned)node & WM) * REV_BLOCK] += lam_next[e];
        else adj[(unsigned)node * chunk] += lam_next[e];
    }
    const V* a0 = tape_a0 + t;
    const V* a1 = tape_a1 + t;
    const int32_t* par = tape_par + t;
    double th0 = 0.0, th1 = 0.0, th2 = 0.0, th3 = 0.0;
    // queue slot j holds, while node k = k0 - j is swept, its tape entry and
    // the adj value of node k + REV_LAG - REV_WIN
    double lag[REV_LAG];
    V qa0[REV_LAG], qa1[REV_LAG];
    int32_t qp[REV_LAG];
#pragma unroll
    for (int j = 0; j < REV_LAG; ++j) {
        const int k = nn - 1 - j;
        lag[j] = 0.0;
        qa0[j] = qa1[j] = V(0);
        qp[j] = -1;  // both parents REV_NONE
        if (k >= 0) {
            const unsigned at = (unsigned)k * (unsigned)NT;
            qp[j] = par[at];
            qa0[j] = a0[at];
            qa1[j] = a1[at];
        }
    }
    auto add = [&](int q, int k, double x) {
        if (q >= k - REV_WIN) win[((unsigned)q & WM) * REV_BLOCK] += x;
        else atomicAdd(&adj[(unsigned)q * chunk], x);
    };
    // one sweep step; CHECK: near the start of the tape, where the window,
    // the far values and the prefetch reach below node 0 (the groups of
    // REV_LAG nodes from the end that lie wholly above REV_WIN need none)
    auto sweep = [&](auto check, int k, int j) {
        constexpr bool CHECK = decltype(check)::value;
        if (!CHECK || k + REV_LAG - REV_WIN >= 0) win[((unsigned)(k + REV_LAG) & WM) * REV_BLOCK] += lag[j];
        double* ws = win + ((unsigned)k & WM) * REV_BLOCK;
        const double a = *ws;
        *ws = 0.0;  // from now on the slot of node k - REV_WIN
        lag[j] = !CHECK || k >= REV_WIN ? adj[(unsigned)(k - REV_WIN) * chunk] : 0.0;
        const int q0 = (int16_t)(qp[j] & 0xffff), q1 = qp[j] >> 16;
        const V v0 = qa0[j];
        const double x0 = (double)v0, x1 = (double)qa1[j];
        if (!CHECK || k >= REV_LAG) {
            const unsigned at = (unsigned)(k - REV_LAG) * (unsigned)NT;
            qp[j] = par[at];
            qa0[j] = a0[at];
            qa1[j] = a1[at];
        }
        if (a == 0.0) return;
        if (q0 >= 0) {
            add(q0, k, a * x0);
        } else if (q0 == REV_STATE) {
            atomicAdd(&lam[rev_index_of(v0) - ebase], a);
        } else if (q0 == REV_THETA) {
            const double d = a * x1;
            const int m = (int)x0;
            th0 += m == 0 ? d : 0.0;
            th1 += m == 1 ? d : 0.0;
            th2 += m == 2 ? d : 0.0;
            th3 += m == 3 ? d : 0.0;
        }
        if (q1 >= 0) add(q1, k, a * x1);
    };
    int k0 = nn - 1;
    for (; k0 - (REV_LAG - 1) >= REV_WIN; k0 -= REV_LAG) {
#pragma unroll
        for (int j = 0; j < REV_LAG; ++j) sweep(std::false_type{}, k0 - j, j);
    }
    for (; k0 >= 0; k0 -= REV_LAG) {
#pragma unroll
        for (int j = 0; j < REV_LAG; ++j) {
            if (k0 - j < 0) break;
            sweep(std::true_type{}, k0 - j, j);
        }
    }
    if (th0 != 0.0) atomicAdd(&dtheta[0], th0);
    if (th1 != 0.0) atomicAdd(&dtheta[1], th1);
    if (th2 != 0.0) atomicAdd(&dtheta[2], th2);
    if (th3 != 0.0) atomicAdd(&dtheta[3], th3);
}

// the parameters as reverse-mode constants, except those that depend on
// theta: they name the parameter leaves that each thread pushes first (node
// 0: A dt, 1: Ta, 2: the isothermal wall and solid temperatures, 3: u_in)
template <typename V>
static StepParams<RevT<V>> rev_params(const StepParams<double>& D)
{
    using Rv = RevT<V>;
    StepParams<Rv> P;
    memset(&P, 0, sizeof P);  // zero bytes are constants (node 0)
    P.dim = D.dim;
    P.nx = D.nx;
    P.ny = D.ny;
    P.nz = D.nz;
    P.ncell = D.ncell;
    P.N = D.N;
    for (int f = 0; f < 6; ++f) {
        P.bc[f] = D.bc[f];
        P.T_wall[f] = D.bc[f] == BC_WALL_ISOTHERMAL ? Rv(D.T_wall[f], 2) : Rv(D.T_wall[f]);
        P.face_solid[f] = D.face_solid[f];
    }
    for (int k = 0; k < NSP; ++k) {
        P.inv_Wk[k] = Rv(D.inv_Wk[k]);
        P.yield[k] = Rv(D.yield[k]);
        P.a_diff[k] = Rv(D.a_diff[k]);
        P.a12[k] = Rv(D.a12[k]);
        P.Y_in[k] = Rv(D.Y_in[k]);
    }
    P.fuel = D.fuel;
    P.oxid = D.oxid;
    P.A_lat = Rv(D.A_lat, 0);
    P.Ta = Rv(D.Ta, 1);
    P.Q_cp = Rv(D.Q_cp);
    P.A_lat_d = D.A_lat_d;
    P.Ta_d = D.Ta_d;
    P.T_fp64 = Rv(D.T_fp64);
    P.omega_s = Rv(D.omega_s);
    P.omega_b = Rv(D.omega_b);
    P.omega_hi = Rv(D.omega_hi);
    P.alpha = Rv(D.alpha);
    P.alpha12 = Rv(D.alpha12);
    P.lam_yield = Rv(D.lam_yield);
    P.u_in = Rv(D.u_in, 3);
    P.T_in = Rv(D.T_in);
    P.invW_in = Rv(D.invW_in);
    P.rho_in = Rv(D.rho_in);
    P.T_solid = D.solid_isothermal ? Rv(D.T_solid, 2) : Rv(D.T_solid);
    P.solid_isothermal = D.solid_isothermal;
    P.poiseuille = D.poiseuille;
    P.epsY = Rv(D.epsY);
    P.epsT = Rv(D.epsT);
    P.cs = Rv(D.cs);
    P.curved = 0;
    P.link_row = nullptr;
    P.link_q = nullptr;
    P.ghost_row = nullptr;
    P.gval = nullptr;
    return P;
}

size_t adjoint_node_bytes(bool fp32) { return 2 * (fp32 ? sizeof(float) : sizeof(double)) + sizeof(int32_t); }
size_t rev_store_bytes(bool fp32) { return fp32 ? sizeof(RevStoreT<float>) : sizeof(RevStoreT<double>); }

template <typename V>
static cudaError_t record_steps(const StepParams<double>& Pd, int planes, const void* states, size_t state_bytes,
                                int slots, bool fp32, const uint8_t* solid, long long c0, long long n,
                                const AdjointWork& w, cudaStream_t stream)
{
    const long long nel = (long long)planes * Pd.N;
    RevStoreT<V>* rin = (RevStoreT<V>*)w.rin;
    cudaError_t e;
    const unsigned nb = (unsigned)((nel + 255) / 256);
    for (int j = 0; j < slots; ++j) {
        const char* st = (const char*)states + (size_t)j * state_bytes;
        if (fp32)
            to_rev_kernel<float, V><<<nb, 256, 0, stream>>>(nel, (const float*)st, rin + (long long)j * nel);
        else
            to_rev_kernel<double, V><<<nb, 256, 0, stream>>>(nel, (const double*)st, rin + (long long)j * nel);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    RevTape tp;
    tp.a0 = w.a0;
    tp.a1 = w.a1;
    tp.par = w.par;
    tp.in_base = rin;
    tp.maxn = w.maxn;
    tp.overflow = w.flags;
    if ((e = cudaMemcpyToSymbolAsync(rev_tape, &tp, sizeof tp, 0, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return e;
    const StepParams<RevT<V>> P = rev_params<V>(Pd);
    // the tape is sized for w.slots * w.chunk threads: launch that many per
    // slot (idle ones return at once) so that the interleaved layout has a
    // fixed stride
    const unsigned blocks = (unsigned)((w.slots * w.chunk + REV_BLOCK - 1) / REV_BLOCK);
    adjoint_record_kernel<2, V><<<blocks, REV_BLOCK, REV_BLOCK * sizeof(int), stream>>>(
        P, rin, (RevStoreT<V>*)w.rout, solid, c0, n, w.chunk, nel, w.count);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_record(int dim, const StepParams<double>& Pd, int planes, const void* states,
                                  size_t state_bytes, int slots, bool fp32, const uint8_t* solid, long long c0,
                                  long long n, const AdjointWork& w, cudaStream_t stream)
{
    if (dim != 2 || slots < 1 || slots > w.slots) return cudaErrorInvalidValue;
    // the FP32 tape names state elements in 31 bits
    if (fp32 && (long long)w.slots * planes * Pd.N >= (1ll << 31)) return cudaErrorInvalidValue;
    if (fp32) return record_steps<float>(Pd, planes, states, state_bytes, slots, fp32, solid, c0, n, w, stream);
    return record_steps<double>(Pd, planes, states, state_bytes, slots, fp32, solid, c0, n, w, stream);
}

template <typename V>
static cudaError_t sweep_step(const StepParams<double>& Pd, int planes, int slot, const uint8_t* solid, long long c0,
                              long long n, const double* lam_next, double* lam, double* dtheta, const AdjointWork& w,
                              cudaStream_t stream)
{
    const long long nel = (long long)planes * Pd.N;
    constexpr size_t smem = REV_BLOCK * REV_WIN * sizeof(double);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(adjoint_sweep_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
        return e;
    const unsigned blocks = (unsigned)(w.chunk / REV_BLOCK);
    adjoint_sweep_kernel<V><<<blocks, REV_BLOCK, smem, stream>>>(
        (const RevStoreT<V>*)w.rout + slot * nel, solid, c0, n, Pd.ncell, Pd.N, planes, slot,
        (long long)w.slots * w.chunk, slot * nel, w.count, lam_next, lam, dtheta, w.adj, (const V*)w.a0,
        (const V*)w.a1, w.par, w.flags + 1);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_sweep(const StepParams<double>& Pd, int planes, int slot, bool fp32, const uint8_t* solid,
                                 long long c0, long long n, const double* lam_next, double* lam, double* dtheta,
                                 const AdjointWork& w, cudaStream_t stream)
{
    if (slot < 0 || slot >= w.slots) return cudaErrorInvalidValue;
    if ((unsigned long long)w.maxn * w.slots * w.chunk >= (1ull << 32)) return cudaErrorInvalidValue;  // 32-bit offsets
    if (fp32) return sweep_step<float>(Pd, planes, slot, solid, c0, n, lam_next, lam, dtheta, w, stream);
    return sweep_step<double>(Pd, planes, slot, solid, c0, n, lam_next, lam, dtheta, w, stream);
}

// ---------------------------------------------------------------------------
// Objectives of the final state and their adjoint seeds
// ---------------------------------------------------------------------------

// heat release of one cell, h = rho (Q/cp) q (Sec. IV observables), and its
// partial derivatives with respect to T and Y_k
template <typename S>
__device__ __forceinline__ double cell_hrr(const StepParams<double>& P, const S* T, const S* Y, long long c,
                                           double* dT, double* dY)
{
    const double Tc = (double)T[c];
    double Yc[NSP], invW = 0.0;
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
        Yc[k] = (double)Y[(long long)k * P.N + c];
        invW += Yc[k] * P.inv_Wk[k];
    }
    const double rho = P.T_in * P.invW_in / (Tc * invW);
    const double yf = pick_species(Yc, P.fuel), yo = pick_species(Yc, P.oxid);
    const double yfp = yf > 0.0 ? yf : 0.0, yop = yo > 0.0 ? yo : 0.0;
    const double e = P.A_lat * ::exp(-P.Ta / Tc);
    const double h = rho * P.Q_cp * e * yfp * yop;
    if (dT) {
        *dT = h * (P.Ta / (Tc * Tc) - 1.0 / Tc);
#pragma unroll
        for (int k = 0; k < NSP; ++k) {
            double d = -h * P.inv_Wk[k] / invW;  // through rho
            if (k == P.fuel && yf > 0.0) d += rho * P.Q_cp * e * yop;
            if (k == P.oxid && yo > 0.0) d += rho * P.Q_cp * e * yfp;
            dY[k] = d;
        }
    }
    return h;
}

// red[0] += sum h, red[1] += sum h w (FP64, warp shuffles + atomics)
template <typename S>
__global__ void __launch_bounds__(256) quench_sums_kernel(StepParams<double> P, const S* __restrict__ T,
                                                          const S* __restrict__ Y, const uint8_t* __restrict__ solid,
                                                          const double* __restrict__ wgt, double* red)
{
    double a0 = 0.0, a1 = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < P.ncell; c += stride) {
        if (solid[c]) continue;
        const double h = cell_hrr(P, T, Y, c, nullptr, nullptr);
        a0 += h;
        a1 += h * wgt[c];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a0 += __shfl_down_sync(0xffffffffu, a0, off);
        a1 += __shfl_down_sync(0xffffffffu, a1, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&red[0], a0);
        atomicAdd(&red[1], a1);
    }
}

// lam = seed * dJ/dstate for J = (S1/S0)^(-1/4), S0 = sum h, S1 = sum h w;
// dtheta += seed * (the explicit dJ/d ln A and dJ/dTa through h)
template <typename S>
__global__ void __launch_bounds__(256) quench_seed_kernel(StepParams<double> P, const S* __restrict__ T,
                                                          const S* __restrict__ Y, const uint8_t* __restrict__ solid,
                                                          const double* __restrict__ wgt, double S0, double S1,
                                                          double J, double seed, double* __restrict__ lam,
                                                          double* dtheta, int Q)
{
    double gA = 0.0, gTa = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < P.ncell; c += stride) {
        if (solid[c]) continue;
        double dT, dY[NSP];
        const double h = cell_hrr(P, T, Y, c, &dT, dY);
        const double dJdh = seed * (-0.25) * J * (wgt[c] / S1 - 1.0 / S0);
        lam[(long long)Q * P.N + c] += dJdh * dT;
#pragma unroll
        for (int k = 0; k < NSP; ++k) lam[(long long)(Q + 1 + k) * P.N + c] += dJdh * dY[k];
        gA += dJdh * h;                           // dh / d ln A = h
        gTa += dJdh * (-h / (double)T[c]);        // dh / dTa = -h / T
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        gA += __shfl_down_sync(0xffffffffu, gA, off);
        gTa += __shfl_down_sync(0xffffffffu, gTa, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&dtheta[0], gA);
        atomicAdd(&dtheta[1], gTa);
    }
}

static unsigned red_blocks(long long ncell)
{
    const long long want = (ncell + 255) / 256;
    return (unsigned)(want < 1024 ? (want > 0 ? want : 1) : 1024);
}

cudaError_t launch_quench_sums(const StepParams<double>& Pd, StateView st, bool fp32, const uint8_t* solid,
                               const double* wgt, double* red, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(red, 0, 2 * sizeof(double), stream);
    if (e != cudaSuccess) return e;
    const unsigned nb = red_blocks(Pd.ncell);
    if (fp32)
        quench_sums_kernel<float><<<nb, 256, 0, stream>>>(Pd, (const float*)st.T, (const float*)st.Y, solid, wgt, red);
    else
        quench_sums_kernel<double><<<nb, 256, 0, stream>>>(Pd, (const double*)st.T, (const double*)st.Y, solid, wgt,
                                                            red);
    return cudaGetLastError();
}

cudaError_t launch_quench_seed(const StepParams<double>& Pd, StateView st, bool fp32, const uint8_t* solid,
                               const double* wgt, double S0, double S1, double J, double seed, double* lam,
                               double* dtheta, int Q, cudaStream_t stream)
{
    const unsigned nb = red_blocks(Pd.ncell);
    if (fp32)
        quench_seed_kernel<float><<<nb, 256, 0, stream>>>(Pd, (const float*)st.T, (const float*)st.Y, solid, wgt, S0,
                                                          S1, J, seed, lam, dtheta, Q);
    else
        quench_seed_kernel<double><<<nb, 256, 0, stream>>>(Pd, (const double*)st.T, (const double*)st.Y, solid, wgt,
                                                           S0, S1, J, seed, lam, dtheta, Q);
    return cudaGetLastError();
}

}  // namespace lbfd
