// lbfd_adjoint.cu -- reverse-mode (discrete adjoint) step: given the adjoint
// lambda^{n+1} of the state after a step, the adjoint lambda^n of the state
// before it and the contribution to dJ/dtheta, theta = (ln A, Ta, T_wall,
// u_in).  One thread per fluid cell records the general-form step of its
// cell on a tape (lbfd_rev.cuh) and sweeps it backwards.
#include "lbfd_internal.h"
#include "lbfd_step_general.cuh"
#include "lbfd_rev.cuh"

namespace lbfd {

constexpr int REV_BLOCK = 64;

// the state (FP64, or the FP32 state of the mixed form widened to FP64) as
// tape input (values only)
template <typename S>
__global__ void __launch_bounds__(256) to_rev_kernel(long long n, const S* __restrict__ in,
                                                     RevStore* __restrict__ out)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = RevStore(Rev((double)in[e]));
}

template <int DIM>
__global__ void __launch_bounds__(REV_BLOCK)
    adjoint_kernel(StepParams<Rev> P, const RevStore* __restrict__ in, RevStore* __restrict__ out,
                   const uint8_t* __restrict__ solid, long long c0, long long n, int planes,
                   const double* __restrict__ lam_next, double* __restrict__ lam, double* __restrict__ dtheta,
                   int* __restrict__ max_nodes)
{
    constexpr int Q = DIM == 2 ? 9 : 27;
    rev_count_dyn[threadIdx.x] = 0;
    const long long t = rev_thread();
    const long long c = c0 + t;
    if (t >= n || c >= P.ncell || solid[c]) return;
    const long long N = P.N;
    // forward: the step of cell c, recorded, with theta as parameter leaves
    {
        StepParams<Rev> Pl = P;
        Pl.A_lat = rev_theta(P.A_lat.v, 0, P.A_lat.v);  // d(A dt)/d(ln A)
        Pl.Ta = rev_theta(P.Ta.v, 1, 1.0);
        for (int f = 0; f < 6; ++f)
            if (P.bc[f] == BC_WALL_ISOTHERMAL) Pl.T_wall[f] = rev_theta(P.T_wall[f].v, 2, 1.0);
        if (P.solid_isothermal) Pl.T_solid = rev_theta(P.T_solid.v, 2, 1.0);
        Pl.u_in = rev_theta(P.u_in.v, 3, 1.0);
        int p[3];
        p[0] = (int)(c % P.nx);
        const long long r = c / P.nx;
        p[1] = (int)(r % P.ny);
        p[2] = (int)(r / P.ny);
        cell_step_general<DIM, RevStore, Rev>(Pl, p, c, in, out, in + (long long)Q * N, out + (long long)Q * N,
                                              in + (long long)(Q + 1) * N, out + (long long)(Q + 1) * N, solid);
    }
    // reverse sweep: seed the outputs of the cell with lambda^{n+1}
    const int nn = rev_count_dyn[threadIdx.x];
    atomicMax(max_nodes, nn);
    const long long NT = rev_threads();
    double* adj = rev_tape.adj + t;
    for (int k = 0; k < nn; ++k) adj[(long long)k * NT] = 0.0;
    for (int j = 0; j < planes; ++j) {
        const long long e = (long long)j * N + c;
        const int node = out[e].i - 1;
        if (node >= 0) adj[(long long)node * NT] += lam_next[e];
    }
    const double* a0 = rev_tape.a0 + t;
    const double* a1 = rev_tape.a1 + t;
    const int16_t* p0 = rev_tape.p0 + t;
    const int16_t* p1 = rev_tape.p1 + t;
    for (int k = nn - 1; k >= 0; --k) {
        const long long at = (long long)k * NT;
        const double a = adj[at];
        if (a == 0.0) continue;
        const int q0 = p0[at], q1 = p1[at];
        if (q0 >= 0) adj[(long long)q0 * NT] += a * a0[at];
        else if (q0 == REV_STATE) atomicAdd(&lam[__double_as_longlong(a0[at])], a);
        else if (q0 == REV_THETA) atomicAdd(&dtheta[(int)a0[at]], a * a1[at]);
        if (q1 >= 0) adj[(long long)q1 * NT] += a * a1[at];
    }
}

// the parameters as reverse-mode constants (theta becomes leaves per cell)
static StepParams<Rev> rev_params(const StepParams<double>& D)
{
    StepParams<Rev> P;
    memset(&P, 0, sizeof P);  // zero bytes are constants (node 0)
    P.dim = D.dim;
    P.nx = D.nx;
    P.ny = D.ny;
    P.nz = D.nz;
    P.ncell = D.ncell;
    P.N = D.N;
    for (int f = 0; f < 6; ++f) {
        P.bc[f] = D.bc[f];
        P.T_wall[f] = Rev(D.T_wall[f]);
        P.face_solid[f] = D.face_solid[f];
    }
    for (int k = 0; k < NSP; ++k) {
        P.inv_Wk[k] = Rev(D.inv_Wk[k]);
        P.yield[k] = Rev(D.yield[k]);
        P.a_diff[k] = Rev(D.a_diff[k]);
        P.a12[k] = Rev(D.a12[k]);
        P.Y_in[k] = Rev(D.Y_in[k]);
    }
    P.fuel = D.fuel;
    P.oxid = D.oxid;
    P.A_lat = Rev(D.A_lat);
    P.Ta = Rev(D.Ta);
    P.Q_cp = Rev(D.Q_cp);
    P.A_lat_d = D.A_lat_d;
    P.Ta_d = D.Ta_d;
    P.T_fp64 = Rev(D.T_fp64);
    P.omega_s = Rev(D.omega_s);
    P.omega_b = Rev(D.omega_b);
    P.omega_hi = Rev(D.omega_hi);
    P.alpha = Rev(D.alpha);
    P.alpha12 = Rev(D.alpha12);
    P.lam_yield = Rev(D.lam_yield);
    P.u_in = Rev(D.u_in);
    P.T_in = Rev(D.T_in);
    P.invW_in = Rev(D.invW_in);
    P.rho_in = Rev(D.rho_in);
    P.T_solid = Rev(D.T_solid);
    P.solid_isothermal = D.solid_isothermal;
    P.poiseuille = D.poiseuille;
    P.epsY = Rev(D.epsY);
    P.epsT = Rev(D.epsT);
    P.cs = Rev(D.cs);
    P.curved = 0;
    P.link_row = nullptr;
    P.link_q = nullptr;
    P.ghost_row = nullptr;
    P.gval = nullptr;
    return P;
}

size_t adjoint_node_bytes() { return 2 * sizeof(double) + 2 * sizeof(int16_t) + sizeof(double); }
size_t rev_store_bytes() { return sizeof(RevStore); }

cudaError_t launch_adjoint_step(int dim, const StepParams<double>& Pd, int planes, const void* state, bool fp32,
                                const uint8_t* solid, const double* lam_next, double* lam, double* dtheta,
                                const AdjointWork& w, cudaStream_t stream)
{
    if (dim != 2) return cudaErrorInvalidValue;
    const long long nel = (long long)planes * Pd.N;
    RevStore* rin = (RevStore*)w.rin;
    RevStore* rout = (RevStore*)w.rout;
    const unsigned nb = (unsigned)((nel + 255) / 256);
    if (fp32)
        to_rev_kernel<float><<<nb, 256, 0, stream>>>(nel, (const float*)state, rin);
    else
        to_rev_kernel<double><<<nb, 256, 0, stream>>>(nel, (const double*)state, rin);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    RevTape tp;
    tp.a0 = w.a0;
    tp.a1 = w.a1;
    tp.p0 = w.p0;
    tp.p1 = w.p1;
    tp.adj = w.adj;
    tp.in_base = rin;
    tp.maxn = w.maxn;
    tp.overflow = w.flags;
    if ((e = cudaMemcpyToSymbolAsync(rev_tape, &tp, sizeof tp, 0, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return e;
    const StepParams<Rev> P = rev_params(Pd);
    for (long long c0 = 0; c0 < Pd.ncell; c0 += w.chunk) {
        const long long n = Pd.ncell - c0 < w.chunk ? Pd.ncell - c0 : w.chunk;
        // the tape is sized for w.chunk threads: launch that many (idle ones
        // return at once) so that the interleaved layout has a fixed stride
        const unsigned blocks = (unsigned)((w.chunk + REV_BLOCK - 1) / REV_BLOCK);
        adjoint_kernel<2><<<blocks, REV_BLOCK, REV_BLOCK * sizeof(int), stream>>>(
            P, rin, rout, solid, c0, n, planes, lam_next, lam, dtheta, w.flags + 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
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
