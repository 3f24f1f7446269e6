// lbfd_tangent.cu -- the coupled step in tangent-linear (forward-mode)
// arithmetic, and the reductions of its objectives.
//
// The general-form step kernel is instantiated with Dual<double, 4> (or
// Dual<float, 4> for the mixed tangent form): every state value carries its
// derivative with respect to
//   theta = (ln A, Ta, T_wall, u_in)
// (T_wall seeds every isothermal wall face and isothermal solid).  One
// tangent step costs about five plain steps and gives the exact derivative
// of the discrete scheme; for four parameters and scalar objectives this
// needs no reverse sweep and no checkpoints.
#include "lbfd_internal.h"
#include "lbfd_step_general.cuh"

namespace lbfd {

template <int DIM, typename TT>
__global__ void __launch_bounds__(128) step_kernel_tangent(StepParams<TT> P, const TT* __restrict__ g_in,
                                                           TT* __restrict__ g_out, const TT* __restrict__ T_in,
                                                           TT* __restrict__ T_out, const TT* __restrict__ Y_in,
                                                           TT* __restrict__ Y_out,
                                                           const uint8_t* __restrict__ solid)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.ncell) return;
    if (solid[c]) return;
    int p[3];
    p[0] = (int)(c % P.nx);
    const long long r = c / P.nx;
    p[1] = (int)(r % P.ny);
    p[2] = (int)(r / P.ny);
    cell_step_general<DIM, TT, TT>(P, p, c, g_in, g_out, T_in, T_out, Y_in, Y_out, solid);
}

template <typename TT>
static cudaError_t step_tangent(int dim, const StepParams<TT>& P, StateView in, StateView out, const uint8_t* solid,
                                cudaStream_t stream)
{
    if (dim != 2) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)((P.ncell + 127) / 128);
    step_kernel_tangent<2, TT><<<blocks, 128, 0, stream>>>(P, (const TT*)in.g, (TT*)out.g, (const TT*)in.T,
                                                           (TT*)out.T, (const TT*)in.Y, (TT*)out.Y, solid);
    return cudaGetLastError();
}
cudaError_t launch_step_tangent(int dim, const StepParams<Tan>& P, StateView in, StateView out, const uint8_t* solid,
                                cudaStream_t stream)
{
    return step_tangent(dim, P, in, out, solid, stream);
}
cudaError_t launch_step_tangent(int dim, const StepParams<Tanf>& P, StateView in, StateView out, const uint8_t* solid,
                                cudaStream_t stream)
{
    return step_tangent(dim, P, in, out, solid, stream);
}

// derivative k of a raw field (T, Y_k, g_i) into double out[ncell]
template <typename TT>
__global__ void __launch_bounds__(256) tangent_field_kernel(long long ncell, long long N, const TT* __restrict__ base,
                                                            int plane, int k, double* __restrict__ out)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    out[c] = (double)base[(long long)plane * N + c].d[k];
}

cudaError_t launch_tangent_field(bool fp32, long long ncell, long long N, const void* state_base, int plane, int k,
                                 double* out, cudaStream_t stream)
{
    const unsigned blocks = (unsigned)((ncell + 255) / 256);
    if (fp32)
        tangent_field_kernel<Tanf><<<blocks, 256, 0, stream>>>(ncell, N, (const Tanf*)state_base, plane, k, out);
    else
        tangent_field_kernel<Tan><<<blocks, 256, 0, stream>>>(ncell, N, (const Tan*)state_base, plane, k, out);
    return cudaGetLastError();
}

// Objectives over fluid cells, evaluated in tangent arithmetic so that the
// parameters' own seeds (A and Ta in the rate) enter too:
//   0: sum Y_F                                (the flame position up to a constant)
//   1: sum rho (Q/cp) A dt Y_F Y_O exp(-Ta/T) (total heat release)
//   2: the same heat release, and its sum weighted by the cell's wall
//      weight wgt (the two sums of the quenching distance)
// red[0] = value, red[1 + k] = derivative k (objective 2 adds the weighted
// sum at red[5 + ...]); accumulated in FP64.
template <typename TT>
__global__ void __launch_bounds__(256) objective_kernel(StepParams<TT> P, const TT* __restrict__ T,
                                                        const TT* __restrict__ Y, const uint8_t* __restrict__ solid,
                                                        int objective, const double* __restrict__ wgt, double* red)
{
    constexpr int NV = 1 + NTAN;
    double acc[2 * NV] = {};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < P.ncell; c += stride) {
        if (solid[c]) continue;
        TT j;
        if (objective == 0) {
            j = Y[(long long)P.fuel * P.N + c];
        } else {
            TT Yc[NSP];
#pragma unroll
            for (int k = 0; k < NSP; ++k) Yc[k] = Y[(long long)k * P.N + c];
            const TT Tc = T[c];
            const TT rho = eos(P, Tc, inv_molar_mass(P, Yc));
            j = rho * P.Q_cp * arrhenius(P, Tc, pick_species(Yc, P.fuel), pick_species(Yc, P.oxid));
        }
        acc[0] += (double)j.v;
#pragma unroll
        for (int k = 0; k < NTAN; ++k) acc[1 + k] += (double)j.d[k];
        if (objective == 2) {
            const double w = wgt[c];
            acc[NV] += w * (double)j.v;
#pragma unroll
            for (int k = 0; k < NTAN; ++k) acc[NV + 1 + k] += w * (double)j.d[k];
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < 2 * NV; ++k) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], off);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < 2 * NV; ++k) atomicAdd(&red[k], acc[k]);
}

template <typename TT>
static cudaError_t objective(const StepParams<TT>& P, StateView st, const uint8_t* solid, int obj, const double* wgt,
                             double* red, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(red, 0, 2 * (1 + NTAN) * sizeof(double), stream);
    if (e != cudaSuccess) return e;
    long long want = (P.ncell + 255) / 256;
    const unsigned blocks = (unsigned)(want < 1024 ? (want > 0 ? want : 1) : 1024);
    objective_kernel<TT><<<blocks, 256, 0, stream>>>(P, (const TT*)st.T, (const TT*)st.Y, solid, obj, wgt, red);
    return cudaGetLastError();
}
cudaError_t launch_objective(const StepParams<Tan>& P, StateView st, const uint8_t* solid, int obj, const double* wgt,
                             double* red, cudaStream_t stream)
{
    return objective(P, st, solid, obj, wgt, red, stream);
}
cudaError_t launch_objective(const StepParams<Tanf>& P, StateView st, const uint8_t* solid, int obj, const double* wgt,
                             double* red, cudaStream_t stream)
{
    return objective(P, st, solid, obj, wgt, red, stream);
}

}  // namespace lbfd
