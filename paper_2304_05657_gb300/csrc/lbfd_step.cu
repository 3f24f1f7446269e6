// lbfd_step.cu -- the fused coupled LB/FD step kernel (sm_103a).
//
// One thread updates one cell: pull streaming, FD scalar update and cumulant
// collision are fused so that each step reads the state once and writes it
// once (populations A/B double-buffered, SoA planes, x fastest).
#include "lbfd_internal.h"
#include "lbfd_step_general.cuh"

namespace lbfd {

template <int DIM, typename S, typename R>
__global__ void __launch_bounds__(256) step_kernel_general(StepParams<R> P, const S* __restrict__ g_in,
                                                           S* __restrict__ g_out, const S* __restrict__ T_in,
                                                           S* __restrict__ T_out, const S* __restrict__ Y_in,
                                                           S* __restrict__ Y_out, const uint8_t* __restrict__ solid)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.ncell) return;
    if (solid[c]) return;
    int p[3];
    p[0] = (int)(c % P.nx);
    const long long r = c / P.nx;
    p[1] = (int)(r % P.ny);
    p[2] = (int)(r / P.ny);
    cell_step_general<DIM, S, R>(P, p, c, g_in, g_out, T_in, T_out, Y_in, Y_out, solid);
}

template <int DIM, typename S, typename R>
static cudaError_t launch_general(const StepParams<R>& P, StateView in, StateView out, const uint8_t* solid,
                                  cudaStream_t stream)
{
    const int threads = 256;
    const long long blocks = (P.ncell + threads - 1) / threads;
    step_kernel_general<DIM, S, R><<<(unsigned)blocks, threads, 0, stream>>>(
        P, (const S*)in.g, (S*)out.g, (const S*)in.T, (S*)out.T, (const S*)in.Y, (S*)out.Y, solid);
    return cudaGetLastError();
}

cudaError_t launch_step(int dim, int precision, const StepParams<double>& Pd, const StepParams<float>& Pf,
                        StateView in, StateView out, const uint8_t* solid, cudaStream_t stream)
{
    if (precision == 0) {
        if (dim == 2) return launch_general<2, double, double>(Pd, in, out, solid, stream);
        return launch_general<3, double, double>(Pd, in, out, solid, stream);
    }
    if (dim == 2) return launch_general<2, float, float>(Pf, in, out, solid, stream);
    return launch_general<3, float, float>(Pf, in, out, solid, stream);
}

}  // namespace lbfd
