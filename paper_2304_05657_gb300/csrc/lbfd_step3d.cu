// lbfd_step3d.cu -- launchers of the 3-D (D3Q27) tile kernels.
#include "lbfd_internal.h"
#include "lbfd_step_tiled3d.cuh"

namespace lbfd {

template <typename S, typename R, int TX, int TY, int ZC>
static cudaError_t launch_t3(const StepParams<R>& P, StateView in, StateView out, const uint8_t* solid,
                             const long long* bnd, long long nbnd, const SideStream& side, cudaStream_t stream)
{
    constexpr size_t smem = tile3_smem_bytes<R, TX, TY>();
    auto kern = step_kernel_tiled3d<S, R, TX, TY, ZC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const bool fork = nbnd > 0 && side.stream != nullptr;
    if (fork) {
        if ((e = cudaEventRecord(side.fork, stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side.stream, side.fork, 0)) != cudaSuccess) return e;
    }
    if (nbnd > 0) {
        const unsigned nb = (unsigned)((nbnd + 127) / 128);
        e = launch_prio(step_kernel_boundary<3, S, R>, dim3(nb), dim3(128), 0, fork ? side.stream : stream,
                        fork ? side.priority : 0, P, (const S*)in.g, (S*)out.g, (const S*)in.T, (S*)out.T,
                        (const S*)in.Y, (S*)out.Y, solid, bnd, nbnd);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY, (P.nz + ZC - 1) / ZC);
    kern<<<grid, dim3(TX, TY), smem, stream>>>(P, (const S*)in.g, (S*)out.g, (const S*)in.T, (S*)out.T,
                                               (const S*)in.Y, (S*)out.Y, solid);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (fork) {
        if ((e = cudaEventRecord(side.join, side.stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(stream, side.join, 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename S, typename R>
static cudaError_t launch_3d_tiles(int variant, const StepParams<R>& P, StateView in, StateView out,
                                   const uint8_t* solid, const long long* bnd, long long nbnd, const SideStream& side,
                                   cudaStream_t stream)
{
    switch (variant) {
    case 1: return launch_t3<S, R, 32, 4, 16>(P, in, out, solid, bnd, nbnd, side, stream);
    case 2: return launch_t3<S, R, 32, 4, 32>(P, in, out, solid, bnd, nbnd, side, stream);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step3d_tiled(int precision, int variant, const StepParams<double>& Pd, const StepParams<float>& Pf,
                                StateView in, StateView out, const uint8_t* solid, const long long* bnd,
                                long long nbnd, const SideStream& side, cudaStream_t stream)
{
    if (precision == 0) return launch_3d_tiles<double, double>(variant, Pd, in, out, solid, bnd, nbnd, side, stream);
    return launch_3d_tiles<float, float>(variant, Pf, in, out, solid, bnd, nbnd, side, stream);
}

}  // namespace lbfd
