// lbfd_step3d.cu -- launchers of the 3-D (D3Q27) tile kernels.
#include "lbfd_internal.h"
#include "lbfd_step_tiled3d.cuh"

namespace lbfd {

// The interior cells go to the tile kernel; on the side stream (same input
// state, disjoint writes) the cells near inlet and outlet faces go through
// their coded neighbourhoods (b.face_coded) and the general form takes the
// other cells near domain faces (b.face), and the cells next to in-domain
// solids (b.wall) go through their coded neighbourhoods (or, with curved
// walls, the general form with the face rules compiled out).
// the tile kernel instance: MINB > 0 caps its registers for MINB blocks per SM
template <typename S, typename R, int TX, int TY, int ZC, int MINB, bool HI1 = false>
static auto tile3_kernel()
{
    if constexpr (MINB > 0) return step_kernel_tiled3d_capped<S, R, TX, TY, ZC, MINB, HI1>;
    else return step_kernel_tiled3d<S, R, TX, TY, ZC, HI1>;
}

// SPLIT: the tile kernel does a1-a7 and a per-cell kernel a8-a10 (two
// smaller kernels instead of one; Lambda and grad rho pass through aux)
// WALLS: the wall-aware tile kernel also updates the cells next to
// in-domain solids, so the wall list runs only with curved walls
template <typename S, typename R, int TX, int TY, int ZC, int MINB = 0, bool SPLIT = false, bool WALLS = false>
static cudaError_t launch_t3(const StepParams<R>& P, StateView in, StateView out, const uint8_t* solid,
                             const BoundaryLists& bin, const SideStream& side, cudaStream_t stream)
{
    constexpr size_t smem = tile3_smem_bytes<R, TX, TY>();
    // FP32 with omega_hi = 1 (the usual setting): the tile and coded kernels
    // that skip the pre-collision cumulants of order >= 3
    constexpr bool F32 = sizeof(R) == 4;
    const bool hi1 = F32 && P.omega_hi == R(1);
    auto kern = hi1 ? tile3_kernel<S, R, TX, TY, ZC, MINB, F32>() : tile3_kernel<S, R, TX, TY, ZC, MINB>();
    auto fkern = step_kernel_fd3d<S, R, TX, TY, ZC>;
    auto wkern = step_kernel_tiled3d_walls<S, R, TX, TY, ZC>;
    auto fcode = hi1 ? step_kernel_wallcode<3, S, R, true, F32> : step_kernel_wallcode<3, S, R, true>;
    auto wcode = hi1 ? step_kernel_wallcode<3, S, R, false, F32> : step_kernel_wallcode<3, S, R, false>;
    cudaError_t e = SPLIT   ? cudaFuncSetAttribute(fkern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                    : WALLS ? cudaFuncSetAttribute(wkern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                            : cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (bin.interior == nullptr || (SPLIT && bin.aux == nullptr)) return cudaErrorInvalidValue;
    BoundaryLists b = bin;
    if (WALLS && !P.curved) b.nwall = 0;
    const bool fork = (b.nface > 0 || b.nface_coded > 0 || b.nwall > 0) && side.stream != nullptr;
    if (fork) {
        if ((e = cudaEventRecord(side.fork, stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side.stream, side.fork, 0)) != cudaSuccess) return e;
    }
    cudaStream_t bs = fork ? side.stream : stream;
    const int prio = fork ? side.priority : 0;
    if (b.nface > 0) {
        const unsigned nb = (unsigned)((b.nface + 127) / 128);
        e = launch_prio(step_kernel_boundary<3, S, R, true>, dim3(nb), dim3(128), 0, bs, prio, P, (const S*)in.g,
                        (S*)out.g, (const S*)in.T, (S*)out.T, (const S*)in.Y, (S*)out.Y, solid, b.face, b.nface);
        if (e != cudaSuccess) return e;
    }
    if (b.nface_coded > 0) {  // cells near inlet/outlet faces with their codes
        const unsigned nb = (unsigned)((b.nface_coded + 127) / 128);
        e = launch_prio(fcode, dim3(nb), dim3(128), 0, bs, prio, P, (const S*)in.g,
                        (S*)out.g, (const S*)in.T, (S*)out.T, (const S*)in.Y, (S*)out.Y, b.face_coded, b.face_code,
                        b.nface_coded);
        if (e != cudaSuccess) return e;
    }
    if (b.nwall > 0) {
        const unsigned nb = (unsigned)((b.nwall + 127) / 128);
        if (!P.curved && b.wall_code != nullptr)  // staircase walls: the coded neighbourhoods
            e = launch_prio(wcode, dim3(nb), dim3(128), 0, bs, prio, P, (const S*)in.g,
                            (S*)out.g, (const S*)in.T, (S*)out.T, (const S*)in.Y, (S*)out.Y, b.wall, b.wall_code,
                            b.nwall);
        else
            e = launch_prio(step_kernel_boundary<3, S, R, false>, dim3(nb), dim3(128), 0, bs, prio, P,
                            (const S*)in.g, (S*)out.g, (const S*)in.T, (S*)out.T, (const S*)in.Y, (S*)out.Y, solid,
                            b.wall, b.nwall);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY, (P.nz + ZC - 1) / ZC);
    if constexpr (SPLIT) {
        fkern<<<grid, dim3(TX, TY), smem, stream>>>(P, (const S*)in.g, (const S*)in.T, (S*)out.T, (const S*)in.Y,
                                                    (S*)out.Y, b.interior, (R*)b.aux);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        step_kernel_collide3d<S, R><<<dim3((P.nx + 127) / 128, P.ny, P.nz), 128, 0, stream>>>(
            P, (const S*)in.g, (S*)out.g, (const S*)in.T, (const S*)in.Y, b.interior, (const R*)b.aux);
    } else if constexpr (WALLS) {
        wkern<<<grid, dim3(TX, TY), smem, stream>>>(P, (const S*)in.g, (S*)out.g, (const S*)in.T, (S*)out.T,
                                                    (const S*)in.Y, (S*)out.Y, b.interior, solid);
    } else {
        kern<<<grid, dim3(TX, TY), smem, stream>>>(P, (const S*)in.g, (S*)out.g, (const S*)in.T, (S*)out.T,
                                                   (const S*)in.Y, (S*)out.Y, b.interior);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (fork) {
        if ((e = cudaEventRecord(side.join, side.stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(stream, side.join, 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename S, typename R>
static cudaError_t launch_3d_tiles(int variant, const StepParams<R>& P, StateView in, StateView out,
                                   const uint8_t* solid, const BoundaryLists& b, const SideStream& side,
                                   cudaStream_t stream)
{
    switch (variant) {
    case 1: return launch_t3<S, R, 32, 4, 16>(P, in, out, solid, b, side, stream);
    case 2: return launch_t3<S, R, 32, 4, 32>(P, in, out, solid, b, side, stream);
    // variant 3: as 1 with the registers capped for four blocks per SM (FP32)
    case 3: return launch_t3<S, R, 32, 4, 16, sizeof(R) == 4 ? 4 : 0>(P, in, out, solid, b, side, stream);
    // variants 4, 5: as 1, 2 split into an FD tile kernel and a collision kernel
    case 4: return launch_t3<S, R, 32, 4, 16, 0, true>(P, in, out, solid, b, side, stream);
    case 5: return launch_t3<S, R, 32, 4, 32, 0, true>(P, in, out, solid, b, side, stream);
    // variants 6, 7: as 1, 2 with the cells next to in-domain solids in the
    // tile kernel (wall-aware), no wall list
    case 6: return launch_t3<S, R, 32, 4, 16, 0, false, true>(P, in, out, solid, b, side, stream);
    case 7: return launch_t3<S, R, 32, 4, 32, 0, false, true>(P, in, out, solid, b, side, stream);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step3d_tiled(int precision, int variant, const StepParams<double>& Pd, const StepParams<float>& Pf,
                                StateView in, StateView out, const uint8_t* solid, const BoundaryLists& b,
                                const SideStream& side, cudaStream_t stream)
{
    if (precision == 0) return launch_3d_tiles<double, double>(variant, Pd, in, out, solid, b, side, stream);
    return launch_3d_tiles<float, float>(variant, Pf, in, out, solid, b, side, stream);
}

}  // namespace lbfd
