// lbfd_step.cu -- launchers of the fused coupled LB/FD step (sm_103a).
//
// Variant 0 is the general form (one thread per cell, every access through
// the boundary classification; D2Q9 and D3Q27).  Variants 1.. are 2-D
// shared-memory tiles of different shapes (lbfd_step_tiled.cuh); the
// autotuner picks among them by timing.  All variants compute the same
// step; they differ only in rounding order.
#include <vector>

#include "lbfd_internal.h"
#include "lbfd_step_tiled.cuh"

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

template <typename S, typename R, int TX, int TY, bool WALLS>
static cudaError_t launch_tiled(const StepParams<R>& P, StateView in, StateView out, const uint8_t* solid,
                                const long long* bnd, long long nbnd, const SideStream& side, cudaStream_t stream)
{
    constexpr size_t smem = tile_smem_bytes<R, TX, TY>();
    auto kern = step_kernel_tiled2d<S, R, TX, TY, WALLS>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
    // the cells the tile kernel skips go to the boundary kernel: disjoint
    // writes, same input state, so it runs concurrently on the side stream
    const bool fork = nbnd > 0 && side.stream != nullptr;
    cudaError_t e = cudaSuccess;
    if (fork) {
        if ((e = cudaEventRecord(side.fork, stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side.stream, side.fork, 0)) != cudaSuccess) return e;
    }
    cudaStream_t bs = fork ? side.stream : stream;
    if (nbnd > 0) {
        const unsigned nb = (unsigned)((nbnd + 127) / 128);
        step_kernel_boundary<2, S, R><<<nb, 128, 0, bs>>>(P, (const S*)in.g, (S*)out.g, (const S*)in.T, (S*)out.T,
                                                          (const S*)in.Y, (S*)out.Y, solid, bnd, nbnd);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
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
static cudaError_t launch_2d(int variant, const StepParams<R>& P, StateView in, StateView out, const uint8_t* solid,
                             const BoundaryLists& b, const SideStream& side, cudaStream_t stream)
{
    // variants 5-8 also update cells next to in-domain solid cells in the
    // tile kernel, so their boundary list holds only cells near domain faces
    // (or every non-interior cell once curved walls are set)
    const long long* bf = b.face;
    const long long nf = b.nface;
    switch (variant) {
    case 0: return launch_general<2, S, R>(P, in, out, solid, stream);
    case 1: return launch_tiled<S, R, 32, 8, false>(P, in, out, solid, b.all, b.nall, side, stream);
    case 2: return launch_tiled<S, R, 32, 4, false>(P, in, out, solid, b.all, b.nall, side, stream);
    case 3: return launch_tiled<S, R, 64, 4, false>(P, in, out, solid, b.all, b.nall, side, stream);
    case 4: return launch_tiled<S, R, 32, 16, false>(P, in, out, solid, b.all, b.nall, side, stream);
    case 5: return launch_tiled<S, R, 32, 8, true>(P, in, out, solid, bf, nf, side, stream);
    case 6: return launch_tiled<S, R, 32, 4, true>(P, in, out, solid, bf, nf, side, stream);
    case 7: return launch_tiled<S, R, 64, 4, true>(P, in, out, solid, bf, nf, side, stream);
    case 8: return launch_tiled<S, R, 32, 16, true>(P, in, out, solid, bf, nf, side, stream);
    default: return cudaErrorInvalidValue;
    }
}

int num_variants(int dim) { return dim == 2 ? 9 : 3; }

cudaError_t launch_step(int dim, int precision, int variant, const StepParams<double>& Pd,
                        const StepParams<float>& Pf, StateView in, StateView out, const uint8_t* solid,
                        const BoundaryLists& b, const SideStream& side, cudaStream_t stream)
{
    if (variant < 0 || variant >= num_variants(dim)) return cudaErrorInvalidValue;
    if (dim == 3 && variant > 0)
        return launch_step3d_tiled(precision, variant, Pd, Pf, in, out, solid, b.all, b.nall, side, stream);
    if (precision == 0) {
        if (dim == 2) return launch_2d<double, double>(variant, Pd, in, out, solid, b, side, stream);
        return launch_general<3, double, double>(Pd, in, out, solid, stream);
    }
    if (dim == 2) return launch_2d<float, float>(variant, Pf, in, out, solid, b, side, stream);
    return launch_general<3, float, float>(Pf, in, out, solid, stream);
}

void boundary_cells(int dim, int nx, int ny, int nz, const uint8_t* solid, std::vector<long long>& out,
                    bool faces_only)
{
    out.clear();
    if (dim == 3) {
        // the 3-D tile kernel's fast-path condition: +-2 along the three axes
        // and the 26 neighbours are fluid cells inside the domain
        const long long plane = (long long)nx * ny;
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const long long c = (long long)x + (long long)nx * y + plane * z;
                    if (solid[c]) continue;
                    bool fast = x >= 2 && x < nx - 2 && y >= 2 && y < ny - 2 && z >= 2 && z < nz - 2;
                    for (int d = -2; d <= 2 && fast; ++d) {
                        if (d == 0) continue;
                        fast = !solid[c + d] && !solid[c + (long long)nx * d] && !solid[c + plane * d];
                    }
                    for (int dz = -1; dz <= 1 && fast; ++dz)
                        for (int dy = -1; dy <= 1 && fast; ++dy)
                            for (int dx = -1; dx <= 1 && fast; ++dx)
                                fast = !solid[c + dx + (long long)nx * dy + plane * dz];
                    if (!fast) out.push_back(c);
                }
        return;
    }
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const long long c = (long long)x + (long long)nx * y;
            if (solid[c]) continue;
            bool fast = true;
            // the tile kernel's fast-path condition: +-2 along both axes and
            // the 8 neighbours are fluid cells inside the domain
            for (int dy = -2; dy <= 2 && fast; ++dy)
                for (int dx = -2; dx <= 2 && fast; ++dx) {
                    const bool axis = (dx == 0 || dy == 0);
                    const bool near = (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1);
                    if (!(axis || near)) continue;
                    const int qx = x + dx, qy = y + dy;
                    if (qx < 0 || qx >= nx || qy < 0 || qy >= ny) fast = false;
                    else if (!faces_only && solid[(long long)qx + (long long)nx * qy]) fast = false;
                }
            if (!fast) out.push_back(c);
        }
    (void)nz;
}

}  // namespace lbfd
