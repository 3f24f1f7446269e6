// lbfd_step.cu -- launchers of the fused coupled LB/FD step (sm_103a).
//
// Variant 0 is the general form (one thread per cell, every access through
// the boundary classification; D2Q9 and D3Q27).  Variants 1.. are 2-D
// shared-memory tiles of different shapes, with or without the wall-tile
// kernel, one or two cells per thread (lbfd_step_tiled.cuh,
// lbfd_step_pair.cuh; 3-D: lbfd_step3d.cu); the autotuner picks among them
// by timing.  All variants compute the same step; they differ only in
// rounding order.  Also: the host-side classification of boundary cells.
#include <vector>

#include "lbfd_internal.h"
#include "lbfd_step_pair.cuh"
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

// PAIR: the interior tiles compute two cells per thread in packed FP32
// (FP32 storage only; the FP64 form keeps one cell per thread)
template <typename S, typename R, int TX, int TY, bool WALLS, bool PAIR = false, int MINB = 1>
static cudaError_t launch_tiled(const StepParams<R>& P, StateView in, StateView out, const uint8_t* solid,
                                const BoundaryLists& b, const SideStream& side, cudaStream_t stream)
{
    constexpr bool pair = PAIR && std::is_same<S, float>::value && std::is_same<R, float>::value;
    constexpr size_t smem = tile_smem_bytes<R, TX, TY>();
    auto kern = step_kernel_tiled2d<S, R, TX, TY>;
    const dim3 block(pair ? TX / 2 : TX, TY);
    constexpr size_t wsmem = tile_smem_bytes<R, WALL_TX, WALL_TY>();
    auto wkern = step_kernel_tiled2d_walls<S, R, WALL_TX, WALL_TY>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
    // the interior cells go to the tile kernel; the others, on the side
    // stream (disjoint writes, same input state), to the wall-tile kernel
    // (WALLS variants, cells next to in-domain solids) and the boundary
    // kernel (the rest)
    const bool walls = WALLS && !P.curved && b.nwall_tiles > 0;
    const long long* bl = walls ? b.face : b.all;
    const long long nb = walls ? b.nface : b.nall;
    const bool fork = (nb > 0 || walls) && side.stream != nullptr;
    cudaError_t e = cudaSuccess;
    if (fork) {
        if ((e = cudaEventRecord(side.fork, stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side.stream, side.fork, 0)) != cudaSuccess) return e;
    }
    cudaStream_t bs = fork ? side.stream : stream;
    const int prio = fork ? side.priority : 0;
    if (nb > 0) {  // the longest-latency blocks first
        const unsigned nbk = (unsigned)((nb + 127) / 128);
        e = launch_prio(step_kernel_boundary<2, S, R>, dim3(nbk), dim3(128), 0, bs, prio, P, (const S*)in.g,
                        (S*)out.g, (const S*)in.T, (S*)out.T, (const S*)in.Y, (S*)out.Y, solid, bl, nb);
        if (e != cudaSuccess) return e;
    }
    if (walls) {
        // after the boundary kernel, at the least priority: its blocks fill
        // the SMs that the tile grid leaves idle in its last wave
        e = launch_prio(wkern, dim3((unsigned)b.nwall_tiles), dim3(WALL_TX, WALL_TY), wsmem, bs,
                        fork ? side.low : 0, P,
                        (const S*)in.g, (S*)out.g, (const S*)in.T, (S*)out.T, (const S*)in.Y, (S*)out.Y, solid,
                        (const int*)b.wall_tiles);
        if (e != cudaSuccess) return e;
    }
    if constexpr (pair) {
        auto pk = step_kernel_pair2d<TX / 2, TY, MINB>;
        constexpr size_t psmem = pair_smem_bytes<TX, TY>();
        if (psmem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem)) != cudaSuccess)
            return e;
        pk<<<grid, block, psmem, stream>>>(P, (const float*)in.g, (float*)out.g, (const float*)in.T, (float*)out.T,
                                          (const float*)in.Y, (float*)out.Y, b.interior);
    } else {
        kern<<<grid, block, smem, stream>>>(P, (const S*)in.g, (S*)out.g, (const S*)in.T, (S*)out.T,
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
static cudaError_t launch_2d(int variant, const StepParams<R>& P, StateView in, StateView out, const uint8_t* solid,
                             const BoundaryLists& b, const SideStream& side, cudaStream_t stream)
{
    // variants 5-8: the same tiles, plus a wall-tile kernel for the cells
    // next to in-domain solid cells, so that only cells near domain faces
    // go through the general form
    switch (variant) {
    case 0: return launch_general<2, S, R>(P, in, out, solid, stream);
    case 1: return launch_tiled<S, R, 32, 8, false>(P, in, out, solid, b, side, stream);
    case 2: return launch_tiled<S, R, 32, 4, false>(P, in, out, solid, b, side, stream);
    case 3: return launch_tiled<S, R, 64, 4, false>(P, in, out, solid, b, side, stream);
    case 4: return launch_tiled<S, R, 32, 16, false>(P, in, out, solid, b, side, stream);
    case 5: return launch_tiled<S, R, 32, 8, true>(P, in, out, solid, b, side, stream);
    case 6: return launch_tiled<S, R, 32, 4, true>(P, in, out, solid, b, side, stream);
    case 7: return launch_tiled<S, R, 64, 4, true>(P, in, out, solid, b, side, stream);
    case 8: return launch_tiled<S, R, 32, 16, true>(P, in, out, solid, b, side, stream);
    // variants 9-12: as 5-8 with two cells per thread in packed FP32, at
    // 128 registers (9, 10) or 96 (11, 12, five 128-thread blocks per SM;
    // six blocks at 80 registers spill and are slower)
    case 9: return launch_tiled<S, R, 32, 8, true, true, 4>(P, in, out, solid, b, side, stream);
    case 10: return launch_tiled<S, R, 64, 8, true, true, 2>(P, in, out, solid, b, side, stream);
    case 11: return launch_tiled<S, R, 32, 8, true, true, 5>(P, in, out, solid, b, side, stream);
    case 12: return launch_tiled<S, R, 64, 4, true, true, 5>(P, in, out, solid, b, side, stream);
    default: return cudaErrorInvalidValue;
    }
}

int num_variants(int dim) { return dim == 2 ? 13 : 8; }

void wall_tiles(int nx, int ny, const std::vector<long long>& all, const std::vector<long long>& face,
                std::vector<int>& out)
{
    // tiles (WALL_TX x WALL_TY) holding a cell of `all` that is not in `face`
    out.clear();
    std::vector<char> in_face;
    const int gx = (nx + WALL_TX - 1) / WALL_TX, gy = (ny + WALL_TY - 1) / WALL_TY;
    std::vector<char> mark((size_t)gx * gy, 0);
    size_t j = 0;
    for (long long c : all) {  // both lists are sorted by cell index
        while (j < face.size() && face[j] < c) ++j;
        if (j < face.size() && face[j] == c) continue;
        const int x = (int)(c % nx), y = (int)(c / nx);
        mark[(size_t)(y / WALL_TY) * gx + x / WALL_TX] = 1;
    }
    for (size_t t = 0; t < mark.size(); ++t)
        if (mark[t]) out.push_back((int)t);
}

cudaError_t launch_step(int dim, int precision, int variant, const StepParams<double>& Pd,
                        const StepParams<float>& Pf, StateView in, StateView out, const uint8_t* solid,
                        const BoundaryLists& b, const SideStream& side, cudaStream_t stream)
{
    if (variant < 0 || variant >= num_variants(dim)) return cudaErrorInvalidValue;
    if (dim == 3 && variant > 0)
        return launch_step3d_tiled(precision, variant, Pd, Pf, in, out, solid, b, side, stream);
    if (precision == 0) {
        if (dim == 2) return launch_2d<double, double>(variant, Pd, in, out, solid, b, side, stream);
        return launch_general<3, double, double>(Pd, in, out, solid, stream);
    }
    if (dim == 2) return launch_2d<float, float>(variant, Pf, in, out, solid, b, side, stream);
    return launch_general<3, float, float>(Pf, in, out, solid, stream);
}

void wall_codes(int nx, int ny, int nz, const int* bc, const uint8_t* solid, const std::vector<long long>& cells,
                std::vector<unsigned long long>& out)
{
    // every neighbour within reach of a listed cell is inside the domain up
    // to periodic wrap (the list leaves out the cells near other faces)
    const int n[3] = {nx, ny, nz};
    auto at = [&](int x, int y, int z) {
        x = ((x % nx) + nx) % nx;
        y = ((y % ny) + ny) % ny;
        z = ((z % nz) + nz) % nz;
        return solid[(long long)x + (long long)nx * ((long long)y + (long long)ny * z)] != 0;
    };
    (void)bc;
    (void)n;
    out.resize(cells.size());
    for (size_t t = 0; t < cells.size(); ++t) {
        const long long c = cells[t];
        const int p[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long long)nx * ny))};
        unsigned long long code = 0;
        for (int i = 0; i < 27; ++i)  // the source x - c_i is solid: bounce-back
            if (at(p[0] - cx_of(i), p[1] - cy_of(i), p[2] - cz_of(i))) code |= 1ull << i;
        for (int a = 0; a < 3; ++a) {
            unsigned bits6 = 0;
            for (int side = -1; side <= 1; side += 2) {
                int q1[3] = {p[0], p[1], p[2]}, q2[3] = {p[0], p[1], p[2]}, qo[3] = {p[0], p[1], p[2]};
                q1[a] += side;
                q2[a] += 2 * side;
                qo[a] -= side;
                const unsigned w = at(q1[0], q1[1], q1[2]) ? 1u : (at(q2[0], q2[1], q2[2]) ? 2u : 0u);
                const unsigned opp = at(qo[0], qo[1], qo[2]) ? 1u : 0u;
                const unsigned b3 = w | (opp << 2);
                bits6 |= (side < 0 ? b3 : b3 << 3);
            }
            if (!(bits6 & 3u)) bits6 &= ~7u;          // no wall on this side: the flag is unused
            if (!((bits6 >> 3) & 3u)) bits6 &= ~56u;
            code |= (unsigned long long)bits6 << (32 + 6 * a);
        }
        out[t] = code;
    }
}

void face_codes(int nx, int ny, int nz, const int* bc, const uint8_t* solid, const std::vector<long long>& cells,
                std::vector<long long>& coded, std::vector<unsigned long long>& codes, std::vector<long long>& rest)
{
    const int n[3] = {nx, ny, nz};
    coded.clear();
    codes.clear();
    rest.clear();
    // point q: 0 fluid, 1 solid, 2 beyond a non-periodic face (periodic axes wrapped)
    auto kind = [&](int q[3], int* face) {
        *face = -1;
        for (int a = 0; a < 3; ++a) {
            if (q[a] >= 0 && q[a] < n[a]) continue;
            const int f = 2 * a + (q[a] < 0 ? 0 : 1);
            if (bc[f] != BC_PERIODIC) {
                *face = f;
                return 2;
            }
            q[a] = ((q[a] % n[a]) + n[a]) % n[a];
        }
        return solid[(long long)q[0] + (long long)nx * ((long long)q[1] + (long long)ny * q[2])] ? 1 : 0;
    };
    auto open_face = [&](int f) { return bc[f] == BC_INLET || bc[f] == BC_OUTLET || bc[f] == BC_OUTLET_PRESSURE; };
    for (const long long c : cells) {
        const int p[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long long)nx * ny))};
        bool ok = true;
        int axis = -1;  // the one axis whose faces are in reach
        for (int a = 0; a < 3 && ok; ++a)
            for (int side = -1; side <= 1; side += 2) {
                const int f = 2 * a + (side < 0 ? 0 : 1);
                const bool reach = side < 0 ? p[a] - 2 < 0 : p[a] + 2 >= n[a];
                if (!reach || bc[f] == BC_PERIODIC) continue;
                if (!open_face(f) || (axis >= 0 && axis != a)) ok = false;
                axis = a;
            }
        unsigned long long code = 0;
        for (int i = 0; i < 27 && ok; ++i) {
            const int ci[3] = {cx_of(i), cy_of(i), cz_of(i)};
            int q[3] = {p[0] - ci[0], p[1] - ci[1], p[2] - ci[2]}, f = -1;
            const int k = kind(q, &f);
            if (k == 1) code |= 1ull << i;  // bounce-back from a solid source
            if (k != 2) continue;
            // beyond a face: the general form bounces back where the boundary
            // column is solid, and takes the convective outlet's inner value
            // from the cell itself where the inner cell is solid
            // (the column: periodic axes wrapped, the others clamped)
            int qc[3] = {p[0] - ci[0], p[1] - ci[1], p[2] - ci[2]};
            for (int a = 0; a < 3; ++a) {
                if (qc[a] >= 0 && qc[a] < n[a]) continue;
                if (bc[2 * a + (qc[a] < 0 ? 0 : 1)] == BC_PERIODIC) qc[a] = ((qc[a] % n[a]) + n[a]) % n[a];
                else qc[a] = qc[a] < 0 ? 0 : n[a] - 1;
            }
            if (solid[(long long)qc[0] + (long long)nx * ((long long)qc[1] + (long long)ny * qc[2])]) ok = false;
            if (bc[f] == BC_OUTLET) {
                const int a = f / 2, ns = (f % 2 == 1) ? 1 : -1;
                int qi[3] = {p[0], p[1], p[2]};
                qi[a] -= ns;
                int fi = -1;
                if (qi[a] < 0 || qi[a] >= n[a] || kind(qi, &fi) != 0) ok = false;
            }
        }
        for (int a = 0; a < 3 && ok; ++a) {
            unsigned bits6 = 0, faces2 = 0;
            for (int side = -1; side <= 1; side += 2) {
                unsigned w = 0, face = 0;
                for (int j = 1; j <= 2 && !w; ++j) {
                    int q[3] = {p[0], p[1], p[2]}, f = -1;
                    q[a] += side * j;
                    const int k = kind(q, &f);
                    if (k != 0) {
                        w = (unsigned)j;
                        face = k == 2 ? 1u : 0u;
                    }
                }
                int qo[3] = {p[0], p[1], p[2]}, fo = -1;
                qo[a] -= side;
                const unsigned opp = w != 0 && kind(qo, &fo) != 0 ? 1u : 0u;
                const unsigned b3 = w | (opp << 2);
                bits6 |= side < 0 ? b3 : b3 << 3;
                faces2 |= face << (side < 0 ? 0 : 1);
            }
            code |= (unsigned long long)bits6 << (32 + 6 * a);
            code |= (unsigned long long)faces2 << (50 + 2 * a);
        }
        if (ok) {
            coded.push_back(c);
            codes.push_back(code);
        } else {
            rest.push_back(c);
        }
    }
}

void boundary_cells(int dim, int nx, int ny, int nz, const int* bc, const uint8_t* solid, std::vector<long long>& out,
                    bool faces_only, const int* face_solid)
{
    out.clear();
    auto wrap = [](int q, int n, bool periodic, bool* out) {
        if (q >= 0 && q < n) return q;
        if (!periodic) {
            *out = true;
            return 0;
        }
        return ((q % n) + n) % n;
    };
    const bool px = bc[0] == 0, py = bc[2] == 0, pz = bc[4] == 0;  // periodic axes
    if (dim == 3) {
        // the 3-D tile kernel's fast-path condition: +-2 along the three axes
        // and the 26 neighbours are fluid cells (periodic axes wrapped);
        // faces_only: only the cells whose stencil leaves the domain across
        // a non-periodic face
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const long long c = (long long)x + (long long)nx * ((long long)y + (long long)ny * z);
                    if (solid[c]) continue;
                    bool fast = true;
                    for (int dz = -2; dz <= 2 && fast; ++dz)
                        for (int dy = -2; dy <= 2 && fast; ++dy)
                            for (int dx = -2; dx <= 2 && fast; ++dx) {
                                const int nzero = (dx != 0) + (dy != 0) + (dz != 0);
                                const bool axis = nzero <= 1;
                                const bool near = dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1;
                                if (!(axis || near)) continue;
                                bool out = false;
                                const int qx = wrap(x + dx, nx, px, &out), qy = wrap(y + dy, ny, py, &out),
                                          qz = wrap(z + dz, nz, pz, &out);
                                if (out || (!faces_only &&
                                            solid[(long long)qx + (long long)nx * ((long long)qy + (long long)ny * qz)]))
                                    fast = false;
                            }
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
                    bool outx = false, outy = false;
                    const int qx = wrap(x + dx, nx, px, &outx), qy = wrap(y + dy, ny, py, &outy);
                    if (outx || outy) {
                        // outside: fine for the wall-aware tiles only beyond walls
                        // that act like the solid cells
                        const int rx = x + dx, ry = y + dy;
                        const bool okx = !outx || (face_solid && face_solid[rx < 0 ? 0 : 1]);
                        const bool oky = !outy || (face_solid && face_solid[ry < 0 ? 2 : 3]);
                        if (!(faces_only && okx && oky)) fast = false;
                    } else if (!faces_only && solid[(long long)qx + (long long)nx * qy]) {
                        fast = false;
                    }
                }
            if (!fast) out.push_back(c);
        }
    (void)nz;
}

}  // namespace lbfd
