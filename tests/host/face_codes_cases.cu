// Host-side check of the 3-D code builders: for a few small geometries, the
// cells near domain faces (boundary_cells, faces only) split by face_codes
// into the coded ones (with their codes) and the rest, and the wall codes of
// the cells around one solid cell, printed one JSON object per case.  Built and run by tests/test_face_codes_host.py
// on the CPU; no GPU call is made.
#include <cstdio>
#include <vector>

#include "lbfd_internal.h"

namespace lbfd {
// lbfd_step.cu calls the 3-D tile launcher, which this check does not link
cudaError_t launch_step3d_tiled(int, int, const StepParams<double>&, const StepParams<float>&, StateView, StateView,
                                const uint8_t*, const BoundaryLists&, const SideStream&, cudaStream_t)
{
    return cudaErrorNotSupported;
}
}  // namespace lbfd

static void run(const char* name, int nx, int ny, int nz, const int* bc, const std::vector<int>& solid_xyz)
{
    std::vector<uint8_t> solid((size_t)nx * ny * nz, 0);
    for (size_t s = 0; s + 2 < solid_xyz.size(); s += 3)
        solid[(size_t)solid_xyz[s] + (size_t)nx * (solid_xyz[s + 1] + (size_t)ny * solid_xyz[s + 2])] = 1;
    std::vector<long long> face, coded, rest;
    std::vector<unsigned long long> codes;
    lbfd::boundary_cells(3, nx, ny, nz, bc, solid.data(), face, true, nullptr);
    lbfd::face_codes(nx, ny, nz, bc, solid.data(), face, coded, codes, rest);
    printf("{\"case\": \"%s\", \"nx\": %d, \"ny\": %d, \"nz\": %d, \"coded\": [", name, nx, ny, nz);
    for (size_t t = 0; t < coded.size(); ++t) printf("%s[%lld, %llu]", t ? ", " : "", coded[t], codes[t]);
    printf("], \"rest\": [");
    for (size_t t = 0; t < rest.size(); ++t) printf("%s%lld", t ? ", " : "", rest[t]);
    printf("]}\n");
}

// the neighbourhood codes of the cells next to one solid cell in a periodic
// domain (wall_codes; listed in index order)
static void run_walls(const char* name, int nx, int ny, int nz, int sx, int sy, int sz)
{
    const int bc[6] = {0, 0, 0, 0, 0, 0};
    std::vector<uint8_t> solid((size_t)nx * ny * nz, 0);
    solid[(size_t)sx + (size_t)nx * (sy + (size_t)ny * sz)] = 1;
    std::vector<long long> all, face, cells;
    lbfd::boundary_cells(3, nx, ny, nz, bc, solid.data(), all, false, nullptr);
    std::vector<unsigned long long> codes;
    lbfd::wall_codes(nx, ny, nz, bc, solid.data(), all, codes);
    printf("{\"case\": \"%s\", \"nx\": %d, \"ny\": %d, \"nz\": %d, \"coded\": [", name, nx, ny, nz);
    for (size_t t = 0; t < all.size(); ++t) printf("%s[%lld, %llu]", t ? ", " : "", all[t], codes[t]);
    printf("], \"rest\": []}\n");
}

int main()
{
    const int open_x[6] = {3, 5, 0, 0, 0, 0};        // inlet, constant-pressure outlet, periodic y and z
    const int eq32_x[6] = {3, 4, 0, 0, 0, 0};        // inlet, convective outlet (Eq. 32)
    const int walls_y[6] = {3, 5, 2, 2, 0, 0};       // and isothermal walls at the y faces
    run("open", 12, 6, 5, open_x, {});
    run("seam", 12, 6, 5, open_x, {0, 5, 0});
    run("inner_pressure", 12, 6, 5, open_x, {10, 2, 2});
    run("inner_eq32", 12, 6, 5, eq32_x, {10, 2, 2});
    run("walls_y", 12, 8, 5, walls_y, {});
    run_walls("one_solid", 9, 9, 9, 4, 4, 4);
    return 0;
}
