// lbfd_step_tiled.cuh -- 2-D fused coupled step with shared-memory staging.
//
// A block owns a TX x TY tile of cells.  It stages T, Y_k and the derived
// point values 1/W, X_k and rho of the tile plus a 2-cell halo in shared
// memory (each derived value is computed once per point instead of once per
// stencil use).  Cells whose +-2 FD lines and LB neighbours are all fluid
// cells inside the domain take the fast path: FD stencils from shared
// memory, populations pulled straight from global memory (coalesced, one
// plane at a time).  Every other cell (walls, solids, inlet, outlet,
// periodic wrap) is left to step_kernel_boundary, which runs the general
// form of lbfd_step_general.cuh over a precomputed list of those cells.
#pragma once
#include "lbfd_step_general.cuh"

namespace lbfd {

template <typename R>
struct TileSmem {
    // layout: [field][point], point = sy * SX + sx
    R* T;
    R* Y;     // NSP planes
    R* X;     // NSP planes
    R* invW;
    R* rho;
    uint8_t* mask;  // 0 fluid, 1 solid, 2 outside the domain
};

template <int TX, int TY>
struct TileGeom {
    static constexpr int SX = TX + 4;
    static constexpr int SY = TY + 4;
    static constexpr int NPT = SX * SY;
};

template <typename R, int TX, int TY>
__host__ __device__ constexpr size_t tile_smem_bytes()
{
    return sizeof(R) * (size_t)TileGeom<TX, TY>::NPT * (3 + 2 * NSP) + (size_t)TileGeom<TX, TY>::NPT;
}

// fast-path FD terms along one axis from shared memory; `st` is the point
// stride of the axis (1 for x, SX for y) and p0 the centre point
template <typename R>
__device__ __forceinline__ void fd_axis_smem(const StepParams<R>& P, const TileSmem<R>& sm, int npt, int p0, int st,
                                             int a, R u_a, R T0, const R* Y0, R invW0, R rho0, FDAccum<R>& acc)
{
    R v[5], w[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) v[j] = sm.rho[p0 + (j - 2) * st];
    const R drho = fd_d1(v);
    acc.grad_rho[a] = drho;
    const R drho_r = fdiv(drho, rho0);
#pragma unroll
    for (int j = 0; j < 5; ++j) v[j] = sm.T[p0 + (j - 2) * st];
    acc.conv_T += u_a * weno3_deriv_fast(v, u_a, P.epsT);
    acc.diff_T += P.alpha * (fd_d2(v) + drho_r * fd_d1(v));
#pragma unroll
    for (int j = 0; j < 5; ++j) w[j] = sm.invW[p0 + (j - 2) * st];
    const R dinvW = fd_d1(w);
    R Lk[NSP], m[NSP], dm[NSP], dY[NSP];
    R sumL = R(0), M = R(0), dM = R(0);
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] = sm.Y[k * npt + p0 + (j - 2) * st];
        Lk[k] = weno3_deriv_fast(v, u_a, P.epsY);
        sumL += Lk[k];
        dY[k] = fd_d1(v);
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] = sm.X[k * npt + p0 + (j - 2) * st];
        const R dX = fd_d1(v), d2X = fd_d2(v);
        m[k] = P.a_diff[k] * invW0 * dX;
        dm[k] = P.a_diff[k] * (invW0 * d2X + dinvW * dX);
        M += m[k];
        dM += dm[k];
    }
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
        acc.conv_Y[k] += u_a * (Lk[k] - Y0[k] * sumL);
        acc.diff_Y[k] += dm[k] - dY[k] * M - Y0[k] * dM + (m[k] - Y0[k] * M) * drho_r;
    }
}

// FD terms along one axis for a cell next to in-domain solid cells (staircase
// walls), from shared memory: pts are the five line points after the mirror
// rule, `ghost` flags the points that are ghosts (bit j), whose T and rho
// take the Dirichlet form when the solid is isothermal (Y, X, 1/W mirror).
template <typename R>
__device__ __forceinline__ void fd_axis_smem_walls(const StepParams<R>& P, const TileSmem<R>& sm, int npt,
                                                   const int* pts, int ghost, int a, R u_a, const R* Y0, R invW0,
                                                   R rho0, FDAccum<R>& acc)
{
    const bool iso = P.solid_isothermal;
    const R TB = P.T_solid;
    R v[5], w[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        w[j] = sm.invW[pts[j]];
        v[j] = sm.rho[pts[j]];
        if (iso && ((ghost >> j) & 1)) v[j] = R(2) * eos(P, TB, w[j]) - v[j];
    }
    const R drho = fd_d1(v);
    acc.grad_rho[a] = drho;
    const R drho_r = fdiv(drho, rho0);
    const R dinvW = fd_d1(w);
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        v[j] = sm.T[pts[j]];
        if (iso && ((ghost >> j) & 1)) v[j] = R(2) * TB - v[j];
    }
    const bool near = ghost != 0;
    acc.conv_T += u_a * (near ? fd_c2(v) : weno3_deriv_fast(v, u_a, P.epsT));
    acc.diff_T += P.alpha * (fd_d2(v) + drho_r * fd_d1(v));
    R Lk[NSP], m[NSP], dm[NSP], dY[NSP];
    R sumL = R(0), M = R(0), dM = R(0);
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] = sm.Y[k * npt + pts[j]];
        Lk[k] = near ? fd_c2(v) : weno3_deriv_fast(v, u_a, P.epsY);
        sumL += Lk[k];
        dY[k] = fd_d1(v);
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] = sm.X[k * npt + pts[j]];
        const R dX = fd_d1(v), d2X = fd_d2(v);
        m[k] = P.a_diff[k] * invW0 * dX;
        dm[k] = P.a_diff[k] * (invW0 * d2X + dinvW * dX);
        M += m[k];
        dM += dm[k];
    }
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
        acc.conv_Y[k] += u_a * (Lk[k] - Y0[k] * sumL);
        acc.diff_Y[k] += dm[k] - dY[k] * M - Y0[k] * dM + (m[k] - Y0[k] * M) * drho_r;
    }
}

// the five points of an axis line after the mirror rule of Eq. 34 for
// in-domain solid cells (the ghost at distance j mirrors the fluid point at
// distance j-1 across the wall; the centre when that point is solid)
__device__ __forceinline__ int wall_line(const uint8_t* mask, int p0, int st, int* pts)
{
    int ghost = 0;
#pragma unroll
    for (int j = 0; j < 5; ++j) pts[j] = p0 + (j - 2) * st;
#pragma unroll
    for (int side = -1; side <= 1; side += 2) {
        const int w = mask[p0 + side * st] ? 1 : (mask[p0 + 2 * side * st] ? 2 : 0);
        if (!w) continue;
#pragma unroll
        for (int j = 1; j <= 2; ++j) {
            if (j < w) continue;
            const int m = 2 * w - 1 - j;
            int mp;
            if (m >= 0) mp = p0 + side * m * st;
            else mp = mask[p0 - side * st] ? p0 : p0 - side * st;
            pts[2 + side * j] = mp;
            ghost |= 1 << (2 + side * j);
        }
    }
    return ghost;
}

// body of the 2-D tile kernels.  WALLS == false: the interior cells of
// every tile.  WALLS == true: only the cells next to in-domain solid cells
// (or walls that act like them), in the tiles listed in `tiles`.
template <typename S, typename R, int TX, int TY, bool WALLS>
__device__ __forceinline__ void tiled2d_body(const StepParams<R>& P, const S* __restrict__ g_in, S* __restrict__ g_out,
                                             const S* __restrict__ T_in, S* __restrict__ T_out,
                                             const S* __restrict__ Y_in, S* __restrict__ Y_out,
                                             const uint8_t* __restrict__ solid, const int* __restrict__ tiles)
{
    using G = TileGeom<TX, TY>;
    constexpr int SX = G::SX, NPT = G::NPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<R> sm;
    sm.T = reinterpret_cast<R*>(smem_raw);
    sm.Y = sm.T + NPT;
    sm.X = sm.Y + NSP * NPT;
    sm.invW = sm.X + NSP * NPT;
    sm.rho = sm.invW + NPT;
    sm.mask = reinterpret_cast<uint8_t*>(sm.rho + NPT);

    int bx = blockIdx.x, by = blockIdx.y;
    if constexpr (WALLS) {
        const int t = tiles[blockIdx.x];
        const int gxn = (P.nx + TX - 1) / TX;
        bx = t % gxn;
        by = t / gxn;
    }
    const int x0 = bx * TX, y0 = by * TY;
    const int tid = threadIdx.x + TX * threadIdx.y;
    const long long N = P.N;
    // stage the tile and its halo (points outside the domain are marked 2
    // and never read by a fast-path cell)
    for (int pt = tid; pt < NPT; pt += TX * TY) {
        const int sx = pt % SX, sy = pt / SX;
        int gx = x0 + sx - 2, gy = y0 + sy - 2;
        // across a periodic face the halo holds the wrapped cells
        // (at most two periods away: the halo is two cells wide)
        if (P.bc[0] == BC_PERIODIC) {
            if (gx < 0) gx += P.nx;
            if (gx < 0) gx += P.nx;
            if (gx >= P.nx) gx -= P.nx;
            if (gx >= P.nx) gx -= P.nx;
        }
        if (P.bc[2] == BC_PERIODIC) {
            if (gy < 0) gy += P.ny;
            if (gy < 0) gy += P.ny;
            if (gy >= P.ny) gy -= P.ny;
            if (gy >= P.ny) gy -= P.ny;
        }
        if (gx < 0 || gx >= P.nx || gy < 0 || gy >= P.ny) {
            uint8_t m = 2;
            if constexpr (WALLS) {  // beyond walls that act like the solid cells
                const bool okx = gx >= 0 && gx < P.nx ? true : P.face_solid[gx < 0 ? 0 : 1];
                const bool oky = gy >= 0 && gy < P.ny ? true : P.face_solid[gy < 0 ? 2 : 3];
                if (okx && oky) m = 1;
            }
            sm.mask[pt] = m;
            continue;
        }
        const long long c = (long long)gx + (long long)P.nx * gy;
        const uint8_t s = solid[c];
        sm.mask[pt] = s ? 1 : 0;
        if (s) continue;
        const R T = R(T_in[c]);
        R Y[NSP];
#pragma unroll
        for (int k = 0; k < NSP; ++k) Y[k] = R(Y_in[(long long)k * N + c]);
        const R invW = inv_molar_mass(P, Y);
        const R W = fdiv(R(1), invW);
        sm.T[pt] = T;
#pragma unroll
        for (int k = 0; k < NSP; ++k) {
            sm.Y[k * NPT + pt] = Y[k];
            sm.X[k * NPT + pt] = Y[k] * P.inv_Wk[k] * W;
        }
        sm.invW[pt] = invW;
        sm.rho[pt] = fdiv(P.T_in * P.invW_in * W, T);
    }
    __syncthreads();

    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const int p0 = (threadIdx.y + 2) * SX + threadIdx.x + 2;
    if (sm.mask[p0]) return;  // solid
    const long long c = (long long)x + (long long)P.nx * y;
    // fast path: the +-2 lines and the 8 neighbours are fluid cells of the domain
    bool fast = true;
#pragma unroll
    for (int j = 1; j <= 2; ++j)
        fast = fast && !sm.mask[p0 + j] && !sm.mask[p0 - j] && !sm.mask[p0 + j * SX] && !sm.mask[p0 - j * SX];
    fast = fast && !sm.mask[p0 + SX + 1] && !sm.mask[p0 + SX - 1] && !sm.mask[p0 - SX + 1] && !sm.mask[p0 - SX - 1];
    if constexpr (WALLS) {
        // next to in-domain solid cells only (staircase walls); the interior
        // cells belong to the plain tile kernel, the rest to the boundary list
        if (fast || P.curved) return;
        bool walls = true;
#pragma unroll
        for (int j = 1; j <= 2; ++j)
            walls = walls && sm.mask[p0 + j] != 2 && sm.mask[p0 - j] != 2 && sm.mask[p0 + j * SX] != 2 &&
                    sm.mask[p0 - j * SX] != 2;
        walls = walls && sm.mask[p0 + SX + 1] != 2 && sm.mask[p0 + SX - 1] != 2 && sm.mask[p0 - SX + 1] != 2 &&
                sm.mask[p0 - SX - 1] != 2;
        if (!walls) return;
    } else {
        if (!fast) return;  // boundary cell: another kernel updates it
    }
    // a1: pull from the neighbours (Eq. 8), half-way bounce-back from an
    // in-domain solid neighbour (Eq. 28) in the wall-aware variants
    R g[9];
    {
        // offsets of the x-1, x+1, y-1, y+1 neighbours, wrapped on periodic axes
        const int oxm = x == 0 ? P.nx - 1 : -1, oxp = x == P.nx - 1 ? 1 - P.nx : 1;
        const int oym = y == 0 ? (P.ny - 1) * P.nx : -P.nx, oyp = y == P.ny - 1 ? (1 - P.ny) * P.nx : P.nx;
        const S* gc = g_in + c;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ox = cx_of(i) > 0 ? oxm : (cx_of(i) < 0 ? oxp : 0);
            const int oy = cy_of(i) > 0 ? oym : (cy_of(i) < 0 ? oyp : 0);
            long long off = (long long)i * N + (ox + oy);
            if constexpr (WALLS) {
                if (sm.mask[p0 - cx_of(i) - cy_of(i) * SX]) off = (long long)opposite<2>(i) * N;
            }
            g[i] = R(__ldg(gc + off));
        }
    }
    // a2
    const R T0 = sm.T[p0], invW0 = sm.invW[p0], rho0 = sm.rho[p0];
    R Y0[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) Y0[k] = sm.Y[k * NPT + p0];
    R u[3];
    {
        const R inv = fdiv(R(3), rho0);
        u[0] = ((g[2] + g[5] + g[8]) - (g[0] + g[3] + g[6])) * inv;
        u[1] = ((g[6] + g[7] + g[8]) - (g[0] + g[1] + g[2])) * inv;
        u[2] = R(0);
    }
    // a3-a5
    FDAccum<R> acc;
    acc.conv_T = acc.diff_T = R(0);
#pragma unroll
    for (int k = 0; k < NSP; ++k) acc.conv_Y[k] = acc.diff_Y[k] = R(0);
    acc.grad_rho[2] = R(0);
    if constexpr (WALLS) {
        int pts[5];
        int gh = wall_line(sm.mask, p0, 1, pts);
        fd_axis_smem_walls<R>(P, sm, NPT, pts, gh, 0, u[0], Y0, invW0, rho0, acc);
        gh = wall_line(sm.mask, p0, SX, pts);
        fd_axis_smem_walls<R>(P, sm, NPT, pts, gh, 1, u[1], Y0, invW0, rho0, acc);
    } else {
        fd_axis_smem<R>(P, sm, NPT, p0, 1, 0, u[0], T0, Y0, invW0, rho0, acc);
        fd_axis_smem<R>(P, sm, NPT, p0, SX, 1, u[1], T0, Y0, invW0, rho0, acc);
    }
    // a6
    const R q = arrhenius(P, T0, Y0[P.fuel], Y0[P.oxid]);
    const R reac_T = P.Q_cp * q;
    // a7
    const R DT = acc.diff_T + reac_T;
    T_out[c] = S(T0 + (DT - acc.conv_T));
    R lam_Y = R(0);
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
        const R DY = acc.diff_Y[k] + P.yield[k] * q;
        Y_out[(long long)k * N + c] = S(Y0[k] + (DY - acc.conv_Y[k]));
        lam_Y += P.inv_Wk[k] * DY;
    }
    const R Lam = fdiv(DT, T0) + fdiv(lam_Y, invW0);
    // a8-a10
    collide<2, R>(P, g, rho0, u, acc.grad_rho, Lam);
#pragma unroll
    for (int i = 0; i < 9; ++i) g_out[(long long)i * N + c] = S(g[i]);
}

// FP32: four 256-thread blocks (1024 threads) per SM, i.e. <= 64 registers
template <typename S, typename R, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, sizeof(R) == 4 ? 1024 / (TX * TY) : 1) step_kernel_tiled2d(StepParams<R> P, const S* __restrict__ g_in,
                                                               S* __restrict__ g_out, const S* __restrict__ T_in,
                                                               S* __restrict__ T_out, const S* __restrict__ Y_in,
                                                               S* __restrict__ Y_out,
                                                               const uint8_t* __restrict__ solid)
{
    tiled2d_body<S, R, TX, TY, false>(P, g_in, g_out, T_in, T_out, Y_in, Y_out, solid, nullptr);
}

// the cells next to in-domain solid cells, over the tiles that contain any
template <typename S, typename R, int TX, int TY>
__global__ void __launch_bounds__(TX * TY)
    step_kernel_tiled2d_walls(StepParams<R> P, const S* __restrict__ g_in, S* __restrict__ g_out,
                              const S* __restrict__ T_in, S* __restrict__ T_out, const S* __restrict__ Y_in,
                              S* __restrict__ Y_out, const uint8_t* __restrict__ solid, const int* __restrict__ tiles)
{
    tiled2d_body<S, R, TX, TY, true>(P, g_in, g_out, T_in, T_out, Y_in, Y_out, solid, tiles);
}

// The cells the tiled kernel leaves out: general form over a cell list.
template <int DIM, typename S, typename R>
__global__ void __launch_bounds__(128) step_kernel_boundary(StepParams<R> P, const S* __restrict__ g_in,
                                                            S* __restrict__ g_out, const S* __restrict__ T_in,
                                                            S* __restrict__ T_out, const S* __restrict__ Y_in,
                                                            S* __restrict__ Y_out, const uint8_t* __restrict__ solid,
                                                            const long long* __restrict__ cells, long long ncells)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncells) return;
    const long long c = cells[t];
    int p[3];
    p[0] = (int)(c % P.nx);
    const long long r = c / P.nx;
    p[1] = (int)(r % P.ny);
    p[2] = (int)(r / P.ny);
    cell_step_general<DIM, S, R>(P, p, c, g_in, g_out, T_in, T_out, Y_in, Y_out, solid);
}

}  // namespace lbfd
