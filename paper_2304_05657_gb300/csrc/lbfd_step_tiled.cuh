// lbfd_step_tiled.cuh -- 2-D fused coupled step with shared-memory staging.
//
// A block owns a TX x TY tile of cells.  It stages T, Y_k and the derived
// point values 1/W, X_k and rho of the tile plus a 2-cell halo in shared
// memory (each derived value is computed once per point instead of once per
// stencil use; across periodic faces the halo holds the wrapped cells).
// Interior cells (+-2 FD lines and the 8 LB neighbours are fluid cells of
// the domain; a per-cell flag computed at create) take the fast path: FD
// stencils from shared memory, populations pulled straight from global
// memory (coalesced, one plane at a time).  The wall-tile kernel updates
// the cells next to in-domain solid cells over the listed tiles, from the
// same staging plus the mask; step_kernel_boundary runs the general form
// of lbfd_step_general.cuh over the list of the remaining cells (near
// inlet, outlet and wall faces).
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

// FD sums of the tile kernels: T's convective and non-convective parts,
// and for the species the net rate rhs_Y = sum over axes of (diffusion -
// convection) plus lamY = sum_k (diffusion of Y_k) / W_k, the FD part of
// Lambda's species sum (Eq. 6), which is all that Lambda needs of them
template <typename R>
struct TileAccum {
    R conv_T, diff_T;
    R rhs_Y[NSP];
    R lamY;
    R grad_rho[3];
    __device__ __forceinline__ void clear()
    {
        conv_T = diff_T = lamY = R(0);
#pragma unroll
        for (int k = 0; k < NSP; ++k) rhs_Y[k] = R(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) grad_rho[a] = R(0);
    }
};

// FD terms along one axis of an interior cell (Eq. 25-27): `line(f, v)`
// gathers the five points of the staged field f along the axis into v.
// R is the compute type (float, double, or F2 for a pair of cells), PR the
// parameters' type.
template <typename R, typename PR, typename SR, typename Line>
__device__ __forceinline__ void fd_axis_core(const StepParams<PR>& P, const TileSmem<SR>& sm, int npt, Line line,
                                             int a, R u_a, const R* Y0, R invW0, R rho0, TileAccum<R>& acc)
{
    R v[5], w[5];
    line(sm.rho, v);
    const R drho = fd_d1(v);
    acc.grad_rho[a] = drho;
    const R drho_r = fdiv(drho, rho0);
    line(sm.T, v);
    acc.conv_T += u_a * weno3_deriv_fast(v, u_a, R(P.epsT));
    acc.diff_T += R(P.alpha12) * (fd_D2(v) + drho_r * fd_D1(v));  // 12x stencils, alpha / 12
    line(sm.invW, w);
    const R dinvW = fd_d1(w);
    // diffusion fluxes from the staged Y_k W lines first (X_k = Y_k W / W_k;
    // 1/W_k and 1/12 are folded into a12): their sums M, dM enter every
    // species' correction term
    R m[NSP], dm[NSP];
    R M = R(0), dM = R(0);
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
        line(sm.X + k * npt, v);
        const R dX = fd_D1(v), d2X = fd_D2(v);
        const R ak = R(P.a12[k]);
        m[k] = ak * invW0 * dX;
        dm[k] = ak * (invW0 * d2X + dinvW * dX);
        M += m[k];
        dM += dm[k];
    }
    // then the Y_k lines; the convective correction -Y_k u_a sum_j L_j is
    // added once the sum is known
    R sumL = R(0);
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
        line(sm.Y + k * npt, v);
        const R Lk = weno3_deriv_fast(v, u_a, R(P.epsY));
        sumL += Lk;
        const R dY = fd_d1(v);
        const R dk = dm[k] - dY * M - Y0[k] * dM + (m[k] - Y0[k] * M) * drho_r;
        acc.rhs_Y[k] += dk - u_a * Lk;
        acc.lamY += R(P.inv_Wk[k]) * dk;
    }
    const R us = u_a * sumL;
#pragma unroll
    for (int k = 0; k < NSP; ++k) acc.rhs_Y[k] += Y0[k] * us;
}

// fast-path FD terms along one axis from shared memory; `st` is the point
// stride of the axis (1 for x, SX for y) and p0 the centre point
template <typename R>
__device__ __forceinline__ void fd_axis_smem(const StepParams<R>& P, const TileSmem<R>& sm, int npt, int p0, int st,
                                             int a, R u_a, R T0, const R* Y0, R invW0, R rho0, TileAccum<R>& acc)
{
    auto line = [&](const R* f, R* v) {
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] = f[p0 + (j - 2) * st];
    };
    fd_axis_core<R>(P, sm, npt, line, a, u_a, Y0, invW0, rho0, acc);
}

// FD terms along one axis for a cell next to in-domain solid cells (staircase
// walls), from shared memory: pts are the five line points after the mirror
// rule, `ghost` flags the points that are ghosts (bit j), whose T and rho
// take the Dirichlet form when the solid is isothermal (Y, X, 1/W mirror).
template <typename R>
__device__ __forceinline__ void fd_axis_smem_walls(const StepParams<R>& P, const TileSmem<R>& sm, int npt,
                                                   const int* pts, int ghost, int a, R u_a, const R* Y0, R invW0,
                                                   R rho0, TileAccum<R>& acc)
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
        for (int j = 0; j < 5; ++j) v[j] = sm.X[k * npt + pts[j]];  // Y_k W
        const R dX = fd_D1(v), d2X = fd_D2(v);
        m[k] = P.a12[k] * invW0 * dX;
        dm[k] = P.a12[k] * (invW0 * d2X + dinvW * dX);
        M += m[k];
        dM += dm[k];
    }
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
        const R dk = dm[k] - dY[k] * M - Y0[k] * dM + (m[k] - Y0[k] * M) * drho_r;
        acc.rhs_Y[k] += dk - u_a * (Lk[k] - Y0[k] * sumL);
        acc.lamY += P.inv_Wk[k] * dk;
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

// a1 (Eq. 8) for a cell whose 8 neighbours are fluid cells of the domain:
// plain pull, the x-1, x+1, y-1, y+1 neighbours wrapped on periodic axes
// (the offsets stay inside the domain for any in-range cell)
template <typename S, typename R>
__device__ __forceinline__ void pull_interior(const StepParams<R>& P, const S* LBFD_RESTRICT g_in, long long c, int x,
                                              int y, R* g)
{
    const int oxm = x == 0 ? P.nx - 1 : -1, oxp = x == P.nx - 1 ? 1 - P.nx : 1;
    const int oym = y == 0 ? (P.ny - 1) * P.nx : -P.nx, oyp = y == P.ny - 1 ? (1 - P.ny) * P.nx : P.nx;
    const S* gc = g_in + c;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ox = cx_of(i) > 0 ? oxm : (cx_of(i) < 0 ? oxp : 0);
        const int oy = cy_of(i) > 0 ? oym : (cy_of(i) < 0 ? oyp : 0);
        g[i] = R(LBFD_LDG(gc + (long long)i * P.N + (ox + oy)));
    }
}

// Stage T, Y_k, X_k, 1/W, rho and the mask of a tile (origin x0, y0) and
// its 2-cell halo with NTHR threads, this one numbered tid.  All of a
// thread's global loads are issued before any of them is used, so that
// their latencies overlap.  WALLS == false (interior tiles, whose cells are
// flagged interior from a per-cell array): no mask; solid points are staged
// like fluid ones, their values are never read.
template <typename S, typename R, int TX, int TY, bool WALLS, int NTHR>
__device__ __forceinline__ void stage_tile2d(const StepParams<R>& P, const TileSmem<R>& sm, int x0, int y0, int tid,
                                             const S* LBFD_RESTRICT T_in, const S* LBFD_RESTRICT Y_in,
                                             const uint8_t* LBFD_RESTRICT solid)
{
    using G = TileGeom<TX, TY>;
    constexpr int SX = G::SX, NPT = G::NPT;
    constexpr int NIT = (NPT + NTHR - 1) / NTHR;
    const long long N = P.N;
    long long cell[NIT];  // -1: outside the domain
    uint8_t s[NIT];
    R T[NIT], Y[NIT][NSP];
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        const int pt = tid + it * NTHR;
        cell[it] = -1;
        if (pt >= NPT) continue;
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
            // outside the domain: marked 2 and never read by a fast-path cell
            uint8_t m = 2;
            if constexpr (WALLS) {  // beyond walls that act like the solid cells
                const bool okx = gx >= 0 && gx < P.nx ? true : P.face_solid[gx < 0 ? 0 : 1];
                const bool oky = gy >= 0 && gy < P.ny ? true : P.face_solid[gy < 0 ? 2 : 3];
                if (okx && oky) m = 1;
                sm.mask[pt] = m;
            }
            continue;
        }
        const long long c = (long long)gx + (long long)P.nx * gy;
        cell[it] = c;
        if constexpr (WALLS) s[it] = solid[c];
        T[it] = R(T_in[c]);
#pragma unroll
        for (int k = 0; k < NSP; ++k) Y[it][k] = R(Y_in[(long long)k * N + c]);
    }
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        if (cell[it] < 0) continue;
        const int pt = tid + it * NTHR;
        if constexpr (WALLS) {
            sm.mask[pt] = s[it] ? 1 : 0;
            if (s[it]) continue;
        }
        const R invW = inv_molar_mass(P, Y[it]);
        const R W = fdiv(R(1), invW);
        sm.T[pt] = T[it];
#pragma unroll
        for (int k = 0; k < NSP; ++k) {
            sm.Y[k * NPT + pt] = Y[it][k];
            sm.X[k * NPT + pt] = Y[it][k] * W;  // X_k W_k (1/W_k folded into a12)
        }
        sm.invW[pt] = invW;
        sm.rho[pt] = fdiv(P.T_in * P.invW_in * W, T[it]);
    }
}

// the +-2 FD lines and the 8 LB neighbours of point p0 are fluid cells of the domain
template <int SX>
__device__ __forceinline__ bool interior_point(const uint8_t* mask, int p0)
{
    bool fast = !mask[p0];
#pragma unroll
    for (int j = 1; j <= 2; ++j)
        fast = fast && !mask[p0 + j] && !mask[p0 - j] && !mask[p0 + j * SX] && !mask[p0 - j * SX];
    return fast && !mask[p0 + SX + 1] && !mask[p0 + SX - 1] && !mask[p0 - SX + 1] && !mask[p0 - SX - 1];
}

// body of the 2-D tile kernels: the tile (bx, by), this thread at (tx, ty)
// of its TX x TY threads.  WALLS == false: the interior cells of the tile.
// WALLS == true: only the cells next to in-domain solid cells (or walls that
// act like them).  Every thread of the block calls it (it synchronises the
// block once, after the staging).
template <typename S, typename R, int TX, int TY, bool WALLS>
__device__ __forceinline__ void tiled2d_body(const StepParams<R>& P, const S* LBFD_RESTRICT g_in, S* LBFD_RESTRICT g_out,
                                             const S* LBFD_RESTRICT T_in, S* LBFD_RESTRICT T_out,
                                             const S* LBFD_RESTRICT Y_in, S* LBFD_RESTRICT Y_out,
                                             const uint8_t* LBFD_RESTRICT solid,
                                             const uint8_t* LBFD_RESTRICT interior, int tx, int ty, int bx, int by)
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

    const int x0 = bx * TX, y0 = by * TY;
    const int tid = tx + TX * ty;
    const long long N = P.N;
    const int x = x0 + tx, y = y0 + ty;
    const bool inside = x < P.nx && y < P.ny;
    const long long c = (long long)x + (long long)P.nx * y;
    R g[9];
    // interior tiles: the cell's class (the +-2 lines and the 8 neighbours
    // are fluid cells of the domain, precomputed per cell) and a1, issued
    // before the staging so that the loads are in flight while the tile is
    // staged
    bool fast = false;
    if constexpr (!WALLS) {
        if (inside) {
            fast = interior[c] != 0;
            pull_interior<S, R>(P, g_in, c, x, y, g);
        }
    }
    stage_tile2d<S, R, TX, TY, WALLS, TX * TY>(P, sm, x0, y0, tid, T_in, Y_in, solid);
    __syncthreads();

    if (!inside) return;
    const int p0 = (ty + 2) * SX + tx + 2;
    if constexpr (WALLS) {
        if (sm.mask[p0]) return;  // solid
        fast = interior_point<SX>(sm.mask, p0);
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
        if (!fast) return;  // solid, or a boundary cell: another kernel updates it
    }
    // a1 for the wall tiles: pull from the neighbours (Eq. 8), half-way
    // bounce-back from an in-domain solid neighbour (Eq. 28)
    if constexpr (WALLS) {
        const int oxm = x == 0 ? P.nx - 1 : -1, oxp = x == P.nx - 1 ? 1 - P.nx : 1;
        const int oym = y == 0 ? (P.ny - 1) * P.nx : -P.nx, oyp = y == P.ny - 1 ? (1 - P.ny) * P.nx : P.nx;
        const S* gc = g_in + c;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ox = cx_of(i) > 0 ? oxm : (cx_of(i) < 0 ? oxp : 0);
            const int oy = cy_of(i) > 0 ? oym : (cy_of(i) < 0 ? oyp : 0);
            long long off = (long long)i * N + (ox + oy);
            if (sm.mask[p0 - cx_of(i) - cy_of(i) * SX]) off = (long long)opposite<2>(i) * N;
            g[i] = R(LBFD_LDG(gc + off));
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
    TileAccum<R> acc;
    acc.clear();
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
    const R q = arrhenius(P, T0, pick_species(Y0, P.fuel), pick_species(Y0, P.oxid));
    const R reac_T = P.Q_cp * q;
    // a7
    const R DT = acc.diff_T + reac_T;
    T_out[c] = S(T0 + (DT - acc.conv_T));
#pragma unroll
    for (int k = 0; k < NSP; ++k) Y_out[(long long)k * N + c] = S(Y0[k] + (acc.rhs_Y[k] + P.yield[k] * q));
    const R lam_Y = acc.lamY + P.lam_yield * q;
    const R Lam = fdiv(DT, T0) + fdiv(lam_Y, invW0);
    // a8-a10
    collide<2, R>(P, g, rho0, u, acc.grad_rho, Lam);
#pragma unroll
    for (int i = 0; i < 9; ++i) g_out[(long long)i * N + c] = S(g[i]);
}

// FP32: four 256-thread blocks (1024 threads) per SM, i.e. <= 64 registers
template <typename S, typename R, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, sizeof(R) == 4 ? 1024 / (TX * TY) : 1)
    step_kernel_tiled2d(StepParams<R> P, const S* LBFD_RESTRICT g_in, S* LBFD_RESTRICT g_out,
                        const S* LBFD_RESTRICT T_in, S* LBFD_RESTRICT T_out, const S* LBFD_RESTRICT Y_in,
                        S* LBFD_RESTRICT Y_out, const uint8_t* LBFD_RESTRICT interior)
{
    tiled2d_body<S, R, TX, TY, false>(P, g_in, g_out, T_in, T_out, Y_in, Y_out, nullptr, interior, threadIdx.x,
                                      threadIdx.y, blockIdx.x, blockIdx.y);
}

// the cells next to in-domain solid cells, over the tiles that contain any
template <typename S, typename R, int TX, int TY>
__global__ void __launch_bounds__(TX * TY)
    step_kernel_tiled2d_walls(StepParams<R> P, const S* LBFD_RESTRICT g_in, S* LBFD_RESTRICT g_out,
                              const S* LBFD_RESTRICT T_in, S* LBFD_RESTRICT T_out, const S* LBFD_RESTRICT Y_in,
                              S* LBFD_RESTRICT Y_out, const uint8_t* LBFD_RESTRICT solid, const int* LBFD_RESTRICT tiles)
{
    const int t = tiles[blockIdx.x];
    const int gxn = (P.nx + TX - 1) / TX;
    tiled2d_body<S, R, TX, TY, true>(P, g_in, g_out, T_in, T_out, Y_in, Y_out, solid, nullptr, threadIdx.x,
                                     threadIdx.y, t % gxn, t / gxn);
}

// The cells of a coded list: next to in-domain solids (staircase walls, no
// non-periodic face in reach), or (FACES) near inlet and outlet faces:
// cell_step_coded
template <int DIM, typename S, typename R, bool FACES = false, bool HI1 = false>
__global__ void __launch_bounds__(128) step_kernel_wallcode(StepParams<R> P, const S* LBFD_RESTRICT g_in,
                                                            S* LBFD_RESTRICT g_out, const S* LBFD_RESTRICT T_in,
                                                            S* LBFD_RESTRICT T_out, const S* LBFD_RESTRICT Y_in,
                                                            S* LBFD_RESTRICT Y_out,
                                                            const long long* LBFD_RESTRICT cells,
                                                            const unsigned long long* LBFD_RESTRICT codes,
                                                            long long ncells)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncells) return;
    const long long c = cells[t];
    int p[3];
    p[0] = (int)(c % P.nx);
    const long long r = c / P.nx;
    p[1] = (int)(r % P.ny);
    p[2] = (int)(r / P.ny);
    cell_step_coded<DIM, S, R, FACES, HI1>(P, p, c, codes[t], g_in, g_out, T_in, T_out, Y_in, Y_out);
}

// The cells the tiled kernel leaves out: general form over a cell list
// (FACES == false: cells whose stencils reach no non-periodic face).
template <int DIM, typename S, typename R, bool FACES = true>
__global__ void __launch_bounds__(128) step_kernel_boundary(StepParams<R> P, const S* LBFD_RESTRICT g_in,
                                                            S* LBFD_RESTRICT g_out, const S* LBFD_RESTRICT T_in,
                                                            S* LBFD_RESTRICT T_out, const S* LBFD_RESTRICT Y_in,
                                                            S* LBFD_RESTRICT Y_out, const uint8_t* LBFD_RESTRICT solid,
                                                            const long long* LBFD_RESTRICT cells, long long ncells)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncells) return;
    const long long c = cells[t];
    int p[3];
    p[0] = (int)(c % P.nx);
    const long long r = c / P.nx;
    p[1] = (int)(r % P.ny);
    p[2] = (int)(r / P.ny);
    cell_step_general<DIM, S, R, FACES>(P, p, c, g_in, g_out, T_in, T_out, Y_in, Y_out, solid);
}

}  // namespace lbfd
