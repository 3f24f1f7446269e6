// lbfd_step_tiled3d.cuh -- 3-D (D3Q27) fused coupled step, 2.5-D tiling.
//
// A block of TX x TY threads owns a TX x TY column of cells and marches it
// through ZC consecutive z-planes.  Shared memory holds a ring of five
// z-planes (z-2 .. z+2) of the tile plus its 2-cell x/y halo, with T, Y_k
// and the derived W, 1/W, rho of every point (X_k = Y_k W / W_k is formed
// when used); each plane is loaded once per column pass.  Interior cells
// (every +-2 axis neighbour and all 26 LB neighbours are fluid cells of the
// domain; per-cell class 1, computed at create) are updated here.  The
// wall-aware variants (WALLS) also update the cells next to in-domain
// solids whose stencils reach no domain face (class 2): their FD lines take
// ghost points by the mirror rule of Eq. 34 from the staged tile and mask,
// and their pull bounces back from solid neighbours (Eq. 28), so only the
// cells near domain faces are left to step_kernel_boundary.
#pragma once
#include "lbfd_step_tiled.cuh"

namespace lbfd {

template <int TX, int TY>
struct Tile3Geom {
    static constexpr int SX = TX + 4;
    static constexpr int SY = TY + 4;
    static constexpr int NPP = SX * SY;  // points per plane
    static constexpr int NPL = 5;        // planes in the ring
    static constexpr int NPT = NPP * NPL;
};

template <typename R, int TX, int TY>
__host__ __device__ constexpr size_t tile3_smem_bytes()
{
    // T, Y_k, 1/W, W, rho per point (X_k = Y_k W / W_k is formed when used)
    return sizeof(R) * (size_t)Tile3Geom<TX, TY>::NPT * (4 + NSP) + (size_t)Tile3Geom<TX, TY>::NPT;
}

// FD terms along one axis from five explicit shared-memory points (the
// X_k lines first, as in fd_axis_core); returns d rho / d x_a.  `ghost`
// flags (bit j) the points that are ghosts of an in-domain solid (pts then
// holds their mirror points): T and rho take the Dirichlet form at
// isothermal solids, Y_k and W mirror, and the convection of the axis is
// centred (Sec. II.D, next to a boundary).  ghost == 0 for interior cells.
template <typename R>
__device__ __forceinline__ R fd_axis_pts(const StepParams<R>& P, const TileSmem<R>& sm, int npt, const int* pts,
                                         int ghost, R u_a, const R* Y0, R invW0, R rho0, TileAccum<R>& acc)
{
    R v[5], w[5];
    const bool dir = ghost != 0 && P.solid_isothermal;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        v[j] = sm.rho[pts[j]];
        if (dir && ((ghost >> j) & 1)) v[j] = R(2) * eos(P, P.T_solid, sm.invW[pts[j]]) - v[j];
    }
    const R drho = fd_d1(v);
    const R drho_r = fdiv(drho, rho0);
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        v[j] = sm.T[pts[j]];
        if (dir && ((ghost >> j) & 1)) v[j] = R(2) * P.T_solid - v[j];
    }
    // next to a wall the axis is centred: both are formed and one is kept,
    // so that a warp mixing wall and interior cells does not branch
    const bool near = ghost != 0;
    const R wT = weno3_deriv_fast(v, u_a, P.epsT);
    acc.conv_T += u_a * (near ? fd_c2(v) : wT);
    acc.diff_T += P.alpha12 * (fd_D2(v) + drho_r * fd_D1(v));  // 12x stencils, alpha / 12
#pragma unroll
    for (int j = 0; j < 5; ++j) w[j] = sm.invW[pts[j]];
    const R dinvW = fd_d1(w);
    R Wl[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) Wl[j] = sm.X[pts[j]];  // W (the 3-D tile keeps W in the X slot)
    R m[NSP], dm[NSP];
    R M = R(0), dM = R(0);
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] = sm.Y[k * npt + pts[j]] * Wl[j];  // X_k W_k (1/W_k and 1/12 in a12)
        const R dX = fd_D1(v), d2X = fd_D2(v);
        m[k] = P.a12[k] * invW0 * dX;
        dm[k] = P.a12[k] * (invW0 * d2X + dinvW * dX);
        M += m[k];
        dM += dm[k];
    }
    R sumL = R(0);
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] = sm.Y[k * npt + pts[j]];
        const R wk = weno3_deriv_fast(v, u_a, P.epsY);
        const R Lk = near ? fd_c2(v) : wk;
        sumL += Lk;
        const R dY = fd_d1(v);
        const R dk = dm[k] - dY * M - Y0[k] * dM + (m[k] - Y0[k] * M) * drho_r;
        acc.rhs_Y[k] += dk - u_a * Lk;
        acc.lamY += P.inv_Wk[k] * dk;
    }
    const R us = u_a * sumL;
#pragma unroll
    for (int k = 0; k < NSP; ++k) acc.rhs_Y[k] += Y0[k] * us;
    return drho;
}

// the five points of an axis line after the mirror rule of Eq. 34 for a
// cell next to in-domain solid cells: raw[j] are the staged points at
// offsets -2..2; the ghost at distance j beyond a wall at distance w
// mirrors the point at offset 2w - 1 - j (the neighbour on the other side,
// or the centre when that is solid, for offset -1).  Returns the ghost bits.
__device__ __forceinline__ int wall_line_pts(const uint8_t* mask, const int* raw, int* pts)
{
    int ghost = 0;
#pragma unroll
    for (int j = 0; j < 5; ++j) pts[j] = raw[j];
#pragma unroll
    for (int side = -1; side <= 1; side += 2) {
        const int w = mask[raw[2 + side]] ? 1 : (mask[raw[2 + 2 * side]] ? 2 : 0);
        if (!w) continue;
#pragma unroll
        for (int j = 1; j <= 2; ++j) {
            if (j < w) continue;
            const int m = 2 * w - 1 - j;
            const int mp = m >= 0 ? raw[2 + side * m] : (mask[raw[2 - side]] ? raw[2] : raw[2 - side]);
            pts[2 + side * j] = mp;
            ghost |= 1 << (2 + side * j);
        }
    }
    return ghost;
}

// stage plane z (grid coordinate) into ring slot `slot`; solid points are
// staged like fluid ones (never read by an interior cell; with WALLS the
// mask marks them, 1 solid, 2 outside the domain, for the wall cells)
template <typename S, typename R, int TX, int TY, bool WALLS = false>
__device__ __forceinline__ void stage_plane(const StepParams<R>& P, const TileSmem<R>& sm, int slot, int x0, int y0,
                                            int z, const S* LBFD_RESTRICT T_in, const S* LBFD_RESTRICT Y_in,
                                            const uint8_t* LBFD_RESTRICT solid = nullptr)
{
    using G = Tile3Geom<TX, TY>;
    constexpr int NPT = G::NPT;
    const long long N = P.N;
    constexpr int NTHR = TX * TY, NIT = (G::NPP + NTHR - 1) / NTHR;
    const int tid = threadIdx.x + TX * threadIdx.y;
    // all of this thread's global loads first, then the derived values
    long long cell[NIT];  // -1: outside the domain
    R T[NIT], Y[NIT][NSP];
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        const int q = tid + it * NTHR;
        cell[it] = -1;
        if (q >= G::NPP) continue;
        const int sx = q % G::SX, sy = q / G::SX;
        int gx = x0 + sx - 2, gy = y0 + sy - 2, gz = z;
        // across a periodic face the halo holds the wrapped cells
        if ((gx < 0 || gx >= P.nx) && P.bc[0] == BC_PERIODIC) gx = ((gx % P.nx) + P.nx) % P.nx;
        if ((gy < 0 || gy >= P.ny) && P.bc[2] == BC_PERIODIC) gy = ((gy % P.ny) + P.ny) % P.ny;
        if ((gz < 0 || gz >= P.nz) && P.bc[4] == BC_PERIODIC) gz = ((gz % P.nz) + P.nz) % P.nz;
        if (gx < 0 || gx >= P.nx || gy < 0 || gy >= P.ny || gz < 0 || gz >= P.nz) {
            if constexpr (WALLS) sm.mask[slot * G::NPP + q] = 2;
            continue;
        }
        const long long c = (long long)gx + (long long)P.nx * (gy + (long long)P.ny * gz);
        cell[it] = c;
        if constexpr (WALLS) sm.mask[slot * G::NPP + q] = solid[c] ? 1 : 0;
        T[it] = R(T_in[c]);
#pragma unroll
        for (int k = 0; k < NSP; ++k) Y[it][k] = R(Y_in[(long long)k * N + c]);
    }
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        if (cell[it] < 0) continue;
        const int pt = slot * G::NPP + tid + it * NTHR;
        const R invW = inv_molar_mass(P, Y[it]);
        const R W = fdiv(R(1), invW);
        sm.T[pt] = T[it];
#pragma unroll
        for (int k = 0; k < NSP; ++k) sm.Y[k * NPT + pt] = Y[it][k];
        sm.X[pt] = W;  // the 3-D tile keeps W in the X slot
        sm.invW[pt] = invW;
        sm.rho[pt] = fdiv(P.T_in * P.invW_in * W, T[it]);
    }
}

// SPLIT: steps a1-a7 only; Lambda and grad rho of every interior cell go
// to aux (four planes) for step_kernel_collide3d, which does a8-a10
template <typename S, typename R, int TX, int TY, int ZC, bool SPLIT = false, bool WALLS = false, bool HI1 = false>
__device__ __forceinline__ void tiled3d_body(const StepParams<R>& P, const S* LBFD_RESTRICT g_in,
                                             S* LBFD_RESTRICT g_out, const S* LBFD_RESTRICT T_in,
                                             S* LBFD_RESTRICT T_out, const S* LBFD_RESTRICT Y_in,
                                             S* LBFD_RESTRICT Y_out, const uint8_t* LBFD_RESTRICT interior,
                                             R* LBFD_RESTRICT aux = nullptr,
                                             const uint8_t* LBFD_RESTRICT solid = nullptr)
{
    using G = Tile3Geom<TX, TY>;
    constexpr int SX = G::SX, NPP = G::NPP, NPT = G::NPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<R> sm;
    sm.T = reinterpret_cast<R*>(smem_raw);
    sm.Y = sm.T + NPT;
    sm.X = sm.Y + NSP * NPT;  // one plane: W
    sm.invW = sm.X + NPT;
    sm.rho = sm.invW + NPT;
    sm.mask = reinterpret_cast<uint8_t*>(sm.rho + NPT);

    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, zb = blockIdx.z * ZC;
    const long long N = P.N;
    const long long plane = (long long)P.nx * P.ny;
    // ring slot of grid plane z: (z + 5*big) % 5 keeps it non-negative
    auto slot_of = [](int z) { return (z + 10) % 5; };
    for (int dz = -2; dz <= 1; ++dz)
        stage_plane<S, R, TX, TY, WALLS>(P, sm, slot_of(zb + dz), x0, y0, zb + dz, T_in, Y_in, solid);
    if constexpr (WALLS) __syncthreads();  // the masks of planes z-1..z+1 are read by the first pull
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const int q0 = (threadIdx.y + 2) * SX + threadIdx.x + 2;  // in-plane point of this thread
    const int zend = zb + ZC < P.nz ? zb + ZC : P.nz;
    const bool inside = x < P.nx && y < P.ny;
    for (int z = zb; z < zend; ++z) {
        // a1 issued before the staging of plane z+2, so that the population
        // loads are in flight meanwhile (pull with periodic wrap; the
        // offsets stay inside the domain for any in-range cell)
        const long long c = (long long)x + (long long)P.nx * y + plane * z;
        R g[27];
        // the cell's class (1: +-2 along the three axes and the 26 neighbours
        // are fluid cells of the domain; 2: next to in-domain solids, no
        // domain face in reach), precomputed per cell
        bool active = false, wall = false;
        if (inside) {
            const int cls = interior[c];
            wall = WALLS && cls == 2 && !P.curved;
            active = cls == 1 || wall;
            const int oxm = x == 0 ? P.nx - 1 : -1, oxp = x == P.nx - 1 ? 1 - P.nx : 1;
            const long long oym = y == 0 ? (long long)(P.ny - 1) * P.nx : -(long long)P.nx;
            const long long oyp = y == P.ny - 1 ? (long long)(1 - P.ny) * P.nx : (long long)P.nx;
            const long long ozm = z == 0 ? (P.nz - 1) * plane : -plane;
            const long long ozp = z == P.nz - 1 ? (1 - P.nz) * plane : plane;
            const S* gc = g_in + c;
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                long long o = (long long)i * N + (cx_of(i) > 0 ? oxm : (cx_of(i) < 0 ? oxp : 0)) +
                              (cy_of(i) > 0 ? oym : (cy_of(i) < 0 ? oyp : 0)) +
                              (cz_of(i) > 0 ? ozm : (cz_of(i) < 0 ? ozp : 0));
                if constexpr (WALLS) {
                    // half-way bounce-back from a solid neighbour (Eq. 28)
                    const int src = slot_of(z - cz_of(i)) * NPP + q0 - cx_of(i) - cy_of(i) * SX;
                    const bool bb = (sm.mask[src] != 0) & wall;
                    o = bb ? (long long)opposite<3>(i) * N : o;
                }
                g[i] = R(LBFD_LDG(gc + o));
            }
        }
        stage_plane<S, R, TX, TY, WALLS>(P, sm, slot_of(z + 2), x0, y0, z + 2, T_in, Y_in, solid);
        __syncthreads();
        const int sc = slot_of(z);
        const int p0 = sc * NPP + q0;
        if (active) {
            const R T0 = sm.T[p0], invW0 = sm.invW[p0], rho0 = sm.rho[p0];
            R Y0[NSP];
#pragma unroll
            for (int k = 0; k < NSP; ++k) Y0[k] = sm.Y[k * NPT + p0];
            R u[3];
            {
                const R inv = fdiv(R(3), rho0);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    R m = R(0);
#pragma unroll
                    for (int i = 0; i < 27; ++i) {
                        const int ci = ccomp<3>(i, a);
                        if (ci) m += R(ci) * g[i];
                    }
                    u[a] = m * inv;
                }
            }
            TileAccum<R> acc;
            acc.clear();
            // the three axes share one copy of the FD code (a rolled loop keeps
            // the kernel small enough for the instruction cache)
#pragma unroll 1
            for (int a = 0; a < 3; ++a) {
                int pts[5];
#pragma unroll
                for (int j = 0; j < 5; ++j)
                    pts[j] = a == 0 ? p0 + (j - 2) : (a == 1 ? p0 + (j - 2) * SX : slot_of(z + j - 2) * NPP + q0);
                int ghost = 0;
                if constexpr (WALLS) {
                    if (wall) {
                        int raw[5];
#pragma unroll
                        for (int j = 0; j < 5; ++j) raw[j] = pts[j];
                        ghost = wall_line_pts(sm.mask, raw, pts);
                    }
                }
                const R u_a = a == 0 ? u[0] : (a == 1 ? u[1] : u[2]);
                const R drho = fd_axis_pts<R>(P, sm, NPT, pts, ghost, u_a, Y0, invW0, rho0, acc);
                acc.grad_rho[0] = a == 0 ? drho : acc.grad_rho[0];
                acc.grad_rho[1] = a == 1 ? drho : acc.grad_rho[1];
                acc.grad_rho[2] = a == 2 ? drho : acc.grad_rho[2];
            }
            const R q = arrhenius(P, T0, pick_species(Y0, P.fuel), pick_species(Y0, P.oxid));
            const R DT = acc.diff_T + P.Q_cp * q;
            T_out[c] = S(T0 + (DT - acc.conv_T));
#pragma unroll
            for (int k = 0; k < NSP; ++k) Y_out[(long long)k * N + c] = S(Y0[k] + (acc.rhs_Y[k] + P.yield[k] * q));
            const R lam_Y = acc.lamY + P.lam_yield * q;
            const R Lam = fdiv(DT, T0) + fdiv(lam_Y, invW0);
            if constexpr (SPLIT) {
                aux[c] = Lam;
#pragma unroll
                for (int a = 0; a < 3; ++a) aux[(long long)(1 + a) * N + c] = acc.grad_rho[a];
            } else {
                collide<3, R, R, HI1>(P, g, rho0, u, acc.grad_rho, Lam);
#pragma unroll
                for (int i = 0; i < 27; ++i) g_out[(long long)i * N + c] = S(g[i]);
            }
        }
        __syncthreads();  // the slot of z-2 is restaged next iteration
    }
}

template <typename S, typename R, int TX, int TY, int ZC, bool HI1 = false>
__global__ void __launch_bounds__(TX * TY) step_kernel_tiled3d(StepParams<R> P, const S* LBFD_RESTRICT g_in,
                                                               S* LBFD_RESTRICT g_out, const S* LBFD_RESTRICT T_in,
                                                               S* LBFD_RESTRICT T_out, const S* LBFD_RESTRICT Y_in,
                                                               S* LBFD_RESTRICT Y_out,
                                                               const uint8_t* LBFD_RESTRICT interior)
{
    tiled3d_body<S, R, TX, TY, ZC, false, false, HI1>(P, g_in, g_out, T_in, T_out, Y_in, Y_out, interior);
}

// interior cells and, from the same staging, the cells next to in-domain
// solids (class 2): no separate wall-list kernel
template <typename S, typename R, int TX, int TY, int ZC>
__global__ void __launch_bounds__(TX * TY) step_kernel_tiled3d_walls(StepParams<R> P, const S* LBFD_RESTRICT g_in,
                                                                     S* LBFD_RESTRICT g_out,
                                                                     const S* LBFD_RESTRICT T_in,
                                                                     S* LBFD_RESTRICT T_out,
                                                                     const S* LBFD_RESTRICT Y_in,
                                                                     S* LBFD_RESTRICT Y_out,
                                                                     const uint8_t* LBFD_RESTRICT interior,
                                                                     const uint8_t* LBFD_RESTRICT solid)
{
    tiled3d_body<S, R, TX, TY, ZC, false, true>(P, g_in, g_out, T_in, T_out, Y_in, Y_out, interior, nullptr, solid);
}

// the same with the registers capped so that MINB blocks fit on an SM
template <typename S, typename R, int TX, int TY, int ZC, int MINB, bool HI1 = false>
__global__ void __launch_bounds__(TX * TY, MINB)
    step_kernel_tiled3d_capped(StepParams<R> P, const S* LBFD_RESTRICT g_in, S* LBFD_RESTRICT g_out,
                               const S* LBFD_RESTRICT T_in, S* LBFD_RESTRICT T_out, const S* LBFD_RESTRICT Y_in,
                               S* LBFD_RESTRICT Y_out, const uint8_t* LBFD_RESTRICT interior)
{
    tiled3d_body<S, R, TX, TY, ZC, false, false, HI1>(P, g_in, g_out, T_in, T_out, Y_in, Y_out, interior);
}

// a1-a7 of the interior cells (the FD half of a split step); FP32 held to
// four 128-thread blocks per SM
template <typename S, typename R, int TX, int TY, int ZC>
__global__ void __launch_bounds__(TX * TY, sizeof(R) == 4 ? 512 / (TX * TY) : 1)
    step_kernel_fd3d(StepParams<R> P, const S* LBFD_RESTRICT g_in, const S* LBFD_RESTRICT T_in, S* LBFD_RESTRICT T_out,
                     const S* LBFD_RESTRICT Y_in, S* LBFD_RESTRICT Y_out, const uint8_t* LBFD_RESTRICT interior,
                     R* LBFD_RESTRICT aux)
{
    tiled3d_body<S, R, TX, TY, ZC, true>(P, g_in, nullptr, T_in, T_out, Y_in, Y_out, interior, aux);
}

// a1, a2 and a8-a10 of the interior cells (the LB half of a split step):
// the pull and the density are recomputed exactly as in the FD half, Lambda
// and grad rho read from aux.  One thread per cell, 128 cells of an x-row
// per block.
template <typename S, typename R>
__global__ void __launch_bounds__(128)
    step_kernel_collide3d(StepParams<R> P, const S* LBFD_RESTRICT g_in, S* LBFD_RESTRICT g_out,
                          const S* LBFD_RESTRICT T_in, const S* LBFD_RESTRICT Y_in,
                          const uint8_t* LBFD_RESTRICT interior, const R* LBFD_RESTRICT aux)
{
    const int x = blockIdx.x * 128 + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const long long N = P.N;
    const long long plane = (long long)P.nx * P.ny;
    const long long c = (long long)x + (long long)P.nx * y + plane * z;
    if (interior[c] != 1) return;
    R g[27];
    {
        const int oxm = x == 0 ? P.nx - 1 : -1, oxp = x == P.nx - 1 ? 1 - P.nx : 1;
        const long long oym = y == 0 ? (long long)(P.ny - 1) * P.nx : -(long long)P.nx;
        const long long oyp = y == P.ny - 1 ? (long long)(1 - P.ny) * P.nx : (long long)P.nx;
        const long long ozm = z == 0 ? (P.nz - 1) * plane : -plane;
        const long long ozp = z == P.nz - 1 ? (1 - P.nz) * plane : plane;
        const S* gc = g_in + c;
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const long long o = (cx_of(i) > 0 ? oxm : (cx_of(i) < 0 ? oxp : 0)) +
                                (cy_of(i) > 0 ? oym : (cy_of(i) < 0 ? oyp : 0)) +
                                (cz_of(i) > 0 ? ozm : (cz_of(i) < 0 ? ozp : 0));
            g[i] = R(LBFD_LDG(gc + (long long)i * N + o));
        }
    }
    // the density as staged by the FD half
    const R T0 = R(T_in[c]);
    R Y0[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) Y0[k] = R(Y_in[(long long)k * N + c]);
    const R invW0 = inv_molar_mass(P, Y0);
    const R W = fdiv(R(1), invW0);
    const R rho0 = fdiv(P.T_in * P.invW_in * W, T0);
    R u[3];
    {
        const R inv = fdiv(R(3), rho0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R m = R(0);
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const int ci = ccomp<3>(i, a);
                if (ci) m += R(ci) * g[i];
            }
            u[a] = m * inv;
        }
    }
    const R Lam = aux[c];
    R grad[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) grad[a] = aux[(long long)(1 + a) * N + c];
    collide<3, R>(P, g, rho0, u, grad, Lam);
#pragma unroll
    for (int i = 0; i < 27; ++i) g_out[(long long)i * N + c] = S(g[i]);
}

}  // namespace lbfd
