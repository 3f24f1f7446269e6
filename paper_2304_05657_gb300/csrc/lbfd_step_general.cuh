// lbfd_step_general.cuh -- the fused coupled step for one fluid cell, general
// form: every neighbour access goes through the boundary classification, so
// it is valid for any cell (walls, solid mask, inlet, outlet, periodic
// wrap).  One call = steps a1-a10 of one cell:
//   a1 pull streaming with half-way bounce-back (Eq. 28), velocity inlet
//      (Eq. 31) and convective outlet (Eq. 32);
//   a2 EOS density and velocity (Eq. 13b);
//   a3 ghost-node FD lines (Eq. 34); a4 WENO3/centred convection with the
//      mass-conserving correction (Eq. 26); a5 4th-order diffusion of
//      T (Eq. 7) and Y_k with the correction velocity (Eq. 1-2);
//   a6 single-step Arrhenius source; a7 explicit Euler and Lambda (Eq. 6);
//   a8-a9 source Xi (Eq. 9), pre-conditioning (Eq. 19) and cumulant
//      collision (Eq. 14-24); a10 write g*.
#pragma once
#include "lbfd_device.cuh"

namespace lbfd {

// ---------------------------------------------------------------------------
// a1: pull one population with the boundary rules
// ---------------------------------------------------------------------------
template <int DIM, typename S, typename R, bool FACES = true>
__device__ __forceinline__ R pull_general(const StepParams<R>& P, int i, const int p[3], long long c,
                                          const S* LBFD_RESTRICT g, const uint8_t* LBFD_RESTRICT solid,
                                          R rho_cell)
{
    const long long N = P.N;
    int src[3] = {p[0] - ccomp<DIM>(i, 0), p[1] - ccomp<DIM>(i, 1), DIM == 3 ? p[2] - ccomp<DIM>(i, 2) : 0};
    int wall = 0, inlet = -1, outlet = -1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const int n = extent(P, a);
        int f = -1;
        if (src[a] < 0) f = 2 * a;
        else if (src[a] >= n) f = 2 * a + 1;
        if (f < 0) continue;
        const int t = P.bc[f];
        if (!FACES || t == BC_PERIODIC) src[a] = ((src[a] % n) + n) % n;
        else if (t == BC_INLET) { if (inlet < 0) inlet = f; }
        else if (t == BC_OUTLET || t == BC_OUTLET_PRESSURE) { if (outlet < 0) outlet = f; }
        else wall = 1;
    }
    const int ib = opposite<DIM>(i);
    if (!wall && (inlet >= 0 || outlet >= 0)) {
        // leaving through an inlet/outlet face where the boundary column is
        // solid: the link hits the solid (bounce-back, as at a wall corner)
        int q[3] = {src[0], src[1], src[2]};
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const int n = extent(P, a);
            q[a] = q[a] < 0 ? 0 : (q[a] >= n ? n - 1 : q[a]);
        }
        if (solid[cell_of(P, q[0], q[1], DIM == 3 ? q[2] : 0)]) wall = 1;
    }
    if (wall) return R(g[(long long)ib * N + c]);  // Eq. 28
    if (inlet >= 0) {                              // Eq. 31 applied to g
        const int a = inlet / 2;
        R mag = P.u_in;
        if (P.poiseuille && DIM == 2 && a == 0) {
            const R ny = R(P.ny), y = R(p[1]) + R(0.5);
            mag = R(6) * P.u_in * y * (ny - y) / (ny * ny);
        }
        const R un = (inlet % 2 == 0) ? mag : -mag;  // along the inward normal
        const R cu = R(ccomp<DIM>(i, a)) * un;
        return R(g[(long long)ib * N + c]) + R(2) * weight<DIM, R>(i) * P.rho_in * cu;
    }
    if (outlet >= 0 && P.bc[outlet] == BC_OUTLET_PRESSURE) {
        // constant P_h = 0: anti-bounce-back with twice the even part of g^eq
        R uc[3] = {R(0), R(0), R(0)};
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            R m = R(0);
#pragma unroll
            for (int j = 0; j < (DIM == 2 ? 9 : 27); ++j) {
                const int cj = ccomp<DIM>(j, a);
                if (cj != 0) m += R(cj) * R(g[(long long)j * N + c]);
            }
            uc[a] = m * fdiv(R(3), rho_cell);
        }
        R cu = R(0), uu = R(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            cu += R(ccomp<DIM>(i, a)) * uc[a];
            uu += uc[a] * uc[a];
        }
        const R wi = weight<DIM, R>(i);
        const R geq_even = wi * rho_cell * (R(1.5) * cu * cu - R(0.5) * uu);
        return R(2) * geq_even - R(g[(long long)ib * N + c]);
    }
    if (outlet >= 0) {  // Eq. 32 in lattice units
        const int a = outlet / 2;
        const int ns = (outlet % 2 == 1) ? 1 : -1;  // outward normal along a
        R mom = R(0);
#pragma unroll
        for (int j = 0; j < (DIM == 2 ? 9 : 27); ++j) {
            const int cj = ccomp<DIM>(j, a) * ns;
            if (cj != 0) mom += R(cj) * R(g[(long long)j * N + c]);
        }
        const R un = fdiv(R(3) * mom, rho_cell);
        int q[3] = {p[0], p[1], p[2]};
        q[a] -= ns;
        R inner = R(g[(long long)i * N + c]);
        if (q[a] >= 0 && q[a] < extent(P, a)) {
            const long long qi = cell_of(P, q[0], q[1], DIM == 3 ? q[2] : 0);
            if (!solid[qi]) inner = R(g[(long long)i * N + qi]);
        }
        return (P.cs - un) * inner + (R(1) - P.cs + un) * R(g[(long long)i * N + c]);
    }
    const long long s = cell_of(P, src[0], src[1], DIM == 3 ? src[2] : 0);
    if (solid[s]) {
        const int row = P.curved ? P.link_row[c] : -1;
        const double qd = row >= 0 ? P.link_q[(long long)row * (DIM == 2 ? 9 : 27) + i] : -1.0;
        if (qd < 0.0) return R(g[(long long)ib * N + c]);  // Eq. 28
        // interpolated bounce-back (Eq. 29-30), post-collision values at t
        const R q = R(qd);
        if (qd < 0.5) {
            int r[3] = {p[0] + ccomp<DIM>(i, 0), p[1] + ccomp<DIM>(i, 1), DIM == 3 ? p[2] + ccomp<DIM>(i, 2) : 0};
            long long ridx = 0;
            int face = -1;
            if (classify<DIM, R, FACES>(P, r, solid, &ridx, &face) == PT_FLUID)
                return R(2) * q * R(g[(long long)ib * N + c]) + (R(1) - R(2) * q) * R(g[(long long)ib * N + ridx]);
            return R(g[(long long)ib * N + c]);
        }
        return R(g[(long long)ib * N + c]) / (R(2) * q) + (R(2) * q - R(1)) / (R(2) * q) * R(g[(long long)i * N + c]);
    }
    return R(g[(long long)i * N + s]);  // Eq. 8
}

// a1 for a cell whose lattice neighbours are all inside the domain up to
// periodic wrap and whose walls are staircase: plain pull, half-way
// bounce-back (Eq. 28) from solid neighbours
template <int DIM, typename S, typename R>
__device__ __forceinline__ void pull_walls(const StepParams<R>& P, const int p[3], long long c,
                                           const S* LBFD_RESTRICT g, const uint8_t* LBFD_RESTRICT solid, R* out)
{
    constexpr int Q = DIM == 2 ? 9 : 27;
    const long long N = P.N;
    const long long plane = (long long)P.nx * P.ny;
    // offsets to the x-1, x+1, ... neighbours (wrapped on periodic axes)
    const long long oxm = p[0] == 0 ? P.nx - 1 : -1, oxp = p[0] == P.nx - 1 ? 1 - P.nx : 1;
    const long long oym = p[1] == 0 ? (long long)(P.ny - 1) * P.nx : -(long long)P.nx;
    const long long oyp = p[1] == P.ny - 1 ? (long long)(1 - P.ny) * P.nx : (long long)P.nx;
    long long ozm = 0, ozp = 0;
    if (DIM == 3) {
        ozm = p[2] == 0 ? (P.nz - 1) * plane : -plane;
        ozp = p[2] == P.nz - 1 ? (1 - P.nz) * plane : plane;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = ccomp<DIM>(i, 0), cy = ccomp<DIM>(i, 1), cz = ccomp<DIM>(i, 2);
        const long long s = c + (cx > 0 ? oxm : (cx < 0 ? oxp : 0)) + (cy > 0 ? oym : (cy < 0 ? oyp : 0)) +
                            (cz > 0 ? ozm : (cz < 0 ? ozp : 0));
        out[i] = solid[s] ? R(g[(long long)opposite<DIM>(i) * N + c]) : R(g[(long long)i * N + s]);
    }
}

// ---------------------------------------------------------------------------
// a3: one FD line through the cell along an axis, with ghost points
// ---------------------------------------------------------------------------
template <typename R>
struct LineDesc {
    long long src[5];  // cell whose values feed the point (itself or its mirror)
    int mode[5];       // G_DIRECT / G_NEUMANN / G_DIRICHLET_T / G_INLET
    R TB[5];           // boundary temperature of Dirichlet ghosts
    int near;          // some point of the line is not a fluid cell
};

template <int DIM, typename R>
__device__ __forceinline__ void ghost_mode(const StepParams<R>& P, int type, int face, int* mode, R* TB)
{
    *TB = R(0);
    if (type == PT_SOLID) {
        *mode = P.solid_isothermal ? G_DIRICHLET_T : G_NEUMANN;
        *TB = P.T_solid;
    } else if (type == BC_WALL_ISOTHERMAL) {
        *mode = G_DIRICHLET_T;
        *TB = P.T_wall[face];
    } else if (type == BC_INLET) {
        *mode = G_INLET;
        *TB = P.T_in;
    } else {
        *mode = G_NEUMANN;  // adiabatic wall, outlet
    }
}

template <int DIM, typename R, bool FACES = true>
__device__ __forceinline__ void build_line(const StepParams<R>& P, const int p[3], long long c, int a,
                                           const uint8_t* LBFD_RESTRICT solid, LineDesc<R>& L)
{
    L.near = 0;
    L.src[2] = c;
    L.mode[2] = G_DIRECT;
    L.TB[2] = R(0);
#pragma unroll
    for (int side = -1; side <= 1; side += 2) {
        int w = 0, wtype = 0, wface = -1;
#pragma unroll
        for (int j = 1; j <= 2; ++j) {
            if (w) break;
            int q[3] = {p[0], p[1], p[2]};
            q[a] += side * j;
            long long idx = 0;
            int face = -1;
            const int t = classify<DIM, R, FACES>(P, q, solid, &idx, &face);
            if (t == PT_FLUID) {
                L.src[2 + side * j] = idx;
                L.mode[2 + side * j] = G_DIRECT;
                L.TB[2 + side * j] = R(0);
            } else {
                w = j;
                wtype = t;
                wface = face;
            }
        }
        if (!w) continue;
        L.near = 1;
        int mode;
        R TB;
        ghost_mode<DIM>(P, wtype, wface, &mode, &TB);
#pragma unroll
        for (int j = 1; j <= 2; ++j) {
            if (j < w) continue;
            if (P.curved) {  // a solid cell with an image-point ghost (Eq. 34-38)
                int q[3] = {p[0], p[1], p[2]};
                q[a] += side * j;
                long long idx = 0;
                int face = -1;
                if (classify<DIM, R, FACES>(P, q, solid, &idx, &face) == PT_SOLID && P.ghost_row[idx] >= 0) {
                    L.src[2 + side * j] = P.ghost_row[idx];
                    L.mode[2 + side * j] = G_CURVED;
                    L.TB[2 + side * j] = R(0);
                    continue;
                }
            }
            const int m = 2 * w - 1 - j;  // mirror offset on this side
            long long ms;
            if (m >= 0) {
                ms = L.src[2 + side * m];
            } else {
                int q[3] = {p[0], p[1], p[2]};
                q[a] -= side;
                long long idx = 0;
                int face = -1;
                ms = (classify<DIM, R, FACES>(P, q, solid, &idx, &face) == PT_FLUID) ? idx : c;
            }
            L.src[2 + side * j] = ms;
            L.mode[2 + side * j] = mode;
            L.TB[2 + side * j] = TB;
        }
    }
}

// values of one line point: T, Y_k, 1/W, rho (ghost rules of Eq. 34; the
// density of a ghost is reconstructed directly, with rho_B = EOS(T_B, Y))
template <typename S, typename R>
__device__ __forceinline__ void line_point(const StepParams<R>& P, const LineDesc<R>& L, int j,
                                           const S* LBFD_RESTRICT T, const S* LBFD_RESTRICT Y, R& Tj, R* Yj,
                                           R& invWj, R& rhoj)
{
    const long long s = L.src[j];
    if (L.mode[j] == G_CURVED) {  // precomputed image-point ghost of this step
        const R* gv = P.gval + s * GHOST_VALUES;
        Tj = gv[0];
#pragma unroll
        for (int k = 0; k < NSP; ++k) Yj[k] = gv[1 + k];
        invWj = gv[1 + NSP];
        rhoj = gv[2 + 2 * NSP];
        return;
    }
    const R Tm = R(T[s]);
    R Ym[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) Ym[k] = R(Y[(long long)k * P.N + s]);
    const R invWm = inv_molar_mass(P, Ym);
    const R rhom = eos(P, Tm, invWm);
    const int mode = L.mode[j];
    if (mode == G_DIRECT || mode == G_NEUMANN) {
        Tj = Tm;
#pragma unroll
        for (int k = 0; k < NSP; ++k) Yj[k] = Ym[k];
        invWj = invWm;
        rhoj = rhom;
    } else if (mode == G_DIRICHLET_T) {
        Tj = R(2) * L.TB[j] - Tm;
#pragma unroll
        for (int k = 0; k < NSP; ++k) Yj[k] = Ym[k];
        invWj = invWm;
        rhoj = R(2) * eos(P, L.TB[j], invWm) - rhom;
    } else {  // inlet: Dirichlet T_in and Y_in
        Tj = R(2) * P.T_in - Tm;
#pragma unroll
        for (int k = 0; k < NSP; ++k) Yj[k] = R(2) * P.Y_in[k] - Ym[k];
        invWj = inv_molar_mass(P, Yj);
        rhoj = R(2) * P.rho_in - rhom;
    }
}

// ---------------------------------------------------------------------------
// FD right-hand side along one axis, accumulated into the cell's terms.
// ---------------------------------------------------------------------------
template <typename R>
struct FDAccum {
    R conv_T, diff_T;
    R conv_Y[NSP], diff_Y[NSP];
    R grad_rho[3];
};

template <typename R>
__device__ __forceinline__ void fd_axis(const StepParams<R>& P, int a, int near, const R* Tl, const R (*Yl)[5],
                                        const R* invWl, const R* rhol, R u_a, R T0, const R* Y0, R invW0, R rho0,
                                        FDAccum<R>& acc)
{
    const R drho = fd_d1(rhol);
    acc.grad_rho[a] = drho;
    const R drho_r = fdiv(drho, rho0);
    // temperature: convection without correction, diffusion (Eq. 7)
    acc.conv_T += u_a * (near ? fd_c2(Tl) : weno3_deriv_fast(Tl, u_a, P.epsT));
    acc.diff_T += P.alpha * (fd_d2(Tl) + drho_r * fd_d1(Tl));
    // species convection with the correction of Eq. 26
    R Lk[NSP], sumL = R(0);
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
        Lk[k] = near ? fd_c2(Yl[k]) : weno3_deriv_fast(Yl[k], u_a, P.epsY);
        sumL += Lk[k];
    }
#pragma unroll
    for (int k = 0; k < NSP; ++k) acc.conv_Y[k] += u_a * (Lk[k] - Y0[k] * sumL);
    // species diffusion with the correction velocity (Eq. 1-2), expanded
    const R dinvW = fd_d1(invWl);
    R Wl[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) Wl[j] = fdiv(R(1), invWl[j]);
    R m[NSP], dm[NSP], dY[NSP], M = R(0), dM = R(0);
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
        R Xl[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) Xl[j] = Yl[k][j] * P.inv_Wk[k] * Wl[j];
        const R dX = fd_d1(Xl), d2X = fd_d2(Xl);
        m[k] = P.a_diff[k] * invW0 * dX;
        dm[k] = P.a_diff[k] * (invW0 * d2X + dinvW * dX);
        dY[k] = fd_d1(Yl[k]);
        M += m[k];
        dM += dm[k];
    }
#pragma unroll
    for (int k = 0; k < NSP; ++k)
        acc.diff_Y[k] += dm[k] - dY[k] * M - Y0[k] * dM + (m[k] - Y0[k] * M) * drho_r;
}

// ---------------------------------------------------------------------------
// The whole coupled update of one fluid cell (general form).  FACES ==
// false: a cell whose stencils reach no non-periodic domain face (the face
// rules are compiled out).
// ---------------------------------------------------------------------------
template <int DIM, typename S, typename R, bool FACES = true>
__device__ __forceinline__ void cell_step_general(const StepParams<R>& P, const int p[3], long long c,
                                                  const S* LBFD_RESTRICT g_in, S* LBFD_RESTRICT g_out,
                                                  const S* LBFD_RESTRICT T_in, S* LBFD_RESTRICT T_out,
                                                  const S* LBFD_RESTRICT Y_in, S* LBFD_RESTRICT Y_out,
                                                  const uint8_t* LBFD_RESTRICT solid)
{
    constexpr int Q = DIM == 2 ? 9 : 27;
    const long long N = P.N;
    // a2 (density first: the outlet rule needs it)
    const R T0 = R(T_in[c]);
    R Y0[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) Y0[k] = R(Y_in[(long long)k * N + c]);
    const R invW0 = inv_molar_mass(P, Y0);
    const R rho0 = eos(P, T0, invW0);
    // a1: a rolled loop (one copy of the boundary rules keeps this kernel
    // small enough for the instruction cache; the pulled values pass
    // through a local array)
    R g[Q];
    bool pulled = false;
    if constexpr (!FACES) {  // no face rules: the compact form (staircase walls)
        if (!P.curved) {
            pull_walls<DIM, S, R>(P, p, c, g_in, solid, g);
            pulled = true;
        }
    }
    if (!pulled) {
        R gl[Q];
#pragma unroll 1
        for (int i = 0; i < Q; ++i) gl[i] = pull_general<DIM, S, R, FACES>(P, i, p, c, g_in, solid, rho0);
#pragma unroll
        for (int i = 0; i < Q; ++i) g[i] = gl[i];
    }
    // a2: velocity, Eq. 13b
    R u[3] = {R(0), R(0), R(0)};
    {
        const R inv = fdiv(R(3), rho0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            R m = R(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int ci = ccomp<DIM>(i, a);
                if (ci) m += R(ci) * g[i];
            }
            u[a] = m * inv;
        }
    }
    // a3-a5
    FDAccum<R> acc;
    acc.conv_T = acc.diff_T = R(0);
#pragma unroll
    for (int k = 0; k < NSP; ++k) acc.conv_Y[k] = acc.diff_Y[k] = R(0);
    acc.grad_rho[0] = acc.grad_rho[1] = acc.grad_rho[2] = R(0);
#pragma unroll 1
    for (int a = 0; a < DIM; ++a) {
        LineDesc<R> L;
        build_line<DIM, R, FACES>(P, p, c, a, solid, L);
        R Tl[5], Yl[NSP][5], invWl[5], rhol[5];
#pragma unroll 1
        for (int j = 0; j < 5; ++j) {
            R Yj[NSP];
            line_point<S, R>(P, L, j, T_in, Y_in, Tl[j], Yj, invWl[j], rhol[j]);
#pragma unroll
            for (int k = 0; k < NSP; ++k) Yl[k][j] = Yj[k];
        }
        fd_axis<R>(P, a, L.near, Tl, Yl, invWl, rhol, u[a], T0, Y0, invW0, rho0, acc);
    }
    // a6: reaction
    const R q = arrhenius(P, T0, pick_species(Y0, P.fuel), pick_species(Y0, P.oxid));
    const R reac_T = P.Q_cp * q;
    // a7: Euler update and Lambda from the non-convective rates (Eq. 6)
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
    // a8-a9
    collide<DIM, R>(P, g, rho0, u, acc.grad_rho, Lam);
    // a10
#pragma unroll
    for (int i = 0; i < Q; ++i) g_out[(long long)i * N + c] = S(g[i]);
}

// ---------------------------------------------------------------------------
// The same update for a cell next to in-domain solids whose stencils reach
// no non-periodic face (staircase walls), or (FACES) for a cell near inlet
// and outlet faces of one axis, with its neighbourhood given by a code
// computed at create instead of mask reads:
//   bits 0..26   population i is pulled from a solid cell (bounce-back)
//   bits 32..49  per axis a (6 bits at 32 + 6a), per side (low 3 bits: -,
//                high 3 bits: +): the distance 1 or 2 of the first point
//                along the line that is not a fluid cell (0: none within 2)
//                and, in the third bit, whether the neighbour on the other
//                side is not a fluid cell either
//   bits 50..55  (FACES) per axis (2 bits at 50 + 2a, -: low, +: high): that
//                first point lies beyond the domain face (inlet: Dirichlet
//                T_in, Y_in ghosts; outlets: zero gradient), not in a solid
// so that all loads of the cell can be issued at once.  A population whose
// source lies beyond an inlet or outlet face takes the rules of Eq. 31, 32
// or the constant-pressure outlet; the code builder leaves out the cells
// where the general form would bounce such a population back or take the
// convective outlet's inner value from the cell itself.
// ---------------------------------------------------------------------------
template <int DIM, typename R>
__device__ __forceinline__ void coded_line(const StepParams<R>& P, const int p[3], long long c, int a, unsigned code,
                                           unsigned faces, LineDesc<R>& L)
{
    // the line's cells (periodic wrap: points beyond a non-periodic face
    // are ghosts, replaced below), without indexing an array by the
    // run-time axis
    const int pa = a == 0 ? p[0] : (a == 1 ? p[1] : p[2]);
    const int n = a == 0 ? P.nx : (a == 1 ? P.ny : P.nz);
    const long long stride = a == 0 ? 1LL : (a == 1 ? (long long)P.nx : (long long)P.nx * P.ny);
    long long raw[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        int qa = pa + j - 2;
        qa = qa < 0 ? qa + n : (qa >= n ? qa - n : qa);
        qa = qa < 0 ? qa + n : (qa >= n ? qa - n : qa);  // extents down to 1
        raw[j] = c + (long long)(qa - pa) * stride;
        L.src[j] = raw[j];
        L.mode[j] = G_DIRECT;
        L.TB[j] = R(0);
    }
    L.near = code != 0;
    const int solid_mode = P.solid_isothermal ? G_DIRICHLET_T : G_NEUMANN;
#pragma unroll
    for (int side = -1; side <= 1; side += 2) {
        const unsigned bits = side < 0 ? (code & 7u) : (code >> 3);
        const int w = (int)(bits & 3u);
        if (!w) continue;
        const bool opp_solid = (bits >> 2) & 1u;
        const bool face = (faces >> (side < 0 ? 0 : 1)) & 1u;
        const int ftype = P.bc[2 * a + (side < 0 ? 0 : 1)];
        const int mode = !face ? solid_mode : (ftype == BC_INLET ? G_INLET : G_NEUMANN);
        const R TB = !face ? P.T_solid : (ftype == BC_INLET ? P.T_in : R(0));
#pragma unroll
        for (int j = 1; j <= 2; ++j) {
            if (j < w) continue;
            const int m = 2 * w - 1 - j;  // mirror offset on this side (Eq. 34)
            L.src[2 + side * j] = m >= 0 ? L.src[2 + side * m] : (opp_solid ? c : raw[2 - side]);
            L.mode[2 + side * j] = mode;
            L.TB[2 + side * j] = TB;
        }
    }
}

template <int DIM, typename S, typename R, bool FACES = false, bool HI1 = false>
__device__ __forceinline__ void cell_step_coded(const StepParams<R>& P, const int p[3], long long c,
                                                unsigned long long code, const S* LBFD_RESTRICT g_in,
                                                S* LBFD_RESTRICT g_out, const S* LBFD_RESTRICT T_in,
                                                S* LBFD_RESTRICT T_out, const S* LBFD_RESTRICT Y_in,
                                                S* LBFD_RESTRICT Y_out)
{
    constexpr int Q = DIM == 2 ? 9 : 27;
    const long long N = P.N;
    const R T0 = R(T_in[c]);
    R Y0[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) Y0[k] = R(Y_in[(long long)k * N + c]);
    const R invW0 = inv_molar_mass(P, Y0);
    const R rho0 = eos(P, T0, invW0);
    // a1: pull, half-way bounce-back (Eq. 28) where the code says solid
    R g[Q];
    {
        const long long plane = (long long)P.nx * P.ny;
        const long long oxm = p[0] == 0 ? P.nx - 1 : -1, oxp = p[0] == P.nx - 1 ? 1 - P.nx : 1;
        const long long oym = p[1] == 0 ? (long long)(P.ny - 1) * P.nx : -(long long)P.nx;
        const long long oyp = p[1] == P.ny - 1 ? (long long)(1 - P.ny) * P.nx : (long long)P.nx;
        long long ozm = 0, ozp = 0;
        if (DIM == 3) {
            ozm = p[2] == 0 ? (P.nz - 1) * plane : -plane;
            ozp = p[2] == P.nz - 1 ? (1 - P.nz) * plane : plane;
        }
        // FACES: the cell's own velocity for the outlet rules, when one of
        // its populations comes from beyond an outlet face
        R uc[3] = {R(0), R(0), R(0)}, mc[3] = {R(0), R(0), R(0)};
        if constexpr (FACES) {
            bool own = false;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const int n = a == 0 ? P.nx : (a == 1 ? P.ny : P.nz);
                const int pa = a == 0 ? p[0] : (a == 1 ? p[1] : p[2]);
                const int lo = P.bc[2 * a], hi = P.bc[2 * a + 1];
                own |= pa == 0 && (lo == BC_OUTLET || lo == BC_OUTLET_PRESSURE);
                own |= pa == n - 1 && (hi == BC_OUTLET || hi == BC_OUTLET_PRESSURE);
            }
            if (own) {
                R gc[Q];
#pragma unroll
                for (int j = 0; j < Q; ++j) gc[j] = R(g_in[(long long)j * N + c]);
                const R inv = fdiv(R(3), rho0);
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    R m = R(0);
#pragma unroll
                    for (int j = 0; j < Q; ++j) {
                        const int cj = ccomp<DIM>(j, a);
                        if (cj != 0) m += R(cj) * gc[j];
                    }
                    mc[a] = m;
                    uc[a] = m * inv;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cx = ccomp<DIM>(i, 0), cy = ccomp<DIM>(i, 1), cz = ccomp<DIM>(i, 2);
            const long long s = c + (cx > 0 ? oxm : (cx < 0 ? oxp : 0)) + (cy > 0 ? oym : (cy < 0 ? oyp : 0)) +
                                (cz > 0 ? ozm : (cz < 0 ? ozp : 0));
            const bool bb = (code >> i) & 1ull;
            if constexpr (FACES) {
                // the face the source x - c_i lies beyond (at most one)
                int f = -1;
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    const int ca = ccomp<DIM>(i, a);
                    const int n = a == 0 ? P.nx : (a == 1 ? P.ny : P.nz);
                    const int sa = (a == 0 ? p[0] : (a == 1 ? p[1] : p[2])) - ca;
                    if (ca > 0 && sa < 0 && P.bc[2 * a] != BC_PERIODIC) f = 2 * a;
                    if (ca < 0 && sa >= n && P.bc[2 * a + 1] != BC_PERIODIC) f = 2 * a + 1;
                }
                if (f >= 0) {
                    const int ib = opposite<DIM>(i);
                    const R gib = R(g_in[(long long)ib * N + c]);
                    const int a = f / 2, t = P.bc[f];
                    const R ci = R(f / 2 == 0 ? cx : (f / 2 == 1 ? cy : cz));
                    if (t == BC_INLET) {  // Eq. 31 applied to g, u_in along the inward normal
                        const R un = (f % 2 == 0) ? P.u_in : -P.u_in;
                        g[i] = gib + R(2) * weight<DIM, R>(i) * P.rho_in * ci * un;
                    } else if (t == BC_OUTLET_PRESSURE) {  // constant P_h = 0: anti-bounce-back
                        R cu = R(0), uu = R(0);
#pragma unroll
                        for (int b = 0; b < DIM; ++b) {
                            cu += R(ccomp<DIM>(i, b)) * uc[b];
                            uu += uc[b] * uc[b];
                        }
                        const R geq_even = weight<DIM, R>(i) * rho0 * (R(1.5) * cu * cu - R(0.5) * uu);
                        g[i] = R(2) * geq_even - gib;
                    } else {  // Eq. 32 in lattice units, outward normal along a
                        const int ns = (f % 2 == 1) ? 1 : -1;
                        const R mom = R(ns) * (a == 0 ? mc[0] : (a == 1 ? mc[1] : mc[2]));
                        const R un = fdiv(R(3) * mom, rho0);
                        const long long st = a == 0 ? 1LL : (a == 1 ? (long long)P.nx : plane);
                        const R inner = R(g_in[(long long)i * N + c - ns * st]);
                        g[i] = (P.cs - un) * inner + (R(1) - P.cs + un) * R(g_in[(long long)i * N + c]);
                    }
                    continue;
                }
            }
            g[i] = R(g_in[bb ? (long long)opposite<DIM>(i) * N + c : (long long)i * N + s]);
        }
    }
    R u[3] = {R(0), R(0), R(0)};
    {
        const R inv = fdiv(R(3), rho0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            R m = R(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int ci = ccomp<DIM>(i, a);
                if (ci) m += R(ci) * g[i];
            }
            u[a] = m * inv;
        }
    }
    FDAccum<R> acc;
    acc.conv_T = acc.diff_T = R(0);
#pragma unroll
    for (int k = 0; k < NSP; ++k) acc.conv_Y[k] = acc.diff_Y[k] = R(0);
    acc.grad_rho[0] = acc.grad_rho[1] = acc.grad_rho[2] = R(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        LineDesc<R> L;
        coded_line<DIM, R>(P, p, c, a, (unsigned)(code >> (32 + 6 * a)) & 63u,
                           FACES ? (unsigned)(code >> (50 + 2 * a)) & 3u : 0u, L);
        R Tl[5], Yl[NSP][5], invWl[5], rhol[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) {  // every point's loads at once
            R Yj[NSP];
            line_point<S, R>(P, L, j, T_in, Y_in, Tl[j], Yj, invWl[j], rhol[j]);
#pragma unroll
            for (int k = 0; k < NSP; ++k) Yl[k][j] = Yj[k];
        }
        fd_axis<R>(P, a, L.near, Tl, Yl, invWl, rhol, u[a], T0, Y0, invW0, rho0, acc);
    }
    const R q = arrhenius(P, T0, pick_species(Y0, P.fuel), pick_species(Y0, P.oxid));
    const R reac_T = P.Q_cp * q;
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
    collide<DIM, R, R, HI1>(P, g, rho0, u, acc.grad_rho, Lam);
#pragma unroll
    for (int i = 0; i < Q; ++i) g_out[(long long)i * N + c] = S(g[i]);
}

}  // namespace lbfd
