// lbfd_params.h -- parameters of one fused step as seen by the kernels,
// already converted to the compute type R and to lattice units.
#pragma once

// Read-only hints of the step's state loads.  A kernel that writes the
// state buffers and reads them back within one launch (the persistent
// step) defines both before including the step headers: no restrict
// qualifier and plain loads, so that no load takes the non-coherent path.
#ifndef LBFD_RESTRICT
#define LBFD_RESTRICT __restrict__
#endif
#ifndef LBFD_LDG
#define LBFD_LDG(p) __ldg(p)
#endif

namespace lbfd {

constexpr int NSP = 5;  // species count the kernels are built for

template <typename R>
struct StepParams {
    int dim, nx, ny, nz;
    long long ncell;  // nx*ny*nz
    long long N;      // stride between SoA planes (ncell rounded up)
    int bc[6];
    R T_wall[6];
    R inv_Wk[NSP];   // 1/W_k
    R yield[NSP];    // nu_k W_k / (-nu_F W_F)
    R a_diff[NSP];   // D_k W_k, D_k = alpha / Le_k
    R a12[NSP];      // a_diff / (12 W_k): the tiles' diffusion on Y_k W with 12x stencils
    R alpha12;       // alpha / 12
    R lam_yield;     // sum_k yield_k / W_k (the reaction's share of Lambda's species sum)
    int fuel, oxid;
    R A_lat;         // A * dt (per step)
    R Ta;            // activation temperature [K]
    R Q_cp;          // Q / cp [K per unit fuel mass fraction]
    double A_lat_d, Ta_d;  // FP64 copies for the mixed-precision Arrhenius
    R T_fp64;
    R omega_s, omega_b, omega_hi;
    R alpha;
    R u_in, T_in, Y_in[NSP], invW_in, rho_in;
    R T_solid;
    int solid_isothermal;
    int poiseuille;
    R epsY, epsT;
    R cs;            // lattice sound speed 1/sqrt(3)
    // face f is a wall that acts exactly like the solid cells (same thermal
    // condition): the wall-aware tiles treat the layer beyond it as solid
    int face_solid[6];
    // curved walls (lbfd_set_curved_walls); curved == 0: staircase walls
    int curved;
    const int* link_row;    // [ncell] row of link_q, -1 when no link is cut
    const double* link_q;   // [rows][Q] wall distance fraction of cut links, < 0: half-way
    const int* ghost_row;   // [ncell] ghost index of a solid cell, -1 if none
    const R* gval;          // [nghost][GHOST_VALUES] ghost values of the current step
};

// values stored per ghost node: T, Y_k, 1/W, X_k, rho
constexpr int GHOST_VALUES = 3 + 2 * NSP;

}  // namespace lbfd
