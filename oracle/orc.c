/*
 * orc.c -- plain, slow FP64 CPU oracle for one coupled time step of the
 * hybrid low-Mach lattice Boltzmann / finite-difference solver of
 * Hosseini & Thevenin, "Towards pore-scale simulation of combustion in
 * porous media using a low-Mach hybrid lattice Boltzmann/finite difference
 * solver" (arXiv 2304.05657).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the package smoke check and the
 * CPU-baseline leg of bench.py load this file's shared object; the CUDA
 * library never does, and this file includes no header of it.  Every
 * constant here (lattice, weights, stencil coefficients) is written out
 * again on purpose.
 *
 * Equation numbers follow the paper's order of display:
 *   Eq. 1 species balance, Eq. 2 diffusion velocity with correction,
 *   Eq. 5 hydrodynamic-pressure closure, Eq. 6 Lambda, Eq. 7 energy,
 *   Eq. 8 LB equation, Eq. 9 source Xi, Eq. 10 f^eq, Eq. 12 g^eq,
 *   Eq. 13 moments (P_h, rho u), Eq. 14 post-collision g*, Eq. 15 MRT
 *   relaxation, Eq. 18 omega_s, Eq. 19 pre-conditioning, Eq. 21 central
 *   moments, Eq. 22 forward cumulants, Eq. 23 relaxation of cumulants,
 *   Eq. 24 backward cumulants, Eq. 26 corrected convection (Sec. II.D),
 *   Eq. 28 half-way bounce-back, Eq. 31 inlet, Eq. 32 outlet,
 *   Eq. 34 ghost node (Sec. III.B).
 *
 * Where the paper is silent or garbled, this file takes the following
 * readings (each also stated where it is used):
 *   - order of one step: pull-stream with boundary rules; u from the pulled
 *     populations; FD right-hand side from state n and u^n; Lambda^n from
 *     the non-convective part of that right-hand side; collision with
 *     rho^n, grad rho^n, Lambda^n, P_h^n.  The stored populations are
 *     post-collision.
 *   - omega_s = 1 / (nu/(cs^2 dt) + 1/2): Eq. 18 prints tau, not omega.
 *   - relaxation (Eq. 15, 23): K*_j = Keq_j + (1 - omega_j)(K_j - Keq_j),
 *     Keq from the same transform applied to g^eq/(rho cs^2) about the same
 *     u; orders 0 and 1 are carried unchanged.  Second order: deviatoric
 *     parts at omega_s, trace at omega_bulk; orders >= 3 at omega_hi.
 *   - cumulant formulas: the index typos of Eq. 22 are fixed by permutation
 *     symmetry (Pi_xx Pi_yy in K_xxyy, Pi_zz Pi_xyy in K_xyyzz, Pi_zz Pi_xxyy
 *     in K_xxyyzz) and the backward map is the exact algebraic inverse of
 *     the forward one, not Eq. 24 as printed.
 *   - outlet (Eq. 32): g_i(x,t+1) = (cs - u.n) g*_i(x-n,t)
 *     + (1 - cs + u.n) g*_i(x,t) in lattice units, u.n from the first
 *     moment of g*(x) divided by rho(x) of the current scalar state.
 *   - inlet (Eq. 31) applied to g: g_i = g*_ibar + 2 w_i rho_in u_in.c_i.
 *   - constant-pressure outlet (the outlet of the validation cases,
 *     Sec. IV.A and IV.C): anti-bounce-back,
 *     g_i = -g*_ibar + 2 [w_i P_out + w_i rho ((c_i.u)^2/(2 cs^2) - u.u/2)]
 *     with P_out = 0 and rho, u of the boundary cell (u from g*), i.e. twice
 *     the even part of g^eq (Eq. 12) at the outlet pressure.  Eq. 32 alone
 *     leaves the pressure level free to drift in this pressure-based scheme.
 *   - transport: constant kinematic nu, alpha = nu/Pr, D_k = alpha/Le_k;
 *     fluxes in expanded form with 4th-order central first and second
 *     derivatives; equal constant c_p for all species.
 *   - reaction: single-step global, rate per unit mass
 *     q = A dt max(Y_F,0) max(Y_O,0) exp(-Ta/T).
 *   - EOS: rho = (T_in/T)(W/W_in), so rho = 1 at the inlet state.
 *   - ghosts per axis line; the ghost at distance j from the wall mirrors
 *     the fluid point at distance j-1 on the other side; if that point is
 *     not fluid the centre cell is used.  Density at ghost points is
 *     reconstructed directly (Dirichlet rule on rho with rho_B = EOS(T_B,Y)),
 *     following the paper's note on ghost-node properties.
 *   - convection: WENO3 (Jiang-Shu, r = 2) upwinded on the sign of the
 *     local velocity component; centred 2nd order on an axis when a point
 *     of the +-2 stencil on that axis is not a fluid cell of the domain.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXSP 8

enum { ORC_PERIODIC = 0, ORC_WALL_ADIABATIC = 1, ORC_WALL_ISOTHERMAL = 2,
       ORC_INLET = 3, ORC_OUTLET = 4, ORC_OUTLET_PRESSURE = 5 };
/* classification of a point next to a fluid cell */
enum { PT_FLUID = 0, PT_SOLID = 16 };

typedef struct {
    int dim, nx, ny, nz;
    int bc[6];                 /* faces -x,+x,-y,+y,-z,+z */
    double T_wall[6];
    int n_species;
    double W[ORC_MAXSP];       /* molar masses */
    double nu_stoich[ORC_MAXSP];
    double Le[ORC_MAXSP];
    int fuel, oxid;
    double A, Ta, Q, cp, dt;   /* A [1/s], Ta [K], Q [J/kg fuel], cp [J/kg/K], dt [s] */
    double nu, Pr, omega_bulk, omega_hi;  /* omega_bulk <= 0 means omega_s */
    double u_in, T_in, Y_in[ORC_MAXSP];
    double T_solid;
    int solid_isothermal;
    int poiseuille_inlet;
    double weno_eps;           /* species; temperature uses weno_eps * T_in^2 */
} orc_setup;

typedef struct {
    orc_setup s;
    int Q, nsp;
    long N;
    int c[27][3];
    double w[27];
    int opp[27];
    double *g, *T, *Y;         /* state: g post-collision [Q][N], T [N], Y [nsp][N] */
    double *gn, *Tn, *Yn;      /* next state */
    unsigned char *solid;
    double cs2, cs, omega_s, omega_b, alpha, D[ORC_MAXSP], A_lat;
    double invW_in, rho_in;
    long steps;
    /* curved walls (optional) */
    int curved, nprims;
    double *prims;      /* 5 per primitive */
    double *linkq;      /* [Q][N] wall distance fraction of cut links, -1 elsewhere */
    long *ghost_of;     /* [N] ghost index of a solid cell, -1 if none */
    long nghost;
    long *gh_start;     /* [nghost+1] CSR of the image-point neighbours */
    long *gh_idx;
    double *gh_w;
    double *gh_B;       /* [nghost][3] boundary points */
} orc_sim;

/* one point of an FD line: primitive and derived values */
typedef struct {
    double T, Y[ORC_MAXSP], invW, X[ORC_MAXSP], rho;
} orc_pt;

/* ------------------------------------------------------------------ */
/* lattice                                                              */
/* ------------------------------------------------------------------ */

/* D2Q9 / D3Q27 as tensor products of D1Q3 {-1,0,1} with weights
 * {1/6, 2/3, 1/6}; population index i = (cx+1) + 3(cy+1) + 9(cz+1). */
static void lattice_init(orc_sim *S)
{
    const double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
    int i = 0;
    S->Q = (S->s.dim == 2) ? 9 : 27;
    for (int cz = -1; cz <= 1; ++cz) {
        if (S->s.dim == 2 && cz != 0) continue;
        for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
                int idx = (cx + 1) + 3 * (cy + 1) + (S->s.dim == 3 ? 9 * (cz + 1) : 0);
                S->c[idx][0] = cx;
                S->c[idx][1] = cy;
                S->c[idx][2] = cz;
                S->w[idx] = w1[cx + 1] * w1[cy + 1] * (S->s.dim == 3 ? w1[cz + 1] : 1.0);
                ++i;
            }
    }
    for (int a = 0; a < S->Q; ++a)
        for (int b = 0; b < S->Q; ++b)
            if (S->c[a][0] == -S->c[b][0] && S->c[a][1] == -S->c[b][1] &&
                S->c[a][2] == -S->c[b][2])
                S->opp[a] = b;
    (void)i;
}

/* ------------------------------------------------------------------ */
/* thermochemistry                                                      */
/* ------------------------------------------------------------------ */

static double inv_molar_mass(const orc_sim *S, const double *Y)
{
    double s = 0.0;
    for (int k = 0; k < S->nsp; ++k) s += Y[k] / S->s.W[k];
    return s;
}

/* ideal-gas EOS at constant P_0 (Sec. II.A), scaled so that rho(T_in, Y_in) = 1 */
static double eos_rho(const orc_sim *S, double T, double invW)
{
    return (S->s.T_in / T) * (S->invW_in / invW);
}

/* single-step rate per unit mass of fuel consumed, per time step */
static double rate_q(const orc_sim *S, double T, const double *Y)
{
    double yf = Y[S->s.fuel] > 0.0 ? Y[S->s.fuel] : 0.0;
    double yo = Y[S->s.oxid] > 0.0 ? Y[S->s.oxid] : 0.0;
    return S->A_lat * yf * yo * exp(-S->s.Ta / T);
}

/* mass yield of species k per unit mass of fuel consumed: nu_k W_k / (-nu_F W_F) */
static double yield(const orc_sim *S, int k)
{
    return S->s.nu_stoich[k] * S->s.W[k] / (-S->s.nu_stoich[S->s.fuel] * S->s.W[S->s.fuel]);
}

/* ------------------------------------------------------------------ */
/* geometry helpers                                                     */
/* ------------------------------------------------------------------ */

static int extent(const orc_sim *S, int a)
{
    return a == 0 ? S->s.nx : (a == 1 ? S->s.ny : S->s.nz);
}

static long cell_index(const orc_sim *S, const int p[3])
{
    return (long)p[0] + (long)S->s.nx * ((long)p[1] + (long)S->s.ny * (long)p[2]);
}

/* Classify position p (may lie outside the box along one axis).  Returns
 * PT_FLUID with *idx set (periodic axes wrapped), PT_SOLID for a solid cell,
 * or the boundary type of the face that is crossed, with *face set. */
static int classify(const orc_sim *S, const int pin[3], long *idx, int *face)
{
    int p[3] = {pin[0], pin[1], pin[2]};
    int wall = -1;
    for (int a = 0; a < S->s.dim; ++a) {
        int n = extent(S, a);
        int f = -1;
        if (p[a] < 0) f = 2 * a;
        else if (p[a] >= n) f = 2 * a + 1;
        if (f < 0) continue;
        if (S->s.bc[f] == ORC_PERIODIC) {
            p[a] = ((p[a] % n) + n) % n;
        } else if (wall < 0) {
            wall = f;
        }
    }
    if (wall >= 0) {
        *face = wall;
        return S->s.bc[wall];
    }
    *idx = cell_index(S, p);
    if (S->solid[*idx]) return PT_SOLID;
    return PT_FLUID;
}

/* ------------------------------------------------------------------ */
/* FD line points and ghosts (Sec. III.B, Eq. 34)                        */
/* ------------------------------------------------------------------ */

static void fluid_pt(const orc_sim *S, long idx, orc_pt *pt)
{
    pt->T = S->T[idx];
    for (int k = 0; k < S->nsp; ++k) pt->Y[k] = S->Y[(long)k * S->N + idx];
    pt->invW = inv_molar_mass(S, pt->Y);
    for (int k = 0; k < S->nsp; ++k) pt->X[k] = pt->Y[k] / (S->s.W[k] * pt->invW);
    pt->rho = eos_rho(S, pt->T, pt->invW);
}

/* ghost value from its mirror point m: phi_G = 2 phi_B - phi_I (Dirichlet)
 * or phi_G = phi_I (Neumann). type is PT_SOLID or a face boundary type. */
static void ghost_pt(const orc_sim *S, int type, int face, const orc_pt *m, orc_pt *g)
{
    int dirichlet_T = 0, dirichlet_Y = 0;
    double TB = 0.0;
    const double *YB = m->Y;
    if (type == PT_SOLID) {
        if (S->s.solid_isothermal) { dirichlet_T = 1; TB = S->s.T_solid; }
    } else if (type == ORC_WALL_ISOTHERMAL) {
        dirichlet_T = 1; TB = S->s.T_wall[face];
    } else if (type == ORC_INLET) {
        dirichlet_T = 1; TB = S->s.T_in;
        dirichlet_Y = 1; YB = S->s.Y_in;
    }
    g->T = dirichlet_T ? 2.0 * TB - m->T : m->T;
    for (int k = 0; k < S->nsp; ++k)
        g->Y[k] = dirichlet_Y ? 2.0 * S->s.Y_in[k] - m->Y[k] : m->Y[k];
    g->invW = inv_molar_mass(S, g->Y);
    for (int k = 0; k < S->nsp; ++k) g->X[k] = g->Y[k] / (S->s.W[k] * g->invW);
    if (dirichlet_T) {
        double rhoB = eos_rho(S, TB, inv_molar_mass(S, YB));
        g->rho = 2.0 * rhoB - m->rho;
    } else {
        g->rho = m->rho;
    }
}

/* ------------------------------------------------------------------ */
/* curved walls: interpolated bounce-back (Eq. 29-30) and image-point   */
/* ghosts with Shepard inverse-distance weighting (Eq. 34-38)           */
/* ------------------------------------------------------------------ */

/* Primitive k: prim[5k] = type (0: sphere/circle, 1: half-space), then
 * sphere: centre (p0, p1, p2), radius p3, solid inside;
 * half-space: unit normal (p0, p1, p2) pointing into the solid, offset p3,
 * solid where n.x > p3.  Cell (x,y,z) has its centre at (x+.5, y+.5, z+.5);
 * in 2-D the z components are ignored. */

static void cell_centre(const orc_sim *S, const int p[3], double c[3])
{
    c[0] = p[0] + 0.5;
    c[1] = p[1] + 0.5;
    c[2] = S->s.dim == 3 ? p[2] + 0.5 : 0.0;
}

static int prim_inside(const orc_sim *S, int k, const double x[3])
{
    const double *P = &S->prims[5 * k];
    if ((int)P[0] == 0) {
        double d2 = 0.0;
        for (int a = 0; a < S->s.dim; ++a) d2 += (x[a] - P[1 + a]) * (x[a] - P[1 + a]);
        return d2 < P[4] * P[4];
    }
    double s = 0.0;
    for (int a = 0; a < S->s.dim; ++a) s += P[1 + a] * x[a];
    return s > P[4];
}

/* wall distance fraction of the link from centre x along -c_i (Eq. 30):
 * the smallest t in (0, 1] where x - t c_i enters a primitive; -1 if none */
static double link_q(const orc_sim *S, const double x[3], int i)
{
    double best = -1.0;
    double v[3] = {-(double)S->c[i][0], -(double)S->c[i][1], -(double)S->c[i][2]};
    for (int k = 0; k < S->nprims; ++k) {
        const double *P = &S->prims[5 * k];
        double t = -1.0;
        if ((int)P[0] == 0) {
            double d[3] = {0, 0, 0}, vv = 0.0, dv = 0.0, dd = 0.0;
            for (int a = 0; a < S->s.dim; ++a) {
                d[a] = x[a] - P[1 + a];
                vv += v[a] * v[a];
                dv += d[a] * v[a];
                dd += d[a] * d[a];
            }
            double disc = dv * dv - vv * (dd - P[4] * P[4]);
            if (disc >= 0.0 && vv > 0.0) t = (-dv - sqrt(disc)) / vv;
        } else {
            double nv = 0.0, nx = 0.0;
            for (int a = 0; a < S->s.dim; ++a) {
                nv += P[1 + a] * v[a];
                nx += P[1 + a] * x[a];
            }
            if (nv > 0.0) t = (P[4] - nx) / nv;
        }
        if (t > 0.0 && t <= 1.0 && (best < 0.0 || t < best)) best = t;
    }
    return best;
}

/* closest boundary point of the primitive that contains x and whose
 * boundary is nearest; returns 0 when x is in no primitive */
static int closest_boundary(const orc_sim *S, const double x[3], double B[3])
{
    double bestd = INFINITY;
    int found = 0;
    for (int k = 0; k < S->nprims; ++k) {
        if (!prim_inside(S, k, x)) continue;
        const double *P = &S->prims[5 * k];
        double cand[3] = {0, 0, 0}, dist;
        if ((int)P[0] == 0) {
            double d[3] = {0, 0, 0}, n = 0.0;
            for (int a = 0; a < S->s.dim; ++a) {
                d[a] = x[a] - P[1 + a];
                n += d[a] * d[a];
            }
            n = sqrt(n);
            if (n < 1e-12) continue;
            for (int a = 0; a < S->s.dim; ++a) cand[a] = P[1 + a] + P[4] * d[a] / n;
            dist = P[4] - n;
        } else {
            double s = 0.0;
            for (int a = 0; a < S->s.dim; ++a) s += P[1 + a] * x[a];
            dist = s - P[4];
            for (int a = 0; a < S->s.dim; ++a) cand[a] = x[a] - dist * P[1 + a];
        }
        if (dist < bestd) {
            bestd = dist;
            for (int a = 0; a < 3; ++a) B[a] = cand[a];
            found = 1;
        }
    }
    return found;
}

/* Build the link and ghost tables from the primitives and the mask. */
static void build_curved(orc_sim *S)
{
    long N = S->N;
    free(S->linkq);
    free(S->ghost_of);
    free(S->gh_start);
    free(S->gh_idx);
    free(S->gh_w);
    S->linkq = (double *)malloc(sizeof(double) * (size_t)S->Q * N);
    S->ghost_of = (long *)malloc(sizeof(long) * (size_t)N);
    for (long c = 0; c < (long)S->Q * N; ++c) S->linkq[c] = -1.0;
    for (long c = 0; c < N; ++c) S->ghost_of[c] = -1;
    int nz = S->s.nz;
    /* links: fluid cell, pulled population whose source is a solid cell */
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < S->s.ny; ++y)
            for (int x = 0; x < S->s.nx; ++x) {
                int p[3] = {x, y, z};
                long c = cell_index(S, p);
                if (S->solid[c]) continue;
                double xc[3];
                cell_centre(S, p, xc);
                for (int i = 0; i < S->Q; ++i) {
                    int q[3] = {x - S->c[i][0], y - S->c[i][1], z - S->c[i][2]};
                    long idx;
                    int face = -1;
                    if (classify(S, q, &idx, &face) != PT_SOLID) continue;
                    S->linkq[(long)i * N + c] = link_q(S, xc, i);
                }
            }
    /* ghosts: solid cells within two cells of a fluid cell along an axis */
    long ng = 0, cap = 1024, nnz = 0, ncap = 16384;
    S->gh_start = (long *)malloc(sizeof(long) * (size_t)(cap + 1));
    S->gh_idx = (long *)malloc(sizeof(long) * (size_t)ncap);
    S->gh_w = (double *)malloc(sizeof(double) * (size_t)ncap);
    S->gh_B = (double *)realloc(S->gh_B, sizeof(double) * 3 * (size_t)cap);
    S->gh_start[0] = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < S->s.ny; ++y)
            for (int x = 0; x < S->s.nx; ++x) {
                int p[3] = {x, y, z};
                long c = cell_index(S, p);
                if (!S->solid[c]) continue;
                int near = 0;
                for (int a = 0; a < S->s.dim && !near; ++a)
                    for (int d = -2; d <= 2 && !near; ++d) {
                        if (!d) continue;
                        int q[3] = {x, y, z};
                        q[a] += d;
                        long idx;
                        int face = -1;
                        if (classify(S, q, &idx, &face) == PT_FLUID) near = 1;
                    }
                if (!near) continue;
                double xc[3], B[3], I[3] = {0, 0, 0};
                cell_centre(S, p, xc);
                if (!closest_boundary(S, xc, B)) continue;
                for (int a = 0; a < S->s.dim; ++a) I[a] = 2.0 * B[a] - xc[a];
                /* fluid cells within 4 cells of the image point (Eq. 38) */
                long first = nnz;
                int exact = -1;
                int lo[3], hi[3];
                for (int a = 0; a < 3; ++a) {
                    if (a >= S->s.dim) { lo[a] = hi[a] = 0; continue; }
                    lo[a] = (int)floor(I[a] - 0.5 - 4.0) - 1;
                    hi[a] = (int)ceil(I[a] - 0.5 + 4.0) + 1;
                    if (lo[a] < 0) lo[a] = 0;
                    if (hi[a] > extent(S, a) - 1) hi[a] = extent(S, a) - 1;
                }
                double wsum = 0.0;
                for (int zz = lo[2]; zz <= hi[2]; ++zz)
                    for (int yy = lo[1]; yy <= hi[1]; ++yy)
                        for (int xx = lo[0]; xx <= hi[0]; ++xx) {
                            int r[3] = {xx, yy, zz};
                            long j = cell_index(S, r);
                            if (S->solid[j]) continue;
                            double rc[3], d2 = 0.0;
                            cell_centre(S, r, rc);
                            for (int a = 0; a < S->s.dim; ++a) d2 += (rc[a] - I[a]) * (rc[a] - I[a]);
                            if (d2 > 16.0) continue;
                            if (nnz >= ncap) {
                                ncap *= 2;
                                S->gh_idx = (long *)realloc(S->gh_idx, sizeof(long) * (size_t)ncap);
                                S->gh_w = (double *)realloc(S->gh_w, sizeof(double) * (size_t)ncap);
                            }
                            if (d2 < 1e-18) exact = (int)(nnz - first);
                            S->gh_idx[nnz] = j;
                            S->gh_w[nnz] = d2 < 1e-18 ? 0.0 : 1.0 / d2;   /* p = 2 (Eq. 36) */
                            wsum += S->gh_w[nnz];
                            ++nnz;
                        }
                if (nnz == first) continue;  /* no fluid around the image: staircase */
                for (long e = first; e < nnz; ++e) {
                    if (exact >= 0) S->gh_w[e] = (e - first == exact) ? 1.0 : 0.0;
                    else S->gh_w[e] /= wsum;                               /* Eq. 37 */
                }
                if (ng >= cap) {
                    cap *= 2;
                    S->gh_start = (long *)realloc(S->gh_start, sizeof(long) * (size_t)(cap + 1));
                    S->gh_B = (double *)realloc(S->gh_B, sizeof(double) * 3 * (size_t)cap);
                }
                for (int a = 0; a < 3; ++a) S->gh_B[3 * ng + a] = B[a];
                S->ghost_of[c] = ng;
                S->gh_start[ng + 1] = nnz;
                ++ng;
            }
    S->nghost = ng;
}

/* Shepard value of the image point of ghost k: T, Y, rho (Eq. 35) */
static void ghost_image(const orc_sim *S, long k, orc_pt *I)
{
    I->T = 0.0;
    I->rho = 0.0;
    for (int s = 0; s < S->nsp; ++s) I->Y[s] = 0.0;
    for (long e = S->gh_start[k]; e < S->gh_start[k + 1]; ++e) {
        orc_pt f;
        fluid_pt(S, S->gh_idx[e], &f);
        double w = S->gh_w[e];
        I->T += w * f.T;
        I->rho += w * f.rho;   /* the property itself is reconstructed */
        for (int s = 0; s < S->nsp; ++s) I->Y[s] += w * f.Y[s];
    }
}

/* ghost node value (Eq. 34) of solid cell with ghost index k */
static void curved_ghost_pt(const orc_sim *S, long k, orc_pt *g)
{
    orc_pt I;
    ghost_image(S, k, &I);
    for (int s = 0; s < S->nsp; ++s) g->Y[s] = I.Y[s];            /* Neumann */
    g->invW = inv_molar_mass(S, g->Y);
    for (int s = 0; s < S->nsp; ++s) g->X[s] = g->Y[s] / (S->s.W[s] * g->invW);
    if (S->s.solid_isothermal) {
        double TB = S->s.T_solid;
        g->T = 2.0 * TB - I.T;
        g->rho = 2.0 * eos_rho(S, TB, inv_molar_mass(S, I.Y)) - I.rho;
    } else {
        g->T = I.T;
        g->rho = I.rho;
    }
}

/* Build the 5-point line (offsets -2..2) through cell p along axis a.
 * Returns 1 when a point of the line is not a fluid cell of the domain. */
static int build_line(const orc_sim *S, const int p[3], long cidx, int a, orc_pt line[5])
{
    int near = 0;
    fluid_pt(S, cidx, &line[2]);
    for (int side = -1; side <= 1; side += 2) {
        int w = 0, wtype = 0, wface = -1;
        for (int j = 1; j <= 2; ++j) {
            int q[3] = {p[0], p[1], p[2]};
            long idx;
            int face = -1;
            q[a] += side * j;
            int t = classify(S, q, &idx, &face);
            if (t == PT_FLUID) {
                fluid_pt(S, idx, &line[2 + side * j]);
            } else {
                w = j; wtype = t; wface = face;
                break;
            }
        }
        if (!w) continue;
        near = 1;
        for (int j = w; j <= 2; ++j) {
            if (S->curved) {  /* a solid cell with an image-point ghost (Eq. 34-38) */
                int q[3] = {p[0], p[1], p[2]};
                long idx;
                int face = -1;
                q[a] += side * j;
                if (classify(S, q, &idx, &face) == PT_SOLID && S->ghost_of[idx] >= 0) {
                    curved_ghost_pt(S, S->ghost_of[idx], &line[2 + side * j]);
                    continue;
                }
            }
            int m = 2 * w - 1 - j;  /* mirror offset on this side (may be -1) */
            orc_pt mpt;
            if (m >= 0) {
                mpt = line[2 + side * m];
            } else {
                int q[3] = {p[0], p[1], p[2]};
                long idx;
                int face = -1;
                q[a] -= side;  /* one step on the opposite side */
                if (classify(S, q, &idx, &face) == PT_FLUID) fluid_pt(S, idx, &mpt);
                else mpt = line[2];
            }
            ghost_pt(S, wtype, wface, &mpt, &line[2 + side * j]);
        }
    }
    return near;
}

/* ------------------------------------------------------------------ */
/* FD operators (Sec. II.D)                                              */
/* ------------------------------------------------------------------ */

/* 4th-order central first derivative, unit spacing */
double orc_d1(const double v[5])
{
    return (v[0] - 8.0 * v[1] + 8.0 * v[3] - v[4]) / 12.0;
}

/* 4th-order central second derivative, unit spacing */
double orc_d2(const double v[5])
{
    return (-v[0] + 16.0 * v[1] - 30.0 * v[2] + 16.0 * v[3] - v[4]) / 12.0;
}

/* centred 2nd-order first derivative */
double orc_c2(const double v[5])
{
    return 0.5 * (v[3] - v[1]);
}

/* WENO3 face value (Jiang-Shu, r = 2).  a: far upwind, b: upwind cell,
 * c: downwind cell of the face. */
static double weno3_face(double a, double b, double c, double eps)
{
    double q0 = -0.5 * a + 1.5 * b;
    double q1 = 0.5 * b + 0.5 * c;
    double b0 = (b - a) * (b - a);
    double b1 = (c - b) * (c - b);
    double a0 = (1.0 / 3.0) / ((eps + b0) * (eps + b0));
    double a1 = (2.0 / 3.0) / ((eps + b1) * (eps + b1));
    return (a0 * q0 + a1 * q1) / (a0 + a1);
}

/* WENO3 approximation of d(phi)/dx at the centre of v[0..4], upwinded
 * for the sign of the advecting velocity u (u = 0 takes the u > 0 branch). */
double orc_weno3(const double v[5], double u, double eps)
{
    double fp, fm;
    if (u >= 0.0) {
        fp = weno3_face(v[1], v[2], v[3], eps);
        fm = weno3_face(v[0], v[1], v[2], eps);
    } else {
        fp = weno3_face(v[4], v[3], v[2], eps);
        fm = weno3_face(v[3], v[2], v[1], eps);
    }
    return fp - fm;
}

/* ------------------------------------------------------------------ */
/* central moments and cumulants (Sec. II.C, Eq. 21, 22, 24)              */
/* ------------------------------------------------------------------ */

static double ipow(double x, int p)
{
    double r = 1.0;
    for (int k = 0; k < p; ++k) r *= x;
    return r;
}

/* moment index j = p + 3q + 9r, exponents p, q, r in {0,1,2} */
static void moment_exponents(int j, int *p, int *q, int *r)
{
    *p = j % 3;
    *q = (j / 3) % 3;
    *r = j / 9;
}

/* Eq. 21: Pi_j = sum_i (c_ix-u_x)^p (c_iy-u_y)^q (c_iz-u_z)^r f_i */
static void central_moments(const orc_sim *S, const double *f, const double u[3], double *Pi)
{
    for (int j = 0; j < S->Q; ++j) {
        int p, q, r;
        moment_exponents(j, &p, &q, &r);
        double s = 0.0;
        for (int i = 0; i < S->Q; ++i)
            s += ipow(S->c[i][0] - u[0], p) * ipow(S->c[i][1] - u[1], q) *
                 ipow(S->c[i][2] - u[2], r) * f[i];
        Pi[j] = s;
    }
}

/* Inverse of Eq. 21: solve the Q x Q linear system by Gaussian elimination
 * with partial pivoting. */
static void central_moments_inverse(const orc_sim *S, const double *Pi, const double u[3], double *f)
{
    int Q = S->Q;
    double M[27][28];
    for (int j = 0; j < Q; ++j) {
        int p, q, r;
        moment_exponents(j, &p, &q, &r);
        for (int i = 0; i < Q; ++i)
            M[j][i] = ipow(S->c[i][0] - u[0], p) * ipow(S->c[i][1] - u[1], q) *
                      ipow(S->c[i][2] - u[2], r);
        M[j][Q] = Pi[j];
    }
    for (int col = 0; col < Q; ++col) {
        int piv = col;
        for (int r = col + 1; r < Q; ++r)
            if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
        if (piv != col)
            for (int k = 0; k <= Q; ++k) {
                double t = M[col][k]; M[col][k] = M[piv][k]; M[piv][k] = t;
            }
        for (int r = col + 1; r < Q; ++r) {
            double fac = M[r][col] / M[col][col];
            for (int k = col; k <= Q; ++k) M[r][k] -= fac * M[col][k];
        }
    }
    for (int r = Q - 1; r >= 0; --r) {
        double s = M[r][Q];
        for (int k = r + 1; k < Q; ++k) s -= M[r][k] * f[k];
        f[r] = s / M[r][r];
    }
}

#define MI(p, q, r) ((p) + 3 * (q) + 9 * (r))

/* Eq. 22, with the index typos fixed by permutation symmetry.  Orders <= 3
 * are the central moments themselves. */
void orc_cumulants(int dim, const double *Pi, double *K)
{
    int Q = dim == 2 ? 9 : 27;
    for (int j = 0; j < Q; ++j) K[j] = Pi[j];
#define M_(p, q, r) Pi[MI(p, q, r)]
    if (dim == 2) {
        K[MI(2, 2, 0)] = M_(2, 2, 0) - M_(2, 0, 0) * M_(0, 2, 0) - 2.0 * M_(1, 1, 0) * M_(1, 1, 0);
        return;
    }
    /* fourth order: xxyy class */
    K[MI(2, 2, 0)] = M_(2, 2, 0) - M_(2, 0, 0) * M_(0, 2, 0) - 2.0 * M_(1, 1, 0) * M_(1, 1, 0);
    K[MI(2, 0, 2)] = M_(2, 0, 2) - M_(2, 0, 0) * M_(0, 0, 2) - 2.0 * M_(1, 0, 1) * M_(1, 0, 1);
    K[MI(0, 2, 2)] = M_(0, 2, 2) - M_(0, 2, 0) * M_(0, 0, 2) - 2.0 * M_(0, 1, 1) * M_(0, 1, 1);
    /* fourth order: xxyz class */
    K[MI(2, 1, 1)] = M_(2, 1, 1) - M_(2, 0, 0) * M_(0, 1, 1) - 2.0 * M_(1, 1, 0) * M_(1, 0, 1);
    K[MI(1, 2, 1)] = M_(1, 2, 1) - M_(0, 2, 0) * M_(1, 0, 1) - 2.0 * M_(1, 1, 0) * M_(0, 1, 1);
    K[MI(1, 1, 2)] = M_(1, 1, 2) - M_(0, 0, 2) * M_(1, 1, 0) - 2.0 * M_(1, 0, 1) * M_(0, 1, 1);
    /* fifth order: xyyzz class */
    K[MI(1, 2, 2)] = M_(1, 2, 2) - M_(0, 0, 2) * M_(1, 2, 0) - M_(0, 2, 0) * M_(1, 0, 2)
                   - 4.0 * M_(0, 1, 1) * M_(1, 1, 1) - 2.0 * M_(1, 0, 1) * M_(0, 2, 1)
                   - 2.0 * M_(1, 1, 0) * M_(0, 1, 2);
    K[MI(2, 1, 2)] = M_(2, 1, 2) - M_(0, 0, 2) * M_(2, 1, 0) - M_(2, 0, 0) * M_(0, 1, 2)
                   - 4.0 * M_(1, 0, 1) * M_(1, 1, 1) - 2.0 * M_(0, 1, 1) * M_(2, 0, 1)
                   - 2.0 * M_(1, 1, 0) * M_(1, 0, 2);
    K[MI(2, 2, 1)] = M_(2, 2, 1) - M_(2, 0, 0) * M_(0, 2, 1) - M_(0, 2, 0) * M_(2, 0, 1)
                   - 4.0 * M_(1, 1, 0) * M_(1, 1, 1) - 2.0 * M_(1, 0, 1) * M_(1, 2, 0)
                   - 2.0 * M_(0, 1, 1) * M_(2, 1, 0);
    /* sixth order */
    K[MI(2, 2, 2)] = M_(2, 2, 2)
        - M_(2, 0, 0) * M_(0, 2, 2) - M_(0, 2, 0) * M_(2, 0, 2) - M_(0, 0, 2) * M_(2, 2, 0)
        - 4.0 * M_(1, 1, 0) * M_(1, 1, 2) - 4.0 * M_(1, 0, 1) * M_(1, 2, 1)
        - 4.0 * M_(0, 1, 1) * M_(2, 1, 1)
        - 4.0 * M_(1, 1, 1) * M_(1, 1, 1)
        - 2.0 * M_(2, 1, 0) * M_(0, 1, 2) - 2.0 * M_(2, 0, 1) * M_(0, 2, 1)
        - 2.0 * M_(1, 2, 0) * M_(1, 0, 2)
        + 2.0 * M_(2, 0, 0) * M_(0, 2, 0) * M_(0, 0, 2)
        + 4.0 * M_(2, 0, 0) * M_(0, 1, 1) * M_(0, 1, 1)
        + 4.0 * M_(0, 2, 0) * M_(1, 0, 1) * M_(1, 0, 1)
        + 4.0 * M_(0, 0, 2) * M_(1, 1, 0) * M_(1, 1, 0)
        + 16.0 * M_(1, 1, 0) * M_(1, 0, 1) * M_(0, 1, 1);
#undef M_
}

/* Exact inverse of orc_cumulants (stands in for Eq. 24): central moments of
 * order <= 3 equal the cumulants; higher orders are rebuilt from the
 * cumulant and the already rebuilt lower-order central moments. */
void orc_cumulants_inverse(int dim, const double *K, double *Pi)
{
    int Q = dim == 2 ? 9 : 27;
    for (int j = 0; j < Q; ++j) Pi[j] = K[j];
#define M_(p, q, r) Pi[MI(p, q, r)]
    if (dim == 2) {
        Pi[MI(2, 2, 0)] = K[MI(2, 2, 0)] + M_(2, 0, 0) * M_(0, 2, 0) + 2.0 * M_(1, 1, 0) * M_(1, 1, 0);
        return;
    }
    Pi[MI(2, 2, 0)] = K[MI(2, 2, 0)] + M_(2, 0, 0) * M_(0, 2, 0) + 2.0 * M_(1, 1, 0) * M_(1, 1, 0);
    Pi[MI(2, 0, 2)] = K[MI(2, 0, 2)] + M_(2, 0, 0) * M_(0, 0, 2) + 2.0 * M_(1, 0, 1) * M_(1, 0, 1);
    Pi[MI(0, 2, 2)] = K[MI(0, 2, 2)] + M_(0, 2, 0) * M_(0, 0, 2) + 2.0 * M_(0, 1, 1) * M_(0, 1, 1);
    Pi[MI(2, 1, 1)] = K[MI(2, 1, 1)] + M_(2, 0, 0) * M_(0, 1, 1) + 2.0 * M_(1, 1, 0) * M_(1, 0, 1);
    Pi[MI(1, 2, 1)] = K[MI(1, 2, 1)] + M_(0, 2, 0) * M_(1, 0, 1) + 2.0 * M_(1, 1, 0) * M_(0, 1, 1);
    Pi[MI(1, 1, 2)] = K[MI(1, 1, 2)] + M_(0, 0, 2) * M_(1, 1, 0) + 2.0 * M_(1, 0, 1) * M_(0, 1, 1);
    Pi[MI(1, 2, 2)] = K[MI(1, 2, 2)] + M_(0, 0, 2) * M_(1, 2, 0) + M_(0, 2, 0) * M_(1, 0, 2)
                    + 4.0 * M_(0, 1, 1) * M_(1, 1, 1) + 2.0 * M_(1, 0, 1) * M_(0, 2, 1)
                    + 2.0 * M_(1, 1, 0) * M_(0, 1, 2);
    Pi[MI(2, 1, 2)] = K[MI(2, 1, 2)] + M_(0, 0, 2) * M_(2, 1, 0) + M_(2, 0, 0) * M_(0, 1, 2)
                    + 4.0 * M_(1, 0, 1) * M_(1, 1, 1) + 2.0 * M_(0, 1, 1) * M_(2, 0, 1)
                    + 2.0 * M_(1, 1, 0) * M_(1, 0, 2);
    Pi[MI(2, 2, 1)] = K[MI(2, 2, 1)] + M_(2, 0, 0) * M_(0, 2, 1) + M_(0, 2, 0) * M_(2, 0, 1)
                    + 4.0 * M_(1, 1, 0) * M_(1, 1, 1) + 2.0 * M_(1, 0, 1) * M_(1, 2, 0)
                    + 2.0 * M_(0, 1, 1) * M_(2, 1, 0);
    Pi[MI(2, 2, 2)] = K[MI(2, 2, 2)]
        + M_(2, 0, 0) * M_(0, 2, 2) + M_(0, 2, 0) * M_(2, 0, 2) + M_(0, 0, 2) * M_(2, 2, 0)
        + 4.0 * M_(1, 1, 0) * M_(1, 1, 2) + 4.0 * M_(1, 0, 1) * M_(1, 2, 1)
        + 4.0 * M_(0, 1, 1) * M_(2, 1, 1)
        + 4.0 * M_(1, 1, 1) * M_(1, 1, 1)
        + 2.0 * M_(2, 1, 0) * M_(0, 1, 2) + 2.0 * M_(2, 0, 1) * M_(0, 2, 1)
        + 2.0 * M_(1, 2, 0) * M_(1, 0, 2)
        - 2.0 * M_(2, 0, 0) * M_(0, 2, 0) * M_(0, 0, 2)
        - 4.0 * M_(2, 0, 0) * M_(0, 1, 1) * M_(0, 1, 1)
        - 4.0 * M_(0, 2, 0) * M_(1, 0, 1) * M_(1, 0, 1)
        - 4.0 * M_(0, 0, 2) * M_(1, 1, 0) * M_(1, 1, 0)
        - 16.0 * M_(1, 1, 0) * M_(1, 0, 1) * M_(0, 1, 1);
#undef M_
}

/* ------------------------------------------------------------------ */
/* collision (Sec. II.B-C)                                               */
/* ------------------------------------------------------------------ */

static int moment_order(int j)
{
    int p, q, r;
    moment_exponents(j, &p, &q, &r);
    return p + q + r;
}

/* One cell: pre-collision populations g (after streaming), density rho,
 * velocity u, density gradient grad_rho, expansion source Lambda.
 * Writes post-collision g* (Eq. 14).  Optionally returns P_h and Xi. */
static void collide(const orc_sim *S, const double *g, double rho, const double u[3],
                    const double grad_rho[3], double Lam, double *gstar,
                    double *P_h_out, double *Xi_out)
{
    int Q = S->Q;
    double cs2 = S->cs2;
    double sum_g = 0.0;
    for (int i = 0; i < Q; ++i) sum_g += g[i];
    double P_h = sum_g + 0.5 * rho * cs2 * Lam;                       /* Eq. 13a */
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double Xi[27], fp[27], fpeq[27];
    for (int i = 0; i < Q; ++i) {
        double cu = S->c[i][0] * u[0] + S->c[i][1] * u[1] + S->c[i][2] * u[2];
        double feq = S->w[i] * rho * (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2)); /* Eq. 10 */
        double cmu_grad = (S->c[i][0] - u[0]) * grad_rho[0] + (S->c[i][1] - u[1]) * grad_rho[1] +
                          (S->c[i][2] - u[2]) * grad_rho[2];
        Xi[i] = cs2 * (feq / rho - S->w[i]) * cmu_grad + S->w[i] * rho * cs2 * Lam;  /* Eq. 9 */
        double geq = S->w[i] * (P_h - rho * cs2) + cs2 * feq;                      /* Eq. 12 */
        fp[i] = g[i] / (rho * cs2) + Xi[i] / (2.0 * rho * cs2);                     /* Eq. 19 */
        fpeq[i] = geq / (rho * cs2);
    }
    double Pi[27], Pieq[27], K[27], Keq[27], Ks[27], Pis[27], fps[27];
    central_moments(S, fp, u, Pi);
    central_moments(S, fpeq, u, Pieq);
    orc_cumulants(S->s.dim, Pi, K);
    orc_cumulants(S->s.dim, Pieq, Keq);
    /* Eq. 15/23 read as relaxation toward the equilibrium cumulants */
    for (int j = 0; j < Q; ++j) {
        int o = moment_order(j);
        if (o <= 1) Ks[j] = K[j];
        else if (o >= 3) Ks[j] = Keq[j] + (1.0 - S->s.omega_hi) * (K[j] - Keq[j]);
        else Ks[j] = 0.0; /* second order handled below */
    }
    double ws = S->omega_s, wb = S->omega_b;
    if (S->s.dim == 2) {
        int ixx = MI(2, 0, 0), iyy = MI(0, 2, 0), ixy = MI(1, 1, 0);
        double tr = K[ixx] + K[iyy], treq = Keq[ixx] + Keq[iyy];
        double dv = K[ixx] - K[iyy], dveq = Keq[ixx] - Keq[iyy];
        double trs = treq + (1.0 - wb) * (tr - treq);
        double dvs = dveq + (1.0 - ws) * (dv - dveq);
        Ks[ixx] = 0.5 * (trs + dvs);
        Ks[iyy] = 0.5 * (trs - dvs);
        Ks[ixy] = Keq[ixy] + (1.0 - ws) * (K[ixy] - Keq[ixy]);
    } else {
        int ixx = MI(2, 0, 0), iyy = MI(0, 2, 0), izz = MI(0, 0, 2);
        double tr = K[ixx] + K[iyy] + K[izz], treq = Keq[ixx] + Keq[iyy] + Keq[izz];
        double d1 = K[ixx] - K[iyy], d1eq = Keq[ixx] - Keq[iyy];
        double d2 = K[ixx] - K[izz], d2eq = Keq[ixx] - Keq[izz];
        double trs = treq + (1.0 - wb) * (tr - treq);
        double d1s = d1eq + (1.0 - ws) * (d1 - d1eq);
        double d2s = d2eq + (1.0 - ws) * (d2 - d2eq);
        Ks[ixx] = (trs + d1s + d2s) / 3.0;
        Ks[iyy] = Ks[ixx] - d1s;
        Ks[izz] = Ks[ixx] - d2s;
        int off[3] = {MI(1, 1, 0), MI(1, 0, 1), MI(0, 1, 1)};
        for (int t = 0; t < 3; ++t)
            Ks[off[t]] = Keq[off[t]] + (1.0 - ws) * (K[off[t]] - Keq[off[t]]);
    }
    orc_cumulants_inverse(S->s.dim, Ks, Pis);
    central_moments_inverse(S, Pis, u, fps);
    for (int i = 0; i < Q; ++i) gstar[i] = rho * cs2 * fps[i] + 0.5 * Xi[i];   /* Eq. 14 */
    if (P_h_out) *P_h_out = P_h;
    if (Xi_out)
        for (int i = 0; i < Q; ++i) Xi_out[i] = Xi[i];
}

/* ------------------------------------------------------------------ */
/* streaming with boundary rules (Eq. 8, 28, 31, 32)                     */
/* ------------------------------------------------------------------ */

/* inlet velocity vector for an inlet on face f at position p */
static void inlet_velocity(const orc_sim *S, int f, const int p[3], double uin[3])
{
    int a = f / 2;
    double sgn = (f % 2 == 0) ? 1.0 : -1.0;  /* inward normal */
    double mag = S->s.u_in;
    if (S->s.poiseuille_inlet && S->s.dim == 2 && a == 0) {
        double ny = S->s.ny, y = p[1] + 0.5;
        mag = 6.0 * S->s.u_in * y * (ny - y) / (ny * ny);
    }
    uin[0] = uin[1] = uin[2] = 0.0;
    uin[a] = sgn * mag;
}

/* pulled population i at cell p (post-streaming, time n+1) */
static double pull(const orc_sim *S, int i, const int p[3], long cidx)
{
    int src[3] = {p[0] - S->c[i][0], p[1] - S->c[i][1], p[2] - S->c[i][2]};
    int wall = 0, inlet = -1, outlet = -1;
    for (int a = 0; a < S->s.dim; ++a) {
        int n = extent(S, a), f = -1;
        if (src[a] < 0) f = 2 * a;
        else if (src[a] >= n) f = 2 * a + 1;
        if (f < 0) continue;
        switch (S->s.bc[f]) {
        case ORC_PERIODIC: src[a] = ((src[a] % n) + n) % n; break;
        case ORC_INLET: if (inlet < 0) inlet = f; break;
        case ORC_OUTLET:
        case ORC_OUTLET_PRESSURE: if (outlet < 0) outlet = f; break;
        default: wall = 1; break;
        }
    }
    const double *g = S->g;
    long N = S->N;
    int ib = S->opp[i];
    if (!wall && (inlet >= 0 || outlet >= 0)) {
        /* a link that leaves through an inlet or outlet face where the
         * boundary column is solid hits the solid: bounce-back, as when it
         * also crosses a wall face */
        int q[3] = {src[0], src[1], src[2]};
        for (int a = 0; a < S->s.dim; ++a) {
            if (q[a] < 0) q[a] = 0;
            else if (q[a] >= extent(S, a)) q[a] = extent(S, a) - 1;
        }
        if (S->solid[cell_index(S, q)]) wall = 1;
    }
    if (wall) return g[(long)ib * N + cidx];                              /* Eq. 28 */
    if (inlet >= 0) {                                                     /* Eq. 31 */
        double uin[3];
        inlet_velocity(S, inlet, p, uin);
        double cu = S->c[i][0] * uin[0] + S->c[i][1] * uin[1] + S->c[i][2] * uin[2];
        return g[(long)ib * N + cidx] + (S->w[i] + S->w[ib]) * S->rho_in * cu;
    }
    if (outlet >= 0 && S->s.bc[outlet] == ORC_OUTLET_PRESSURE) {         /* constant P_h */
        double T = S->T[cidx], Y[ORC_MAXSP], u[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < S->nsp; ++k) Y[k] = S->Y[(long)k * N + cidx];
        double rho = eos_rho(S, T, inv_molar_mass(S, Y));
        for (int a = 0; a < S->s.dim; ++a) {
            double m = 0.0;
            for (int j = 0; j < S->Q; ++j) m += S->c[j][a] * g[(long)j * N + cidx];
            u[a] = m / (rho * S->cs2);
        }
        double cu = S->c[i][0] * u[0] + S->c[i][1] * u[1] + S->c[i][2] * u[2];
        double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        double geq_even = S->w[i] * (0.0 - rho * S->cs2) +
                          S->cs2 * S->w[i] * rho * (1.0 + cu * cu / (2.0 * S->cs2 * S->cs2) - uu / (2.0 * S->cs2));
        return -g[(long)ib * N + cidx] + 2.0 * geq_even;
    }
    if (outlet >= 0) {                                                    /* Eq. 32 */
        int a = outlet / 2;
        int nsign = (outlet % 2 == 1) ? 1 : -1;  /* outward normal along axis a */
        double T = S->T[cidx], Y[ORC_MAXSP];
        for (int k = 0; k < S->nsp; ++k) Y[k] = S->Y[(long)k * N + cidx];
        double rho = eos_rho(S, T, inv_molar_mass(S, Y));
        double mom = 0.0;
        for (int j = 0; j < S->Q; ++j) mom += S->c[j][a] * nsign * g[(long)j * N + cidx];
        double un = mom / (rho * S->cs2);
        int q[3] = {p[0], p[1], p[2]};
        q[a] -= nsign;
        double inner = g[(long)i * N + cidx];
        if (q[a] >= 0 && q[a] < extent(S, a)) {
            long qi = cell_index(S, q);
            if (!S->solid[qi]) inner = g[(long)i * N + qi];
        }
        return (S->cs - un) * inner + (1.0 - S->cs + un) * g[(long)i * N + cidx];
    }
    long sidx = cell_index(S, src);
    if (S->solid[sidx]) {
        double q = S->curved ? S->linkq[(long)i * N + cidx] : -1.0;
        if (q < 0.0) return g[(long)ib * N + cidx];                        /* Eq. 28 */
        /* interpolated bounce-back (Eq. 29-30), post-collision values at t */
        if (q < 0.5) {
            int r[3] = {p[0] + S->c[i][0], p[1] + S->c[i][1], p[2] + S->c[i][2]};
            long ridx;
            int face = -1;
            if (classify(S, r, &ridx, &face) == PT_FLUID)
                return 2.0 * q * g[(long)ib * N + cidx] + (1.0 - 2.0 * q) * g[(long)ib * N + ridx];
            return g[(long)ib * N + cidx];
        }
        return g[(long)ib * N + cidx] / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * g[(long)i * N + cidx];
    }
    return g[(long)i * N + sidx];                                          /* Eq. 8 */
}

/* ------------------------------------------------------------------ */
/* one cell of the coupled step                                          */
/* ------------------------------------------------------------------ */

/* Per-cell quantities, also returned to the tests by orc_cell_terms. */
typedef struct {
    double rho, u[3], grad_rho[3];
    double conv_T, diff_T, reac_T;
    double conv_Y[ORC_MAXSP], diff_Y[ORC_MAXSP], reac_Y[ORC_MAXSP];
    double Lambda, P_h;
} orc_terms;

static void cell_update(const orc_sim *S, const int p[3], long cidx, double *gin,
                        orc_terms *tm, double *T_new, double *Y_new, double *gstar)
{
    int nsp = S->nsp, dim = S->s.dim;
    /* a1: pull-stream with boundary rules */
    for (int i = 0; i < S->Q; ++i) gin[i] = pull(S, i, p, cidx);

    /* a2: density from the EOS, velocity from Eq. 13b */
    orc_pt c0;
    fluid_pt(S, cidx, &c0);
    double rho = c0.rho;
    double u[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < dim; ++a) {
        double m = 0.0;
        for (int i = 0; i < S->Q; ++i) m += S->c[i][a] * gin[i];
        u[a] = m / (rho * S->cs2);
    }

    /* a3-a5: per-axis FD lines */
    double conv_T = 0.0, diff_T = 0.0;
    double conv_Y[ORC_MAXSP] = {0}, diff_Y[ORC_MAXSP] = {0};
    double grad_rho[3] = {0.0, 0.0, 0.0};
    double epsY = S->s.weno_eps, epsT = S->s.weno_eps * S->s.T_in * S->s.T_in;
    for (int a = 0; a < dim; ++a) {
        orc_pt line[5];
        int near = build_line(S, p, cidx, a, line);
        double v[5];
        /* density gradient, 4th order (used by diffusion and by Xi) */
        for (int j = 0; j < 5; ++j) v[j] = line[j].rho;
        double drho = orc_d1(v);
        grad_rho[a] = drho;
        /* temperature: convection (no correction) and diffusion, Eq. 7 */
        for (int j = 0; j < 5; ++j) v[j] = line[j].T;
        conv_T += u[a] * (near ? orc_c2(v) : orc_weno3(v, u[a], epsT));
        diff_T += S->alpha * (orc_d2(v) + drho * orc_d1(v) / rho);
        /* species convection with the correction of Eq. 26 */
        double L[ORC_MAXSP], sumL = 0.0;
        for (int k = 0; k < nsp; ++k) {
            for (int j = 0; j < 5; ++j) v[j] = line[j].Y[k];
            L[k] = near ? orc_c2(v) : orc_weno3(v, u[a], epsY);
            sumL += L[k];
        }
        for (int k = 0; k < nsp; ++k) conv_Y[k] += u[a] * (L[k] - c0.Y[k] * sumL);
        /* species diffusion, Eq. 1-2 with constant D_k, expanded form */
        double vW[5];
        for (int j = 0; j < 5; ++j) vW[j] = line[j].invW;
        double dinvW = orc_d1(vW);
        double m[ORC_MAXSP], dm[ORC_MAXSP], dY[ORC_MAXSP], Msum = 0.0, dMsum = 0.0;
        for (int k = 0; k < nsp; ++k) {
            double ak = S->D[k] * S->s.W[k];
            for (int j = 0; j < 5; ++j) v[j] = line[j].X[k];
            double dX = orc_d1(v), d2X = orc_d2(v);
            m[k] = ak * c0.invW * dX;
            dm[k] = ak * (c0.invW * d2X + dinvW * dX);
            for (int j = 0; j < 5; ++j) v[j] = line[j].Y[k];
            dY[k] = orc_d1(v);
            Msum += m[k];
            dMsum += dm[k];
        }
        for (int k = 0; k < nsp; ++k)
            diff_Y[k] += dm[k] - dY[k] * Msum - c0.Y[k] * dMsum +
                         (m[k] - c0.Y[k] * Msum) * drho / rho;
    }

    /* a6: reaction */
    double q = rate_q(S, c0.T, c0.Y);
    double reac_T = S->s.Q / S->s.cp * q;
    double reac_Y[ORC_MAXSP];
    for (int k = 0; k < nsp; ++k) reac_Y[k] = yield(S, k) * q;

    /* a7: explicit Euler and Lambda (Eq. 6, from the non-convective rates) */
    *T_new = c0.T + (-conv_T + diff_T + reac_T);
    double Lam = (diff_T + reac_T) / c0.T;
    double W = 1.0 / c0.invW;
    for (int k = 0; k < nsp; ++k) {
        Y_new[k] = c0.Y[k] + (-conv_Y[k] + diff_Y[k] + reac_Y[k]);
        Lam += W / S->s.W[k] * (diff_Y[k] + reac_Y[k]);
    }

    /* a8-a9: source, pre-conditioning and cumulant collision */
    double P_h;
    collide(S, gin, rho, u, grad_rho, Lam, gstar, &P_h, NULL);

    if (tm) {
        tm->rho = rho;
        for (int a = 0; a < 3; ++a) { tm->u[a] = u[a]; tm->grad_rho[a] = grad_rho[a]; }
        tm->conv_T = conv_T; tm->diff_T = diff_T; tm->reac_T = reac_T;
        for (int k = 0; k < nsp; ++k) {
            tm->conv_Y[k] = conv_Y[k]; tm->diff_Y[k] = diff_Y[k]; tm->reac_Y[k] = reac_Y[k];
        }
        tm->Lambda = Lam;
        tm->P_h = P_h;
    }
}

/* ------------------------------------------------------------------ */
/* public oracle interface (ctypes)                                      */
/* ------------------------------------------------------------------ */

orc_sim *orc_new(const orc_setup *s, const unsigned char *solid)
{
    orc_sim *S = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!S) return NULL;
    S->s = *s;
    if (S->s.dim == 2) S->s.nz = 1;
    S->nsp = s->n_species;
    S->N = (long)S->s.nx * S->s.ny * S->s.nz;
    lattice_init(S);
    S->cs2 = 1.0 / 3.0;
    S->cs = sqrt(S->cs2);
    S->omega_s = 1.0 / (s->nu / S->cs2 + 0.5);   /* Eq. 18 read as 1/tau */
    S->omega_b = s->omega_bulk > 0.0 ? s->omega_bulk : S->omega_s;
    S->alpha = s->nu / s->Pr;
    for (int k = 0; k < S->nsp; ++k) S->D[k] = S->alpha / s->Le[k];
    S->A_lat = s->A * s->dt;
    S->invW_in = inv_molar_mass(S, s->Y_in);
    S->rho_in = eos_rho(S, s->T_in, S->invW_in);
    long N = S->N;
    S->g = (double *)calloc((size_t)S->Q * N, sizeof(double));
    S->gn = (double *)calloc((size_t)S->Q * N, sizeof(double));
    S->T = (double *)calloc((size_t)N, sizeof(double));
    S->Tn = (double *)calloc((size_t)N, sizeof(double));
    S->Y = (double *)calloc((size_t)S->nsp * N, sizeof(double));
    S->Yn = (double *)calloc((size_t)S->nsp * N, sizeof(double));
    S->solid = (unsigned char *)calloc((size_t)N, 1);
    if (!S->g || !S->gn || !S->T || !S->Tn || !S->Y || !S->Yn || !S->solid) return NULL;
    if (solid) memcpy(S->solid, solid, (size_t)N);
    return S;
}

/* Curved walls from n primitives (5 doubles each, see build_curved). */
void orc_set_geometry(orc_sim *S, int n, const double *prims)
{
    free(S->prims);
    S->prims = (double *)malloc(sizeof(double) * 5 * (size_t)(n > 0 ? n : 1));
    if (n > 0) memcpy(S->prims, prims, sizeof(double) * 5 * (size_t)n);
    S->nprims = n;
    build_curved(S);
    S->curved = 1;
}

long orc_num_ghosts(const orc_sim *S) { return S->nghost; }

void orc_free(orc_sim *S)
{
    if (!S) return;
    free(S->prims); free(S->linkq); free(S->ghost_of); free(S->gh_start); free(S->gh_idx);
    free(S->gh_w); free(S->gh_B);
    free(S->g); free(S->gn); free(S->T); free(S->Tn); free(S->Y); free(S->Yn); free(S->solid);
    free(S);
}

long orc_ncells(const orc_sim *S) { return S->N; }
int orc_q(const orc_sim *S) { return S->Q; }
double orc_omega_s(const orc_sim *S) { return S->omega_s; }

/* T [N], Y [nsp][N], g [Q][N] (g may be NULL: zero populations) */
void orc_set_state(orc_sim *S, const double *T, const double *Y, const double *g)
{
    long N = S->N;
    memcpy(S->T, T, sizeof(double) * (size_t)N);
    memcpy(S->Y, Y, sizeof(double) * (size_t)S->nsp * N);
    if (g) memcpy(S->g, g, sizeof(double) * (size_t)S->Q * N);
    else memset(S->g, 0, sizeof(double) * (size_t)S->Q * N);
    S->steps = 0;
}

void orc_get_state(const orc_sim *S, double *T, double *Y, double *g)
{
    long N = S->N;
    if (T) memcpy(T, S->T, sizeof(double) * (size_t)N);
    if (Y) memcpy(Y, S->Y, sizeof(double) * (size_t)S->nsp * N);
    if (g) memcpy(g, S->g, sizeof(double) * (size_t)S->Q * N);
}

/* Threads of orc_step (OpenMP over grid rows when the library is built
 * with -fopenmp; 1 by default).  Every cell's update reads state n only and
 * writes its own outputs, so the result does not depend on the count; the
 * threaded form exists to time the oracle on all host cores. */
static int orc_nthreads = 1;

void orc_set_threads(int n) { orc_nthreads = n > 0 ? n : 1; }

int orc_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* Advance n coupled steps.  Solid cells keep their state. */
void orc_step(orc_sim *S, int n)
{
    long N = S->N;
    int rows = S->s.ny * S->s.nz;
    for (int it = 0; it < n; ++it) {
        memcpy(S->gn, S->g, sizeof(double) * (size_t)S->Q * N);
        memcpy(S->Tn, S->T, sizeof(double) * (size_t)N);
        memcpy(S->Yn, S->Y, sizeof(double) * (size_t)S->nsp * N);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(orc_nthreads)
#endif
        for (int row = 0; row < rows; ++row) {
            double gin[27], gst[27], Yn[ORC_MAXSP], Tn;
            int y = row % S->s.ny, z = row / S->s.ny;
            for (int x = 0; x < S->s.nx; ++x) {
                int p[3] = {x, y, z};
                long c = cell_index(S, p);
                if (S->solid[c]) continue;
                cell_update(S, p, c, gin, NULL, &Tn, Yn, gst);
                S->Tn[c] = Tn;
                for (int k = 0; k < S->nsp; ++k) S->Yn[(long)k * N + c] = Yn[k];
                for (int i = 0; i < S->Q; ++i) S->gn[(long)i * N + c] = gst[i];
            }
        }
        double *t;
        t = S->g; S->g = S->gn; S->gn = t;
        t = S->T; S->T = S->Tn; S->Tn = t;
        t = S->Y; S->Y = S->Yn; S->Yn = t;
        S->steps++;
    }
}

/* One step of the cells with x0 <= x < x1 only (a slab of a domain
 * decomposition along x); every other cell keeps its current state.  Used
 * by the decomposition test: the update of a slab reads nothing beyond
 * two cells on each side of it. */
void orc_step_slab(orc_sim *S, int x0, int x1)
{
    long N = S->N;
    double gin[27], gst[27], Yn[ORC_MAXSP], Tn;
    memcpy(S->gn, S->g, sizeof(double) * (size_t)S->Q * N);
    memcpy(S->Tn, S->T, sizeof(double) * (size_t)N);
    memcpy(S->Yn, S->Y, sizeof(double) * (size_t)S->nsp * N);
    for (int z = 0; z < S->s.nz; ++z)
        for (int y = 0; y < S->s.ny; ++y)
            for (int x = x0; x < x1; ++x) {
                int p[3] = {x, y, z};
                long c = cell_index(S, p);
                if (S->solid[c]) continue;
                cell_update(S, p, c, gin, NULL, &Tn, Yn, gst);
                S->Tn[c] = Tn;
                for (int k = 0; k < S->nsp; ++k) S->Yn[(long)k * N + c] = Yn[k];
                for (int i = 0; i < S->Q; ++i) S->gn[(long)i * N + c] = gst[i];
            }
    double *t;
    t = S->g; S->g = S->gn; S->gn = t;
    t = S->T; S->T = S->Tn; S->Tn = t;
    t = S->Y; S->Y = S->Yn; S->Yn = t;
    S->steps++;
}

/* Per-cell terms of the next step at cell (x,y,z), without advancing.
 * out layout: rho, u[3], grad_rho[3], conv_T, diff_T, reac_T, Lambda, P_h,
 * then conv_Y[nsp], diff_Y[nsp], reac_Y[nsp], then g_in[Q], g*[Q],
 * T_new, Y_new[nsp]. */
void orc_cell_terms(const orc_sim *S, int x, int y, int z, double *out)
{
    int p[3] = {x, y, z};
    long c = cell_index(S, p);
    orc_terms tm;
    double gin[27], gst[27], Yn[ORC_MAXSP], Tn;
    memset(&tm, 0, sizeof tm);
    cell_update(S, p, c, gin, &tm, &Tn, Yn, gst);
    int o = 0, nsp = S->nsp;
    out[o++] = tm.rho;
    for (int a = 0; a < 3; ++a) out[o++] = tm.u[a];
    for (int a = 0; a < 3; ++a) out[o++] = tm.grad_rho[a];
    out[o++] = tm.conv_T; out[o++] = tm.diff_T; out[o++] = tm.reac_T;
    out[o++] = tm.Lambda; out[o++] = tm.P_h;
    for (int k = 0; k < nsp; ++k) out[o++] = tm.conv_Y[k];
    for (int k = 0; k < nsp; ++k) out[o++] = tm.diff_Y[k];
    for (int k = 0; k < nsp; ++k) out[o++] = tm.reac_Y[k];
    for (int i = 0; i < S->Q; ++i) out[o++] = gin[i];
    for (int i = 0; i < S->Q; ++i) out[o++] = gst[i];
    out[o++] = Tn;
    for (int k = 0; k < nsp; ++k) out[o++] = Yn[k];
}

/* Single-cell collision for the tests: g (pre-collision), rho, u, grad_rho,
 * Lambda -> g*, Xi, P_h.  Uses the sim's lattice and relaxation rates. */
void orc_collide_cell(const orc_sim *S, const double *g, double rho, const double *u,
                      const double *grad_rho, double Lam, double *gstar, double *Xi, double *P_h)
{
    double uu[3] = {u[0], u[1], u[2]}, gr[3] = {grad_rho[0], grad_rho[1], grad_rho[2]};
    collide(S, g, rho, uu, gr, Lam, gstar, P_h, Xi);
}

/* Central moments (Eq. 21) and their inverse, for the tests. */
void orc_central_moments(const orc_sim *S, const double *f, const double *u, double *Pi)
{
    double uu[3] = {u[0], u[1], u[2]};
    central_moments(S, f, uu, Pi);
}

void orc_central_moments_inverse(const orc_sim *S, const double *Pi, const double *u, double *f)
{
    double uu[3] = {u[0], u[1], u[2]};
    central_moments_inverse(S, Pi, uu, f);
}

/* Diagnostics over fluid cells (a11):
 * out[0] x_f = sum Y_F / (Y_F,in * fluid cells in the x = 0 section) [cells]
 * out[1] mass = sum rho
 * out[2] heat release = sum rho (Q/cp) q   [K per step, rho-weighted]
 * out[3] fuel consumption = sum rho q
 * out[4] max T
 * out[5] x of the maximum heat release on the centre line y = ny/2, z = nz/2
 *        (smallest x on ties; -1 when no fluid cell there)
 * out[6] number of fluid cells with a non-finite state value
 * out[7] number of fluid cells */
void orc_diagnostics(const orc_sim *S, double *out)
{
    long N = S->N;
    int nsp = S->nsp;
    double sumYF = 0.0, mass = 0.0, hrr = 0.0, fuel = 0.0, Tmax = -INFINITY;
    double nonfinite = 0.0, nfluid = 0.0, section = 0.0;
    double best = -INFINITY;
    int bestx = -1;
    int yc = S->s.ny / 2, zc = S->s.nz / 2;
    for (int z = 0; z < S->s.nz; ++z)
        for (int y = 0; y < S->s.ny; ++y)
            for (int x = 0; x < S->s.nx; ++x) {
                int p[3] = {x, y, z};
                long c = cell_index(S, p);
                if (S->solid[c]) continue;
                nfluid += 1.0;
                if (x == 0) section += 1.0;
                double Y[ORC_MAXSP];
                int bad = !isfinite(S->T[c]);
                for (int k = 0; k < nsp; ++k) {
                    Y[k] = S->Y[(long)k * N + c];
                    bad |= !isfinite(Y[k]);
                }
                for (int i = 0; i < S->Q; ++i) bad |= !isfinite(S->g[(long)i * N + c]);
                if (bad) { nonfinite += 1.0; continue; }
                double T = S->T[c];
                double rho = eos_rho(S, T, inv_molar_mass(S, Y));
                double q = rate_q(S, T, Y);
                double h = rho * S->s.Q / S->s.cp * q;
                sumYF += Y[S->s.fuel];
                mass += rho;
                hrr += h;
                fuel += rho * q;
                if (T > Tmax) Tmax = T;
                if (y == yc && z == zc && h > best) { best = h; bestx = x; }
            }
    out[0] = section > 0.0 ? sumYF / (S->s.Y_in[S->s.fuel] * section) : 0.0;
    out[1] = mass;
    out[2] = hrr;
    out[3] = fuel;
    out[4] = Tmax;
    out[5] = (double)bestx;
    out[6] = nonfinite;
    out[7] = nfluid;
}

/* Reaction front per column (the dead zone of Sec. IV.A), 2-D: for every
 * column x, the largest heat release rho (Q/cp) q over the fluid cells of
 * rows y0 <= y < y1 into peak[x] (0 when there is none) and the distance of
 * that cell's centre from the nearer edge of the row band, walls half-way
 * between cells, into dist[x]; ties go to the smallest y. */
void orc_column_peaks(const orc_sim *S, int y0, int y1, double *peak, double *dist)
{
    long N = S->N;
    for (int x = 0; x < S->s.nx; ++x) {
        double best = -1.0;
        int by = y0;
        for (int y = y0; y < y1; ++y) {
            int p[3] = {x, y, 0};
            long c = cell_index(S, p);
            if (S->solid[c]) continue;
            double Y[ORC_MAXSP];
            for (int k = 0; k < S->nsp; ++k) Y[k] = S->Y[(long)k * N + c];
            double rho = eos_rho(S, S->T[c], inv_molar_mass(S, Y));
            double h = rho * S->s.Q / S->s.cp * rate_q(S, S->T[c], Y);
            if (h > best) { best = h; by = y; }
        }
        double d0 = by - y0 + 0.5, d1 = y1 - 0.5 - by;
        peak[x] = best < 0.0 ? 0.0 : best;
        dist[x] = d0 < d1 ? d0 : d1;
    }
}
