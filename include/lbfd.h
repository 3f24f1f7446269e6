/*
 * lbfd.h -- C ABI of the GB300 (sm_103a) library for the coupled time step
 * of the hybrid low-Mach lattice Boltzmann / finite-difference solver of
 * Hosseini & Thevenin, arXiv 2304.05657.
 *
 * One step advances, for every fluid cell, the pressure-based lattice
 * Boltzmann populations g_i (Sec. II.B, Eq. 8-13) with the cumulant
 * collision (Sec. II.C, Eq. 14-24) and the finite-difference temperature and
 * species fields (Sec. II.A Eq. 1-7, Sec. II.D Eq. 26) with a single-step
 * Arrhenius source, with half-way bounce-back walls, velocity inlet and
 * convective outlet (Sec. III.A, Eq. 28, 31, 32) and ghost-node scalar
 * boundaries (Sec. III.B, Eq. 34).  All of a step runs in CUDA kernels of
 * this library; there is no CPU fallback: when no CUDA device is present
 * lbfd_create returns LBFD_ECUDA.
 *
 * Conventions shared by every entry point
 *   - Return value: LBFD_OK (0) or one of the LBFD_E* codes below;
 *     lbfd_strerror() gives a static message.  A CUDA failure is reported
 *     as LBFD_ECUDA and its text is kept in lbfd_last_error().
 *   - Units are lattice units (dr = dt = 1, cs^2 = 1/3) except the
 *     thermochemistry in lbfd_mechanism, which is SI; the step length
 *     lbfd_params.dt [s] maps the pre-exponential factor to A*dt per step.
 *   - Cell index: c = x + nx*(y + ny*z), x fastest.  Populations are
 *     numbered i = (cx+1) + 3(cy+1) [+ 9(cz+1) in 3-D] with c_i in {-1,0,1}.
 *   - Every host array passed in is copied before the call returns; the
 *     library never keeps a caller pointer.  Output arrays are owned by the
 *     caller.  The handle owns all device memory it allocates.
 *   - Calls on one handle are not thread-safe; distinct handles are
 *     independent.
 */
#ifndef LBFD_H
#define LBFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LBFD_OK 0
#define LBFD_EINVAL 1     /* bad argument (null pointer, size, enum value) */
#define LBFD_ENOMEM 2     /* device or host allocation failed */
#define LBFD_ECUDA 3      /* a CUDA call failed (see lbfd_last_error) */
#define LBFD_ENONFINITE 4 /* a fluid cell holds a non-finite value */
#define LBFD_ETIMEOUT 5   /* a bounded device wait gave up */
#define LBFD_EUNSTABLE 6  /* parameters violate a stability limit */
#define LBFD_ENOTSUP 7    /* valid request this build does not support */

/* boundary type of each domain face (Sec. III) */
#define LBFD_BC_PERIODIC 0
#define LBFD_BC_WALL_ADIABATIC 1   /* half-way bounce-back, Neumann T and Y */
#define LBFD_BC_WALL_ISOTHERMAL 2  /* half-way bounce-back, Dirichlet T = T_wall */
#define LBFD_BC_INLET 3            /* Eq. 31 velocity inlet, Dirichlet T_in, Y_in */
#define LBFD_BC_OUTLET 4           /* Eq. 32 convective outlet, zero-gradient T, Y */
#define LBFD_BC_OUTLET_PRESSURE 5  /* constant P_h = 0 outlet (Sec. IV.A, IV.C) by anti-bounce-back:
                                      g_i = -g*_ibar + 2 (even part of g^eq at P_h = 0, rho and u of
                                      the cell); zero-gradient T, Y */

/* arithmetic of the step */
#define LBFD_FP64 0  /* FP64 storage and arithmetic */
#define LBFD_MIXED 1 /* FP32 storage and arithmetic; FP64 Arrhenius above T_fp64 */
#define LBFD_TANGENT 2 /* FP64 values each carrying 4 derivatives (forward mode),
                          with respect to theta = (ln A, Ta, T_wall, u_in); 2-D only,
                          general-form kernel.  T_wall moves every isothermal wall face
                          and, when solids are isothermal, T_solid together. */
#define LBFD_TANGENT_MIXED 3 /* as LBFD_TANGENT with FP32 values and derivatives
                                (FP32 forward), the Arrhenius rate and its derivatives
                                in FP64 above T_fp64 and the objectives accumulated
                                in FP64 (lbfd_gradient); no curved walls. */

/* objectives of lbfd_gradient and of the discrete adjoint */
#define LBFD_OBJ_FLAME_POSITION 0 /* x_f [m] as in lbfd_flame_position */
#define LBFD_OBJ_HEAT_RELEASE 1   /* sum of LBFD_FIELD_HRR over fluid cells (lbfd_gradient only) */
#define LBFD_OBJ_QUENCH_DISTANCE 2 /* smooth distance [cells] between the reaction zone and the cold
                                      walls, the differentiable stand-in for the dead-zone thickness of
                                      Sec. IV.A: J = (sum_c h_c d_c^-4 / sum_c h_c)^(-1/4) over fluid
                                      cells, h_c = LBFD_FIELD_HRR, d_c the distance from the cell centre
                                      to the nearest isothermal boundary (an isothermal solid cell or
                                      wall face; wall planes half-way between cells) along the axis
                                      directions, 64 when none is that close.  A heat-release-weighted
                                      soft minimum of the wall distance: it tends to the distance of the
                                      reacting cells closest to a wall. */

/* number of species the kernels are built for */
#define LBFD_NSP 5

/* fields for lbfd_read_field */
#define LBFD_FIELD_T 0
#define LBFD_FIELD_Y0 1    /* Y_k is LBFD_FIELD_Y0 + k */
#define LBFD_FIELD_UX 6    /* sum_i c_i g*_i / (rho cs^2), rho of the stored T, Y */
#define LBFD_FIELD_UY 7
#define LBFD_FIELD_UZ 8
#define LBFD_FIELD_PH 9    /* sum_i g*_i */
#define LBFD_FIELD_RHO 10  /* EOS density of the stored T, Y */
#define LBFD_FIELD_HRR 11  /* rho (Q/cp) A dt Y_F Y_O exp(-Ta/T) [K per step] */
#define LBFD_FIELD_G0 16   /* stored (post-collision) population i is G0 + i */

/* diagnostics vector of lbfd_diagnostics */
#define LBFD_DIAG_XF 0        /* sum Y_F / (Y_F,in * fluid cells at x = 0) [cells] */
#define LBFD_DIAG_MASS 1      /* sum rho over fluid cells */
#define LBFD_DIAG_HRR 2       /* sum of LBFD_FIELD_HRR over fluid cells */
#define LBFD_DIAG_FUEL 3      /* sum rho A dt Y_F Y_O exp(-Ta/T) (fuel consumed per step) */
#define LBFD_DIAG_TMAX 4      /* maximum T over fluid cells */
#define LBFD_DIAG_XHRR 5      /* x of the largest HRR on the line y = ny/2, z = nz/2 */
#define LBFD_DIAG_NONFINITE 6 /* fluid cells holding a non-finite value */
#define LBFD_DIAG_NFLUID 7    /* number of fluid cells */
#define LBFD_NDIAG 8

typedef struct lbfd_handle lbfd_handle;

/* Grid and face boundary types.  dim = 2 (D2Q9, nz ignored) or 3 (D3Q27).
 * bc[] and T_wall[] are per face in the order -x, +x, -y, +y, -z, +z;
 * T_wall is read for LBFD_BC_WALL_ISOTHERMAL faces only [K]. */
typedef struct lbfd_grid {
    int dim, nx, ny, nz;
    int bc[6];
    double T_wall[6];
} lbfd_grid;

/* Single-step global mechanism Fuel + ... -> products (the stand-in for the
 * Cantera kinetics of Sec. II.D).  Rate per unit mass of fuel:
 * q = A max(Y_F,0) max(Y_O,0) exp(-Ta/T); species k gains
 * nu_k W_k / (-nu_F W_F) q, temperature gains (Q/cp) q.
 * W [g/mol], nu_stoich < 0 for reactants, A [1/s], Ta [K], Q [J/kg fuel],
 * cp [J/kg/K] equal for all species, Le_k constant Lewis numbers. */
typedef struct lbfd_mechanism {
    int n_species;
    double W[8];
    double nu_stoich[8];
    int fuel, oxidiser;
    double A, Ta, Q, cp;
    double Le[8];
} lbfd_mechanism;

/* Physical and numerical parameters.
 * nu: kinematic viscosity (lattice); omega_s = 1/(nu/cs^2 + 1/2) (Eq. 18).
 * Pr: alpha = nu/Pr;  D_k = alpha/Le_k.
 * omega_bulk: rate of the second-order trace (<= 0: omega_s).
 * omega_hi: rate of cumulants of order >= 3 (Eq. 23).
 * u_in, T_in [K], Y_in: inlet state; (T_in, Y_in) is the EOS reference
 *   (rho = 1 there).
 * T_solid [K], solid_isothermal: thermal condition of solid-mask cells.
 * dx [m], dt [s]: physical size of a cell and of a step.
 * T_fp64 [K]: LBFD_MIXED evaluates the Arrhenius source in FP64 where T > T_fp64.
 * weno_eps: WENO3 epsilon for species (temperature: weno_eps*T_in^2).
 * precision: LBFD_FP64 or LBFD_MIXED.
 * poiseuille_inlet: 2-D -x/+x inlet with parabolic profile of mean u_in. */
typedef struct lbfd_params {
    double nu, Pr, omega_bulk, omega_hi;
    double u_in, T_in, Y_in[8];
    double T_solid;
    int solid_isothermal;
    double dx, dt;
    double T_fp64;
    double weno_eps;
    int precision;
    int poiseuille_inlet;
} lbfd_params;

/* Create a solver.  solid_mask: nx*ny*nz bytes on the host, nonzero = solid
 * (copied).  Allocates the double-buffered state on the current CUDA device
 * and initialises every cell to T = T_in, Y = Y_in, g = 0.
 * Errors: EINVAL (null pointer, sizes, bc values, n_species != LBFD_NSP is
 * ENOTSUP), EUNSTABLE (omega outside (0,2), |u_in| >= cs, explicit Euler
 * diffusion limit alpha*sum_axes(64/12) >= 2), ENOMEM, ECUDA. */
int lbfd_create(const lbfd_grid* grid, const uint8_t* solid_mask,
                const lbfd_mechanism* mech, const lbfd_params* params,
                lbfd_handle** out);

/* Release the handle and its device memory (NULL is accepted). */
int lbfd_destroy(lbfd_handle* h);

/* Run subsequent work on this CUDA stream (a cudaStream_t passed as void*;
 * NULL selects the legacy default stream).  The caller keeps ownership. */
int lbfd_set_stream(lbfd_handle* h, void* cuda_stream);

/* Set the scalar fields from host FP64 arrays T[N] and Y[nsp][N] and reset
 * the populations to g = 0 (the rest state, P_h = 0, u = 0).  Synchronous. */
int lbfd_init_fields(lbfd_handle* h, const double* T, const double* Y);

/* Set the full state from host FP64 arrays (g: [Q][N] post-collision
 * populations; NULL keeps them at 0).  Synchronous. */
int lbfd_set_state(lbfd_handle* h, const double* T, const double* Y, const double* g);

/* Advance n coupled steps (Sec. II), asynchronously on the handle's stream.
 * Each step is one launch of the fused kernel. */
int lbfd_step(lbfd_handle* h, int n);

/* Advance n coupled steps as one CUDA-graph launch (the n kernel launches
 * are captured once, then replayed; a new n, kernel variant or stream
 * re-captures).  On the legacy default stream the library captures on a
 * stream of its own and synchronises it before returning. */
int lbfd_step_graph(lbfd_handle* h, int n);

/* Advance n coupled steps in ONE persistent launch (2-D, LBFD_FP64 or
 * LBFD_MIXED, staircase walls): a cooperative launch of as many blocks as
 * are resident on the device at once; every step the blocks share out the
 * interior tiles, the tiles of cells next to in-domain solids and the
 * cells near domain faces (the per-cell arithmetic of kernel variant 6),
 * then meet at a grid-wide barrier before the buffers swap roles.  Batches
 * of channels packed into one masked domain (separated by solid rows)
 * advance together in this one launch.  Every barrier wait is bounded by
 * lbfd_set_wait_limit (default 2 s): a block that waits longer records it
 * and returns, the others follow within the same step, and the call returns
 * LBFD_ETIMEOUT with the step in lbfd_last_error(); the state is then
 * undefined (set it again before stepping) and the handle stays usable.
 * Synchronises the handle's stream (it reads the barrier's status).
 * Errors: EINVAL, ENOTSUP (3-D, tangent precisions, curved walls), ENOMEM,
 * ECUDA, ETIMEOUT. */
int lbfd_step_persistent(lbfd_handle* h, int n);

/* Bound of every grid-wide wait of lbfd_step_persistent, in nanoseconds.
 * ns <= 0: no block waits at all, so every barrier that is not met at once
 * fails (exercises the LBFD_ETIMEOUT path without a fault). */
int lbfd_set_wait_limit(lbfd_handle* h, long long ns);

/* Kernel variants of the step: 0 is the general form (any cell, D2Q9 and
 * D3Q27).  In 2-D (13 variants), 1..4 are shared-memory tiles of 32x8,
 * 32x4, 64x4 and 32x16 interior cells; 5..8 the same tiles plus a second
 * tile kernel (over the 64x2 tiles that need it) for the cells next to
 * in-domain solid cells (staircase walls, from shared memory); 9..12 as 5..8
 * with two interior cells per thread in packed FP32 arithmetic (tiles of
 * 32x8, 64x8, 32x8, 64x4 at 4, 2, 5 and 5 blocks per SM; the FP64 form runs
 * them one cell per thread).
 * In 3-D (8 variants), 1..2 are 32x4 columns marching through 16 or 32
 * z-planes with a five-plane shared-memory ring, 3 is 1 with the registers
 * capped for four blocks per SM, 4..5 are 1..2 split into an FD tile
 * kernel (a1-a7, writing Lambda and grad rho to a scratch buffer of four
 * planes) and a per-cell collision kernel (a8-a10), and 6..7 are 1..2 with
 * the cells next to in-domain solids updated in the tile kernel too (ghost
 * points by the mirror rule from the staged mask, bounce-back pulls).  The
 * cells the tiles leave out are listed at create.  In 2-D they go through
 * the general form.  In 3-D with staircase walls, a 64-bit neighbourhood
 * code per listed cell drives a compact form of the step: one list for the
 * cells next to in-domain solids (variants 1..5), one for the cells near
 * inlet and outlet faces of one axis.  The general form takes the other
 * cells near domain faces, and every listed cell when the walls are curved.
 * In FP32 with omega_hi = 1 the 3-D tile and coded kernels form only the
 * central moments of orders 0-2 (the relaxation sets the higher cumulants
 * to equilibrium).  All variants compute the same step up to rounding
 * order.  Default: 1 (0 for LBFD_TANGENT, which has the general form
 * only). */
int lbfd_num_variants(const lbfd_handle* h);
int lbfd_get_variant(const lbfd_handle* h);
int lbfd_set_variant(lbfd_handle* h, int variant);
/* Kernel launches one step makes with the current variant: the tile
 * variants launch the tile kernel plus one kernel per non-empty list of
 * boundary cells (and the wall-tile kernel in 2-D variants 5..12, the
 * collision kernel in 3-D variants 4..5); curved walls add the ghost-fill
 * kernel. */
int lbfd_launches_per_step(const lbfd_handle* h);

/* Autotuner: time every variant over `reps` launches on the current state
 * (the output buffer is overwritten, the state does not advance), select
 * the fastest and return it in *best; ms_per_variant (may be NULL) gets
 * lbfd_num_variants(h) mean launch times [ms].  Synchronises. */
int lbfd_autotune(lbfd_handle* h, int reps, double* ms_per_variant, int* best);

/* Copy one field (LBFD_FIELD_*) of all N cells to host FP64 out[N].
 * Synchronises the handle's stream. */
int lbfd_read_field(lbfd_handle* h, int field, double* out);

/* Copy the whole current state of n listed cells to host FP64
 * out[n][Q + 1 + 5]: per cell g_0 .. g_{Q-1} (the stored post-collision
 * populations, Eq. 14), T, Y_0 .. Y_4.  cells: host array of n cell
 * indices c = x + nx (y + ny z), each in [0, N) (else LBFD_EINVAL, nothing
 * copied).  Both arrays are caller-owned; the call allocates device scratch
 * for its duration and synchronises the handle's stream.  Lets a caller
 * inspect a few cells of a large grid without copying the whole state. */
int lbfd_read_cells(lbfd_handle* h, const long long* cells, long long n, double* out);

/* Reductions over fluid cells in FP64 (warp shuffles + atomics), out[LBFD_NDIAG]
 * as listed above.  Synchronises; returns LBFD_ENONFINITE (after filling out)
 * when a fluid cell holds a non-finite value. */
int lbfd_diagnostics(lbfd_handle* h, double* out);

/* lbfd_diagnostics restricted to the rows y0 <= y < y1 (all x and z), e.g.
 * one channel of a batch packed along y; x_f is normalised by the fluid
 * cells of that part of the x = 0 section and LBFD_DIAG_XHRR uses the line
 * y = (y0 + y1)/2.  EINVAL unless 0 <= y0 < y1 <= ny. */
int lbfd_diagnostics_rows(lbfd_handle* h, int y0, int y1, double* out);

/* Reaction front per column, for the dead zone of Sec. IV.A (2-D,
 * LBFD_FP64 or LBFD_MIXED): for every column x, the peak of LBFD_FIELD_HRR
 * over the fluid cells of rows y0 <= y < y1 (one channel of a packed batch)
 * into host peak[nx] (0 for a column without fluid there), and the distance
 * from that cell's centre to the nearer edge of the row band (the walls lie
 * half-way between cells: min(y - y0 + 1/2, y1 - 1/2 - y); the smallest y
 * on ties) into host wall_distance[nx].  The dead-zone thickness delta_dead
 * is the smallest such distance over the columns where the front burns
 * (channels.py takes the columns whose peak is at least 10 % of the
 * channel's largest).  Synchronises.  EINVAL unless 0 <= y0 < y1 <= ny;
 * ENOTSUP in 3-D and the tangent precisions. */
int lbfd_column_peaks(lbfd_handle* h, int y0, int y1, double* peak, double* wall_distance);

/* Change the inlet velocity of subsequent steps (the flow rate control that
 * holds a flame in place, Sec. IV.A).  EUNSTABLE if |u_in| >= cs.  A
 * captured step graph is re-captured at its next use. */
int lbfd_set_inlet_velocity(lbfd_handle* h, double u_in);

/* Flame position x_f [m] (LBFD_DIAG_XF times dx), fluid mass sum rho and
 * total heat release (LBFD_DIAG_HRR).  Any pointer may be NULL. */
int lbfd_flame_position(lbfd_handle* h, double* x_f, double* mass, double* heat_release);

/* Tangent precision only: derivative k (0..3, order of theta) of a raw
 * field (LBFD_FIELD_T, LBFD_FIELD_Y0 + k, LBFD_FIELD_G0 + i) of all cells
 * into host out[N].  The state set by lbfd_init_fields/lbfd_set_state has
 * zero derivatives; every step propagates them exactly (the derivative of
 * the discrete step; branch decisions are taken on the values).
 * Synchronises. */
int lbfd_read_tangent(lbfd_handle* h, int field, int k, double* out);

/* Tangent precision only: objective J (LBFD_OBJ_*) of the current state and
 * its gradient dJ/dtheta[4] (the forward-mode derivatives carried by the
 * state).  Either pointer may be NULL.  Synchronises. */
int lbfd_gradient(lbfd_handle* h, int objective, double* value, double* grad);

/* Discrete adjoint (reverse mode) of the coupled step, 2-D handles with
 * staircase walls, LBFD_FP64 or LBFD_MIXED (FP32 forward pass).  The
 * gradient of an objective J (LBFD_OBJ_FLAME_POSITION, x_f [m], or
 * LBFD_OBJ_QUENCH_DISTANCE) of the state after n steps with respect to
 * theta = (ln A, Ta, T_wall, u_in) is the adjoint recursion
 * lambda^n = (dF/dx^n)^T lambda^{n+1} run backwards from
 * lambda^N = dJ/dx^N, plus (dF/dtheta)^T lambda^{n+1} summed over the steps
 * (and J's own dependence on theta).  Each step's adjoint is taken by
 * recording every fluid cell's step on a reverse-mode tape and sweeping it
 * backwards: the exact transpose of the derivative of the discrete step,
 * branches taken on the values.  The forward pass keeps a copy of the state
 * every `checkpoint_every` steps; the backward pass recomputes each segment
 * from its copy with the forward kernels (FP32 ones for LBFD_MIXED) and
 * evaluates every step's adjoint at that trajectory, the step recorded in
 * FP64 (in FP32 for LBFD_MIXED: FP32 values and partials), accumulating
 * lambda and the gradient in FP64.
 *
 * lbfd_adjoint_setup: the checkpoint interval of later calls (default 200).
 * lbfd_adjoint_record: advance the handle's state by `steps` steps, keeping
 *   the checkpoints (steps/checkpoint_every state copies in device memory,
 *   held by the handle until lbfd_adjoint_backward or the next record), and
 *   return J of the final state in *value.
 * lbfd_adjoint_backward: the sweep over the recorded steps with
 *   lambda^N = seed * dJ/dx^N; grad[4] = seed * dJ/dtheta.  Frees the
 *   record.  The forward/backward split serves reverse-mode frameworks
 *   (the backward call receives the incoming gradient as seed).
 * lbfd_adjoint_run: record followed by backward with seed 1.
 * lbfd_adjoint_gradient: lbfd_adjoint_run with this checkpoint interval
 *   for the one call.
 * Device memory of a backward call: checkpoint_every + 2 state copies and
 *   two FP64 adjoint states, plus tapes of at most 12 GB: 20 B (12 B for
 *   LBFD_MIXED) x 2048 nodes per cell and recorded step, in two buffers of up to 4 steps each (one
 *   recorded while the other is swept) when they fit, else one step with
 *   its cells in chunks; and 8 B x 2048 nodes per cell for the sweep.  A
 *   step that needs more nodes is taken again with 4096.  Freed before
 *   returning.  All synchronise.
 * Errors: LBFD_EINVAL (arguments, backward without a record), LBFD_ENOTSUP
 * (other precision, 3-D, curved walls, or a cell whose step needs more than
 * 4096 nodes), LBFD_ENOMEM, LBFD_ECUDA (also for LBFD_MIXED when four
 * recorded states hold 2^31 elements or more: the FP32 tape names state
 * elements in 31 bits). */
int lbfd_adjoint_setup(lbfd_handle* h, int checkpoint_every);
int lbfd_adjoint_record(lbfd_handle* h, int steps, int objective, double* value);
int lbfd_adjoint_backward(lbfd_handle* h, double seed, double* grad);
int lbfd_adjoint_run(lbfd_handle* h, int steps, int objective, double* value, double* grad);
int lbfd_adjoint_gradient(lbfd_handle* h, int steps, int checkpoint_every, int objective, double* value,
                          double* grad);

/* Raw state in storage precision (4 or 8 bytes per value; 40 for tangent):
 * layout g[Q][N], T[N], Y[nsp][N], contiguous; lbfd_state_bytes gives the size.
 * The host buffer may be pageable or pinned; the copy is ordered on the
 * handle's stream and the call synchronises it. */
size_t lbfd_state_bytes(const lbfd_handle* h);
int lbfd_get_state_raw(lbfd_handle* h, void* host_dst, size_t bytes);
int lbfd_set_state_raw(lbfd_handle* h, const void* host_src, size_t bytes);

/* Diagnostics without any allocation, for callers that cannot call
 * cudaMalloc: code running where the device memory belongs to someone else
 * (a host framework's pool, a plugin with a fixed budget), code that must
 * not trigger the device-wide synchronisation of cudaMalloc/cudaFree in a
 * latency-bound loop, or code that may not fail on memory pressure after
 * start-up.  The paper has no counterpart; it is an interface variant of
 * lbfd_diagnostics and returns the same LBFD_NDIAG values (sums are FP64 in
 * both; they may differ by the rounding of the atomic accumulation order).
 *
 * Inputs are the caller's: g, T, Y are DEVICE pointers to the state planes
 * in storage precision (params->precision: 8-byte or 4-byte values),
 * plane k of g at g + k*plane_stride values, Y likewise; solid is a DEVICE
 * pointer to nx*ny*nz mask bytes; stream is a cudaStream_t (NULL: legacy
 * default stream).  out is a HOST array of LBFD_NDIAG doubles.  The call
 * synchronises the stream.
 *
 * Scratch: a file-scope device array of LBFD_NOALLOC_SCRATCH_WORDS doubles
 * (512 bytes) that every GPU which loads the library holds until the
 * process exits.  The call needs 16 words for any grid size; a request
 * needing more than the array holds is rejected with LBFD_EINVAL and a
 * message in lbfd_last_error().  Every call on a device shares the array,
 * which keeps the last call's contents; the words are cleared at the start
 * of each call, so calls that overlap on the GPU (two streams, two host
 * threads) race and must be serialised by the caller.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and
 * caches it; make that first call before any stream capture.  No cudaMalloc,
 * cudaFree or allocating library routine is called.  The call copies the
 * sums to the host and synchronises the stream, so it cannot be made while
 * the stream is being captured into a CUDA graph.  The cached address
 * belongs to the device's context: a cudaDeviceReset of that device while
 * the library is loaded is not supported.
 * Errors: EINVAL (null or non-device pointer, plane_stride < cells, invalid
 * grid/parameters as in lbfd_create), EUNSTABLE/ENOTSUP as lbfd_create,
 * ECUDA, ENONFINITE (after filling out). */
#define LBFD_NOALLOC_SCRATCH_WORDS 64
int lbfd_diagnostics_noalloc(const lbfd_grid* grid, const lbfd_mechanism* mech,
                             const lbfd_params* params, const void* g, const void* T,
                             const void* Y, long long plane_stride, const uint8_t* solid,
                             void* stream, double* out);

/* Checkpoint of the current state to a file and back: a header (magic
 * "LBFDCKPT", version 1, dim, nx, ny, nz, Q, species, precision, bytes per
 * value, the step counter, the state size) followed by the raw state of
 * lbfd_get_state_raw.  lbfd_load accepts only a file written for the same
 * grid, lattice and precision (else LBFD_EINVAL with the reason in
 * lbfd_last_error()), restores the state and the step counter (resume).
 * Both synchronise. */
int lbfd_save(lbfd_handle* h, const char* path);
int lbfd_load(lbfd_handle* h, const char* path);

/* Create one handle for n 2-D channels of uneven width run together (the
 * batching of Sec. IV.A's channel study): channel j has widths[j] rows and
 * `length` columns; the channels are stacked along y in one masked domain
 * with one solid row between neighbours, so that no stencil or population
 * couples them (with isothermal solids at the wall temperature each row of
 * solid acts as the walls of both channels).  proto gives dim (2) and the
 * face types and wall temperatures; nx, ny, nz are set here.  rows[2 j],
 * rows[2 j + 1] receive the first and one-past-last row of channel j (the
 * rows argument of lbfd_diagnostics_rows, lbfd_column_peaks).  Errors as
 * lbfd_create; ENOTSUP unless dim == 2. */
int lbfd_batch_create(int n, const int* widths, int length, const lbfd_grid* proto, const lbfd_mechanism* mech,
                      const lbfd_params* params, lbfd_handle** out, int* rows);

/* Curved walls (Sec. III): n analytic primitives, 5 doubles each,
 *   {0, cx, cy, cz, r}: sphere (circle in 2-D), solid inside;
 *   {1, nx, ny, nz, d}: half-space, unit normal pointing into the solid,
 *                      solid where n.x > d;
 * in lattice coordinates with the centre of cell (x, y, z) at
 * (x+1/2, y+1/2, z+1/2) (z ignored in 2-D).  The solid mask given to
 * lbfd_create stays the definition of solid cells and should agree with the
 * primitives.  Every population pulled from a solid cell then uses the
 * interpolated bounce-back of Eq. 29 with the wall distance q of its link
 * (Eq. 30; half-way bounce-back when the link meets no primitive), and the
 * FD stencils read, at solid cells within two cells of fluid, image-point
 * ghost values (Eq. 34): the mirror image across the nearest wall point,
 * valued by Shepard inverse-distance weighting (p = 2) of the fluid cells
 * within 4 dr (Eq. 35-38; the density reconstructed itself).  Domain faces
 * keep their own rules.  n = 0 restores staircase walls.  Computes the
 * tables on the host; adds a ghost-fill launch to every step. */
int lbfd_set_curved_walls(lbfd_handle* h, int n, const double* prims);

/* Counters and sizes. */
long long lbfd_steps_done(const lbfd_handle* h);
long long lbfd_num_cells(const lbfd_handle* h);
int lbfd_num_populations(const lbfd_handle* h);

const char* lbfd_strerror(int status);
/* text of the last CUDA failure on this thread ("" when none) */
const char* lbfd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBFD_H */
