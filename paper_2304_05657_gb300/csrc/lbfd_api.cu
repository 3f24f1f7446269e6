// lbfd_api.cu -- host side of the C ABI declared in include/lbfd.h.
//
// The handle owns a double-buffered device state (populations and scalar
// fields in SoA planes), the solid mask, the per-cell interior flags and
// boundary lists, a small reduction scratch and a read-out buffer.  All
// arithmetic of a step runs in the kernels; this file validates, converts
// parameters to lattice units, moves data, launches, and drives the
// checkpointed backward sweep of the discrete adjoint.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <iterator>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbfd.h"
#include "lbfd_internal.h"

using lbfd::StateView;
using lbfd::StepParams;
using lbfd::Tan;
using lbfd::Tanf;

struct lbfd_handle {
    lbfd_grid grid;
    lbfd_mechanism mech;
    lbfd_params prm;
    int dim, Q, precision;
    long long ncell, stride;
    size_t esz;           // bytes per stored value
    size_t planes;        // Q + 1 + NSP
    void* buf[2];         // device state buffers
    int cur;
    uint8_t* solid;       // device mask
    long long* bnd;       // device list of the cells the tile kernels skip
    long long nbnd;
    long long* bndf;      // the subset near domain faces (wall-aware 2-D tiles)
    long long nbndf;
    long long* bndw;      // 3-D: the others (next to in-domain solids only)
    long long nbndw;
    unsigned long long* bndw_code;  // 3-D: their neighbourhood codes
    long long* bndfc;     // 3-D: the cells near faces that take the coded form (staircase walls)
    long long nbndfc;
    unsigned long long* bndfc_code;
    long long* bndfg;     // 3-D: the other cells near faces (general form)
    long long nbndfg;
    uint8_t* interior;    // per cell, 1 = updated by the interior tile kernels
    void* aux;            // 3-D: Lambda and grad rho planes of the split variants
    int* wtiles;          // tiles holding the other boundary cells (2-D)
    long long nwtiles;
    double* red;          // device reduction scratch
    double* tmp;          // device read-out buffer (ncell doubles)
    cudaStream_t stream;
    long long steps;
    int variant;          // kernel variant (lbfd::launch_step)
    StepParams<double> Pd;
    StepParams<float> Pf;
    StepParams<lbfd::Tan> Pt;    // tangent precision: parameters with their seeds
    StepParams<lbfd::Tanf> Ptf;  // mixed tangent precision
    double section;            // fluid cells of the x = 0 section
    // CUDA graph of `graph_n` steps starting from buffer `graph_parity`
    cudaGraphExec_t graph;
    int graph_n, graph_parity, graph_variant;
    cudaStream_t graph_stream;  // stream the graph was captured on
    cudaStream_t own_stream;    // created when capture needs a non-legacy stream
    lbfd::SideStream side;      // boundary kernel next to the tile kernel
    std::vector<uint8_t> mask_host;
    // curved walls: device tables and the per-step ghost values
    int* link_row;
    double* link_q;
    int* ghost_row;
    long long *gh_start, *gh_idx;
    double* gh_w;
    void* gval;
    long long nghost;
    // persistent step: barrier words and the bound of each grid-wide wait
    lbfd::PersistentWait* pwait;
    long long wait_limit_ns;
    // quenching-distance objective: per-cell wall weights d^-4 (device)
    double* qwgt;
    // discrete adjoint: checkpoint interval and the recorded forward run
    int adj_K;
    char* adj_ck;      // one state copy per segment (storage precision)
    int adj_steps, adj_nseg, adj_obj;
    double adj_J;
};

namespace {

// NVTX range around an entry point (visible in a profiler timeline; no
// cost without one attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

thread_local char g_last_error[512] = "";

int cuda_fail(cudaError_t e, const char* what)
{
    snprintf(g_last_error, sizeof g_last_error, "%s: %s", what, cudaGetErrorString(e));
    return LBFD_ECUDA;
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
    } while (0)

StateView view(const lbfd_handle* h, int which)
{
    char* base = (char*)h->buf[which];
    const size_t plane = (size_t)h->stride * h->esz;
    StateView v;
    v.g = base;
    v.T = base + plane * h->Q;
    v.Y = base + plane * (h->Q + 1);
    return v;
}

template <typename R>
void fill_params(const lbfd_handle* h, StepParams<R>& P)
{
    const lbfd_grid& G = h->grid;
    const lbfd_mechanism& M = h->mech;
    const lbfd_params& p = h->prm;
    memset(&P, 0, sizeof P);
    P.dim = G.dim;
    P.nx = G.nx;
    P.ny = G.ny;
    P.nz = G.dim == 3 ? G.nz : 1;
    P.ncell = h->ncell;
    P.N = h->stride;
    for (int f = 0; f < 6; ++f) {
        P.bc[f] = (f < 2 * G.dim) ? G.bc[f] : LBFD_BC_PERIODIC;
        P.T_wall[f] = (R)G.T_wall[f];
    }
    const double cs2 = 1.0 / 3.0;
    const double alpha = p.nu / p.Pr;
    double invW_in = 0.0;
    for (int k = 0; k < lbfd::NSP; ++k) invW_in += p.Y_in[k] / M.W[k];
    const double yF = -M.nu_stoich[M.fuel] * M.W[M.fuel];
    for (int k = 0; k < lbfd::NSP; ++k) {
        P.inv_Wk[k] = (R)(1.0 / M.W[k]);
        P.yield[k] = (R)(M.nu_stoich[k] * M.W[k] / yF);
        P.a_diff[k] = (R)(alpha / M.Le[k] * M.W[k]);
        P.a12[k] = (R)(alpha / M.Le[k] / 12.0);
        P.Y_in[k] = (R)p.Y_in[k];
    }
    P.fuel = M.fuel;
    P.oxid = M.oxidiser;
    P.A_lat = (R)(M.A * p.dt);
    P.Ta = (R)M.Ta;
    P.Q_cp = (R)(M.Q / M.cp);
    P.A_lat_d = M.A * p.dt;
    P.Ta_d = M.Ta;
    P.T_fp64 = (R)p.T_fp64;
    const double omega_s = 1.0 / (p.nu / cs2 + 0.5);  // Eq. 18 read as 1/tau
    P.omega_s = (R)omega_s;
    P.omega_b = (R)(p.omega_bulk > 0.0 ? p.omega_bulk : omega_s);
    P.omega_hi = (R)p.omega_hi;
    P.alpha = (R)alpha;
    P.alpha12 = (R)(alpha / 12.0);
    {
        double ly = 0.0;
        for (int k = 0; k < lbfd::NSP; ++k) ly += M.nu_stoich[k] / yF;  // yield_k / W_k
        P.lam_yield = (R)ly;
    }
    P.u_in = (R)p.u_in;
    P.T_in = (R)p.T_in;
    P.invW_in = (R)invW_in;
    P.rho_in = (R)1.0;  // EOS reference state (T_in, Y_in)
    P.T_solid = (R)p.T_solid;
    P.solid_isothermal = p.solid_isothermal;
    P.poiseuille = p.poiseuille_inlet;
    for (int f = 0; f < 6; ++f) {
        const int b = P.bc[f];
        P.face_solid[f] = (b == LBFD_BC_WALL_ISOTHERMAL && p.solid_isothermal && G.T_wall[f] == p.T_solid) ||
                          (b == LBFD_BC_WALL_ADIABATIC && !p.solid_isothermal);
    }
    P.epsY = (R)p.weno_eps;
    P.epsT = (R)(p.weno_eps * p.T_in * p.T_in);
    P.cs = (R)sqrt(cs2);
}

static bool is_tangent(int precision) { return precision == LBFD_TANGENT || precision == LBFD_TANGENT_MIXED; }

// derivative directions of the tangent precisions: (ln A, Ta, T_wall, u_in)
template <typename TT>
void seed_tangents(const lbfd_handle* h, StepParams<TT>& P)
{
    P.A_lat.d[0] = P.A_lat.v;  // d(A dt)/d(ln A)
    P.Ta.d[1] = 1.0;
    for (int f = 0; f < 6; ++f)
        if (P.bc[f] == LBFD_BC_WALL_ISOTHERMAL) P.T_wall[f].d[2] = 1.0;
    if (h->prm.solid_isothermal) P.T_solid.d[2] = 1.0;
    P.u_in.d[3] = 1.0;
}

int validate(const lbfd_grid* G, const lbfd_mechanism* M, const lbfd_params* p)
{
    if (G->dim != 2 && G->dim != 3) return LBFD_EINVAL;
    if (G->nx < 1 || G->ny < 1 || (G->dim == 3 && G->nz < 1)) return LBFD_EINVAL;
    if ((long long)G->nx * G->ny * (G->dim == 3 ? G->nz : 1) > (1ll << 40)) return LBFD_EINVAL;
    for (int f = 0; f < 2 * G->dim; ++f) {
        if (G->bc[f] < LBFD_BC_PERIODIC || G->bc[f] > LBFD_BC_OUTLET_PRESSURE) return LBFD_EINVAL;
        const int o = f ^ 1;  // periodic faces come in pairs
        if ((G->bc[f] == LBFD_BC_PERIODIC) != (G->bc[o] == LBFD_BC_PERIODIC)) return LBFD_EINVAL;
        if (G->bc[f] == LBFD_BC_WALL_ISOTHERMAL && !(G->T_wall[f] > 0.0)) return LBFD_EINVAL;
    }
    if (M->n_species != lbfd::NSP) return LBFD_ENOTSUP;
    if (M->fuel < 0 || M->fuel >= lbfd::NSP || M->oxidiser < 0 || M->oxidiser >= lbfd::NSP ||
        M->fuel == M->oxidiser)
        return LBFD_EINVAL;
    if (!(M->nu_stoich[M->fuel] < 0.0)) return LBFD_EINVAL;
    for (int k = 0; k < lbfd::NSP; ++k)
        if (!(M->W[k] > 0.0) || !(M->Le[k] > 0.0)) return LBFD_EINVAL;
    if (!(M->A >= 0.0) || !(M->Ta >= 0.0) || !(M->cp > 0.0) || !std::isfinite(M->Q)) return LBFD_EINVAL;
    if (!(p->T_in > 0.0) || !(p->dt > 0.0) || !(p->Pr > 0.0) || !(p->weno_eps > 0.0)) return LBFD_EINVAL;
    if (p->precision != LBFD_FP64 && p->precision != LBFD_MIXED && !is_tangent(p->precision)) return LBFD_EINVAL;
    if (is_tangent(p->precision) && G->dim != 2) return LBFD_ENOTSUP;
    double ysum = 0.0;
    for (int k = 0; k < lbfd::NSP; ++k) ysum += p->Y_in[k];
    if (fabs(ysum - 1.0) > 1e-6) return LBFD_EINVAL;
    // stability limits
    if (!(p->nu > 0.0)) return LBFD_EUNSTABLE;
    const double omega_s = 1.0 / (3.0 * p->nu + 0.5);
    if (!(omega_s > 0.0 && omega_s < 2.0)) return LBFD_EUNSTABLE;
    if (p->omega_bulk > 0.0 && !(p->omega_bulk < 2.0)) return LBFD_EUNSTABLE;
    if (!(p->omega_hi > 0.0 && p->omega_hi < 2.0)) return LBFD_EUNSTABLE;
    if (!(fabs(p->u_in) < sqrt(1.0 / 3.0))) return LBFD_EUNSTABLE;
    double dmax = p->nu / p->Pr;
    for (int k = 0; k < lbfd::NSP; ++k) dmax = fmax(dmax, p->nu / p->Pr / M->Le[k]);
    // explicit Euler with the 4th-order Laplacian: |eigenvalue| <= dim * 64/12
    if (!(dmax * G->dim * 64.0 / 12.0 < 2.0)) return LBFD_EUNSTABLE;
    return LBFD_OK;
}

void free_handle(lbfd_handle* h)
{
    if (!h) return;
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    if (h->side.stream) cudaStreamDestroy(h->side.stream);
    if (h->side.fork) cudaEventDestroy(h->side.fork);
    if (h->side.join) cudaEventDestroy(h->side.join);
    for (int b = 0; b < 2; ++b)
        if (h->buf[b]) cudaFree(h->buf[b]);
    if (h->solid) cudaFree(h->solid);
    if (h->red) cudaFree(h->red);
    if (h->tmp) cudaFree(h->tmp);
    if (h->bnd) cudaFree(h->bnd);
    if (h->bndf) cudaFree(h->bndf);
    if (h->bndw) cudaFree(h->bndw);
    if (h->bndw_code) cudaFree(h->bndw_code);
    if (h->bndfc) cudaFree(h->bndfc);
    if (h->bndfc_code) cudaFree(h->bndfc_code);
    if (h->bndfg) cudaFree(h->bndfg);
    if (h->interior) cudaFree(h->interior);
    if (h->aux) cudaFree(h->aux);
    if (h->wtiles) cudaFree(h->wtiles);
    if (h->pwait) cudaFree(h->pwait);
    if (h->qwgt) cudaFree(h->qwgt);
    if (h->adj_ck) cudaFree(h->adj_ck);
    void* curved[] = {h->link_row, h->link_q, h->ghost_row, h->gh_start, h->gh_idx, h->gh_w, h->gval};
    for (void* p : curved)
        if (p) cudaFree(p);
    delete h;
}

// host values (double, dense planes) -> storage precision -> device buffer `which`
int upload_planes(lbfd_handle* h, int which, int first_plane, int nplanes, const double* src)
{
    const size_t n = (size_t)h->ncell;
    std::vector<char> stage(n * h->esz * nplanes);
    if (h->precision == LBFD_FP64) {
        memcpy(stage.data(), src, n * sizeof(double) * nplanes);
    } else if (h->precision == LBFD_MIXED) {
        float* d = (float*)stage.data();
        for (size_t i = 0; i < n * nplanes; ++i) d[i] = (float)src[i];
    } else if (h->precision == LBFD_TANGENT) {  // the given state carries no derivative
        Tan* d = (Tan*)stage.data();
        for (size_t i = 0; i < n * nplanes; ++i) d[i] = Tan(src[i]);
    } else {
        Tanf* d = (Tanf*)stage.data();
        for (size_t i = 0; i < n * nplanes; ++i) d[i] = Tanf(src[i]);
    }
    char* dst = (char*)h->buf[which] + (size_t)first_plane * h->stride * h->esz;
    CK(cudaMemcpy2DAsync(dst, (size_t)h->stride * h->esz, stage.data(), n * h->esz, n * h->esz, nplanes,
                         cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBFD_OK;
}

int sync_other_buffer(lbfd_handle* h)
{
    const size_t bytes = h->planes * (size_t)h->stride * h->esz;
    CK(cudaMemcpyAsync(h->buf[h->cur ^ 1], h->buf[h->cur], bytes, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBFD_OK;
}

// the boundary lists of the current geometry: with curved walls every cell
// next to a solid goes through the general form
lbfd::BoundaryLists lists(const lbfd_handle* h)
{
    lbfd::BoundaryLists b;
    b.all = h->bnd;
    b.nall = h->nbnd;
    const bool curved = h->nghost > 0 || h->Pd.curved;
    b.face = curved ? h->bnd : h->bndf;
    b.nface = curved ? h->nbnd : h->nbndf;
    b.wall_tiles = h->wtiles;
    b.nwall_tiles = curved ? 0 : h->nwtiles;
    b.wall = nullptr;
    b.nwall = 0;
    b.wall_code = nullptr;
    b.face_coded = nullptr;
    b.nface_coded = 0;
    b.face_code = nullptr;
    if (h->dim == 3) {  // the general form takes curved walls in both lists
        b.face = h->bndf;
        b.nface = h->nbndf;
        b.wall = h->bndw;
        b.nwall = h->nbndw;
        b.wall_code = h->bndw_code;
        if (!curved) {  // staircase walls: most cells near faces take their codes
            b.face = h->bndfg;
            b.nface = h->nbndfg;
            b.face_coded = h->bndfc;
            b.nface_coded = h->nbndfc;
            b.face_code = h->bndfc_code;
        }
    }
    b.interior = h->interior;
    b.aux = h->aux;
    return b;
}

// one step from buffer `from` to buffer `from ^ 1` with kernel variant v
cudaError_t launch_one(lbfd_handle* h, int from, int v, cudaStream_t s)
{
    if (h->nghost > 0) {  // image-point ghost values of the input state
        cudaError_t e = lbfd::launch_ghost_fill(h->precision, h->Pd, h->Pf, h->Pt, view(h, from), h->gh_start,
                                                h->gh_idx, h->gh_w, h->nghost, s);
        if (e != cudaSuccess) return e;
    }
    if (h->precision == LBFD_TANGENT)
        return lbfd::launch_step_tangent(h->dim, h->Pt, view(h, from), view(h, from ^ 1), h->solid, s);
    if (h->precision == LBFD_TANGENT_MIXED)
        return lbfd::launch_step_tangent(h->dim, h->Ptf, view(h, from), view(h, from ^ 1), h->solid, s);
    return lbfd::launch_step(h->dim, h->precision, v, h->Pd, h->Pf, view(h, from), view(h, from ^ 1), h->solid,
                             lists(h), h->side, s);
}

int num_variants_of(const lbfd_handle* h)
{
    return is_tangent(h->precision) ? 1 : lbfd::num_variants(h->dim);
}

}  // namespace

extern "C" {

const char* lbfd_strerror(int s)
{
    switch (s) {
    case LBFD_OK: return "ok";
    case LBFD_EINVAL: return "invalid argument";
    case LBFD_ENOMEM: return "out of memory";
    case LBFD_ECUDA: return "CUDA error";
    case LBFD_ENONFINITE: return "non-finite value in a fluid cell";
    case LBFD_ETIMEOUT: return "bounded device wait timed out";
    case LBFD_EUNSTABLE: return "parameters violate a stability limit";
    case LBFD_ENOTSUP: return "not supported by this build";
    default: return "unknown status";
    }
}

const char* lbfd_last_error(void) { return g_last_error; }

int lbfd_create(const lbfd_grid* grid, const uint8_t* solid_mask, const lbfd_mechanism* mech,
                const lbfd_params* params, lbfd_handle** out)
{
    if (!grid || !mech || !params || !out) return LBFD_EINVAL;
    *out = nullptr;
    int st = validate(grid, mech, params);
    if (st != LBFD_OK) return st;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1) {
        snprintf(g_last_error, sizeof g_last_error, "no CUDA device: %s",
                 e == cudaSuccess ? "device count is 0" : cudaGetErrorString(e));
        return LBFD_ECUDA;
    }
    lbfd_handle* h = new (std::nothrow) lbfd_handle();
    if (!h) return LBFD_ENOMEM;
    h->grid = *grid;
    if (grid->dim == 2) h->grid.nz = 1;
    h->mech = *mech;
    h->prm = *params;
    h->dim = grid->dim;
    h->Q = grid->dim == 2 ? 9 : 27;
    h->precision = params->precision;
    h->ncell = (long long)h->grid.nx * h->grid.ny * h->grid.nz;
    h->stride = (h->ncell + 63) / 64 * 64;  // 256-byte aligned FP32 planes
    h->esz = h->precision == LBFD_FP64 ? 8
             : h->precision == LBFD_MIXED ? 4
             : h->precision == LBFD_TANGENT ? sizeof(Tan) : sizeof(Tanf);
    h->planes = (size_t)h->Q + 1 + lbfd::NSP;
    h->stream = nullptr;
    h->variant = is_tangent(h->precision) ? 0 : 1;
    h->wait_limit_ns = 2000000000LL;  // 2 s per grid-wide wait of the persistent step
    h->adj_K = 200;
    const size_t bytes = h->planes * (size_t)h->stride * h->esz;
    for (int b = 0; b < 2; ++b) {
        e = cudaMalloc(&h->buf[b], bytes);
        if (e != cudaSuccess) {
            free_handle(h);
            cuda_fail(e, "cudaMalloc(state)");
            return LBFD_ENOMEM;
        }
    }
    if ((e = cudaMalloc(&h->solid, (size_t)h->ncell)) != cudaSuccess ||
        (e = cudaMalloc(&h->red, lbfd::RED_WORDS * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&h->tmp, (size_t)h->ncell * sizeof(double))) != cudaSuccess) {
        free_handle(h);
        cuda_fail(e, "cudaMalloc");
        return LBFD_ENOMEM;
    }
    fill_params(h, h->Pd);
    fill_params(h, h->Pf);
    fill_params(h, h->Pt);
    seed_tangents(h, h->Pt);
    fill_params(h, h->Ptf);
    seed_tangents(h, h->Ptf);
    // mask
    std::vector<uint8_t> m((size_t)h->ncell, 0);
    if (solid_mask)
        for (long long c = 0; c < h->ncell; ++c) m[c] = solid_mask[c] ? 1 : 0;
    if ((e = cudaMemcpy(h->solid, m.data(), (size_t)h->ncell, cudaMemcpyHostToDevice)) != cudaSuccess) {
        free_handle(h);
        return cuda_fail(e, "cudaMemcpy(mask)");
    }
    if (!is_tangent(h->precision) &&
        ((e = cudaDeviceGetStreamPriorityRange(&h->side.low, &h->side.priority)) != cudaSuccess ||
         (e = cudaStreamCreateWithPriority(&h->side.stream, cudaStreamNonBlocking, h->side.priority)) !=
             cudaSuccess ||
         (e = cudaEventCreateWithFlags(&h->side.fork, cudaEventDisableTiming)) != cudaSuccess ||
         (e = cudaEventCreateWithFlags(&h->side.join, cudaEventDisableTiming)) != cudaSuccess)) {
        free_handle(h);
        return cuda_fail(e, "side stream");
    }
    h->mask_host = m;
    h->section = 0.0;
    for (long long c = 0; c < h->ncell; c += h->grid.nx)
        if (!m[c]) h->section += 1.0;
    std::vector<long long> lists_host[2];
    for (int faces_only = 0; faces_only <= 1; ++faces_only) {
        std::vector<long long>& list = lists_host[faces_only];
        lbfd::boundary_cells(h->dim, h->grid.nx, h->grid.ny, h->grid.nz, h->Pd.bc, m.data(), list, faces_only != 0,
                             h->Pd.face_solid);
        long long** dst = faces_only ? &h->bndf : &h->bnd;
        (faces_only ? h->nbndf : h->nbnd) = (long long)list.size();
        if (list.empty()) continue;
        if ((e = cudaMalloc(dst, list.size() * sizeof(long long))) != cudaSuccess) {
            free_handle(h);
            cuda_fail(e, "cudaMalloc(boundary list)");
            return LBFD_ENOMEM;
        }
        if ((e = cudaMemcpy(*dst, list.data(), list.size() * sizeof(long long), cudaMemcpyHostToDevice)) !=
            cudaSuccess) {
            free_handle(h);
            return cuda_fail(e, "cudaMemcpy(boundary list)");
        }
    }
    {
        // per-cell flag of the cells the tile kernels update (fluid cells
        // outside the boundary list)
        std::vector<uint8_t> inter((size_t)h->ncell, 0);
        for (long long c = 0; c < h->ncell; ++c) inter[c] = m[c] ? 0 : 1;
        for (long long c : lists_host[0]) inter[c] = 0;
        if ((e = cudaMalloc(&h->interior, (size_t)h->ncell)) != cudaSuccess ||
            (e = cudaMemcpy(h->interior, inter.data(), (size_t)h->ncell, cudaMemcpyHostToDevice)) != cudaSuccess) {
            free_handle(h);
            return cuda_fail(e, "interior flags");
        }
    }
    if (h->dim == 3) {  // all \ face (both sorted)
        std::vector<long long> wl;
        std::set_difference(lists_host[0].begin(), lists_host[0].end(), lists_host[1].begin(), lists_host[1].end(),
                            std::back_inserter(wl));
        h->nbndw = (long long)wl.size();
        // class 2: next to in-domain solids, no domain face in reach (the
        // wall-aware tiles update these cells themselves)
        if (!wl.empty()) {
            std::vector<uint8_t> cls((size_t)h->ncell);
            if ((e = cudaMemcpy(cls.data(), h->interior, (size_t)h->ncell, cudaMemcpyDeviceToHost)) != cudaSuccess) {
                free_handle(h);
                return cuda_fail(e, "interior flags");
            }
            for (long long c : wl) cls[c] = 2;
            if ((e = cudaMemcpy(h->interior, cls.data(), (size_t)h->ncell, cudaMemcpyHostToDevice)) != cudaSuccess) {
                free_handle(h);
                return cuda_fail(e, "interior flags");
            }
        }
        // the Lambda / grad rho planes of the split variants
        if (!is_tangent(h->precision) &&
            (e = cudaMalloc(&h->aux, (size_t)4 * h->stride * h->esz)) != cudaSuccess) {
            free_handle(h);
            return cuda_fail(e, "split-step buffers");
        }
        {  // the cells near faces: coded where the coded form applies
            std::vector<long long> fc, fg;
            std::vector<unsigned long long> fcodes;
            lbfd::face_codes(h->grid.nx, h->grid.ny, h->grid.nz, h->Pd.bc, m.data(), lists_host[1], fc, fcodes, fg);
            h->nbndfc = (long long)fc.size();
            h->nbndfg = (long long)fg.size();
            if ((!fc.empty() &&
                 ((e = cudaMalloc(&h->bndfc, fc.size() * sizeof(long long))) != cudaSuccess ||
                  (e = cudaMemcpy(h->bndfc, fc.data(), fc.size() * sizeof(long long), cudaMemcpyHostToDevice)) !=
                      cudaSuccess ||
                  (e = cudaMalloc(&h->bndfc_code, fcodes.size() * sizeof(unsigned long long))) != cudaSuccess ||
                  (e = cudaMemcpy(h->bndfc_code, fcodes.data(), fcodes.size() * sizeof(unsigned long long),
                                  cudaMemcpyHostToDevice)) != cudaSuccess)) ||
                (!fg.empty() &&
                 ((e = cudaMalloc(&h->bndfg, fg.size() * sizeof(long long))) != cudaSuccess ||
                  (e = cudaMemcpy(h->bndfg, fg.data(), fg.size() * sizeof(long long), cudaMemcpyHostToDevice)) !=
                      cudaSuccess))) {
                free_handle(h);
                return cuda_fail(e, "face lists");
            }
        }
        if (!wl.empty()) {
            std::vector<unsigned long long> codes;
            lbfd::wall_codes(h->grid.nx, h->grid.ny, h->grid.nz, h->Pd.bc, m.data(), wl, codes);
            if ((e = cudaMalloc(&h->bndw, wl.size() * sizeof(long long))) != cudaSuccess ||
                (e = cudaMemcpy(h->bndw, wl.data(), wl.size() * sizeof(long long), cudaMemcpyHostToDevice)) !=
                    cudaSuccess ||
                (e = cudaMalloc(&h->bndw_code, codes.size() * sizeof(unsigned long long))) != cudaSuccess ||
                (e = cudaMemcpy(h->bndw_code, codes.data(), codes.size() * sizeof(unsigned long long),
                                cudaMemcpyHostToDevice)) != cudaSuccess) {
                free_handle(h);
                return cuda_fail(e, "wall list");
            }
        }
    }
    if (h->dim == 2) {
        std::vector<int> tiles;
        lbfd::wall_tiles(h->grid.nx, h->grid.ny, lists_host[0], lists_host[1], tiles);
        h->nwtiles = (long long)tiles.size();
        if (!tiles.empty()) {
            if ((e = cudaMalloc(&h->wtiles, tiles.size() * sizeof(int))) != cudaSuccess ||
                (e = cudaMemcpy(h->wtiles, tiles.data(), tiles.size() * sizeof(int), cudaMemcpyHostToDevice)) !=
                    cudaSuccess) {
                free_handle(h);
                return cuda_fail(e, "wall tiles");
            }
        }
    }
    // initial state: T_in, Y_in, g = 0
    h->cur = 0;
    if ((e = cudaMemset(h->buf[0], 0, bytes)) != cudaSuccess) {
        free_handle(h);
        return cuda_fail(e, "cudaMemset");
    }
    std::vector<double> TY((size_t)h->ncell * (1 + lbfd::NSP));
    for (long long c = 0; c < h->ncell; ++c) TY[c] = params->T_in;
    for (int k = 0; k < lbfd::NSP; ++k)
        for (long long c = 0; c < h->ncell; ++c) TY[(size_t)(k + 1) * h->ncell + c] = params->Y_in[k];
    st = upload_planes(h, 0, h->Q, 1 + lbfd::NSP, TY.data());
    if (st == LBFD_OK) st = sync_other_buffer(h);
    if (st != LBFD_OK) {
        free_handle(h);
        return st;
    }
    *out = h;
    return LBFD_OK;
}

int lbfd_destroy(lbfd_handle* h)
{
    if (!h) return LBFD_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    free_handle(h);
    return LBFD_OK;
}

int lbfd_set_stream(lbfd_handle* h, void* s)
{
    if (!h) return LBFD_EINVAL;
    h->stream = (cudaStream_t)s;
    return LBFD_OK;
}

int lbfd_set_state(lbfd_handle* h, const double* T, const double* Y, const double* g)
{
    if (!h || !T || !Y) return LBFD_EINVAL;
    const size_t n = (size_t)h->ncell;
    std::vector<double> all(n * h->planes, 0.0);
    if (g) memcpy(all.data(), g, n * h->Q * sizeof(double));
    memcpy(all.data() + n * h->Q, T, n * sizeof(double));
    memcpy(all.data() + n * (h->Q + 1), Y, n * lbfd::NSP * sizeof(double));
    int st = upload_planes(h, h->cur, 0, (int)h->planes, all.data());
    if (st != LBFD_OK) return st;
    return sync_other_buffer(h);
}

int lbfd_init_fields(lbfd_handle* h, const double* T, const double* Y)
{
    return lbfd_set_state(h, T, Y, nullptr);
}

int lbfd_step(lbfd_handle* h, int n)
{
    NvtxRange nvtx_("lbfd_step");
    if (!h || n < 0) return LBFD_EINVAL;
    for (int it = 0; it < n; ++it) {
        cudaError_t e = launch_one(h, h->cur, h->variant, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
        h->cur ^= 1;
        h->steps++;
    }
    return LBFD_OK;
}

int lbfd_step_graph(lbfd_handle* h, int n)
{
    NvtxRange nvtx_("lbfd_step_graph");
    if (!h || n < 1) return LBFD_EINVAL;
    cudaStream_t s = h->stream;
    if (s == nullptr) {  // the legacy default stream cannot be captured
        if (!h->own_stream) CK(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
        s = h->own_stream;
        CK(cudaDeviceSynchronize());
    }
    if (!h->graph || h->graph_n != n || h->graph_parity != h->cur || h->graph_variant != h->variant ||
        h->graph_stream != s) {
        if (h->graph) {
            cudaGraphExecDestroy(h->graph);
            h->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int cur = h->cur;
        cudaError_t le = cudaSuccess;
        for (int it = 0; it < n && le == cudaSuccess; ++it) {
            le = launch_one(h, cur, h->variant, s);
            cur ^= 1;
        }
        cudaError_t ee = cudaStreamEndCapture(s, &g);
        if (le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(le, "step launch during capture");
        }
        if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture");
        // honour the kernel nodes' priorities (boundary kernels ahead of the tiles)
        cudaError_t ie = cudaGraphInstantiate(&h->graph, g, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            h->graph = nullptr;
            return cuda_fail(ie, "cudaGraphInstantiate");
        }
        h->graph_n = n;
        h->graph_parity = h->cur;
        h->graph_variant = h->variant;
        h->graph_stream = s;
    }
    CK(cudaGraphLaunch(h->graph, s));
    if (s != h->stream) CK(cudaStreamSynchronize(s));
    h->cur ^= (n & 1);
    h->steps += n;
    return LBFD_OK;
}

int lbfd_set_wait_limit(lbfd_handle* h, long long ns)
{
    if (!h) return LBFD_EINVAL;
    h->wait_limit_ns = ns;
    return LBFD_OK;
}

int lbfd_step_persistent(lbfd_handle* h, int n)
{
    NvtxRange nvtx_("lbfd_step_persistent");
    if (!h || n < 0) return LBFD_EINVAL;
    if (h->dim != 2 || is_tangent(h->precision) || h->nghost > 0 || h->Pd.curved) return LBFD_ENOTSUP;
    if (n == 0) return LBFD_OK;
    if (!h->pwait) {
        if (cudaMalloc((void**)&h->pwait, sizeof(lbfd::PersistentWait)) != cudaSuccess) {
            h->pwait = nullptr;
            return LBFD_ENOMEM;
        }
    }
    int blocks = 0;
    cudaError_t e = lbfd::launch_step_persistent(h->precision, h->Pd, h->Pf, view(h, h->cur), view(h, h->cur ^ 1), n,
                                                 h->solid, lists(h), h->pwait, h->wait_limit_ns, h->stream, &blocks);
    if (e != cudaSuccess) return cuda_fail(e, "persistent step launch");
    lbfd::PersistentWait w{};
    CK(cudaMemcpyAsync(&w, h->pwait, sizeof w, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (w.error) {
        snprintf(g_last_error, sizeof g_last_error,
                 "persistent step: a grid-wide wait gave up at step %d of %d (%d blocks, limit %lld ns)", w.step, n,
                 blocks, h->wait_limit_ns);
        return LBFD_ETIMEOUT;
    }
    h->cur ^= (n & 1);
    h->steps += n;
    return LBFD_OK;
}

int lbfd_num_variants(const lbfd_handle* h) { return h ? num_variants_of(h) : -1; }

int lbfd_get_variant(const lbfd_handle* h) { return h ? h->variant : -1; }

int lbfd_launches_per_step(const lbfd_handle* h)
{
    if (!h) return -1;
    const lbfd::BoundaryLists b = lists(h);
    int n = 1;
    if (h->variant > 0 && !is_tangent(h->precision)) {
        if (h->dim == 3) {
            const bool wall_list = b.nwall > 0 && (h->variant < 6 || h->Pd.curved);
            n += (b.nface > 0 ? 1 : 0) + (b.nface_coded > 0 ? 1 : 0) + (wall_list ? 1 : 0) +
                 (h->variant == 4 || h->variant == 5 ? 1 : 0);
        } else {
            const bool wv = h->variant >= 5 && b.nwall_tiles > 0;
            n += ((wv ? b.nface : b.nall) > 0 ? 1 : 0) + (wv ? 1 : 0);
        }
    }
    return n + (h->nghost > 0 ? 1 : 0);
}

int lbfd_set_curved_walls(lbfd_handle* h, int n, const double* prims)
{
    if (!h || n < 0 || (n > 0 && !prims)) return LBFD_EINVAL;
    if (h->precision == LBFD_TANGENT_MIXED && n > 0) return LBFD_ENOTSUP;
    for (int k = 0; k < n; ++k) {
        const double* P = prims + 5 * k;
        const int t = (int)P[0];
        if (t != 0 && t != 1) return LBFD_EINVAL;
        if (t == 0 && !(P[4] > 0.0)) return LBFD_EINVAL;
        if (t == 1) {
            double nn = 0.0;
            for (int a = 0; a < h->dim; ++a) nn += P[1 + a] * P[1 + a];
            if (fabs(nn - 1.0) > 1e-9) return LBFD_EINVAL;
        }
    }
    CK(cudaStreamSynchronize(h->stream));
    void* old[] = {h->link_row, h->link_q, h->ghost_row, h->gh_start, h->gh_idx, h->gh_w, h->gval};
    for (void* p : old)
        if (p) cudaFree(p);
    h->link_row = nullptr;
    h->link_q = nullptr;
    h->ghost_row = nullptr;
    h->gh_start = h->gh_idx = nullptr;
    h->gh_w = nullptr;
    h->gval = nullptr;
    h->nghost = 0;
    h->Pd.curved = h->Pf.curved = h->Pt.curved = h->Ptf.curved = 0;
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    if (n == 0) return LBFD_OK;
    lbfd::CurvedTables t;
    lbfd::build_curved_tables(h->dim, h->grid.nx, h->grid.ny, h->grid.nz, h->grid.bc, h->mask_host.data(), n, prims,
                              t);
    auto upload = [&](void** dst, const void* src, size_t bytes) -> cudaError_t {
        if (bytes == 0) bytes = 8;  // keep a valid pointer for empty tables
        cudaError_t e = cudaMalloc(dst, bytes);
        if (e != cudaSuccess) return e;
        return src ? cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    CK(upload((void**)&h->link_row, t.link_row.data(), t.link_row.size() * sizeof(int)));
    CK(upload((void**)&h->link_q, t.link_q.empty() ? nullptr : t.link_q.data(), t.link_q.size() * sizeof(double)));
    CK(upload((void**)&h->ghost_row, t.ghost_row.data(), t.ghost_row.size() * sizeof(int)));
    CK(upload((void**)&h->gh_start, t.gh_start.data(), t.gh_start.size() * sizeof(long long)));
    CK(upload((void**)&h->gh_idx, t.gh_idx.empty() ? nullptr : t.gh_idx.data(), t.gh_idx.size() * sizeof(long long)));
    CK(upload((void**)&h->gh_w, t.gh_w.empty() ? nullptr : t.gh_w.data(), t.gh_w.size() * sizeof(double)));
    h->nghost = t.nghost;
    CK(upload(&h->gval, nullptr, (size_t)(h->nghost > 0 ? h->nghost : 1) * lbfd::GHOST_VALUES * h->esz));
    h->Pd.curved = h->Pf.curved = h->Pt.curved = 1;
    h->Pd.link_row = h->Pf.link_row = h->Pt.link_row = h->link_row;
    h->Pd.link_q = h->Pf.link_q = h->Pt.link_q = h->link_q;
    h->Pd.ghost_row = h->Pf.ghost_row = h->Pt.ghost_row = h->ghost_row;
    h->Pd.gval = (const double*)h->gval;
    h->Pf.gval = (const float*)h->gval;
    h->Pt.gval = (const Tan*)h->gval;
    return LBFD_OK;
}

int lbfd_set_variant(lbfd_handle* h, int variant)
{
    if (!h || variant < 0 || variant >= num_variants_of(h)) return LBFD_EINVAL;
    h->variant = variant;
    return LBFD_OK;
}

int lbfd_autotune(lbfd_handle* h, int reps, double* ms_per_variant, int* best)
{
    NvtxRange nvtx_("lbfd_autotune");
    if (!h || reps < 1) return LBFD_EINVAL;
    const int nv = num_variants_of(h);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int arg = h->variant;
    float best_ms = 3.4e38f;
    for (int v = 0; v < nv; ++v) {
        // the input buffer is never written: the state does not advance
        cudaError_t e = cudaSuccess;
        for (int r = 0; r < 2 && e == cudaSuccess; ++r)
            e = launch_one(h, h->cur, v, h->stream);
        cudaEventRecord(e0, h->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r)
            e = launch_one(h, h->cur, v, h->stream);
        cudaEventRecord(e1, h->stream);
        cudaError_t se = cudaEventSynchronize(e1);
        if (e != cudaSuccess || se != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(e != cudaSuccess ? e : se, "autotune");
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms_per_variant) ms_per_variant[v] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            arg = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->variant = arg;
    if (best) *best = arg;
    return LBFD_OK;
}


int lbfd_read_cells(lbfd_handle* h, const long long* cells, long long n, double* out)
{
    if (!h || n < 0 || (n > 0 && (!cells || !out))) return LBFD_EINVAL;
    if (n == 0) return LBFD_OK;
    for (long long t = 0; t < n; ++t)
        if (cells[t] < 0 || cells[t] >= h->ncell) return LBFD_EINVAL;
    const size_t per = (size_t)h->Q + 1 + lbfd::NSP;
    long long* dc = nullptr;
    double* dout = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&dc, (size_t)n * sizeof(long long))) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&dout, (size_t)n * per * sizeof(double))) != cudaSuccess) {
        cudaFree(dc);
        return cuda_fail(e, "cudaMalloc");
    }
    if ((e = cudaMemcpyAsync(dc, cells, (size_t)n * sizeof(long long), cudaMemcpyHostToDevice, h->stream)) ==
            cudaSuccess &&
        (e = lbfd::launch_cells(h->dim, h->precision, h->Pd, view(h, h->cur), dc, n, dout, h->stream)) ==
            cudaSuccess &&
        (e = cudaMemcpyAsync(out, dout, (size_t)n * per * sizeof(double), cudaMemcpyDeviceToHost, h->stream)) ==
            cudaSuccess)
        e = cudaStreamSynchronize(h->stream);
    cudaFree(dc);
    cudaFree(dout);
    if (e != cudaSuccess) return cuda_fail(e, "lbfd_read_cells");
    return LBFD_OK;
}

int lbfd_read_field(lbfd_handle* h, int field, double* out)
{
    if (!h || !out) return LBFD_EINVAL;
    const bool ok = (field >= 0 && field <= LBFD_FIELD_HRR) ||
                    (field >= LBFD_FIELD_G0 && field < LBFD_FIELD_G0 + h->Q);
    if (!ok) return LBFD_EINVAL;
    CK(lbfd::launch_field(h->dim, h->precision, h->Pd, view(h, h->cur), h->solid, field, h->tmp, h->stream));
    CK(cudaMemcpyAsync(out, h->tmp, (size_t)h->ncell * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBFD_OK;
}

int lbfd_diagnostics_rows(lbfd_handle* h, int y0, int y1, double* out)
{
    NvtxRange nvtx_("lbfd_diagnostics");
    if (!h || !out || y0 < 0 || y1 > h->grid.ny || y0 >= y1) return LBFD_EINVAL;
    double r[lbfd::RED_WORDS];
    CK(lbfd::launch_diagnostics(h->dim, h->precision, h->Pd, view(h, h->cur), h->solid, y0, y1, h->red, h->stream));
    CK(cudaMemcpyAsync(r, h->red, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    unsigned long long u[lbfd::RED_WORDS];
    memcpy(u, r, sizeof r);
    const double section = (double)u[7];
    const double yf_in = h->prm.Y_in[h->mech.fuel];
    out[LBFD_DIAG_XF] = section > 0.0 ? r[0] / (yf_in * section) : 0.0;
    out[LBFD_DIAG_MASS] = r[1];
    out[LBFD_DIAG_HRR] = r[2];
    out[LBFD_DIAG_FUEL] = r[3];
    {
        const unsigned long long k = u[4];
        double t;
        if (k == 0ull) {
            t = -INFINITY;
        } else {
            const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
            memcpy(&t, &b, sizeof t);
        }
        out[LBFD_DIAG_TMAX] = t;
    }
    out[LBFD_DIAG_XHRR] = r[9];
    out[LBFD_DIAG_NONFINITE] = (double)u[5];
    out[LBFD_DIAG_NFLUID] = (double)u[6];
    return u[5] ? LBFD_ENONFINITE : LBFD_OK;
}

int lbfd_column_peaks(lbfd_handle* h, int y0, int y1, double* peak, double* wall_distance)
{
    if (!h || !peak || !wall_distance || y0 < 0 || y1 > h->grid.ny || y0 >= y1) return LBFD_EINVAL;
    if (h->dim != 2 || (h->precision != LBFD_FP64 && h->precision != LBFD_MIXED)) return LBFD_ENOTSUP;
    const int nx = h->grid.nx;
    double* out = h->tmp;
    double* own = nullptr;
    if (h->ncell < 2LL * nx) {  // a one-row grid: tmp holds nx values only
        if (cudaMalloc((void**)&own, 2 * (size_t)nx * sizeof(double)) != cudaSuccess) return LBFD_ENOMEM;
        out = own;
    }
    std::vector<double> r(2 * (size_t)nx);
    cudaError_t e = lbfd::launch_column_peaks(h->precision, h->Pd, view(h, h->cur), h->solid, y0, y1, out, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r.data(), out, r.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (own) cudaFree(own);
    if (e != cudaSuccess) return cuda_fail(e, "column peaks");
    memcpy(peak, r.data(), (size_t)nx * sizeof(double));
    memcpy(wall_distance, r.data() + nx, (size_t)nx * sizeof(double));
    return LBFD_OK;
}

int lbfd_diagnostics(lbfd_handle* h, double* out)
{
    if (!h) return LBFD_EINVAL;
    return lbfd_diagnostics_rows(h, 0, h->grid.ny, out);
}

int lbfd_set_inlet_velocity(lbfd_handle* h, double u_in)
{
    if (!h) return LBFD_EINVAL;
    if (!(fabs(u_in) < sqrt(1.0 / 3.0))) return LBFD_EUNSTABLE;
    h->prm.u_in = u_in;
    h->Pd.u_in = u_in;
    h->Pf.u_in = (float)u_in;
    const double seed = h->Pt.u_in.d[3];
    h->Pt.u_in = Tan(u_in);
    h->Pt.u_in.d[3] = seed;
    const float seedf = h->Ptf.u_in.d[3];
    h->Ptf.u_in = Tanf(u_in);
    h->Ptf.u_in.d[3] = seedf;
    if (h->graph) {  // kernel parameters are baked into a captured graph
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    return LBFD_OK;
}

// the view of an FP64 state buffer laid out as the handle's
static StateView view_of(const lbfd_handle* h, void* base)
{
    const size_t plane = (size_t)h->stride * h->esz;
    StateView v;
    v.g = base;
    v.T = (char*)base + plane * h->Q;
    v.Y = (char*)base + plane * (h->Q + 1);
    return v;
}

// wall weights of the quenching-distance objective: d^-4 with d the distance
// (cells, to the wall plane half-way between cells) from a fluid cell to the
// nearest isothermal boundary along the axis directions: an isothermal solid
// cell, or the layer beyond an isothermal wall face (periodic axes wrap);
// 64 cells when there is none that close
static int quench_weights(lbfd_handle* h)
{
    if (h->qwgt) return LBFD_OK;
    const int nx = h->grid.nx, ny = h->grid.ny, nz = h->grid.nz, dim = h->dim;
    const int n[3] = {nx, ny, nz};
    const int* bc = h->grid.bc;
    const bool iso_solid = h->prm.solid_isothermal != 0;
    constexpr int CAP = 64;
    std::vector<double> w((size_t)h->stride, 0.0);
    for (long long c = 0; c < h->ncell; ++c) {
        if (h->mask_host[c]) continue;
        const int p[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long long)nx * ny))};
        double d = CAP;
        for (int a = 0; a < dim; ++a)
            for (int side = -1; side <= 1; side += 2)
                for (int j = 1; j <= CAP && j - 0.5 < d; ++j) {
                    int q[3] = {p[0], p[1], p[2]};
                    q[a] += side * j;
                    if (q[a] < 0 || q[a] >= n[a]) {
                        const int f = 2 * a + (q[a] < 0 ? 0 : 1);
                        if (bc[f] == LBFD_BC_PERIODIC) {
                            q[a] = ((q[a] % n[a]) + n[a]) % n[a];
                        } else {
                            if (bc[f] == LBFD_BC_WALL_ISOTHERMAL) d = j - 0.5;
                            break;
                        }
                    }
                    const long long e = (long long)q[0] + (long long)nx * ((long long)q[1] + (long long)ny * q[2]);
                    if (h->mask_host[e]) {
                        if (iso_solid) d = j - 0.5;
                        break;
                    }
                }
        w[c] = 1.0 / (d * d * d * d);
    }
    if (cudaMalloc((void**)&h->qwgt, w.size() * sizeof(double)) != cudaSuccess) {
        h->qwgt = nullptr;
        return LBFD_ENOMEM;
    }
    CK(cudaMemcpy(h->qwgt, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
    return LBFD_OK;
}

static bool adjoint_precision(const lbfd_handle* h) { return h->precision == LBFD_FP64 || h->precision == LBFD_MIXED; }

static void adjoint_release(lbfd_handle* h)
{
    if (h->adj_ck) cudaFree(h->adj_ck);
    h->adj_ck = nullptr;
    h->adj_steps = h->adj_nseg = 0;
}

int lbfd_adjoint_setup(lbfd_handle* h, int checkpoint_every)
{
    if (!h || checkpoint_every < 1) return LBFD_EINVAL;
    h->adj_K = checkpoint_every;
    return LBFD_OK;
}

int lbfd_adjoint_record(lbfd_handle* h, int steps, int objective, double* value)
{
    NvtxRange nvtx_("lbfd_adjoint_record");
    if (!h || steps < 1 || (objective != LBFD_OBJ_FLAME_POSITION && objective != LBFD_OBJ_QUENCH_DISTANCE))
        return LBFD_EINVAL;
    if (!adjoint_precision(h) || h->dim != 2 || h->nghost > 0 || h->Pd.curved) return LBFD_ENOTSUP;
    adjoint_release(h);
    const int K = h->adj_K < steps ? h->adj_K : steps;
    const int nseg = (steps + K - 1) / K;
    const size_t sbytes = h->planes * (size_t)h->stride * h->esz;
    if (objective == LBFD_OBJ_QUENCH_DISTANCE) {
        const int st = quench_weights(h);
        if (st != LBFD_OK) return st;
    }
    if (cudaMalloc((void**)&h->adj_ck, sbytes * nseg) != cudaSuccess) {
        h->adj_ck = nullptr;
        snprintf(g_last_error, sizeof g_last_error, "cudaMalloc(adjoint checkpoints, %zu bytes)", sbytes * nseg);
        return LBFD_ENOMEM;
    }
    // forward pass from the handle's state, one checkpoint per segment
    for (int g = 0; g < nseg; ++g) {
        CK(cudaMemcpyAsync(h->adj_ck + (size_t)g * sbytes, h->buf[h->cur], sbytes, cudaMemcpyDeviceToDevice,
                           h->stream));
        const int len = steps - g * K < K ? steps - g * K : K;
        const int st = lbfd_step(h, len);
        if (st != LBFD_OK) {
            adjoint_release(h);
            return st;
        }
    }
    double J = 0.0;
    if (objective == LBFD_OBJ_FLAME_POSITION) {
        double d[LBFD_NDIAG];
        const int dst = lbfd_diagnostics(h, d);
        if (dst != LBFD_OK) {
            adjoint_release(h);
            return dst;
        }
        J = d[LBFD_DIAG_XF] * h->prm.dx;
    } else {
        double r[2];
        CK(lbfd::launch_quench_sums(h->Pd, view(h, h->cur), h->precision == LBFD_MIXED, h->solid, h->qwgt, h->red,
                                    h->stream));
        CK(cudaMemcpyAsync(r, h->red, sizeof r, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        J = r[1] > 0.0 && r[0] > 0.0 ? pow(r[1] / r[0], -0.25) : 0.0;
    }
    h->adj_steps = steps;
    h->adj_nseg = nseg;
    h->adj_obj = objective;
    h->adj_J = J;
    if (value) *value = J;
    return LBFD_OK;
}

// One backward sweep with tapes of maxn nodes per thread; *overflow is set
// when a cell's step needed more.  The tapes of groups of steps are recorded
// on a second stream into two alternating buffers while the steps of the
// previous group are swept on the handle's stream (the record is bound by
// FP64 arithmetic, the sweep by latency: together they share the SMs).
static int adjoint_backward_pass(lbfd_handle* h, double seed, int maxn, double* grad, bool* overflow)
{
    const int steps = h->adj_steps, nseg = h->adj_nseg;
    const int K = h->adj_K < steps ? h->adj_K : steps;
    const bool fp32 = h->precision == LBFD_MIXED;
    const size_t sbytes = h->planes * (size_t)h->stride * h->esz;       // a state copy, storage precision
    const size_t lbytes = h->planes * (size_t)h->stride * sizeof(double);  // an adjoint state, FP64
    const long long nel = (long long)h->planes * h->stride;
    const int planes = (int)h->planes;
    // tapes: at most 12 GB.  When a step's tapes fit several times, two
    // buffers of several steps each (recorded per launch); else one step
    // recorded and swept in chunks of cells.
    lbfd::AdjointWork w[2];
    memset(w, 0, sizeof w);
    const size_t budget = (size_t)12 << 30;
    const size_t node = lbfd::adjoint_node_bytes(fp32);
    const long long need = (h->ncell + 63) / 64 * 64;
    const size_t far = (size_t)maxn * sizeof(double);  // adj, per thread
    const size_t per_slot = (size_t)need * ((size_t)maxn * node + sizeof(int)) + 2 * nel * lbfd::rev_store_bytes(fp32);
    int nbuf = 1;
    w[0].maxn = maxn;
    if ((size_t)need * far + 2 * per_slot <= budget) {
        w[0].chunk = need;
        const size_t fit = (budget - (size_t)need * far) / (2 * per_slot);
        w[0].slots = (int)(fit < (size_t)K ? fit : (size_t)K);
        if (w[0].slots > 4) w[0].slots = 4;
        nbuf = K > w[0].slots ? 2 : 1;
    } else {
        long long chunk = (long long)((budget - 2 * nel * lbfd::rev_store_bytes(fp32)) /
                                      ((size_t)maxn * node + sizeof(int) + far));
        w[0].chunk = chunk / 64 * 64;
        w[0].slots = 1;
    }
    w[1].maxn = maxn;
    w[1].chunk = w[0].chunk;
    w[1].slots = w[0].slots;
    const size_t tape = (size_t)maxn * w[0].chunk * w[0].slots;
    const bool pipelined = w[0].chunk >= h->ncell;
    const size_t vsz = fp32 ? sizeof(float) : sizeof(double);  // a recorded partial
    char* seg = nullptr;
    double *lam0 = nullptr, *lam1 = nullptr, *dth = nullptr;
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev[5] = {};  // records done (2), sweeps done (2), segment ready
    std::vector<void*> owned;
    auto alloc = [&](void** p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) owned.push_back(*p);
        return e;
    };
    auto release = [&]() {
        if (s2) cudaStreamSynchronize(s2);
        cudaStreamSynchronize(h->stream);
        for (void* p : owned) cudaFree(p);
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
        if (s2) cudaStreamDestroy(s2);
    };
    cudaError_t e = cudaSuccess;
    if ((e = alloc((void**)&seg, sbytes * K)) != cudaSuccess || (e = alloc((void**)&lam0, lbytes)) != cudaSuccess ||
        (e = alloc((void**)&lam1, lbytes)) != cudaSuccess ||
        (e = alloc((void**)&dth, lbfd::NTAN * sizeof(double))) != cudaSuccess ||
        (e = alloc((void**)&w[0].adj, (size_t)maxn * w[0].chunk * sizeof(double))) != cudaSuccess ||
        (e = alloc((void**)&w[0].flags, 2 * sizeof(int))) != cudaSuccess) {
        release();
        cuda_fail(e, "cudaMalloc(adjoint)");
        return LBFD_ENOMEM;
    }
    w[1].adj = w[0].adj;
    w[1].flags = w[0].flags;
    for (int i = 0; i < nbuf; ++i)
        if ((e = alloc(&w[i].rin, w[i].slots * nel * lbfd::rev_store_bytes(fp32))) != cudaSuccess ||
            (e = alloc(&w[i].rout, w[i].slots * nel * lbfd::rev_store_bytes(fp32))) != cudaSuccess ||
            (e = alloc(&w[i].a0, tape * vsz)) != cudaSuccess || (e = alloc(&w[i].a1, tape * vsz)) != cudaSuccess ||
            (e = alloc((void**)&w[i].par, tape * sizeof(int32_t))) != cudaSuccess ||
            (e = alloc((void**)&w[i].count, w[i].slots * w[i].chunk * sizeof(int))) != cudaSuccess) {
            release();
            cuda_fail(e, "cudaMalloc(adjoint)");
            return LBFD_ENOMEM;
        }
    cudaStream_t s = h->stream;
#define AK(call)                         \
    do {                                 \
        cudaError_t e_ = (call);         \
        if (e_ != cudaSuccess) {         \
            release();                   \
            return cuda_fail(e_, #call); \
        }                                \
    } while (0)
    if (nbuf == 2) {
        AK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
        for (cudaEvent_t& x : ev) AK(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
    }
    cudaStream_t rs = nbuf == 2 ? s2 : s;  // the stream of the records
    AK(cudaMemsetAsync(w[0].flags, 0, 2 * sizeof(int), s));
    AK(cudaMemsetAsync(dth, 0, lbfd::NTAN * sizeof(double), s));
    // the adjoint of J with respect to the final state (FP64), times seed
    AK(cudaMemsetAsync(lam1, 0, lbytes, s));
    if (h->adj_obj == LBFD_OBJ_FLAME_POSITION) {
        // x_f = dx sum_fluid Y_F / (Y_F,in * section)
        const double scale = h->section > 0.0 ? seed * h->prm.dx / (h->prm.Y_in[h->mech.fuel] * h->section) : 0.0;
        std::vector<double> lam((size_t)h->stride, 0.0);
        for (long long c = 0; c < h->ncell; ++c)
            if (!h->mask_host[c]) lam[c] = scale;
        AK(cudaMemcpyAsync(lam1 + (size_t)(h->Q + 1 + h->mech.fuel) * h->stride, lam.data(),
                           (size_t)h->stride * sizeof(double), cudaMemcpyHostToDevice, s));
        AK(cudaStreamSynchronize(s));
    } else {
        double r[2];
        AK(lbfd::launch_quench_sums(h->Pd, view(h, h->cur), fp32, h->solid, h->qwgt, h->red, s));
        AK(cudaMemcpyAsync(r, h->red, sizeof r, cudaMemcpyDeviceToHost, s));
        AK(cudaStreamSynchronize(s));
        if (r[0] > 0.0 && r[1] > 0.0)
            AK(lbfd::launch_quench_seed(h->Pd, view(h, h->cur), fp32, h->solid, h->qwgt, r[0], r[1], h->adj_J, seed,
                                        lam1, dth, h->Q, s));
    }
    // backward pass: each segment recomputed from its checkpoint with the
    // forward kernels (FP32 in the mixed form), every step's adjoint in FP64
    const lbfd::BoundaryLists b = lists(h);
    const int G = w[0].slots;
    for (int g = nseg - 1; g >= 0; --g) {
        const int len = steps - g * K < K ? steps - g * K : K;
        for (int j = 0; j < len; ++j)  // every slot starts as the checkpoint (solid cells never change)
            AK(cudaMemcpyAsync(seg + (size_t)j * sbytes, h->adj_ck + (size_t)g * sbytes, sbytes,
                               cudaMemcpyDeviceToDevice, s));
        for (int j = 1; j < len; ++j)
            AK(lbfd::launch_step(h->dim, h->precision, h->variant, h->Pd, h->Pf,
                                 view_of(h, seg + (size_t)(j - 1) * sbytes), view_of(h, seg + (size_t)j * sbytes),
                                 h->solid, b, h->side, s));
        if (!pipelined) {  // one step at a time (j0 == j1), recorded and swept in chunks of cells
            for (int j = len - 1; j >= 0; --j) {
                AK(cudaMemsetAsync(lam0, 0, lbytes, s));
                for (long long c0 = 0; c0 < h->ncell; c0 += w[0].chunk) {
                    const long long n = h->ncell - c0 < w[0].chunk ? h->ncell - c0 : w[0].chunk;
                    AK(lbfd::launch_adjoint_record(h->dim, h->Pd, planes, seg + (size_t)j * sbytes, sbytes, 1, fp32,
                                                   h->solid, c0, n, w[0], s));
                    AK(lbfd::launch_adjoint_sweep(h->Pd, planes, 0, fp32, h->solid, c0, n, lam1, lam0, dth, w[0], s));
                }
                std::swap(lam0, lam1);
            }
            continue;
        }
        // groups of G steps from the end of the segment: group i holds the
        // steps j1(i) - G + 1 .. j1(i) (clipped at 0) and uses buffer i % 2
        const int ngroups = (len + G - 1) / G;
        auto first = [&](int i) { return len - 1 - i * G - (G - 1) > 0 ? len - 1 - i * G - (G - 1) : 0; };
        auto record = [&](int i) -> cudaError_t {
            const int j1 = len - 1 - i * G, j0 = first(i);
            return lbfd::launch_adjoint_record(h->dim, h->Pd, planes, seg + (size_t)j0 * sbytes, sbytes, j1 - j0 + 1,
                                               fp32, h->solid, 0, h->ncell, w[i % nbuf], rs);
        };
        if (nbuf == 2) {  // the segment's states are ready for the records
            AK(cudaEventRecord(ev[4], s));
            AK(cudaStreamWaitEvent(s2, ev[4], 0));
        }
        AK(record(0));
        if (nbuf == 2) AK(cudaEventRecord(ev[0], s2));
        for (int i = 0; i < ngroups; ++i) {
            const int bi = i % nbuf;
            if (nbuf == 2) {
                AK(cudaStreamWaitEvent(s, ev[bi], 0));  // group i recorded
                if (i + 1 < ngroups) {
                    // group i + 1 into the other buffer once its last sweeps (group i - 1) are done
                    if (i >= 1) AK(cudaStreamWaitEvent(s2, ev[2 + (i + 1) % 2], 0));
                    AK(record(i + 1));
                    AK(cudaEventRecord(ev[(i + 1) % 2], s2));
                }
            } else if (i >= 1) {
                AK(record(i));
            }
            const int j1 = len - 1 - i * G, j0 = first(i);
            for (int j = j1; j >= j0; --j) {
                AK(cudaMemsetAsync(lam0, 0, lbytes, s));
                AK(lbfd::launch_adjoint_sweep(h->Pd, planes, j - j0, fp32, h->solid, 0, h->ncell, lam1, lam0, dth, w[bi],
                                              s));
                std::swap(lam0, lam1);
            }
            if (nbuf == 2) AK(cudaEventRecord(ev[2 + bi], s));
        }
    }
    int flags[2];
    double gr[lbfd::NTAN];
    AK(cudaMemcpyAsync(flags, w[0].flags, sizeof flags, cudaMemcpyDeviceToHost, s));
    AK(cudaMemcpyAsync(gr, dth, sizeof gr, cudaMemcpyDeviceToHost, s));
    AK(cudaStreamSynchronize(s));
#undef AK
    release();
    *overflow = flags[0] != 0;
    for (int k = 0; k < lbfd::NTAN; ++k) grad[k] = gr[k];
    return LBFD_OK;
}

int lbfd_adjoint_backward(lbfd_handle* h, double seed, double* grad)
{
    NvtxRange nvtx_("lbfd_adjoint_backward");
    if (!h || !grad) return LBFD_EINVAL;
    if (!h->adj_ck || h->adj_steps < 1) return LBFD_EINVAL;  // nothing recorded
    // tapes of 2048 nodes per cell and step hold every step of the 2-D
    // general form with room to spare; a step that needs more is taken again
    // with the 16-bit node limit's share of 4096
    double g[lbfd::NTAN];
    bool overflow = false;
    for (int maxn : {2048, 4096}) {
        const int st = adjoint_backward_pass(h, seed, maxn, g, &overflow);
        if (st != LBFD_OK) {
            adjoint_release(h);
            return st;
        }
        if (!overflow) break;
    }
    adjoint_release(h);
    if (overflow) return LBFD_ENOTSUP;  // a cell's step needs more tape than provided
    for (int k = 0; k < lbfd::NTAN; ++k) grad[k] = g[k];
    return LBFD_OK;
}

int lbfd_adjoint_run(lbfd_handle* h, int steps, int objective, double* value, double* grad)
{
    const int st = lbfd_adjoint_record(h, steps, objective, value);
    if (st != LBFD_OK) return st;
    double g[lbfd::NTAN];
    const int bt = lbfd_adjoint_backward(h, 1.0, g);
    if (bt != LBFD_OK) return bt;
    if (grad)
        for (int k = 0; k < lbfd::NTAN; ++k) grad[k] = g[k];
    return LBFD_OK;
}

int lbfd_adjoint_gradient(lbfd_handle* h, int steps, int checkpoint_every, int objective, double* value,
                          double* grad)
{
    if (!h || checkpoint_every < 1) return LBFD_EINVAL;
    const int K = h->adj_K;
    h->adj_K = checkpoint_every;
    const int st = lbfd_adjoint_run(h, steps, objective, value, grad);
    h->adj_K = K;
    return st;
}

int lbfd_flame_position(lbfd_handle* h, double* x_f, double* mass, double* heat_release)
{
    double d[LBFD_NDIAG];
    int st = lbfd_diagnostics(h, d);
    if (st != LBFD_OK && st != LBFD_ENONFINITE) return st;
    if (x_f) *x_f = d[LBFD_DIAG_XF] * h->prm.dx;
    if (mass) *mass = d[LBFD_DIAG_MASS];
    if (heat_release) *heat_release = d[LBFD_DIAG_HRR];
    return st;
}

size_t lbfd_state_bytes(const lbfd_handle* h)
{
    return h ? h->planes * (size_t)h->ncell * h->esz : 0;
}

int lbfd_get_state_raw(lbfd_handle* h, void* dst, size_t bytes)
{
    if (!h || !dst || bytes != lbfd_state_bytes(h)) return LBFD_EINVAL;
    const size_t w = (size_t)h->ncell * h->esz;
    if (h->stride == h->ncell)  // unpadded planes: one contiguous copy
        CK(cudaMemcpyAsync(dst, h->buf[h->cur], w * h->planes, cudaMemcpyDeviceToHost, h->stream));
    else
        CK(cudaMemcpy2DAsync(dst, w, h->buf[h->cur], (size_t)h->stride * h->esz, w, h->planes,
                             cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBFD_OK;
}

int lbfd_set_state_raw(lbfd_handle* h, const void* src, size_t bytes)
{
    if (!h || !src || bytes != lbfd_state_bytes(h)) return LBFD_EINVAL;
    const size_t w = (size_t)h->ncell * h->esz;
    if (h->stride == h->ncell)
        CK(cudaMemcpyAsync(h->buf[h->cur], src, w * h->planes, cudaMemcpyHostToDevice, h->stream));
    else
        CK(cudaMemcpy2DAsync(h->buf[h->cur], (size_t)h->stride * h->esz, src, w, w, h->planes,
                             cudaMemcpyHostToDevice, h->stream));
    // the other buffer too: the step never rewrites solid cells
    const size_t all = h->planes * (size_t)h->stride * h->esz;
    CK(cudaMemcpyAsync(h->buf[h->cur ^ 1], h->buf[h->cur], all, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBFD_OK;
}

// checkpoint file: a fixed header, then the raw state (lbfd_get_state_raw)
struct CheckpointHeader {
    char magic[8];  // "LBFDCKPT"
    int version, dim, nx, ny, nz, Q, nsp, precision;
    long long esz, steps, state_bytes;
};

int lbfd_save(lbfd_handle* h, const char* path)
{
    NvtxRange nvtx_("lbfd_save");
    if (!h || !path) return LBFD_EINVAL;
    CheckpointHeader hd;
    memset(&hd, 0, sizeof hd);
    memcpy(hd.magic, "LBFDCKPT", 8);
    hd.version = 1;
    hd.dim = h->dim;
    hd.nx = h->grid.nx;
    hd.ny = h->grid.ny;
    hd.nz = h->grid.nz;
    hd.Q = h->Q;
    hd.nsp = lbfd::NSP;
    hd.precision = h->precision;
    hd.esz = (long long)h->esz;
    hd.steps = h->steps;
    hd.state_bytes = (long long)lbfd_state_bytes(h);
    std::vector<char> state((size_t)hd.state_bytes);
    const int st = lbfd_get_state_raw(h, state.data(), state.size());
    if (st != LBFD_OK) return st;
    FILE* f = fopen(path, "wb");
    if (!f) {
        snprintf(g_last_error, sizeof g_last_error, "lbfd_save: cannot open %s", path);
        return LBFD_EINVAL;
    }
    const bool ok = fwrite(&hd, sizeof hd, 1, f) == 1 && fwrite(state.data(), 1, state.size(), f) == state.size();
    if (fclose(f) != 0 || !ok) {
        snprintf(g_last_error, sizeof g_last_error, "lbfd_save: write to %s failed", path);
        return LBFD_EINVAL;
    }
    return LBFD_OK;
}

int lbfd_load(lbfd_handle* h, const char* path)
{
    NvtxRange nvtx_("lbfd_load");
    if (!h || !path) return LBFD_EINVAL;
    FILE* f = fopen(path, "rb");
    if (!f) {
        snprintf(g_last_error, sizeof g_last_error, "lbfd_load: cannot open %s", path);
        return LBFD_EINVAL;
    }
    CheckpointHeader hd;
    bool ok = fread(&hd, sizeof hd, 1, f) == 1;
    ok = ok && memcmp(hd.magic, "LBFDCKPT", 8) == 0 && hd.version == 1 && hd.dim == h->dim && hd.nx == h->grid.nx &&
         hd.ny == h->grid.ny && hd.nz == h->grid.nz && hd.Q == h->Q && hd.nsp == lbfd::NSP &&
         hd.precision == h->precision && hd.esz == (long long)h->esz &&
         hd.state_bytes == (long long)lbfd_state_bytes(h);
    std::vector<char> state;
    if (ok) {
        state.resize((size_t)hd.state_bytes);
        ok = fread(state.data(), 1, state.size(), f) == state.size();
    }
    fclose(f);
    if (!ok) {
        snprintf(g_last_error, sizeof g_last_error,
                 "lbfd_load: %s is not a checkpoint of this grid, lattice and precision", path);
        return LBFD_EINVAL;
    }
    const int st = lbfd_set_state_raw(h, state.data(), state.size());
    if (st != LBFD_OK) return st;
    h->steps = hd.steps;
    return LBFD_OK;
}

int lbfd_batch_create(int n, const int* widths, int length, const lbfd_grid* proto, const lbfd_mechanism* mech,
                      const lbfd_params* params, lbfd_handle** out, int* rows)
{
    if (n < 1 || !widths || length < 1 || !proto || !mech || !params || !out || !rows) return LBFD_EINVAL;
    if (proto->dim != 2) return LBFD_ENOTSUP;
    long long ny = n - 1;
    for (int j = 0; j < n; ++j) {
        if (widths[j] < 1) return LBFD_EINVAL;
        ny += widths[j];
    }
    if (ny > (1 << 30)) return LBFD_EINVAL;
    lbfd_grid g = *proto;
    g.nx = length;
    g.ny = (int)ny;
    g.nz = 1;
    std::vector<uint8_t> mask((size_t)length * ny, 0);
    int y = 0;
    for (int j = 0; j < n; ++j) {
        rows[2 * j] = y;
        y += widths[j];
        rows[2 * j + 1] = y;
        if (j < n - 1) {  // one solid row between neighbouring channels
            memset(mask.data() + (size_t)y * length, 1, (size_t)length);
            ++y;
        }
    }
    return lbfd_create(&g, mask.data(), mech, params, out);
}

int lbfd_read_tangent(lbfd_handle* h, int field, int k, double* out)
{
    if (!h || !out || !is_tangent(h->precision) || k < 0 || k >= lbfd::NTAN) return LBFD_EINVAL;
    int plane;
    if (field == LBFD_FIELD_T) plane = h->Q;
    else if (field >= LBFD_FIELD_Y0 && field < LBFD_FIELD_Y0 + lbfd::NSP) plane = h->Q + 1 + (field - LBFD_FIELD_Y0);
    else if (field >= LBFD_FIELD_G0 && field < LBFD_FIELD_G0 + h->Q) plane = field - LBFD_FIELD_G0;
    else return LBFD_EINVAL;
    CK(lbfd::launch_tangent_field(h->precision == LBFD_TANGENT_MIXED, h->ncell, h->stride, h->buf[h->cur], plane, k,
                                  h->tmp, h->stream));
    CK(cudaMemcpyAsync(out, h->tmp, (size_t)h->ncell * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return LBFD_OK;
}

int lbfd_gradient(lbfd_handle* h, int objective, double* value, double* grad)
{
    if (!h || !is_tangent(h->precision) ||
        (objective != LBFD_OBJ_FLAME_POSITION && objective != LBFD_OBJ_HEAT_RELEASE &&
         objective != LBFD_OBJ_QUENCH_DISTANCE))
        return LBFD_EINVAL;
    if (objective == LBFD_OBJ_QUENCH_DISTANCE) {
        const int st = quench_weights(h);
        if (st != LBFD_OK) return st;
    }
    double r[2 * (1 + lbfd::NTAN)];
    if (h->precision == LBFD_TANGENT)
        CK(lbfd::launch_objective(h->Pt, view(h, h->cur), h->solid, objective, h->qwgt, h->red, h->stream));
    else
        CK(lbfd::launch_objective(h->Ptf, view(h, h->cur), h->solid, objective, h->qwgt, h->red, h->stream));
    CK(cudaMemcpyAsync(r, h->red, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (objective == LBFD_OBJ_QUENCH_DISTANCE) {
        // J = (S1/S0)^(-1/4): dJ = -J/4 (dS1/S1 - dS0/S0)
        const double S0 = r[0], S1 = r[1 + lbfd::NTAN];
        const double J = S0 > 0.0 && S1 > 0.0 ? pow(S1 / S0, -0.25) : 0.0;
        if (value) *value = J;
        if (grad)
            for (int k = 0; k < lbfd::NTAN; ++k)
                grad[k] = S0 > 0.0 && S1 > 0.0 ? -0.25 * J * (r[2 + lbfd::NTAN + k] / S1 - r[1 + k] / S0) : 0.0;
        return LBFD_OK;
    }
    double scale = 1.0;
    if (objective == LBFD_OBJ_FLAME_POSITION)  // x_f = dx sum Y_F / (Y_F,in * section)
        scale = h->section > 0.0 ? h->prm.dx / (h->prm.Y_in[h->mech.fuel] * h->section) : 0.0;
    if (value) *value = r[0] * scale;
    if (grad)
        for (int k = 0; k < lbfd::NTAN; ++k) grad[k] = r[1 + k] * scale;
    return LBFD_OK;
}

long long lbfd_steps_done(const lbfd_handle* h) { return h ? h->steps : -1; }
long long lbfd_num_cells(const lbfd_handle* h) { return h ? h->ncell : -1; }
int lbfd_num_populations(const lbfd_handle* h) { return h ? h->Q : -1; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free diagnostics (see lbfd_diagnostics_noalloc in lbfd.h).
// The reduction scratch lives in this file-scope device array instead of
// memory from cudaMalloc.  Host code cannot use the array's name as a device
// address, so the address is looked up once per device with
// cudaGetSymbolAddress and cached (for the life of the device's context: a
// cudaDeviceReset is not supported while the library is loaded).
// ---------------------------------------------------------------------------
static __device__ __align__(256) double lbfd_noalloc_scratch[LBFD_NOALLOC_SCRATCH_WORDS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {};

int noalloc_scratch_address(void** out)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        snprintf(g_last_error, sizeof g_last_error, "lbfd_diagnostics_noalloc: device ordinal %d >= %d", dev,
                 kMaxDevices);
        return LBFD_ENOTSUP;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, lbfd_noalloc_scratch));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return LBFD_OK;
}

bool is_device_pointer(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // a failed query leaves its error set: clear it
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int lbfd_diagnostics_noalloc(const lbfd_grid* grid, const lbfd_mechanism* mech,
                                        const lbfd_params* params, const void* g, const void* T, const void* Y,
                                        long long plane_stride, const uint8_t* solid, void* stream, double* out)
{
    if (!grid || !mech || !params || !g || !T || !Y || !solid || !out) return LBFD_EINVAL;
    int st = validate(grid, mech, params);
    if (st != LBFD_OK) return st;
    // the call needs lbfd::RED_WORDS words of scratch whatever the grid size
    if (lbfd::RED_WORDS > LBFD_NOALLOC_SCRATCH_WORDS) {
        snprintf(g_last_error, sizeof g_last_error,
                 "lbfd_diagnostics_noalloc: needs %d scratch words, the static array holds %d", lbfd::RED_WORDS,
                 LBFD_NOALLOC_SCRATCH_WORDS);
        return LBFD_EINVAL;
    }
    lbfd_handle tmp{};  // parameters only: no buffer is allocated or owned
    tmp.grid = *grid;
    if (grid->dim == 2) tmp.grid.nz = 1;
    tmp.mech = *mech;
    tmp.prm = *params;
    tmp.dim = grid->dim;
    tmp.Q = grid->dim == 2 ? 9 : 27;
    tmp.precision = params->precision;
    tmp.ncell = (long long)tmp.grid.nx * tmp.grid.ny * tmp.grid.nz;
    if (plane_stride < tmp.ncell) {
        snprintf(g_last_error, sizeof g_last_error, "lbfd_diagnostics_noalloc: plane_stride %lld < cells %lld",
                 plane_stride, tmp.ncell);
        return LBFD_EINVAL;
    }
    tmp.stride = plane_stride;
    if (!is_device_pointer(g) || !is_device_pointer(T) || !is_device_pointer(Y) || !is_device_pointer(solid)) {
        snprintf(g_last_error, sizeof g_last_error, "lbfd_diagnostics_noalloc: inputs must be device pointers");
        return LBFD_EINVAL;
    }
    void* red = nullptr;
    st = noalloc_scratch_address(&red);
    if (st != LBFD_OK) return st;
    StepParams<double> P;
    fill_params(&tmp, P);
    StateView v;
    v.g = const_cast<void*>(g);
    v.T = const_cast<void*>(T);
    v.Y = const_cast<void*>(Y);
    cudaStream_t s = (cudaStream_t)stream;
    // launch_diagnostics clears the words it accumulates into before use
    CK(lbfd::launch_diagnostics(tmp.dim, tmp.precision, P, v, solid, 0, tmp.grid.ny, (double*)red, s));
    double r[lbfd::RED_WORDS];
    CK(cudaMemcpyAsync(r, red, sizeof r, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    unsigned long long u[lbfd::RED_WORDS];
    memcpy(u, r, sizeof r);
    const double section = (double)u[7];
    out[LBFD_DIAG_XF] = section > 0.0 ? r[0] / (params->Y_in[mech->fuel] * section) : 0.0;
    out[LBFD_DIAG_MASS] = r[1];
    out[LBFD_DIAG_HRR] = r[2];
    out[LBFD_DIAG_FUEL] = r[3];
    double t = -INFINITY;
    if (u[4] != 0ull) {
        const unsigned long long b = (u[4] >> 63) ? (u[4] & 0x7fffffffffffffffull) : ~u[4];
        memcpy(&t, &b, sizeof t);
    }
    out[LBFD_DIAG_TMAX] = t;
    out[LBFD_DIAG_XHRR] = r[9];
    out[LBFD_DIAG_NONFINITE] = (double)u[5];
    out[LBFD_DIAG_NFLUID] = (double)u[6];
    return u[5] ? LBFD_ENONFINITE : LBFD_OK;
}
