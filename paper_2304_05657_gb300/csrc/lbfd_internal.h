// lbfd_internal.h -- launch interface between the C-ABI host code and the
// kernel translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "lbfd_dual.cuh"
#include "lbfd_params.h"

namespace lbfd {

// Device views of one state buffer: populations g[Q][stride], T[stride],
// Y[NSP][stride], all in storage precision.
struct StateView {
    void* g;
    void* T;
    void* Y;
};

// Launch one fused coupled step: state `in` -> state `out`.
// precision: 0 = FP64 (S = R = double), 1 = mixed (S = R = float).
// variant: 0 = general form, 1.. = 2-D shared-memory tiles (see lbfd_step.cu)
// A second stream and two events used to run the boundary kernel next to
// the tile kernel (fork on `fork`, join on `join`); stream == nullptr runs
// both on the launch stream.
struct SideStream {
    cudaStream_t stream;
    cudaEvent_t fork, join;
    int priority;  // the device's greatest stream priority
    int low;       // and its least
};

// Launch on the side stream at its priority, so that the block scheduler
// dispatches these blocks ahead of the pending blocks of the (much larger)
// tile grid on the main stream; in a captured graph the priority is kept
// as a kernel-node attribute.
template <typename... Exp, typename... Act>
cudaError_t launch_prio(void (*kern)(Exp...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, int prio,
                        Act&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = prio;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Act>(args)...);
}

// Cells the tile kernels leave to the boundary kernel (see boundary_cells):
// `all` every non-interior fluid cell; `face` only those whose stencil
// reaches a domain face (for the 2-D variants that handle in-domain solid
// neighbours themselves).  Unused by the general variant.
struct BoundaryLists {
    const long long* all;
    long long nall;
    const long long* face;
    long long nface;
    const int* wall_tiles;  // 2-D tiles of WALL_TX x WALL_TY cells holding cells of all \ face
    long long nwall_tiles;
    const long long* wall;  // 3-D: all \ face, cells whose stencils reach no non-periodic face
    long long nwall;
    const unsigned long long* wall_code;  // 3-D: their neighbourhood codes (cell_step_coded)
    const long long* face_coded;  // 3-D: cells near inlet/outlet faces taken by cell_step_coded<FACES>
    long long nface_coded;        // (then `face` holds the other cells near faces)
    const unsigned long long* face_code;
    const uint8_t* interior;  // per cell, 1 for the cells the interior tile kernels update
    void* aux;                // 3-D: 4 planes of the compute type for the split variants
};

// tile shape of the 2-D wall-tile kernel
constexpr int WALL_TX = 64, WALL_TY = 2;
// the tiles that hold a cell of `all` not in `face` (host, at create)
void wall_tiles(int nx, int ny, const std::vector<long long>& all, const std::vector<long long>& face,
                std::vector<int>& out);

cudaError_t launch_step(int dim, int precision, int variant, const StepParams<double>& Pd,
                        const StepParams<float>& Pf, StateView in, StateView out, const uint8_t* solid,
                        const BoundaryLists& b, const SideStream& side, cudaStream_t stream);
int num_variants(int dim);

// 3-D tile kernels (variants 1..2 in 3-D), lbfd_step3d.cu
cudaError_t launch_step3d_tiled(int precision, int variant, const StepParams<double>& Pd, const StepParams<float>& Pf,
                                StateView in, StateView out, const uint8_t* solid, const BoundaryLists& b,
                                const SideStream& side, cudaStream_t stream);

// Neighbourhood codes of the cells of a 3-D wall list (host, at create;
// layout in cell_step_coded).
void wall_codes(int nx, int ny, int nz, const int* bc, const uint8_t* solid, const std::vector<long long>& cells,
                std::vector<unsigned long long>& out);
// The cells near domain faces that cell_step_coded<FACES> takes (faces of
// one axis, all of them inlet or outlet faces, no corner of the general
// form's rules in reach; staircase walls) with their codes, and the others
// (general form).  Both in the order of `cells`.
void face_codes(int nx, int ny, int nz, const int* bc, const uint8_t* solid, const std::vector<long long>& cells,
                std::vector<long long>& coded, std::vector<unsigned long long>& codes, std::vector<long long>& rest);

// Fluid cells that are not interior for the tile kernels (host, at create);
// faces_only (2-D): only cells whose stencil leaves the domain.
void boundary_cells(int dim, int nx, int ny, int nz, const int* bc, const uint8_t* solid, std::vector<long long>& out,
                    bool faces_only, const int* face_solid);

// Diagnostics reduction over the rows y0 <= y < y1 (all x, all z) into the
// device scratch `red` (RED_WORDS words, zeroed by the launcher); FP64
// accumulation.
cudaError_t launch_diagnostics(int dim, int precision, const StepParams<double>& Pd, StateView st,
                               const uint8_t* solid, int y0, int y1, double* red, cudaStream_t stream);

// Column peaks of the heat release over rows y0 <= y < y1 of a 2-D grid
// (FP64 or mixed state): out[x] = peak, out[nx + x] = its distance to the
// nearer band edge (device, 2 nx doubles).
cudaError_t launch_column_peaks(int precision, const StepParams<double>& P, StateView st, const uint8_t* solid,
                                int y0, int y1, double* out, cudaStream_t stream);

// Derived or raw field of every cell into double out[ncell] (device).
cudaError_t launch_field(int dim, int precision, const StepParams<double>& Pd, StateView st,
                         const uint8_t* solid, int field, double* out, cudaStream_t stream);
// gather the whole state of n listed cells into out[n][Q + 1 + NSP] (device)
cudaError_t launch_cells(int dim, int precision, const StepParams<double>& Pd, StateView st, const long long* cells,
                         long long n, double* out, cudaStream_t stream);

// Tangent-linear step (precision 2: Dual<double, 4> values; precision 3:
// Dual<float, 4>; general form, 2-D), tangent read-out and objective
// gradients (lbfd_tangent.cu).
cudaError_t launch_step_tangent(int dim, const StepParams<Tan>& P, StateView in, StateView out, const uint8_t* solid,
                                cudaStream_t stream);
cudaError_t launch_step_tangent(int dim, const StepParams<Tanf>& P, StateView in, StateView out, const uint8_t* solid,
                                cudaStream_t stream);
cudaError_t launch_tangent_field(bool fp32, long long ncell, long long N, const void* state_base, int plane, int k,
                                 double* out, cudaStream_t stream);
cudaError_t launch_objective(const StepParams<Tan>& P, StateView st, const uint8_t* solid, int objective,
                             const double* wgt, double* red, cudaStream_t stream);
cudaError_t launch_objective(const StepParams<Tanf>& P, StateView st, const uint8_t* solid, int objective,
                             const double* wgt, double* red, cudaStream_t stream);

// Discrete adjoint of FP64 steps (lbfd_adjoint.cu): scratch of the
// reverse-mode tapes.  A record launch takes the steps of `slots` states at
// once (thread t = slot * chunk + u: cell c0 + u), node k of thread t at
// k * slots * chunk + t; a sweep takes one slot.
struct AdjointWork {
    void* rin;   // the input states as tape input (slots * planes * N elements)
    void* rout;  // the recorded outputs (as many)
    void* a0;         // partials: double, or float for the FP32 forward pass
    void* a1;
    int32_t* par;
    int* count;       // [slots * chunk] nodes each thread recorded
    double* adj;      // [maxn][chunk] adjoints of the far nodes during a sweep
    int maxn;         // nodes per thread
    int slots;        // steps recorded per launch
    long long chunk;  // threads (cells) per slot, a multiple of 64
    int* flags;       // [0] tape overflow, [1] most nodes a thread used
};
size_t adjoint_node_bytes(bool fp32);  // tape bytes per node and slot
size_t rev_store_bytes(bool fp32);
// record the steps from `slots` states (slot j at states + j * state_bytes,
// storage precision) for the cells [c0, c0 + n); fp32: the FP32 state of
// the mixed form, its steps recorded in FP32 (the sweep's adjoints stay
// FP64)
cudaError_t launch_adjoint_record(int dim, const StepParams<double>& Pd, int planes, const void* states,
                                  size_t state_bytes, int slots, bool fp32, const uint8_t* solid, long long c0,
                                  long long n, const AdjointWork& w, cudaStream_t stream);
// sweep the tapes of slot `slot` for the cells [c0, c0 + n): lam (zeroed by
// the caller) += (dF/dx)^T lam_next, dtheta += (dF/dtheta)^T lam_next
cudaError_t launch_adjoint_sweep(const StepParams<double>& Pd, int planes, int slot, bool fp32, const uint8_t* solid,
                                 long long c0, long long n, const double* lam_next, double* lam, double* dtheta,
                                 const AdjointWork& w, cudaStream_t stream);
// quenching-distance objective J = (S1/S0)^(-1/4), S0 = sum_fluid h,
// S1 = sum_fluid h w (h the heat release of a cell, w = d^-4 its wall
// weight): red[0..1] = S0, S1 of state st; and the adjoint seed
// lam += seed dJ/dstate, dtheta += seed (explicit dJ/dtheta)
cudaError_t launch_quench_sums(const StepParams<double>& Pd, StateView st, bool fp32, const uint8_t* solid,
                               const double* wgt, double* red, cudaStream_t stream);
cudaError_t launch_quench_seed(const StepParams<double>& Pd, StateView st, bool fp32, const uint8_t* solid,
                               const double* wgt, double S0, double S1, double J, double seed, double* lam,
                               double* dtheta, int Q, cudaStream_t stream);

// Curved walls (lbfd_geometry.cu): host tables of cut links and ghosts.
struct CurvedTables {
    std::vector<int> link_row;        // [ncell]
    std::vector<double> link_q;       // [rows][Q]
    std::vector<int> ghost_row;       // [ncell]
    std::vector<long long> gh_start;  // [nghost + 1]
    std::vector<long long> gh_idx;
    std::vector<double> gh_w;
    long long nghost;
};
int build_curved_tables(int dim, int nx, int ny, int nz, const int* bc, const uint8_t* solid, int nprims,
                        const double* prims, CurvedTables& out);
// ghost values of state `in` into the gval buffer of the parameters
cudaError_t launch_ghost_fill(int precision, const StepParams<double>& Pd, const StepParams<float>& Pf,
                              const StepParams<Tan>& Pt, StateView in, const long long* start, const long long* nb,
                              const double* w, long long nghost, cudaStream_t stream);

// Grid-wide barrier words of the persistent step (device memory, zeroed
// before each launch): arrival count, generation, a failure flag and the
// first step (1-based) whose barrier gave up.
struct PersistentWait {
    unsigned count;
    unsigned gen;
    int error;
    int step;
    unsigned next[2];  // work-item counters of even and odd steps
};
// n 2-D steps in one cooperative launch (lbfd_persistent.cu), alternating
// a -> b -> a ...; *blocks gets the grid size.  limit_ns bounds every
// barrier wait (<= 0: no waiting at all).
cudaError_t launch_step_persistent(int precision, const StepParams<double>& Pd, const StepParams<float>& Pf,
                                   StateView a, StateView b, int n, const uint8_t* solid, const BoundaryLists& bl,
                                   PersistentWait* w, long long limit_ns, cudaStream_t stream, int* blocks);

// Number of words of the reduction scratch.
constexpr int RED_WORDS = 16;

}  // namespace lbfd
