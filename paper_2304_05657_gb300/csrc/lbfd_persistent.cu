// lbfd_persistent.cu -- n coupled 2-D steps in one persistent launch.
//
// One cooperative launch of as many 128-thread blocks as fit on the GPU
// at once.  Every step, the blocks take work items from a shared counter:
// first the chunks of 128 cells near domain faces (general form, the
// slowest items), then the wall tiles (64 x 2, the cells next to in-domain
// solids), then the interior tiles (32 x 4 cells), with the same per-cell
// code as the multi-kernel step of variant 6; then all blocks meet at a
// grid-wide barrier before the buffers swap roles.  The barrier's wait is
// bounded: a block that waits longer than the limit records the failure
// and returns, the others see the record and return too, and the host
// reports LBFD_ETIMEOUT.  Batching in this library packs many channels
// into one masked domain, so this one launch advances every channel.
//
// The state buffers are written and read back within the launch, so this
// translation unit compiles the step without read-only hints: no restrict
// qualifiers and plain loads (a load through the non-coherent read-only
// path could return data cached before another block wrote it).
#include <cuda_runtime.h>

#define LBFD_RESTRICT
#define LBFD_LDG(p) (*(p))

#include "lbfd_internal.h"
#include "lbfd_step_tiled.cuh"

namespace lbfd {

namespace {

constexpr int PT_TX = 32, PT_TY = 4, PT_THREADS = 128;
static_assert(PT_TX * PT_TY == PT_THREADS && WALL_TX * WALL_TY == PT_THREADS, "one block shape for every phase");

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of step `step`.  Returns false when this block or
// another one gave up waiting; limit_ns <= 0 gives up at once in every block
// but the last to arrive.
__device__ bool grid_wait(PersistentWait* w, unsigned nblocks, long long limit_ns, int step)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = &w->gen;
        volatile int* err = &w->error;
        const unsigned g = *gen;
        __threadfence();  // this block's writes of the step before its arrival
        const unsigned arrived = atomicAdd(&w->count, 1u);
        int res = 1;
        if (arrived == nblocks - 1) {
            atomicExch(&w->count, 0u);
            atomicExch(&w->next[(step + 1) & 1], 0u);  // the next step's items (last used two steps ago)
            __threadfence();
            atomicAdd(&w->gen, 1u);
        } else if (limit_ns <= 0) {
            res = 0;
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g) {
                if (*err) {
                    res = 0;
                    break;
                }
                if ((long long)(global_ns() - t0) > limit_ns) {
                    res = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (!res) {
            atomicCAS(&w->step, 0, step + 1);
            atomicExch(&w->error, 1);
        } else if (*err) {
            res = 0;  // another block gave up: the state is not synchronised
        }
        __threadfence();  // the other blocks' writes before this block's next reads
        ok = res;
    }
    __syncthreads();
    return ok != 0;
}

// FP32: four blocks per SM (128 registers); FP64: two
template <typename S, typename R>
__global__ void __launch_bounds__(PT_THREADS, sizeof(R) == 4 ? 4 : 2)
    step_kernel_persistent2d(StepParams<R> P, StateView a, StateView b, int n, const uint8_t* solid,
                             const uint8_t* interior, const int* wall_tiles, int nwall_tiles,
                             const long long* cells, long long ncells, PersistentWait* w, long long limit_ns)
{
    __shared__ unsigned item_sh;
    const int tid = threadIdx.x;
    const int gx = (P.nx + PT_TX - 1) / PT_TX, gy = (P.ny + PT_TY - 1) / PT_TY;
    const int wgx = (P.nx + WALL_TX - 1) / WALL_TX;
    const unsigned nchunk = (unsigned)((ncells + PT_THREADS - 1) / PT_THREADS);
    const unsigned nitems = nchunk + (unsigned)nwall_tiles + (unsigned)(gx * gy);
    for (int s = 0; s < n; ++s) {
        const StateView in = (s & 1) ? b : a, out = (s & 1) ? a : b;
        const S* g_in = (const S*)in.g;
        const S* T_in = (const S*)in.T;
        const S* Y_in = (const S*)in.Y;
        S* g_out = (S*)out.g;
        S* T_out = (S*)out.T;
        S* Y_out = (S*)out.Y;
        for (;;) {
            if (tid == 0) item_sh = atomicAdd(&w->next[s & 1], 1u);
            __syncthreads();
            const unsigned it = item_sh;
            __syncthreads();  // item_sh is rewritten by the next grab
            if (it >= nitems) break;
            if (it < nchunk) {
                const long long i = (long long)it * PT_THREADS + tid;
                if (i < ncells) {
                    const long long c = cells[i];
                    const int p[3] = {(int)(c % P.nx), (int)(c / P.nx), 0};
                    cell_step_general<2, S, R, true>(P, p, c, g_in, g_out, T_in, T_out, Y_in, Y_out, solid);
                }
            } else if (it < nchunk + (unsigned)nwall_tiles) {
                const int wt = wall_tiles[it - nchunk];
                tiled2d_body<S, R, WALL_TX, WALL_TY, true>(P, g_in, g_out, T_in, T_out, Y_in, Y_out, solid, nullptr,
                                                           tid % WALL_TX, tid / WALL_TX, wt % wgx, wt / wgx);
            } else {
                const int t = (int)(it - nchunk - (unsigned)nwall_tiles);
                tiled2d_body<S, R, PT_TX, PT_TY, false>(P, g_in, g_out, T_in, T_out, Y_in, Y_out, nullptr, interior,
                                                        tid % PT_TX, tid / PT_TX, t % gx, t / gx);
            }
            __syncthreads();  // the next tile restages the shared memory
        }
        if (!grid_wait(w, gridDim.x, limit_ns, s)) return;
    }
}

template <typename S, typename R>
cudaError_t launch_pers(const StepParams<R>& P, StateView a, StateView b, int n, const uint8_t* solid,
                        const BoundaryLists& bl, PersistentWait* w, long long limit_ns, cudaStream_t stream,
                        int* blocks)
{
    auto kern = step_kernel_persistent2d<S, R>;
    const size_t smem = tile_smem_bytes<R, PT_TX, PT_TY>() > tile_smem_bytes<R, WALL_TX, WALL_TY>()
                            ? tile_smem_bytes<R, PT_TX, PT_TY>()
                            : tile_smem_bytes<R, WALL_TX, WALL_TY>();
    cudaError_t e;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PT_THREADS, smem)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    const unsigned nb = (unsigned)(per_sm * sms);
    *blocks = (int)nb;
    // wall tiles only when the variant-6 split has them; otherwise every
    // non-interior cell goes through the general form
    const bool walls = bl.nwall_tiles > 0;
    const long long* cells = walls ? bl.face : bl.all;
    const long long ncells = walls ? bl.nface : bl.nall;
    if ((e = cudaMemsetAsync(w, 0, sizeof(PersistentWait), stream)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(PT_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all blocks resident at once: the barrier can complete
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, P, a, b, n, solid, (const uint8_t*)bl.interior,
                              walls ? bl.wall_tiles : (const int*)nullptr, walls ? (int)bl.nwall_tiles : 0, cells,
                              ncells, w, limit_ns);
}

}  // namespace

cudaError_t launch_step_persistent(int precision, const StepParams<double>& Pd, const StepParams<float>& Pf,
                                   StateView a, StateView b, int n, const uint8_t* solid, const BoundaryLists& bl,
                                   PersistentWait* w, long long limit_ns, cudaStream_t stream, int* blocks)
{
    if (bl.interior == nullptr) return cudaErrorInvalidValue;
    if (precision == 0) return launch_pers<double, double>(Pd, a, b, n, solid, bl, w, limit_ns, stream, blocks);
    return launch_pers<float, float>(Pf, a, b, n, solid, bl, w, limit_ns, stream, blocks);
}

}  // namespace lbfd
