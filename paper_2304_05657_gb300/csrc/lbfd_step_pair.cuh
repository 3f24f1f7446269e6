// lbfd_step_pair.cuh -- 2-D interior tile kernel that computes two
// neighbouring cells (x, x+1) per thread with packed FP32 arithmetic (F2):
// the same staging and the same per-cell arithmetic as step_kernel_tiled2d,
// instantiated on a pair of cells, so that each packed instruction does the
// work of two.  The kernel is issue-bound (not HBM-bound), and the packed
// form halves the floating-point instructions; FD lines along x come from
// three aligned 8-byte shared loads per field, along y from five.
//
// A thread whose two cells are not both interior still computes the pair
// and stores only the interior one(s); the others belong to the boundary
// kernels, exactly as in the one-cell-per-thread tiles.
#pragma once
#include "lbfd_step_tiled.cuh"

namespace lbfd {

// five-point line of a staged field for the cells at points p0 (even) and
// p0 + 1: along x from f[p0-2 .. p0+3], along y from rows p0 +- SX, +- 2 SX
template <bool XLINE, int SX>
__device__ __forceinline__ void pair_line(const float* f, int p0, F2* v)
{
    if constexpr (XLINE) {
        const float2 a = *reinterpret_cast<const float2*>(f + p0 - 2);
        const float2 b = *reinterpret_cast<const float2*>(f + p0);
        const float2 c = *reinterpret_cast<const float2*>(f + p0 + 2);
        v[0] = F2(a);
        v[1] = F2(a.y, b.x);
        v[2] = F2(b);
        v[3] = F2(b.y, c.x);
        v[4] = F2(c);
    } else {
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] = F2(*reinterpret_cast<const float2*>(f + p0 + (j - 2) * SX));
    }
}

__device__ __forceinline__ F2 pair_at(const float* f, int p0) { return F2(*reinterpret_cast<const float2*>(f + p0)); }

// asynchronous global -> shared copy of B bytes (cp.async; both addresses
// aligned to B), completed by cp_async_wait_all in the issuing thread
template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// shared memory of the pair kernel: the staged tile, then (16-byte aligned)
// the pulled populations of its cells, [i][2 * thread + lane]
template <int TX, int TY>
__host__ __device__ constexpr size_t pair_pull_offset()
{
    return (tile_smem_bytes<float, TX, TY>() + 15) / 16 * 16;
}
template <int TX, int TY>
__host__ __device__ constexpr size_t pair_smem_bytes()
{
    return pair_pull_offset<TX, TY>() + sizeof(float) * 9 * TX * TY;
}

// store the lanes that are set: one 8-byte store when both are and p is
// 8-byte aligned (vec), else per lane
__device__ __forceinline__ void pair_store(float* p, const F2& v, bool ok0, bool ok1, bool vec)
{
    if (vec) {
        *reinterpret_cast<float2*>(p) = v.v;
    } else {
        if (ok0) p[0] = v.v.x;
        if (ok1) p[1] = v.v.y;
    }
}

// Staging of the pair kernel's tile, two x-neighbouring points per thread
// in packed FP32 (the same values as stage_tile2d): with nx even, the two
// points of a pair (staged x even) are both inside the domain or both
// outside it, wrap together across a periodic x face and sit at an even
// cell index, so that each field moves as one 8-byte load and one 8-byte
// shared store.  Odd nx takes stage_tile2d.
template <int TX, int TY, int NTHR>
__device__ __forceinline__ void stage_tile2d_pairs(const StepParams<float>& P, const TileSmem<float>& sm, int x0,
                                                   int y0, int tid, const float* LBFD_RESTRICT T_in,
                                                   const float* LBFD_RESTRICT Y_in)
{
    using G = TileGeom<TX, TY>;
    constexpr int SX = G::SX, NPT = G::NPT, NPP = NPT / 2;
    constexpr int NIT = (NPP + NTHR - 1) / NTHR;
    const long long N = P.N;
    long long cell[NIT];  // -1: outside the domain
    F2 T[NIT], Y[NIT][NSP];
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        const int pp = tid + it * NTHR;
        cell[it] = -1;
        if (pp >= NPP) continue;
        const int pt = 2 * pp;
        const int sx = pt % SX, sy = pt / SX;
        int gx = x0 + sx - 2, gy = y0 + sy - 2;
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
        if (gx < 0 || gx >= P.nx || gy < 0 || gy >= P.ny) continue;
        const long long c = (long long)gx + (long long)P.nx * gy;
        cell[it] = c;
        T[it] = F2(*reinterpret_cast<const float2*>(T_in + c));
#pragma unroll
        for (int k = 0; k < NSP; ++k) Y[it][k] = F2(*reinterpret_cast<const float2*>(Y_in + (long long)k * N + c));
    }
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        if (cell[it] < 0) continue;
        const int pt = 2 * (tid + it * NTHR);
        F2 invW = F2(0.f);
#pragma unroll
        for (int k = 0; k < NSP; ++k) invW += Y[it][k] * F2(P.inv_Wk[k]);
        const F2 W = fdiv(F2(1.f), invW);
        auto put = [&](float* f, const F2& v) { *reinterpret_cast<float2*>(f + pt) = v.v; };
        put(sm.T, T[it]);
#pragma unroll
        for (int k = 0; k < NSP; ++k) {
            put(sm.Y + k * NPT, Y[it][k]);
            put(sm.X + k * NPT, Y[it][k] * W);  // X_k W_k (1/W_k folded into a12)
        }
        put(sm.invW, invW);
        put(sm.rho, fdiv(F2(P.T_in * P.invW_in) * W, T[it]));
    }
}

// TXP x TY threads, a tile of 2 TXP x TY cells, at least MINB blocks per
// SM (which caps the registers); FP32 storage and arithmetic
template <int TXP, int TY, int MINB>
__global__ void __launch_bounds__(TXP * TY, MINB)
    step_kernel_pair2d(StepParams<float> P, const float* LBFD_RESTRICT g_in, float* LBFD_RESTRICT g_out,
                       const float* LBFD_RESTRICT T_in, float* LBFD_RESTRICT T_out, const float* LBFD_RESTRICT Y_in,
                       float* LBFD_RESTRICT Y_out, const uint8_t* LBFD_RESTRICT interior)
{
    constexpr int TX = 2 * TXP;
    using G = TileGeom<TX, TY>;
    constexpr int SX = G::SX, NPT = G::NPT;
    static_assert(SX % 2 == 0 && NPT % 2 == 0, "pairs need 8-byte aligned shared rows");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<float> sm;
    sm.T = reinterpret_cast<float*>(smem_raw);
    sm.Y = sm.T + NPT;
    sm.X = sm.Y + NSP * NPT;
    sm.invW = sm.X + NSP * NPT;
    sm.rho = sm.invW + NPT;
    sm.mask = reinterpret_cast<uint8_t*>(sm.rho + NPT);

    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int x = x0 + 2 * threadIdx.x, y = y0 + threadIdx.y;
    const bool inside = x < P.nx && y < P.ny;
    const bool has1 = x + 1 < P.nx;
    const long long c = (long long)x + (long long)P.nx * y;
    const long long N = P.N;

    // a1: pull from the neighbours (Eq. 8) straight into shared memory
    // (cp.async), issued before the staging so that the copies are in flight
    // meanwhile and hold no registers through the FD part; a missing lane 1
    // re-reads lane 0.  The offsets wrap inside the domain for any in-range
    // cell.
    constexpr int NT = TXP * TY;
    const int tid = threadIdx.x + TXP * threadIdx.y;
    float* gs = reinterpret_cast<float*>(smem_raw + pair_pull_offset<TX, TY>()) + 2 * tid;
    bool ok0 = false, ok1 = false;  // the two cells are interior (per-cell class)
    if (inside) {
        ok0 = interior[c] != 0;
        ok1 = has1 && interior[c + 1] != 0;
        const int x1 = has1 ? x + 1 : x;
        const int oym = y == 0 ? (P.ny - 1) * P.nx : -P.nx, oyp = y == P.ny - 1 ? (1 - P.ny) * P.nx : P.nx;
        const int oxm0 = x == 0 ? P.nx - 1 : -1, oxp0 = x == P.nx - 1 ? 1 - P.nx : 1;
        const int oxm1 = x1 == 0 ? P.nx - 1 : -1, oxp1 = x1 == P.nx - 1 ? 1 - P.nx : 1;
        const float* gc0 = g_in + c;
        const float* gc1 = g_in + c + (x1 - x);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int oy = cy_of(i) > 0 ? oym : (cy_of(i) < 0 ? oyp : 0);
            const int o0 = (cx_of(i) > 0 ? oxm0 : (cx_of(i) < 0 ? oxp0 : 0)) + oy;
            const int o1 = (cx_of(i) > 0 ? oxm1 : (cx_of(i) < 0 ? oxp1 : 0)) + oy;
            const float* a0 = gc0 + (long long)i * N + o0;
            float* d = gs + i * 2 * NT;
            if (cx_of(i) == 0 && has1 && (reinterpret_cast<uintptr_t>(a0) & 7) == 0) {
                cp_async<8>(d, a0);
            } else {
                cp_async<4>(d, a0);
                cp_async<4>(d + 1, gc1 + (long long)i * N + o1);
            }
        }
    }
    if ((P.nx & 1) == 0)
        stage_tile2d_pairs<TX, TY, NT>(P, sm, x0, y0, tid, T_in, Y_in);
    else
        stage_tile2d<float, float, TX, TY, false, NT>(P, sm, x0, y0, tid, T_in, Y_in, nullptr);
    cp_async_wait_all();
    __syncthreads();

    if (!inside || (!ok0 && !ok1)) return;
    const int p0 = (threadIdx.y + 2) * SX + 2 * threadIdx.x + 2;
    F2 g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = F2(*reinterpret_cast<const float2*>(gs + i * 2 * NT));

    // a2
    const F2 T0 = pair_at(sm.T, p0), invW0 = pair_at(sm.invW, p0), rho0 = pair_at(sm.rho, p0);
    F2 Y0[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) Y0[k] = pair_at(sm.Y + k * NPT, p0);
    F2 u[3];
    {
        const F2 inv = fdiv(F2(3.f), rho0);
        u[0] = ((g[2] + g[5] + g[8]) - (g[0] + g[3] + g[6])) * inv;
        u[1] = ((g[6] + g[7] + g[8]) - (g[0] + g[1] + g[2])) * inv;
        u[2] = F2(0.f);
    }
    // a3-a5
    TileAccum<F2> acc;
    acc.clear();
    {
        auto line_x = [&](const float* f, F2* v) { pair_line<true, SX>(f, p0, v); };
        auto line_y = [&](const float* f, F2* v) { pair_line<false, SX>(f, p0, v); };
        fd_axis_core<F2>(P, sm, NPT, line_x, 0, u[0], Y0, invW0, rho0, acc);
        // the point values are read again from shared memory for each use
        // (the compiler barrier keeps them out of registers in between)
        asm volatile("" ::: "memory");
#pragma unroll
        for (int k = 0; k < NSP; ++k) Y0[k] = pair_at(sm.Y + k * NPT, p0);
        fd_axis_core<F2>(P, sm, NPT, line_y, 1, u[1], Y0, invW0, rho0, acc);
    }
    asm volatile("" ::: "memory");
#pragma unroll
    for (int k = 0; k < NSP; ++k) Y0[k] = pair_at(sm.Y + k * NPT, p0);
    // a6: per lane (the mixed form switches to FP64 above T_fp64)
    const F2 yf = pick_species(Y0, P.fuel), yo = pick_species(Y0, P.oxid);
    const F2 q(arrhenius(P, T0.v.x, yf.v.x, yo.v.x), arrhenius(P, T0.v.y, yf.v.y, yo.v.y));
    const F2 reac_T = F2(P.Q_cp) * q;
    // a7
    const F2 DT = acc.diff_T + reac_T;
    const bool vec = ok0 && ok1 && (c & 1) == 0;
    pair_store(T_out + c, T0 + (DT - acc.conv_T), ok0, ok1, vec);
#pragma unroll
    for (int k = 0; k < NSP; ++k)
        pair_store(Y_out + (long long)k * N + c, Y0[k] + (acc.rhs_Y[k] + F2(P.yield[k]) * q), ok0, ok1, vec);
    const F2 lam_Y = acc.lamY + F2(P.lam_yield) * q;
    const F2 Lam = fdiv(DT, T0) + fdiv(lam_Y, invW0);
    // a8-a10, on the populations read again from shared memory (the compiler
    // barrier keeps them out of registers during the FD part)
    asm volatile("" ::: "memory");
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = F2(*reinterpret_cast<const float2*>(gs + i * 2 * NT));
    collide<2, F2>(P, g, rho0, u, acc.grad_rho, Lam);
#pragma unroll
    for (int i = 0; i < 9; ++i) pair_store(g_out + (long long)i * N + c, g[i], ok0, ok1, vec);
}

}  // namespace lbfd
