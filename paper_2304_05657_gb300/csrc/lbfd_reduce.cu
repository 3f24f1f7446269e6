// lbfd_reduce.cu -- FP64 reductions over the fluid cells (flame position,
// mass, heat release, fuel consumption, max T, non-finite count) and the
// per-cell field read-out kernel.
//
// Observables: flame front by maximum heat release (Sec. IV.A dead-zone
// analysis; Sec. IV.B burner), consumption speed integrals (Sec. IV.C,
// Eq. 40), and an integral flame position (unburnt length).
#include <cmath>

#include "lbfd_device.cuh"
#include "lbfd_internal.h"

namespace lbfd {

__device__ __forceinline__ unsigned long long order_key(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

template <typename S>
__device__ __forceinline__ double hrr_of(const StepParams<double>& P, double T, const double* Y, double* rho_out,
                                         double* q_out)
{
    double invW = 0.0;
#pragma unroll
    for (int k = 0; k < NSP; ++k) invW += Y[k] * P.inv_Wk[k];
    const double rho = P.T_in * P.invW_in / (T * invW);
    const double yf = Y[P.fuel] > 0.0 ? Y[P.fuel] : 0.0;
    const double yo = Y[P.oxid] > 0.0 ? Y[P.oxid] : 0.0;
    const double q = P.A_lat * yf * yo * ::exp(-P.Ta / T);
    *rho_out = rho;
    *q_out = q;
    return rho * P.Q_cp * q;
}

// red layout: [0] sum Y_F, [1] mass, [2] hrr, [3] fuel, [4] max-T key (u64),
// [5] non-finite count (u64), [6] fluid count (u64), [7] x=0 section count (u64),
// [8] centre-line max hrr, [9] its x
template <int DIM, typename S>
__global__ void __launch_bounds__(256) diag_kernel(StepParams<double> P, const S* __restrict__ g,
                                                   const S* __restrict__ T, const S* __restrict__ Y,
                                                   const uint8_t* __restrict__ solid, int y0, int y1, double* red)
{
    constexpr int Q = DIM == 2 ? 9 : 27;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    unsigned long long tkey = 0ull, nonf = 0ull, nfl = 0ull, sec = 0ull;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int rows = y1 - y0;
    const long long ncount = (long long)P.nx * rows * P.nz;  // cells with y0 <= y < y1
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < ncount; t += stride) {
        const long long r = t / P.nx;
        const long long c = t % P.nx + (long long)P.nx * (y0 + r % rows + (long long)P.ny * (r / rows));
        if (solid[c]) continue;
        ++nfl;
        if (c % P.nx == 0) ++sec;
        const double Tc = val(T[c]);
        double Yc[NSP];
        bool bad = !isfinite(Tc);
#pragma unroll
        for (int k = 0; k < NSP; ++k) {
            Yc[k] = val(Y[(long long)k * P.N + c]);
            bad |= !isfinite(Yc[k]);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) bad |= !isfinite(val(g[(long long)i * P.N + c]));
        if (bad) {
            ++nonf;
            continue;
        }
        double rho, q;
        const double h = hrr_of<S>(P, Tc, Yc, &rho, &q);
        s[0] += Yc[P.fuel];
        s[1] += rho;
        s[2] += h;
        s[3] += rho * q;
        const unsigned long long k = order_key(Tc);
        tkey = k > tkey ? k : tkey;
    }
    // warp then block reduction
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int j = 0; j < 4; ++j) s[j] += __shfl_down_sync(0xffffffffu, s[j], off);
        const unsigned long long o = __shfl_down_sync(0xffffffffu, tkey, off);
        tkey = o > tkey ? o : tkey;
        nonf += __shfl_down_sync(0xffffffffu, nonf, off);
        nfl += __shfl_down_sync(0xffffffffu, nfl, off);
        sec += __shfl_down_sync(0xffffffffu, sec, off);
    }
    __shared__ double sh[8][4];
    __shared__ unsigned long long shk[8][4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) sh[wid][j] = s[j];
        shk[wid][0] = tkey;
        shk[wid][1] = nonf;
        shk[wid][2] = nfl;
        shk[wid][3] = sec;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int w = 1; w < nw; ++w) {
            for (int j = 0; j < 4; ++j) s[j] += sh[w][j];
            tkey = shk[w][0] > tkey ? shk[w][0] : tkey;
            nonf += shk[w][1];
            nfl += shk[w][2];
            sec += shk[w][3];
        }
        for (int j = 0; j < 4; ++j) atomicAdd(&red[j], s[j]);
        unsigned long long* ru = reinterpret_cast<unsigned long long*>(red);
        atomicMax(&ru[4], tkey);
        atomicAdd(&ru[5], nonf);
        atomicAdd(&ru[6], nfl);
        atomicAdd(&ru[7], sec);
    }
}

// one block: argmax of the heat release on the line y = ny/2, z = nz/2
template <int DIM, typename S>
__global__ void __launch_bounds__(1024) centreline_kernel(StepParams<double> P, const S* __restrict__ T,
                                                          const S* __restrict__ Y,
                                                          const uint8_t* __restrict__ solid, int y0, int y1,
                                                          double* red)
{
    double best = -INFINITY;
    int bx = -1;
    const int yc = (y0 + y1) / 2, zc = DIM == 3 ? P.nz / 2 : 0;
    for (int x = threadIdx.x; x < P.nx; x += blockDim.x) {
        const long long c = x + (long long)P.nx * (yc + (long long)P.ny * zc);
        if (solid[c]) continue;
        const double Tc = val(T[c]);
        double Yc[NSP];
        bool bad = !isfinite(Tc);
#pragma unroll
        for (int k = 0; k < NSP; ++k) {
            Yc[k] = val(Y[(long long)k * P.N + c]);
            bad |= !isfinite(Yc[k]);
        }
        if (bad) continue;
        double rho, q;
        const double h = hrr_of<S>(P, Tc, Yc, &rho, &q);
        if (h > best) {  // x increases along the loop: ties keep the smaller x
            best = h;
            bx = x;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int ox = __shfl_down_sync(0xffffffffu, bx, off);
        if (ox >= 0 && (bx < 0 || ob > best || (ob == best && ox < bx))) {
            best = ob;
            bx = ox;
        }
    }
    __shared__ double sb[32];
    __shared__ int sx[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sb[wid] = best;
        sx[wid] = bx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int w = 1; w < nw; ++w) {
            if (sx[w] >= 0 && (bx < 0 || sb[w] > best || (sb[w] == best && sx[w] < bx))) {
                best = sb[w];
                bx = sx[w];
            }
        }
        red[8] = best;
        red[9] = (double)bx;
    }
}

template <int DIM, typename S>
static cudaError_t diag_launch(const StepParams<double>& P, StateView st, const uint8_t* solid, int y0, int y1,
                               double* red, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(red, 0, RED_WORDS * sizeof(double), stream);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = ((long long)P.nx * (y1 - y0) * P.nz + 255) / 256;
    long long cap = (long long)(sms > 0 ? sms : 1) * 8;
    const unsigned blocks = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
    diag_kernel<DIM, S><<<blocks, 256, 0, stream>>>(P, (const S*)st.g, (const S*)st.T, (const S*)st.Y, solid, y0, y1,
                                                    red);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    centreline_kernel<DIM, S><<<1, 1024, 0, stream>>>(P, (const S*)st.T, (const S*)st.Y, solid, y0, y1, red);
    return cudaGetLastError();
}

cudaError_t launch_diagnostics(int dim, int precision, const StepParams<double>& P, StateView st,
                               const uint8_t* solid, int y0, int y1, double* red, cudaStream_t stream)
{
    if (precision == 0)
        return dim == 2 ? diag_launch<2, double>(P, st, solid, y0, y1, red, stream)
                        : diag_launch<3, double>(P, st, solid, y0, y1, red, stream);
    if (precision == 2)
        return dim == 2 ? diag_launch<2, Tan>(P, st, solid, y0, y1, red, stream) : cudaErrorInvalidValue;
    if (precision == 3)
        return dim == 2 ? diag_launch<2, Tanf>(P, st, solid, y0, y1, red, stream) : cudaErrorInvalidValue;
    return dim == 2 ? diag_launch<2, float>(P, st, solid, y0, y1, red, stream)
                    : diag_launch<3, float>(P, st, solid, y0, y1, red, stream);
}

// Per column x of a 2-D grid: the peak heat release over the fluid cells of
// rows y0 <= y < y1 (the reaction front where it crosses the column, Sec.
// IV.A) and the distance of that cell's centre to the nearer edge of the
// row band (walls half-way between cells): out[x] = peak (0 when the column
// has no fluid cell there), out[nx + x] = distance (smallest y on ties).
template <typename S>
__global__ void __launch_bounds__(256) column_peaks_kernel(StepParams<double> P, const S* __restrict__ T,
                                                           const S* __restrict__ Y,
                                                           const uint8_t* __restrict__ solid, int y0, int y1,
                                                           double* __restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= P.nx) return;
    double best = -1.0;
    int by = y0;
    for (int y = y0; y < y1; ++y) {
        const long long c = (long long)x + (long long)P.nx * y;
        if (solid[c]) continue;
        double Yc[NSP];
#pragma unroll
        for (int k = 0; k < NSP; ++k) Yc[k] = val(Y[(long long)k * P.N + c]);
        double rho, q;
        const double h = hrr_of<S>(P, val(T[c]), Yc, &rho, &q);
        if (h > best) {
            best = h;
            by = y;
        }
    }
    const double d0 = by - y0 + 0.5, d1 = y1 - 0.5 - by;
    out[x] = best < 0.0 ? 0.0 : best;
    out[P.nx + x] = d0 < d1 ? d0 : d1;
}

cudaError_t launch_column_peaks(int precision, const StepParams<double>& P, StateView st, const uint8_t* solid,
                                int y0, int y1, double* out, cudaStream_t stream)
{
    const unsigned nb = (unsigned)((P.nx + 255) / 256);
    if (precision == 0)
        column_peaks_kernel<double><<<nb, 256, 0, stream>>>(P, (const double*)st.T, (const double*)st.Y, solid, y0,
                                                            y1, out);
    else if (precision == 1)
        column_peaks_kernel<float><<<nb, 256, 0, stream>>>(P, (const float*)st.T, (const float*)st.Y, solid, y0, y1,
                                                           out);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// field ids follow include/lbfd.h
template <int DIM, typename S>
__global__ void __launch_bounds__(256) field_kernel(StepParams<double> P, const S* __restrict__ g,
                                                    const S* __restrict__ T, const S* __restrict__ Y,
                                                    const uint8_t* __restrict__ solid, int field,
                                                    double* __restrict__ out)
{
    constexpr int Q = DIM == 2 ? 9 : 27;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.ncell) return;
    if (field >= 16) {
        out[c] = val(g[(long long)(field - 16) * P.N + c]);
        return;
    }
    if (field == 0) {
        out[c] = val(T[c]);
        return;
    }
    if (field >= 1 && field <= NSP) {
        out[c] = val(Y[(long long)(field - 1) * P.N + c]);
        return;
    }
    const double Tc = val(T[c]);
    double Yc[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) Yc[k] = val(Y[(long long)k * P.N + c]);
    double rho, q;
    const double h = hrr_of<S>(P, Tc, Yc, &rho, &q);
    double v = 0.0;
    if (field >= 6 && field <= 8) {
        const int a = field - 6;
        if (a < DIM) {
            double m = 0.0;
#pragma unroll
            for (int i = 0; i < Q; ++i) m += (double)ccomp<DIM>(i, a) * val(g[(long long)i * P.N + c]);
            v = 3.0 * m / rho;
        }
    } else if (field == 9) {
#pragma unroll
        for (int i = 0; i < Q; ++i) v += val(g[(long long)i * P.N + c]);
    } else if (field == 10) {
        v = rho;
    } else if (field == 11) {
        v = h;
    }
    out[c] = v;
}

// the whole state (g_0..g_{Q-1}, T, Y_0..Y_{NSP-1}) of listed cells
template <typename S>
__global__ void __launch_bounds__(256) cells_kernel(long long N, int Q, const S* __restrict__ g,
                                                    const S* __restrict__ T, const S* __restrict__ Y,
                                                    const long long* __restrict__ cells, long long n,
                                                    double* __restrict__ out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const long long c = cells[t];
    double* o = out + t * (Q + 1 + NSP);
    for (int i = 0; i < Q; ++i) o[i] = val(g[(long long)i * N + c]);
    o[Q] = val(T[c]);
    for (int k = 0; k < NSP; ++k) o[Q + 1 + k] = val(Y[(long long)k * N + c]);
}

cudaError_t launch_cells(int dim, int precision, const StepParams<double>& P, StateView st, const long long* cells,
                         long long n, double* out, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    const int Q = dim == 2 ? 9 : 27;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (precision == 2)
        cells_kernel<Tan><<<blocks, 256, 0, stream>>>(P.N, Q, (const Tan*)st.g, (const Tan*)st.T, (const Tan*)st.Y,
                                                      cells, n, out);
    else if (precision == 3)
        cells_kernel<Tanf><<<blocks, 256, 0, stream>>>(P.N, Q, (const Tanf*)st.g, (const Tanf*)st.T,
                                                       (const Tanf*)st.Y, cells, n, out);
    else if (precision == 0)
        cells_kernel<double><<<blocks, 256, 0, stream>>>(P.N, Q, (const double*)st.g, (const double*)st.T,
                                                         (const double*)st.Y, cells, n, out);
    else
        cells_kernel<float><<<blocks, 256, 0, stream>>>(P.N, Q, (const float*)st.g, (const float*)st.T,
                                                        (const float*)st.Y, cells, n, out);
    return cudaGetLastError();
}

cudaError_t launch_field(int dim, int precision, const StepParams<double>& P, StateView st, const uint8_t* solid,
                         int field, double* out, cudaStream_t stream)
{
    const unsigned blocks = (unsigned)((P.ncell + 255) / 256);
    if (precision == 2) {
        if (dim != 2) return cudaErrorInvalidValue;
        field_kernel<2, Tan><<<blocks, 256, 0, stream>>>(P, (const Tan*)st.g, (const Tan*)st.T, (const Tan*)st.Y,
                                                          solid, field, out);
        return cudaGetLastError();
    }
    if (precision == 3) {
        if (dim != 2) return cudaErrorInvalidValue;
        field_kernel<2, Tanf><<<blocks, 256, 0, stream>>>(P, (const Tanf*)st.g, (const Tanf*)st.T, (const Tanf*)st.Y,
                                                          solid, field, out);
        return cudaGetLastError();
    }
    if (precision == 0) {
        if (dim == 2)
            field_kernel<2, double><<<blocks, 256, 0, stream>>>(P, (const double*)st.g, (const double*)st.T,
                                                                 (const double*)st.Y, solid, field, out);
        else
            field_kernel<3, double><<<blocks, 256, 0, stream>>>(P, (const double*)st.g, (const double*)st.T,
                                                                 (const double*)st.Y, solid, field, out);
    } else {
        if (dim == 2)
            field_kernel<2, float><<<blocks, 256, 0, stream>>>(P, (const float*)st.g, (const float*)st.T,
                                                                (const float*)st.Y, solid, field, out);
        else
            field_kernel<3, float><<<blocks, 256, 0, stream>>>(P, (const float*)st.g, (const float*)st.T,
                                                                (const float*)st.Y, solid, field, out);
    }
    return cudaGetLastError();
}

}  // namespace lbfd
