// lbfd_geometry.cu -- curved walls described by analytic primitives.
//
// Host side, once per geometry: the wall distance fraction q of every cut
// lattice link (Sec. III.A, Eq. 30) and, for every solid cell within two
// cells of a fluid cell along an axis, its image point across the wall and
// the Shepard inverse-distance weights (p = 2) of the fluid cells within
// 4 dr of that point (Sec. III.B, Eq. 34-38).
// Device side, every step: the ghost values of the current state.
#include <cmath>
#include <vector>

#include "lbfd_device.cuh"
#include "lbfd_internal.h"

namespace lbfd {

namespace {

struct Geo {
    int dim, n[3];
    const int* bc;
    const uint8_t* solid;
    int nprims;
    const double* prims;  // 5 per primitive

    long long idx(int x, int y, int z) const { return (long long)x + (long long)n[0] * (y + (long long)n[1] * z); }
    void centre(int x, int y, int z, double c[3]) const
    {
        c[0] = x + 0.5;
        c[1] = y + 0.5;
        c[2] = dim == 3 ? z + 0.5 : 0.0;
    }
    bool inside(int k, const double* p) const
    {
        const double* P = prims + 5 * k;
        if ((int)P[0] == 0) {
            double r2 = 0.0;
            for (int a = 0; a < dim; ++a) r2 += (p[a] - P[1 + a]) * (p[a] - P[1 + a]);
            return r2 < P[4] * P[4];
        }
        double s = 0.0;
        for (int a = 0; a < dim; ++a) s += P[1 + a] * p[a];
        return s > P[4];
    }
    // point q (one step from a fluid cell along axis offsets) classification:
    // 0 fluid (periodic axes wrapped into *w), 1 solid cell (*w its index),
    // 2 outside through a non-periodic face
    int kind(int q[3], long long* w) const
    {
        for (int a = 0; a < dim; ++a) {
            if (q[a] >= 0 && q[a] < n[a]) continue;
            const int f = q[a] < 0 ? 2 * a : 2 * a + 1;
            if (bc[f] != BC_PERIODIC) return 2;
            q[a] = ((q[a] % n[a]) + n[a]) % n[a];
        }
        *w = idx(q[0], q[1], dim == 3 ? q[2] : 0);
        return solid[*w] ? 1 : 0;
    }
    // smallest t in (0, 1] at which x + t v enters a primitive, -1 if none
    double entry(const double x[3], const double v[3]) const
    {
        double best = -1.0;
        for (int k = 0; k < nprims; ++k) {
            const double* P = prims + 5 * k;
            double t = -1.0;
            if ((int)P[0] == 0) {
                double vv = 0.0, dv = 0.0, dd = 0.0;
                for (int a = 0; a < dim; ++a) {
                    const double d = x[a] - P[1 + a];
                    vv += v[a] * v[a];
                    dv += d * v[a];
                    dd += d * d;
                }
                const double disc = dv * dv - vv * (dd - P[4] * P[4]);
                if (disc >= 0.0 && vv > 0.0) t = (-dv - std::sqrt(disc)) / vv;
            } else {
                double nv = 0.0, nx = 0.0;
                for (int a = 0; a < dim; ++a) {
                    nv += P[1 + a] * v[a];
                    nx += P[1 + a] * x[a];
                }
                if (nv > 0.0) t = (P[4] - nx) / nv;
            }
            if (t > 0.0 && t <= 1.0 && (best < 0.0 || t < best)) best = t;
        }
        return best;
    }
    // nearest wall point of the primitives containing p
    bool wall_point(const double p[3], double B[3]) const
    {
        double bestd = INFINITY;
        bool found = false;
        for (int k = 0; k < nprims; ++k) {
            if (!inside(k, p)) continue;
            const double* P = prims + 5 * k;
            double c[3] = {0.0, 0.0, 0.0}, dist;
            if ((int)P[0] == 0) {
                double r = 0.0;
                for (int a = 0; a < dim; ++a) r += (p[a] - P[1 + a]) * (p[a] - P[1 + a]);
                r = std::sqrt(r);
                if (r < 1e-12) continue;
                for (int a = 0; a < dim; ++a) c[a] = P[1 + a] + P[4] * (p[a] - P[1 + a]) / r;
                dist = P[4] - r;
            } else {
                double s = 0.0;
                for (int a = 0; a < dim; ++a) s += P[1 + a] * p[a];
                dist = s - P[4];
                for (int a = 0; a < dim; ++a) c[a] = p[a] - dist * P[1 + a];
            }
            if (dist < bestd) {
                bestd = dist;
                B[0] = c[0];
                B[1] = c[1];
                B[2] = c[2];
                found = true;
            }
        }
        return found;
    }
};

}  // namespace

int build_curved_tables(int dim, int nx, int ny, int nz, const int* bc, const uint8_t* solid, int nprims,
                        const double* prims, CurvedTables& out)
{
    Geo G{dim, {nx, ny, dim == 3 ? nz : 1}, bc, solid, nprims, prims};
    const int Q = dim == 2 ? 9 : 27;
    const int NZ = G.n[2];
    const long long ncell = (long long)nx * ny * NZ;
    out.link_row.assign((size_t)ncell, -1);
    out.ghost_row.assign((size_t)ncell, -1);
    out.link_q.clear();
    out.gh_start.assign(1, 0);
    out.gh_idx.clear();
    out.gh_w.clear();
    // cut links: a fluid cell pulls population i from a solid cell
    for (int z = 0; z < NZ; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long long c = G.idx(x, y, z);
                if (solid[c]) continue;
                double xc[3];
                G.centre(x, y, z, xc);
                int row = -1;
                for (int i = 0; i < Q; ++i) {
                    const int ci[3] = {i % 3 - 1, (i / 3) % 3 - 1, dim == 3 ? i / 9 - 1 : 0};
                    int q[3] = {x - ci[0], y - ci[1], z - ci[2]};
                    long long w;
                    if (G.kind(q, &w) != 1) continue;
                    if (row < 0) {
                        row = (int)(out.link_q.size() / Q);
                        out.link_q.resize(out.link_q.size() + Q, -1.0);
                        out.link_row[c] = row;
                    }
                    const double v[3] = {-(double)ci[0], -(double)ci[1], -(double)ci[2]};
                    out.link_q[(size_t)row * Q + i] = G.entry(xc, v);
                }
            }
    // ghosts: solid cells within two cells of a fluid cell along an axis
    long long ng = 0;
    for (int z = 0; z < NZ; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long long c = G.idx(x, y, z);
                if (!solid[c]) continue;
                bool near = false;
                for (int a = 0; a < dim && !near; ++a)
                    for (int d = -2; d <= 2 && !near; ++d) {
                        if (!d) continue;
                        int q[3] = {x, y, z};
                        q[a] += d;
                        long long w;
                        near = G.kind(q, &w) == 0;
                    }
                if (!near) continue;
                double pc[3], B[3], I[3] = {0.0, 0.0, 0.0};
                G.centre(x, y, z, pc);
                if (!G.wall_point(pc, B)) continue;
                for (int a = 0; a < dim; ++a) I[a] = 2.0 * B[a] - pc[a];
                int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
                for (int a = 0; a < dim; ++a) {
                    lo[a] = std::max(0, (int)std::floor(I[a] - 4.5) - 1);
                    hi[a] = std::min(G.n[a] - 1, (int)std::ceil(I[a] + 3.5) + 1);
                }
                const size_t first = out.gh_idx.size();
                long long exact = -1;
                double wsum = 0.0;
                for (int zz = lo[2]; zz <= hi[2]; ++zz)
                    for (int yy = lo[1]; yy <= hi[1]; ++yy)
                        for (int xx = lo[0]; xx <= hi[0]; ++xx) {
                            const long long j = G.idx(xx, yy, zz);
                            if (solid[j]) continue;
                            double rc[3], d2 = 0.0;
                            G.centre(xx, yy, zz, rc);
                            for (int a = 0; a < dim; ++a) d2 += (rc[a] - I[a]) * (rc[a] - I[a]);
                            if (d2 > 16.0) continue;  // within 4 dr of the image point (Eq. 38)
                            if (d2 < 1e-18) exact = (long long)(out.gh_idx.size() - first);
                            out.gh_idx.push_back(j);
                            out.gh_w.push_back(d2 < 1e-18 ? 0.0 : 1.0 / d2);  // d^-p, p = 2 (Eq. 36)
                            wsum += out.gh_w.back();
                        }
                if (out.gh_idx.size() == first) continue;  // no fluid near the image: staircase
                for (size_t e = first; e < out.gh_idx.size(); ++e)
                    out.gh_w[e] = exact >= 0 ? ((long long)(e - first) == exact ? 1.0 : 0.0) : out.gh_w[e] / wsum;
                out.ghost_row[c] = (int)ng;
                out.gh_start.push_back((long long)out.gh_idx.size());
                ++ng;
            }
    out.nghost = ng;
    return 0;
}

// ghost values of the current state: Shepard values at the image point
// (Eq. 35; the density is reconstructed itself) and Eq. 34 on top
template <typename S, typename R>
__global__ void __launch_bounds__(128) ghost_fill_kernel(StepParams<R> P, const S* __restrict__ T,
                                                         const S* __restrict__ Y,
                                                         const long long* __restrict__ start,
                                                         const long long* __restrict__ nb,
                                                         const double* __restrict__ w, long long nghost,
                                                         R* __restrict__ gval)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nghost) return;
    R TI = R(0), rI = R(0), YI[NSP];
#pragma unroll
    for (int s = 0; s < NSP; ++s) YI[s] = R(0);
    for (long long e = start[k]; e < start[k + 1]; ++e) {
        const long long j = nb[e];
        const R wj = R(w[e]);
        const R Tj = R(T[j]);
        R Yj[NSP];
#pragma unroll
        for (int s = 0; s < NSP; ++s) Yj[s] = R(Y[(long long)s * P.N + j]);
        TI += wj * Tj;
        rI += wj * eos(P, Tj, inv_molar_mass(P, Yj));
#pragma unroll
        for (int s = 0; s < NSP; ++s) YI[s] += wj * Yj[s];
    }
    R* gv = gval + k * GHOST_VALUES;
    const R invW = inv_molar_mass(P, YI);
#pragma unroll
    for (int s = 0; s < NSP; ++s) {
        gv[1 + s] = YI[s];  // species: Neumann
        gv[2 + NSP + s] = YI[s] * P.inv_Wk[s] / invW;
    }
    gv[1 + NSP] = invW;
    if (P.solid_isothermal) {
        gv[0] = R(2) * P.T_solid - TI;
        gv[2 + 2 * NSP] = R(2) * eos(P, P.T_solid, invW) - rI;
    } else {
        gv[0] = TI;
        gv[2 + 2 * NSP] = rI;
    }
}

cudaError_t launch_ghost_fill(int precision, const StepParams<double>& Pd, const StepParams<float>& Pf,
                              const StepParams<Tan>& Pt, StateView in, const long long* start, const long long* nb,
                              const double* w, long long nghost, cudaStream_t stream)
{
    if (nghost <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((nghost + 127) / 128);
    if (precision == 0)
        ghost_fill_kernel<double, double><<<blocks, 128, 0, stream>>>(Pd, (const double*)in.T, (const double*)in.Y,
                                                                      start, nb, w, nghost, (double*)Pd.gval);
    else if (precision == 1)
        ghost_fill_kernel<float, float><<<blocks, 128, 0, stream>>>(Pf, (const float*)in.T, (const float*)in.Y,
                                                                    start, nb, w, nghost, (float*)Pf.gval);
    else
        ghost_fill_kernel<Tan, Tan><<<blocks, 128, 0, stream>>>(Pt, (const Tan*)in.T, (const Tan*)in.Y, start, nb,
                                                                w, nghost, (Tan*)Pt.gval);
    return cudaGetLastError();
}

}  // namespace lbfd
