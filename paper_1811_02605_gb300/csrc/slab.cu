// Radial slabs of a grid for domain decomposition (Sec. 4.2: each MPI rank, one per GPU, owns a
// part of the mesh; a PCG iteration exchanges the boundary values its operator application needs
// and reduces the few scalars of its inner products across the ranks).
//
// A slab grid holds the global rows [i0, i1) of a grid: its metric and operator tables are the
// global ones of those rows, so the diagonal of M_alpha at a slab's edge row includes the face it
// shares with the neighbouring slab. The operator call takes that neighbour's boundary plane as a
// ghost plane and evaluates, row for row, the same expression in the same order as the
// single-grid operator (k_apply64), so a slab's rows of M p have the bits of the global M p.
// The PCG vector kernels are those of the unscaled point-Jacobi form (z = r / diag M): x += a p,
// r -= a q, z = r / d with the slab's shares of <r, z> and <r, r>; p = z + beta p. The caller (the
// distributed driver in dist.py) exchanges the ghost planes and sums the shares over the ranks.
#include <cmath>

#include "mhd_internal.cuh"
#include "reduce.cuh"

using namespace mhd;

namespace {

// interface couplings of the slab's edge rows: alpha times the shared face's weight, 0 at the
// domain's own walls (the Dirichlet weight of r0 sits on the diagonal, r1 has none)
__global__ void k_slab_couplings(Dims d, Geo G, double alpha, int lo_if, int hi_if, double* __restrict__ clo,
                                 double* __restrict__ chi) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d.nt) return;
    clo[j] = lo_if ? alpha * G.wr[j] : 0.0;
    chi[j] = hi_if ? alpha * G.wr[(size_t)d.nr * d.nt + j] : 0.0;
}

__global__ void k_set_alpha_slab(double* a, double v) { *a = v; }

// q = M p on the slab with ghost planes plo (row i0-1) and phi (row i1); share of <p, q>
__global__ void __launch_bounds__(kThreads) k_slab_apply(Dims d, int nc, const double* __restrict__ p,
                                                         const double* __restrict__ plo,
                                                         const double* __restrict__ phi, double* __restrict__ q,
                                                         OpTab64u tu, const double* __restrict__ clo,
                                                         const double* __restrict__ chi, unsigned int* count,
                                                         double* __restrict__ partials, double* __restrict__ out) {
    const int nt = d.nt, np = d.np;
    const long long plane = (long long)nt * np;
    const long long G = d.N;
    double acc = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < G; e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e % np);
        const long long ij = e / np;
        const int j = (int)(ij % nt), i = (int)(ij / nt);
        const double dg = tu.dg[ij];
        const double wl = (i > 0) ? tu.awr[i * nt + j] : clo[j];
        const double wh = (i < d.nr - 1) ? tu.awr[(i + 1) * nt + j] : chi[j];
        const double tl = tu.awt[i * (nt + 1) + j], th = tu.awt[i * (nt + 1) + j + 1];
        const double wp = tu.awp[ij];
        const int km = (k == 0) ? np - 1 : k - 1;
        const int kp = (k == np - 1) ? 0 : k + 1;
        for (int c = 0; c < nc; c++) {
            const double* u = p + c * G;
            const double uc = u[e];
            double mx = dg * uc - wp * (u[e - k + km] + u[e - k + kp]);
            if (i > 0) mx -= wl * u[e - plane];
            else if (plo) mx -= wl * plo[c * plane + j * np + k];
            if (i < d.nr - 1) mx -= wh * u[e + plane];
            else if (phi) mx -= wh * phi[c * plane + j * np + k];
            if (j > 0) mx -= tl * u[e - np];
            if (j < nt - 1) mx -= th * u[e + np];
            q[c * G + e] = mx;
            acc = fma(uc, mx, acc);
        }
    }
    double v[1] = {acc}, o[1];
    if (reduce_last<1>(v, partials, count, o) && threadIdx.x == 0) {
        out[0] = o[0];
        *count = 0u;
    }
}

// x += a p (x may be null), r -= a q, z = r / dg; shares of <r, z> and <r, r>
__global__ void __launch_bounds__(kThreads) k_slab_update(Dims d, int nc, double a, double* __restrict__ x,
                                                          const double* __restrict__ p, double* __restrict__ r,
                                                          const double* __restrict__ q, double* __restrict__ z,
                                                          const double* __restrict__ dg, unsigned int* count,
                                                          double* __restrict__ partials, double* __restrict__ out) {
    const long long G = d.N;
    const int np = d.np;
    double rz = 0.0, rr = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < G; e += (long long)gridDim.x * blockDim.x) {
        const double di = dg[e / np];
        for (int c = 0; c < nc; c++) {
            const long long o = c * G + e;
            if (x) x[o] += a * p[o];
            const double rv = r[o] - a * q[o];
            const double zv = rv / di;
            r[o] = rv;
            z[o] = zv;
            rz = fma(rv, zv, rz);
            rr = fma(rv, rv, rr);
        }
    }
    double v[2] = {rz, rr}, o2[2];
    if (reduce_last<2>(v, partials, count, o2) && threadIdx.x == 0) {
        out[0] = o2[0];
        out[1] = o2[1];
        *count = 0u;
    }
}

// p = z + beta p (p = z when beta == 0, whatever p held)
__global__ void __launch_bounds__(kThreads) k_slab_pupdate(long long n, double beta, const double* __restrict__ z,
                                                           double* __restrict__ p) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        p[e] = (beta == 0.0) ? z[e] : z[e] + beta * p[e];
}

bool is_slab(const mhd_grid_s* g) { return g->slab_nr_global > 0; }

mhd_status_t read_out(mhd_grid_s* g, double* host, int n) {
    if (cudaMemcpyAsync(g->h_alpha, g->slab_out, sizeof(double) * n, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
        cudaStreamSynchronize(g->stream) != cudaSuccess)
        return check_cuda(g, "slab: read");
    for (int q = 0; q < n; q++) host[q] = g->h_alpha[q];
    return MHD_OK;
}

}  // namespace

extern "C" mhd_status_t mhd_slab_apply(mhd_grid_t g, double alpha, int ncomp, const double* p, const double* p_lo,
                                       const double* p_hi, double* q, double* pq) {
    if (!g) return MHD_ERR_ARG;
    if (!is_slab(g)) return set_error(g, MHD_ERR_ARG, "mhd_slab_apply: not a slab grid (mhd_grid_create_slab)");
    if (ncomp < 1 || ncomp > 3 || !p || !q || p == q || !(alpha >= 0.0))
        return set_error(g, MHD_ERR_ARG, "mhd_slab_apply: need 1 <= ncomp <= 3, distinct p, q, alpha >= 0");
    if ((g->slab_i0 > 0) != (p_lo != nullptr) || (g->slab_i0 + g->d.nr < g->slab_nr_global) != (p_hi != nullptr))
        return set_error(g, MHD_ERR_ARG, "mhd_slab_apply: a ghost plane is given exactly where a neighbour slab is");
    const Dims d = g->d;
    k_set_alpha_slab<<<1, 1, 0, g->stream>>>(&g->ss->alpha_user, alpha);
    build_tables(g, &g->ss->alpha_user, false);
    k_slab_couplings<<<(d.nt + 127) / 128, 128, 0, g->stream>>>(d, g->geo, alpha, g->slab_i0 > 0 ? 1 : 0,
                                                               g->slab_i0 + d.nr < g->slab_nr_global ? 1 : 0,
                                                               g->slab_out + 8, g->slab_out + 8 + d.nt);
    k_slab_apply<<<grid_blocks(g, d.N, 8), kThreads, 0, g->stream>>>(d, ncomp, p, p_lo, p_hi, q, g->tu, g->slab_out + 8,
                                                                      g->slab_out + 8 + d.nt, &g->ss->count,
                                                                      g->partials, g->slab_out);
    mhd_status_t st = check_cuda(g, "mhd_slab_apply");
    if (st != MHD_OK) return st;
    if (!pq) return MHD_OK;
    return read_out(g, pq, 1);
}

extern "C" mhd_status_t mhd_slab_update(mhd_grid_t g, double alpha, int ncomp, double a, double* x, const double* p,
                                        double* r, const double* q, double* z, double dots[2]) {
    if (!g) return MHD_ERR_ARG;
    if (!is_slab(g)) return set_error(g, MHD_ERR_ARG, "mhd_slab_update: not a slab grid");
    if (ncomp < 1 || ncomp > 3 || !r || !q || !z || !dots || (x && !p) || !(alpha >= 0.0))
        return set_error(g, MHD_ERR_ARG, "mhd_slab_update: bad argument");
    const Dims d = g->d;
    k_set_alpha_slab<<<1, 1, 0, g->stream>>>(&g->ss->alpha_user, alpha);
    build_tables(g, &g->ss->alpha_user, false);
    k_slab_update<<<grid_blocks(g, d.N, 8), kThreads, 0, g->stream>>>(d, ncomp, a, x, p, r, q, z, g->tu.dg,
                                                                       &g->ss->count, g->partials, g->slab_out);
    mhd_status_t st = check_cuda(g, "mhd_slab_update");
    if (st != MHD_OK) return st;
    return read_out(g, dots, 2);
}

extern "C" mhd_status_t mhd_slab_pupdate(mhd_grid_t g, int ncomp, double beta, const double* z, double* p) {
    if (!g) return MHD_ERR_ARG;
    if (!is_slab(g)) return set_error(g, MHD_ERR_ARG, "mhd_slab_pupdate: not a slab grid");
    if (ncomp < 1 || ncomp > 3 || !z || !p || z == p) return set_error(g, MHD_ERR_ARG, "mhd_slab_pupdate: bad argument");
    const long long n = (long long)ncomp * g->d.N;
    k_slab_pupdate<<<grid_blocks(g, n, 8), kThreads, 0, g->stream>>>(n, beta, z, p);
    return check_cuda(g, "mhd_slab_pupdate");
}
