// Viscosity by RKL2 super time-stepping (Sec. 2.2: the STS option for diffusive terms, the
// paper's GPU choice in algorithm 3; second-order Runge-Kutta-Legendre scheme of Meyer, Balsara &
// Aslam 2014). It advances rho V dv/dt = -nu K v over dt with s explicit stages:
//   Y_1 = Y_0 + b_1 w1 dt L(Y_0)
//   Y_j = mu_j Y_{j-1} + nv_j Y_{j-2} + (1 - mu_j - nv_j) Y_0 + mu_j w1 dt L(Y_{j-1})
//         - (1 - b_{j-1}) mu_j w1 dt L(Y_0)
// with b_j = (j^2 + j - 2) / (2 j (j + 1)) (b_0 = b_1 = 1/3), w1 = 4 / (s^2 + s - 2),
// mu_j = (2j - 1)/j b_j / b_{j-1}, nv_j = -(j - 1)/j b_j / b_{j-2}, L(v) = -nu D^-1 K v.
// s is the smallest s >= 2 with (s^2 + s - 2)/2 >= dt lambda_max, lambda_max the Gershgorin bound
// of nu D^-1 K (computed once per grid).
//
// GPU form: the stages carry the differences D_j = Y_j - Y_0. L is linear (the Dirichlet wall
// value is zero), so dt L(Y_{j-1}) = ly0 + dt L(D_{j-1}) with ly0 = dt L(Y_0), and
//   D_j = mu_j D_{j-1} + nv_j D_{j-2} + mu~_j dt L(D_{j-1}) + (mu~_j + ga~_j) ly0,
// mu~_j = mu_j w1, ga~_j = -(1 - b_{j-1}) mu~_j, D_0 = 0, D_1 = b_1 w1 ly0, Y_s = Y_0 + D_s.
// One fused kernel per stage: stencil of D_{j-1}, reads of D_{j-2} and ly0, one write (4 arrays
// of 3N doubles instead of the 5 of the Y form), and no copy of Y_0 (it stays in the caller's
// buffer until the last stage adds it).
#include <cmath>

#include "mhd_internal.cuh"

namespace mhd {

namespace {

constexpr int kTab = 8;   // doubles per (i, j) in the stage coefficient table

// T[ij] = nu dt / (rho V) * {K diagonal, w_phi, w_r low, w_r high, w_theta low, w_theta high}
// (a face with no neighbour inside the grid contributes 0 off-diagonal; the Dirichlet weight at
// r0 and the Neumann face at r1 are in the diagonal as in K)
__global__ void k_sts_tab(Dims d, Geo G, double nu, const double* __restrict__ dt_p, double* __restrict__ T) {
    const double dt = *dt_p;
    const int nt = d.nt;
    for (int ij = blockIdx.x * blockDim.x + threadIdx.x; ij < d.nr * nt; ij += gridDim.x * blockDim.x) {
        const int i = ij / nt, j = ij - i * nt;
        const double h = nu * dt / G.rhoV[ij];
        const double wrl = G.wr[i * nt + j], wrh = G.wr[(i + 1) * nt + j];
        const double wtl = G.wt[i * (nt + 1) + j], wth = G.wt[i * (nt + 1) + j + 1];
        const double wp = G.wp[ij];
        double* t = T + (size_t)ij * kTab;
        t[0] = h * (wrl + wrh + wtl + wth + 2.0 * wp);
        t[1] = h * wp;
        t[2] = (i > 0) ? h * wrl : 0.0;
        t[3] = (i < d.nr - 1) ? h * wrh : 0.0;
        t[4] = (j > 0) ? h * wtl : 0.0;
        t[5] = (j < nt - 1) ? h * wth : 0.0;
        t[6] = 0.0;
        t[7] = 0.0;
    }
}

struct Pair {
    unsigned int ij;
    int i, j, k0;
    long long base;
};

__device__ __forceinline__ Pair pair_of(const Dims& d, unsigned int g) {
    const unsigned int npv = d.np / 2;
    Pair p;
    p.ij = g / npv;
    p.k0 = (int)(g - p.ij * npv) * 2;
    p.i = (int)(p.ij / d.nt);
    p.j = (int)(p.ij - (unsigned)p.i * d.nt);
    p.base = (long long)p.ij * d.np + p.k0;
    return p;
}

// o = ca u + cp (u_{k-1} + u_{k+1}) + sum over in-grid neighbours c_n u_n, for the two cells of a
// phi-pair (coefficients already scaled by the caller)
__device__ __forceinline__ void stencil2(const Dims& d, const Pair& P, const double* __restrict__ u, double ca,
                                         double cp, double crl, double crh, double ctl, double cth, double2& o) {
    const long long plane = (long long)d.nt * d.np;
    const double2 v = *reinterpret_cast<const double2*>(u + P.base);
    const long long row = P.base - P.k0;
    const int km = (P.k0 == 0) ? d.np - 1 : P.k0 - 1;
    const int kp = (P.k0 + 2 == d.np) ? 0 : P.k0 + 2;
    o.x = fma(cp, u[row + km] + v.y, ca * v.x);
    o.y = fma(cp, v.x + u[row + kp], ca * v.y);
    if (P.i > 0) {
        const double2 n = *reinterpret_cast<const double2*>(u + P.base - plane);
        o.x = fma(crl, n.x, o.x);
        o.y = fma(crl, n.y, o.y);
    }
    if (P.i < d.nr - 1) {
        const double2 n = *reinterpret_cast<const double2*>(u + P.base + plane);
        o.x = fma(crh, n.x, o.x);
        o.y = fma(crh, n.y, o.y);
    }
    if (P.j > 0) {
        const double2 n = *reinterpret_cast<const double2*>(u + P.base - d.np);
        o.x = fma(ctl, n.x, o.x);
        o.y = fma(ctl, n.y, o.y);
    }
    if (P.j < d.nt - 1) {
        const double2 n = *reinterpret_cast<const double2*>(u + P.base + d.np);
        o.x = fma(cth, n.x, o.x);
        o.y = fma(cth, n.y, o.y);
    }
}

// ly0 = dt L(Y_0) = -T K-stencil of Y_0; D_1 = c1 ly0
__global__ void __launch_bounds__(kThreads) k_sts_first(Dims d, const double* __restrict__ T, double c1,
                                                        const double* __restrict__ y0, double* __restrict__ ly0,
                                                        double* __restrict__ d1) {
    const unsigned int G2 = (unsigned int)(d.N / 2);
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G2; g += gridDim.x * blockDim.x) {
        const Pair P = pair_of(d, g);
        const double* t = T + (size_t)P.ij * kTab;
        const double ca = -t[0], cp = t[1], crl = t[2], crh = t[3], ctl = t[4], cth = t[5];
#pragma unroll 1
        for (int c = 0; c < 3; c++) {
            double2 l;
            stencil2(d, P, y0 + c * d.N, ca, cp, crl, crh, ctl, cth, l);
            const long long o = c * d.N + P.base;
            *reinterpret_cast<double2*>(ly0 + o) = l;
            *reinterpret_cast<double2*>(d1 + o) = make_double2(c1 * l.x, c1 * l.y);
        }
    }
}

// D_j = mu D_{j-1} + nv D_{j-2} + mut dt L(D_{j-1}) + cl ly0; the last stage writes Y_0 + D_s
// into y (which holds Y_0)
template <bool HAS_B, bool LAST>
__global__ void __launch_bounds__(kThreads) k_sts_stage(Dims d, const double* __restrict__ T, double mu, double nv,
                                                        double mut, double cl, const double* __restrict__ ly0,
                                                        const double* __restrict__ da, const double* __restrict__ db,
                                                        double* __restrict__ out) {
    const unsigned int G2 = (unsigned int)(d.N / 2);
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G2; g += gridDim.x * blockDim.x) {
        const Pair P = pair_of(d, g);
        const double* t = T + (size_t)P.ij * kTab;
        const double ca = fma(-mut, t[0], mu), cp = mut * t[1], crl = mut * t[2], crh = mut * t[3],
                     ctl = mut * t[4], cth = mut * t[5];
#pragma unroll 1
        for (int c = 0; c < 3; c++) {
            double2 r;
            stencil2(d, P, da + c * d.N, ca, cp, crl, crh, ctl, cth, r);
            const long long o = c * d.N + P.base;
            const double2 l = *reinterpret_cast<const double2*>(ly0 + o);
            r.x = fma(cl, l.x, r.x);
            r.y = fma(cl, l.y, r.y);
            if (HAS_B) {
                const double2 b = *reinterpret_cast<const double2*>(db + o);
                r.x = fma(nv, b.x, r.x);
                r.y = fma(nv, b.y, r.y);
            }
            if (LAST) {
                const double2 y = *reinterpret_cast<const double2*>(out + o);
                r.x += y.x;
                r.y += y.y;
            }
            *reinterpret_cast<double2*>(out + o) = r;
        }
    }
}

double rkl2_b(int j) { return (j < 2) ? 1.0 / 3.0 : (double)(j * j + j - 2) / (2.0 * j * (j + 1)); }

template <bool HAS_B, bool LAST>
void launch_stage(mhd_grid_s* g, int blocks, double mu, double nv, double mut, double cl, const double* ly0,
                  const double* da, const double* db, double* out) {
    k_sts_stage<HAS_B, LAST><<<blocks, kThreads, 0, g->stream>>>(g->d, g->sts_tab, mu, nv, mut, cl, ly0, da, db, out);
}

}  // namespace

int sts_stages(const mhd_grid_s* g, double nu, double dt) {
    const double lam = nu * g->visc_lambda_unit;
    int s = 2;
    while ((double)(s * s + s - 2) / 2.0 < dt * lam) s++;
    return s;
}

// y (stacked 3N, in place) advanced over dt (device scalar; dt_host is its value, which sets the
// stage count). Workspace: ly0 in the FP64 CG vector q, the differences rotate through x, r, p.
int sts_advance(mhd_grid_s* g, double nu, const double* dt_dev, double dt_host, double* y) {
    const int s = sts_stages(g, nu, dt_host);
    const double w1 = 4.0 / (double)(s * s + s - 2);
    const int blocks = grid_blocks(g, g->d.N / 2, 5);
    double* ly0 = g->q64;
    double* const ring[3] = {g->x64, g->r64, g->p64};
    auto dbuf = [&](int j) { return ring[j % 3]; };
    const int nij = g->d.nr * g->d.nt;
    k_sts_tab<<<(nij + kThreads - 1) / kThreads, kThreads, 0, g->stream>>>(g->d, g->geo, nu, dt_dev, g->sts_tab);
    k_sts_first<<<blocks, kThreads, 0, g->stream>>>(g->d, g->sts_tab, rkl2_b(1) * w1, y, ly0, dbuf(1));
    for (int j = 2; j <= s; j++) {
        const double bj = rkl2_b(j), bj1 = rkl2_b(j - 1), bj2 = rkl2_b(j - 2);
        const double mu = (2.0 * j - 1.0) / j * bj / bj1;
        const double nv = -(j - 1.0) / j * bj / bj2;
        const double mut = mu * w1;
        const double cl = bj1 * mut;   // mu~_j + ga~_j
        const bool last = (j == s);
        double* out = last ? y : dbuf(j);
        if (j == 2) {
            if (last) launch_stage<false, true>(g, blocks, mu, nv, mut, cl, ly0, dbuf(1), nullptr, out);
            else launch_stage<false, false>(g, blocks, mu, nv, mut, cl, ly0, dbuf(1), nullptr, out);
        } else {
            if (last) launch_stage<true, true>(g, blocks, mu, nv, mut, cl, ly0, dbuf(j - 1), dbuf(j - 2), out);
            else launch_stage<true, false>(g, blocks, mu, nv, mut, cl, ly0, dbuf(j - 1), dbuf(j - 2), out);
        }
    }
    return s;
}

}  // namespace mhd
