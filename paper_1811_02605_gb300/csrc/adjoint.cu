// Adjoint (reverse-mode derivative) of one zero-beta step with dt, alpha_SI, alpha_nu and the
// upwind directions frozen at the forward values.
//
// The forward step is recomputed from state n. The reverse sweep runs its stages backwards:
//   viscous solve:   lam_v** = D M_nu^-1 lam_v'                   (M symmetric: one PCG solve)
//   corrector solve: lam_bc = M_SI^-1 lam_dc; lam_b1 = lam_b0 = lam_bc / 2
//   F(v_p, B^{n+1}): force transpose -> lam_vp, lam_B^{n+1}
//   CT:              lam_E = -dt C^T lam_B^{n+1}; E transpose -> lam_vbar, lam_B
//   predictor solve: lam_b0 += M_SI^-1 (lam_vp + lam_vbar / 2)
//   F(v^n, B^n):     force transpose -> lam_v, lam_B
// Every transpose is written as a gather over the cells, edges or faces that the forward stencil
// touches (no atomics, deterministic). FP64 throughout.
#include <cmath>
#include <cstring>

#include "mhd_internal.cuh"

using namespace mhd;

namespace {


struct VelA {
    const double *vr, *vt, *vp, *dl;
    double f;
    long long N;
    __device__ __forceinline__ void at(long long c, double (&u)[3]) const {
        u[0] = vr[c];
        u[1] = vt[c];
        u[2] = vp[c];
        if (dl) {
            u[0] += f * dl[c];
            u[1] += f * dl[N + c];
            u[2] += f * dl[2 * N + c];
        }
    }
};

// cell-centred B; bh: first-harmonic sums of the B_theta face rings next to the poles
__device__ __forceinline__ void bcen(const Dims& d, const Geo& G, const double* bh, const double* br,
                                     const double* bt, const double* bp, int i, int j, int k, double (&o)[3]) {
    o[0] = 0.5 * (br[ix(d, i, j, k)] + br[ix(d, i + 1, j, k)]);
    if (j == 0) o[1] = polar_btc(G, d.np, bh + 2 * i, k, bt[ixt(d, i, 1, k)]);
    else if (j == d.nt - 1) o[1] = polar_btc(G, d.np, bh + 2 * (d.nr + i), k, bt[ixt(d, i, d.nt - 1, k)]);
    else o[1] = 0.5 * (bt[ixt(d, i, j, k)] + bt[ixt(d, i, j + 1, k)]);
    o[2] = 0.5 * (bp[ix(d, i, j, k)] + bp[ix(d, i, j, kp1(d, k))]);
}

__device__ __forceinline__ void jcen(const Dims& d, const double* jr, const double* jt, const double* jp, int i,
                                     int j, int k, double (&o)[3]) {
    const int kp = kp1(d, k);
    o[0] = 0.25 * (jr[ixt(d, i, j, k)] + jr[ixt(d, i, j, kp)] + jr[ixt(d, i, j + 1, k)] + jr[ixt(d, i, j + 1, kp)]);
    o[1] = 0.25 * (jt[ix(d, i, j, k)] + jt[ix(d, i, j, kp)] + jt[ix(d, i + 1, j, k)] + jt[ix(d, i + 1, j, kp)]);
    if (j == 0) o[2] = 0.5 * (jp[ixt(d, i, 1, k)] + jp[ixt(d, i + 1, 1, k)]);
    else if (j == d.nt - 1) o[2] = 0.5 * (jp[ixt(d, i, d.nt - 1, k)] + jp[ixt(d, i + 1, d.nt - 1, k)]);
    else
        o[2] = 0.25 * (jp[ixt(d, i, j, k)] + jp[ixt(d, i, j + 1, k)] + jp[ixt(d, i + 1, j, k)] +
                       jp[ixt(d, i + 1, j + 1, k)]);
}

// forward upwind difference of component u at cell (i,j,k) along direction dir with the frozen
// direction chosen by the sign of the cell's own velocity component vd
__device__ double upwind(const Dims& d, const Geo& G, const VelA& v, int m, int dir, double vd, int i, int j, int k,
                         long long c) {
    double uc[3], n[3];
    v.at(c, uc);
    if (dir == 0) {
        if (vd > 0.0) {
            if (i > 0) {
                v.at(c - (long long)d.nt * d.np, n);
                return (uc[m] - n[m]) / (G.rc[i] - G.rc[i - 1]);
            }
            return (uc[m] - (-uc[m])) / (2.0 * (G.rc[0] - G.r0));
        }
        if (i < d.nr - 1) {
            v.at(c + (long long)d.nt * d.np, n);
            return (n[m] - uc[m]) / (G.rc[i + 1] - G.rc[i]);
        }
        return 0.0;
    } else if (dir == 1) {
        const double h = G.rc[i] * G.dth;
        if (vd > 0.0) {
            if (j > 0) {
                v.at(c - d.np, n);
                return (uc[m] - n[m]) / h;
            }
            return 0.0;
        }
        if (j < d.nt - 1) {
            v.at(c + d.np, n);
            return (n[m] - uc[m]) / h;
        }
        return 0.0;
    }
    const double h = G.rc[i] * G.sc[j] * G.dph;
    if (vd > 0.0) {
        v.at(c - k + km1(d, k), n);
        return (uc[m] - n[m]) / h;
    }
    v.at(c - k + kp1(d, k), n);
    return (n[m] - uc[m]) / h;
}

// first-harmonic sums of the theta component of lam_Bc over the two polar rings, into the second
// half of g->bharm (read by k_face_T)
void lbc_harmonics(mhd_grid_s* g, const double* lbc, cudaStream_t st) {
    const Dims d = g->d;
    ring_harmonics(g, lbc + d.N, (long long)d.nt * d.np, 0, (long long)(d.nt - 1) * d.np, g->bharm + 4 * d.nr, st);
}

// ---------------------------------------------------------------------------------------------
// force transpose, cell part: lam_v += (dF/dv)^T (s lam_b); lam_Bc = (s lam_b x J)/rho,
// lam_Jc = (B x s lam_b)/rho (cell arrays, overwritten)
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_adjF_cell(Dims d, Geo G, VelA v, const double* __restrict__ bh,
                                                        const double* __restrict__ br,
                                                        const double* __restrict__ bt, const double* __restrict__ bp,
                                                        const double* __restrict__ jr, const double* __restrict__ jt,
                                                        const double* __restrict__ jp, double dt,
                                                        const double* __restrict__ lb, double* __restrict__ lv,
                                                        double* __restrict__ lbc, double* __restrict__ ljc) {
    const long long N = d.N;
    const long long plane = (long long)d.nt * d.np;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        int k;
        unsigned int ij;
        split_np(d, c, k, ij);
        const int j = (int)(ij % d.nt), i = (int)(ij / d.nt);
        const double s = G.rhoV[ij] * dt;
        const double rho = G.rho[i];
        const double lf[3] = {s * lb[c], s * lb[N + c], s * lb[2 * N + c]};
        double B[3], J[3], u[3];
        bcen(d, G, bh, br, bt, bp, i, j, k, B);
        jcen(d, jr, jt, jp, i, j, k, J);
        v.at(c, u);
        ljc[c] = (B[1] * lf[2] - B[2] * lf[1]) / rho;
        ljc[N + c] = (B[2] * lf[0] - B[0] * lf[2]) / rho;
        ljc[2 * N + c] = (B[0] * lf[1] - B[1] * lf[0]) / rho;
        lbc[c] = (lf[1] * J[2] - lf[2] * J[1]) / rho;
        lbc[N + c] = (lf[2] * J[0] - lf[0] * J[2]) / rho;
        lbc[2 * N + c] = (lf[0] * J[1] - lf[1] * J[0]) / rho;
        const double mu[3] = {-lf[0], -lf[1], -lf[2]};
        double acc[3] = {0.0, 0.0, 0.0};
        // pointwise: lam_u_d += sum_m mu_m D_d(v_m)
        for (int dir = 0; dir < 3; dir++)
            for (int m = 0; m < 3; m++) acc[dir] += mu[m] * upwind(d, G, v, m, dir, u[dir], i, j, k, c);
        // gather of D_d^T (u_d mu_m) from this cell and its two neighbours along d
        // neighbours' weights need their own mu = -s lam_b and velocity component
        auto mu_at = [&](long long cc, long long ijc, double (&o)[3]) {
            const double sc = G.rhoV[ijc] * dt;
            o[0] = -sc * lb[cc];
            o[1] = -sc * lb[N + cc];
            o[2] = -sc * lb[2 * N + cc];
        };
        // r
        {
            const double hl = (i > 0) ? G.rc[i] - G.rc[i - 1] : 0.0;
            const double hh = (i < d.nr - 1) ? G.rc[i + 1] - G.rc[i] : 0.0;
            double cown;
            if (u[0] > 0.0) cown = (i > 0) ? 1.0 / hl : 2.0 / (2.0 * (G.rc[0] - G.r0));
            else cown = (i < d.nr - 1) ? -1.0 / hh : 0.0;
            for (int m = 0; m < 3; m++) acc[m] += cown * u[0] * mu[m];
            if (i + 1 <= d.nr - 1) {
                double un[3], mn[3];
                v.at(c + plane, un);
                if (un[0] > 0.0) {
                    mu_at(c + plane, ij + d.nt, mn);
                    for (int m = 0; m < 3; m++) acc[m] -= un[0] * mn[m] / hh;
                }
            }
            if (i - 1 >= 0) {
                double un[3], mn[3];
                v.at(c - plane, un);
                if (!(un[0] > 0.0)) {
                    mu_at(c - plane, ij - d.nt, mn);
                    for (int m = 0; m < 3; m++) acc[m] += un[0] * mn[m] / hl;
                }
            }
        }
        // theta
        {
            const double h = G.rc[i] * G.dth;
            double cown;
            if (u[1] > 0.0) cown = (j > 0) ? 1.0 / h : 0.0;
            else cown = (j < d.nt - 1) ? -1.0 / h : 0.0;
            for (int m = 0; m < 3; m++) acc[m] += cown * u[1] * mu[m];
            if (j + 1 <= d.nt - 1) {
                double un[3], mn[3];
                v.at(c + d.np, un);
                if (un[1] > 0.0) {
                    mu_at(c + d.np, ij + 1, mn);
                    for (int m = 0; m < 3; m++) acc[m] -= un[1] * mn[m] / h;
                }
            }
            if (j - 1 >= 0) {
                double un[3], mn[3];
                v.at(c - d.np, un);
                if (!(un[1] > 0.0)) {
                    mu_at(c - d.np, ij - 1, mn);
                    for (int m = 0; m < 3; m++) acc[m] += un[1] * mn[m] / h;
                }
            }
        }
        // phi
        {
            const double h = G.rc[i] * G.sc[j] * G.dph;
            const double cown = (u[2] > 0.0) ? 1.0 / h : -1.0 / h;
            for (int m = 0; m < 3; m++) acc[m] += cown * u[2] * mu[m];
            const long long cp = c - k + kp1(d, k), cm = c - k + km1(d, k);
            double un[3], mn[3];
            v.at(cp, un);
            if (un[2] > 0.0) {
                mu_at(cp, ij, mn);
                for (int m = 0; m < 3; m++) acc[m] -= un[2] * mn[m] / h;
            }
            v.at(cm, un);
            if (!(un[2] > 0.0)) {
                mu_at(cm, ij, mn);
                for (int m = 0; m < 3; m++) acc[m] += un[2] * mn[m] / h;
            }
        }
        // curvature Jacobian
        const double r = G.rc[i], cot = G.cc[j] / G.sc[j];
        acc[1] += mu[0] * (-2.0 * u[1] / r);
        acc[2] += mu[0] * (-2.0 * u[2] / r);
        acc[0] += mu[1] * (u[1] / r);
        acc[1] += mu[1] * (u[0] / r);
        acc[2] += mu[1] * (-2.0 * u[2] * cot / r);
        acc[0] += mu[2] * (u[2] / r);
        acc[1] += mu[2] * (u[2] * cot / r);
        acc[2] += mu[2] * ((u[0] + u[1] * cot) / r);
        lv[c] += acc[0];
        lv[N + c] += acc[1];
        lv[2 * N + c] += acc[2];
    }
}

// E transpose, cell part: lam_vbar += lam_Ec x Bc; lam_Bc = vbar x lam_Ec; lam_Jc = eta lam_Ec
__global__ void __launch_bounds__(kThreads) k_adjE_cell(Dims d, Geo G, VelA v, const double* __restrict__ bh,
                                                        const double* __restrict__ br,
                                                        const double* __restrict__ bt, const double* __restrict__ bp,
                                                        const double* __restrict__ lec, double eta,
                                                        double* __restrict__ lvb, double* __restrict__ lbc,
                                                        double* __restrict__ ljc) {
    const long long N = d.N;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        int k;
        unsigned int ij;
        split_np(d, c, k, ij);
        const int j = (int)(ij % d.nt), i = (int)(ij / d.nt);
        double B[3], u[3];
        bcen(d, G, bh, br, bt, bp, i, j, k, B);
        v.at(c, u);
        const double l0 = lec[c], l1 = lec[N + c], l2 = lec[2 * N + c];
        lvb[c] += l1 * B[2] - l2 * B[1];
        lvb[N + c] += l2 * B[0] - l0 * B[2];
        lvb[2 * N + c] += l0 * B[1] - l1 * B[0];
        lbc[c] = u[1] * l2 - u[2] * l1;
        lbc[N + c] = u[2] * l0 - u[0] * l2;
        lbc[2 * N + c] = u[0] * l1 - u[1] * l0;
        if (ljc) {
            ljc[c] = eta * l0;
            ljc[N + c] = eta * l1;
            ljc[2 * N + c] = eta * l2;
        }
    }
}

// polar ring sums of the radial-edge array (j = 0 and j = nt): out[i], out[nr + i]
__global__ void k_ring_edges(Dims d, const double* __restrict__ er, double* __restrict__ out) {
    const int i = blockIdx.x % d.nr;
    const int south = blockIdx.x / d.nr;
    const int j = south ? d.nt : 0;
    double s = 0.0;
    for (int k = threadIdx.x; k < d.np; k += blockDim.x) s += er[ixt(d, i, j, k)];
    __shared__ double sm[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sm[w];
        out[blockIdx.x] = t;
    }
}

// transpose of the edge -> centre averaging of J: lam_J edges (overwritten) from lam_Jc
__global__ void __launch_bounds__(kThreads) k_jcentre_T(Dims d, const double* __restrict__ ljc,
                                                        double* __restrict__ ljr, double* __restrict__ ljt,
                                                        double* __restrict__ ljp) {
    const long long N = d.N;
    const long long n_r = (long long)d.nr * (d.nt + 1) * d.np;
    const long long n_t = (long long)(d.nr + 1) * d.nt * d.np;
    const long long n_p = (long long)(d.nr + 1) * (d.nt + 1) * d.np;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_r + n_t + n_p;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < n_r) {
            int k;
            unsigned int q;
            split_np(d, e, k, q);
            const int j = (int)(q % (d.nt + 1)), i = (int)(q / (d.nt + 1));
            const int km = km1(d, k);
            double s = 0.0;
            if (j - 1 >= 0) s += ljc[ix(d, i, j - 1, km)] + ljc[ix(d, i, j - 1, k)];
            if (j <= d.nt - 1) s += ljc[ix(d, i, j, km)] + ljc[ix(d, i, j, k)];
            ljr[e] = 0.25 * s;
        } else if (e < n_r + n_t) {
            const long long f = e - n_r;
            int k;
            unsigned int q;
            split_np(d, f, k, q);
            const int j = (int)(q % d.nt), i = (int)(q / d.nt);
            const int km = km1(d, k);
            double s = 0.0;
            if (i - 1 >= 0) s += ljc[N + ix(d, i - 1, j, km)] + ljc[N + ix(d, i - 1, j, k)];
            if (i <= d.nr - 1) s += ljc[N + ix(d, i, j, km)] + ljc[N + ix(d, i, j, k)];
            ljt[f] = 0.25 * s;
        } else {
            const long long f = e - n_r - n_t;
            int k;
            unsigned int q;
            split_np(d, f, k, q);
            const int j = (int)(q % (d.nt + 1)), i = (int)(q / (d.nt + 1));
            double s = 0.0;
            if (j >= 1 && j <= d.nt - 1) {
                for (int ic = i - 1; ic <= i; ic++) {
                    if (ic < 0 || ic > d.nr - 1) continue;
                    for (int jc = j - 1; jc <= j; jc++) {
                        if (jc < 0 || jc > d.nt - 1) continue;
                        double w;
                        if (jc == 0) w = (j == 1) ? 0.5 : 0.0;
                        else if (jc == d.nt - 1) w = (j == d.nt - 1) ? 0.5 : 0.0;
                        else w = 0.25;
                        s += w * ljc[2 * N + ix(d, ic, jc, k)];
                    }
                }
            }
            ljp[f] = s;
        }
    }
}

// lam_B faces += P_B^T lam_Bc + (curl_J)^T lam_J (edges). The polar-ring pole value of B_theta,c is
// a symmetric map of the face ring (matrix 2 / (np cos(dth)) cos(phi_k - phi_m)), so its transpose
// evaluates the same first harmonic of the lam_Bc_theta polar ring (lh: its cos and sin sums).
__global__ void __launch_bounds__(kThreads) k_face_T(Dims d, Geo G, const double* __restrict__ lbc,
                                                     const double* __restrict__ lh,
                                                     const double* __restrict__ ljr, const double* __restrict__ ljt,
                                                     const double* __restrict__ ljp, const double* __restrict__ ring,
                                                     int has_j, double* __restrict__ lbr, double* __restrict__ lbt,
                                                     double* __restrict__ lbp) {
    const long long N = d.N;
    const int nr = d.nr, nt = d.nt;
    const long long n_r = (long long)(nr + 1) * nt * d.np;
    const long long n_t = (long long)nr * (nt + 1) * d.np;
    const long long n_p = (long long)nr * nt * d.np;
    const double two_pi = 6.283185307179586;
    auto rlo = [&](int ie) { return (ie > 0) ? G.rc[ie - 1] : 2.0 * G.r0 - G.rc[0]; };
    auto rhi = [&](int ie) { return (ie < nr) ? G.rc[ie] : 2.0 * G.r1 - G.rc[nr - 1]; };
    // J edge cotangents divided by their dual-face areas
    auto wjr = [&](int i, int j, int k) {
        return ljr[ixt(d, i, j, k)] / (G.rc[i] * G.rc[i] * (G.cc[j - 1] - G.cc[j]) * G.dph);
    };
    auto wjt = [&](int ie, int j, int k) {
        const double a = rlo(ie), b = rhi(ie);
        return ljt[ix(d, ie, j, k)] / (G.sc[j] * 0.5 * (b * b - a * a) * G.dph);
    };
    auto wjp = [&](int ie, int j, int k) {
        const double a = rlo(ie), b = rhi(ie);
        return ljp[ixt(d, ie, j, k)] / (0.5 * (b * b - a * a) * G.dth);
    };
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_r + n_t + n_p;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < n_r) {
            int k;
            unsigned int q;
            split_np(d, e, k, q);
            const int j = (int)(q % nt), i = (int)(q / nt);
            double s = 0.0;
            if (i >= 1) s += 0.5 * lbc[ix(d, i - 1, j, k)];
            if (i <= nr - 1) s += 0.5 * lbc[ix(d, i, j, k)];
            if (has_j) {
                const double dR = rhi(i) - rlo(i);
                s += dR * (wjt(i, j, k) - wjt(i, j, kp1(d, k)));
                if (j + 1 <= nt - 1) s += dR * wjp(i, j + 1, k);
                if (j >= 1) s -= dR * wjp(i, j, k);
            }
            lbr[e] += s;
        } else if (e < n_r + n_t) {
            const long long f = e - n_r;
            int k;
            unsigned int q;
            split_np(d, f, k, q);
            const int j = (int)(q % (nt + 1)), i = (int)(q / (nt + 1));
            double s = 0.0;
            for (int jc = j - 1; jc <= j; jc++) {
                if (jc < 0 || jc > nt - 1) continue;
                double w;
                if (jc == 0) w = (j == 1) ? 0.5 : 0.0;
                else if (jc == nt - 1) w = (j == nt - 1) ? 0.5 : 0.0;
                else w = 0.5;
                s += w * lbc[N + ix(d, i, jc, k)];
            }
            if (j == 1) s += 0.5 * G.pole_f * (lh[2 * i] * G.pcs[k] + lh[2 * i + 1] * G.pcs[d.np + k]);
            if (j == nt - 1)
                s += 0.5 * G.pole_f * (lh[2 * (nr + i)] * G.pcs[k] + lh[2 * (nr + i) + 1] * G.pcs[d.np + k]);
            if (has_j && j >= 1 && j <= nt - 1) {
                const double rcd = G.rc[i] * G.dth;
                s += rcd * (wjr(i, j, kp1(d, k)) - wjr(i, j, k));
                s += rhi(i) * G.dth * wjp(i, j, k);
                if (i == nr - 1) s += rhi(nr) * G.dth * wjp(nr, j, k);
                s -= rlo(i + 1) * G.dth * wjp(i + 1, j, k);
                if (i == 0) s -= rlo(0) * G.dth * wjp(0, j, k);
            }
            lbt[f] += s;
        } else {
            const long long f = e - n_r - n_t;
            int k;
            unsigned int q;
            split_np(d, f, k, q);
            const int j = (int)(q % nt), i = (int)(q / nt);
            double s = 0.5 * (lbc[2 * N + ix(d, i, j, k)] + lbc[2 * N + ix(d, i, j, km1(d, k))]);
            if (has_j) {
                const double rc = G.rc[i];
                if (j >= 1) s += rc * G.sc[j] * G.dph * wjr(i, j, k);
                if (j + 1 <= nt - 1) s -= rc * G.sc[j] * G.dph * wjr(i, j + 1, k);
                if (j == 0) s += rc * G.sc[0] * G.dph / (rc * rc * (1.0 - G.cc[0]) * two_pi) * ring[i];
                if (j == nt - 1) s -= rc * G.sc[nt - 1] * G.dph / (rc * rc * (1.0 + G.cc[nt - 1]) * two_pi) * ring[nr + i];
                const double sd = G.sc[j] * G.dph;
                s += rlo(i + 1) * sd * wjt(i + 1, j, k);
                if (i == 0) s += rlo(0) * sd * wjt(0, j, k);
                s -= rhi(i) * sd * wjt(i, j, k);
                if (i == nr - 1) s -= rhi(nr) * sd * wjt(nr, j, k);
            }
            lbp[f] += s;
        }
    }
}

// lam_E (edges, overwritten) = -dt C^T lam_B (faces)
__global__ void __launch_bounds__(kThreads) k_ct_T(Dims d, Geo G, double dt, const double* __restrict__ lbr,
                                                   const double* __restrict__ lbt, const double* __restrict__ lbp,
                                                   double* __restrict__ ler, double* __restrict__ let,
                                                   double* __restrict__ lep) {
    const int nr = d.nr, nt = d.nt;
    const long long n_r = (long long)nr * (nt + 1) * d.np;
    const long long n_t = (long long)(nr + 1) * nt * d.np;
    const long long n_p = (long long)(nr + 1) * (nt + 1) * d.np;
    // scaled face cotangents w = -dt lam_B / A
    auto wbr = [&](int i, int j, int k) {
        const double ri = G.r[i];
        return -dt * lbr[ix(d, i, j, k)] / (ri * ri * (G.cn[j] - G.cn[j + 1]) * G.dph);
    };
    auto wbt = [&](int i, int j, int k) {
        const double ri = G.r[i], ro = G.r[i + 1];
        return -dt * lbt[ixt(d, i, j, k)] / (G.sn[j] * 0.5 * (ro * ro - ri * ri) * G.dph);
    };
    auto wbp = [&](int i, int j, int k) {
        const double ri = G.r[i], ro = G.r[i + 1];
        return -dt * lbp[ix(d, i, j, k)] / (0.5 * (ro * ro - ri * ri) * G.dth);
    };
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_r + n_t + n_p;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < n_r) {
            int k;
            unsigned int q;
            split_np(d, e, k, q);
            const int j = (int)(q % (nt + 1)), i = (int)(q / (nt + 1));
            const double lr = G.r[i + 1] - G.r[i];
            double s = 0.0;
            if (j >= 1 && j <= nt - 1) s += lr * (wbt(i, j, km1(d, k)) - wbt(i, j, k));
            if (j <= nt - 1) s += lr * wbp(i, j, k);
            if (j >= 1) s -= lr * wbp(i, j - 1, k);
            ler[e] = s;
        } else if (e < n_r + n_t) {
            const long long f = e - n_r;
            int k;
            unsigned int q;
            split_np(d, f, k, q);
            const int j = (int)(q % nt), i = (int)(q / nt);
            const double lt = G.r[i] * G.dth;
            double s = lt * (wbr(i, j, k) - wbr(i, j, km1(d, k)));
            if (i >= 1) s += lt * wbp(i - 1, j, k);
            if (i <= nr - 1) s -= lt * wbp(i, j, k);
            let[f] = s;
        } else {
            const long long f = e - n_r - n_t;
            int k;
            unsigned int q;
            split_np(d, f, k, q);
            const int j = (int)(q % (nt + 1)), i = (int)(q / (nt + 1));
            const double lp = G.r[i] * G.sn[j] * G.dph;
            double s = 0.0;
            if (j >= 1) s += lp * wbr(i, j - 1, k);
            if (j <= nt - 1) s -= lp * wbr(i, j, k);
            if (j >= 1 && j <= nt - 1) {
                if (i <= nr - 1) s += lp * wbt(i, j, k);
                if (i >= 1) s -= lp * wbt(i - 1, j, k);
            }
            lep[f] = s;
        }
    }
}

// transpose of the centre -> edge averaging of E: lam_Ec (cells, overwritten) from lam_E edges
__global__ void __launch_bounds__(kThreads) k_eedges_T(Dims d, const double* __restrict__ ler,
                                                       const double* __restrict__ let, const double* __restrict__ lep,
                                                       const double* __restrict__ ring, double* __restrict__ lec) {
    const long long N = d.N;
    const int nr = d.nr, nt = d.nt;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        int k;
        unsigned int ij;
        split_np(d, c, k, ij);
        const int j = (int)(ij % nt), i = (int)(ij / nt);
        const int kp = kp1(d, k);
        double sr = 0.0;
        for (int je = j; je <= j + 1; je++)
            if (je >= 1 && je <= nt - 1) sr += 0.25 * (ler[ixt(d, i, je, k)] + ler[ixt(d, i, je, kp)]);
        if (j == 0) sr += ring[i] / d.np;
        if (j == nt - 1) sr += ring[nr + i] / d.np;
        double st = 0.0;
        if (i >= 1) st += 0.25 * (let[ix(d, i, j, k)] + let[ix(d, i, j, kp)]);
        st += ((i + 1 == nr) ? 0.5 : 0.25) * (let[ix(d, i + 1, j, k)] + let[ix(d, i + 1, j, kp)]);
        double sp = 0.0;
        for (int ie = i; ie <= i + 1; ie++) {
            if (ie == 0) continue;
            const double w = (ie == nr) ? 0.5 : 0.25;
            for (int je = j; je <= j + 1; je++)
                if (je >= 1 && je <= nt - 1) sp += w * lep[ixt(d, ie, je, k)];
        }
        lec[c] = sr;
        lec[N + c] = st;
        lec[2 * N + c] = sp;
    }
}

// small vector kernels
__global__ void k_axpby(long long n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* __restrict__ z) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        z[q] = a * x[q] + (y ? b * y[q] : 0.0);
}
// lv = D y (accumulate), y = D y  (D = rho V per cell, three stacked components)
__global__ void k_scale_rhov(Dims d, Geo G, double* __restrict__ y, double* __restrict__ lv) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 3 * d.N;
         q += (long long)gridDim.x * blockDim.x) {
        const double w = G.rhoV[(q % d.N) / d.np] * y[q];
        y[q] = w;
        lv[q] += w;
    }
}

__global__ void k_unscale_rhov(Dims d, Geo G, const double* __restrict__ x, double* __restrict__ y) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 3 * d.N;
         q += (long long)gridDim.x * blockDim.x)
        y[q] = x[q] / G.rhoV[(q % d.N) / d.np];
}

struct AdjWork {
    double *b1r, *b1t, *b1p;          // B^{n+1}
    double *lb1r, *lb1t, *lb1p;       // cotangent of B^{n+1}
    double *y, *lb, *ldp, *lvp, *lvb; // 3N each
    double *lbc, *ljc;                // cell cotangents of Bc and Jc (3N each)
    double *lv;                       // stacked cotangent of v (3N)
};

}  // namespace

namespace mhd {
void adjoint_free(mhd_grid_s* g) {
    if (g->adj_mem) {
        cudaFree(g->adj_mem);
        g->adj_mem = nullptr;
    }
}
}  // namespace mhd

namespace mhd {
// the adjoint's workspace: B^{n+1} and its cotangent (faces), and 8 stacked cell vectors
mhd_status_t adjoint_reserve(mhd_grid_s* g) {
    if (g->adj_mem) return MHD_OK;
    const Dims d = g->d;
    const long long nbr = (long long)(d.nr + 1) * d.nt * d.np, nbt = (long long)d.nr * (d.nt + 1) * d.np;
    const long long total = 2 * (nbr + nbt + d.N) + 8 * 3 * d.N + 64;
    if (cudaMalloc(&g->adj_mem, sizeof(double) * total) != cudaSuccess) {
        cudaGetLastError();
        g->adj_mem = nullptr;
        return set_error(g, MHD_ERR_OOM, "mhd_adjoint_step: workspace allocation failed");
    }
    return MHD_OK;
}
}  // namespace mhd

extern "C" mhd_status_t mhd_adjoint_step(mhd_grid_t g, const mhd_params_t* p, const mhd_fields_t* s0, double dt,
                                         const mhd_fields_t* a1, mhd_fields_t* a0) {
    if (!g) return MHD_ERR_ARG;
    NvtxRange range("mhd_adjoint_step");
    if (g->slab_nr_global > 0) return set_error(g, MHD_ERR_ARG, "mhd_adjoint_step: not available on a slab grid");
    if (!p || !s0 || !a1 || !a0 || !(dt > 0.0)) return set_error(g, MHD_ERR_ARG, "mhd_adjoint_step: bad argument");
    if (p->precision != MHD_PREC_FP64 || !(p->tol > 0.0) || (p->viscosity_sts != 0 && p->viscosity_sts != 1) ||
        (p->pcg_variant != 0 && p->pcg_variant != 1) || (p->resistivity_implicit != 0 && p->resistivity_implicit != 1) ||
        (p->preconditioner != 0 && p->preconditioner != 1) || (p->preconditioner == 1 && p->pcg_variant != 0))
        return set_error(g, MHD_ERR_ARG, "mhd_adjoint_step: FP64 only, tol > 0, option flags 0 or 1");
    const mhd_fields_t* fl[3] = {s0, a1, a0};
    for (const mhd_fields_t* f : fl)
        if (!f->br || !f->bt || !f->bp || !f->vr || !f->vt || !f->vp)
            return set_error(g, MHD_ERR_ARG, "mhd_adjoint_step: null field pointer");
    const Dims d = g->d;
    const long long N = d.N, n3 = 3 * N;
    const long long nbr = (long long)(d.nr + 1) * d.nt * d.np, nbt = (long long)d.nr * (d.nt + 1) * d.np, nbp = N;
    // workspace, allocated on the first adjoint call of this grid (or by mhd_grid_reserve)
    mhd_status_t sa = adjoint_reserve(g);
    if (sa != MHD_OK) return sa;
    AdjWork w;
    double* m = static_cast<double*>(g->adj_mem);
    auto take = [&](long long n) {
        double* q = m;
        m += (n + 7) / 8 * 8;
        return q;
    };
    w.b1r = take(nbr); w.b1t = take(nbt); w.b1p = take(nbp);
    w.lb1r = take(nbr); w.lb1t = take(nbt); w.lb1p = take(nbp);
    w.y = take(n3); w.lb = take(n3); w.ldp = take(n3); w.lvp = take(n3); w.lvb = take(n3);
    w.lbc = take(n3); w.ljc = take(n3); w.lv = take(n3);
    cudaStream_t st = g->stream;
    const int bc = grid_blocks(g, N, 8);
    const long long ne = (long long)d.nr * (d.nt + 1) * d.np + (long long)(d.nr + 1) * d.nt * d.np +
                         (long long)(d.nr + 1) * (d.nt + 1) * d.np;
    const int be = grid_blocks(g, ne, 8);
    const long long nf = nbr + nbt + nbp;
    const int bf = grid_blocks(g, nf, 8);
    const bool res = (p->resistivity_implicit == 1);
    const double eta = res ? 0.0 : p->eta;   // resistivity in E (explicit) or in the face solve

    // coefficients with dt frozen (alpha_SI frozen too if given)
    mhd_params_t pf = *p;
    pf.dt_fixed = dt;
    mhd_status_t stt = coeffs(g, &pf, s0->vr, s0->vt, s0->vp, s0->br, s0->bt, s0->bp);
    if (stt != MHD_OK) return stt;
    cudaMemcpyAsync(g->h_ss, g->ss, sizeof(StepScalars), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return check_cuda(g, "adjoint coeffs");
    if (g->h_ss->status != MHD_OK) return set_error(g, MHD_ERR_ARG, "mhd_adjoint_step: C_f >= 1");
    const double* asi = &g->ss->alpha_si;
    const double* anu = &g->ss->alpha_nu;
    mhd_status_t worst = MHD_OK;
    auto note = [&](mhd_status_t s) {
        if (s != MHD_OK && worst == MHD_OK) worst = s;
    };
    const VelA vel0{s0->vr, s0->vt, s0->vp, nullptr, 0.0, N};
    const VelA velp{s0->vr, s0->vt, s0->vp, g->dlt, 1.0, N};
    const VelA velb{s0->vr, s0->vt, s0->vp, g->dlt, 0.5, N};

    // ---- forward recomputation: b0, d_p, B^{n+1}
    force(g, s0->vr, s0->vt, s0->vp, nullptr, 0.0, s0->br, s0->bt, s0->bp, nullptr, dt, nullptr, g->b0);
    cudaMemsetAsync(g->dlt, 0, sizeof(double) * n3, st);
    stt = solve(g, asi, 3, g->b0, g->dlt, g->dlt, p, nullptr, nullptr, nullptr);
    if (stt == MHD_ERR_CUDA) return stt;
    note(stt);
    cudaMemcpyAsync(w.b1r, s0->br, sizeof(double) * nbr, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(w.b1t, s0->bt, sizeof(double) * nbt, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(w.b1p, s0->bp, sizeof(double) * nbp, cudaMemcpyDeviceToDevice, st);
    induction(g, s0->vr, s0->vt, s0->vp, g->dlt, 0.5, eta, nullptr, dt, w.b1r, w.b1t, w.b1p);
    if (res) {
        stt = res_solve(g, &g->ss->dt, p->eta, w.b1r, w.b1t, w.b1p, p, nullptr, nullptr);
        if (stt == MHD_ERR_CUDA || stt == MHD_ERR_OOM) return stt;
        note(stt);
    }

    // ---- reverse
    // stacked copy of lam_v' and zeroed accumulators
    cudaMemcpyAsync(w.lvb, a1->vr, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(w.lvb + N, a1->vt, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(w.lvb + 2 * N, a1->vp, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(w.lv, 0, sizeof(double) * n3, st);
    cudaMemsetAsync(w.y, 0, sizeof(double) * n3, st);
    if (p->viscosity_sts) {
        // 5. v' = P v**, P the RKL2 polynomial in dt L (L = -nu D^-1 K, K symmetric), so
        // P^T = D P D^-1: y = P (D^-1 lam_v'), the D factor follows
        k_unscale_rhov<<<bc, kThreads, 0, st>>>(d, g->geo, w.lvb, w.y);
        sts_advance(g, p->nu, &g->ss->dt, dt, w.y);
    } else {
        // 5. viscous solve
        stt = solve(g, anu, 3, w.lvb, w.y, w.y, p, nullptr, nullptr, nullptr);
        if (stt == MHD_ERR_CUDA) return stt;
        note(stt);
    }
    k_scale_rhov<<<bc, kThreads, 0, st>>>(d, g->geo, w.y, w.lv);   // lv = D y, y = lam_dc
    // 4. corrector solve: lam_bc = M_SI^-1 lam_dc; lam_b = lam_bc / 2
    cudaMemsetAsync(w.lb, 0, sizeof(double) * n3, st);
    stt = solve(g, asi, 3, w.y, w.lb, w.lb, p, nullptr, nullptr, nullptr);
    if (stt == MHD_ERR_CUDA) return stt;
    note(stt);
    k_axpby<<<bc, kThreads, 0, st>>>(n3, 0.5, w.lb, 0.0, nullptr, w.lb);
    // F(v_p, B^{n+1}) transpose
    cudaMemcpyAsync(w.lb1r, a1->br, sizeof(double) * nbr, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(w.lb1t, a1->bt, sizeof(double) * nbt, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(w.lb1p, a1->bp, sizeof(double) * nbp, cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(w.lvp, 0, sizeof(double) * n3, st);
    current_edges(g, w.b1r, w.b1t, w.b1p);
    bt_harmonics(g, w.b1t, st);
    k_adjF_cell<<<bc, kThreads, 0, st>>>(d, g->geo, velp, g->bharm, w.b1r, w.b1t, w.b1p, g->er, g->et, g->ep, dt,
                                         w.lb, w.lvp, w.lbc, w.ljc);
    k_jcentre_T<<<be, kThreads, 0, st>>>(d, w.ljc, g->er, g->et, g->ep);
    k_ring_edges<<<2 * d.nr, kThreads, 0, st>>>(d, g->er, g->ring);
    lbc_harmonics(g, w.lbc, st);
    k_face_T<<<bf, kThreads, 0, st>>>(d, g->geo, w.lbc, g->bharm + 4 * d.nr, g->er, g->et, g->ep, g->ring, 1, w.lb1r,
                                      w.lb1t, w.lb1p);
    if (res) {
        // B^{n+1} = M_res^-1 W B* (the face solve): lam_B* = W M_res^-1 lam_B^{n+1}
        stt = res_transpose(g, &g->ss->dt, p->eta, w.lb1r, w.lb1t, w.lb1p, p);
        if (stt == MHD_ERR_CUDA || stt == MHD_ERR_OOM) return stt;
        note(stt);
    }
    // 3. B* = B - dt curl E(vbar, B) (B^{n+1} itself without a face solve): lam_B = lam_B*
    // (copy into the output), lam_E
    cudaMemcpyAsync(a0->br, w.lb1r, sizeof(double) * nbr, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(a0->bt, w.lb1t, sizeof(double) * nbt, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(a0->bp, w.lb1p, sizeof(double) * nbp, cudaMemcpyDeviceToDevice, st);
    k_ct_T<<<be, kThreads, 0, st>>>(d, g->geo, dt, w.lb1r, w.lb1t, w.lb1p, g->er, g->et, g->ep);
    k_ring_edges<<<2 * d.nr, kThreads, 0, st>>>(d, g->er, g->ring);
    k_eedges_T<<<bc, kThreads, 0, st>>>(d, g->er, g->et, g->ep, g->ring, g->ec);
    cudaMemsetAsync(w.lvb, 0, sizeof(double) * n3, st);
    bt_harmonics(g, s0->bt, st);
    k_adjE_cell<<<bc, kThreads, 0, st>>>(d, g->geo, velb, g->bharm, s0->br, s0->bt, s0->bp, g->ec, eta, w.lvb, w.lbc,
                                         eta != 0.0 ? w.ljc : nullptr);
    if (eta != 0.0) {
        k_jcentre_T<<<be, kThreads, 0, st>>>(d, w.ljc, g->er, g->et, g->ep);
        k_ring_edges<<<2 * d.nr, kThreads, 0, st>>>(d, g->er, g->ring);
    }
    lbc_harmonics(g, w.lbc, st);
    k_face_T<<<bf, kThreads, 0, st>>>(d, g->geo, w.lbc, g->bharm + 4 * d.nr, g->er, g->et, g->ep, g->ring,
                                      eta != 0.0 ? 1 : 0, a0->br, a0->bt, a0->bp);
    // v_p = v + d_p, vbar = v + d_p / 2
    k_axpby<<<bc, kThreads, 0, st>>>(n3, 1.0, w.lvp, 1.0, w.lvb, w.ldp);   // ldp = lvp + lvb (temp)
    k_axpby<<<bc, kThreads, 0, st>>>(n3, 1.0, w.lv, 1.0, w.ldp, w.lv);     // lv += lvp + lvb
    k_axpby<<<bc, kThreads, 0, st>>>(n3, 1.0, w.lvp, 0.5, w.lvb, w.ldp);   // ldp = lvp + lvb/2
    // 2. predictor solve: lam_b += M_SI^-1 lam_dp
    cudaMemsetAsync(w.y, 0, sizeof(double) * n3, st);
    stt = solve(g, asi, 3, w.ldp, w.y, w.y, p, nullptr, nullptr, nullptr);
    if (stt == MHD_ERR_CUDA) return stt;
    note(stt);
    k_axpby<<<bc, kThreads, 0, st>>>(n3, 1.0, w.lb, 1.0, w.y, w.lb);
    // F(v, B) transpose
    current_edges(g, s0->br, s0->bt, s0->bp);
    bt_harmonics(g, s0->bt, st);
    k_adjF_cell<<<bc, kThreads, 0, st>>>(d, g->geo, vel0, g->bharm, s0->br, s0->bt, s0->bp, g->er, g->et, g->ep, dt,
                                         w.lb, w.lv, w.lbc, w.ljc);
    k_jcentre_T<<<be, kThreads, 0, st>>>(d, w.ljc, g->er, g->et, g->ep);
    k_ring_edges<<<2 * d.nr, kThreads, 0, st>>>(d, g->er, g->ring);
    lbc_harmonics(g, w.lbc, st);
    k_face_T<<<bf, kThreads, 0, st>>>(d, g->geo, w.lbc, g->bharm + 4 * d.nr, g->er, g->et, g->ep, g->ring, 1, a0->br,
                                      a0->bt, a0->bp);
    cudaMemcpyAsync(a0->vr, w.lv, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(a0->vt, w.lv + N, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(a0->vp, w.lv + 2 * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    if ((stt = check_cuda(g, "mhd_adjoint_step")) != MHD_OK) return stt;
    if (cudaStreamSynchronize(st) != cudaSuccess) return check_cuda(g, "mhd_adjoint_step sync");
    return worst;
}
