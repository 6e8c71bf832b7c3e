// Explicit parts of the zero-beta step (Eq. 1; Sec. 2.2 explicit predictor-corrector
// upwinding), all FP64, one thread per output element:
//   - step coefficients: dt from the flow CFL, C_w, the semi-implicit coefficient (Sec. 2.1)
//   - J = curl_h B on edges (Stokes on the dual faces around each edge)
//   - momentum force b = rho V dt (-(v.grad)v + J x B / rho)
//   - E = -v x B + eta J at cell centres, averaged to edges; B <- B - dt curl_h E (Stokes)
// Pole and boundary rules:
//   - B_theta at a cell centre in the two polar rings is the mean of the non-polar face and of
//     the pole value along the cell's meridian (first phi harmonic of the face ring next to the
//     pole, divided by cos(dth)).
//   - The polar radial edge carries one value: the cap circulation of B_phi for J, the ring
//     mean of the polar cells for E.
//   - The polar phi edges have zero length; their J is 0 and left out of the centre average.
//   - Ghost tangential B beyond r0 and r1 equals the first interior value, at mirrored radii.
//   - Advection: Dirichlet mirror ghost (-u) at r0, zero gradient at r1, no flux from the pole.
//   - Tangential E is 0 on r0 (line-tied); on r1 it is the mean of the two interior cells.
#include <cmath>

#include "mhd_internal.cuh"
#include "reduce.cuh"

namespace mhd {

namespace {


// cell-centred B: mean of opposite faces; in the polar rings B_theta is the mean of the non-polar
// face and the pole value (bh: first-harmonic sums of the B_theta face rings, bt_harmonics)
__device__ __forceinline__ void bcentre(const Dims& d, const Geo& G, const double* __restrict__ bh,
                                        const double* __restrict__ br, const double* __restrict__ bt,
                                        const double* __restrict__ bp, int i, int j, int k, double (&o)[3]) {
    o[0] = 0.5 * (br[ix(d, i, j, k)] + br[ix(d, i + 1, j, k)]);
    if (j == 0) o[1] = polar_btc(G, d.np, bh + 2 * i, k, bt[ixt(d, i, 1, k)]);
    else if (j == d.nt - 1) o[1] = polar_btc(G, d.np, bh + 2 * (d.nr + i), k, bt[ixt(d, i, d.nt - 1, k)]);
    else o[1] = 0.5 * (bt[ixt(d, i, j, k)] + bt[ixt(d, i, j + 1, k)]);
    o[2] = 0.5 * (bp[ix(d, i, j, k)] + bp[ix(d, i, j, kp1(d, k))]);
}

// velocity u = v + f * dlt (dlt may be null)
struct Vel {
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

}  // namespace

// ------------------------------------------------------------------------------------------
// step coefficients
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_coeffs(Dims d, Geo G, Vel v, const double* __restrict__ bh,
                                                     const double* __restrict__ br,
                                                     const double* __restrict__ bt,
                                                     const double* __restrict__ bp, double nu, double cfl,
                                                     double dt_fixed, double dt_max, double asi_fixed,
                                                     StepScalars* ss, double* __restrict__ partials) {
    double mkv = 0.0, mka = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.N;
         c += (long long)gridDim.x * blockDim.x) {
        int k;
        unsigned int ij;
        split_np(d, c, k, ij);
        const int j = (int)(ij % d.nt), i = (int)(ij / d.nt);
        double u[3], B[3];
        v.at(c, u);
        bcentre(d, G, bh, br, bt, bp, i, j, k, B);
        const double kt2 = G.kt2[ij];
        const double vv = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const double bb = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
        mkv = fmax(mkv, kt2 * vv);
        mka = fmax(mka, kt2 * bb / G.rho[i]);
    }
    double val[2] = {mkv, mka}, out[2];
    if (reduce_last<2, OpMax>(val, partials, &ss->count, out) && threadIdx.x == 0) {
        const double kv = sqrt(out[0]), ka = sqrt(out[1]);
        ss->max_kv2 = out[0];
        ss->max_kva2 = out[1];
        ss->max_kt2 = G.max_kt2;
        double dt = 0.0;
        int st = MHD_OK;
        if (dt_fixed > 0.0) dt = dt_fixed;
        else {
            if (kv > 0.0) dt = cfl / kv;
            else if (dt_max > 0.0) dt = dt_max;
            else st = MHD_ERR_ARG;
            if (dt_max > 0.0 && dt > dt_max) dt = dt_max;
        }
        const double cf = dt * kv, cw = dt * ka;
        if (!(cf < 1.0)) st = MHD_ERR_ARG;
        const double X = cw * cw / ((1.0 - cf) * (1.0 - cf)) - 1.0;
        double asi = (X > 0.0) ? X / G.max_kt2 : 0.0;
        if (asi_fixed >= 0.0) asi = asi_fixed;
        ss->dt = dt;
        ss->cf = cf;
        ss->cw = cw;
        ss->alpha_si = (st == MHD_OK) ? asi : 0.0;
        ss->alpha_nu = nu * dt;
        ss->status = st;
    }
}

mhd_status_t coeffs(mhd_grid_s* g, const mhd_params_t* p, const double* vr, const double* vt,
                    const double* vp, const double* br, const double* bt, const double* bp) {
    Vel v{vr, vt, vp, nullptr, 0.0, g->d.N};
    bt_harmonics(g, bt);
    const int blocks = grid_blocks(g, g->d.N, 4);
    k_coeffs<<<blocks, kThreads, 0, g->stream>>>(g->d, g->geo, v, g->bharm, br, bt, bp, p->nu, p->cfl, p->dt_fixed,
                                                 p->dt_max, p->alpha_si_fixed, g->ss, g->partials);
    return check_cuda(g, "coeffs");
}

// ------------------------------------------------------------------------------------------
// polar ring sums: out[i] (north, ring j = 0) and out[nr + i] (south, ring j = nt-1) of a
// cell-centred array (one CTA per ring, fixed-order reduction)
// ------------------------------------------------------------------------------------------
__global__ void k_ring(Dims d, const double* __restrict__ a, double* __restrict__ out) {
    const int i = blockIdx.x % d.nr;
    const int south = blockIdx.x / d.nr;
    const int j = south ? d.nt - 1 : 0;
    double s = 0.0;
    for (int k = threadIdx.x; k < d.np; k += blockDim.x) s += a[ix(d, i, j, k)];
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

// first-harmonic sums of the rows next to the poles (one CTA per row, fixed-order reduction):
// out[2 b] = sum_k a_k cos(phi_c_k), out[2 b + 1] = sum_k a_k sin(phi_c_k), b = i (north row at
// off_n + i stride_i) or nr + i (south row at off_s + i stride_i)
__global__ void k_ring_harm(Dims d, const double* __restrict__ a, long long stride_i, long long off_n,
                            long long off_s, const double* __restrict__ pcs, double* __restrict__ out) {
    const int i = blockIdx.x % d.nr;
    const int south = blockIdx.x / d.nr;
    const double* row = a + (long long)i * stride_i + (south ? off_s : off_n);
    double sc = 0.0, ss = 0.0;
    for (int k = threadIdx.x; k < d.np; k += blockDim.x) {
        sc = fma(row[k], pcs[k], sc);
        ss = fma(row[k], pcs[d.np + k], ss);
    }
    __shared__ double sm[2][kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sm[0][threadIdx.x >> 5] = sc;
        sm[1][threadIdx.x >> 5] = ss;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tc = 0.0, ts = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            tc += sm[0][w];
            ts += sm[1][w];
        }
        out[2 * blockIdx.x] = tc;
        out[2 * blockIdx.x + 1] = ts;
    }
}

void ring_harmonics(mhd_grid_s* g, const double* a, long long stride_i, long long off_n, long long off_s,
                    double* out, cudaStream_t st) {
    k_ring_harm<<<2 * g->d.nr, kThreads, 0, st ? st : g->stream>>>(g->d, a, stride_i, off_n, off_s, g->geo.pcs,
                                                                   out);
}

void bt_harmonics(mhd_grid_s* g, const double* bt, cudaStream_t st) {
    const Dims d = g->d;
    ring_harmonics(g, bt, (long long)(d.nt + 1) * d.np, d.np, (long long)(d.nt - 1) * d.np, g->bharm, st);
}

// ------------------------------------------------------------------------------------------
// current density on edges
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_jr(Dims d, const double* __restrict__ cr,
                                                 const double* __restrict__ bt, const double* __restrict__ bp,
                                                 const double* __restrict__ ring, double* __restrict__ jr) {
    const long long n = (long long)d.nr * (d.nt + 1) * d.np;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int k;
        unsigned int q;
        split_np(d, e, k, q);
        const int j = (int)(q % (d.nt + 1)), i = (int)(q / (d.nt + 1));
        const double* c = cr + 4 * (size_t)q;
        double val;
        if (j == 0) val = ring[i] * c[3];                   // north cap circulation / cap area
        else if (j == d.nt) val = -ring[d.nr + i] * c[3];   // south cap
        else val = c[0] * bp[ix(d, i, j, k)] - c[1] * bp[ix(d, i, j - 1, k)] -
                   c[2] * (bt[ixt(d, i, j, k)] - bt[ixt(d, i, j, km1(d, k))]);
        jr[e] = val;
    }
}

// walls_zero: the resistive operator's current, 0 on the tangential edges of r0 and r1
__global__ void __launch_bounds__(kThreads) k_jt(Dims d, const double* __restrict__ ct,
                                                 const double* __restrict__ br, const double* __restrict__ bp,
                                                 double* __restrict__ jt, int walls_zero) {
    const long long n = (long long)(d.nr + 1) * d.nt * d.np;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int k;
        unsigned int q;
        split_np(d, e, k, q);
        const int j = (int)(q % d.nt), i = (int)(q / d.nt);
        if (walls_zero && (i == 0 || i == d.nr)) {
            jt[e] = 0.0;
            continue;
        }
        // ghost B_phi beyond r0 / r1 = the first interior value (at the mirrored radius in the table)
        const int ilo = (i > 0) ? i - 1 : 0, ihi = (i < d.nr) ? i : d.nr - 1;
        const double* c = ct + 3 * (size_t)q;
        jt[e] = c[0] * bp[ix(d, ilo, j, k)] + c[1] * (br[ix(d, i, j, k)] - br[ix(d, i, j, km1(d, k))]) -
                c[2] * bp[ix(d, ihi, j, k)];
    }
}

__global__ void __launch_bounds__(kThreads) k_jp(Dims d, const double* __restrict__ cp,
                                                 const double* __restrict__ br, const double* __restrict__ bt,
                                                 double* __restrict__ jp, int walls_zero) {
    const long long n = (long long)(d.nr + 1) * (d.nt + 1) * d.np;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int k;
        unsigned int q;
        split_np(d, e, k, q);
        const int j = (int)(q % (d.nt + 1)), i = (int)(q / (d.nt + 1));
        if (j == 0 || j == d.nt || (walls_zero && (i == 0 || i == d.nr))) {
            jp[e] = 0.0;
            continue;
        }
        const int ilo = (i > 0) ? i - 1 : 0, ihi = (i < d.nr) ? i : d.nr - 1;
        const double* c = cp + 3 * (size_t)q;
        jp[e] = c[0] * (br[ix(d, i, j - 1, k)] - br[ix(d, i, j, k)]) + c[1] * bt[ixt(d, ihi, j, k)] -
                c[2] * bt[ixt(d, ilo, j, k)];
    }
}

void current_edges(mhd_grid_s* g, const double* br, const double* bt, const double* bp, bool walls_zero,
                   cudaStream_t st) {
    const Dims d = g->d;
    if (!st) st = g->stream;
    k_ring<<<2 * d.nr, kThreads, 0, st>>>(d, bp, g->ring);
    const long long n = (long long)(d.nr + 1) * (d.nt + 1) * d.np;
    const int blocks = grid_blocks(g, n, 8);
    k_jr<<<blocks, kThreads, 0, st>>>(d, g->ex.jr, bt, bp, g->ring, g->er);
    k_jt<<<blocks, kThreads, 0, st>>>(d, g->ex.jt, br, bp, g->et, walls_zero ? 1 : 0);
    k_jp<<<blocks, kThreads, 0, st>>>(d, g->ex.jp, br, bt, g->ep, walls_zero ? 1 : 0);
}

// J at a cell centre from the edge arrays (polar phi edges left out)
__device__ __forceinline__ void jcentre(const Dims& d, const double* __restrict__ jr, const double* __restrict__ jt,
                                        const double* __restrict__ jp, int i, int j, int k, double (&o)[3]) {
    const int kp = kp1(d, k);
    o[0] = 0.25 * (jr[ixt(d, i, j, k)] + jr[ixt(d, i, j, kp)] + jr[ixt(d, i, j + 1, k)] + jr[ixt(d, i, j + 1, kp)]);
    o[1] = 0.25 * (jt[ix(d, i, j, k)] + jt[ix(d, i, j, kp)] + jt[ix(d, i + 1, j, k)] + jt[ix(d, i + 1, j, kp)]);
    if (j == 0) o[2] = 0.5 * (jp[ixt(d, i, 1, k)] + jp[ixt(d, i + 1, 1, k)]);
    else if (j == d.nt - 1) o[2] = 0.5 * (jp[ixt(d, i, d.nt - 1, k)] + jp[ixt(d, i + 1, d.nt - 1, k)]);
    else
        o[2] = 0.25 * (jp[ixt(d, i, j, k)] + jp[ixt(d, i, j + 1, k)] + jp[ixt(d, i + 1, j, k)] +
                       jp[ixt(d, i + 1, j + 1, k)]);
}

// ------------------------------------------------------------------------------------------
// momentum force
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_force(Dims d, Geo G, ExTab X, Vel v, const double* __restrict__ bh,
                                                    const double* __restrict__ br,
                                                    const double* __restrict__ bt, const double* __restrict__ bp,
                                                    const double* __restrict__ jr, const double* __restrict__ jt,
                                                    const double* __restrict__ jp, const double* __restrict__ dt_dev,
                                                    double dt_host, const double* __restrict__ b_avg,
                                                    double* __restrict__ b) {
    const double dt = dt_dev ? *dt_dev : dt_host;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.N;
         c += (long long)gridDim.x * blockDim.x) {
        int k;
        unsigned int ij;
        split_np(d, c, k, ij);
        const int j = (int)(ij % d.nt), i = (int)(ij / d.nt);
        double u[3];
        v.at(c, u);
        // per-shell reciprocals: 1/d_lo, 1/d_hi, 1/rc, 1/rho, 1/(rc dth)
        const double* sh = X.sh + 5 * (size_t)i;
        // upwind differences of the three components along r, theta, phi
        double Dr[3], Dt[3], Dp[3];
        if (u[0] > 0.0) {
            if (i > 0) {
                double n[3];
                v.at(c - (long long)d.nt * d.np, n);
                const double ih = sh[0];
                for (int m = 0; m < 3; m++) Dr[m] = (u[m] - n[m]) * ih;
            } else {
                const double ih = sh[0];   // Dirichlet mirror ghost at distance 2 (rc_0 - r0)
                for (int m = 0; m < 3; m++) Dr[m] = (u[m] - (-u[m])) * ih;
            }
        } else {
            if (i < d.nr - 1) {
                double n[3];
                v.at(c + (long long)d.nt * d.np, n);
                const double ih = sh[1];
                for (int m = 0; m < 3; m++) Dr[m] = (n[m] - u[m]) * ih;
            } else {
                for (int m = 0; m < 3; m++) Dr[m] = 0.0;
            }
        }
        const double iht = sh[4];
        if (u[1] > 0.0) {
            if (j > 0) {
                double n[3];
                v.at(c - d.np, n);
                for (int m = 0; m < 3; m++) Dt[m] = (u[m] - n[m]) * iht;
            } else {
                for (int m = 0; m < 3; m++) Dt[m] = 0.0;
            }
        } else {
            if (j < d.nt - 1) {
                double n[3];
                v.at(c + d.np, n);
                for (int m = 0; m < 3; m++) Dt[m] = (n[m] - u[m]) * iht;
            } else {
                for (int m = 0; m < 3; m++) Dt[m] = 0.0;
            }
        }
        const double ihp = X.ihp[ij];
        {
            double n[3];
            if (u[2] > 0.0) {
                v.at(c - k + km1(d, k), n);
                for (int m = 0; m < 3; m++) Dp[m] = (u[m] - n[m]) * ihp;
            } else {
                v.at(c - k + kp1(d, k), n);
                for (int m = 0; m < 3; m++) Dp[m] = (n[m] - u[m]) * ihp;
            }
        }
        double adv[3];
        for (int m = 0; m < 3; m++) adv[m] = u[0] * Dr[m] + u[1] * Dt[m] + u[2] * Dp[m];
        const double cot = X.cot[j];
        const double irc = sh[2];
        adv[0] += -(u[1] * u[1] + u[2] * u[2]) * irc;
        adv[1] += (u[0] * u[1] - u[2] * u[2] * cot) * irc;
        adv[2] += (u[0] * u[2] + u[1] * u[2] * cot) * irc;
        double B[3], J[3];
        bcentre(d, G, bh, br, bt, bp, i, j, k, B);
        jcentre(d, jr, jt, jp, i, j, k, J);
        const double irho = sh[3];
        const double jxb0 = J[1] * B[2] - J[2] * B[1];
        const double jxb1 = J[2] * B[0] - J[0] * B[2];
        const double jxb2 = J[0] * B[1] - J[1] * B[0];
        const double s = G.rhoV[ij] * dt;
        double f0 = s * (-adv[0] + jxb0 * irho);
        double f1 = s * (-adv[1] + jxb1 * irho);
        double f2 = s * (-adv[2] + jxb2 * irho);
        if (b_avg) {
            f0 = 0.5 * (b_avg[c] + f0);
            f1 = 0.5 * (b_avg[d.N + c] + f1);
            f2 = 0.5 * (b_avg[2 * d.N + c] + f2);
        }
        b[c] = f0;
        b[d.N + c] = f1;
        b[2 * d.N + c] = f2;
    }
}

void force(mhd_grid_s* g, const double* vr, const double* vt, const double* vp, const double* dlt, double dfac,
           const double* br, const double* bt, const double* bp, const double* dt_dev, double dt_host,
           const double* b_avg, double* b) {
    current_edges(g, br, bt, bp);
    bt_harmonics(g, bt);
    Vel v{vr, vt, vp, dlt, dfac, g->d.N};
    const int blocks = grid_blocks(g, g->d.N, 8);
    k_force<<<blocks, kThreads, 0, g->stream>>>(g->d, g->geo, g->ex, v, g->bharm, br, bt, bp, g->er, g->et, g->ep,
                                                dt_dev, dt_host, b_avg, b);
}

// ------------------------------------------------------------------------------------------
// electric field and constrained transport
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_ecentre(Dims d, Geo G, Vel v, const double* __restrict__ bh,
                                                      const double* __restrict__ br,
                                                      const double* __restrict__ bt, const double* __restrict__ bp,
                                                      const double* __restrict__ jr, const double* __restrict__ jt,
                                                      const double* __restrict__ jp, double eta,
                                                      double* __restrict__ ec) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.N;
         c += (long long)gridDim.x * blockDim.x) {
        int k;
        unsigned int ij;
        split_np(d, c, k, ij);
        const int j = (int)(ij % d.nt), i = (int)(ij / d.nt);
        double u[3], B[3];
        v.at(c, u);
        bcentre(d, G, bh, br, bt, bp, i, j, k, B);
        double e0 = -(u[1] * B[2] - u[2] * B[1]);
        double e1 = -(u[2] * B[0] - u[0] * B[2]);
        double e2 = -(u[0] * B[1] - u[1] * B[0]);
        if (eta != 0.0) {
            double J[3];
            jcentre(d, jr, jt, jp, i, j, k, J);
            e0 += eta * J[0];
            e1 += eta * J[1];
            e2 += eta * J[2];
        }
        ec[c] = e0;
        ec[d.N + c] = e1;
        ec[2 * d.N + c] = e2;
    }
}

__global__ void __launch_bounds__(kThreads) k_eedges(Dims d, const double* __restrict__ ec,
                                                     const double* __restrict__ ring, double* __restrict__ er,
                                                     double* __restrict__ et, double* __restrict__ ep) {
    const double* Er = ec;
    const double* Et = ec + d.N;
    const double* Ep = ec + 2 * d.N;
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
            double val;
            if (j == 0) val = ring[i] / d.np;
            else if (j == d.nt) val = ring[d.nr + i] / d.np;
            else {
                const int km = km1(d, k);
                val = 0.25 * (Er[ix(d, i, j - 1, km)] + Er[ix(d, i, j - 1, k)] + Er[ix(d, i, j, km)] + Er[ix(d, i, j, k)]);
            }
            er[e] = val;
        } else if (e < n_r + n_t) {
            const long long f = e - n_r;
            int k;
            unsigned int q;
            split_np(d, f, k, q);
            const int j = (int)(q % d.nt), i = (int)(q / d.nt);
            const int km = km1(d, k);
            double val;
            if (i == 0) val = 0.0;
            else if (i == d.nr) val = 0.5 * (Et[ix(d, d.nr - 1, j, km)] + Et[ix(d, d.nr - 1, j, k)]);
            else
                val = 0.25 * (Et[ix(d, i - 1, j, km)] + Et[ix(d, i - 1, j, k)] + Et[ix(d, i, j, km)] + Et[ix(d, i, j, k)]);
            et[f] = val;
        } else {
            const long long f = e - n_r - n_t;
            int k;
            unsigned int q;
            split_np(d, f, k, q);
            const int j = (int)(q % (d.nt + 1)), i = (int)(q / (d.nt + 1));
            double val;
            if (j == 0 || j == d.nt || i == 0) val = 0.0;
            else if (i == d.nr) val = 0.5 * (Ep[ix(d, d.nr - 1, j - 1, k)] + Ep[ix(d, d.nr - 1, j, k)]);
            else
                val = 0.25 * (Ep[ix(d, i - 1, j - 1, k)] + Ep[ix(d, i - 1, j, k)] + Ep[ix(d, i, j - 1, k)] +
                              Ep[ix(d, i, j, k)]);
            ep[f] = val;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_ct(Dims d, ExTab X, const double* __restrict__ er,
                                                 const double* __restrict__ et, const double* __restrict__ ep,
                                                 const double* __restrict__ dt_dev, double dt_host,
                                                 double* __restrict__ br, double* __restrict__ bt,
                                                 double* __restrict__ bp) {
    const double dt = dt_dev ? *dt_dev : dt_host;
    const long long n_r = (long long)(d.nr + 1) * d.nt * d.np;
    const long long n_t = (long long)d.nr * (d.nt + 1) * d.np;
    const long long n_p = (long long)d.nr * d.nt * d.np;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_r + n_t + n_p;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < n_r) {
            int k;
            unsigned int q;
            split_np(d, e, k, q);
            const int j = (int)(q % d.nt), i = (int)(q / d.nt);
            const double* c = X.fr + 3 * (size_t)q;
            const double circ = c[0] * (et[ix(d, i, j, k)] - et[ix(d, i, j, kp1(d, k))]) +
                                c[1] * ep[ixt(d, i, j + 1, k)] - c[2] * ep[ixt(d, i, j, k)];
            br[e] -= dt * circ;
        } else if (e < n_r + n_t) {
            const long long f = e - n_r;
            int k;
            unsigned int q;
            split_np(d, f, k, q);
            const int j = (int)(q % (d.nt + 1)), i = (int)(q / (d.nt + 1));
            if (j == 0 || j == d.nt) continue;
            const double* c = X.ft + 3 * (size_t)q;
            const double circ = c[0] * ep[ixt(d, i, j, k)] + c[1] * (er[ixt(d, i, j, kp1(d, k))] - er[ixt(d, i, j, k)]) -
                                c[2] * ep[ixt(d, i + 1, j, k)];
            bt[f] -= dt * circ;
        } else {
            const long long f = e - n_r - n_t;
            int k;
            unsigned int q;
            split_np(d, f, k, q);
            const int j = (int)(q % d.nt), i = (int)(q / d.nt);
            const double* c = X.fp + 3 * (size_t)q;
            const double circ = c[0] * (er[ixt(d, i, j, k)] - er[ixt(d, i, j + 1, k)]) + c[1] * et[ix(d, i + 1, j, k)] -
                                c[2] * et[ix(d, i, j, k)];
            bp[f] -= dt * circ;
        }
    }
}

void induction(mhd_grid_s* g, const double* vr, const double* vt, const double* vp, const double* dlt, double dfac,
               double eta, const double* dt_dev, double dt_host, double* br, double* bt, double* bp) {
    const Dims d = g->d;
    if (eta != 0.0) current_edges(g, br, bt, bp);
    Vel v{vr, vt, vp, dlt, dfac, d.N};
    bt_harmonics(g, bt);
    k_ecentre<<<grid_blocks(g, d.N, 8), kThreads, 0, g->stream>>>(d, g->geo, v, g->bharm, br, bt, bp, g->er, g->et,
                                                                 g->ep, eta, g->ec);
    k_ring<<<2 * d.nr, kThreads, 0, g->stream>>>(d, g->ec, g->ring);
    const long long ne = (long long)d.nr * (d.nt + 1) * d.np + (long long)(d.nr + 1) * d.nt * d.np +
                         (long long)(d.nr + 1) * (d.nt + 1) * d.np;
    k_eedges<<<grid_blocks(g, ne, 8), kThreads, 0, g->stream>>>(d, g->ec, g->ring, g->er, g->et, g->ep);
    k_ct<<<grid_blocks(g, ne, 8), kThreads, 0, g->stream>>>(d, g->ex, g->er, g->et, g->ep, dt_dev, dt_host, br, bt,
                                                           bp);
}

void ring_sums(mhd_grid_s* g, const double* a, cudaStream_t st) {
    k_ring<<<2 * g->d.nr, kThreads, 0, st ? st : g->stream>>>(g->d, a, g->ring);
}

void ct_apply(mhd_grid_s* g, const double* dt_dev, double* br, double* bt, double* bp) {
    const Dims d = g->d;
    const long long ne = (long long)d.nr * (d.nt + 1) * d.np + (long long)(d.nr + 1) * d.nt * d.np +
                         (long long)(d.nr + 1) * (d.nt + 1) * d.np;
    k_ct<<<grid_blocks(g, ne, 8), kThreads, 0, g->stream>>>(d, g->ex, g->er, g->et, g->ep, dt_dev, 0.0, br, bt, bp);
}

// ------------------------------------------------------------------------------------------
// field diagnostics (Sec. 3.1 validates runs by integrated energies and by |J x B| and |J . B|):
// out[0..3] = magnetic energy, kinetic energy, sum |J_c x B_c| V_c, sum |J_c . B_c| V_c; out[4] =
// max |div_h B| (net outward flux over the cell volume). B_c and J_c as in the momentum force.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double cell_volume(const Geo& G, int i, int j) {
    const double ri = G.r[i], ro = G.r[i + 1];
    return (ro * ro * ro - ri * ri * ri) / 3.0 * (G.cn[j] - G.cn[j + 1]) * G.dph;
}

__global__ void __launch_bounds__(kThreads) k_diag_sums(Dims d, Geo G, Vel v, const double* __restrict__ bh,
                                                        const double* __restrict__ br, const double* __restrict__ bt,
                                                        const double* __restrict__ bp, const double* __restrict__ jr,
                                                        const double* __restrict__ jt, const double* __restrict__ jp,
                                                        unsigned int* count, double* __restrict__ partials,
                                                        double* __restrict__ out) {
    double em = 0.0, ek = 0.0, jxb = 0.0, jdb = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.N;
         c += (long long)gridDim.x * blockDim.x) {
        int k;
        unsigned int ij;
        split_np(d, c, k, ij);
        const int j = (int)(ij % d.nt), i = (int)(ij / d.nt);
        double u[3], B[3], J[3];
        v.at(c, u);
        bcentre(d, G, bh, br, bt, bp, i, j, k, B);
        jcentre(d, jr, jt, jp, i, j, k, J);
        const double V = cell_volume(G, i, j);
        const double x0 = J[1] * B[2] - J[2] * B[1], x1 = J[2] * B[0] - J[0] * B[2], x2 = J[0] * B[1] - J[1] * B[0];
        em += 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) * V;
        ek += 0.5 * G.rho[i] * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * V;
        jxb += sqrt(x0 * x0 + x1 * x1 + x2 * x2) * V;
        jdb += fabs(J[0] * B[0] + J[1] * B[1] + J[2] * B[2]) * V;
    }
    double val[4] = {em, ek, jxb, jdb}, o[4];
    if (reduce_last<4>(val, partials, count, o) && threadIdx.x == 0)
        for (int q = 0; q < 4; q++) out[q] = o[q];
}

__global__ void __launch_bounds__(kThreads) k_diag_divmax(Dims d, Geo G, const double* __restrict__ br,
                                                          const double* __restrict__ bt,
                                                          const double* __restrict__ bp, unsigned int* count,
                                                          double* __restrict__ partials, double* __restrict__ out) {
    double m = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.N;
         c += (long long)gridDim.x * blockDim.x) {
        int k;
        unsigned int ij;
        split_np(d, c, k, ij);
        const int j = (int)(ij % d.nt), i = (int)(ij / d.nt);
        const double ri = G.r[i], ro = G.r[i + 1];
        const double ring = 0.5 * (ro * ro - ri * ri);
        const double band = G.cn[j] - G.cn[j + 1];
        const double ari = ri * ri * band * G.dph, aro = ro * ro * band * G.dph;
        const double atj = G.sn[j] * ring * G.dph, atj1 = G.sn[j + 1] * ring * G.dph;
        const double ap = ring * G.dth;
        const double flux = br[ix(d, i + 1, j, k)] * aro - br[ix(d, i, j, k)] * ari + bt[ixt(d, i, j + 1, k)] * atj1 -
                            bt[ixt(d, i, j, k)] * atj + bp[ix(d, i, j, kp1(d, k))] * ap - bp[ix(d, i, j, k)] * ap;
        m = fmax(m, fabs(flux) / cell_volume(G, i, j));
    }
    double val[1] = {m}, o[1];
    if (reduce_last<1, OpMax>(val, partials, count, o) && threadIdx.x == 0) out[0] = o[0];
}

// out (device, 5 doubles): the diagnostics of the fields; enqueued on the grid's stream
void diagnostics(mhd_grid_s* g, const double* vr, const double* vt, const double* vp, const double* br,
                 const double* bt, const double* bp, double* out) {
    const Dims d = g->d;
    current_edges(g, br, bt, bp);
    bt_harmonics(g, bt);
    Vel v{vr, vt, vp, nullptr, 0.0, d.N};
    const int blocks = grid_blocks(g, d.N, 8);
    k_diag_sums<<<blocks, kThreads, 0, g->stream>>>(d, g->geo, v, g->bharm, br, bt, bp, g->er, g->et, g->ep,
                                                    &g->ss->count, g->partials, out);
    k_diag_divmax<<<blocks, kThreads, 0, g->stream>>>(d, g->geo, br, bt, bp, &g->ss->count, g->partials, out + 4);
}

// ------------------------------------------------------------------------------------------
// v** = v + dlt (in place) and b = rho V v**
// ------------------------------------------------------------------------------------------
__global__ void k_vstar(Dims d, Geo G, double* __restrict__ vr, double* __restrict__ vt, double* __restrict__ vp,
                        const double* __restrict__ dlt, double* __restrict__ b) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.N;
         c += (long long)gridDim.x * blockDim.x) {
        const double w = G.rhoV[(unsigned int)c / (unsigned int)d.np];
        const double a = vr[c] + dlt[c], e = vt[c] + dlt[d.N + c], f = vp[c] + dlt[2 * d.N + c];
        vr[c] = a;
        vt[c] = e;
        vp[c] = f;
        b[c] = w * a;
        b[d.N + c] = w * e;
        b[2 * d.N + c] = w * f;
    }
}

void vstar_rhs(mhd_grid_s* g, double* vr, double* vt, double* vp, const double* dlt, double* b) {
    k_vstar<<<grid_blocks(g, g->d.N, 8), kThreads, 0, g->stream>>>(g->d, g->geo, vr, vt, vp, dlt, b);
}

}  // namespace mhd
