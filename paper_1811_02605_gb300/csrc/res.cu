// Implicit resistivity (Eq. 1: the -eta curl curl A term; Sec. 2.2: diffusive terms by PCG, the
// resistive solve always well conditioned and always with PC1), in B form on the faces.
//
// After the ideal CT update B* = B^n - dt curl_h E(v_bar, B^n), solve
//     W (x + dte curl_h J(x)) = W B*,   dte = dt eta,
// with J on the edges the circulation of x around each edge's dual face divided by its area (the
// edge current of the explicit path, set to 0 on the tangential edges of r0 and r1), curl_h the
// CT face circulation, and W_f = A_f l*_f (face area times the centre-to-centre distance across
// the face; half distances on the walls). With these weights J is the weighted adjoint of
// curl_h, so the system is symmetric positive definite. Point-Jacobi PCG on the stacked face
// vector [br | bt | bp] (polar theta faces: identity rows), then B = B* - dte curl_h J(x): the
// last update is a CT circulation, so div_h B keeps its value to rounding whatever the tolerance.
//
// Per iteration: edge current of p (ring sums + three edge kernels), q = M p with <p, q>, the
// x / r update with <r, z> and ||r||^2, and p = z + beta p; the scalar recurrence runs in the
// last CTA of each reducing kernel, and batches of iterations replay as one CUDA graph.
//
// Every geometric factor is a per-row table (a row is the np elements of one (i, j)): the edge
// kernels multiply by dual length / dual area, the face kernels by dte l* x edge length and by
// 1 / diag (formed once per solve), so no kernel of the iteration divides: FP64 division is a long
// instruction sequence on this part and these kernels are bound by the FP64 pipe.
#include <cmath>
#include <vector>

#include "mhd_internal.cuh"
#include "reduce.cuh"

namespace mhd {

namespace {

struct ResSizes {
    long long nbr, nbt, nbp, nf;   // face counts per family and total
    int tr, tt, tp;                // face rows per family
};

ResSizes res_sizes(const Dims& d) {
    ResSizes z;
    z.nbr = (long long)(d.nr + 1) * d.nt * d.np;
    z.nbt = (long long)d.nr * (d.nt + 1) * d.np;
    z.nbp = (long long)d.nr * d.nt * d.np;
    z.nf = z.nbr + z.nbt + z.nbp;
    z.tr = (d.nr + 1) * d.nt;
    z.tt = d.nr * (d.nt + 1);
    z.tp = d.nr * d.nt;
    return z;
}

// flat face index -> (family, row, i, j, k). The stacked face vector is a sequence of rows of np
// faces (r-face rows, then theta-face rows, then phi-face rows) in the order of the per-row
// tables, so the row is f / np; 32-bit arithmetic (nf < 2^31 is checked on the host).
struct Face {
    int fam, i, j, k;
    int t;
};
__device__ __forceinline__ Face face_of(const Dims& d, long long f) {
    Face o;
    const unsigned int uf = (unsigned int)f;
    const unsigned int row = uf / (unsigned int)d.np;
    o.k = (int)(uf - row * (unsigned int)d.np);
    o.t = (int)row;
    const unsigned int tr = (unsigned int)((d.nr + 1) * d.nt), tt = (unsigned int)(d.nr * (d.nt + 1));
    if (row < tr) {
        o.fam = 0;
        o.i = (int)(row / (unsigned int)d.nt);
        o.j = (int)(row - (unsigned int)o.i * d.nt);
    } else if (row < tr + tt) {
        o.fam = 1;
        const unsigned int q = row - tr;
        o.i = (int)(q / (unsigned int)(d.nt + 1));
        o.j = (int)(q - (unsigned int)o.i * (d.nt + 1));
    } else {
        o.fam = 2;
        const unsigned int q = row - tr - tt;
        o.i = (int)(q / (unsigned int)d.nt);
        o.j = (int)(q - (unsigned int)o.i * d.nt);
    }
    return o;
}

__device__ __forceinline__ int face_row(const Dims& d, long long f) {
    return (int)((unsigned int)f / (unsigned int)d.np);
}

// ------------------------------------------------------------------------------------------
// edge current of the resistive operator (interior edges; the tangential edges of r0 and r1
// carry none), from per-row coefficient tables
// ------------------------------------------------------------------------------------------
// radial edges (i, j, k), rows i (nt + 1) + j: c = {w_phi(j), w_phi(j-1), w_theta, w_polar}
__global__ void __launch_bounds__(kThreads) k_res_jr(Dims d, const double* __restrict__ cr,
                                                     const double* __restrict__ ring, const double* __restrict__ bt,
                                                     const double* __restrict__ bp, double* __restrict__ jr) {
    const long long n = (long long)d.nr * (d.nt + 1) * d.np;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int k;
        unsigned int row;
        split_np(d, e, k, row);
        const int i = (int)(row / (unsigned int)(d.nt + 1)), j = (int)(row - (unsigned int)i * (d.nt + 1));
        const double* c = cr + 4 * (size_t)row;
        double val;
        if (j == 0) val = ring[i] * c[3];
        else if (j == d.nt) val = -ring[d.nr + i] * c[3];
        else val = c[0] * bp[ix(d, i, j, k)] - c[1] * bp[ix(d, i, j - 1, k)] -
                   c[2] * (bt[ixt(d, i, j, k)] - bt[ixt(d, i, j, km1(d, k))]);
        jr[e] = val;
    }
}

// theta edges (i, j, k), rows i nt + j: c = {w_phi(i-1), w_r, w_phi(i)}
__global__ void __launch_bounds__(kThreads) k_res_jt(Dims d, const double* __restrict__ ct,
                                                     const double* __restrict__ br, const double* __restrict__ bp,
                                                     double* __restrict__ jt) {
    const long long n = (long long)(d.nr + 1) * d.nt * d.np;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int k;
        unsigned int row;
        split_np(d, e, k, row);
        const int i = (int)(row / (unsigned int)d.nt), j = (int)(row - (unsigned int)i * d.nt);
        double val = 0.0;
        if (i > 0 && i < d.nr) {
            const double* c = ct + 3 * (size_t)row;
            val = c[0] * bp[ix(d, i - 1, j, k)] + c[1] * (br[ix(d, i, j, k)] - br[ix(d, i, j, km1(d, k))]) -
                  c[2] * bp[ix(d, i, j, k)];
        }
        jt[e] = val;
    }
}

// phi edges (i, j, k), rows i (nt + 1) + j: c = {w_r, w_theta(i), w_theta(i-1)}
__global__ void __launch_bounds__(kThreads) k_res_jp(Dims d, const double* __restrict__ cp,
                                                     const double* __restrict__ br, const double* __restrict__ bt,
                                                     double* __restrict__ jp) {
    const long long n = (long long)(d.nr + 1) * (d.nt + 1) * d.np;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        int k;
        unsigned int row;
        split_np(d, e, k, row);
        const int i = (int)(row / (unsigned int)(d.nt + 1)), j = (int)(row - (unsigned int)i * (d.nt + 1));
        double val = 0.0;
        if (i > 0 && i < d.nr && j > 0 && j < d.nt) {
            const double* c = cp + 3 * (size_t)row;
            val = c[0] * (br[ix(d, i, j - 1, k)] - br[ix(d, i, j, k)]) + c[1] * bt[ixt(d, i, j, k)] -
                  c[2] * bt[ixt(d, i - 1, j, k)];
        }
        jp[e] = val;
    }
}

// ------------------------------------------------------------------------------------------
// face kernels; co[4 t + 0..2] = dte l* x the three edge-length factors of row t, co[4 t + 3] =
// 1 / diag (both formed per solve), w[t] = W of row t
// ------------------------------------------------------------------------------------------
// dte l* times the CT circulation of the edge current around face F (og_ct's sign convention;
// the polar radial edges hold the ring value in every k)
__device__ __forceinline__ double face_circ(const Dims& d, const Face& F, const double* __restrict__ co,
                                            const double* __restrict__ er, const double* __restrict__ et,
                                            const double* __restrict__ ep) {
    const int i = F.i, j = F.j, k = F.k;
    const double* c = co + 4 * (size_t)F.t;
    if (F.fam == 0)
        return c[0] * (et[ix(d, i, j, k)] - et[ix(d, i, j, kp1(d, k))]) + c[1] * ep[ixt(d, i, j + 1, k)] -
               c[2] * ep[ixt(d, i, j, k)];
    if (F.fam == 1) {
        if (j == 0 || j == d.nt) return 0.0;
        return c[0] * ep[ixt(d, i, j, k)] + c[1] * (er[ixt(d, i, j, kp1(d, k))] - er[ixt(d, i, j, k)]) -
               c[2] * ep[ixt(d, i + 1, j, k)];
    }
    return c[0] * (er[ixt(d, i, j, k)] - er[ixt(d, i, j + 1, k)]) + c[1] * et[ix(d, i + 1, j, k)] -
           c[2] * et[ix(d, i, j, k)];
}

__global__ void k_res_setup(PcgScalars* sc, double tol, int max_iter, const double* __restrict__ dt_dev, double eta) {
    sc->tol = tol;
    sc->max_iter = max_iter;
    sc->done = 0;
    sc->iter = 0;
    sc->total_iter = 0;
    sc->outer = 0;
    sc->count = 0u;
    sc->dte = *dt_dev * eta;
}

// per-solve row coefficients from the dte-independent tables
__global__ void k_res_coef(int rows, const double* __restrict__ w, const double* __restrict__ dc,
                           const double* __restrict__ el, const PcgScalars* sc, double* __restrict__ co) {
    const double dte = sc->dte;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < rows; t += gridDim.x * blockDim.x) {
        co[4 * t + 0] = dte * el[3 * t + 0];
        co[4 * t + 1] = dte * el[3 * t + 1];
        co[4 * t + 2] = dte * el[3 * t + 2];
        co[4 * t + 3] = 1.0 / fma(dte, dc[t], w[t]);
    }
}

// the edge current of x0 is in the edge arrays: r = b - M x0 with b = W x0 (x0 = B*), so
// r = -dte l* circ; x = x0, p = r / diag; rho = <r, z>, rr = ||r||^2, bb = ||b||^2
__global__ void __launch_bounds__(kThreads) k_res_init(Dims d, const double* __restrict__ w,
                                                       const double* __restrict__ co, const double* __restrict__ x0,
                                                       const double* __restrict__ er, const double* __restrict__ et,
                                                       const double* __restrict__ ep, double* __restrict__ x,
                                                       double* __restrict__ r, double* __restrict__ p, PcgScalars* sc,
                                                       double* __restrict__ partials, long long nf) {
    double a_rho = 0.0, a_rr = 0.0, a_bb = 0.0;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
        const Face F = face_of(d, f);
        const double xv = x0[f];
        const double rv = -face_circ(d, F, co, er, et, ep);
        const double z = rv * co[4 * (size_t)F.t + 3];
        x[f] = xv;
        r[f] = rv;
        p[f] = z;
        const double b = w[F.t] * xv;
        a_rho = fma(rv, z, a_rho);
        a_rr = fma(rv, rv, a_rr);
        a_bb = fma(b, b, a_bb);
    }
    double val[3] = {a_rho, a_rr, a_bb}, out[3];
    if (reduce_last<3>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        sc->rho = out[0];
        sc->rr = out[1];
        sc->bb = out[2];
        sc->beta = 0.0;
        if (!isfinite(out[0]) || !isfinite(out[1]) || !isfinite(out[2])) sc->done = 3;
        else if (out[2] == 0.0 || sqrt(out[1]) <= sc->tol * sqrt(out[2])) sc->done = 1;
        else if (sc->max_iter <= 0) sc->done = 2;
    }
}

// general right-hand side from x0 = 0: x = 0, r = b, p = r / diag; rho, ||r||^2, ||b||^2
__global__ void __launch_bounds__(kThreads) k_res_init_rhs(Dims d, const double* __restrict__ co,
                                                           const double* __restrict__ b, double* __restrict__ x,
                                                           double* __restrict__ r, double* __restrict__ p,
                                                           PcgScalars* sc, double* __restrict__ partials, long long nf) {
    double a_rho = 0.0, a_rr = 0.0;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
        const double rv = b[f];
        const double z = rv * co[4 * (size_t)face_row(d, f) + 3];
        x[f] = 0.0;
        r[f] = rv;
        p[f] = z;
        a_rho = fma(rv, z, a_rho);
        a_rr = fma(rv, rv, a_rr);
    }
    double val[2] = {a_rho, a_rr}, out[2];
    if (reduce_last<2>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        sc->rho = out[0];
        sc->rr = out[1];
        sc->bb = out[1];
        sc->beta = 0.0;
        if (!isfinite(out[0]) || !isfinite(out[1])) sc->done = 3;
        else if (out[1] == 0.0) sc->done = 1;
        else if (sc->max_iter <= 0) sc->done = 2;
    }
}

// out (three face arrays) = W x
__global__ void k_res_scale_w(Dims d, const double* __restrict__ w, const double* __restrict__ x,
                              double* __restrict__ br, double* __restrict__ bt, double* __restrict__ bp, long long nbr,
                              long long nbt, long long nf) {
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
        const double v = w[face_row(d, f)] * x[f];
        if (f < nbr) br[f] = v;
        else if (f < nbr + nbt) bt[f - nbr] = v;
        else bp[f - nbr - nbt] = v;
    }
}

// q = W p + dte l* circ(J(p)), <p, q>; last CTA: alpha
__global__ void __launch_bounds__(kThreads) k_res_apply(Dims d, const double* __restrict__ w,
                                                        const double* __restrict__ co, const double* __restrict__ p,
                                                        const double* __restrict__ er, const double* __restrict__ et,
                                                        const double* __restrict__ ep, double* __restrict__ q,
                                                        PcgScalars* sc, double* __restrict__ partials, long long nf) {
    if (sc->done) return;
    double a = 0.0;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
        const Face F = face_of(d, f);
        const double pv = p[f];
        const double qv = fma(w[F.t], pv, face_circ(d, F, co, er, et, ep));
        q[f] = qv;
        a = fma(pv, qv, a);
    }
    double val[1] = {a}, out[1];
    if (reduce_last<1>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        const double pq = out[0];
        sc->pq = pq;
        if (!isfinite(pq)) sc->done = 3;
        else if (!(pq > 0.0)) sc->done = 4;
        else sc->alpha = sc->rho / pq;
    }
}

// x += alpha p, r -= alpha q, rho = <r, r / diag>, rr = ||r||^2; last CTA: beta, stop test
__global__ void __launch_bounds__(kThreads) k_res_update(Dims d, const double* __restrict__ co, double* __restrict__ x,
                                                         const double* __restrict__ p, double* __restrict__ r,
                                                         const double* __restrict__ q, PcgScalars* sc,
                                                         double* __restrict__ partials, long long nf) {
    if (sc->done) return;
    const double al = sc->alpha;
    double a_rho = 0.0, a_rr = 0.0;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
        const double idg = co[4 * (size_t)face_row(d, f) + 3];
        x[f] = fma(al, p[f], x[f]);
        const double rv = fma(-al, q[f], r[f]);
        r[f] = rv;
        a_rho = fma(rv * rv, idg, a_rho);
        a_rr = fma(rv, rv, a_rr);
    }
    double val[2] = {a_rho, a_rr}, out[2];
    if (reduce_last<2>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        const double rho = out[0], rr = out[1];
        sc->iter += 1;
        sc->total_iter += 1;
        sc->beta = rho / sc->rho;
        sc->rho = rho;
        sc->rr = rr;
        if (!isfinite(rr) || !isfinite(rho)) sc->done = 3;
        else if (sqrt(rr) <= sc->tol * sqrt(sc->bb)) sc->done = 1;
        else if (sc->iter >= sc->max_iter) sc->done = 2;
    }
}

// p = r / diag + beta p
__global__ void __launch_bounds__(kThreads) k_res_pupdate(Dims d, const double* __restrict__ co,
                                                          const double* __restrict__ r, double* __restrict__ p,
                                                          const PcgScalars* sc, long long nf) {
    if (sc->done) return;
    const double be = sc->beta;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x)
        p[f] = fma(be, p[f], r[f] * co[4 * (size_t)face_row(d, f) + 3]);
}

// ------------------------------------------------------------------------------------------
// host tables (FP64, from the grid's node tables)
// ------------------------------------------------------------------------------------------
struct HostTabs {
    std::vector<double> w, dc, el;   // face rows: W, curl-curl diagonal part, l* x edge lengths (3)
    std::vector<double> cr, ct, cp;  // edge rows: dual length / dual area factors (4, 3, 3)
};

void res_tables(const mhd_grid_s* g, HostTabs& H) {
    const Dims d = g->d;
    const int nr = d.nr, nt = d.nt, np = d.np;
    const double PI = 3.14159265358979323846;
    const double dth = PI / nt, dph = 2.0 * PI / np;
    std::vector<double> r(nr + 1), rc(nr), sn(nt + 1), cn(nt + 1), sc(nt), cc(nt);
    cudaMemcpy(r.data(), g->geo.r, sizeof(double) * (nr + 1), cudaMemcpyDeviceToHost);
    cudaMemcpy(rc.data(), g->geo.rc, sizeof(double) * nr, cudaMemcpyDeviceToHost);
    cudaMemcpy(sn.data(), g->geo.sn, sizeof(double) * (nt + 1), cudaMemcpyDeviceToHost);
    cudaMemcpy(cn.data(), g->geo.cn, sizeof(double) * (nt + 1), cudaMemcpyDeviceToHost);
    cudaMemcpy(sc.data(), g->geo.sc, sizeof(double) * nt, cudaMemcpyDeviceToHost);
    cudaMemcpy(cc.data(), g->geo.cc, sizeof(double) * nt, cudaMemcpyDeviceToHost);
    auto lsr = [&](int i) { return i == 0 ? rc[0] - r[0] : (i == nr ? r[nr] - rc[nr - 1] : rc[i] - rc[i - 1]); };
    // dual-face areas of the interior edges: radial (shell i, node j), theta (node i, centre j),
    // phi (node i, any j)
    auto asr = [&](int i, int j) { return rc[i] * rc[i] * (cc[j - 1] - cc[j]) * dph; };
    auto ast = [&](int i, int j) { return sc[j] * 0.5 * (rc[i] * rc[i] - rc[i - 1] * rc[i - 1]) * dph; };
    auto asp = [&](int i) { return 0.5 * (rc[i] * rc[i] - rc[i - 1] * rc[i - 1]) * dth; };
    const int tr = (nr + 1) * nt, tt = nr * (nt + 1), tp = nr * nt;
    H.w.assign(tr + tt + tp, 0.0);
    H.dc.assign(tr + tt + tp, 0.0);
    H.el.assign(3 * (size_t)(tr + tt + tp), 0.0);
    for (int i = 0; i <= nr; i++)
        for (int j = 0; j < nt; j++) {
            const int t = i * nt + j;
            const double l = lsr(i);
            H.w[t] = r[i] * r[i] * (cn[j] - cn[j + 1]) * dph * l;
            H.el[3 * t + 0] = l * (r[i] * dth);
            H.el[3 * t + 1] = l * (r[i] * sn[j + 1] * dph);
            H.el[3 * t + 2] = l * (r[i] * sn[j] * dph);
            if (i >= 1 && i <= nr - 1) {
                double s = 2.0 * r[i] * dth / ast(i, j);
                if (j >= 1) s += r[i] * sn[j] * dph / asp(i);
                if (j + 1 <= nt - 1) s += r[i] * sn[j + 1] * dph / asp(i);
                H.dc[t] = l * l * s;
            }
        }
    for (int i = 0; i < nr; i++)
        for (int j = 0; j <= nt; j++) {
            const int t = tr + i * (nt + 1) + j;
            const double l = rc[i] * dth;
            if (j == 0 || j == nt) {
                H.w[t] = 1.0;
                continue;
            }
            H.w[t] = sn[j] * 0.5 * (r[i + 1] * r[i + 1] - r[i] * r[i]) * dph * l;
            const double lr = r[i + 1] - r[i];
            H.el[3 * t + 0] = l * (r[i] * sn[j] * dph);
            H.el[3 * t + 1] = l * lr;
            H.el[3 * t + 2] = l * (r[i + 1] * sn[j] * dph);
            double s = 2.0 * lr / asr(i, j);
            if (i >= 1) s += r[i] * sn[j] * dph / asp(i);
            if (i + 1 <= nr - 1) s += r[i + 1] * sn[j] * dph / asp(i + 1);
            H.dc[t] = l * l * s;
        }
    for (int i = 0; i < nr; i++) {
        const double lr = r[i + 1] - r[i];
        const double cap_n = rc[i] * rc[i] * (1.0 - cc[0]) * 2.0 * PI;
        const double cap_s = rc[i] * rc[i] * (1.0 + cc[nt - 1]) * 2.0 * PI;
        for (int j = 0; j < nt; j++) {
            const int t = tr + tt + i * nt + j;
            const double l = rc[i] * sc[j] * dph;
            H.w[t] = 0.5 * (r[i + 1] * r[i + 1] - r[i] * r[i]) * dth * l;
            H.el[3 * t + 0] = l * lr;
            H.el[3 * t + 1] = l * (r[i + 1] * dth);
            H.el[3 * t + 2] = l * (r[i] * dth);
            double s = lr / (j == 0 ? cap_n : asr(i, j)) + lr / (j == nt - 1 ? cap_s : asr(i, j + 1));
            if (i >= 1) s += r[i] * dth / ast(i, j);
            if (i + 1 <= nr - 1) s += r[i + 1] * dth / ast(i + 1, j);
            H.dc[t] = l * l * s;
        }
    }
    // edge rows
    H.cr.assign(4 * (size_t)nr * (nt + 1), 0.0);
    for (int i = 0; i < nr; i++) {
        const double cap_n = rc[i] * rc[i] * (1.0 - cc[0]) * 2.0 * PI;
        const double cap_s = rc[i] * rc[i] * (1.0 + cc[nt - 1]) * 2.0 * PI;
        for (int j = 0; j <= nt; j++) {
            double* c = &H.cr[4 * ((size_t)i * (nt + 1) + j)];
            if (j == 0) {
                c[3] = rc[i] * sc[0] * dph / cap_n;
            } else if (j == nt) {
                c[3] = rc[i] * sc[nt - 1] * dph / cap_s;
            } else {
                const double ia = 1.0 / asr(i, j);
                c[0] = rc[i] * sc[j] * dph * ia;
                c[1] = rc[i] * sc[j - 1] * dph * ia;
                c[2] = rc[i] * dth * ia;
            }
        }
    }
    H.ct.assign(3 * (size_t)(nr + 1) * nt, 0.0);
    H.cp.assign(3 * (size_t)(nr + 1) * (nt + 1), 0.0);
    for (int i = 1; i < nr; i++) {
        const double rlo = rc[i - 1], rhi = rc[i];
        for (int j = 0; j < nt; j++) {
            double* c = &H.ct[3 * ((size_t)i * nt + j)];
            const double ia = 1.0 / ast(i, j);
            c[0] = rlo * sc[j] * dph * ia;
            c[1] = (rhi - rlo) * ia;
            c[2] = rhi * sc[j] * dph * ia;
        }
        for (int j = 1; j < nt; j++) {
            double* c = &H.cp[3 * ((size_t)i * (nt + 1) + j)];
            const double ia = 1.0 / asp(i);
            c[0] = (rhi - rlo) * ia;
            c[1] = rhi * dth * ia;
            c[2] = rlo * dth * ia;
        }
    }
}

struct ResWork {
    double *x, *r, *p, *q;           // nf each
    double *w, *dc, *el, *co;        // face-row tables (co: per solve)
    double *cr, *ct, *cp;            // edge-row tables
    cudaGraphExec_t graph;
};

mhd_status_t res_workspace(mhd_grid_s* g, ResWork** out) {
    if (g->res_mem) {
        *out = reinterpret_cast<ResWork*>(g->res_mem);
        return MHD_OK;
    }
    const ResSizes z = res_sizes(g->d);
    if (z.nf >= (1LL << 31)) return set_error(g, MHD_ERR_ARG, "implicit resistivity: grid too large (2^31 faces)");
    HostTabs H;
    res_tables(g, H);
    const size_t rows = (size_t)z.tr + z.tt + z.tp;
    const size_t total = 4 * (size_t)z.nf + rows * (1 + 1 + 3 + 4) + H.cr.size() + H.ct.size() + H.cp.size();
    auto* w = new ResWork{};
    double* m = nullptr;
    if (cudaMalloc(&m, sizeof(double) * total) != cudaSuccess) {
        delete w;
        cudaGetLastError();
        return set_error(g, MHD_ERR_OOM, "implicit resistivity: workspace allocation failed");
    }
    w->x = m;
    w->r = m + z.nf;
    w->p = m + 2 * z.nf;
    w->q = m + 3 * z.nf;
    w->w = m + 4 * z.nf;
    w->dc = w->w + rows;
    w->el = w->dc + rows;
    w->co = w->el + 3 * rows;
    w->cr = w->co + 4 * rows;
    w->ct = w->cr + H.cr.size();
    w->cp = w->ct + H.ct.size();
    cudaMemcpy(w->w, H.w.data(), sizeof(double) * rows, cudaMemcpyHostToDevice);
    cudaMemcpy(w->dc, H.dc.data(), sizeof(double) * rows, cudaMemcpyHostToDevice);
    cudaMemcpy(w->el, H.el.data(), sizeof(double) * 3 * rows, cudaMemcpyHostToDevice);
    cudaMemcpy(w->cr, H.cr.data(), sizeof(double) * H.cr.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(w->ct, H.ct.data(), sizeof(double) * H.ct.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(w->cp, H.cp.data(), sizeof(double) * H.cp.size(), cudaMemcpyHostToDevice);
    g->res_mem = w;
    *out = w;
    return check_cuda(g, "implicit resistivity workspace");
}

// edge current of the stacked face vector v into the grid's edge arrays
void res_current(mhd_grid_s* g, cudaStream_t st, const ResWork* w, const double* v) {
    const Dims d = g->d;
    const ResSizes z = res_sizes(d);
    const double *br = v, *bt = v + z.nbr, *bp = v + z.nbr + z.nbt;
    ring_sums(g, bp, st);
    const long long n = (long long)(d.nr + 1) * (d.nt + 1) * d.np;
    k_res_jr<<<grid_blocks(g, n, resident_per_sm<k_res_jr>()), kThreads, 0, st>>>(d, w->cr, g->ring, bt, bp, g->er);
    k_res_jt<<<grid_blocks(g, n, resident_per_sm<k_res_jt>()), kThreads, 0, st>>>(d, w->ct, br, bp, g->et);
    k_res_jp<<<grid_blocks(g, n, resident_per_sm<k_res_jp>()), kThreads, 0, st>>>(d, w->cp, br, bt, g->ep);
}

void res_enqueue_iteration(mhd_grid_s* g, cudaStream_t st, ResWork* w) {
    const Dims d = g->d;
    const ResSizes z = res_sizes(d);
    res_current(g, st, w, w->p);
    k_res_apply<<<grid_blocks(g, z.nf, resident_per_sm<k_res_apply>()), kThreads, 0, st>>>(
        d, w->w, w->co, w->p, g->er, g->et, g->ep, w->q, g->sc, g->partials, z.nf);
    k_res_update<<<grid_blocks(g, z.nf, resident_per_sm<k_res_update>()), kThreads, 0, st>>>(
        d, w->co, w->x, w->p, w->r, w->q, g->sc, g->partials, z.nf);
    k_res_pupdate<<<grid_blocks(g, z.nf, resident_per_sm<k_res_pupdate>()), kThreads, 0, st>>>(d, w->co, w->r, w->p,
                                                                                               g->sc, z.nf);
}

mhd_status_t res_graph(mhd_grid_s* g, ResWork* w) {
    if (w->graph) return MHD_OK;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return check_cuda(g, "res graph stream");
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return check_cuda(g, "res graph capture");
    }
    for (int it = 0; it < g->graph_batch; it++) res_enqueue_iteration(g, cs, w);
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return set_error(g, MHD_ERR_CUDA, std::string("res end capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&w->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return set_error(g, MHD_ERR_CUDA, std::string("res instantiate: ") + cudaGetErrorString(e));
    return MHD_OK;
}

mhd_status_t res_read(mhd_grid_s* g) {
    if (cudaMemcpyAsync(g->h_sc, g->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
        return check_cuda(g, "res read scalars");
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return check_cuda(g, "res sync");
    return MHD_OK;
}

// scalar set-up and the per-solve row coefficients
void res_begin(mhd_grid_s* g, ResWork* w, const double* dt_dev, double eta, const mhd_params_t* p) {
    const ResSizes z = res_sizes(g->d);
    const int rows = z.tr + z.tt + z.tp;
    k_res_setup<<<1, 1, 0, g->stream>>>(g->sc, p->tol, p->max_iter, dt_dev, eta);
    k_res_coef<<<(rows + kThreads - 1) / kThreads, kThreads, 0, g->stream>>>(rows, w->w, w->dc, w->el, g->sc, w->co);
}

mhd_status_t res_iterate(mhd_grid_s* g, ResWork* w) {
    mhd_status_t st;
    for (;;) {
        if ((st = res_read(g)) != MHD_OK) return st;
        if (g->h_sc->done) return MHD_OK;
        if (cudaGraphLaunch(w->graph, g->stream) != cudaSuccess) return check_cuda(g, "res graph launch");
        if (cudaGraphLaunch(w->graph, g->stream) != cudaSuccess) return check_cuda(g, "res graph launch");
    }
}

}  // namespace

void res_free(mhd_grid_s* g) {
    if (!g->res_mem) return;
    auto* w = reinterpret_cast<ResWork*>(g->res_mem);
    if (w->graph) cudaGraphExecDestroy(w->graph);
    cudaFree(w->x);
    delete w;
    g->res_mem = nullptr;
}

// Transpose of the resistive map for the adjoint: with an exact solve the step's B = B* - dte
// curl_h J(x) equals x = M^-1 W B*, so its transpose is W M^-1. In place on the three face arrays:
// lam <- W y with M y = lam (PCG from y = 0, tolerance and cap from p).
mhd_status_t res_transpose(mhd_grid_s* g, const double* dt_dev, double eta, double* lr, double* lt, double* lp,
                           const mhd_params_t* p) {
    ResWork* w = nullptr;
    mhd_status_t st = res_workspace(g, &w);
    if (st != MHD_OK) return st;
    if ((st = res_graph(g, w)) != MHD_OK) return st;
    const Dims d = g->d;
    const ResSizes z = res_sizes(d);
    const int blocks = grid_blocks(g, z.nf, 8);
    cudaMemcpyAsync(w->q, lr, sizeof(double) * z.nbr, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(w->q + z.nbr, lt, sizeof(double) * z.nbt, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(w->q + z.nbr + z.nbt, lp, sizeof(double) * z.nbp, cudaMemcpyDeviceToDevice, g->stream);
    res_begin(g, w, dt_dev, eta, p);
    k_res_init_rhs<<<blocks, kThreads, 0, g->stream>>>(d, w->co, w->q, w->x, w->r, w->p, g->sc, g->partials, z.nf);
    if ((st = check_cuda(g, "res transpose init")) != MHD_OK) return st;
    if ((st = res_iterate(g, w)) != MHD_OK) return st;
    const int done = g->h_sc->done;
    k_res_scale_w<<<blocks, kThreads, 0, g->stream>>>(d, w->w, w->x, lr, lt, lp, z.nbr, z.nbt, z.nf);
    if ((st = check_cuda(g, "res transpose scale")) != MHD_OK) return st;
    if (done == 1) return MHD_OK;
    if (done == 3) return set_error(g, MHD_ERR_NONFINITE, "resistive transpose: non-finite value");
    return set_error(g, MHD_ERR_NOCONV, "resistive transpose: no convergence within max_iter");
}

// B (caller's face arrays, holding B*) <- B* - dte curl_h J(x), x the PCG solution; dte = dt eta
// with dt the step's device scalar
mhd_status_t res_solve(mhd_grid_s* g, const double* dt_dev, double eta, double* br, double* bt, double* bp,
                       const mhd_params_t* p, int* iters, double* relres) {
    ResWork* w = nullptr;
    mhd_status_t st = res_workspace(g, &w);
    if (st != MHD_OK) return st;
    if ((st = res_graph(g, w)) != MHD_OK) return st;
    const Dims d = g->d;
    const ResSizes z = res_sizes(d);
    const int blocks = grid_blocks(g, z.nf, 8);
    // x0 = B* gathered into the stacked vector
    cudaMemcpyAsync(w->q, br, sizeof(double) * z.nbr, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(w->q + z.nbr, bt, sizeof(double) * z.nbt, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(w->q + z.nbr + z.nbt, bp, sizeof(double) * z.nbp, cudaMemcpyDeviceToDevice, g->stream);
    res_begin(g, w, dt_dev, eta, p);
    res_current(g, g->stream, w, w->q);
    k_res_init<<<blocks, kThreads, 0, g->stream>>>(d, w->w, w->co, w->q, g->er, g->et, g->ep, w->x, w->r, w->p, g->sc,
                                                   g->partials, z.nf);
    if ((st = check_cuda(g, "res init")) != MHD_OK) return st;
    if ((st = res_iterate(g, w)) != MHD_OK) return st;
    const PcgScalars h = *g->h_sc;
    // B = B* - dte curl_h J(x)
    res_current(g, g->stream, w, w->x);
    ct_apply(g, &g->sc->dte, br, bt, bp);
    if ((st = check_cuda(g, "res final update")) != MHD_OK) return st;
    if (iters) *iters = h.iter;
    if (relres) *relres = (h.bb > 0) ? std::sqrt(h.rr) / std::sqrt(h.bb) : 0.0;
    if (h.done == 1) return MHD_OK;
    if (h.done == 3) return set_error(g, MHD_ERR_NONFINITE, "resistive pcg: non-finite value");
    if (h.done == 4) return set_error(g, MHD_ERR_NOCONV, "resistive pcg: breakdown");
    return set_error(g, MHD_ERR_NOCONV, "resistive pcg: no convergence within max_iter");
}

// workspace and iteration graph of the implicit resistive solve, allocated ahead of the first step
mhd_status_t res_reserve(mhd_grid_s* g) {
    ResWork* w = nullptr;
    mhd_status_t st = res_workspace(g, &w);
    if (st != MHD_OK) return st;
    return res_graph(g, w);
}

}  // namespace mhd
