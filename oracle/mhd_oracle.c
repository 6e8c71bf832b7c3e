/*
 * Plain FP64 CPU oracle for the zero-beta MHD step (arXiv 1811.02605). TEST INFRASTRUCTURE:
 * only tests, the smoke check and the benchmark's CPU baseline use it. See mhd_oracle.h for
 * layouts. Each function cites the passage of the paper it restates; where the paper is silent
 * the comment states the reading taken.
 *
 * The default build is plain sequential C. The `omp` pragmas below only take effect in the
 * separate timing build (compiled with -fopenmp, used by the benchmark's CPU baseline on all host
 * cores): they split loops whose iterations are independent, and the inner product then sums
 * fixed chunks and combines them in chunk order, so its value does not depend on the thread
 * count.
 */
#include "mhd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

struct og_grid {
    int nr, nt, np;
    long long N;
    double r0, r1, stretch;
    double dth, dph;
    double *r;        /* nr+1 radial nodes */
    double *rc;       /* nr   radial centres */
    double *sn, *cn;  /* nt+1 sin/cos of theta nodes (exact 0, +-1 at the poles) */
    double *sc, *cc;  /* nt   sin/cos of theta centres */
    /* per (i,j) tables, nr*nt: cell volume, rho at the centre, k~^2 */
    double *vol, *rho, *kt2;
    /* stiffness weights of the symmetric operator K (reading R3):
     *   wr[i*nt+j], i = 0..nr  : radial face i (between cells i-1 and i); wr[0] is the
     *                            Dirichlet weight at r0 (one-sided), wr[nr] = 0 (Neumann)
     *   wt[i*(nt+1)+j], j = 0..nt : theta face j; 0 at the poles (zero face area)
     *   wp[i*nt+j]              : each of the two phi faces of the cell */
    double *wr, *wt, *wp;
};

#define IDX(g, i, j, k) ((((long long)(i)) * (g)->nt + (j)) * (g)->np + (k))
#define IDXT(g, i, j, k) ((((long long)(i)) * ((g)->nt + 1) + (j)) * (g)->np + (k))
#define KP(g, k) (((k) + 1) % (g)->np)
#define KM(g, k) (((k) + (g)->np - 1) % (g)->np)

static double rho0(const og_grid* g, double r) { return (g->r0 / r) * (g->r0 / r); }
static void res_weights(const og_grid* g, double* w);

/* ---------------------------------------------------------------------------------------------
 * Grid (reading R2: geometric radial stretch, uniform theta in [0,pi], periodic phi; exact
 * finite-volume geometry of spherical cells).
 * ------------------------------------------------------------------------------------------- */
/* threads of the timing build (n > 0 sets them); 1 in the plain build */
int og_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

og_grid* og_create(int nr, int nt, int np, double r0, double r1, double stretch) {
    if (nr < 2 || nt < 2 || np < 1 || !(r1 > r0) || !(r0 > 0) || !(stretch > 0)) return NULL;
    og_grid* g = (og_grid*)calloc(1, sizeof(og_grid));
    g->nr = nr; g->nt = nt; g->np = np;
    g->N = (long long)nr * nt * np;
    g->r0 = r0; g->r1 = r1; g->stretch = stretch;
    g->dth = M_PI / nt;
    g->dph = 2.0 * M_PI / np;
    g->r = (double*)malloc(sizeof(double) * (nr + 1));
    g->rc = (double*)malloc(sizeof(double) * nr);
    g->sn = (double*)malloc(sizeof(double) * (nt + 1));
    g->cn = (double*)malloc(sizeof(double) * (nt + 1));
    g->sc = (double*)malloc(sizeof(double) * nt);
    g->cc = (double*)malloc(sizeof(double) * nt);
    g->vol = (double*)malloc(sizeof(double) * nr * nt);
    g->rho = (double*)malloc(sizeof(double) * nr * nt);
    g->kt2 = (double*)malloc(sizeof(double) * nr * nt);
    g->wr = (double*)calloc((size_t)(nr + 1) * nt, sizeof(double));
    g->wt = (double*)calloc((size_t)nr * (nt + 1), sizeof(double));
    g->wp = (double*)calloc((size_t)nr * nt, sizeof(double));

    /* r_{i+1} = r_i + h0 s^i, h0 = (r1-r0)(s-1)/(s^nr-1) */
    double h0;
    if (stretch == 1.0) {
        h0 = (r1 - r0) / nr;
    } else {
        double snr = 1.0;
        for (int i = 0; i < nr; i++) snr *= stretch;
        h0 = (r1 - r0) * (stretch - 1.0) / (snr - 1.0);
    }
    g->r[0] = r0;
    double dr = h0;
    for (int i = 0; i < nr; i++) { g->r[i + 1] = g->r[i] + dr; dr *= stretch; }
    for (int i = 0; i < nr; i++) g->rc[i] = 0.5 * (g->r[i] + g->r[i + 1]);
    for (int j = 0; j <= nt; j++) { g->sn[j] = sin(j * g->dth); g->cn[j] = cos(j * g->dth); }
    g->sn[0] = 0.0; g->sn[nt] = 0.0; g->cn[0] = 1.0; g->cn[nt] = -1.0;
    for (int j = 0; j < nt; j++) { g->sc[j] = sin((j + 0.5) * g->dth); g->cc[j] = cos((j + 0.5) * g->dth); }

    for (int i = 0; i < nr; i++) {
        double ri = g->r[i], ro = g->r[i + 1];
        double ring = 0.5 * (ro * ro - ri * ri);       /* int r dr over the shell */
        for (int j = 0; j < nt; j++) {
            double band = g->cn[j] - g->cn[j + 1];      /* int sin(theta) dtheta over the band */
            g->vol[i * nt + j] = (ro * ro * ro - ri * ri * ri) / 3.0 * band * g->dph;
            g->rho[i * nt + j] = rho0(g, g->rc[i]);
            double a = ro - ri;
            double b = g->rc[i] * g->dth;
            double c = g->rc[i] * g->sc[j] * g->dph;
            g->kt2[i * nt + j] = 1.0 / (a * a) + 1.0 / (b * b) + 1.0 / (c * c);
            /* phi face: area ring*dth, centre distance rc sin(theta_c) dphi, rho at rc */
            g->wp[i * nt + j] = g->rho[i * nt + j] * (ring * g->dth) / c;
        }
        /* theta faces j = 1..nt-1: area sin(theta_j) ring dphi, distance rc dth */
        for (int j = 1; j < nt; j++)
            g->wt[i * (nt + 1) + j] = rho0(g, g->rc[i]) * (g->sn[j] * ring * g->dph) / (g->rc[i] * g->dth);
    }
    for (int j = 0; j < nt; j++) {
        double band = g->cn[j] - g->cn[j + 1];
        /* Dirichlet face at r0: rho0(r0) A / (rc_0 - r0) */
        g->wr[0 * nt + j] = rho0(g, r0) * (r0 * r0 * band * g->dph) / (g->rc[0] - r0);
        /* interior radial faces: rho0(r_i) A / (rc_i - rc_{i-1}) */
        for (int i = 1; i < nr; i++)
            g->wr[i * nt + j] = rho0(g, g->r[i]) * (g->r[i] * g->r[i] * band * g->dph) / (g->rc[i] - g->rc[i - 1]);
        g->wr[nr * nt + j] = 0.0; /* Neumann at r1 */
    }
    return g;
}

void og_destroy(og_grid* g) {
    if (!g) return;
    free(g->r); free(g->rc); free(g->sn); free(g->cn); free(g->sc); free(g->cc);
    free(g->vol); free(g->rho); free(g->kt2); free(g->wr); free(g->wt); free(g->wp);
    free(g);
}

void og_radial_nodes(const og_grid* g, double* r) { memcpy(r, g->r, sizeof(double) * (g->nr + 1)); }
void og_volumes(const og_grid* g, double* v) { memcpy(v, g->vol, sizeof(double) * g->nr * g->nt); }
void og_ktilde2(const og_grid* g, double* k) { memcpy(k, g->kt2, sizeof(double) * g->nr * g->nt); }

/* ---------------------------------------------------------------------------------------------
 * Implicit operator (Eq. 1, viscous and semi-implicit terms; Sec. 4.1: sparse matrix-vector
 * products that are stencil operations). Reading R3: the operator (1/rho) div(rho grad u)
 * acts on each spherical component separately; multiplied by the cell volume it becomes the
 * symmetric finite-volume form M_alpha = D + alpha K with D = rho_c V_c and
 * (K u)_c = sum over faces w_f (u_c - u_nb), Dirichlet u = 0 at r0, Neumann at r1.
 * ------------------------------------------------------------------------------------------- */
static void apply_op(const og_grid* g, double alpha, int with_d, int with_dirichlet, int ncomp,
                     const double* p, double* q) {
    int nr = g->nr, nt = g->nt, np = g->np;
    for (int c = 0; c < ncomp; c++) {
        const double* u = p + c * g->N;
        double* o = q + c * g->N;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < nr; i++)
            for (int j = 0; j < nt; j++)
                for (int k = 0; k < np; k++) {
                    double uc = u[IDX(g, i, j, k)];
                    double s = 0.0;
                    if (i > 0) s += g->wr[i * nt + j] * (uc - u[IDX(g, i - 1, j, k)]);
                    else if (with_dirichlet) s += g->wr[0 * nt + j] * uc;
                    if (i < nr - 1) s += g->wr[(i + 1) * nt + j] * (uc - u[IDX(g, i + 1, j, k)]);
                    if (j > 0) s += g->wt[i * (nt + 1) + j] * (uc - u[IDX(g, i, j - 1, k)]);
                    if (j < nt - 1) s += g->wt[i * (nt + 1) + j + 1] * (uc - u[IDX(g, i, j + 1, k)]);
                    s += g->wp[i * nt + j] * (uc - u[IDX(g, i, j, KM(g, k))]);
                    s += g->wp[i * nt + j] * (uc - u[IDX(g, i, j, KP(g, k))]);
                    double d = with_d ? g->rho[i * nt + j] * g->vol[i * nt + j] * uc : 0.0;
                    o[IDX(g, i, j, k)] = d + alpha * s;
                }
    }
}

void og_apply_M(const og_grid* g, double alpha, int ncomp, const double* p, double* q) {
    apply_op(g, alpha, 1, 1, ncomp, p, q);
}

void og_apply_K_neumann(const og_grid* g, int ncomp, const double* p, double* q) {
    apply_op(g, 1.0, 0, 0, ncomp, p, q);
}

void og_diag(const og_grid* g, double alpha, double* d) {
    int nr = g->nr, nt = g->nt;
    for (int i = 0; i < nr; i++)
        for (int j = 0; j < nt; j++) {
            double s = g->wr[i * nt + j] + g->wr[(i + 1) * nt + j] + g->wt[i * (nt + 1) + j] +
                       g->wt[i * (nt + 1) + j + 1] + 2.0 * g->wp[i * nt + j];
            d[i * nt + j] = g->rho[i * nt + j] * g->vol[i * nt + j] + alpha * s;
        }
}

/* ---------------------------------------------------------------------------------------------
 * PCG with PC1 (Sec. 2.2: preconditioning by the inverse of the matrix diagonal). Reading P12:
 * one stacked system for all components with one alpha and one beta; stop when the
 * recursively updated residual satisfies ||r||_2 <= tol ||b||_2, tested before each iteration;
 * the count is the number of x updates; b = 0 gives x = 0 after 0 iterations.
 * ------------------------------------------------------------------------------------------- */
/* Inner product (reading P12: FP64 dot products whose value does not depend on the order of the
 * terms beyond rounding). Algorithm Dot2 of Ogita, Rump & Oishi (2005): each product is split
 * exactly into p + e (e, its rounding error, from an fma), the products are summed with Knuth's
 * error-free TwoSum, and the collected errors are added at the end. The result is as accurate as a
 * sum taken in twice the working precision and then rounded, whatever the length, so the PCG
 * scalars alpha and beta carry no summation-order error of this side's own. */
static void dot2_range(const double* a, const double* b, long long lo, long long hi, double* sum, double* err) {
    double s = 0.0, c = 0.0;
    for (long long i = lo; i < hi; i++) {
        double p = a[i] * b[i];
        double pe = fma(a[i], b[i], -p);
        double t = s + p;
        double z = t - s;
        c += ((s - (t - z)) + (p - z)) + pe;
        s = t;
    }
    *sum = s;
    *err = c;
}

static double dot(long long n, const double* a, const double* b) {
#ifdef _OPENMP
    /* timing build: 256 fixed chunks, each by Dot2, then the chunk sums by TwoSum in order */
    enum { NCH = 256 };
    double cs[NCH], ce[NCH];
    long long len = (n + NCH - 1) / NCH;
#pragma omp parallel for schedule(static)
    for (int ch = 0; ch < NCH; ch++) {
        long long lo = ch * len, hi = lo + len < n ? lo + len : n;
        if (lo > n) lo = n;
        dot2_range(a, b, lo, hi, &cs[ch], &ce[ch]);
    }
    double s = 0.0, c = 0.0;
    for (int ch = 0; ch < NCH; ch++) {
        double t = s + cs[ch];
        double z = t - s;
        c += ((s - (t - z)) + (cs[ch] - z)) + ce[ch];
        s = t;
    }
    return s + c;
#else
    double s, c;
    dot2_range(a, b, 0, n, &s, &c);
    return s + c;
#endif
}

double og_dot(long long n, const double* a, const double* b) { return dot(n, a, b); }

int og_pcg(const og_grid* g, double alpha, int ncomp, const double* b, double* x, double tol,
           int max_iter, int fixed_iters, int* iters, double* relres) {
    long long N = g->N, n = ncomp * N;
    int nt = g->nt, np = g->np;
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
        *iters = 0; *relres = 0.0;
        return OG_OK;
    }
    double* d = (double*)malloc(sizeof(double) * g->nr * nt);
    double* r = (double*)malloc(sizeof(double) * n);
    double* z = (double*)malloc(sizeof(double) * n);
    double* p = (double*)malloc(sizeof(double) * n);
    double* q = (double*)malloc(sizeof(double) * n);
    og_diag(g, alpha, d);
    og_apply_M(g, alpha, ncomp, x, q);
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n; e++) r[e] = b[e] - q[e];
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n; e++) z[e] = r[e] / d[(e % N) / np];
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n; e++) p[e] = z[e];
    double rz = dot(n, r, z);
    double rn = sqrt(dot(n, r, r));
    int k = 0;
    int status = OG_OK;
    for (;;) {
        if (fixed_iters > 0) {
            if (k >= fixed_iters) break;
        } else {
            if (rn <= tol * bnorm) break;
            if (k >= max_iter) { status = OG_ERR_NOCONV; break; }
        }
        og_apply_M(g, alpha, ncomp, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) { status = OG_ERR_NOCONV; break; }
        double a = rz / pq;
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) x[e] += a * p[e];
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) r[e] -= a * q[e];
        k++;
        rn = sqrt(dot(n, r, r));
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) z[e] = r[e] / d[(e % N) / np];
        double rz_new = dot(n, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) p[e] = z[e] + beta * p[e];
    }
    *iters = k;
    *relres = rn / bnorm;
    free(d); free(r); free(z); free(p); free(q);
    return status;
}

/* ---------------------------------------------------------------------------------------------
 * The same Jacobi PCG in the single-reduction form of Chronopoulos & Gear (1989): the search
 * direction's image s = M p is carried by its own recurrence, so both inner products of an
 * iteration, (r, u) and (M u, u) with u = D^-1 r, come from one pass after one operator
 * application. In exact arithmetic the iterates are those of og_pcg; the stop test, the count and
 * the b = 0 case are the same.
 * ------------------------------------------------------------------------------------------- */
int og_pcg_cg(const og_grid* g, double alpha, int ncomp, const double* b, double* x, double tol,
              int max_iter, int fixed_iters, int* iters, double* relres) {
    long long N = g->N, n = ncomp * N;
    int nt = g->nt, np = g->np;
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
        *iters = 0; *relres = 0.0;
        return OG_OK;
    }
    double* d = (double*)malloc(sizeof(double) * g->nr * nt);
    double* r = (double*)malloc(sizeof(double) * n);
    double* u = (double*)malloc(sizeof(double) * n);
    double* w = (double*)malloc(sizeof(double) * n);
    double* p = (double*)calloc(n, sizeof(double));
    double* sv = (double*)calloc(n, sizeof(double));
    og_diag(g, alpha, d);
    og_apply_M(g, alpha, ncomp, x, w);
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n; e++) r[e] = b[e] - w[e];
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n; e++) u[e] = r[e] / d[(e % N) / np];
    og_apply_M(g, alpha, ncomp, u, w);
    double gam = dot(n, r, u), del = dot(n, w, u);
    double rn = sqrt(dot(n, r, r));
    double a = 0.0, gam_old = 0.0;
    int k = 0;
    int status = OG_OK;
    for (;;) {
        if (fixed_iters > 0) {
            if (k >= fixed_iters) break;
        } else {
            if (rn <= tol * bnorm) break;
            if (k >= max_iter) { status = OG_ERR_NOCONV; break; }
        }
        double beta, den;
        if (k == 0) {
            beta = 0.0;
            den = del;
        } else {
            beta = gam / gam_old;
            den = del - beta * gam / a;
        }
        if (!(den > 0.0)) { status = OG_ERR_NOCONV; break; }
        a = gam / den;
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) p[e] = u[e] + beta * p[e];
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) sv[e] = w[e] + beta * sv[e];
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) x[e] += a * p[e];
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) r[e] -= a * sv[e];
        k++;
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) u[e] = r[e] / d[(e % N) / np];
        og_apply_M(g, alpha, ncomp, u, w);
        gam_old = gam;
        gam = dot(n, r, u);
        del = dot(n, w, u);
        rn = sqrt(dot(n, r, r));
    }
    *iters = k;
    *relres = rn / bnorm;
    free(d); free(r); free(u); free(w); free(p); free(sv);
    return status;
}

/* ---------------------------------------------------------------------------------------------
 * Pole values along a meridian (reading R4, polar rings). Near a pole, the theta and phi
 * components of a smooth vector field, followed along the meridian phi towards the pole, tend
 * to the horizontal field on the axis projected on (cos phi, sin phi) and on (-sin phi, cos phi):
 * pure first harmonics in phi. The value at the pole along the meridian of cell k is therefore
 * taken as the first phi harmonic of the ring of values next to the pole, fitted by the discrete
 * Fourier projection a = (2/np) sum_m f_m cos(phi_m), b = (2/np) sum_m f_m sin(phi_m) over the
 * ring's centres phi_m, and evaluated at phi_k: a cos(phi_k) + b sin(phi_k). The projection
 * removes the ring's harmonics 0 and 2, which carry the field's O(h) change between the ring and
 * the axis, so the pole value is second-order accurate (np >= 3).
 * ------------------------------------------------------------------------------------------- */
static double first_harmonic_at(const og_grid* g, const double* row, int k) {
    double a = 0.0, b = 0.0;
    for (int m = 0; m < g->np; m++) {
        double ph = (m + 0.5) * g->dph;
        a += row[m] * cos(ph);
        b += row[m] * sin(ph);
    }
    double ph = (k + 0.5) * g->dph;
    return (2.0 / g->np) * (a * cos(ph) + b * sin(ph));
}

/* ---------------------------------------------------------------------------------------------
 * Cell-centred B (reading R4): mean of the two opposite faces. In the two polar rings the theta
 * component is the mean of its non-polar face and of its pole value along the cell's meridian:
 * the first harmonic of the B_theta ring on the faces j = 1 (north) or nt-1 (south), divided by
 * cos(dtheta), the factor by which the horizontal part of the theta unit vector shrinks between
 * the axis and that ring (so a uniform field's pole value is exact).
 * ------------------------------------------------------------------------------------------- */
static void bcentre_at(const og_grid* g, const double* br, const double* bt, const double* bp,
                       int i, int j, int k, double* o) {
    int nt = g->nt;
    o[0] = 0.5 * (br[IDX(g, i, j, k)] + br[IDX(g, i + 1, j, k)]);
    if (j == 0 || j == nt - 1) {
        int jf = (j == 0) ? 1 : nt - 1;
        double pole = first_harmonic_at(g, &bt[IDXT(g, i, jf, 0)], k) / cos(g->dth);
        o[1] = 0.5 * (bt[IDXT(g, i, jf, k)] + pole);
    } else {
        o[1] = 0.5 * (bt[IDXT(g, i, j, k)] + bt[IDXT(g, i, j + 1, k)]);
    }
    o[2] = 0.5 * (bp[IDX(g, i, j, k)] + bp[IDX(g, i, j, KP(g, k))]);
}

void og_bcentre(const og_grid* g, const double* br, const double* bt, const double* bp, double* bc) {
    for (int i = 0; i < g->nr; i++)
        for (int j = 0; j < g->nt; j++)
            for (int k = 0; k < g->np; k++) {
                double o[3];
                bcentre_at(g, br, bt, bp, i, j, k, o);
                for (int c = 0; c < 3; c++) bc[c * g->N + IDX(g, i, j, k)] = o[c];
            }
}

/* ---------------------------------------------------------------------------------------------
 * Current density J = curl B (Eq. 1, code units c = 4 pi = 1) on the edges, by Stokes'
 * theorem on the dual face around each edge, whose corners are the surrounding cell centres
 * (reading R4). Polar radial edges use the cap around the pole; the tangential field beyond
 * r0 and r1 is taken equal to the first interior value (ghost centres mirrored in radius).
 * ------------------------------------------------------------------------------------------- */
void og_current_edges(const og_grid* g, const double* br, const double* bt, const double* bp,
                      double* jr, double* jt, double* jp) {
    int nr = g->nr, nt = g->nt, np = g->np;
    double dth = g->dth, dph = g->dph;
    /* radial edges: (i, j, k), j = 0..nt, at (theta_j, phi_k), dual face at rc_i */
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nr; i++) {
        double rc = g->rc[i];
        double circ_n = 0.0, circ_s = 0.0;
        for (int k = 0; k < np; k++) {
            circ_n += bp[IDX(g, i, 0, k)] * rc * g->sc[0] * dph;
            circ_s -= bp[IDX(g, i, nt - 1, k)] * rc * g->sc[nt - 1] * dph;
        }
        double cap_n = rc * rc * (1.0 - g->cc[0]) * 2.0 * M_PI;
        double cap_s = rc * rc * (1.0 + g->cc[nt - 1]) * 2.0 * M_PI;
        for (int k = 0; k < np; k++) {
            jr[IDXT(g, i, 0, k)] = circ_n / cap_n;
            jr[IDXT(g, i, nt, k)] = circ_s / cap_s;
        }
        for (int j = 1; j < nt; j++) {
            double area = rc * rc * (g->cc[j - 1] - g->cc[j]) * dph;
            for (int k = 0; k < np; k++) {
                double c = bp[IDX(g, i, j, k)] * rc * g->sc[j] * dph
                         - bp[IDX(g, i, j - 1, k)] * rc * g->sc[j - 1] * dph
                         - bt[IDXT(g, i, j, k)] * rc * dth
                         + bt[IDXT(g, i, j, KM(g, k))] * rc * dth;
                jr[IDXT(g, i, j, k)] = c / area;
            }
        }
    }
    /* theta edges (i, j, k), i = 0..nr, at (r_i, phi_k); dual face at theta_c_j spanning
     * r_lo..r_hi (cell centres on either side, mirrored ghosts at the boundaries) */
#pragma omp parallel for schedule(static)
    for (int i = 0; i <= nr; i++) {
        double rlo = (i > 0) ? g->rc[i - 1] : 2.0 * g->r0 - g->rc[0];
        double rhi = (i < nr) ? g->rc[i] : 2.0 * g->r[nr] - g->rc[nr - 1];
        int ilo = (i > 0) ? i - 1 : 0;
        int ihi = (i < nr) ? i : nr - 1;
        for (int j = 0; j < nt; j++) {
            double area = g->sc[j] * 0.5 * (rhi * rhi - rlo * rlo) * dph;
            for (int k = 0; k < np; k++) {
                double c = bp[IDX(g, ilo, j, k)] * rlo * g->sc[j] * dph
                         + br[IDX(g, i, j, k)] * (rhi - rlo)
                         - bp[IDX(g, ihi, j, k)] * rhi * g->sc[j] * dph
                         - br[IDX(g, i, j, KM(g, k))] * (rhi - rlo);
                jt[IDX(g, i, j, k)] = c / area;
            }
        }
    }
    /* phi edges (i, j, k), i = 0..nr, j = 0..nt, at (r_i, theta_j); zero on the polar axis */
#pragma omp parallel for schedule(static)
    for (int i = 0; i <= nr; i++) {
        double rlo = (i > 0) ? g->rc[i - 1] : 2.0 * g->r0 - g->rc[0];
        double rhi = (i < nr) ? g->rc[i] : 2.0 * g->r[nr] - g->rc[nr - 1];
        int ilo = (i > 0) ? i - 1 : 0;
        int ihi = (i < nr) ? i : nr - 1;
        double area = 0.5 * (rhi * rhi - rlo * rlo) * dth;
        for (int k = 0; k < np; k++) {
            jp[IDXT(g, i, 0, k)] = 0.0;
            jp[IDXT(g, i, nt, k)] = 0.0;
        }
        for (int j = 1; j < nt; j++)
            for (int k = 0; k < np; k++) {
                double c = br[IDX(g, i, j - 1, k)] * (rhi - rlo)
                         + bt[IDXT(g, ihi, j, k)] * rhi * dth
                         - br[IDX(g, i, j, k)] * (rhi - rlo)
                         - bt[IDXT(g, ilo, j, k)] * rlo * dth;
                jp[IDXT(g, i, j, k)] = c / area;
            }
    }
}

/* J at cell centres: mean of the four edges of each direction around the cell; the polar
 * phi edges (zero length) are left out of the phi average. */
static void current_centre_from_edges(const og_grid* g, const double* jr, const double* jt,
                                      const double* jp, int i, int j, int k, double* o) {
    int nt = g->nt;
    int kp = KP(g, k);
    o[0] = 0.25 * (jr[IDXT(g, i, j, k)] + jr[IDXT(g, i, j, kp)] + jr[IDXT(g, i, j + 1, k)] + jr[IDXT(g, i, j + 1, kp)]);
    o[1] = 0.25 * (jt[IDX(g, i, j, k)] + jt[IDX(g, i, j, kp)] + jt[IDX(g, i + 1, j, k)] + jt[IDX(g, i + 1, j, kp)]);
    if (j == 0) o[2] = 0.5 * (jp[IDXT(g, i, 1, k)] + jp[IDXT(g, i + 1, 1, k)]);
    else if (j == nt - 1) o[2] = 0.5 * (jp[IDXT(g, i, nt - 1, k)] + jp[IDXT(g, i + 1, nt - 1, k)]);
    else o[2] = 0.25 * (jp[IDXT(g, i, j, k)] + jp[IDXT(g, i, j + 1, k)] + jp[IDXT(g, i + 1, j, k)] + jp[IDXT(g, i + 1, j + 1, k)]);
}

typedef struct { double *jr, *jt, *jp; } edges3;

static edges3 edges_alloc(const og_grid* g) {
    edges3 e;
    e.jr = (double*)malloc(sizeof(double) * g->nr * (g->nt + 1) * g->np);
    e.jt = (double*)malloc(sizeof(double) * (g->nr + 1) * g->nt * g->np);
    e.jp = (double*)malloc(sizeof(double) * (g->nr + 1) * (g->nt + 1) * g->np);
    return e;
}
static void edges_free(edges3 e) { free(e.jr); free(e.jt); free(e.jp); }

void og_current_centre(const og_grid* g, const double* br, const double* bt, const double* bp, double* jc) {
    edges3 e = edges_alloc(g);
    og_current_edges(g, br, bt, bp, e.jr, e.jt, e.jp);
    for (int i = 0; i < g->nr; i++)
        for (int j = 0; j < g->nt; j++)
            for (int k = 0; k < g->np; k++) {
                double o[3];
                current_centre_from_edges(g, e.jr, e.jt, e.jp, i, j, k, o);
                for (int c = 0; c < 3; c++) jc[c * g->N + IDX(g, i, j, k)] = o[c];
            }
    edges_free(e);
}

/* ---------------------------------------------------------------------------------------------
 * Explicit momentum force (Eq. 1: -v.grad v + J x B / rho; Sec. 2.2: explicit upwinding).
 * Reading R4: first-order upwind differences per direction, chosen by the sign of the cell's
 * own velocity component, over centre distances; Dirichlet mirror ghost (-u) at r0, zero
 * gradient at r1, no flux from the pole side. Spherical curvature terms of (v.grad)v added.
 * Output b = rho_c V_c dt F.
 * ------------------------------------------------------------------------------------------- */
static double upwind_r(const og_grid* g, const double* u, double vr, int i, int j, int k) {
    double uc = u[IDX(g, i, j, k)];
    if (vr > 0.0) {
        if (i > 0) return (uc - u[IDX(g, i - 1, j, k)]) / (g->rc[i] - g->rc[i - 1]);
        return (uc - (-uc)) / (2.0 * (g->rc[0] - g->r0));
    }
    if (i < g->nr - 1) return (u[IDX(g, i + 1, j, k)] - uc) / (g->rc[i + 1] - g->rc[i]);
    return 0.0;
}
static double upwind_t(const og_grid* g, const double* u, double vt, int i, int j, int k) {
    double uc = u[IDX(g, i, j, k)];
    double h = g->rc[i] * g->dth;
    if (vt > 0.0) {
        if (j > 0) return (uc - u[IDX(g, i, j - 1, k)]) / h;
        return 0.0;
    }
    if (j < g->nt - 1) return (u[IDX(g, i, j + 1, k)] - uc) / h;
    return 0.0;
}
static double upwind_p(const og_grid* g, const double* u, double vp, int i, int j, int k) {
    double uc = u[IDX(g, i, j, k)];
    double h = g->rc[i] * g->sc[j] * g->dph;
    if (vp > 0.0) return (uc - u[IDX(g, i, j, KM(g, k))]) / h;
    return (u[IDX(g, i, j, KP(g, k))] - uc) / h;
}

void og_force(const og_grid* g, const double* v, const double* br, const double* bt,
              const double* bp, double dt, double* b) {
    long long N = g->N;
    int nt = g->nt;
    edges3 e = edges_alloc(g);
    og_current_edges(g, br, bt, bp, e.jr, e.jt, e.jp);
    const double* vr = v;
    const double* vt = v + N;
    const double* vp = v + 2 * N;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < g->nr; i++)
        for (int j = 0; j < nt; j++)
            for (int k = 0; k < g->np; k++) {
                long long c = IDX(g, i, j, k);
                double ur = vr[c], ut = vt[c], up = vp[c];
                double B[3], J[3];
                bcentre_at(g, br, bt, bp, i, j, k, B);
                current_centre_from_edges(g, e.jr, e.jt, e.jp, i, j, k, J);
                double rr = g->rc[i];
                double cot = g->cc[j] / g->sc[j];
                /* (v.grad) of each component */
                double ar = ur * upwind_r(g, vr, ur, i, j, k) + ut * upwind_t(g, vr, ut, i, j, k) + up * upwind_p(g, vr, up, i, j, k);
                double at = ur * upwind_r(g, vt, ur, i, j, k) + ut * upwind_t(g, vt, ut, i, j, k) + up * upwind_p(g, vt, up, i, j, k);
                double ap = ur * upwind_r(g, vp, ur, i, j, k) + ut * upwind_t(g, vp, ut, i, j, k) + up * upwind_p(g, vp, up, i, j, k);
                /* curvature terms of (v.grad)v in spherical components */
                ar += -(ut * ut + up * up) / rr;
                at += (ur * ut - up * up * cot) / rr;
                ap += (ur * up + ut * up * cot) / rr;
                double rho = g->rho[i * nt + j];
                double jxb_r = J[1] * B[2] - J[2] * B[1];
                double jxb_t = J[2] * B[0] - J[0] * B[2];
                double jxb_p = J[0] * B[1] - J[1] * B[0];
                double s = rho * g->vol[i * nt + j] * dt;
                b[c] = s * (-ar + jxb_r / rho);
                b[N + c] = s * (-at + jxb_t / rho);
                b[2 * N + c] = s * (-ap + jxb_p / rho);
            }
    edges_free(e);
}

/* ---------------------------------------------------------------------------------------------
 * Electric field on edges (Eq. 1 in B form: dB/dt = -curl E, E = -v x B + eta J; reading R5).
 * E at cell centres, averaged to each edge over the cells sharing it; the polar radial edge
 * takes the mean of the whole polar ring (k = 0..np-1 in order); tangential E = 0 on r0
 * (line-tied); at r1 the mean of the two interior cells.
 * ------------------------------------------------------------------------------------------- */
void og_efield_edges(const og_grid* g, const double* vbar, const double* br, const double* bt,
                     const double* bp, double eta, double* er, double* et, double* ep) {
    int nr = g->nr, nt = g->nt, np = g->np;
    long long N = g->N;
    double* ec = (double*)malloc(sizeof(double) * 3 * N);
    double* jc = NULL;
    if (eta != 0.0) {
        jc = (double*)malloc(sizeof(double) * 3 * N);
        og_current_centre(g, br, bt, bp, jc);
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nr; i++)
        for (int j = 0; j < nt; j++)
            for (int k = 0; k < np; k++) {
                long long c = IDX(g, i, j, k);
                double B[3];
                bcentre_at(g, br, bt, bp, i, j, k, B);
                double ur = vbar[c], ut = vbar[N + c], up = vbar[2 * N + c];
                double vxb_r = ut * B[2] - up * B[1];
                double vxb_t = up * B[0] - ur * B[2];
                double vxb_p = ur * B[1] - ut * B[0];
                ec[c] = -vxb_r;
                ec[N + c] = -vxb_t;
                ec[2 * N + c] = -vxb_p;
                if (jc) {
                    ec[c] += eta * jc[c];
                    ec[N + c] += eta * jc[N + c];
                    ec[2 * N + c] += eta * jc[2 * N + c];
                }
            }
    const double* Er = ec;
    const double* Et = ec + N;
    const double* Ep = ec + 2 * N;
    /* radial edges */
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nr; i++) {
        double sn = 0.0, ss = 0.0;
        for (int k = 0; k < np; k++) { sn += Er[IDX(g, i, 0, k)]; ss += Er[IDX(g, i, nt - 1, k)]; }
        for (int k = 0; k < np; k++) { er[IDXT(g, i, 0, k)] = sn / np; er[IDXT(g, i, nt, k)] = ss / np; }
        for (int j = 1; j < nt; j++)
            for (int k = 0; k < np; k++) {
                int km = KM(g, k);
                er[IDXT(g, i, j, k)] = 0.25 * (Er[IDX(g, i, j - 1, km)] + Er[IDX(g, i, j - 1, k)] +
                                               Er[IDX(g, i, j, km)] + Er[IDX(g, i, j, k)]);
            }
    }
    /* theta edges */
#pragma omp parallel for schedule(static)
    for (int i = 0; i <= nr; i++)
        for (int j = 0; j < nt; j++)
            for (int k = 0; k < np; k++) {
                int km = KM(g, k);
                double val;
                if (i == 0) val = 0.0;
                else if (i == nr) val = 0.5 * (Et[IDX(g, nr - 1, j, km)] + Et[IDX(g, nr - 1, j, k)]);
                else val = 0.25 * (Et[IDX(g, i - 1, j, km)] + Et[IDX(g, i - 1, j, k)] +
                                   Et[IDX(g, i, j, km)] + Et[IDX(g, i, j, k)]);
                et[IDX(g, i, j, k)] = val;
            }
    /* phi edges */
#pragma omp parallel for schedule(static)
    for (int i = 0; i <= nr; i++)
        for (int j = 0; j <= nt; j++)
            for (int k = 0; k < np; k++) {
                double val;
                if (j == 0 || j == nt || i == 0) val = 0.0;
                else if (i == nr) val = 0.5 * (Ep[IDX(g, nr - 1, j - 1, k)] + Ep[IDX(g, nr - 1, j, k)]);
                else val = 0.25 * (Ep[IDX(g, i - 1, j - 1, k)] + Ep[IDX(g, i - 1, j, k)] +
                                   Ep[IDX(g, i, j - 1, k)] + Ep[IDX(g, i, j, k)]);
                ep[IDXT(g, i, j, k)] = val;
            }
    free(ec);
    free(jc);
}

/* ---------------------------------------------------------------------------------------------
 * Constrained-transport update (reading R5): each face flux changes by -dt times the
 * circulation of E around the face (Stokes), divided by the face area. Polar theta faces have
 * zero area and stay 0.
 * ------------------------------------------------------------------------------------------- */
void og_ct(const og_grid* g, const double* er, const double* et, const double* ep, double dt,
           double* br, double* bt, double* bp) {
    int nr = g->nr, nt = g->nt, np = g->np;
    double dth = g->dth, dph = g->dph;
    /* radial faces (i, j, k), i = 0..nr */
#pragma omp parallel for schedule(static)
    for (int i = 0; i <= nr; i++) {
        double ri = g->r[i];
        double lt = ri * dth;
        for (int j = 0; j < nt; j++) {
            double area = ri * ri * (g->cn[j] - g->cn[j + 1]) * dph;
            double lpj = ri * g->sn[j] * dph, lpj1 = ri * g->sn[j + 1] * dph;
            for (int k = 0; k < np; k++) {
                double c = et[IDX(g, i, j, k)] * lt + ep[IDXT(g, i, j + 1, k)] * lpj1
                         - et[IDX(g, i, j, KP(g, k))] * lt - ep[IDXT(g, i, j, k)] * lpj;
                br[IDX(g, i, j, k)] -= dt * c / area;
            }
        }
    }
    /* theta faces (i, j, k), interior j */
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nr; i++) {
        double ri = g->r[i], ro = g->r[i + 1];
        double lr = ro - ri;
        for (int j = 1; j < nt; j++) {
            double area = g->sn[j] * 0.5 * (ro * ro - ri * ri) * dph;
            double lpi = ri * g->sn[j] * dph, lpo = ro * g->sn[j] * dph;
            for (int k = 0; k < np; k++) {
                double c = ep[IDXT(g, i, j, k)] * lpi + er[IDXT(g, i, j, KP(g, k))] * lr
                         - ep[IDXT(g, i + 1, j, k)] * lpo - er[IDXT(g, i, j, k)] * lr;
                bt[IDXT(g, i, j, k)] -= dt * c / area;
            }
        }
    }
    /* phi faces (i, j, k) */
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nr; i++) {
        double ri = g->r[i], ro = g->r[i + 1];
        double lr = ro - ri;
        double area = 0.5 * (ro * ro - ri * ri) * dth;
        for (int j = 0; j < nt; j++)
            for (int k = 0; k < np; k++) {
                double c = er[IDXT(g, i, j, k)] * lr + et[IDX(g, i + 1, j, k)] * ro * dth
                         - er[IDXT(g, i, j + 1, k)] * lr - et[IDX(g, i, j, k)] * ri * dth;
                bp[IDX(g, i, j, k)] -= dt * c / area;
            }
    }
}

void og_divb(const og_grid* g, const double* br, const double* bt, const double* bp, double* div) {
    int nr = g->nr, nt = g->nt, np = g->np;
    for (int i = 0; i < nr; i++) {
        double ri = g->r[i], ro = g->r[i + 1];
        double ring = 0.5 * (ro * ro - ri * ri);
        for (int j = 0; j < nt; j++) {
            double band = g->cn[j] - g->cn[j + 1];
            double ari = ri * ri * band * g->dph, aro = ro * ro * band * g->dph;
            double atj = g->sn[j] * ring * g->dph, atj1 = g->sn[j + 1] * ring * g->dph;
            double ap = ring * g->dth;
            for (int k = 0; k < np; k++)
                div[IDX(g, i, j, k)] = br[IDX(g, i + 1, j, k)] * aro - br[IDX(g, i, j, k)] * ari
                                     + bt[IDXT(g, i, j + 1, k)] * atj1 - bt[IDXT(g, i, j, k)] * atj
                                     + bp[IDX(g, i, j, KP(g, k))] * ap - bp[IDX(g, i, j, k)] * ap;
        }
    }
}

/* ---------------------------------------------------------------------------------------------
 * Field diagnostics (Sec. 3.1 validates runs by the integrated energies and by |J x B| and
 * |J . B|): out[0] = magnetic energy 1/2 sum_c |B_c|^2 V_c, out[1] = kinetic energy
 * 1/2 sum_c rho_c |v_c|^2 V_c, out[2] = sum_c |J_c x B_c| V_c, out[3] = sum_c |J_c . B_c| V_c,
 * out[4] = max_c |div_h B|_c, the net outward flux of the cell over its volume. B_c and J_c are
 * the cell-centred fields of the momentum force.
 * ------------------------------------------------------------------------------------------- */
void og_diagnostics(const og_grid* g, const double* v, const double* br, const double* bt, const double* bp,
                    double* out) {
    long long N = g->N;
    int nt = g->nt;
    edges3 e = edges_alloc(g);
    og_current_edges(g, br, bt, bp, e.jr, e.jt, e.jp);
    double* div = (double*)malloc(sizeof(double) * N);
    og_divb(g, br, bt, bp, div);
    double em = 0.0, ek = 0.0, jxb = 0.0, jdb = 0.0, dmax = 0.0;
    for (int i = 0; i < g->nr; i++)
        for (int j = 0; j < nt; j++)
            for (int k = 0; k < g->np; k++) {
                long long c = IDX(g, i, j, k);
                double V = g->vol[i * nt + j], rho = g->rho[i * nt + j];
                double B[3], J[3];
                bcentre_at(g, br, bt, bp, i, j, k, B);
                current_centre_from_edges(g, e.jr, e.jt, e.jp, i, j, k, J);
                double u0 = v[c], u1 = v[N + c], u2 = v[2 * N + c];
                double x0 = J[1] * B[2] - J[2] * B[1];
                double x1 = J[2] * B[0] - J[0] * B[2];
                double x2 = J[0] * B[1] - J[1] * B[0];
                em += 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) * V;
                ek += 0.5 * rho * (u0 * u0 + u1 * u1 + u2 * u2) * V;
                jxb += sqrt(x0 * x0 + x1 * x1 + x2 * x2) * V;
                jdb += fabs(J[0] * B[0] + J[1] * B[1] + J[2] * B[2]) * V;
                double dv = fabs(div[c]) / V;
                if (dv > dmax) dmax = dv;
            }
    out[0] = em; out[1] = ek; out[2] = jxb; out[3] = jdb; out[4] = dmax;
    free(div);
    edges_free(e);
}

/* ---------------------------------------------------------------------------------------------
 * Step coefficients (Sec. 2.1: S = (dt^2 k~^2)^-1 (C_w^2/(1-C_f)^2 - 1), k~^2 the upper limit
 * of the combined inverse grid spacing). Reading R3: dt = cfl / max_c k~_c |v_c| (clipped to
 * dt_max, or fixed); C_f = dt max k~|v|, C_w = dt max k~ |B_c| / sqrt(rho_c);
 * alpha_SI = max(C_w^2/(1-C_f)^2 - 1, 0) / max k~^2 (the dt^2 of the printed S cancels against
 * the time discretisation of d v / dt); alpha_nu = nu dt.
 * ------------------------------------------------------------------------------------------- */
int og_coeffs(const og_grid* g, double nu, double cfl, double dt_fixed, double dt_max,
              double asi_fixed, const double* v, const double* br, const double* bt,
              const double* bp, double* out) {
    long long N = g->N;
    int nt = g->nt;
    double mkv = 0.0, mka = 0.0, mk2 = 0.0;
#pragma omp parallel for schedule(static) reduction(max : mkv, mka, mk2)
    for (int i = 0; i < g->nr; i++)
        for (int j = 0; j < nt; j++) {
            double kt2 = g->kt2[i * nt + j];
            double kt = sqrt(kt2);
            if (kt2 > mk2) mk2 = kt2;
            for (int k = 0; k < g->np; k++) {
                long long c = IDX(g, i, j, k);
                double vv = sqrt(v[c] * v[c] + v[N + c] * v[N + c] + v[2 * N + c] * v[2 * N + c]);
                double B[3];
                bcentre_at(g, br, bt, bp, i, j, k, B);
                double bb = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
                double a = kt * vv;
                double w = kt * bb / sqrt(g->rho[i * nt + j]);
                if (a > mkv) mkv = a;
                if (w > mka) mka = w;
            }
        }
    double dt;
    if (dt_fixed > 0.0) dt = dt_fixed;
    else {
        if (mkv > 0.0) dt = cfl / mkv;
        else if (dt_max > 0.0) dt = dt_max;
        else return OG_ERR_ARG;
        if (dt_max > 0.0 && dt > dt_max) dt = dt_max;
    }
    double cf = dt * mkv, cw = dt * mka;
    if (!(cf < 1.0)) return OG_ERR_ARG;
    double X = cw * cw / ((1.0 - cf) * (1.0 - cf)) - 1.0;
    double asi = (X > 0.0) ? X / mk2 : 0.0;
    if (asi_fixed >= 0.0) asi = asi_fixed;
    out[0] = dt; out[1] = cf; out[2] = cw; out[3] = asi; out[4] = nu * dt;
    return OG_OK;
}

/* ---------------------------------------------------------------------------------------------
 * One zero-beta step (Sec. 2.2: explicit predictor-corrector upwinding for the advective and
 * reactive terms; the semi-implicit term inside the predictor-corrector with two PCG solves;
 * viscosity by a third PCG solve). Reading R6:
 *   1. dt, alpha_SI, alpha_nu from (v^n, B^n)
 *   2. predictor: M_SI d_p = rho V dt F(v^n, B^n), x0 = 0; v_p = v^n + d_p
 *   3. B^{n+1} = B^n - dt curl_h E(v_bar, B^n), v_bar = (v^n + v_p)/2
 *   4. corrector: M_SI d_c = rho V dt (F(v^n,B^n) + F(v_p,B^{n+1}))/2, x0 = d_p; v** = v^n + d_c
 *   5. viscosity: M_nu v^{n+1} = rho V v**, x0 = v**
 * ------------------------------------------------------------------------------------------- */
typedef int (*pcg_fn)(const og_grid*, double, int, const double*, double*, double, int, int, int*, double*);

static int pcg_pc2_lines(const og_grid* g, double alpha, int ncomp, const double* b, double* x, double tol,
                         int max_iter, int fixed_iters, int* iters, double* relres) {
    return og_pcg_pc2(g, alpha, 1, ncomp, b, x, tol, max_iter, fixed_iters, iters, relres);
}

/* the step of algorithm 1 with the options of og_step_opts (info: 11 entries, 13 with
 * OG_OPT_RES_IMPLICIT) */
static int step_impl(const og_grid* g, int opts, double nu, double eta, double cfl, double dt_fixed,
                     double dt_max, double asi_fixed, double tol, int max_iter, double* v, double* br,
                     double* bt, double* bp, double* info) {
    pcg_fn pcg = (opts & OG_OPT_PC2) ? pcg_pc2_lines : ((opts & OG_OPT_PCG_CG) ? og_pcg_cg : og_pcg);
    int res_it = 0;
    double res_rr = 0.0;
    long long N = g->N, n3 = 3 * N;
    int nt = g->nt, np = g->np;
    double co[5];
    int st = og_coeffs(g, nu, cfl, dt_fixed, dt_max, asi_fixed, v, br, bt, bp, co);
    if (st != OG_OK) return st;
    double dt = co[0], asi = co[3], anu = co[4];
    double* b0 = (double*)malloc(sizeof(double) * n3);
    double* b1 = (double*)malloc(sizeof(double) * n3);
    double* dlt = (double*)calloc(n3, sizeof(double));
    double* vp = (double*)malloc(sizeof(double) * n3);
    double* vb = (double*)malloc(sizeof(double) * n3);
    edges3 e = edges_alloc(g);
    int it[3] = {0, 0, 0};
    double rr[3] = {0, 0, 0};
    int status = OG_OK, s;

    og_force(g, v, br, bt, bp, dt, b0);
    s = pcg(g, asi, 3, b0, dlt, tol, max_iter, 0, &it[0], &rr[0]);
    if (s != OG_OK) status = s;
#pragma omp parallel for schedule(static)
    for (long long e2 = 0; e2 < n3; e2++) vp[e2] = v[e2] + dlt[e2];
#pragma omp parallel for schedule(static)
    for (long long e2 = 0; e2 < n3; e2++) vb[e2] = 0.5 * (v[e2] + vp[e2]);
    if (opts & OG_OPT_RES_IMPLICIT) {
        /* ideal CT update, then the resistive solve on the faces */
        og_efield_edges(g, vb, br, bt, bp, 0.0, e.jr, e.jt, e.jp);
        og_ct(g, e.jr, e.jt, e.jp, dt, br, bt, bp);
        s = og_res_solve(g, dt * eta, br, bt, bp, tol, max_iter, &res_it, &res_rr);
        if (s != OG_OK) status = s;
    } else {
        og_efield_edges(g, vb, br, bt, bp, eta, e.jr, e.jt, e.jp);
        og_ct(g, e.jr, e.jt, e.jp, dt, br, bt, bp);
    }
    og_force(g, vp, br, bt, bp, dt, b1);
#pragma omp parallel for schedule(static)
    for (long long e2 = 0; e2 < n3; e2++) b1[e2] = 0.5 * (b0[e2] + b1[e2]);
    s = pcg(g, asi, 3, b1, dlt, tol, max_iter, 0, &it[1], &rr[1]);
    if (s != OG_OK) status = s;
#pragma omp parallel for schedule(static)
    for (long long e2 = 0; e2 < n3; e2++) v[e2] = v[e2] + dlt[e2];          /* v** */
    for (int c = 0; c < 3; c++)
#pragma omp parallel for schedule(static)
        for (long long q = 0; q < N; q++) {
            long long ij = q / np;
            b0[c * N + q] = g->rho[ij] * g->vol[ij] * v[c * N + q];
        }
    (void)nt;
    if (opts & OG_OPT_STS) {
        it[2] = og_rkl2(g, nu, dt, 0, v);   /* viscosity by RKL2 from v** (algorithm 3) */
    } else {
        s = pcg(g, anu, 3, b0, v, tol, max_iter, 0, &it[2], &rr[2]);
        if (s != OG_OK) status = s;
    }
    if (info) {
        for (int q = 0; q < 5; q++) info[q] = co[q];
        for (int q = 0; q < 3; q++) { info[5 + q] = it[q]; info[8 + q] = rr[q]; }
        if (opts & OG_OPT_RES_IMPLICIT) { info[11] = res_it; info[12] = res_rr; }
    }
    free(b0); free(b1); free(dlt); free(vp); free(vb);
    edges_free(e);
    return status;
}

int og_step(const og_grid* g, double nu, double eta, double cfl, double dt_fixed, double dt_max,
            double asi_fixed, double tol, int max_iter, double* v, double* br, double* bt,
            double* bp, double* info) {
    return step_impl(g, 0, nu, eta, cfl, dt_fixed, dt_max, asi_fixed, tol, max_iter, v, br, bt, bp, info);
}

/* og_step with every solve in the single-reduction PCG form (og_pcg_cg) */
int og_step_cg(const og_grid* g, double nu, double eta, double cfl, double dt_fixed, double dt_max,
               double asi_fixed, double tol, int max_iter, double* v, double* br, double* bt,
               double* bp, double* info) {
    return step_impl(g, OG_OPT_PCG_CG, nu, eta, cfl, dt_fixed, dt_max, asi_fixed, tol, max_iter, v, br, bt, bp,
                     info);
}

int og_step_opts(const og_grid* g, int opts, double nu, double eta, double cfl, double dt_fixed, double dt_max,
                 double asi_fixed, double tol, int max_iter, double* v, double* br, double* bt, double* bp,
                 double* info) {
    return step_impl(g, opts, nu, eta, cfl, dt_fixed, dt_max, asi_fixed, tol, max_iter, v, br, bt, bp, info);
}

/* =============================================================================================
 * Adjoint of the step (reading P15: dt, alpha_SI, alpha_nu and the upwind directions frozen at
 * the forward values). Every linear piece of the forward step has its transpose written below as
 * a loop over the same stencil that scatters the output cotangent back onto the inputs; the
 * bilinear pieces (v x B, J x B, (v.grad)v) are linearised at the recomputed forward state. The
 * solves use M^-T = M^-1 (M symmetric).
 * =========================================================================================== */

/* transpose of og_ct's map E -> dB = -dt curl_h E: lam_E += -dt (circulation weights) lam_B */
static void ct_T(const og_grid* g, double dt, const double* lbr, const double* lbt, const double* lbp,
                 double* ler, double* let, double* lep) {
    int nr = g->nr, nt = g->nt, np = g->np;
    double dth = g->dth, dph = g->dph;
    for (int i = 0; i <= nr; i++) {
        double ri = g->r[i];
        double lt = ri * dth;
        for (int j = 0; j < nt; j++) {
            double area = ri * ri * (g->cn[j] - g->cn[j + 1]) * dph;
            double lpj = ri * g->sn[j] * dph, lpj1 = ri * g->sn[j + 1] * dph;
            for (int k = 0; k < np; k++) {
                double w = -dt * lbr[IDX(g, i, j, k)] / area;
                let[IDX(g, i, j, k)] += w * lt;
                lep[IDXT(g, i, j + 1, k)] += w * lpj1;
                let[IDX(g, i, j, KP(g, k))] -= w * lt;
                lep[IDXT(g, i, j, k)] -= w * lpj;
            }
        }
    }
    for (int i = 0; i < nr; i++) {
        double ri = g->r[i], ro = g->r[i + 1];
        double lr = ro - ri;
        for (int j = 1; j < nt; j++) {
            double area = g->sn[j] * 0.5 * (ro * ro - ri * ri) * dph;
            double lpi = ri * g->sn[j] * dph, lpo = ro * g->sn[j] * dph;
            for (int k = 0; k < np; k++) {
                double w = -dt * lbt[IDXT(g, i, j, k)] / area;
                lep[IDXT(g, i, j, k)] += w * lpi;
                ler[IDXT(g, i, j, KP(g, k))] += w * lr;
                lep[IDXT(g, i + 1, j, k)] -= w * lpo;
                ler[IDXT(g, i, j, k)] -= w * lr;
            }
        }
    }
    for (int i = 0; i < nr; i++) {
        double ri = g->r[i], ro = g->r[i + 1];
        double lr = ro - ri;
        double area = 0.5 * (ro * ro - ri * ri) * dth;
        for (int j = 0; j < nt; j++)
            for (int k = 0; k < np; k++) {
                double w = -dt * lbp[IDX(g, i, j, k)] / area;
                ler[IDXT(g, i, j, k)] += w * lr;
                let[IDX(g, i + 1, j, k)] += w * ro * dth;
                ler[IDXT(g, i, j + 1, k)] -= w * lr;
                let[IDX(g, i, j, k)] -= w * ri * dth;
            }
    }
}

/* transpose of the centre -> edge averaging of E (og_efield_edges): lam_Ec += weights lam_E */
static void eedges_T(const og_grid* g, const double* ler, const double* let, const double* lep, double* lec) {
    int nr = g->nr, nt = g->nt, np = g->np;
    long long N = g->N;
    double* Er = lec;
    double* Et = lec + N;
    double* Ep = lec + 2 * N;
    for (int i = 0; i < nr; i++) {
        double sn = 0.0, ss = 0.0;
        for (int k = 0; k < np; k++) { sn += ler[IDXT(g, i, 0, k)]; ss += ler[IDXT(g, i, nt, k)]; }
        for (int k = 0; k < np; k++) { Er[IDX(g, i, 0, k)] += sn / np; Er[IDX(g, i, nt - 1, k)] += ss / np; }
        for (int j = 1; j < nt; j++)
            for (int k = 0; k < np; k++) {
                int km = KM(g, k);
                double w = 0.25 * ler[IDXT(g, i, j, k)];
                Er[IDX(g, i, j - 1, km)] += w; Er[IDX(g, i, j - 1, k)] += w;
                Er[IDX(g, i, j, km)] += w; Er[IDX(g, i, j, k)] += w;
            }
    }
    for (int i = 0; i <= nr; i++)
        for (int j = 0; j < nt; j++)
            for (int k = 0; k < np; k++) {
                int km = KM(g, k);
                double l = let[IDX(g, i, j, k)];
                if (i == 0) continue;
                if (i == nr) { Et[IDX(g, nr - 1, j, km)] += 0.5 * l; Et[IDX(g, nr - 1, j, k)] += 0.5 * l; }
                else {
                    Et[IDX(g, i - 1, j, km)] += 0.25 * l; Et[IDX(g, i - 1, j, k)] += 0.25 * l;
                    Et[IDX(g, i, j, km)] += 0.25 * l; Et[IDX(g, i, j, k)] += 0.25 * l;
                }
            }
    for (int i = 0; i <= nr; i++)
        for (int j = 0; j <= nt; j++)
            for (int k = 0; k < np; k++) {
                double l = lep[IDXT(g, i, j, k)];
                if (j == 0 || j == nt || i == 0) continue;
                if (i == nr) { Ep[IDX(g, nr - 1, j - 1, k)] += 0.5 * l; Ep[IDX(g, nr - 1, j, k)] += 0.5 * l; }
                else {
                    Ep[IDX(g, i - 1, j - 1, k)] += 0.25 * l; Ep[IDX(g, i - 1, j, k)] += 0.25 * l;
                    Ep[IDX(g, i, j - 1, k)] += 0.25 * l; Ep[IDX(g, i, j, k)] += 0.25 * l;
                }
            }
}

/* transpose of first_harmonic_at for one output cell k with weight w: the map f -> pole value
 * has the matrix (2/np)(cos phi_k cos phi_m + sin phi_k sin phi_m), so column k is added to row */
static void first_harmonic_T(const og_grid* g, double* row, int k, double w) {
    double phk = (k + 0.5) * g->dph;
    for (int m = 0; m < g->np; m++) {
        double ph = (m + 0.5) * g->dph;
        row[m] += w * (2.0 / g->np) * (cos(ph) * cos(phk) + sin(ph) * sin(phk));
    }
}

/* transpose of the face -> centre averaging of B (bcentre_at) */
static void bcentre_T(const og_grid* g, const double* lbc, double* lbr, double* lbt, double* lbp) {
    int nt = g->nt;
    long long N = g->N;
    for (int i = 0; i < g->nr; i++)
        for (int j = 0; j < nt; j++)
            for (int k = 0; k < g->np; k++) {
                long long c = IDX(g, i, j, k);
                lbr[IDX(g, i, j, k)] += 0.5 * lbc[c];
                lbr[IDX(g, i + 1, j, k)] += 0.5 * lbc[c];
                if (j == 0 || j == nt - 1) {
                    int jf = (j == 0) ? 1 : nt - 1;
                    lbt[IDXT(g, i, jf, k)] += 0.5 * lbc[N + c];
                    first_harmonic_T(g, &lbt[IDXT(g, i, jf, 0)], k, 0.5 * lbc[N + c] / cos(g->dth));
                } else {
                    lbt[IDXT(g, i, j, k)] += 0.5 * lbc[N + c];
                    lbt[IDXT(g, i, j + 1, k)] += 0.5 * lbc[N + c];
                }
                lbp[IDX(g, i, j, k)] += 0.5 * lbc[2 * N + c];
                lbp[IDX(g, i, j, KP(g, k))] += 0.5 * lbc[2 * N + c];
            }
}

/* transpose of the edge -> centre averaging of J (current_centre_from_edges) */
static void jcentre_T(const og_grid* g, const double* ljc, double* ljr, double* ljt, double* ljp) {
    int nt = g->nt;
    long long N = g->N;
    for (int i = 0; i < g->nr; i++)
        for (int j = 0; j < nt; j++)
            for (int k = 0; k < g->np; k++) {
                long long c = IDX(g, i, j, k);
                int kp = KP(g, k);
                double a = 0.25 * ljc[c], b = 0.25 * ljc[N + c], e = ljc[2 * N + c];
                ljr[IDXT(g, i, j, k)] += a; ljr[IDXT(g, i, j, kp)] += a;
                ljr[IDXT(g, i, j + 1, k)] += a; ljr[IDXT(g, i, j + 1, kp)] += a;
                ljt[IDX(g, i, j, k)] += b; ljt[IDX(g, i, j, kp)] += b;
                ljt[IDX(g, i + 1, j, k)] += b; ljt[IDX(g, i + 1, j, kp)] += b;
                if (j == 0) { ljp[IDXT(g, i, 1, k)] += 0.5 * e; ljp[IDXT(g, i + 1, 1, k)] += 0.5 * e; }
                else if (j == nt - 1) { ljp[IDXT(g, i, nt - 1, k)] += 0.5 * e; ljp[IDXT(g, i + 1, nt - 1, k)] += 0.5 * e; }
                else {
                    ljp[IDXT(g, i, j, k)] += 0.25 * e; ljp[IDXT(g, i, j + 1, k)] += 0.25 * e;
                    ljp[IDXT(g, i + 1, j, k)] += 0.25 * e; ljp[IDXT(g, i + 1, j + 1, k)] += 0.25 * e;
                }
            }
}

/* transpose of og_current_edges (B faces -> J edges) */
static void curlJ_T(const og_grid* g, const double* ljr, const double* ljt, const double* ljp, double* lbr,
                    double* lbt, double* lbp) {
    int nr = g->nr, nt = g->nt, np = g->np;
    double dth = g->dth, dph = g->dph;
    for (int i = 0; i < nr; i++) {
        double rc = g->rc[i];
        double cap_n = rc * rc * (1.0 - g->cc[0]) * 2.0 * M_PI;
        double cap_s = rc * rc * (1.0 + g->cc[nt - 1]) * 2.0 * M_PI;
        double sn = 0.0, ss = 0.0;
        for (int k = 0; k < np; k++) { sn += ljr[IDXT(g, i, 0, k)]; ss += ljr[IDXT(g, i, nt, k)]; }
        for (int k = 0; k < np; k++) {
            lbp[IDX(g, i, 0, k)] += sn / cap_n * (rc * g->sc[0] * dph);
            lbp[IDX(g, i, nt - 1, k)] -= ss / cap_s * (rc * g->sc[nt - 1] * dph);
        }
        for (int j = 1; j < nt; j++) {
            double area = rc * rc * (g->cc[j - 1] - g->cc[j]) * dph;
            for (int k = 0; k < np; k++) {
                double w = ljr[IDXT(g, i, j, k)] / area;
                lbp[IDX(g, i, j, k)] += w * rc * g->sc[j] * dph;
                lbp[IDX(g, i, j - 1, k)] -= w * rc * g->sc[j - 1] * dph;
                lbt[IDXT(g, i, j, k)] -= w * rc * dth;
                lbt[IDXT(g, i, j, KM(g, k))] += w * rc * dth;
            }
        }
    }
    for (int i = 0; i <= nr; i++) {
        double rlo = (i > 0) ? g->rc[i - 1] : 2.0 * g->r0 - g->rc[0];
        double rhi = (i < nr) ? g->rc[i] : 2.0 * g->r[nr] - g->rc[nr - 1];
        int ilo = (i > 0) ? i - 1 : 0;
        int ihi = (i < nr) ? i : nr - 1;
        for (int j = 0; j < nt; j++) {
            double area = g->sc[j] * 0.5 * (rhi * rhi - rlo * rlo) * dph;
            for (int k = 0; k < np; k++) {
                double w = ljt[IDX(g, i, j, k)] / area;
                lbp[IDX(g, ilo, j, k)] += w * rlo * g->sc[j] * dph;
                lbr[IDX(g, i, j, k)] += w * (rhi - rlo);
                lbp[IDX(g, ihi, j, k)] -= w * rhi * g->sc[j] * dph;
                lbr[IDX(g, i, j, KM(g, k))] -= w * (rhi - rlo);
            }
        }
        double area = 0.5 * (rhi * rhi - rlo * rlo) * dth;
        for (int j = 1; j < nt; j++)
            for (int k = 0; k < np; k++) {
                double w = ljp[IDXT(g, i, j, k)] / area;
                lbr[IDX(g, i, j - 1, k)] += w * (rhi - rlo);
                lbt[IDXT(g, ihi, j, k)] += w * rhi * dth;
                lbr[IDX(g, i, j, k)] -= w * (rhi - rlo);
                lbt[IDXT(g, ilo, j, k)] -= w * rlo * dth;
            }
    }
}

/* lam_B += (J-dependence of) the adjoint of a cell-centred J cotangent */
static void jc_cotangent_to_faces(const og_grid* g, const double* ljc, double* lbr, double* lbt, double* lbp) {
    edges3 e = edges_alloc(g);
    memset(e.jr, 0, sizeof(double) * g->nr * (g->nt + 1) * g->np);
    memset(e.jt, 0, sizeof(double) * (g->nr + 1) * g->nt * g->np);
    memset(e.jp, 0, sizeof(double) * (g->nr + 1) * (g->nt + 1) * g->np);
    jcentre_T(g, ljc, e.jr, e.jt, e.jp);
    curlJ_T(g, e.jr, e.jt, e.jp, lbr, lbt, lbp);
    edges_free(e);
}

/* transpose of one upwind difference D_d u at cell (i,j,k) with the frozen direction: scatter
 * w * (coefficients) onto lu */
static void upwind_T(const og_grid* g, int dir, double vdir, double w, int i, int j, int k, double* lu) {
    long long c = IDX(g, i, j, k);
    if (dir == 0) {
        if (vdir > 0.0) {
            if (i > 0) { double h = g->rc[i] - g->rc[i - 1]; lu[c] += w / h; lu[IDX(g, i - 1, j, k)] -= w / h; }
            else { double h = 2.0 * (g->rc[0] - g->r0); lu[c] += 2.0 * w / h; }
        } else if (i < g->nr - 1) {
            double h = g->rc[i + 1] - g->rc[i];
            lu[IDX(g, i + 1, j, k)] += w / h; lu[c] -= w / h;
        }
    } else if (dir == 1) {
        double h = g->rc[i] * g->dth;
        if (vdir > 0.0) { if (j > 0) { lu[c] += w / h; lu[IDX(g, i, j - 1, k)] -= w / h; } }
        else if (j < g->nt - 1) { lu[IDX(g, i, j + 1, k)] += w / h; lu[c] -= w / h; }
    } else {
        double h = g->rc[i] * g->sc[j] * g->dph;
        if (vdir > 0.0) { lu[c] += w / h; lu[IDX(g, i, j, KM(g, k))] -= w / h; }
        else { lu[IDX(g, i, j, KP(g, k))] += w / h; lu[c] -= w / h; }
    }
}

/* adjoint of b = rho V dt F(v, B) at the base (v, B): lam_v += (dF/dv)^T (s lam_b),
 * lam_B += (dF/dB)^T (s lam_b) */
static void force_T(const og_grid* g, const double* v, const double* br, const double* bt, const double* bp,
                    double dt, const double* lb, double* lv, double* lbr, double* lbt, double* lbp) {
    long long N = g->N;
    int nt = g->nt;
    double* jc = (double*)malloc(sizeof(double) * 3 * N);
    double* ljc = (double*)calloc(3 * N, sizeof(double));
    double* lbc = (double*)calloc(3 * N, sizeof(double));
    og_current_centre(g, br, bt, bp, jc);
    const double* vv[3] = {v, v + N, v + 2 * N};
    for (int i = 0; i < g->nr; i++)
        for (int j = 0; j < nt; j++)
            for (int k = 0; k < g->np; k++) {
                long long c = IDX(g, i, j, k);
                double s = g->rho[i * nt + j] * g->vol[i * nt + j] * dt;
                double rho = g->rho[i * nt + j];
                double lf[3] = {s * lb[c], s * lb[N + c], s * lb[2 * N + c]};
                double B[3], J[3] = {jc[c], jc[N + c], jc[2 * N + c]};
                bcentre_at(g, br, bt, bp, i, j, k, B);
                /* Lorentz term (J x B)/rho */
                ljc[c] += (B[1] * lf[2] - B[2] * lf[1]) / rho;
                ljc[N + c] += (B[2] * lf[0] - B[0] * lf[2]) / rho;
                ljc[2 * N + c] += (B[0] * lf[1] - B[1] * lf[0]) / rho;
                lbc[c] += (lf[1] * J[2] - lf[2] * J[1]) / rho;
                lbc[N + c] += (lf[2] * J[0] - lf[0] * J[2]) / rho;
                lbc[2 * N + c] += (lf[0] * J[1] - lf[1] * J[0]) / rho;
                /* advection: adv_m = sum_d u_d D_d(v_m) + curv_m; F = -adv */
                double u[3] = {vv[0][c], vv[1][c], vv[2][c]};
                double mu[3] = {-lf[0], -lf[1], -lf[2]};
                for (int m = 0; m < 3; m++) {
                    double D[3] = {upwind_r(g, vv[m], u[0], i, j, k), upwind_t(g, vv[m], u[1], i, j, k),
                                   upwind_p(g, vv[m], u[2], i, j, k)};
                    for (int d = 0; d < 3; d++) {
                        lv[d * N + c] += mu[m] * D[d];
                        upwind_T(g, d, u[d], u[d] * mu[m], i, j, k, lv + m * N);
                    }
                }
                double r = g->rc[i], cot = g->cc[j] / g->sc[j];
                /* curvature Jacobian rows: r: -(ut^2+up^2)/r; t: (ur ut - up^2 cot)/r; p: (ur up + ut up cot)/r */
                lv[N + c] += mu[0] * (-2.0 * u[1] / r);
                lv[2 * N + c] += mu[0] * (-2.0 * u[2] / r);
                lv[c] += mu[1] * (u[1] / r);
                lv[N + c] += mu[1] * (u[0] / r);
                lv[2 * N + c] += mu[1] * (-2.0 * u[2] * cot / r);
                lv[c] += mu[2] * (u[2] / r);
                lv[N + c] += mu[2] * (u[2] * cot / r);
                lv[2 * N + c] += mu[2] * ((u[0] + u[1] * cot) / r);
            }
    bcentre_T(g, lbc, lbr, lbt, lbp);
    jc_cotangent_to_faces(g, ljc, lbr, lbt, lbp);
    free(jc); free(ljc); free(lbc);
}

/* adjoint of E edges(vbar, B) given lam_E on edges: lam_vbar += ..., lam_B += ... */
static void efield_T(const og_grid* g, const double* vb, const double* br, const double* bt, const double* bp,
                     double eta, const double* ler, const double* let, const double* lep, double* lvb,
                     double* lbr, double* lbt, double* lbp) {
    long long N = g->N;
    double* lec = (double*)calloc(3 * N, sizeof(double));
    double* lbc = (double*)calloc(3 * N, sizeof(double));
    eedges_T(g, ler, let, lep, lec);
    for (int i = 0; i < g->nr; i++)
        for (int j = 0; j < g->nt; j++)
            for (int k = 0; k < g->np; k++) {
                long long c = IDX(g, i, j, k);
                double B[3], u[3] = {vb[c], vb[N + c], vb[2 * N + c]};
                double l[3] = {lec[c], lec[N + c], lec[2 * N + c]};
                bcentre_at(g, br, bt, bp, i, j, k, B);
                /* E_c = -u x B: lam_u = l x B, lam_B = u x l */
                lvb[c] += l[1] * B[2] - l[2] * B[1];
                lvb[N + c] += l[2] * B[0] - l[0] * B[2];
                lvb[2 * N + c] += l[0] * B[1] - l[1] * B[0];
                lbc[c] += u[1] * l[2] - u[2] * l[1];
                lbc[N + c] += u[2] * l[0] - u[0] * l[2];
                lbc[2 * N + c] += u[0] * l[1] - u[1] * l[0];
            }
    bcentre_T(g, lbc, lbr, lbt, lbp);
    if (eta != 0.0) {
        for (long long q = 0; q < 3 * N; q++) lec[q] *= eta;
        jc_cotangent_to_faces(g, lec, lbr, lbt, lbp);
    }
    free(lec); free(lbc);
}

static int adjoint_step(const og_grid* g, double nu, double eta, double cfl, double dt, double asi_fixed,
                        double tol, int max_iter, int opts, const double* v0, const double* br0, const double* bt0,
                        const double* bp0, const double* lv1, const double* lbr1, const double* lbt1,
                        const double* lbp1, double* lv, double* lbr, double* lbt, double* lbp) {
    long long N = g->N, n3 = 3 * N;
    int np = g->np;
    long long nbr = (long long)(g->nr + 1) * g->nt * np, nbt = (long long)g->nr * (g->nt + 1) * np, nbp = N;
    long long ner = (long long)g->nr * (g->nt + 1) * np, net = (long long)(g->nr + 1) * g->nt * np,
              nep = (long long)(g->nr + 1) * (g->nt + 1) * np;
    double co[5];
    int st = og_coeffs(g, nu, cfl, dt, 0.0, asi_fixed, v0, br0, bt0, bp0, co);
    if (st != OG_OK) return st;
    double asi = co[3], anu = co[4];
    int it, status = OG_OK, s;
    double rr;
    /* ---- forward recomputation */
    double* b0 = (double*)malloc(sizeof(double) * n3);
    double* b1 = (double*)malloc(sizeof(double) * n3);
    double* dp = (double*)calloc(n3, sizeof(double));
    double* vp = (double*)malloc(sizeof(double) * n3);
    double* vb = (double*)malloc(sizeof(double) * n3);
    double* B1r = (double*)malloc(sizeof(double) * nbr);
    double* B1t = (double*)malloc(sizeof(double) * nbt);
    double* B1p = (double*)malloc(sizeof(double) * nbp);
    edges3 e = edges_alloc(g);
    og_force(g, v0, br0, bt0, bp0, dt, b0);
    s = og_pcg(g, asi, 3, b0, dp, tol, max_iter, 0, &it, &rr);
    if (s != OG_OK) status = s;
    for (long long q = 0; q < n3; q++) { vp[q] = v0[q] + dp[q]; vb[q] = 0.5 * (v0[q] + vp[q]); }
    memcpy(B1r, br0, sizeof(double) * nbr); memcpy(B1t, bt0, sizeof(double) * nbt); memcpy(B1p, bp0, sizeof(double) * nbp);
    const int res = (opts & OG_OPT_RES_IMPLICIT) != 0;
    const double eta_e = res ? 0.0 : eta;   /* resistivity in E (explicit) or in the face solve */
    og_efield_edges(g, vb, br0, bt0, bp0, eta_e, e.jr, e.jt, e.jp);
    og_ct(g, e.jr, e.jt, e.jp, dt, B1r, B1t, B1p);
    if (res) {
        int rit;
        double rrr;
        s = og_res_solve(g, dt * eta, B1r, B1t, B1p, tol, max_iter, &rit, &rrr);
        if (s != OG_OK) status = s;
    }
    /* ---- reverse */
    double* y = (double*)calloc(n3, sizeof(double));
    double* lb = (double*)calloc(n3, sizeof(double));
    double* ldp = (double*)calloc(n3, sizeof(double));
    double* lvp = (double*)calloc(n3, sizeof(double));
    double* lvb = (double*)calloc(n3, sizeof(double));
    double* lB1r = (double*)malloc(sizeof(double) * nbr);
    double* lB1t = (double*)malloc(sizeof(double) * nbt);
    double* lB1p = (double*)malloc(sizeof(double) * nbp);
    memset(lv, 0, sizeof(double) * n3);
    memset(lbr, 0, sizeof(double) * nbr); memset(lbt, 0, sizeof(double) * nbt); memset(lbp, 0, sizeof(double) * nbp);
    memcpy(lB1r, lbr1, sizeof(double) * nbr); memcpy(lB1t, lbt1, sizeof(double) * nbt); memcpy(lB1p, lbp1, sizeof(double) * nbp);
    if (opts & OG_OPT_STS) {
        /* 5. v' = P v** with P the RKL2 polynomial in dt L, L = -nu D^-1 K; K symmetric gives
         * P^T = D P D^-1, so lam_v** = D P (D^-1 lam_v') (the D factor is applied below) */
        for (int c = 0; c < 3; c++)
            for (long long q = 0; q < N; q++) {
                long long ij = q / np;
                y[c * N + q] = lv1[c * N + q] / (g->rho[ij] * g->vol[ij]);
            }
        og_rkl2(g, nu, dt, 0, y);
    } else {
        /* 5. v' = M_nu^-1 D v**  ->  lam_v** = D M_nu^-1 lam_v' */
        s = og_pcg(g, anu, 3, lv1, y, tol, max_iter, 0, &it, &rr);
        if (s != OG_OK) status = s;
    }
    for (int c = 0; c < 3; c++)
        for (long long q = 0; q < N; q++) {
            long long ij = q / np;
            double w = g->rho[ij] * g->vol[ij] * y[c * N + q];
            lv[c * N + q] += w;      /* v** = v + d_c */
            y[c * N + q] = w;        /* lam_dc */
        }
    /* 4. d_c = M_SI^-1 (b0 + b1)/2 */
    memset(lb, 0, sizeof(double) * n3);
    s = og_pcg(g, asi, 3, y, lb, tol, max_iter, 0, &it, &rr);   /* lb = M_SI^-1 lam_dc = lam_bc */
    if (s != OG_OK) status = s;
    for (long long q = 0; q < n3; q++) { lb[q] *= 0.5; }            /* lam_b0 (partial) = lam_b1 = lam_bc/2 */
    /* b1 = F(vp, B1): lam_vp, lam_B1 */
    force_T(g, vp, B1r, B1t, B1p, dt, lb, lvp, lB1r, lB1t, lB1p);
    if (res) {
        /* 3b. B1 = R B*, R = M_res^-1 W for the exact face solve (W (x + dte curl_h J x) = W B*
         * gives B* - dte curl_h J x = x), so lam_B* = W M_res^-1 lam_B1 (M_res symmetric) */
        long long nf = og_res_size(g);
        double* lb1 = (double*)malloc(sizeof(double) * nf);
        double* yr = (double*)calloc(nf, sizeof(double));
        double* wv = (double*)malloc(sizeof(double) * nf);
        memcpy(lb1, lB1r, sizeof(double) * nbr);
        memcpy(lb1 + nbr, lB1t, sizeof(double) * nbt);
        memcpy(lb1 + nbr + nbt, lB1p, sizeof(double) * nbp);
        int rit;
        double rrr;
        s = og_res_pcg(g, dt * eta, lb1, yr, tol, max_iter, 0, &rit, &rrr);
        if (s != OG_OK) status = s;
        res_weights(g, wv);
        for (long long q = 0; q < nf; q++) yr[q] *= wv[q];
        memcpy(lB1r, yr, sizeof(double) * nbr);
        memcpy(lB1t, yr + nbr, sizeof(double) * nbt);
        memcpy(lB1p, yr + nbr + nbt, sizeof(double) * nbp);
        free(lb1); free(yr); free(wv);
    }
    /* 3. B* = B - dt curl E(vb, B) (B1 itself without the face solve): lam_B += lam_B*;
     * lam_E = -dt C^T lam_B* */
    for (long long q = 0; q < nbr; q++) lbr[q] += lB1r[q];
    for (long long q = 0; q < nbt; q++) lbt[q] += lB1t[q];
    for (long long q = 0; q < nbp; q++) lbp[q] += lB1p[q];
    memset(e.jr, 0, sizeof(double) * ner); memset(e.jt, 0, sizeof(double) * net); memset(e.jp, 0, sizeof(double) * nep);
    ct_T(g, dt, lB1r, lB1t, lB1p, e.jr, e.jt, e.jp);
    efield_T(g, vb, br0, bt0, bp0, eta_e, e.jr, e.jt, e.jp, lvb, lbr, lbt, lbp);
    /* vp = v + dp, vb = v + dp/2 */
    for (long long q = 0; q < n3; q++) {
        lv[q] += lvp[q] + lvb[q];
        ldp[q] = lvp[q] + 0.5 * lvb[q];
    }
    /* 2. dp = M_SI^-1 b0: lam_b0 += M_SI^-1 lam_dp */
    memset(y, 0, sizeof(double) * n3);
    s = og_pcg(g, asi, 3, ldp, y, tol, max_iter, 0, &it, &rr);
    if (s != OG_OK) status = s;
    for (long long q = 0; q < n3; q++) lb[q] += y[q];
    /* b0 = F(v, B) */
    force_T(g, v0, br0, bt0, bp0, dt, lb, lv, lbr, lbt, lbp);
    free(b0); free(b1); free(dp); free(vp); free(vb); free(B1r); free(B1t); free(B1p);
    free(y); free(lb); free(ldp); free(lvp); free(lvb); free(lB1r); free(lB1t); free(lB1p);
    edges_free(e);
    return status;
}

/* =============================================================================================
 * Viscosity by RKL2 super time-stepping (Sec. 2.2: the STS option for the viscous term, the
 * paper's GPU choice in algorithm 3; the method is the second-order Runge-Kutta-Legendre scheme of
 * Meyer, Balsara & Aslam 2014). It integrates rho V dv/dt = -nu K v over dt explicitly with s
 * stages:
 *   b_j = (j^2 + j - 2) / (2 j (j + 1)) for j >= 2, b_0 = b_1 = 1/3, a_j = 1 - b_j,
 *   w1 = 4 / (s^2 + s - 2),
 *   Y_1 = Y_0 + (b_1 w1) dt L(Y_0)
 *   Y_j = mu_j Y_{j-1} + nv_j Y_{j-2} + (1 - mu_j - nv_j) Y_0 + mu_j w1 dt L(Y_{j-1})
 *         - a_{j-1} mu_j w1 dt L(Y_0),   j = 2..s,
 *   with mu_j = (2j - 1)/j b_j/b_{j-1}, nv_j = -(j - 1)/j b_j/b_{j-2}, L(v) = -nu D^-1 K v.
 * The stage count is the smallest s >= 2 with (s^2 + s - 2)/2 >= dt lambda_max, lambda_max
 * bounded above by Gershgorin: nu max_c (2 sum_f w_f + w_Dirichlet) / (rho_c V_c).
 * =========================================================================================== */
static double rkl2_b(int j) { return (j < 2) ? 1.0 / 3.0 : (double)(j * j + j - 2) / (2.0 * j * (j + 1)); }

int og_rkl2_stages(const og_grid* g, double nu, double dt) {
    int nr = g->nr, nt = g->nt;
    double lam = 0.0;
    for (int i = 0; i < nr; i++)
        for (int j = 0; j < nt; j++) {
            double s = g->wr[i * nt + j] + g->wr[(i + 1) * nt + j] + g->wt[i * (nt + 1) + j] +
                       g->wt[i * (nt + 1) + j + 1] + 2.0 * g->wp[i * nt + j];
            double off = s - (i == 0 ? g->wr[j] : 0.0);  /* the Dirichlet weight has no partner */
            double l = nu * (s + off) / (g->rho[i * nt + j] * g->vol[i * nt + j]);
            if (l > lam) lam = l;
        }
    int s = 2;
    while ((double)(s * s + s - 2) / 2.0 < dt * lam) s++;
    return s;
}

/* v (3N) advanced in place by s RKL2 stages over dt; s <= 0 picks the stage count */
int og_rkl2(const og_grid* g, double nu, double dt, int s, double* v) {
    long long N = g->N, n3 = 3 * N;
    int np = g->np;
    if (s <= 0) s = og_rkl2_stages(g, nu, dt);
    double w1 = 4.0 / (double)(s * s + s - 2);
    double* y0 = (double*)malloc(sizeof(double) * n3);
    double* ly0 = (double*)malloc(sizeof(double) * n3);
    double* ym1 = (double*)malloc(sizeof(double) * n3);
    double* ym2 = (double*)malloc(sizeof(double) * n3);
    double* yj = (double*)malloc(sizeof(double) * n3);
    double* lk = (double*)malloc(sizeof(double) * n3);
    memcpy(y0, v, sizeof(double) * n3);
    /* L(Y) = -nu D^-1 K Y, K with its Dirichlet term, D = rho V */
    apply_op(g, 1.0, 0, 1, 3, y0, lk);
    for (long long q = 0; q < n3; q++) {
        long long ij = (q % N) / np;
        ly0[q] = -nu * lk[q] / (g->rho[ij] * g->vol[ij]);
    }
    for (long long q = 0; q < n3; q++) { ym2[q] = y0[q]; ym1[q] = y0[q] + rkl2_b(1) * w1 * dt * ly0[q]; }
    for (int j = 2; j <= s; j++) {
        double bj = rkl2_b(j), bj1 = rkl2_b(j - 1), bj2 = rkl2_b(j - 2);
        double mu = (2.0 * j - 1.0) / j * bj / bj1;
        double nv = -(j - 1.0) / j * bj / bj2;
        double mut = mu * w1;
        double gat = -(1.0 - bj1) * mut;
        apply_op(g, 1.0, 0, 1, 3, ym1, lk);
        for (long long q = 0; q < n3; q++) {
            long long ij = (q % N) / np;
            double l = -nu * lk[q] / (g->rho[ij] * g->vol[ij]);
            yj[q] = mu * ym1[q] + nv * ym2[q] + (1.0 - mu - nv) * y0[q] + mut * dt * l + gat * dt * ly0[q];
        }
        double* t = ym2; ym2 = ym1; ym1 = yj; yj = t;
    }
    memcpy(v, ym1, sizeof(double) * n3);
    free(y0); free(ly0); free(ym1); free(ym2); free(yj); free(lk);
    return s;
}

/* og_step with viscosity by RKL2 (algorithm 3 of the paper: SI by PCG, viscosity by STS);
 * info[7] holds the stage count */
int og_step_sts(const og_grid* g, double nu, double eta, double cfl, double dt_fixed, double dt_max,
                double asi_fixed, double tol, int max_iter, double* v, double* br, double* bt, double* bp,
                double* info) {
    return step_impl(g, OG_OPT_STS, nu, eta, cfl, dt_fixed, dt_max, asi_fixed, tol, max_iter, v, br, bt, bp, info);
}

int og_adjoint_step(const og_grid* g, double nu, double eta, double cfl, double dt, double asi_fixed, double tol,
                    int max_iter, const double* v0, const double* br0, const double* bt0, const double* bp0,
                    const double* lv1, const double* lbr1, const double* lbt1, const double* lbp1, double* lv,
                    double* lbr, double* lbt, double* lbp) {
    return adjoint_step(g, nu, eta, cfl, dt, asi_fixed, tol, max_iter, 0, v0, br0, bt0, bp0, lv1, lbr1, lbt1, lbp1,
                        lv, lbr, lbt, lbp);
}

/* adjoint of og_step_sts (same frozen map: dt, alpha_SI, the stage count, upwind directions) */
int og_adjoint_step_sts(const og_grid* g, double nu, double eta, double cfl, double dt, double asi_fixed,
                        double tol, int max_iter, const double* v0, const double* br0, const double* bt0,
                        const double* bp0, const double* lv1, const double* lbr1, const double* lbt1,
                        const double* lbp1, double* lv, double* lbr, double* lbt, double* lbp) {
    return adjoint_step(g, nu, eta, cfl, dt, asi_fixed, tol, max_iter, OG_OPT_STS, v0, br0, bt0, bp0, lv1, lbr1,
                        lbt1, lbp1, lv, lbr, lbt, lbp);
}

/* adjoint of og_step_opts with OG_OPT_STS and / or OG_OPT_RES_IMPLICIT (the other options do not
 * change the map) */
int og_adjoint_step_opts(const og_grid* g, int opts, double nu, double eta, double cfl, double dt, double asi_fixed,
                         double tol, int max_iter, const double* v0, const double* br0, const double* bt0,
                         const double* bp0, const double* lv1, const double* lbr1, const double* lbt1,
                         const double* lbp1, double* lv, double* lbr, double* lbt, double* lbp) {
    return adjoint_step(g, nu, eta, cfl, dt, asi_fixed, tol, max_iter, opts, v0, br0, bt0, bp0, lv1, lbr1, lbt1,
                        lbp1, lv, lbr, lbt, lbp);
}

/* =============================================================================================
 * Implicit resistivity (Eq. 1: the -eta curl curl A term; Sec. 2.2: diffusive terms by PCG,
 * the resistive solve always well conditioned and always with PC1). Reading R8, in B form:
 * after the ideal CT update B* = B^n - dt curl_h E(v_bar, B^n) with eta = 0, solve
 *     B^{n+1} + dt eta curl_h J(B^{n+1}) = B*,
 * curl_h the face circulation of og_ct and J_e = (1/A*_e) sum_f s_fe l*_f B_f the circulation of
 * B around the dual face of edge e (og_current_edges on interior edges): s_fe is the sign that
 * og_ct gives edge e in face f and l*_f the centre-to-centre distance across f. Tangential edges
 * on r0 and r1 carry no resistive E (line-tied inner wall; no resistive flux through the outer
 * one), so every dual loop in the system is complete and B_r on both walls is unchanged. With
 * the face weights W_f = A_f l*_f the system
 *     W (B + dte curl_h J(B)) = W B*,   dte = dt eta,
 * is W + dte G^T diag(l_e / A*_e) G with G_ef = s_fe l*_f: symmetric positive definite. The
 * unknown is the stacked face vector [br | bt | bp]; the polar theta faces (zero area, stored
 * 0) are identity rows.
 * =========================================================================================== */
static double lstar_r(const og_grid* g, int i) {
    if (i == 0) return g->rc[0] - g->r0;
    if (i == g->nr) return g->r[g->nr] - g->rc[g->nr - 1];
    return g->rc[i] - g->rc[i - 1];
}

long long og_res_size(const og_grid* g) {
    return (long long)(g->nr + 1) * g->nt * g->np + (long long)g->nr * (g->nt + 1) * g->np + g->N;
}

/* W_f per face, stacked */
static void res_weights(const og_grid* g, double* w) {
    int nr = g->nr, nt = g->nt, np = g->np;
    double dth = g->dth, dph = g->dph;
    double* wr = w;
    double* wt = w + (long long)(nr + 1) * nt * np;
    double* wp = wt + (long long)nr * (nt + 1) * np;
    for (int i = 0; i <= nr; i++)
        for (int j = 0; j < nt; j++) {
            double a = g->r[i] * g->r[i] * (g->cn[j] - g->cn[j + 1]) * dph;
            for (int k = 0; k < np; k++) wr[IDX(g, i, j, k)] = a * lstar_r(g, i);
        }
    for (int i = 0; i < nr; i++)
        for (int j = 0; j <= nt; j++) {
            double a = g->sn[j] * 0.5 * (g->r[i + 1] * g->r[i + 1] - g->r[i] * g->r[i]) * dph;
            double wv = (j == 0 || j == nt) ? 1.0 : a * g->rc[i] * dth;
            for (int k = 0; k < np; k++) wt[IDXT(g, i, j, k)] = wv;
        }
    for (int i = 0; i < nr; i++)
        for (int j = 0; j < nt; j++) {
            double a = 0.5 * (g->r[i + 1] * g->r[i + 1] - g->r[i] * g->r[i]) * dth;
            for (int k = 0; k < np; k++) wp[IDX(g, i, j, k)] = a * g->rc[i] * g->sc[j] * dph;
        }
}

/* J of the resistive operator on the edge arrays (og_current_edges layouts) */
void og_res_current(const og_grid* g, const double* br, const double* bt, const double* bp, double* jr,
                    double* jt, double* jp) {
    int nr = g->nr, nt = g->nt, np = g->np;
    og_current_edges(g, br, bt, bp, jr, jt, jp);
    for (int j = 0; j < nt; j++)
        for (int k = 0; k < np; k++) {
            jt[IDX(g, 0, j, k)] = 0.0;
            jt[IDX(g, nr, j, k)] = 0.0;
        }
    for (int j = 0; j <= nt; j++)
        for (int k = 0; k < np; k++) {
            jp[IDXT(g, 0, j, k)] = 0.0;
            jp[IDXT(g, nr, j, k)] = 0.0;
        }
}

/* y = W (x + dte curl_h J(x)) on stacked face vectors */
void og_res_apply(const og_grid* g, double dte, const double* x, double* y) {
    int nr = g->nr, nt = g->nt, np = g->np;
    long long nbr = (long long)(nr + 1) * nt * np, nbt = (long long)nr * (nt + 1) * np, n = og_res_size(g);
    edges3 e = edges_alloc(g);
    double* w = (double*)malloc(sizeof(double) * n);
    og_res_current(g, x, x + nbr, x + nbr + nbt, e.jr, e.jt, e.jp);
    memcpy(y, x, sizeof(double) * n);
    og_ct(g, e.jr, e.jt, e.jp, -dte, y, y + nbr, y + nbr + nbt);
    res_weights(g, w);
    for (long long q = 0; q < n; q++) y[q] *= w[q];
    free(w);
    edges_free(e);
}

/* diagonal of the system: W_f + dte l*_f^2 sum over the edges of f in the system of l_e / A*_e */
void og_res_diag(const og_grid* g, double dte, double* d) {
    int nr = g->nr, nt = g->nt, np = g->np;
    double dth = g->dth, dph = g->dph;
    long long nbr = (long long)(nr + 1) * nt * np, nbt = (long long)nr * (nt + 1) * np;
    res_weights(g, d);
    double* dr = d;
    double* dt_ = d + nbr;
    double* dp = d + nbr + nbt;
    /* dual-face areas: radial edge (shell i, node j), theta edge (node i, centre j), phi edge
     * (node i, node j); interior edges only */
#define ASR(i, j) (g->rc[i] * g->rc[i] * (g->cc[(j) - 1] - g->cc[j]) * dph)
#define AST(i, j) (g->sc[j] * 0.5 * (g->rc[i] * g->rc[i] - g->rc[(i) - 1] * g->rc[(i) - 1]) * dph)
#define ASP(i) (0.5 * (g->rc[i] * g->rc[i] - g->rc[(i) - 1] * g->rc[(i) - 1]) * dth)
    for (int i = 1; i < nr; i++)
        for (int j = 0; j < nt; j++) {
            double ls = lstar_r(g, i);
            double sum = 2.0 * g->r[i] * dth / AST(i, j);
            if (j >= 1) sum += g->r[i] * g->sn[j] * dph / ASP(i);
            if (j + 1 <= nt - 1) sum += g->r[i] * g->sn[j + 1] * dph / ASP(i);
            for (int k = 0; k < np; k++) dr[IDX(g, i, j, k)] += dte * ls * ls * sum;
        }
    for (int i = 0; i < nr; i++)
        for (int j = 1; j < nt; j++) {
            double ls = g->rc[i] * dth, lr = g->r[i + 1] - g->r[i];
            double sum = 2.0 * lr / ASR(i, j);
            if (i >= 1) sum += g->r[i] * g->sn[j] * dph / ASP(i);
            if (i + 1 <= nr - 1) sum += g->r[i + 1] * g->sn[j] * dph / ASP(i + 1);
            for (int k = 0; k < np; k++) dt_[IDXT(g, i, j, k)] += dte * ls * ls * sum;
        }
    for (int i = 0; i < nr; i++) {
        double lr = g->r[i + 1] - g->r[i];
        double cap_n = g->rc[i] * g->rc[i] * (1.0 - g->cc[0]) * 2.0 * M_PI;
        double cap_s = g->rc[i] * g->rc[i] * (1.0 + g->cc[nt - 1]) * 2.0 * M_PI;
        for (int j = 0; j < nt; j++) {
            double ls = g->rc[i] * g->sc[j] * dph;
            double sum = lr / (j == 0 ? cap_n : ASR(i, j)) + lr / (j == nt - 1 ? cap_s : ASR(i, j + 1));
            if (i >= 1) sum += g->r[i] * dth / AST(i, j);
            if (i + 1 <= nr - 1) sum += g->r[i + 1] * dth / AST(i + 1, j);
            for (int k = 0; k < np; k++) dp[IDX(g, i, j, k)] += dte * ls * ls * sum;
        }
    }
#undef ASR
#undef AST
#undef ASP
}

/* Jacobi PCG on the resistive system (same stop test, count and b = 0 rule as og_pcg) */
int og_res_pcg(const og_grid* g, double dte, const double* b, double* x, double tol, int max_iter,
               int fixed_iters, int* iters, double* relres) {
    long long n = og_res_size(g);
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
        *iters = 0; *relres = 0.0;
        return OG_OK;
    }
    double* d = (double*)malloc(sizeof(double) * n);
    double* r = (double*)malloc(sizeof(double) * n);
    double* z = (double*)malloc(sizeof(double) * n);
    double* p = (double*)malloc(sizeof(double) * n);
    double* q = (double*)malloc(sizeof(double) * n);
    og_res_diag(g, dte, d);
    og_res_apply(g, dte, x, q);
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n; e++) r[e] = b[e] - q[e];
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n; e++) z[e] = r[e] / d[e];
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n; e++) p[e] = z[e];
    double rz = dot(n, r, z);
    double rn = sqrt(dot(n, r, r));
    int k = 0, status = OG_OK;
    for (;;) {
        if (fixed_iters > 0) {
            if (k >= fixed_iters) break;
        } else {
            if (rn <= tol * bnorm) break;
            if (k >= max_iter) { status = OG_ERR_NOCONV; break; }
        }
        og_res_apply(g, dte, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) { status = OG_ERR_NOCONV; break; }
        double a = rz / pq;
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) x[e] += a * p[e];
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) r[e] -= a * q[e];
        k++;
        rn = sqrt(dot(n, r, r));
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) z[e] = r[e] / d[e];
        double rz_new = dot(n, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) p[e] = z[e] + beta * p[e];
    }
    *iters = k;
    *relres = rn / bnorm;
    free(d); free(r); free(z); free(p); free(q);
    return status;
}

/* B (three face arrays) <- B* - dte curl_h J(x), x the PCG solution of W (x + dte curl_h J(x)) = W B*
 * started from B*: the final update is a CT circulation, so div_h B keeps its value to rounding
 * whatever the solver tolerance, and B differs from x by the solver error only */
int og_res_solve(const og_grid* g, double dte, double* br, double* bt, double* bp, double tol, int max_iter,
                 int* iters, double* relres) {
    int nr = g->nr, nt = g->nt, np = g->np;
    long long nbr = (long long)(nr + 1) * nt * np, nbt = (long long)nr * (nt + 1) * np, n = og_res_size(g);
    double* x = (double*)malloc(sizeof(double) * n);
    double* b = (double*)malloc(sizeof(double) * n);
    memcpy(x, br, sizeof(double) * nbr);
    memcpy(x + nbr, bt, sizeof(double) * nbt);
    memcpy(x + nbr + nbt, bp, sizeof(double) * g->N);
    res_weights(g, b);
    for (long long q = 0; q < n; q++) b[q] *= x[q];
    int st = og_res_pcg(g, dte, b, x, tol, max_iter, 0, iters, relres);
    edges3 e = edges_alloc(g);
    og_res_current(g, x, x + nbr, x + nbr + nbt, e.jr, e.jt, e.jp);
    og_ct(g, e.jr, e.jt, e.jp, dte, br, bt, bp);
    edges_free(e);
    free(x); free(b);
    return st;
}

/* =============================================================================================
 * PC2 (Sec. 2.2): block-Jacobi with a zero-fill incomplete LU factorisation (ILU(0)) in each
 * block. Reading R9: the blocks are a choice (the paper's are the MPI ranks' subdomains); two
 * block structures are provided:
 *   blocks = 0: one block, the whole grid, in the natural order of the memory layout (i slowest,
 *               then j, then k; the periodic phi neighbour of k = np-1 at k = 0 comes earlier);
 *   blocks = 1: one block per periodic phi line (i, j): the couplings in r and theta are dropped
 *               from the preconditioner, each line keeps its own tridiagonal-plus-wrap block.
 * The three components share the factorisation. For these patterns (np >= 4) zero fill changes
 * only the diagonal:
 *     dt_c = M_cc - sum over the earlier in-block neighbours l of c of M_cl^2 / dt_l,
 * and the preconditioner is P = (dt + L) dt^-1 (dt + U), L / U the strict lower / upper parts of
 * the block-diagonal part of M_alpha: symmetric, equal to M_alpha on each block's pattern. z =
 * P^-1 r by one forward and one backward substitution in that order.
 * =========================================================================================== */
/* off-diagonal entries of M_alpha at cell (i, j, k) towards its six neighbours: -alpha w */
static void m_offdiag(const og_grid* g, double alpha, int i, int j, double* wrl, double* wrh, double* wtl,
                      double* wth, double* wp) {
    int nr = g->nr, nt = g->nt;
    *wrl = (i > 0) ? -alpha * g->wr[i * nt + j] : 0.0;
    *wrh = (i < nr - 1) ? -alpha * g->wr[(i + 1) * nt + j] : 0.0;
    *wtl = (j > 0) ? -alpha * g->wt[i * (nt + 1) + j] : 0.0;
    *wth = (j < nt - 1) ? -alpha * g->wt[i * (nt + 1) + j + 1] : 0.0;
    *wp = -alpha * g->wp[i * nt + j];
}

/* dt (N entries) of the ILU(0) factorisation; returns 0, or -1 if a pivot is not positive */
int og_ilu0(const og_grid* g, double alpha, int blocks, double* dt) {
    int nr = g->nr, nt = g->nt, np = g->np;
    int whole = (blocks == 0);
    double* dg = (double*)malloc(sizeof(double) * nr * nt);
    og_diag(g, alpha, dg);
    int bad = 0;
    for (int i = 0; i < nr; i++)
        for (int j = 0; j < nt; j++)
            for (int k = 0; k < np; k++) {
                double wrl, wrh, wtl, wth, wp;
                m_offdiag(g, alpha, i, j, &wrl, &wrh, &wtl, &wth, &wp);
                double d = dg[i * nt + j];
                if (whole && i > 0) d -= wrl * wrl / dt[IDX(g, i - 1, j, k)];
                if (whole && j > 0) d -= wtl * wtl / dt[IDX(g, i, j - 1, k)];
                if (k > 0) d -= wp * wp / dt[IDX(g, i, j, k - 1)];
                if (k == np - 1) d -= wp * wp / dt[IDX(g, i, j, 0)];
                if (!(d > 0.0)) bad = 1;
                dt[IDX(g, i, j, k)] = d;
            }
    free(dg);
    return bad ? -1 : 0;
}

/* z = P^-1 r for ncomp stacked components, dt from og_ilu0 with the same blocks */
void og_ilu0_apply(const og_grid* g, double alpha, int blocks, const double* dt, int ncomp, const double* r,
                   double* z) {
    int nr = g->nr, nt = g->nt, np = g->np;
    int whole = (blocks == 0);
    for (int c = 0; c < ncomp; c++) {
        const double* rc = r + c * g->N;
        double* zc = z + c * g->N;
        /* forward: (dt + L) u = r, u stored in z */
        for (int i = 0; i < nr; i++)
            for (int j = 0; j < nt; j++)
                for (int k = 0; k < np; k++) {
                    double wrl, wrh, wtl, wth, wp;
                    m_offdiag(g, alpha, i, j, &wrl, &wrh, &wtl, &wth, &wp);
                    double s = rc[IDX(g, i, j, k)];
                    if (whole && i > 0) s -= wrl * zc[IDX(g, i - 1, j, k)];
                    if (whole && j > 0) s -= wtl * zc[IDX(g, i, j - 1, k)];
                    if (k > 0) s -= wp * zc[IDX(g, i, j, k - 1)];
                    if (k == np - 1) s -= wp * zc[IDX(g, i, j, 0)];
                    zc[IDX(g, i, j, k)] = s / dt[IDX(g, i, j, k)];
                }
        /* backward: (dt + U) z = dt u */
        for (int i = nr - 1; i >= 0; i--)
            for (int j = nt - 1; j >= 0; j--)
                for (int k = np - 1; k >= 0; k--) {
                    double wrl, wrh, wtl, wth, wp;
                    m_offdiag(g, alpha, i, j, &wrl, &wrh, &wtl, &wth, &wp);
                    double s = 0.0;
                    if (whole && i < nr - 1) s += wrh * zc[IDX(g, i + 1, j, k)];
                    if (whole && j < nt - 1) s += wth * zc[IDX(g, i, j + 1, k)];
                    if (k < np - 1) s += wp * zc[IDX(g, i, j, k + 1)];
                    if (k == 0) s += wp * zc[IDX(g, i, j, np - 1)];
                    zc[IDX(g, i, j, k)] -= s / dt[IDX(g, i, j, k)];
                }
    }
}

/* PCG with PC2 (same stop test, count and b = 0 rule as og_pcg) */
int og_pcg_pc2(const og_grid* g, double alpha, int blocks, int ncomp, const double* b, double* x, double tol,
               int max_iter, int fixed_iters, int* iters, double* relres) {
    long long N = g->N, n = ncomp * N;
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
        *iters = 0; *relres = 0.0;
        return OG_OK;
    }
    double* dt = (double*)malloc(sizeof(double) * N);
    double* r = (double*)malloc(sizeof(double) * n);
    double* z = (double*)malloc(sizeof(double) * n);
    double* p = (double*)malloc(sizeof(double) * n);
    double* q = (double*)malloc(sizeof(double) * n);
    int status = OG_OK;
    if (og_ilu0(g, alpha, blocks, dt) != 0) status = OG_ERR_NOCONV;
    og_apply_M(g, alpha, ncomp, x, q);
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n; e++) r[e] = b[e] - q[e];
    og_ilu0_apply(g, alpha, blocks, dt, ncomp, r, z);
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n; e++) p[e] = z[e];
    double rz = dot(n, r, z);
    double rn = sqrt(dot(n, r, r));
    int k = 0;
    while (status == OG_OK) {
        if (fixed_iters > 0) {
            if (k >= fixed_iters) break;
        } else {
            if (rn <= tol * bnorm) break;
            if (k >= max_iter) { status = OG_ERR_NOCONV; break; }
        }
        og_apply_M(g, alpha, ncomp, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) { status = OG_ERR_NOCONV; break; }
        double a = rz / pq;
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) x[e] += a * p[e];
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) r[e] -= a * q[e];
        k++;
        rn = sqrt(dot(n, r, r));
        og_ilu0_apply(g, alpha, blocks, dt, ncomp, r, z);
        double rz_new = dot(n, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < n; e++) p[e] = z[e] + beta * p[e];
    }
    *iters = k;
    *relres = rn / bnorm;
    free(dt); free(r); free(z); free(p); free(q);
    return status;
}
