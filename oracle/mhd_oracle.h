/*
 * Plain FP64 CPU oracle for the zero-beta MHD time step of Caplan et al. (arXiv 1811.02605).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's CPU
 * baseline load this library. The CUDA library shares no code, header, table or constant with
 * it; both sides take their inputs from the seeded generator in the package's inputs module.
 *
 * Everything is double precision, single threaded, written in the order of the definitions
 * it restates (Sec. 2.1 Eq. 1 for the model, Sec. 2.2 for the scheme family and the PCG
 * solver with the point-Jacobi preconditioner PC1). Where the paper is silent the readings are
 * stated beside each function. Compiled with -ffp-contract=off so no multiply-add is fused.
 *
 * Layouts (phi fastest, C order). N = nr*nt*np cells.
 *   vectors      v[c][i][j][k], c = 0 (r), 1 (theta), 2 (phi)
 *   br [nr+1][nt][np]  bt [nr][nt+1][np]  bp [nr][nt][np]          faces
 *   er [nr][nt+1][np]  et [nr+1][nt][np]  ep [nr+1][nt+1][np]      edges (E and J)
 */
#ifndef MHD_ORACLE_H
#define MHD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct og_grid og_grid;

enum { OG_OK = 0, OG_ERR_ARG = 1, OG_ERR_NOCONV = 3 };

og_grid* og_create(int nr, int nt, int np, double r0, double r1, double stretch);
void og_destroy(og_grid* g);

/* geometry tables exported for tests: r nodes (nr+1), cell volume (nr*nt), k~^2 (nr*nt) */
void og_radial_nodes(const og_grid* g, double* r);
void og_volumes(const og_grid* g, double* vol);
void og_ktilde2(const og_grid* g, double* kt2);

/* q = M_alpha p for ncomp stacked components (Sec. 4.1: the implicit operators are sparse
 * symmetric stencils). M_alpha = D + alpha K, D = rho_c V_c. */
void og_apply_M(const og_grid* g, double alpha, int ncomp, const double* p, double* q);
/* same with the Dirichlet term and D switched off: the pure-Neumann stiffness K (tests) */
void og_apply_K_neumann(const og_grid* g, int ncomp, const double* p, double* q);
/* diagonal of M_alpha per (i,j) row, nr*nt entries */
void og_diag(const og_grid* g, double alpha, double* d);

/* threads of the OpenMP timing build (n > 0 sets them); the plain build returns 1 */
int og_set_threads(int n);

/* field diagnostics (Sec. 3.1): out[5] = magnetic energy, kinetic energy, sum |J x B| V,
 * sum |J . B| V, max |div_h B| (flux over volume); v stacked [3][N] */
void og_diagnostics(const og_grid* g, const double* v, const double* br, const double* bt, const double* bp,
                    double* out);

/* the inner product every PCG form of the oracle uses (compensated, reading P12) */
double og_dot(long long n, const double* a, const double* b);

/* point-Jacobi PCG (PC1). x holds x0 on entry. fixed_iters > 0 runs exactly that many
 * iterations. Returns OG_OK or OG_ERR_NOCONV. */
int og_pcg(const og_grid* g, double alpha, int ncomp, const double* b, double* x, double tol,
           int max_iter, int fixed_iters, int* iters, double* relres);
/* og_pcg in the single-reduction (Chronopoulos-Gear) form */
int og_pcg_cg(const og_grid* g, double alpha, int ncomp, const double* b, double* x, double tol,
           int max_iter, int fixed_iters, int* iters, double* relres);

/* step coefficients: out = {dt, C_f, C_w, alpha_SI, alpha_nu} */
int og_coeffs(const og_grid* g, double nu, double cfl, double dt_fixed, double dt_max,
              double asi_fixed, const double* v, const double* br, const double* bt, const double* bp,
              double* out);

void og_bcentre(const og_grid* g, const double* br, const double* bt, const double* bp,
                double* bc);
void og_current_edges(const og_grid* g, const double* br, const double* bt, const double* bp,
                      double* jr, double* jt, double* jp);
void og_current_centre(const og_grid* g, const double* br, const double* bt, const double* bp,
                       double* jc);
/* b = rho_c V_c dt F(v, B) */
void og_force(const og_grid* g, const double* v, const double* br, const double* bt,
              const double* bp, double dt, double* b);
void og_efield_edges(const og_grid* g, const double* vbar, const double* br, const double* bt,
                     const double* bp, double eta, double* er, double* et, double* ep);
/* B <- B - dt * curl_h E */
void og_ct(const og_grid* g, const double* er, const double* et, const double* ep, double dt,
           double* br, double* bt, double* bp);
/* discrete divergence (net outward flux) per cell, N entries */
void og_divb(const og_grid* g, const double* br, const double* bt, const double* bp, double* div);

/* one predictor-corrector step, in place. dt_fixed > 0 bypasses the CFL rule; asi_fixed >= 0
 * replaces the computed alpha_SI (frozen map for finite differences). info = {dt, cf, cw, asi, anu, it0, it1, it2,
 * rr0, rr1, rr2} (11 doubles) */
/* step options (bit mask) of og_step_opts */
enum { OG_OPT_PCG_CG = 1, OG_OPT_STS = 2, OG_OPT_RES_IMPLICIT = 4, OG_OPT_PC2 = 8 };
int og_step(const og_grid* g, double nu, double eta, double cfl, double dt_fixed, double dt_max,
            double asi_fixed, double tol, int max_iter, double* v, double* br, double* bt,
            double* bp, double* info);
int og_step_cg(const og_grid* g, double nu, double eta, double cfl, double dt_fixed, double dt_max,
            double asi_fixed, double tol, int max_iter, double* v, double* br, double* bt,
            double* bp, double* info);

/* Adjoint of og_step with dt = `dt` (fixed), alpha_SI = asi_fixed if >= 0 (else computed from
 * state n), alpha_nu = nu dt, and the upwind directions of the forward step frozen (reading P15).
 * Given state n (v [3N], br, bt, bp) and the cotangent of state n+1 (lv1, lbr1, lbt1, lbp1),
 * writes the cotangent of state n (lv, lbr, lbt, lbp). PCG solves use `tol`. */
int og_adjoint_step(const og_grid* g, double nu, double eta, double cfl, double dt, double asi_fixed,
                    double tol, int max_iter, const double* v, const double* br, const double* bt,
                    const double* bp, const double* lv1, const double* lbr1, const double* lbt1,
                    const double* lbp1, double* lv, double* lbr, double* lbt, double* lbp);
int og_adjoint_step_sts(const og_grid* g, double nu, double eta, double cfl, double dt, double asi_fixed,
                    double tol, int max_iter, const double* v, const double* br, const double* bt,
                    const double* bp, const double* lv1, const double* lbr1, const double* lbt1,
                    const double* lbp1, double* lv, double* lbr, double* lbt, double* lbp);

/* Viscosity by RKL2 super time-stepping: stage count for (nu, dt), and v (3N) advanced in place
 * over dt with s stages (s <= 0: chosen by og_rkl2_stages). Returns s. */
int og_rkl2_stages(const og_grid* g, double nu, double dt);
int og_rkl2(const og_grid* g, double nu, double dt, int s, double* v);
/* og_step with the viscous PCG solve replaced by RKL2 (info[7] = stage count) */
int og_step_sts(const og_grid* g, double nu, double eta, double cfl, double dt_fixed, double dt_max,
                double asi_fixed, double tol, int max_iter, double* v, double* br, double* bt, double* bp,
                double* info);


/* og_step with options: OG_OPT_PCG_CG every solve in the single-reduction form, OG_OPT_STS
 * viscosity by RKL2, OG_OPT_RES_IMPLICIT resistivity by the implicit face solve (info then has
 * 13 entries: [11] its iterations, [12] its relative residual), OG_OPT_PC2 every cell solve
 * preconditioned by PC2 with phi-line blocks */
int og_step_opts(const og_grid* g, int opts, double nu, double eta, double cfl, double dt_fixed, double dt_max,
                 double asi_fixed, double tol, int max_iter, double* v, double* br, double* bt, double* bp,
                 double* info);

/* implicit resistivity: stacked face vectors [br | bt | bp] of og_res_size entries */
long long og_res_size(const og_grid* g);
void og_res_current(const og_grid* g, const double* br, const double* bt, const double* bp, double* jr,
                    double* jt, double* jp);
void og_res_apply(const og_grid* g, double dte, const double* x, double* y);
void og_res_diag(const og_grid* g, double dte, double* d);
int og_res_pcg(const og_grid* g, double dte, const double* b, double* x, double tol, int max_iter,
               int fixed_iters, int* iters, double* relres);
int og_res_solve(const og_grid* g, double dte, double* br, double* bt, double* bp, double tol, int max_iter,
                 int* iters, double* relres);


/* PC2: block-Jacobi ILU(0) of M_alpha; blocks 0: one block in the natural order, 1: one block per
 * periodic phi line. og_ilu0 writes the modified diagonal (N entries; returns -1 on a non-positive
 * pivot); og_ilu0_apply gives z = P^-1 r; og_pcg_pc2 is og_pcg with that preconditioner. */
int og_ilu0(const og_grid* g, double alpha, int blocks, double* dt);
void og_ilu0_apply(const og_grid* g, double alpha, int blocks, const double* dt, int ncomp, const double* r,
                   double* z);
int og_pcg_pc2(const og_grid* g, double alpha, int blocks, int ncomp, const double* b, double* x, double tol,
               int max_iter, int fixed_iters, int* iters, double* relres);


/* adjoint of og_step_opts with OG_OPT_STS and / or OG_OPT_RES_IMPLICIT */
int og_adjoint_step_opts(const og_grid* g, int opts, double nu, double eta, double cfl, double dt, double asi_fixed,
                         double tol, int max_iter, const double* v0, const double* br0, const double* bt0,
                         const double* bp0, const double* lv1, const double* lbr1, const double* lbt1,
                         const double* lbp1, double* lv, double* lbr, double* lbt, double* lbp);

#ifdef __cplusplus
}
#endif
#endif
