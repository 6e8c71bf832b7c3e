/*
 * mhd.h -- C ABI of a GB300-native (sm_103a) library for the zero-beta MHD time step of
 * Caplan et al., "GPU Acceleration of an Established Solar MHD Code using OpenACC"
 * (arXiv 1811.02605).
 *
 * The model (Sec. 2.1, Eq. 1): magnetic field B = curl A advanced by dA/dt = v x curl A -
 * eta curl curl A (code units: c = 4 pi = 1), velocity advanced by
 *   dv/dt = -v.grad v + (J x B)/rho + (1/rho) div(nu rho grad v) + (1/rho) div(S rho grad dv/dt),
 * density frozen (rho = rho0(r) = (r0/r)^2), pressure zero. The scheme (Sec. 2.2): explicit
 * predictor-corrector upwinding for the advective and reactive terms, the semi-implicit (SI)
 * term solved implicitly inside the predictor-corrector with two preconditioned conjugate
 * gradient (PCG) solves, and viscosity by a third PCG solve, all with the point-Jacobi
 * preconditioner (PC1). Grid (Sec. 2.2: a staggered, logically rectangular, non-uniform mesh):
 * spherical shell r in [r0, r1] with geometric radial stretch, theta in [0, pi] uniform,
 * phi periodic; B on faces, E and J on edges, v at cell centres.
 *
 * Conventions common to every call:
 *  - All field and vector pointers are DEVICE pointers to caller-owned, contiguous float64
 *    arrays, phi fastest (C order), 16-byte aligned. The library never frees them.
 *  - N = nr*nt*np cells. Array shapes:
 *      br [nr+1][nt][np]  radial faces at r_i
 *      bt [nr][nt+1][np]  theta faces at theta_j; j = 0 and j = nt are the poles, held at 0
 *      bp [nr][nt][np]    phi faces at phi_k
 *      vr, vt, vp [nr][nt][np] cell centres; "stacked" vectors hold ncomp such blocks back
 *      to back ([ncomp][nr][nt][np]).
 *  - A grid owns its metric tables and all workspace. It allocates in mhd_grid_create, and
 *    features that need more allocate on first use: PC2 and implicit resistivity (their
 *    workspaces), mhd_adjoint_step (its workspace), pcg_solve_batched (the plan of a batch), and
 *    every PCG form (the CUDA graph of its iterations). mhd_grid_reserve and pcg_batch_reserve do
 *    those allocations up front.
 *  - All work is enqueued on the grid's CUDA stream. Calls that return scalars (step info,
 *    iteration counts) synchronise that stream once at their end; the others return after
 *    enqueueing.
 *  - Status codes only: nothing throws or aborts across the ABI. After an error,
 *    mhd_last_error(grid) describes it. On MHD_ERR_NOCONV the best iterate is left in x.
 *  - One grid per stream; a grid is not thread-safe.
 *  - np must be even (double2 loads along phi); nt >= 2, nr >= 2.
 */
#ifndef MHD_H
#define MHD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mhd_grid_s* mhd_grid_t; /* opaque, library-owned */

typedef enum {
    MHD_OK = 0,
    MHD_ERR_ARG = 1,       /* invalid argument (sizes, pointers, parameters) */
    MHD_ERR_CUDA = 2,      /* a CUDA runtime call failed */
    MHD_ERR_NOCONV = 3,    /* PCG reached max_iter (or max_outer) before the tolerance */
    MHD_ERR_NONFINITE = 4, /* NaN or Inf met in a reduction */
    MHD_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up (batched persistent solver) */
    MHD_ERR_OOM = 6        /* device allocation failed */
} mhd_status_t;

/* Grid: nr x nt x np cells. Radial nodes r_0 = r0, r_{i+1} = r_i + h0 s^i with
 * h0 = (r1 - r0)(s - 1)/(s^nr - 1) (s = stretch, uniform if s == 1). theta_j = j pi/nt,
 * phi_k = 2 pi k/np. (Sec. 3: the production run refines the grid strongly near the erupting
 * region and coarsens it with distance; the geometric stretch stands in for that.) */
typedef struct {
    int nr, nt, np;
    double r0, r1, stretch;
} mhd_grid_desc_t;

enum { MHD_PREC_FP64 = 0, MHD_PREC_MIXED = 1 };

/* Step and solver parameters.
 *  nu        kinematic viscosity (Eq. 1), code units
 *  eta       resistivity (Eq. 1); explicit in E = -v x B + eta J
 *  cfl       flow CFL number C_f: dt = cfl / max_c(k~_c |v_c|)
 *  dt_fixed  > 0: use this dt instead of the CFL rule
 *  dt_max    > 0: upper bound on the CFL dt
 *  alpha_si_fixed >= 0: use this SI coefficient instead of the computed one (frozen map)
 *  tol       relative residual ||b - M x||_2 / ||b||_2 at which PCG stops (Sec. 2.2)
 *  inner_tol mixed precision only: FP32 inner solves stop at inner_tol times the outer residual
 *  max_iter  PCG iteration cap per solve (inner iterations in mixed precision)
 *  max_outer mixed precision: cap on FP64 iterative-refinement passes
 *  precision MHD_PREC_FP64 or MHD_PREC_MIXED (FP32 stencil and inner PCG, FP64 residuals,
 *            corrections and reductions)
 *  mixed_restart  mixed precision only. 0 (default): reliable updates. When the FP32 recursive
 *            residual has fallen by inner_tol, x is corrected in FP64, the true FP64 residual
 *            replaces the recursive one, and the CG recurrence continues with the same search
 *            direction. 1: classic iterative refinement, restarting the FP32 CG from the new
 *            residual at each correction.
 *  viscosity_sts  0 (default): viscosity by the implicit solve M_nu v^{n+1} = rho V v** (PCG).
 *            1: viscosity by RKL2 super time-stepping (second-order Runge-Kutta-Legendre, the
 *            STS option of Sec. 2.2 / algorithm 3): rho V dv/dt = -nu K v is advanced explicitly
 *            from v** over dt in s stages, s the smallest s >= 2 with (s^2 + s - 2)/2 >=
 *            dt lambda, lambda the Gershgorin bound of nu (rho V)^-1 K. info->iters[2] then holds
 *            s and outer[2], relres[2] are 0. Always FP64 (the SI solves keep `precision`).
 *  pcg_variant  0 (default): Hestenes-Stiefel PCG (three kernels and two reductions per
 *            iteration). 1: the same Jacobi PCG in the single-reduction form of Chronopoulos &
 *            Gear (1989): s = M p is updated by its own recurrence, so one operator application
 *            gives both inner products and an iteration is two kernels with one reduction. Same
 *            iterates in exact arithmetic; rounding differs. FP64 only (MHD_ERR_ARG with
 *            precision = MHD_PREC_MIXED); applies to every solve of pcg_solve, mhd_step and
 *            mhd_adjoint_step (pcg_solve_batched ignores it).
 *  resistivity_implicit  0 (default): resistivity explicit, E = -v x B + eta J in the CT update.
 *            1: resistivity implicit (Eq. 1's -eta curl curl term, Sec. 2.2: PCG with PC1): after
 *            the ideal CT update to B*, solve W (B + dt eta curl_h J(B)) = W B* on the faces,
 *            curl_h the CT face circulation, J on each edge the circulation of B around the
 *            edge's dual face over its area (0 on the tangential edges of r0 and r1), W_f = face
 *            area x centre-to-centre distance across the face (SPD system); then B = B* - dt eta
 *            curl_h J(x) from the solution x, which keeps div_h B to rounding. Uses tol and
 *            max_iter; FP64 (either precision setting). info->iters_res / relres_res report it.
 *            The first such step allocates its workspace (4 face vectors). mhd_adjoint_step
 *            differentiates it: the face solve's transpose is W M^-1 (one more face PCG solve).
 *  preconditioner  0 (default): PC1, point Jacobi (Sec. 2.2). 1: PC2, block Jacobi with a
 *            zero-fill incomplete LU factorisation (ILU(0)) in each block (Sec. 2.2); the blocks
 *            are the periodic phi lines (i, j) of each component, so the r and theta couplings
 *            are left out of the preconditioner and every line is solved independently (one warp
 *            per line, forward and backward substitution as affine scans). In mixed precision
 *            the FP32 inner solves use it too (FP32 factor copy; after each FP64 residual
 *            replacement one preconditioner pass recomputes z and <r, z>). Needs pcg_variant 0
 *            (MHD_ERR_ARG otherwise); applies to every solve of pcg_solve, mhd_step and
 *            mhd_adjoint_step; the first PC2 solve allocates N doubles + N floats for the
 *            factorisation and 3N floats for z of the FP32 iteration. pcg_solve_batched ignores it.
 *
 * Kernel variants of the FP32 inner iteration (split p update and stencil, the two folded into
 * one kernel, the recompute pair that stores no A p, the single-reduction pair, or plane-marching
 * tiles) and of the FP64 iteration (split, components overlapped on two streams, tiles) are chosen
 * per grid by timing on its first solve of each precision (or in mhd_grid_reserve); results agree
 * to the order of the dot products' reductions. Diagnostics only: the environment variable
 * MHD_FORCE_SLAB skips the timing (-1 split, -2 folded, -3 recompute pair, -4 recompute pair with
 * the second kernel walking the grid backwards, -5 recompute pair at 6 CTAs per SM, -6 / -7 / -8
 * single-reduction pair (-7: its residual kernel unrolled over the components, both kernels at 3
 * CTAs per SM; -8: unrolled residual kernel, update kernel at 4), -64 the FP64 iteration with its
 * components overlapped, n > 0 tiles of n planes). */
typedef struct {
    double nu, eta, cfl, dt_fixed, dt_max, alpha_si_fixed;
    double tol, inner_tol;
    int max_iter, max_outer;
    int precision;
    int mixed_restart;
    int viscosity_sts;
    int pcg_variant;
    int resistivity_implicit;
    int preconditioner;
} mhd_params_t;

/* Caller-owned DEVICE pointers (layouts above). */
typedef struct {
    double *br, *bt, *bp, *vr, *vt, *vp;
} mhd_fields_t;

/* Per-step report. iters/outer/relres: [0] SI predictor, [1] SI corrector, [2] viscosity.
 * relres is the final ||r||_2/||b||_2 (recursive residual in FP64 mode, true FP64 residual in
 * mixed mode). */
typedef struct {
    double dt, cf, cw, alpha_si, alpha_nu;
    int iters[3], outer[3];
    double relres[3];
    int iters_res;      /* implicit resistivity: PCG iterations (0 otherwise) */
    double relres_res;  /* implicit resistivity: final ||r||_2 / ||b||_2 */
} mhd_step_info_t;

/* Create a grid on the CUDA stream `cuda_stream` (a cudaStream_t; NULL = legacy default
 * stream) of the current device. Builds the metric tables (exact finite-volume geometry of
 * spherical cells) and allocates all workspace for one 3-component solve in either precision.
 * Errors: MHD_ERR_ARG (sizes, r1 <= r0, stretch <= 0, np odd, 3 (nr+1)(nt+1) np >= 2^31),
 * MHD_ERR_OOM, MHD_ERR_CUDA. */
mhd_status_t mhd_grid_create(const mhd_grid_desc_t* desc, void* cuda_stream, mhd_grid_t* out);

/* Free the grid's tables and workspace (synchronises its stream). NULL is accepted. */
mhd_status_t mhd_grid_destroy(mhd_grid_t grid);

/* Element counts of br, bt, bp, vr, vt, vp. */
mhd_status_t mhd_grid_sizes(mhd_grid_t grid, long long sizes[6]);

/* Step coefficients (Sec. 2.1 definition of S; Sec. 3: the time step varies from step to step):
 * dt = cfl / max_c(k~_c |v_c|) (or dt_fixed; clipped to dt_max), C_f = dt max k~|v|,
 * C_w = dt max k~ |B_c|/sqrt(rho_c), alpha_SI = max(C_w^2/(1-C_f)^2 - 1, 0)/max k~^2,
 * alpha_nu = nu dt, where k~_c^2 = 1/dr^2 + 1/(r dtheta)^2 + 1/(r sin(theta) dphi)^2 at the cell
 * centre. Fills info->dt, cf, cw, alpha_si, alpha_nu; synchronises. MHD_ERR_ARG if C_f >= 1 or
 * no dt can be formed (v = 0 without dt_fixed or dt_max). */
mhd_status_t mhd_step_coeffs(mhd_grid_t grid, const mhd_params_t* params,
                             const mhd_fields_t* fields, mhd_step_info_t* info);

/* One zero-beta predictor-corrector step, in place on `inout` (Sec. 2.2):
 *   1. coefficients as in mhd_step_coeffs from (v^n, B^n)
 *   2. predictor: M_SI d_p = rho V dt F(v^n, B^n), x0 = 0; v_p = v^n + d_p
 *   3. B^{n+1} = B^n - dt curl_h E, E = -v_bar x B^n + eta J(B^n), v_bar = (v^n + v_p)/2,
 *      averaged from cell centres to edges (constrained transport: div_h B is unchanged)
 *   4. corrector: M_SI d_c = rho V dt (F(v^n,B^n) + F(v_p,B^{n+1}))/2, x0 = d_p; v** = v^n + d_c
 *   5. viscosity: M_nu v^{n+1} = rho V v**, x0 = v**
 * M_alpha = D + alpha K is the symmetric finite-volume form of rho - alpha div(rho grad .) per
 * component (see mhd_apply_operator). `info` may be NULL. Returns the first non-OK status of the
 * three solves (the step still completes), MHD_ERR_ARG for bad parameters. */
mhd_status_t mhd_step(mhd_grid_t grid, const mhd_params_t* params, mhd_fields_t* inout,
                      mhd_step_info_t* info);

/* q = M_alpha p for ncomp (1..3) stacked components: the implicit viscous/SI operator
 * (Eq. 1; Sec. 4.1: the implicit matrices are applied as stencils, never stored):
 * (M_alpha u)_c = rho_c V_c u_c + alpha sum_faces w_f (u_c - u_nb), w_f = rho A_f / d_f,
 * Dirichlet u = 0 at r0, Neumann at r1, no flux through the poles, periodic in phi.
 * p and q: device, [ncomp][nr][nt][np]; must not overlap. Enqueued only. */
mhd_status_t mhd_apply_operator(mhd_grid_t grid, double alpha, int ncomp, const double* p,
                                double* q);

/* b = rho_c V_c dt F(v, B) with F = -(v.grad)v + (J x B)/rho (Eq. 1), first-order upwind
 * advection with spherical curvature terms, J = curl_h B on edges averaged to centres. v from
 * fields->vr/vt/vp, B from fields->br/bt/bp. b: device [3][nr][nt][np]. Enqueued only. */
mhd_status_t mhd_force(mhd_grid_t grid, const mhd_fields_t* fields, double dt, double* b);

/* Constrained-transport induction (Eq. 1 in B form): B <- B - dt curl_h E with
 * E = -vbar x B + eta J on edges. vbar: device [3][nr][nt][np]; B in fields->br/bt/bp updated
 * in place (fields->v* ignored). Enqueued only. */
mhd_status_t mhd_induction(mhd_grid_t grid, const double* vbar, double eta, double dt,
                           mhd_fields_t* fields);

/* Solve M_alpha x = b by PCG with the point-Jacobi preconditioner (Sec. 2.2 PC1), for ncomp
 * (1..3) stacked components sharing one CG alpha/beta. x holds x0 on entry (NULL-free; pass
 * zeros for a cold start) and the solution on exit. Stop: ||r||_2 <= tol ||b||_2 (recursive
 * residual, tested before each iteration; FP64 mode) or on the true FP64 residual (mixed
 * mode, FP32 inner solves to inner_tol). b = 0 gives x = 0 after 0 iterations.
 * iters/outer/relres may be NULL. Synchronises. MHD_ERR_NOCONV at max_iter/max_outer,
 * MHD_ERR_NONFINITE if a reduction is not finite. */
mhd_status_t pcg_solve(mhd_grid_t grid, double alpha, int ncomp, const double* b, double* x,
                       const mhd_params_t* params, int* iters, int* outer, double* relres);

/* Batched FP64 PCG: n independent 3-component systems M_alpha[i] x[i] = b[i] on grids[i]
 * (grids of different sizes allowed; all on the stream of grids[0]) in ONE persistent
 * cooperative launch per CUDA-graph replay, with per-system scalars and bounded grid barriers.
 * x[i] holds x0 on entry. iters/relres: host arrays of n (may be NULL). Returns MHD_ERR_NOCONV
 * if any system missed the tolerance, MHD_ERR_TIMEOUT if a device barrier gave up. */
mhd_status_t pcg_solve_batched(int n, const mhd_grid_t* grids, const double* alpha,
                               const double* const* b, double* const* x,
                               const mhd_params_t* params, int* iters, double* relres);

/* Adjoint (reverse-mode derivative) of one mhd_step with dt frozen to `dt`, alpha_SI to
 * params->alpha_si_fixed if >= 0 (else the value computed from state_n), alpha_nu = nu dt, and
 * the upwind directions of the forward step. Given state_n and the cotangent adj_np1 =
 * dL/d(state_{n+1}) (same layout as the fields), writes adj_n = dL/d(state_n). The step's
 * intermediates are recomputed from state_n. PCG solves inside use params->tol. With
 * params->viscosity_sts = 1 it differentiates the RKL2 step (same stage count): the viscous
 * transpose is D P D^-1 with D = rho V and P the stage polynomial. adj_n must not alias adj_np1
 * or state_n. Synchronises. */
mhd_status_t mhd_adjoint_step(mhd_grid_t grid, const mhd_params_t* params,
                              const mhd_fields_t* state_n, double dt,
                              const mhd_fields_t* adj_np1, mhd_fields_t* adj_n);

/* The momentum force of mhd_force for callers that cannot allocate device memory (a host code
 * that owns all device memory under a fixed budget, a latency-bound loop where cudaMalloc may
 * synchronise the device, an allocator policy that forbids new allocations). The paper has no
 * counterpart: it is an interface variant, not part of the method. No grid object is needed:
 * the grid is described by `desc`, and the metric tables, the current density on edges and the
 * polar ring sums are kept in one static device array of 10 MiB (1,310,720 doubles) that every
 * GPU loading this library holds until the process exits. Limits: at most 262,144 cells and the
 * tables and edge arrays must fit that array; larger grids return MHD_ERR_ARG. The call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine). The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture. All calls share the array: calls whose work
 * overlaps on the GPU (different streams or host threads) race on it. Inputs and output as in
 * mhd_force (device pointers); work is enqueued on `cuda_stream` (a cudaStream_t, NULL = legacy
 * default stream). Errors: MHD_ERR_ARG (null pointer, bad or too large grid), MHD_ERR_CUDA. */
mhd_status_t mhd_force_noalloc(const mhd_grid_desc_t* desc, const mhd_fields_t* fields, double dt,
                               double* b, void* cuda_stream);

/* Field diagnostics (Sec. 3.1 validates its runs by the integrated magnetic and kinetic energies
 * and by |J x B| and |J . B|): out[0] = magnetic energy 1/2 sum_c |B_c|^2 V_c, out[1] = kinetic
 * energy 1/2 sum_c rho_c |v_c|^2 V_c, out[2] = sum_c |J_c x B_c| V_c, out[3] = sum_c |J_c . B_c| V_c,
 * out[4] = max_c |div_h B|, the net outward flux of a cell over its volume (0 to rounding while B
 * evolves by constrained transport). B_c and J_c are the cell-centred fields of the momentum force.
 * FP64 device reductions; synchronises the grid's stream. */
mhd_status_t mhd_diagnostics(mhd_grid_t grid, const mhd_fields_t* fields, double out[5]);

/* Domain decomposition in r (Sec. 4.2: the code runs one MPI rank per GPU, each rank owning a part
 * of the mesh; a PCG iteration exchanges the boundary values its operator application needs and
 * sums the few scalars of its inner products over the ranks with an allreduce). A slab grid holds
 * the radial rows [i0, i1) of the grid `desc` describes (at least 2 rows), with the
 * global metric and operator tables of those rows; its vectors are [ncomp][i1-i0][nt][np]. The
 * calls of a whole grid (mhd_step, pcg_solve, mhd_apply_operator, ...) refuse a slab grid; the
 * distributed point-Jacobi PCG of paper_1811_02605_gb300/dist.py drives these three calls and does
 * the exchange and the sums. */
mhd_status_t mhd_grid_create_slab(const mhd_grid_desc_t* desc, int i0, int i1, void* cuda_stream, mhd_grid_t* out);

/* q = M_alpha p on the slab's rows (Sec. 4.1 operator; same arithmetic and order as the whole
 * grid's operator, so the rows are bit-identical to it). p_lo / p_hi: the neighbours' boundary
 * planes, global rows i0-1 and i1 ([ncomp][nt][np] device arrays); NULL exactly where the slab
 * touches r0 or r1 (MHD_ERR_ARG otherwise). *pq (nullable, host): the slab's share of <p, q>
 * (synchronises the stream when given). */
mhd_status_t mhd_slab_apply(mhd_grid_t slab, double alpha, int ncomp, const double* p, const double* p_lo,
                            const double* p_hi, double* q, double* pq);

/* One iteration's vector updates of point-Jacobi PCG (Sec. 2.2, PC1) on the slab: x += a p (skipped
 * when x is NULL), r -= a q, z = r / diag(M_alpha); dots (host) = the slab's shares of <r, z> and
 * <r, r>. Synchronises the stream. */
mhd_status_t mhd_slab_update(mhd_grid_t slab, double alpha, int ncomp, double a, double* x, const double* p,
                             double* r, const double* q, double* z, double dots[2]);

/* p = z + beta p (p = z when beta = 0, whatever p held). */
mhd_status_t mhd_slab_pupdate(mhd_grid_t slab, int ncomp, double beta, const double* z, double* p);

/* Workspace reservation (not part of the method; the paper has no counterpart). Some features
 * allocate on their first use: the PC2 factorisation, the implicit-resistivity face vectors, the
 * adjoint workspace, and the CUDA graphs of the PCG iterations (instantiating a graph can take
 * device memory), after the per-grid kernel choice that those graphs record. mhd_grid_reserve does
 * all of that now for the features named, so that afterwards mhd_step, pcg_solve and
 * mhd_adjoint_step on 3-component systems with those features allocate no device memory on this
 * grid (a code that captures them in its own CUDA graph, or that budgets device memory up front,
 * needs that). The PCG vectors' contents are overwritten (the timed trial iterations of the kernel
 * choice); fields are not touched. Synchronises the grid's stream. Errors: MHD_ERR_ARG (unknown
 * feature bit), MHD_ERR_OOM, MHD_ERR_CUDA. */
enum {
    MHD_RESERVE_PC1 = 1,           /* FP64 point-Jacobi PCG: FP64 kernel choice, iteration graph */
    MHD_RESERVE_MIXED = 2,         /* mixed precision: FP32 kernel choice (timed), iteration graph */
    MHD_RESERVE_CG = 4,            /* single-reduction PCG (pcg_variant = 1): iteration graph */
    MHD_RESERVE_PC2 = 8,           /* preconditioner = 1: workspace, FP64 (and with MIXED FP32) graphs */
    MHD_RESERVE_RESISTIVITY = 16,  /* resistivity_implicit = 1: face workspace and iteration graph */
    MHD_RESERVE_ADJOINT = 32,      /* mhd_adjoint_step workspace */
    MHD_RESERVE_ALL = 63
};
mhd_status_t mhd_grid_reserve(mhd_grid_t grid, int features);

/* The same for a batch of pcg_solve_batched: builds (and times) the plan of exactly this batch
 * (the grids and the b and x pointers, as a later call passes them) and instantiates its CUDA graph
 * for these params; a later pcg_solve_batched with the same batch and the same tol and max_iter
 * allocates nothing. Solves nothing; x is not written. Errors as pcg_solve_batched. */
mhd_status_t pcg_batch_reserve(int n, const mhd_grid_t* grids, const double* alpha, const double* const* b,
                               double* const* x, const mhd_params_t* params);

/* Diagnostics (not part of the method): device time of the library's kernels, measured with
 * CUDA events recorded on the grid's stream immediately before and after each launch, summed
 * per kernel while profiling is enabled. Enabling resets the counters and makes the PCG loop
 * launch its kernels directly instead of replaying CUDA graphs (so each launch can be
 * bracketed); results are otherwise identical. */
enum {
    MHD_KERNEL_PUPDATE64 = 0, MHD_KERNEL_SPMV64 = 1, MHD_KERNEL_UPDATE64 = 2,
    MHD_KERNEL_PUPDATE32 = 3, MHD_KERNEL_SPMV32 = 4, MHD_KERNEL_UPDATE32 = 5,
    MHD_KERNEL_OUTER_RES = 6, MHD_KERNEL_FORCE = 7, MHD_KERNEL_INDUCTION = 8,
    MHD_KERNEL_COEFFS = 9, MHD_KERNEL_STS = 10, MHD_KERNEL_RES = 11, MHD_KERNEL_PC2 = 12,
    MHD_KERNEL_PSPMV32 = 13, /* FP32 p update folded into the stencil */
    MHD_KERNEL_PFOLD32 = 14, /* FP32 p update folded into <p, A p>, no q stored */
    MHD_KERNEL_RUPD32 = 15,  /* FP32 r update with A p recomputed, x every second iteration */
    MHD_KERNEL_CGR32 = 16,   /* FP32 single-reduction pair: <r, r>, <r, A r> and the scalars */
    MHD_KERNEL_CGU32 = 17,   /* FP32 single-reduction pair: p, A p, r and x updates */
    MHD_KERNEL_COUNT = 18
};
mhd_status_t mhd_profile_enable(mhd_grid_t grid, int enable);
/* Total milliseconds and launch count of one kernel id since profiling was enabled.
 * Synchronises the grid's stream. */
mhd_status_t mhd_profile_read(mhd_grid_t grid, int kernel, double* total_ms, long long* launches);
/* The kernel forms the grid's autotuner chose, in the codes of MHD_FORCE_SLAB: *fp64_form for the
 * FP64 iteration (-1 split, -2 components overlapped, n > 0 tiles of n planes) and *fp32_form for
 * the FP32 inner iteration (-1 split, -2 folded, -3/-4/-5 recompute pair, -6/-7/-8 single-reduction
 * pair, <= -100 bulk-staged pair, n > 0 tiles); 0 where that precision has not been tuned yet.
 * Either pointer may be NULL. */
mhd_status_t mhd_grid_kernel_forms(mhd_grid_t grid, int* fp64_form, int* fp32_form);

/* Text of the last error on this grid ("" if none); NULL grid gives the last create error. */
const char* mhd_last_error(mhd_grid_t grid);

#ifdef __cplusplus
}
#endif
#endif /* MHD_H */
