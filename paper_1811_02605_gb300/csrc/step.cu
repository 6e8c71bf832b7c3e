// C-ABI entry points: the zero-beta step (Sec. 2.2 predictor-corrector with two SI PCG solves
// and a viscous PCG solve) and the single-row calls used to test each part.
#include <cmath>
#include <cstring>

#include "mhd_internal.cuh"

using namespace mhd;

namespace {

__global__ void k_set_alpha(StepScalars* ss, double a) { ss->alpha_user = a; }

mhd_status_t check_params(mhd_grid_s* g, const mhd_params_t* p) {
    if (!p) return set_error(g, MHD_ERR_ARG, "params is NULL");
    if (!(p->tol > 0.0) || p->max_iter < 0)
        return set_error(g, MHD_ERR_ARG, "params: need tol > 0 and max_iter >= 0");
    if (p->precision != MHD_PREC_FP64 && p->precision != MHD_PREC_MIXED)
        return set_error(g, MHD_ERR_ARG, "params: precision must be 0 (FP64) or 1 (mixed)");
    if (p->precision == MHD_PREC_MIXED && (!(p->inner_tol > 0.0) || p->inner_tol >= 1.0 || p->max_outer < 1))
        return set_error(g, MHD_ERR_ARG, "params: mixed precision needs 0 < inner_tol < 1, max_outer >= 1");
    if (!(p->nu >= 0.0) || !(p->cfl > 0.0))
        return set_error(g, MHD_ERR_ARG, "params: need nu >= 0 and cfl > 0");
    if (p->viscosity_sts != 0 && p->viscosity_sts != 1)
        return set_error(g, MHD_ERR_ARG, "params: viscosity_sts must be 0 (implicit PCG) or 1 (RKL2)");
    if (p->pcg_variant != 0 && p->pcg_variant != 1)
        return set_error(g, MHD_ERR_ARG, "params: pcg_variant must be 0 (Hestenes-Stiefel) or 1 (single reduction)");
    if (p->pcg_variant == 1 && p->precision != MHD_PREC_FP64)
        return set_error(g, MHD_ERR_ARG, "params: the single-reduction PCG form is FP64 only");
    if (p->preconditioner != 0 && p->preconditioner != 1)
        return set_error(g, MHD_ERR_ARG, "params: preconditioner must be 0 (PC1) or 1 (PC2)");
    if (p->preconditioner == 1 && p->pcg_variant != 0)
        return set_error(g, MHD_ERR_ARG, "params: PC2 runs with pcg_variant 0");
    if (p->resistivity_implicit != 0 && p->resistivity_implicit != 1)
        return set_error(g, MHD_ERR_ARG, "params: resistivity_implicit must be 0 or 1");
    if (!(p->eta >= 0.0)) return set_error(g, MHD_ERR_ARG, "params: need eta >= 0");
    return MHD_OK;
}

bool fields_ok(const mhd_fields_t* f, bool need_v) {
    if (!f || !f->br || !f->bt || !f->bp) return false;
    if (need_v && (!f->vr || !f->vt || !f->vp)) return false;
    return true;
}

// the calls of a whole grid are refused on a slab of one (its edge rows couple to ghost planes)
mhd_status_t whole_grid(mhd_grid_s* g, const char* what) {
    if (g->slab_nr_global > 0)
        return set_error(g, MHD_ERR_ARG, std::string(what) + ": not available on a slab grid (mhd_slab_* calls)");
    return MHD_OK;
}

mhd_status_t read_step_scalars(mhd_grid_s* g) {
    if (cudaMemcpyAsync(g->h_ss, g->ss, sizeof(StepScalars), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
        return check_cuda(g, "read step scalars");
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return check_cuda(g, "sync");
    return MHD_OK;
}

}  // namespace

extern "C" mhd_status_t mhd_step_coeffs(mhd_grid_t g, const mhd_params_t* p, const mhd_fields_t* f,
                                        mhd_step_info_t* info) {
    if (!g) return MHD_ERR_ARG;
    if (whole_grid(g, "mhd_step_coeffs") != MHD_OK) return MHD_ERR_ARG;
    mhd_status_t st = check_params(g, p);
    if (st != MHD_OK) return st;
    if (!fields_ok(f, true)) return set_error(g, MHD_ERR_ARG, "mhd_step_coeffs: null field pointer");
    if ((st = coeffs(g, p, f->vr, f->vt, f->vp, f->br, f->bt, f->bp)) != MHD_OK) return st;
    if ((st = read_step_scalars(g)) != MHD_OK) return st;
    const StepScalars& h = *g->h_ss;
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->dt = h.dt;
        info->cf = h.cf;
        info->cw = h.cw;
        info->alpha_si = h.alpha_si;
        info->alpha_nu = h.alpha_nu;
    }
    if (h.status != MHD_OK) return set_error(g, MHD_ERR_ARG, "step coefficients: C_f >= 1 or no time step");
    return MHD_OK;
}

extern "C" mhd_status_t mhd_step(mhd_grid_t g, const mhd_params_t* p, mhd_fields_t* f, mhd_step_info_t* info) {
    if (!g) return MHD_ERR_ARG;
    if (whole_grid(g, "mhd_step") != MHD_OK) return MHD_ERR_ARG;
    mhd_status_t st = check_params(g, p);
    if (st != MHD_OK) return st;
    if (!fields_ok(f, true)) return set_error(g, MHD_ERR_ARG, "mhd_step: null field pointer");
    const Dims d = g->d;
    const size_t bytes3 = sizeof(double) * 3 * (size_t)d.N;
    NvtxRange range("mhd_step");
    NvtxPhase phase;
    // 1. coefficients from (v^n, B^n)
    phase.next("coefficients");
    int pc = prof_begin(g, g->stream, MHD_KERNEL_COEFFS);
    if ((st = coeffs(g, p, f->vr, f->vt, f->vp, f->br, f->bt, f->bp)) != MHD_OK) return st;
    prof_end(g, g->stream, pc);
    if ((st = read_step_scalars(g)) != MHD_OK) return st;
    if (g->h_ss->status != MHD_OK) return set_error(g, MHD_ERR_ARG, "mhd_step: C_f >= 1 or no time step");
    const double* dt_dev = &g->ss->dt;
    int it[3] = {0, 0, 0}, ou[3] = {0, 0, 0};
    double rr[3] = {0, 0, 0};
    mhd_status_t worst = MHD_OK;
    // 2. predictor: M_SI d_p = rho V dt F(v^n, B^n), x0 = 0
    phase.next("predictor");
    int ps = prof_begin(g, g->stream, MHD_KERNEL_FORCE);
    force(g, f->vr, f->vt, f->vp, nullptr, 0.0, f->br, f->bt, f->bp, dt_dev, 0.0, nullptr, g->b0);
    prof_end(g, g->stream, ps);
    cudaMemsetAsync(g->dlt, 0, bytes3, g->stream);
    st = solve(g, &g->ss->alpha_si, 3, g->b0, g->dlt, g->dlt, p, &it[0], &ou[0], &rr[0]);
    if (st == MHD_ERR_CUDA) return st;
    if (st != MHD_OK && worst == MHD_OK) worst = st;
    // 3. B^{n+1} = B^n - dt curl_h E(v^n + d_p / 2, B^n)
    phase.next("induction");
    int it_res = 0;
    double rr_res = 0.0;
    ps = prof_begin(g, g->stream, MHD_KERNEL_INDUCTION);
    induction(g, f->vr, f->vt, f->vp, g->dlt, 0.5, p->resistivity_implicit ? 0.0 : p->eta, dt_dev, 0.0, f->br,
              f->bt, f->bp);
    prof_end(g, g->stream, ps);
    if (p->resistivity_implicit) {
        // resistive part implicit on the faces: W (B + dt eta curl_h J(B)) = W B*
        ps = prof_begin(g, g->stream, MHD_KERNEL_RES);
        st = res_solve(g, dt_dev, p->eta, f->br, f->bt, f->bp, p, &it_res, &rr_res);
        prof_end(g, g->stream, ps);
        if (st == MHD_ERR_CUDA || st == MHD_ERR_OOM) return st;
        if (st != MHD_OK && worst == MHD_OK) worst = st;
    }
    // 4. corrector: M_SI d_c = (b0 + rho V dt F(v^n + d_p, B^{n+1})) / 2, x0 = d_p
    phase.next("corrector");
    ps = prof_begin(g, g->stream, MHD_KERNEL_FORCE);
    force(g, f->vr, f->vt, f->vp, g->dlt, 1.0, f->br, f->bt, f->bp, dt_dev, 0.0, g->b0, g->b1);
    prof_end(g, g->stream, ps);
    st = solve(g, &g->ss->alpha_si, 3, g->b1, g->dlt, g->dlt, p, &it[1], &ou[1], &rr[1]);
    if (st == MHD_ERR_CUDA) return st;
    if (st != MHD_OK && worst == MHD_OK) worst = st;
    // 5. viscosity: M_nu v^{n+1} = rho V v**, x0 = v**  (v** is formed in the stacked buffer)
    phase.next("viscosity");
    cudaMemcpyAsync(g->b1, f->vr, bytes3 / 3, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(g->b1 + d.N, f->vt, bytes3 / 3, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(g->b1 + 2 * d.N, f->vp, bytes3 / 3, cudaMemcpyDeviceToDevice, g->stream);
    vstar_rhs(g, g->b1, g->b1 + d.N, g->b1 + 2 * d.N, g->dlt, g->b0);
    if (p->viscosity_sts) {
        // RKL2 super time-stepping of rho V dv/dt = -nu K v from v** over dt (algorithm 3)
        ps = prof_begin(g, g->stream, MHD_KERNEL_STS);
        it[2] = sts_advance(g, p->nu, dt_dev, g->h_ss->dt, g->b1);
        prof_end(g, g->stream, ps);
    } else {
        st = solve(g, &g->ss->alpha_nu, 3, g->b0, g->b1, g->b1, p, &it[2], &ou[2], &rr[2]);
        if (st == MHD_ERR_CUDA) return st;
        if (st != MHD_OK && worst == MHD_OK) worst = st;
    }
    cudaMemcpyAsync(f->vr, g->b1, bytes3 / 3, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(f->vt, g->b1 + d.N, bytes3 / 3, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(f->vp, g->b1 + 2 * d.N, bytes3 / 3, cudaMemcpyDeviceToDevice, g->stream);
    if ((st = check_cuda(g, "mhd_step")) != MHD_OK) return st;
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return check_cuda(g, "mhd_step sync");
    prof_flush(g);
    if (info) {
        const StepScalars& h = *g->h_ss;
        info->dt = h.dt;
        info->cf = h.cf;
        info->cw = h.cw;
        info->alpha_si = h.alpha_si;
        info->alpha_nu = h.alpha_nu;
        for (int q = 0; q < 3; q++) {
            info->iters[q] = it[q];
            info->outer[q] = ou[q];
            info->relres[q] = rr[q];
        }
        info->iters_res = it_res;
        info->relres_res = rr_res;
    }
    return worst;
}

extern "C" mhd_status_t mhd_apply_operator(mhd_grid_t g, double alpha, int ncomp, const double* p, double* q) {
    if (!g) return MHD_ERR_ARG;
    if (whole_grid(g, "mhd_apply_operator") != MHD_OK) return MHD_ERR_ARG;
    if (ncomp < 1 || ncomp > 3 || !p || !q || p == q)
        return set_error(g, MHD_ERR_ARG, "mhd_apply_operator: need 1 <= ncomp <= 3, distinct non-null p, q");
    if (!(alpha >= 0.0)) return set_error(g, MHD_ERR_ARG, "mhd_apply_operator: alpha must be >= 0");
    k_set_alpha<<<1, 1, 0, g->stream>>>(g->ss, alpha);
    apply_operator(g, &g->ss->alpha_user, ncomp, p, q);
    return check_cuda(g, "mhd_apply_operator");
}

extern "C" mhd_status_t mhd_force(mhd_grid_t g, const mhd_fields_t* f, double dt, double* b) {
    if (!g) return MHD_ERR_ARG;
    if (whole_grid(g, "mhd_force") != MHD_OK) return MHD_ERR_ARG;
    if (!fields_ok(f, true) || !b) return set_error(g, MHD_ERR_ARG, "mhd_force: null pointer");
    force(g, f->vr, f->vt, f->vp, nullptr, 0.0, f->br, f->bt, f->bp, nullptr, dt, nullptr, b);
    return check_cuda(g, "mhd_force");
}

extern "C" mhd_status_t mhd_induction(mhd_grid_t g, const double* vbar, double eta, double dt, mhd_fields_t* f) {
    if (!g) return MHD_ERR_ARG;
    if (whole_grid(g, "mhd_induction") != MHD_OK) return MHD_ERR_ARG;
    if (!fields_ok(f, false) || !vbar) return set_error(g, MHD_ERR_ARG, "mhd_induction: null pointer");
    const long long N = g->d.N;
    induction(g, vbar, vbar + N, vbar + 2 * N, nullptr, 0.0, eta, nullptr, dt, f->br, f->bt, f->bp);
    return check_cuda(g, "mhd_induction");
}

extern "C" mhd_status_t pcg_solve(mhd_grid_t g, double alpha, int ncomp, const double* b, double* x,
                                  const mhd_params_t* p, int* iters, int* outer, double* relres) {
    if (!g) return MHD_ERR_ARG;
    if (whole_grid(g, "pcg_solve") != MHD_OK) return MHD_ERR_ARG;
    mhd_status_t st = check_params(g, p);
    if (st != MHD_OK) return st;
    if (ncomp < 1 || ncomp > 3 || !b || !x || (const double*)x == b)
        return set_error(g, MHD_ERR_ARG, "pcg_solve: need 1 <= ncomp <= 3 and distinct non-null b, x");
    if (!(alpha >= 0.0)) return set_error(g, MHD_ERR_ARG, "pcg_solve: alpha must be >= 0");
    NvtxRange range("pcg_solve");
    k_set_alpha<<<1, 1, 0, g->stream>>>(g->ss, alpha);
    return solve(g, &g->ss->alpha_user, ncomp, b, x, x, p, iters, outer, relres);
}

extern "C" mhd_status_t mhd_diagnostics(mhd_grid_t g, const mhd_fields_t* f, double out[5]) {
    if (!g) return MHD_ERR_ARG;
    if (whole_grid(g, "mhd_diagnostics") != MHD_OK) return MHD_ERR_ARG;
    if (!fields_ok(f, true) || !out) return set_error(g, MHD_ERR_ARG, "mhd_diagnostics: null pointer");
    diagnostics(g, f->vr, f->vt, f->vp, f->br, f->bt, f->bp, g->slab_out);
    if (cudaMemcpyAsync(g->h_alpha, g->slab_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
        cudaStreamSynchronize(g->stream) != cudaSuccess)
        return check_cuda(g, "mhd_diagnostics");
    for (int q = 0; q < 5; q++) out[q] = g->h_alpha[q];
    return MHD_OK;
}
