// Batched persistent PCG (filled in below as it is built).
#include "mhd_internal.cuh"

using namespace mhd;

extern "C" mhd_status_t pcg_solve_batched(int n, const mhd_grid_t* grids, const double* alpha,
                                          const double* const* b, double* const* x,
                                          const mhd_params_t* params, int* iters, double* relres) {
    (void)n; (void)grids; (void)alpha; (void)b; (void)x; (void)params; (void)iters; (void)relres;
    return set_error(nullptr, MHD_ERR_ARG, "pcg_solve_batched: not available in this build");
}
