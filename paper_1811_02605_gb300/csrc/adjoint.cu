// Adjoint of the zero-beta step (filled in below as it is built).
#include "mhd_internal.cuh"

using namespace mhd;

extern "C" mhd_status_t mhd_adjoint_step(mhd_grid_t g, const mhd_params_t* params, const mhd_fields_t* state_n,
                                         double dt, const mhd_fields_t* adj_np1, mhd_fields_t* adj_n) {
    (void)params; (void)state_n; (void)dt; (void)adj_np1; (void)adj_n;
    return set_error(g, MHD_ERR_ARG, "mhd_adjoint_step: not available in this build");
}
