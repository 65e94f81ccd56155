// Mixed-precision (tcgen05 BF16) path.
#include "tc_path.cuh"

kfac_status_t tc_alloc(kfac_pinn_handle*) { return KFAC_OK; }
void tc_free(kfac_pinn_handle*) {}
kfac_status_t tc_factors(kfac_pinn_handle*, cudaStream_t, const double*, const double*, int,
                         const double*, const double*, int, const double*, double*) {
    return KFAC_BAD_ARG;
}
kfac_status_t tc_forward_laplacian(kfac_pinn_handle*, cudaStream_t, const double*, const double*, int,
                                   double*, double*, double*) {
    return KFAC_BAD_ARG;
}
