// Mixed-precision (tcgen05 BF16) path: declarations (implemented in tc_path.cu).
#pragma once
#include "kfac_internal.cuh"

kfac_status_t tc_alloc(kfac_pinn_handle* h);
void tc_free(kfac_pinn_handle* h);
kfac_status_t tc_factors(kfac_pinn_handle* h, cudaStream_t s, const double* theta,
                         const double* X_int, int N_int, const double* f,
                         const double* X_bdy, int N_bdy, const double* g, double* loss);
kfac_status_t tc_forward_laplacian(kfac_pinn_handle* h, cudaStream_t s, const double* theta,
                                   const double* X, int N, double* u, double* grad, double* lap);
// Loss (3 doubles: total, interior, boundary) of theta on the batch, written to dst.
kfac_status_t tc_eval_loss(kfac_pinn_handle* h, cudaStream_t s, const double* theta,
                           const double* X_int, int N_int, const double* f,
                           const double* X_bdy, int N_bdy, const double* g, double* dst);
// Reverse mode of the forward Laplacian on one chunk (N <= max_n_int): dtheta
// (overwritten, or accumulated into), and dX when not NULL.
kfac_status_t tc_forward_laplacian_backward(kfac_pinn_handle* h, cudaStream_t s, const double* theta,
                                            const double* X, int N, const double* du, const double* dgrad,
                                            const double* dlap, double* dtheta, double* dX, bool accumulate);
// J_theta r . v for the interior and boundary residuals of the last kfac_pinn_step's
// batch (forward activations at theta still held by the handle), KFAC*.
kfac_status_t tc_residual_jvp(kfac_pinn_handle* h, cudaStream_t s, const double* v, int N_int, int N_bdy,
                              double* jv_int, double* jv_bdy);
// Self-check of the engine's bounded mbarrier wait (kfac_pinn_check_wait_timeout).
kfac_status_t tc_check_wait(kfac_pinn_handle* h, cudaStream_t s, uint64_t limit_ns);
