// Damped Kronecker-sum preconditioning and the parameter update (Sec. 3.4).
//
// With V_A, a and V_B, b from the simultaneous diagonalisation of the damped
// factor pairs (eig.cu: V^T A~_Omega V = I, V^T A~_bdy V = diag(a)),
//     (A~_Omega (x) B~_Omega + A~_bdy (x) B~_bdy)^{-1} vec G
//         = vec( V_B [ (V_B^T G V_A) / (1 + b a^T) ] V_A^T ),
// which is exact because vec(B X A) = (A^T (x) B) vec X (Sec. 2).
#include "kfac_internal.cuh"
#include "tc_path.cuh"

namespace {

__global__ void k_div_kron(double* Y, int nb, int na, const double* wb, const double* wa) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nb * na) return;
    int p = (int)(idx / na), q = (int)(idx % na);
    Y[idx] /= (1.0 + wb[p] * wa[q]);
}

// delta = lr (mu delta_prev + Delta); theta += delta (Sec. 3.4, fixed learning rate).
__global__ void k_update(double* theta, const double* dir, double* delta_prev, long long D, double lr,
                         double mom) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    double dlt = lr * (mom * delta_prev[i] + dir[i]);
    delta_prev[i] = dlt;
    theta[i] += dlt;
}

// Line search over the grid alpha_k = 2^-k, k = 0..LS_GRID-1 (Sec. 3.4).
constexpr int LS_GRID = 31;

// dhat = mu delta_prev + Delta (delta_prev is zero before the first step).
__global__ void k_dhat(const double* dir, const double* delta_prev, double* dhat, long long D, double mom) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    dhat[i] = mom * delta_prev[i] + dir[i];
}

__global__ void k_trial(const double* theta, const double* dhat, double* trial, long long D, double alpha) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    trial[i] = theta[i] + alpha * dhat[i];
}

// alpha* = argmin over the finite trial losses; equal losses keep the larger
// alpha.  With no finite trial the step is skipped and NONFINITE latched.
__device__ int ls_argmin(const double* ls_loss) {
    int best = -1;
    double bl = 0.0;
    for (int k = 0; k < LS_GRID; k++) {
        double v = ls_loss[3 * k];
        if (!isfinite(v)) continue;
        if (best < 0 || v < bl) {
            best = k;
            bl = v;
        }
    }
    return best;
}

// delta = alpha* dhat; theta += delta.
__global__ void k_ls_apply(double* theta, const double* dhat, double* delta_prev, long long D,
                           const double* ls_loss, int* status) {
    __shared__ int best;
    if (threadIdx.x == 0) {
        best = ls_argmin(ls_loss);
        if (best < 0 && blockIdx.x == 0) latch_status(status, KFAC_NONFINITE);
    }
    __syncthreads();
    const double alpha = best < 0 ? 0.0 : ldexp(1.0, -best);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < D;
         i += (long long)gridDim.x * blockDim.x) {
        double dlt = alpha * dhat[i];
        delta_prev[i] = dlt;
        theta[i] += dlt;
    }
}

kfac_status_t precondition_impl(kfac_pinn_handle* h, cudaStream_t s, const double* grad, double* dir) {
    // The mixed-precision path applies the (FP64) inverse with FP32 products:
    // its gradient already carries BF16-level errors.
    const bool f32 = (h->cfg.precision == KFAC_MIXED_BF16);
    for (int l = 1; l <= h->cfg.L; l++) {
        const int na = h->dims[l - 1] + 1, nb = h->dims[l];
        const double* G = grad + h->woff[l - 1];
        double* X1 = h->tmp;
        double* Y = h->tmp + (size_t)nb * na;
        const double* VA = h->VA[l - 1];
        const double* VB = h->VB[l - 1];
        kfac_status_t st;
        // X1 = V_B^T G      (nb x na, row-major)
        st = dgemm_strided(h, s, nb, na, nb, VB, 1, nb, G, 1, nb, X1, na, 1, 1.0, 0.0, f32);
        if (st) return st;
        // Y = X1 V_A, then the element-wise division by 1 + b a^T
        st = dgemm_strided(h, s, nb, na, na, X1, na, 1, VA, na, 1, Y, na, 1, 1.0, 0.0, f32);
        if (st) return st;
        k_div_kron<<<ceil_div_u((long long)nb * na, 256), 256, 0, s>>>(Y, nb, na, h->wb[l - 1], h->wa[l - 1]);
        KFAC_LAUNCH_CHECK(h);
        // X1 = V_B Y
        st = dgemm_strided(h, s, nb, na, nb, VB, nb, 1, Y, na, 1, X1, na, 1, 1.0, 0.0, f32);
        if (st) return st;
        // Delta = -X1 V_A^T, stored column-stacked like theta
        st = dgemm_strided(h, s, nb, na, na, X1, na, 1, VA, 1, na, dir + h->woff[l - 1], 1, nb, -1.0, 0.0, f32);
        if (st) return st;
    }
    return KFAC_OK;
}

}  // namespace

size_t linalg_workspace_elems(const kfac_pinn_handle*) { return 1; }

kfac_status_t linalg_invert(kfac_pinn_handle* h, cudaStream_t s) {
    // algorithmic work of the generalized eigendecomposition, about 10 n^3 per factor pair
    double work = 0.0;
    for (int l = 1; l <= h->cfg.L; l++) {
        double na = h->dims[l - 1] + 1, nb = h->dims[l];
        work += 10.0 * (na * na * na + nb * nb * nb);
    }
    timer_begin(h, KFAC_KC_EIG, s);
    kfac_status_t st = eig_run(h, s);
    timer_end(h, KFAC_KC_EIG, s, work);
    return st;
}

kfac_status_t linalg_precondition(kfac_pinn_handle* h, cudaStream_t s, const double* grad, double* dir) {
    double work = 0.0;
    for (int l = 1; l <= h->cfg.L; l++) {
        double na = h->dims[l - 1] + 1, nb = h->dims[l];
        work += 4.0 * (nb * nb * na + nb * na * na);
    }
    timer_begin(h, KFAC_KC_PRECOND, s);
    kfac_status_t r = precondition_impl(h, s, grad, dir);
    timer_end(h, KFAC_KC_PRECOND, s, work);
    return r;
}

kfac_status_t linalg_update(kfac_pinn_handle* h, cudaStream_t s, double* theta) {
    k_update<<<ceil_div_u(h->D, 256), 256, 0, s>>>(theta, h->dir, h->delta_prev, h->D, h->cfg.lr,
                                                   h->cfg.momentum);
    KFAC_LAUNCH_CHECK(h);
    return KFAC_OK;
}

kfac_status_t linalg_line_search_update(kfac_pinn_handle* h, cudaStream_t s, double* theta, const double* X_int,
                                        int N_int, const double* f, const double* X_bdy, int N_bdy,
                                        const double* g) {
    const unsigned blocks = ceil_div_u(h->D, 256);
    k_dhat<<<blocks, 256, 0, s>>>(h->dir, h->delta_prev, h->dhat, h->D, h->cfg.momentum);
    KFAC_LAUNCH_CHECK(h);
    const bool mixed = (h->cfg.precision == KFAC_MIXED_BF16);
    for (int k = 0; k < LS_GRID; k++) {
        k_trial<<<blocks, 256, 0, s>>>(theta, h->dhat, h->trial, h->D, ldexp(1.0, -k));
        KFAC_LAUNCH_CHECK(h);
        double* dst = h->ls_loss + 3 * k;
        kfac_status_t st = mixed ? tc_eval_loss(h, s, h->trial, X_int, N_int, f, X_bdy, N_bdy, g, dst)
                                 : fp64_eval_loss(h, s, h->trial, X_int, N_int, f, X_bdy, N_bdy, g, dst);
        if (st) return st;
    }
    unsigned ab = blocks < (unsigned)(4 * h->sm_count) ? blocks : (unsigned)(4 * h->sm_count);
    k_ls_apply<<<ab, 256, 0, s>>>(theta, h->dhat, h->delta_prev, h->D, h->ls_loss, h->status);
    KFAC_LAUNCH_CHECK(h);
    return KFAC_OK;
}
