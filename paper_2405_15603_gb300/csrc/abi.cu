// C-ABI entry points of libkfacpinn.so (declared in include/kfac_pinn.h).
#include <stdlib.h>
#include <string.h>
#include <math.h>

#include <atomic>
#include <vector>

#include "kfac_internal.cuh"
#include "tc_path.cuh"

namespace {

}  // namespace

// Allocation-failure injection (kfac_pinn_inject_alloc_failure): the number of
// device allocations still to succeed before one fails, or -1 for none.
static std::atomic<long long> g_alloc_fail_in{-1};

kfac_status_t kfac_device_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 1;
    long long left = g_alloc_fail_in.load();
    while (left >= 0) {
        if (g_alloc_fail_in.compare_exchange_weak(left, left - 1)) {
            if (left == 0) return KFAC_OOM;      // the injected failure: nothing allocated
            break;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); *p = nullptr; return KFAC_OOM; }
    if (e != cudaSuccess) { *p = nullptr; return KFAC_CUDA_ERROR; }
    return KFAC_OK;
}

// The network and operator part of a configuration: d, L, widths (each at
// most 1023, the last 1, d + 1 at most 1024) and the operator.
bool kfac_valid_network(const kfac_config_t* c) {
    if (!c) return false;
    if (c->d < 1 || c->L < 1 || c->L > KFAC_MAX_LAYERS) return false;
    for (int l = 0; l < c->L; l++)
        if (c->widths[l] < 1 || c->widths[l] > 1023) return false;
    if (c->widths[c->L - 1] != 1) return false;
    if (c->d + 1 > 1024) return false;
    if (c->op != KFAC_OP_LAPLACE && c->op != KFAC_OP_HEAT && c->op != KFAC_OP_GENERAL) return false;
    if (c->op == KFAC_OP_HEAT && c->d < 2) return false;
    return true;
}

namespace {

// Cholesky factor of the M x M symmetric matrix W (row-major, lower
// triangle into Lw); false unless W is positive definite.
bool host_cholesky(const double* W, int M, double* Lw) {
    for (int i = 0; i < M * M; i++) Lw[i] = 0.0;
    for (int j = 0; j < M; j++) {
        double dsum = W[j * M + j];
        for (int k = 0; k < j; k++) dsum -= Lw[j * M + k] * Lw[j * M + k];
        if (!(dsum > 0.0) || !isfinite(dsum)) return false;
        const double ljj = sqrt(dsum);
        Lw[j * M + j] = ljj;
        for (int i = j + 1; i < M; i++) {
            double v = W[i * M + j];
            for (int k = 0; k < j; k++) v -= Lw[i * M + k] * Lw[j * M + k];
            Lw[i * M + j] = v / ljj;
        }
    }
    return true;
}

// The general residual: 1 <= M <= KFAC_MAX_RESIDUALS, finite b, Q symmetric in
// its last two indices, W symmetric positive definite; the SIMT precisions,
// the LAPLACE or HEAT operator (coordinate tangents), KFAC-expand, and the
// FIXED or LINE_SEARCH update.
bool valid_residual(const kfac_config_t* c) {
    const kfac_residual_t* r = c->residual;
    if (r->M < 1 || r->M > KFAC_MAX_RESIDUALS || !r->b) return false;
    if (c->op != KFAC_OP_LAPLACE && c->op != KFAC_OP_HEAT) return false;
    if (c->precision != KFAC_FP64 && c->precision != KFAC_FP32) return false;
    if (c->variant != KFAC_EXPAND || c->update == KFAC_UPDATE_AUTO) return false;
    const int M = r->M, S = c->d + 2;
    for (int i = 0; i < M * S; i++)
        if (!isfinite(r->b[i])) return false;
    if (r->Q) {
        for (int k = 0; k < M; k++)
            for (int a = 0; a < S; a++)
                for (int b = 0; b < S; b++) {
                    const double q = r->Q[((size_t)k * S + a) * S + b];
                    if (!isfinite(q) || fabs(q - r->Q[((size_t)k * S + b) * S + a]) > 1e-12 * (1.0 + fabs(q)))
                        return false;
                }
    }
    if (r->W) {
        for (int i = 0; i < M; i++)
            for (int j = 0; j < M; j++)
                if (!isfinite(r->W[i * M + j]) || fabs(r->W[i * M + j] - r->W[j * M + i]) >
                                                       1e-12 * (1.0 + fabs(r->W[i * M + j])))
                    return false;
        std::vector<double> Lw((size_t)M * M);
        if (!host_cholesky(r->W, M, Lw.data())) return false;
    }
    return true;
}

bool valid_config(const kfac_config_t* c) {
    if (!kfac_valid_network(c)) return false;
    if (c->op == KFAC_OP_GENERAL) {
        if (!c->op_coef || c->variant != KFAC_EXPAND) return false;
        double mx = 0.0;
        for (int i = 0; i < c->d * c->d; i++) {
            if (!isfinite(c->op_coef[i])) return false;
            mx = fmax(mx, fabs(c->op_coef[i]));
        }
        for (int i = 0; i < c->d; i++)
            for (int j = 0; j < i; j++)
                if (fabs(c->op_coef[i * c->d + j] - c->op_coef[j * c->d + i]) > 1e-12 * mx) return false;
    }
    if (c->precision != KFAC_FP64 && c->precision != KFAC_MIXED_BF16 && c->precision != KFAC_MIXED_SPLIT &&
        c->precision != KFAC_FP32)
        return false;
    if (c->residual && !valid_residual(c)) return false;
    if (c->variant != KFAC_EXPAND && c->variant != KFAC_REDUCE) return false;
    if (!(c->beta >= 0.0 && c->beta < 1.0)) return false;
    if (!(c->lambda > 0.0) || !isfinite(c->lambda)) return false;
    if (!isfinite(c->lr) || !isfinite(c->momentum) || !isfinite(c->kappa)) return false;
    if (c->max_n_int < 1 || c->max_n_bdy < 1) return false;
    if (c->update < KFAC_UPDATE_FIXED || c->update > KFAC_UPDATE_AUTO) return false;
    if (c->eig_sm_budget < 0) return false;
    long long rows = (long long)(c->d + 2) * c->max_n_int;
    if (rows > (1LL << 30)) return false;
    return true;
}

kfac_status_t dalloc_bytes(void** p, size_t bytes) { return kfac_device_alloc(p, bytes); }

template <class T>
kfac_status_t dalloc(T** p, size_t elems) {
    void* v = nullptr;
    kfac_status_t st = dalloc_bytes(&v, elems * sizeof(T));
    *p = (T*)v;
    return st;
}

// Symmetric eigendecomposition C = Q diag(lam) Q^T on the host (cyclic
// Jacobi rotations; C is small and read once per handle).  Q row-major,
// Q[i * d + m] = component i of eigenvector m.
void host_sym_eig(const double* C, int d, std::vector<double>& Q, std::vector<double>& lam) {
    std::vector<double> A(C, C + (size_t)d * d);
    Q.assign((size_t)d * d, 0.0);
    for (int i = 0; i < d; i++) Q[(size_t)i * d + i] = 1.0;
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < d; i++)
            for (int j = 0; j < d; j++) {
                double a = A[(size_t)i * d + j] * A[(size_t)i * d + j];
                tot += a;
                if (i != j) off += a;
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < d; p++)
            for (int q = p + 1; q < d; q++) {
                const double apq = A[(size_t)p * d + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * d + p], aqq = A[(size_t)q * d + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < d; k++) {     // columns p, q
                    const double akp = A[(size_t)k * d + p], akq = A[(size_t)k * d + q];
                    A[(size_t)k * d + p] = c * akp - sn * akq;
                    A[(size_t)k * d + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < d; k++) {     // rows p, q
                    const double apk = A[(size_t)p * d + k], aqk = A[(size_t)q * d + k];
                    A[(size_t)p * d + k] = c * apk - sn * aqk;
                    A[(size_t)q * d + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < d; k++) {
                    const double qkp = Q[(size_t)k * d + p], qkq = Q[(size_t)k * d + q];
                    Q[(size_t)k * d + p] = c * qkp - sn * qkq;
                    Q[(size_t)k * d + q] = sn * qkp + c * qkq;
                }
            }
    }
    lam.resize(d);
    for (int i = 0; i < d; i++) lam[i] = A[(size_t)i * d + i];
}

// Operator description on the device: residual coefficients, tangent
// directions and channel weights of the second-order column.
kfac_status_t setup_operator(kfac_pinn_handle* h) {
    const int d = h->dims[0];
    std::vector<double> w(d, 1.0);
    h->cT = 0.0;
    h->cD = -1.0;
    if (h->cfg.op == KFAC_OP_HEAT) {
        h->cT = 1.0;
        h->cD = -h->cfg.kappa;
        w[0] = 0.0;                     // time is outside the spatial Laplacian
    }
    kfac_status_t st;
    if (h->cfg.op == KFAC_OP_GENERAL) {
        std::vector<double> Q, lam;
        host_sym_eig(h->cfg.op_coef, d, Q, lam);
        w = lam;
        h->cD = 1.0;
        if ((st = dalloc(&h->opQ, (size_t)d * d))) return st;
        if ((st = dalloc(&h->w1q, (size_t)h->dims[1] * d))) return st;
        if ((st = dalloc(&h->w1q2, (size_t)h->dims[1] * d))) return st;
        KFAC_CUDA_TRY(cudaMemcpy(h->opQ, Q.data(), sizeof(double) * d * d, cudaMemcpyHostToDevice));
    }
    h->cfg.op_coef = nullptr;           // read only here
    h->fM = 1;
    if (h->cfg.residual) {
        const kfac_residual_t* r = h->cfg.residual;
        const int M = r->M, S = d + 2;
        std::vector<double> coef((size_t)M * S + 2 * (size_t)M * M + (r->Q ? (size_t)M * S * S : 0), 0.0);
        double* b = coef.data();
        double* W = b + (size_t)M * S;
        double* Lw = W + (size_t)M * M;
        for (int i = 0; i < M * S; i++) b[i] = r->b[i];
        for (int i = 0; i < M; i++) W[i * M + i] = 1.0;
        if (r->W)
            for (int i = 0; i < M * M; i++) W[i] = r->W[i];
        if (!host_cholesky(W, M, Lw)) return KFAC_BAD_ARG;
        if (r->Q)
            for (size_t i = 0; i < (size_t)M * S * S; i++) Lw[(size_t)M * M + i] = r->Q[i];
        if ((st = dalloc(&h->res_coef, coef.size()))) return st;
        KFAC_CUDA_TRY(cudaMemcpy(h->res_coef, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice));
        if ((st = dalloc(&h->res_r, (size_t)h->cfg.max_n_int * M))) return st;
        h->res_M = M;
        h->res_has_Q = r->Q ? 1 : 0;
        h->fM = M;
    }
    h->cfg.residual = nullptr;          // read only here
    std::vector<float> wf(w.begin(), w.end());
    if ((st = dalloc(&h->chw64, (size_t)d))) return st;
    if ((st = dalloc(&h->chw32, (size_t)d))) return st;
    KFAC_CUDA_TRY(cudaMemcpy(h->chw64, w.data(), sizeof(double) * d, cudaMemcpyHostToDevice));
    KFAC_CUDA_TRY(cudaMemcpy(h->chw32, wf.data(), sizeof(float) * d, cudaMemcpyHostToDevice));
    return KFAC_OK;
}

void free_pass(PassBuffers& pb) {
    for (int l = 0; l < KFAC_MAX_LAYERS; l++) {
        cudaFree(pb.Z[l]);
        cudaFree(pb.T[l]);
        cudaFree(pb.Zb[l]);
    }
    cudaFree(pb.r);
    cudaFree(pb.red_a);
    cudaFree(pb.red_g);
}

void free_handle(kfac_pinn_handle* h) {
    if (!h) return;
    timers_free(h);
    free_pass(h->in);
    free_pass(h->bd);
    tc_free(h);
    eig_free(h);
    cudaFree(h->grad);
    cudaFree(h->dir);
    cudaFree(h->delta_prev);
    cudaFree(h->dhat);
    cudaFree(h->trial);
    cudaFree(h->ls_loss);
    cudaFree(h->ks_jv);
    cudaFree(h->ks_part);
    cudaFree(h->coef);
    cudaFree(h->opQ);
    cudaFree(h->chw64);
    cudaFree(h->chw32);
    cudaFree(h->res_coef);
    cudaFree(h->res_r);
    cudaFree(h->w1q);
    cudaFree(h->w1q2);
    for (int w = 0; w < 4; w++)
        for (int l = 0; l < KFAC_MAX_LAYERS; l++) cudaFree(h->fac[w][l]);
    for (int l = 0; l < KFAC_MAX_LAYERS; l++) {
        cudaFree(h->VA[l]);
        cudaFree(h->wa[l]);
        cudaFree(h->VB[l]);
        cudaFree(h->wb[l]);
    }
    cudaFree(h->loss);
    cudaFree(h->part);
    cudaFree(h->lin);
    cudaFree(h->tmp);
    cudaFree(h->status);
    cudaFree(h->stage);
    for (cudaEvent_t e : h->tune_ev)
        if (e) cudaEventDestroy(e);
    free(h);
}

kfac_status_t alloc_pass(kfac_pinn_handle* h, PassBuffers& pb, int N, int S) {
    pb.N = N;
    pb.S = S;
    const int L = h->cfg.L;
    kfac_status_t st;
    int maxw = 0;
    if (is_mixed(h)) {   // the mixed path keeps its own BF16 activations
        return dalloc(&pb.r, (size_t)N);
    }
    const size_t eb = simt_elem_bytes(h);   // FP64 or FP32 activations
    for (int l = 1; l <= L; l++) {
        size_t e = (size_t)S * N * h->dims[l] * eb;
        if ((st = dalloc_bytes(&pb.Z[l - 1], e))) return st;
        if ((st = dalloc_bytes(&pb.Zb[l - 1], e))) return st;
        if (l < L && (st = dalloc_bytes(&pb.T[l - 1], e))) return st;
        if (h->dims[l] > maxw) maxw = h->dims[l];
    }
    if (h->dims[0] + 1 > maxw) maxw = h->dims[0] + 1;
    for (int l = 0; l < L; l++)
        if (h->dims[l] + 1 > maxw) maxw = h->dims[l] + 1;
    if ((st = dalloc(&pb.r, (size_t)N))) return st;
    if (S > 1 && h->cfg.variant == KFAC_REDUCE) {
        if ((st = dalloc_bytes(&pb.red_a, (size_t)N * maxw * eb))) return st;
        if ((st = dalloc_bytes(&pb.red_g, (size_t)N * maxw * eb))) return st;
    }
    return KFAC_OK;
}

size_t partial_elems_needed(const kfac_pinn_handle* h) {
    // Enough for the split-K partials of every Gram / weight-gradient GEMM.
    size_t need = 0;
    const int S = h->S;
    for (int l = 1; l <= h->cfg.L; l++) {
        int nin = h->dims[l - 1] + 1, hout = h->dims[l];
        int K = S * h->cfg.max_n_int;
        int dimsP[3] = {hout, nin, hout};
        int dimsQ[3] = {nin, nin, hout};
        for (int t = 0; t < 3; t++) {
            long long tiles = (long long)((dimsP[t] + 63) / 64) * ((dimsQ[t] + 63) / 64);
            long long want = (2LL * h->sm_count + tiles - 1) / tiles;
            long long maxs = (K + 511) / 512;
            if (want > maxs) want = maxs;
            if (want < 1) want = 1;
            size_t e = (size_t)want * dimsP[t] * dimsQ[t];
            if (e > need) need = e;
        }
    }
    return need;
}

__global__ void k_init_factor(double* M, int n, double diag) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)n * n) return;
    M[i] = ((int)(i / n) == (int)(i % n)) ? diag : 0.0;
}

kfac_status_t reset_state(kfac_pinn_handle* h, cudaStream_t s) {
    double diag = h->cfg.factor_init_identity ? 1.0 : 0.0;
    for (int l = 1; l <= h->cfg.L; l++) {
        int na = h->dims[l - 1] + 1, nb = h->dims[l];
        for (int w = 0; w < 4; w++) {
            int n = (w == KFAC_A_INT || w == KFAC_A_BDY) ? na : nb;
            k_init_factor<<<ceil_div_u((long long)n * n, 256), 256, 0, s>>>(h->fac[w][l - 1], n, diag);
            KFAC_LAUNCH_CHECK(h);
        }
    }
    KFAC_CUDA_TRY(cudaMemsetAsync(h->delta_prev, 0, h->D * sizeof(double), s));
    KFAC_CUDA_TRY(cudaMemsetAsync(h->dir, 0, h->D * sizeof(double), s));
    KFAC_CUDA_TRY(cudaMemsetAsync(h->grad, 0, h->D * sizeof(double), s));
    h->t = 0;
    h->have_inverse = 0;
    h->have_direction = 0;
    return KFAC_OK;
}

inline cudaStream_t S_(void* p) { return (cudaStream_t)p; }

kfac_status_t check_batch(kfac_pinn_handle* h, const void* X_int, int N_int, const void* f,
                          const void* X_bdy, int N_bdy, const void* g) {
    if (!h) return KFAC_BAD_ARG;
    if (!X_int || !f || !X_bdy || !g) return KFAC_BAD_ARG;
    if (N_int < 1 || N_int > h->cfg.max_n_int) return KFAC_BAD_ARG;
    if (N_bdy < 1 || N_bdy > h->cfg.max_n_bdy) return KFAC_BAD_ARG;
    return KFAC_OK;
}

kfac_status_t run_factors(kfac_pinn_handle* h, cudaStream_t s, const double* theta,
                          const double* X_int, int N_int, const double* f,
                          const double* X_bdy, int N_bdy, const double* g, double* loss) {
    h->fwd_valid = 0;       // the pass buffers are about to be overwritten
    if (is_mixed(h))
        return tc_factors(h, s, theta, X_int, N_int, f, X_bdy, N_bdy, g, loss);
    kfac_status_t st;
    const int S = h->S;
    if (h->res_M > 0) {      // general residual: M + 1 seeded interior adjoint passes
        if ((st = simt_forward(h, s, theta, X_int, N_int, h->in, S))) return st;
        if ((st = simt_residual_general(h, s, N_int, f))) return st;
        if ((st = simt_forward(h, s, theta, X_bdy, N_bdy, h->bd, 1))) return st;
        if ((st = simt_residual_and_seed(h, s, h->bd, N_bdy, 1, g, false))) return st;
        if ((st = simt_backward(h, s, theta, h->bd, N_bdy, 1))) return st;
        if ((st = fp64_loss(h, s, N_int, N_bdy, loss))) return st;
        return simt_backward_and_factors_general(h, s, theta, X_int, N_int, f, X_bdy, N_bdy);
    }
    if ((st = simt_forward(h, s, theta, X_int, N_int, h->in, S))) return st;
    if ((st = simt_residual_and_seed(h, s, h->in, N_int, S, f, true))) return st;
    if ((st = simt_backward(h, s, theta, h->in, N_int, S))) return st;
    if ((st = simt_forward(h, s, theta, X_bdy, N_bdy, h->bd, 1))) return st;
    if ((st = simt_residual_and_seed(h, s, h->bd, N_bdy, 1, g, false))) return st;
    if ((st = simt_backward(h, s, theta, h->bd, N_bdy, 1))) return st;
    if ((st = fp64_loss(h, s, N_int, N_bdy, loss))) return st;
    if ((st = simt_grad_and_factors(h, s, X_int, N_int, X_bdy, N_bdy))) return st;
    return KFAC_OK;
}

constexpr int TIMER_CAP = 4096;

void timer_fold(kfac_pinn_handle* h, int cls) {
    auto& t = h->timers[cls];
    if (t.n == 0) return;
    cudaEventSynchronize(t.ev[2 * t.n - 1]);
    for (int i = 0; i < t.n; i++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.ev[2 * i], t.ev[2 * i + 1]) == cudaSuccess) t.ms += ms;
    }
    t.n = 0;
}

}  // namespace

void timer_begin(kfac_pinn_handle* h, int cls, cudaStream_t s) {
    if (!h->timing) return;
    auto& t = h->timers[cls];
    if (t.n >= t.cap) timer_fold(h, cls);
    cudaEventRecord(t.ev[2 * t.n], s);
}

void timer_end(kfac_pinn_handle* h, int cls, cudaStream_t s, double work, double exec) {
    if (!h->timing) return;
    auto& t = h->timers[cls];
    cudaEventRecord(t.ev[2 * t.n + 1], s);
    t.n++;
    t.launches++;
    t.work += work;
    t.exec += exec < 0.0 ? work : exec;
}

void timers_free(kfac_pinn_handle* h) {
    for (int c = 0; c < KFAC_KC_COUNT; c++) {
        auto& t = h->timers[c];
        if (t.ev) {
            for (int i = 0; i < 2 * t.cap; i++) cudaEventDestroy(t.ev[i]);
            free(t.ev);
        }
        t.ev = nullptr;
        t.cap = t.n = 0;
    }
}

namespace {
thread_local int g_last_cuda_error = 0;
}

void kfac_record_cuda_error(cudaError_t e) { g_last_cuda_error = (int)e; }

extern "C" {

int kfac_pinn_last_cuda_error(void) { return g_last_cuda_error; }

const char* kfac_pinn_last_cuda_error_string(void) {
    return cudaGetErrorString((cudaError_t)g_last_cuda_error);
}

kfac_status_t kfac_pinn_timing_enable(kfac_handle_t h, int enable) {
    if (!h) return KFAC_BAD_ARG;
    if (enable) {
        for (int c = 0; c < KFAC_KC_COUNT; c++) {
            auto& t = h->timers[c];
            if (!t.ev) {
                t.ev = (cudaEvent_t*)calloc(2 * TIMER_CAP, sizeof(cudaEvent_t));
                if (!t.ev) return KFAC_OOM;
                for (int i = 0; i < 2 * TIMER_CAP; i++)
                    KFAC_CUDA_TRY(cudaEventCreate(&t.ev[i]));
                t.cap = TIMER_CAP;
            }
            t.n = 0;
            t.launches = 0;
            t.work = 0.0;
            t.exec = 0.0;
            t.ms = 0.0;
        }
    }
    h->timing = enable ? 1 : 0;
    return KFAC_OK;
}

kfac_status_t kfac_pinn_timing_read_ex(kfac_handle_t h, int kernel_class, double* total_ms, int64_t* launches,
                                       double* work, double* exec_work) {
    if (!h || kernel_class < 0 || kernel_class >= KFAC_KC_COUNT) return KFAC_BAD_ARG;
    auto& t = h->timers[kernel_class];
    if (t.ev) timer_fold(h, kernel_class);
    if (total_ms) *total_ms = t.ms;
    if (launches) *launches = t.launches;
    if (work) *work = t.work;
    if (exec_work) *exec_work = t.exec;
    t.ms = 0.0;
    t.launches = 0;
    t.work = 0.0;
    t.exec = 0.0;
    return KFAC_OK;
}

kfac_status_t kfac_pinn_timing_read(kfac_handle_t h, int kernel_class, double* total_ms,
                                    int64_t* launches, double* work) {
    return kfac_pinn_timing_read_ex(h, kernel_class, total_ms, launches, work, nullptr);
}


int64_t kfac_pinn_param_count(const kfac_config_t* cfg) {
    if (!valid_config(cfg)) return -1;
    int64_t D = 0;
    int prev = cfg->d;
    for (int l = 0; l < cfg->L; l++) {
        D += (int64_t)cfg->widths[l] * (prev + 1);
        prev = cfg->widths[l];
    }
    return D;
}

const char* kfac_pinn_status_string(kfac_status_t st) {
    switch (st) {
        case KFAC_OK: return "KFAC_OK";
        case KFAC_BAD_ARG: return "KFAC_BAD_ARG";
        case KFAC_NOT_PD: return "KFAC_NOT_PD";
        case KFAC_NONFINITE: return "KFAC_NONFINITE";
        case KFAC_TIMEOUT: return "KFAC_TIMEOUT";
        case KFAC_OOM: return "KFAC_OOM";
        case KFAC_CUDA_ERROR: return "KFAC_CUDA_ERROR";
        case KFAC_NOT_READY: return "KFAC_NOT_READY";
    }
    return "KFAC_UNKNOWN";
}

kfac_status_t kfac_pinn_check_wait_timeout(kfac_handle_t h, void* stream, int kind, int limit_ms) {
    if (!h || limit_ms < 1 || limit_ms > 10000 || (kind != 0 && kind != 1)) return KFAC_BAD_ARG;
    const uint64_t ns = (uint64_t)limit_ms * 1000000ull;
    return kind == 0 ? eig_check_wait(h, S_(stream), ns) : tc_check_wait(h, S_(stream), ns);
}

kfac_status_t kfac_pinn_inject_alloc_failure(long long n) {
    if (n < -1) return KFAC_BAD_ARG;
    g_alloc_fail_in.store(n);
    return KFAC_OK;
}

kfac_status_t kfac_pinn_create(const kfac_config_t* cfg, kfac_handle_t* out) {
    if (!out) return KFAC_BAD_ARG;
    *out = nullptr;
    if (!valid_config(cfg)) return KFAC_BAD_ARG;
    kfac_pinn_handle* h = (kfac_pinn_handle*)calloc(1, sizeof(kfac_pinn_handle));
    if (!h) return KFAC_OOM;
    h->cfg = *cfg;
    h->cta_pairs = 0;
    KFAC_CUDA_TRY(cudaGetDevice(&h->device));
    KFAC_CUDA_TRY(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device));
    h->dims[0] = cfg->d;
    for (int l = 0; l < cfg->L; l++) h->dims[l + 1] = cfg->widths[l];
    h->woff[0] = 0;
    for (int l = 1; l <= cfg->L; l++)
        h->woff[l] = h->woff[l - 1] + (int64_t)h->dims[l] * (h->dims[l - 1] + 1);
    h->D = h->woff[cfg->L];
    h->S = cfg->d + 2;

    kfac_status_t st = KFAC_OK;
#define TRY(x) do { st = (x); if (st != KFAC_OK) { free_handle(h); return st; } } while (0)
    TRY(setup_operator(h));
    TRY(alloc_pass(h, h->in, cfg->max_n_int, h->S));
    TRY(alloc_pass(h, h->bd, cfg->max_n_bdy, 1));
    TRY(dalloc(&h->grad, (size_t)h->D));
    TRY(dalloc(&h->dir, (size_t)h->D));
    TRY(dalloc(&h->delta_prev, (size_t)h->D));
    if (cfg->update == KFAC_UPDATE_LINE_SEARCH) {
        TRY(dalloc(&h->dhat, (size_t)h->D));
        TRY(dalloc(&h->trial, (size_t)h->D));
        TRY(dalloc(&h->ls_loss, 3 * 31));
    }
    if (cfg->update == KFAC_UPDATE_AUTO) {
        TRY(dalloc(&h->ks_jv, 2 * ((size_t)cfg->max_n_int + cfg->max_n_bdy)));
        TRY(dalloc(&h->ks_part, linalg_auto_part_elems()));
    }
    TRY(dalloc(&h->coef, 8));
    size_t tmp = 0;
    for (int l = 1; l <= cfg->L; l++) {
        size_t na = h->dims[l - 1] + 1, nb = h->dims[l];
        TRY(dalloc(&h->fac[KFAC_A_INT][l - 1], na * na));
        TRY(dalloc(&h->fac[KFAC_A_BDY][l - 1], na * na));
        TRY(dalloc(&h->fac[KFAC_B_INT][l - 1], nb * nb));
        TRY(dalloc(&h->fac[KFAC_B_BDY][l - 1], nb * nb));
        TRY(dalloc(&h->VA[l - 1], na * na));
        TRY(dalloc(&h->wa[l - 1], na));
        TRY(dalloc(&h->VB[l - 1], nb * nb));
        TRY(dalloc(&h->wb[l - 1], nb));
        if (2 * na * nb > tmp) tmp = 2 * na * nb;
    }
    // the mixed path's batched preconditioning holds every layer's two
    // scratch matrices at once
    if (is_mixed(h)) tmp = std::max(tmp, 2 * (size_t)h->D);
    h->tmp_elems = tmp;
    TRY(dalloc(&h->tmp, tmp));
    TRY(dalloc(&h->loss, 3));
    h->part_elems = partial_elems_needed(h);
    TRY(dalloc(&h->part, h->part_elems));
    h->lin_elems = linalg_workspace_elems(h);
    TRY(dalloc(&h->lin, h->lin_elems));
    TRY(dalloc(&h->status, 1));
    h->stage_elems = (size_t)cfg->max_n_int * (cfg->d + h->fM) + (size_t)cfg->max_n_bdy * (cfg->d + 1) + 8;
    TRY(dalloc(&h->stage, h->stage_elems));
    if (is_mixed(h)) TRY(tc_alloc(h));
    TRY(eig_alloc(h));
    if (cudaMemset(h->status, 0, sizeof(int)) != cudaSuccess) { free_handle(h); return KFAC_CUDA_ERROR; }
    TRY(reset_state(h, 0));
    if (cudaDeviceSynchronize() != cudaSuccess) { free_handle(h); return KFAC_CUDA_ERROR; }
#undef TRY
    *out = h;
    return KFAC_OK;
}

kfac_status_t kfac_pinn_destroy(kfac_handle_t h) {
    if (!h) return KFAC_BAD_ARG;
    cudaDeviceSynchronize();
    handle_graph_free(h);
    free_handle(h);
    return KFAC_OK;
}

kfac_status_t kfac_pinn_reset(kfac_handle_t h, void* stream) {
    if (!h) return KFAC_BAD_ARG;
    return reset_state(h, S_(stream));
}

kfac_status_t kfac_pinn_forward_laplacian(kfac_handle_t h, void* stream, const double* theta,
                                          const double* X, int N, double* u, double* grad,
                                          double* lap) {
    if (!h || !theta || N < 0) return KFAC_BAD_ARG;
    if (N == 0) return KFAC_OK;                  // nothing to evaluate
    if (!X || !u) return KFAC_BAD_ARG;
    cudaStream_t s = S_(stream);
    const int S = h->S, d = h->dims[0];
    for (int off = 0; off < N; off += h->cfg.max_n_int) {
        int n = N - off < h->cfg.max_n_int ? N - off : h->cfg.max_n_int;
        kfac_status_t st;
        if (is_mixed(h)) {
            st = tc_forward_laplacian(h, s, theta, X + (long long)off * d, n, u + off,
                                      grad ? grad + (long long)off * d : nullptr, lap ? lap + off : nullptr);
        } else {
            st = simt_forward(h, s, theta, X + (long long)off * d, n, h->in, S);
            if (st == KFAC_OK)
                st = simt_extract_outputs(h, s, h->in, n, S, u + off,
                                          grad ? grad + (long long)off * d : nullptr, lap ? lap + off : nullptr);
        }
        if (st) return st;
    }
    h->fwd_valid = h->store_forward && !is_mixed(h) && N <= h->cfg.max_n_int;
    h->fwd_theta = theta;
    h->fwd_X = X;
    h->fwd_N = N;
    return KFAC_OK;
}

kfac_status_t kfac_pinn_forward_laplacian_backward(kfac_handle_t h, void* stream, const double* theta,
                                                   const double* X, int N, const double* du,
                                                   const double* dgrad, const double* dlap, double* dtheta,
                                                   double* dX) {
    if (!h || !theta || !X || !dtheta || N < 0) return KFAC_BAD_ARG;
    cudaStream_t s = S_(stream);
    const int d = h->dims[0];
    if (N == 0) {
        KFAC_CUDA_TRY(cudaMemsetAsync(dtheta, 0, h->D * sizeof(double), s));
        return KFAC_OK;
    }
    if (is_mixed(h)) {
        h->fwd_valid = 0;
        for (int off = 0; off < N; off += h->cfg.max_n_int) {
            int n = N - off < h->cfg.max_n_int ? N - off : h->cfg.max_n_int;
            kfac_status_t st = tc_forward_laplacian_backward(
                h, s, theta, X + (long long)off * d, n, du ? du + off : nullptr,
                dgrad ? dgrad + (long long)off * d : nullptr, dlap ? dlap + off : nullptr, dtheta,
                dX ? dX + (long long)off * d : nullptr, off > 0);
            if (st) return st;
        }
        return KFAC_OK;
    }
    const bool reuse = h->store_forward && h->fwd_valid && h->fwd_theta == theta && h->fwd_X == X &&
                       h->fwd_N == N && N <= h->cfg.max_n_int;
    for (int off = 0; off < N; off += h->cfg.max_n_int) {
        int n = N - off < h->cfg.max_n_int ? N - off : h->cfg.max_n_int;
        kfac_status_t st = simt_forward_laplacian_backward(
            h, s, theta, X + (long long)off * d, n, du ? du + off : nullptr,
            dgrad ? dgrad + (long long)off * d : nullptr, dlap ? dlap + off : nullptr, dtheta,
            dX ? dX + (long long)off * d : nullptr, off > 0, reuse);
        if (st) return st;
    }
    // the pass buffers now hold this chunk's forward activations either way
    h->fwd_valid = h->store_forward && N <= h->cfg.max_n_int;
    h->fwd_theta = theta;
    h->fwd_X = X;
    h->fwd_N = N;
    return KFAC_OK;
}

kfac_status_t kfac_pinn_set_store_forward(kfac_handle_t h, int enable) {
    if (!h) return KFAC_BAD_ARG;
    h->store_forward = enable ? 1 : 0;
    h->fwd_valid = 0;
    return KFAC_OK;
}

kfac_status_t kfac_pinn_set_cta_pairs(kfac_handle_t h, int enable) {
    if (!h) return KFAC_BAD_ARG;
    h->cta_pairs = enable ? 1 : 0;
    handle_graph_free(h);
    return KFAC_OK;
}

kfac_status_t kfac_pinn_set_graph(kfac_handle_t h, int enable) {
    if (!h) return KFAC_BAD_ARG;
    h->graph_mode = enable ? 1 : 0;
    if (!enable) handle_graph_free(h);
    return KFAC_OK;
}

kfac_status_t kfac_pinn_set_autotune(kfac_handle_t h, int enable) {
    if (!h) return KFAC_BAD_ARG;
    h->autotune = enable ? 1 : 0;
    if (enable) handle_graph_free(h);
    return KFAC_OK;
}

kfac_status_t kfac_pinn_get_tuning(kfac_handle_t h, kfac_tune_entry_t* out, int cap, int* count) {
    if (!h || !count || cap < 0 || (cap > 0 && !out)) return KFAC_BAD_ARG;
    const int n = h->n_tune < cap ? h->n_tune : cap;
    if (n > 0) memcpy(out, h->tune, (size_t)n * sizeof(kfac_tune_entry_t));
    *count = h->n_tune;
    return KFAC_OK;
}

kfac_status_t kfac_pinn_set_tuning(kfac_handle_t h, const kfac_tune_entry_t* in, int count) {
    if (!h || count < 0 || count > KFAC_TUNE_CAP || (count > 0 && !in)) return KFAC_BAD_ARG;
    for (int i = 0; i < count; i++) {
        const kfac_tune_entry_t& e = in[i];
        if (e.P < 1 || e.Q < 1 || e.K < 1 || (e.sym != 0 && e.sym != 1) || (e.split != 0 && e.split != 1))
            return KFAC_BAD_ARG;
        if (e.kind == KFAC_TUNE_GRAM) {
            const long long top = ((long long)e.K + 63) / 64 * 64;
            if (e.tiles != 0 || e.chunk < 64 || e.chunk % 64 != 0 || e.chunk > top) return KFAC_BAD_ARG;
        } else if (e.kind == KFAC_TUNE_FWD_TAN || e.kind == KFAC_TUNE_BWD_TAN) {
            if (e.sym != 0 || e.tiles < 1 || e.chunk < 1 || e.chunk > e.tiles) return KFAC_BAD_ARG;
        } else {
            return KFAC_BAD_ARG;
        }
    }
    for (int i = 0; i < count; i++) {
        h->tune[i] = in[i];
        h->tune[i].us = 0.f;
        h->tune[i].model_us = 0.f;
    }
    h->n_tune = count;
    handle_graph_free(h);
    return KFAC_OK;
}

kfac_status_t kfac_pinn_factors(kfac_handle_t h, void* stream, const double* theta,
                                const double* X_int, int N_int, const double* f,
                                const double* X_bdy, int N_bdy, const double* g, double* loss) {
    kfac_status_t st = check_batch(h, X_int, N_int, f, X_bdy, N_bdy, g);
    if (st) return st;
    if (!theta) return KFAC_BAD_ARG;
    return run_factors(h, S_(stream), theta, X_int, N_int, f, X_bdy, N_bdy, g, loss);
}

kfac_status_t kfac_pinn_invert(kfac_handle_t h, void* stream) {
    if (!h) return KFAC_BAD_ARG;
    kfac_status_t st = linalg_invert(h, S_(stream));
    if (st == KFAC_OK) h->have_inverse = 1;
    return st;
}

kfac_status_t kfac_pinn_precondition(kfac_handle_t h, void* stream, const double* grad, double* direction) {
    if (!h) return KFAC_BAD_ARG;
    if (!h->have_inverse) return KFAC_NOT_READY;
    cudaStream_t s = S_(stream);
    kfac_status_t st = linalg_precondition(h, s, grad ? grad : h->grad, h->dir);
    if (st) return st;
    h->have_direction = 1;
    if (direction)
        KFAC_CUDA_TRY(cudaMemcpyAsync(direction, h->dir, h->D * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return KFAC_OK;
}

kfac_status_t kfac_pinn_update(kfac_handle_t h, void* stream, double* theta) {
    if (!h || !theta) return KFAC_BAD_ARG;
    if (!h->have_direction) return KFAC_NOT_READY;
    kfac_status_t st = linalg_update(h, S_(stream), theta);
    if (st == KFAC_OK) h->t++;
    return st;
}

kfac_status_t kfac_pinn_step(kfac_handle_t h, void* stream, double* theta,
                             const double* X_int, int N_int, const double* f,
                             const double* X_bdy, int N_bdy, const double* g, double* loss) {
    kfac_status_t st = check_batch(h, X_int, N_int, f, X_bdy, N_bdy, g);
    if (st) return st;
    if (!theta) return KFAC_BAD_ARG;
    cudaStream_t s = S_(stream);
    if (h->graph_mode && !h->in_graph) {
        // stage the batch where the graph expects it (unless it is there already)
        const int d = h->dims[0];
        double* xi = h->stage;
        double* fi = xi + (size_t)N_int * d;
        double* xb = fi + (size_t)N_int * h->fM;
        double* gb = xb + (size_t)N_bdy * d;
        if (X_int != xi) {
            KFAC_CUDA_TRY(cudaMemcpyAsync(xi, X_int, (size_t)N_int * d * sizeof(double), cudaMemcpyDeviceToDevice, s));
            KFAC_CUDA_TRY(cudaMemcpyAsync(fi, f, (size_t)N_int * h->fM * sizeof(double), cudaMemcpyDeviceToDevice, s));
            KFAC_CUDA_TRY(cudaMemcpyAsync(xb, X_bdy, (size_t)N_bdy * d * sizeof(double), cudaMemcpyDeviceToDevice, s));
            KFAC_CUDA_TRY(cudaMemcpyAsync(gb, g, (size_t)N_bdy * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        return handle_graph_step(h, s, theta, xi, N_int, fi, xb, N_bdy, gb, loss);
    }
    if ((st = run_factors(h, s, theta, X_int, N_int, f, X_bdy, N_bdy, g, loss))) return st;
    if ((st = kfac_pinn_invert(h, stream))) return st;
    if ((st = kfac_pinn_precondition(h, stream, nullptr, nullptr))) return st;
    if (h->cfg.update == KFAC_UPDATE_FIXED) return kfac_pinn_update(h, stream, theta);
    if (h->cfg.update == KFAC_UPDATE_LINE_SEARCH)
        st = linalg_line_search_update(h, s, theta, X_int, N_int, f, X_bdy, N_bdy, g);
    else
        st = linalg_auto_update(h, s, theta, X_int, N_int, X_bdy, N_bdy);
    if (st) return st;
    h->t++;
    return KFAC_OK;
}

kfac_status_t kfac_pinn_get_update_coefficients(kfac_handle_t h, void* stream, double* dst) {
    if (!h || !dst) return KFAC_BAD_ARG;
    if (h->t == 0) return KFAC_NOT_READY;
    KFAC_CUDA_TRY(cudaMemcpyAsync(dst, h->coef, 2 * sizeof(double), cudaMemcpyDeviceToDevice, S_(stream)));
    return KFAC_OK;
}

kfac_status_t kfac_pinn_get_line_search_losses(kfac_handle_t h, void* stream, double* dst) {
    if (!h || !dst) return KFAC_BAD_ARG;
    if (h->cfg.update != KFAC_UPDATE_LINE_SEARCH || h->t == 0) return KFAC_NOT_READY;
    KFAC_CUDA_TRY(cudaMemcpyAsync(dst, h->ls_loss, 3 * 31 * sizeof(double), cudaMemcpyDeviceToDevice, S_(stream)));
    return KFAC_OK;
}

kfac_status_t kfac_pinn_step_host(kfac_handle_t h, void* stream, double* theta,
                                  const double* X_int_host, int N_int, const double* f_host,
                                  const double* X_bdy_host, int N_bdy, const double* g_host,
                                  double* loss_host) {
    kfac_status_t st = check_batch(h, X_int_host, N_int, f_host, X_bdy_host, N_bdy, g_host);
    if (st) return st;
    if (!theta) return KFAC_BAD_ARG;
    cudaStream_t s = S_(stream);
    const int d = h->dims[0];
    double* xi = h->stage;
    double* fi = xi + (size_t)N_int * d;
    double* xb = fi + (size_t)N_int * h->fM;
    double* gb = xb + (size_t)N_bdy * d;
    KFAC_CUDA_TRY(cudaMemcpyAsync(xi, X_int_host, (size_t)N_int * d * sizeof(double), cudaMemcpyHostToDevice, s));
    KFAC_CUDA_TRY(cudaMemcpyAsync(fi, f_host, (size_t)N_int * h->fM * sizeof(double), cudaMemcpyHostToDevice, s));
    KFAC_CUDA_TRY(cudaMemcpyAsync(xb, X_bdy_host, (size_t)N_bdy * d * sizeof(double), cudaMemcpyHostToDevice, s));
    KFAC_CUDA_TRY(cudaMemcpyAsync(gb, g_host, (size_t)N_bdy * sizeof(double), cudaMemcpyHostToDevice, s));
    if ((st = kfac_pinn_step(h, stream, theta, xi, N_int, fi, xb, N_bdy, gb, h->loss))) return st;
    if (loss_host)
        KFAC_CUDA_TRY(cudaMemcpyAsync(loss_host, h->loss, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    KFAC_CUDA_TRY(cudaStreamSynchronize(s));
    return KFAC_OK;
}

kfac_status_t kfac_pinn_get_factor(kfac_handle_t h, void* stream, int layer, int which, double* dst) {
    if (!h || !dst || layer < 1 || layer > h->cfg.L || which < 0 || which > 3) return KFAC_BAD_ARG;
    size_t n = (which == KFAC_A_INT || which == KFAC_A_BDY) ? h->dims[layer - 1] + 1 : h->dims[layer];
    KFAC_CUDA_TRY(cudaMemcpyAsync(dst, h->fac[which][layer - 1], n * n * sizeof(double),
                                  cudaMemcpyDeviceToDevice, S_(stream)));
    return KFAC_OK;
}

kfac_status_t kfac_pinn_set_factor(kfac_handle_t h, void* stream, int layer, int which, const double* src) {
    if (!h || !src || layer < 1 || layer > h->cfg.L || which < 0 || which > 3) return KFAC_BAD_ARG;
    size_t n = (which == KFAC_A_INT || which == KFAC_A_BDY) ? h->dims[layer - 1] + 1 : h->dims[layer];
    KFAC_CUDA_TRY(cudaMemcpyAsync(h->fac[which][layer - 1], src, n * n * sizeof(double),
                                  cudaMemcpyDeviceToDevice, S_(stream)));
    return KFAC_OK;
}

kfac_status_t kfac_pinn_get_gradient(kfac_handle_t h, void* stream, double* dst) {
    if (!h || !dst) return KFAC_BAD_ARG;
    KFAC_CUDA_TRY(cudaMemcpyAsync(dst, h->grad, h->D * sizeof(double), cudaMemcpyDeviceToDevice, S_(stream)));
    return KFAC_OK;
}

kfac_status_t kfac_pinn_get_direction(kfac_handle_t h, void* stream, double* dst) {
    if (!h || !dst) return KFAC_BAD_ARG;
    KFAC_CUDA_TRY(cudaMemcpyAsync(dst, h->dir, h->D * sizeof(double), cudaMemcpyDeviceToDevice, S_(stream)));
    return KFAC_OK;
}

kfac_status_t kfac_pinn_sync_status(kfac_handle_t h, kfac_status_t* status) {
    if (!h || !status) return KFAC_BAD_ARG;
    KFAC_CUDA_TRY(cudaDeviceSynchronize());
    int v = 0;
    KFAC_CUDA_TRY(cudaMemcpy(&v, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    KFAC_CUDA_TRY(cudaMemset(h->status, 0, sizeof(int)));
    *status = (kfac_status_t)v;
    return KFAC_OK;
}

int64_t kfac_pinn_launch_count(kfac_handle_t h) { return h ? h->launches : -1; }

}  // extern "C"
