// Internal declarations shared by the translation units of libkfacpinn.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/kfac_pinn.h"

#define KFAC_DEV __device__ __forceinline__

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------
// Activations of one pass are stored column-block-major: the S Taylor columns
// of all N points form S consecutive blocks of N rows, each row holding the h
// features of one (column, point) pair:  X[(s * N + n) * h + j].  A layer's
// linear map is then one GEMM over M = S*N rows, the value rows are the
// first block (the only rows that see the bias) and the Laplacian rows the
// last block.
// The SIMT path stores them in its precision (double for KFAC_FP64, float
// for KFAC_FP32: simt_elem_bytes), hence the untyped pointers.
struct PassBuffers {
    int N;           // capacity in points
    int S;           // shared columns (d + 2 for the interior, 1 for the boundary)
    void* Z[KFAC_MAX_LAYERS];      // pre-activation outputs Z^{(l)}       (S*N x h_l)
    void* T[KFAC_MAX_LAYERS];      // post-activation T^{(l)}, l < L       (S*N x h_l)
    void* Zb[KFAC_MAX_LAYERS];     // adjoints g^{(l)} = dr/dZ^{(l)}       (S*N x h_l)
    double* r;                     // residuals, FP64                      (N)
    // reduce-variant scratch: per-point column sums (N x max width)
    void* red_a;
    void* red_g;
    // mixed-precision path (bf16 operands, see tc_path.cu)
    void* mx;
};

struct kfac_pinn_handle {
    kfac_config_t cfg;
    int dims[KFAC_MAX_LAYERS + 1];          // h_0..h_L
    int64_t woff[KFAC_MAX_LAYERS + 1];      // offset of W~_l in theta (l = 0..L-1), woff[L] = D
    int64_t D;
    int S;
    int device;
    int sm_count;

    PassBuffers in;   // interior pass
    PassBuffers bd;   // boundary pass

    double* grad;         // D
    double* dir;          // D
    double* delta_prev;   // D
    double* dhat;         // D: momentum direction of the line search
    double* trial;        // D: trial parameters of the line search
    double* ls_loss;      // 3 x 31 trial losses
    double* ks_jv;        // residual JVPs of the automatic update (2 (max_n_int + max_n_bdy))
    double* ks_part;      // block partial sums of the automatic update
    double* coef;         // (c0, c1) of the last update delta = c0 Delta + c1 delta_prev, + diagnostics
    // operator: interior residual r = cT z_t + cD z_D - f; tangent channel m of the
    // Taylor pass has direction v_m = opQ e_m (opQ == nullptr: e_m) and weight chw[m]
    // in the second-order column (App. C.3)
    double cT, cD;
    // general interior residual (kfac_residual_t; res_M == 0: the operator's own)
    int res_M;
    int res_has_Q;
    int fM;               // interior data values per point: res_M, or 1
    double* res_coef;     // b (M x S), W (M x M), L_W (M x M, Cholesky of W), Q (M x S x S)
    double* res_r;        // residuals r_{n,k} of the last interior pass (max_n_int x M)
    double* opQ;          // d x d row-major (general operator only)
    double* chw64;        // d
    float* chw32;         // d
    double* w1q;          // h_1 x d: W_1 Q (general operator only)
    double* w1q2;         // h_1 x d: V_1 Q for forward-mode products
    double* fac[4][KFAC_MAX_LAYERS];      // EMA factors A_int, B_int, A_bdy, B_bdy (n x n)
    double* VA[KFAC_MAX_LAYERS];          // generalized eigenvectors (na x na, row-major)
    double* wa[KFAC_MAX_LAYERS];          // generalized eigenvalues (na)
    double* VB[KFAC_MAX_LAYERS];
    double* wb[KFAC_MAX_LAYERS];
    double* loss;                         // 3 doubles
    double* part;                         // split-K partial sums
    size_t part_elems;
    double* lin;                          // linear-algebra workspace
    size_t lin_elems;
    double* tmp;                          // precondition temporaries
    size_t tmp_elems;
    int* status;                          // device status word
    // host staging for kfac_pinn_step_host
    double* stage;                        // device copy of the host batch
    size_t stage_elems;
    void* mx;                             // mixed-precision state (tc_path.cu)
    void* eig;                            // batched eigensolver state (eig.cu)

    // per-class device timers (kfac_pinn_timing_*)
    int timing;
    struct Timer {
        cudaEvent_t* ev;   // 2 * cap events
        int cap, n;
        long long launches;
        double work;       // algorithmic work of the method (FLOPs or bytes)
        double exec;       // work the hardware executed (padded tiles, split-BF16 products)
        double ms;         // folded-in time of earlier batches
    } timers[KFAC_KC_COUNT];

    int t;                 // completed steps
    int have_inverse;
    int have_direction;
    // reverse mode with stored activations: the interior pass buffers hold the
    // forward Laplacian of (fwd_theta, fwd_X, fwd_N) while fwd_valid is set
    int store_forward;
    // the forward layer GEMMs of the tensor-core precisions on CTA pairs
    // (kfac_pinn_set_cta_pairs; off by default)
    int cta_pairs;
    // graph mode (kfac_pinn_set_graph): a batch of this handle alone; in_graph
    // marks the eager step run inside it (capture or first call)
    int graph_mode;
    int in_graph;
    struct kfac_pinn_batch* gbatch;
    // Gram tile autotuner (kfac_pinn_set_autotune): measured row-chunk lengths
    int autotune;
    int n_tune;
    kfac_tune_entry_t tune[KFAC_TUNE_CAP];
    cudaEvent_t tune_ev[2];
    int fwd_valid;
    const double* fwd_theta;
    const double* fwd_X;
    int fwd_N;
    long long launches;    // kernels launched (host counter)
};

// ---------------------------------------------------------------------------
// Status helpers
// ---------------------------------------------------------------------------
KFAC_DEV void latch_status(int* status, int code) {
    // first error wins
    atomicCAS(status, 0, code);
}

// The CUDA error behind the last KFAC_CUDA_ERROR on this host thread
// (kfac_pinn_last_cuda_error).
void kfac_record_cuda_error(cudaError_t e);

#define KFAC_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) {                              \
            kfac_record_cuda_error(_e);                       \
            return KFAC_CUDA_ERROR;                           \
        }                                                     \
    } while (0)

#define KFAC_TRY(expr)                  \
    do {                                \
        kfac_status_t _st = (expr);     \
        if (_st != KFAC_OK) return _st; \
    } while (0)

#define KFAC_LAUNCH_CHECK(h)                                  \
    do {                                                      \
        (h)->launches++;                                      \
        cudaError_t _e = cudaGetLastError();                  \
        if (_e != cudaSuccess) {                              \
            kfac_record_cuda_error(_e);                       \
            return KFAC_CUDA_ERROR;                           \
        }                                                     \
    } while (0)

// Graph mode (batch.cu): one step of h through its own single-handle batch.
kfac_status_t handle_graph_step(kfac_pinn_handle* h, cudaStream_t s, double* theta, const double* X_int, int N_int,
                                const double* f, const double* X_bdy, int N_bdy, const double* g, double* loss);
void handle_graph_free(kfac_pinn_handle* h);

// The tensor-core path (BF16, or split-BF16 everywhere) vs the SIMT path
// (FP64 or FP32).
static inline bool is_mixed(const kfac_pinn_handle* h) {
    return h->cfg.precision == KFAC_MIXED_BF16 || h->cfg.precision == KFAC_MIXED_SPLIT;
}
static inline bool is_split_all(const kfac_pinn_handle* h) { return h->cfg.precision == KFAC_MIXED_SPLIT; }

// The network and operator checks of kfac_pinn_create (abi.cu).
bool kfac_valid_network(const kfac_config_t* c);

// Every device allocation of the library (abi.cu): cudaMalloc of `bytes`
// (at least 1), KFAC_OOM when the device is out of memory or when the
// injected failure of kfac_pinn_inject_alloc_failure is due, KFAC_CUDA_ERROR
// for any other failure; *p is NULL unless KFAC_OK.
kfac_status_t kfac_device_alloc(void** p, size_t bytes);

// Device timers: bracket a launch with events when timing is enabled.
void timer_begin(kfac_pinn_handle* h, int cls, cudaStream_t s);
// work: algorithmic work of the launch; exec: work as executed (padding and
// split-BF16 products included), exec < 0 meaning the same as work.
void timer_end(kfac_pinn_handle* h, int cls, cudaStream_t s, double work, double exec = -1.0);
void timers_free(kfac_pinn_handle* h);

static inline unsigned ceil_div_u(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// SIMT path in the handle's precision, FP64 or FP32 (simt_path.cu)
// ---------------------------------------------------------------------------
size_t simt_elem_bytes(const kfac_pinn_handle* h);
kfac_status_t simt_forward(kfac_pinn_handle* h, cudaStream_t s, const double* theta,
                           const double* X, int N, PassBuffers& pb, int S);
kfac_status_t simt_residual_and_seed(kfac_pinn_handle* h, cudaStream_t s, PassBuffers& pb, int N,
                                     int S, const double* target, bool interior);
kfac_status_t simt_backward(kfac_pinn_handle* h, cudaStream_t s, const double* theta,
                            PassBuffers& pb, int N, int S);
kfac_status_t simt_grad_and_factors(kfac_pinn_handle* h, cudaStream_t s, const double* X_int,
                                    int N_int, const double* X_bdy, int N_bdy);
// Loss (Eq. 1) of the FP64 residuals in h->in.r and h->bd.r (both paths)
kfac_status_t fp64_loss(kfac_pinn_handle* h, cudaStream_t s, int N_int, int N_bdy, double* loss_out);
kfac_status_t fp64_loss_to(kfac_pinn_handle* h, cudaStream_t s, int N_int, int N_bdy, double* dst);
kfac_status_t simt_eval_loss(kfac_pinn_handle* h, cudaStream_t s, const double* theta, const double* X_int,
                             int N_int, const double* f, const double* X_bdy, int N_bdy, const double* g,
                             double* dst);
kfac_status_t simt_jvp(kfac_pinn_handle* h, cudaStream_t s, const double* theta, const double* v,
                       const double* X, int N, PassBuffers& pb, int S, bool interior, double* jv);
// General interior residual (Sec. 3.3): r_{n,k} into h->res_r and r_n^T W r_n into
// h->in.r from the interior pass's outputs; the whole curvature-and-gradient part
// of a step after both forward passes (M + 1 interior adjoint passes).
kfac_status_t simt_residual_general(kfac_pinn_handle* h, cudaStream_t s, int N, const double* f);
kfac_status_t simt_backward_and_factors_general(kfac_pinn_handle* h, cudaStream_t s, const double* theta,
                                                const double* X_int, int N_int, const double* f,
                                                const double* X_bdy, int N_bdy);
// Automatic learning rate and momentum (linalg.cu), FP64 handles
kfac_status_t linalg_auto_update(kfac_pinn_handle* h, cudaStream_t s, double* theta, const double* X_int,
                                 int N_int, const double* X_bdy, int N_bdy);
// Line-search update (linalg.cu): theta += alpha* dhat, alpha* from the grid 2^-k
kfac_status_t linalg_line_search_update(kfac_pinn_handle* h, cudaStream_t s, double* theta, const double* X_int,
                                        int N_int, const double* f, const double* X_bdy, int N_bdy,
                                        const double* g);
kfac_status_t simt_forward_laplacian_backward(kfac_pinn_handle* h, cudaStream_t s, const double* theta,
                                              const double* X, int N, const double* du, const double* dgrad,
                                              const double* dlap, double* dtheta, double* dX, bool accumulate,
                                              bool reuse_forward);
kfac_status_t simt_extract_outputs(kfac_pinn_handle* h, cudaStream_t s, PassBuffers& pb, int N,
                                   int S, double* u, double* grad, double* lap);

// ---------------------------------------------------------------------------
// Linear algebra (linalg.cu)
// ---------------------------------------------------------------------------
size_t linalg_workspace_elems(const kfac_pinn_handle* h);
size_t linalg_auto_part_elems();
// Batched FP64 generalized eigensolver (eig.cu)
kfac_status_t eig_alloc(kfac_pinn_handle* h);
void eig_free(kfac_pinn_handle* h);
kfac_status_t eig_run(kfac_pinn_handle* h, cudaStream_t s);
// One eigensolve over every factor pair of `count` handles (the grouped batch
// step): problems on the handles' own workspaces, schedules of their own.
kfac_status_t eig_batch_alloc(kfac_pinn_handle* const* hs, int count, void** out);
kfac_status_t eig_batch_run(kfac_pinn_handle* h0, void* eb, cudaStream_t s);
void eig_batch_free(void* eb);
// Self-check of the eigensolver's bounded group barrier (kfac_pinn_check_wait_timeout).
kfac_status_t eig_check_wait(kfac_pinn_handle* h, cudaStream_t s, uint64_t limit_ns);
kfac_status_t linalg_invert(kfac_pinn_handle* h, cudaStream_t s);
kfac_status_t linalg_precondition(kfac_pinn_handle* h, cudaStream_t s, const double* grad,
                                  double* dir);
kfac_status_t linalg_update(kfac_pinn_handle* h, cudaStream_t s, double* theta);

// ---------------------------------------------------------------------------
// Generic FP64 GEMM launcher (simt_path.cu)
// ---------------------------------------------------------------------------
// C(p, q) = sum_k A(p, k) B(k, q) with strided operands:
//   A(p, k) = A[p * a_sp + k * a_sk],  B(k, q) = B[k * b_sk + q * b_sq]
// and C(p, q) written to C[p * c_sp + q * c_sq] as alpha * acc (+ beta * C if
// beta != 0).  Strides are in elements.  fp32: products and sums in FP32.
kfac_status_t dgemm_strided(kfac_pinn_handle* h, cudaStream_t s, int P, int Q, int K,
                            const double* A, long long a_sp, long long a_sk,
                            const double* B, long long b_sk, long long b_sq,
                            double* C, long long c_sp, long long c_sq, double alpha, double beta,
                            bool fp32 = false);
