/*
 * kfac_pinn.h -- C-ABI of the GB300 (sm_103a) KFAC-for-PINNs hot path.
 *
 * One KFAC step for a tanh MLP on a Poisson- or heat-type PINN loss, after
 * Dangel, Mueller, Zeinhofer, "Kronecker-Factored Approximate Curvature for
 * Physics-Informed Neural Networks" (NeurIPS 2024):
 *   - the Taylor-mode forward Laplacian (Sec. 3.1, Eq. 5-6; App. C.2);
 *   - the per-layer Kronecker factors A_l, B_l of the interior term
 *     (KFAC-expand, Eq. 8, or KFAC-reduce) and of the boundary term (Eq. 3);
 *   - the damped Kronecker-sum inverse and the preconditioned update
 *     (Sec. 3.4; App. B, Algorithm 1).
 *
 * Conventions shared by every call
 *   - Layers l = 1..L, widths h_0 = d, h_1, .., h_L = 1, tanh after every
 *     layer but the last.  theta packs the augmented weights
 *     W~_l = (W_l b_l) (h_l x (h_{l-1}+1)) one after another, each stacked
 *     column by column (first index fastest), as in Sec. 2.  Its length is
 *     D = sum_l h_l (h_{l-1} + 1)  (kfac_pinn_param_count).
 *   - Points X are N x d, row-major (point-major), FP64.  f has N entries
 *     (right-hand side at interior points), g has N_bdy entries (boundary
 *     data).  For the heat operator coordinate 0 of each point is time.
 *   - Unless a name ends in _host, every pointer argument is a DEVICE pointer
 *     on the handle's device, owned by the caller, and must stay valid until
 *     the work queued on `stream` has finished.  The handle owns only its
 *     internal buffers (activations, factors, inverses, momentum, scratch).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls queue work asynchronously and return at once; argument
 *     errors are returned immediately (KFAC_BAD_ARG) and nothing is queued.
 *   - Errors found on the device (a factor that is not positive definite, a
 *     non-finite loss, a bounded wait that ran out) are latched in a device
 *     status word; kfac_pinn_sync_status reads and clears it.  No call traps,
 *     asserts or aborts on the device.
 *   - A handle is not thread-safe; calls on one handle must be serialised by
 *     the caller (they share the handle's buffers).
 */
#ifndef KFAC_PINN_H
#define KFAC_PINN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KFAC_OK = 0,
    KFAC_BAD_ARG = 1,      /* invalid size, pointer or configuration          */
    KFAC_NOT_PD = 2,       /* a damped factor failed its Cholesky             */
    KFAC_NONFINITE = 3,    /* NaN/Inf in the loss or the factors               */
    KFAC_TIMEOUT = 4,      /* a bounded device-side wait gave up               */
    KFAC_OOM = 5,          /* cudaMalloc failed in kfac_pinn_create            */
    KFAC_CUDA_ERROR = 6,   /* a CUDA runtime call or launch failed             */
    KFAC_NOT_READY = 7     /* precondition/update called before invert         */
} kfac_status_t;

typedef enum {
    KFAC_FP64 = 0,         /* every stage in FP64 SIMT arithmetic              */
    KFAC_MIXED_BF16 = 1,   /* tensor-core BF16 (split-BF16 on the value and
                              Laplacian columns) with FP32 accumulation for the
                              Taylor pass, adjoint, gradient and Grams; FP64
                              for loss, factors, Cholesky and eigensolver      */
    KFAC_MIXED_SPLIT = 2,  /* the same tensor-core path with split-BF16 (hi +
                              lo, about 16 significant bits, three products
                              per contraction) on every Taylor column, every
                              adjoint and every Gram: per-result errors near
                              1e-5 against FP64, at about three times the
                              tensor work.  For d >= 32 the 31 trial losses
                              of the LINE_SEARCH update run the
                              KFAC_MIXED_BF16 forward pass (split value,
                              second-order and time columns; plain BF16
                              tangents, whose roundings average over the d
                              tangents of the second-order column): a trial
                              loss only ranks the grid points                */
    KFAC_FP32 = 3          /* the SIMT path of KFAC_FP64 with FP32 storage and
                              FP32 arithmetic (CUDA cores) for the Taylor pass
                              and its adjoint; the sums over the collocation
                              points (gradient and factor Grams) multiply the
                              FP32 operands exactly in FP64 and accumulate in
                              FP64; FP64 for residuals, loss, factors (EMA),
                              Cholesky, eigensolver and preconditioning.
                              Per-result errors near 1e-7 against FP64       */
} kfac_precision_t;

typedef enum { KFAC_EXPAND = 0, KFAC_REDUCE = 1 } kfac_variant_t;

/* Residual operator of the interior term.
 * LAPLACE: r = -Laplacian(u) - f   (Eq. 1 with L = -Laplacian)
 * HEAT:    r = du/dt - kappa * Laplacian_x(u) - f, where the Laplacian runs
 *          over coordinates 1..d-1 and coordinate 0 is time (App. A.6).
 * GENERAL: r = sum_ij c_ij d^2 u / dx_i dx_j - f with the symmetric d x d
 *          coefficient matrix cfg.op_coef (Sec. 3.1; App. C.3).  The Taylor
 *          pass propagates the derivatives along the eigenvectors q_m of C
 *          and the second-order column sum_m lambda_m d^2u/dq_m^2, which is
 *          the same operator; the gradient output is rotated back to the
 *          coordinate axes.  KFAC-expand only. */
typedef enum { KFAC_OP_LAPLACE = 0, KFAC_OP_HEAT = 1, KFAC_OP_GENERAL = 2 } kfac_operator_t;

/* Update rule of kfac_pinn_step (Sec. 3.4), with Delta the preconditioned
 * direction and delta_prev the previous update:
 * FIXED:       delta = lr (momentum delta_prev + Delta)
 * LINE_SEARCH: delta = alpha* dhat, dhat = momentum delta_prev + Delta and
 *              alpha* = argmin over {2^0, 2^-1, .., 2^-30} of L(theta + alpha dhat)
 *              on the step's batch (KFAC of the paper; lr unused)
 * AUTO:        delta = alpha* Delta + mu* delta_prev with (alpha*, mu*) the
 *              minimiser of the quadratic model with the exact damped Gramian
 *              G + lambda I (KFAC* of the paper; lr and momentum unused).  The
 *              Gramian products need J v per point: on an FP64 handle a
 *              forward-mode pass through the Taylor pass; on a tensor-core
 *              handle sum_l sum_s g_{n,s}^T V_l T^_{n,s} from the activations
 *              and adjoints the step's curvature pass stored (Sec. 3.2), in
 *              that handle's precision. */
typedef enum { KFAC_UPDATE_FIXED = 0, KFAC_UPDATE_LINE_SEARCH = 1, KFAC_UPDATE_AUTO = 2 } kfac_update_t;

/* Factor selector of kfac_pinn_get_factor / kfac_pinn_set_factor. */
typedef enum { KFAC_A_INT = 0, KFAC_B_INT = 1, KFAC_A_BDY = 2, KFAC_B_BDY = 3 } kfac_factor_t;

#define KFAC_MAX_LAYERS 16
#define KFAC_MAX_RESIDUALS 8

/* A general interior residual (Sec. 3.3, Eq. 9-10) in place of the operator's
 * own: M outputs that are polynomials of degree two in the network's Taylor
 * outputs at each point, z_n = (u, du/dx_1, .., du/dx_d, the operator's
 * second-order column) in R^S, S = d + 2,
 *     r_{n,k} = sum_s b[k,s] z_{n,s} + 1/2 sum_{s,t} Q[k,s,t] z_{n,s} z_{n,t} - f_{n,k},
 * fed into the criterion l(r) = 1/2 r^T W r, so that the interior loss is
 * (1/N) sum_n l(r_n) and the criterion Hessian of Eq. 10 is Lambda = W.
 * First-order terms of a linear operator are b on the derivative columns, a
 * term such as |grad u|^2 is Q on them, M > 1 residuals share one network.
 * B_Omega = (1/N) sum_{n,s} (J_{Z_{n,s}} r_n)^T W (J_{Z_{n,s}} r_n) is formed by
 * M adjoint passes seeded with the columns of the Cholesky factor of W (the
 * outer-product rewrite of Sec. 3.3), the gradient by one more seeded with
 * W r_n.  The interior data f of every call then holds N x M values,
 * point-major.  Host pointers, read by kfac_pinn_create only. */
typedef struct {
    int M;               /* residual outputs, 1..KFAC_MAX_RESIDUALS                 */
    const double* b;     /* M x S row-major, b[k * S + s]                            */
    const double* Q;     /* M x S x S, Q[(k * S + s) * S + t], symmetric in s and t;
                            NULL: r linear in z                                      */
    const double* W;     /* M x M symmetric positive definite; NULL: the identity   */
} kfac_residual_t;

typedef struct {
    int d;                         /* input dimension h_0 (>= 1)                       */
    int L;                         /* number of linear layers, 1..KFAC_MAX_LAYERS      */
    int widths[KFAC_MAX_LAYERS];   /* h_1..h_L, each >= 1, h_L == 1                    */
    int op;                        /* kfac_operator_t                                  */
    double kappa;                  /* heat diffusivity (op == HEAT)                    */
    int precision;                 /* kfac_precision_t                                 */
    int variant;                   /* kfac_variant_t (interior factors)                */
    double beta;                   /* EMA factor of the Kronecker factors, [0, 1)      */
    double lambda;                 /* damping lambda > 0                               */
    int damping_sqrt;              /* 0: factor + lambda*I (paper); 1: + sqrt(lambda)*I */
    int factor_init_identity;      /* 0: EMA starts from 0; 1: from the identity      */
    double lr;                     /* fixed learning rate                              */
    double momentum;               /* momentum mu on the previous update               */
    int max_n_int;                 /* capacity: interior points per call (>= 1)        */
    int max_n_bdy;                 /* capacity: boundary points per call (>= 1)        */
    int update;                    /* kfac_update_t of kfac_pinn_step                  */
    int eig_sm_budget;             /* SMs the cooperative tridiagonalisation may
                                      occupy (0: all).  It is used only for factors too
                                      large for one thread-block cluster's shared memory
                                      (h_l + 1 above about 890); the others run one
                                      cluster per factor pair.  Handles stepped
                                      concurrently (kfac_pinn_batch_step) should split
                                      the GPU between them.                          */
    const double* op_coef;         /* GENERAL: host pointer to the d x d coefficient
                                      matrix C (row-major, symmetric), read by
                                      kfac_pinn_create only; otherwise ignored        */
    const kfac_residual_t* residual; /* NULL: the operator's own residual (Eq. 1);
                                      else the general residual above (LAPLACE or
                                      HEAT operator, FP64 or FP32 precision,
                                      KFAC-expand, FIXED or LINE_SEARCH update;
                                      create returns KFAC_BAD_ARG otherwise)  */
} kfac_config_t;

typedef struct kfac_pinn_handle* kfac_handle_t;

/* D = sum_l h_l (h_{l-1} + 1), or -1 for an invalid configuration. */
int64_t kfac_pinn_param_count(const kfac_config_t* cfg);

/* Human-readable name of a status code (static string). */
const char* kfac_pinn_status_string(kfac_status_t st);

/* The cudaError_t behind the last KFAC_CUDA_ERROR returned on the calling host
 * thread (0 if none), and its description (static string). */
int kfac_pinn_last_cuda_error(void);
const char* kfac_pinn_last_cuda_error_string(void);

/* Create a handle on the current CUDA device: validates cfg, allocates every
 * internal buffer for max_n_int / max_n_bdy points, and sets the EMA factors
 * to their initial value (0 or I), momentum to 0 and the step counter to 0.
 * Returns KFAC_BAD_ARG (cfg invalid, out NULL), KFAC_OOM or KFAC_CUDA_ERROR;
 * *out is NULL on failure.  Blocks until the initialisation has finished. */
kfac_status_t kfac_pinn_create(const kfac_config_t* cfg, kfac_handle_t* out);

/* Free every buffer of the handle (synchronises its device first). */
kfac_status_t kfac_pinn_destroy(kfac_handle_t h);

/* Reset EMA factors to their initial value, momentum to 0, step counter to 0. */
kfac_status_t kfac_pinn_reset(kfac_handle_t h, void* stream);

/* Forward Laplacian (Sec. 3.1 Eq. 5-6; App. C.2): for each of N points, u,
 * the d input derivatives and the Laplacian (the partial spatial Laplacian
 * for the heat operator).  u: N; grad: N x d row-major (may be NULL); lap: N
 * (may be NULL).  N may exceed max_n_int (processed in chunks). */
kfac_status_t kfac_pinn_forward_laplacian(kfac_handle_t h, void* stream, const double* theta,
                                          const double* X, int N,
                                          double* u, double* grad, double* lap);

/* Reverse mode through the forward Laplacian (the backward pass of Sec. 3.2,
 * seeded by the caller instead of by a residual): for a scalar phi of the
 * outputs with upstream gradients du = dphi/du (N), dgrad = dphi/d(grad u)
 * (N x d row-major) and dlap = dphi/d(lap u) (N), each may be NULL (zero),
 * writes dtheta = dphi/dtheta (D doubles, overwritten; same packing as theta)
 * and, if dX is not NULL, dX = dphi/dX (N x d).  The Taylor activations of
 * the forward pass are recomputed in chunks of max_n_int points, so memory
 * does not grow with N.  Both precisions: a mixed-precision handle runs the
 * pass and its adjoint on the tensor cores (BF16 with split-BF16 value and
 * second-order rows, FP32 accumulation) and sums the gradient in FP64. */
kfac_status_t kfac_pinn_forward_laplacian_backward(kfac_handle_t h, void* stream, const double* theta,
                                                   const double* X, int N, const double* du,
                                                   const double* dgrad, const double* dlap,
                                                   double* dtheta, double* dX);

/* Store instead of recompute: when enabled, the Taylor activations of the last
 * kfac_pinn_forward_laplacian (FP64, N <= max_n_int, one chunk) stay in the
 * handle and a kfac_pinn_forward_laplacian_backward with the same theta and X
 * pointers and N reuses them instead of recomputing the forward pass; any
 * factors or step call discards them.  The caller must not change theta or X
 * in between.  Larger N is always recomputed chunk by chunk, so memory does
 * not grow with N.  Default: disabled. */
kfac_status_t kfac_pinn_set_store_forward(kfac_handle_t h, int enable);

/* CTA pairs for the forward layer GEMMs of the tensor-core precisions (no
 * counterpart in the paper: a kernel option).  When enabled, each 128-point
 * block of the layer GEMMs T^{(l)} = T^{(l-1)} W~_l^T (Sec. 3.1, Eq. 5) runs
 * with the next point block on a cluster of two CTAs that share one 256-row
 * tensor-core product, each loading half of the weight tile (an odd number
 * of point blocks leaves one CTA of the last pair idle).  The products and their
 * order are the same either way, so the results are bit-identical whenever the
 * two forms split the tangent columns into the same chunks (the wave model
 * counts the idle CTA, so with an odd number of point blocks it may choose
 * another split, which changes only the rounding of the partial sums).  No effect on the
 * FP64 and FP32 precisions.  Default: disabled (on GB300 the pair form fed
 * 25 % fewer bytes per SM but ran the benchmark's step about 3 % slower).
 * Takes effect at the handle's next step (its own captured graph is
 * dropped); a batch step captured earlier (kfac_pinn_batch_step) keeps the
 * form it was captured with.  Errors: KFAC_BAD_ARG for a NULL handle. */
kfac_status_t kfac_pinn_set_cta_pairs(kfac_handle_t h, int enable);

/* Graph mode for kfac_pinn_step and kfac_pinn_step_host (no counterpart in the
 * paper: a runtime option).  When enabled, a step copies its batch into the
 * handle's staging buffers (device to device; step_host copies there from the
 * host anyway) and runs as a CUDA graph: the first step after enabling runs
 * eagerly, the second is captured, later steps with the same theta and loss
 * pointers and point counts replay it (a change re-captures).  The results
 * are bit-identical to eager steps.  The graph runs on a stream of its own,
 * ordered after the work queued on `stream` and before what follows it.
 * Device timers (kfac_pinn_timing_enable) make steps eager.  Default:
 * disabled.  Errors: KFAC_BAD_ARG for a NULL handle. */
kfac_status_t kfac_pinn_set_graph(kfac_handle_t h, int enable);

/* Autotuner of the split-K partitions of the tensor-core precisions (no
 * counterpart in the paper: a runtime option).  Three kinds of launch are
 * split into chunks, one CTA per (output tile, chunk), whose FP32 partial
 * sums are then added in a fixed order:
 *   KFAC_TUNE_GRAM     the Grams of the Kronecker factors (Eq. 8, Eq. 3) and
 *                      the weight-gradient contractions: their K = S * N_cap
 *                      rows (N_cap = max_n_int or max_n_bdy rounded up to
 *                      128) are split into row chunks of at most 2048 rows
 *                      (each chunk sums in FP32, the chunks in FP64);
 *   KFAC_TUNE_FWD_TAN  the layer GEMM of the tangent and Laplacian columns of
 *                      the Taylor pass: its tiles (one per tangent column) are
 *                      split into chunks, each adding its share of the
 *                      Laplacian's sum of squares;
 *   KFAC_TUNE_BWD_TAN  the adjoint GEMM of the tangent columns, likewise.
 * By default the chunk length comes from a wave model: full waves of one CTA
 * per SM and chunks of equal length.  While autotuning is enabled, the first
 * eager call that meets a launch shape not yet in the handle's table times
 * the model's chunk length and up to three runners-up by the model (one
 * warm-up and three timed launches each, CUDA events on the launching
 * stream, which the host then waits for), records the fastest and computes
 * with it; later launches of that shape use the recorded length, so results
 * are deterministic once the table is filled.  Different chunk lengths add
 * the partial sums in different orders: results agree to FP32 rounding, not
 * bit for bit.  Nothing is measured while the stream is being captured into
 * a graph.  Enabling frees the handle's graph (kfac_pinn_set_graph), so the
 * next step runs eagerly and measures; a kfac_pinn_batch holding the handle
 * keeps the lengths its graph was captured with until it re-captures.  The
 * FP64 precision and the Jacobian-vector products of the AUTO update have no
 * tuned launches.  Default: disabled.  Errors: KFAC_BAD_ARG for a NULL
 * handle. */
#define KFAC_TUNE_CAP 128
typedef enum { KFAC_TUNE_GRAM = 0, KFAC_TUNE_FWD_TAN = 1, KFAC_TUNE_BWD_TAN = 2 } kfac_tune_kind_t;
typedef struct {
    int kind;              /* kfac_tune_kind_t                                     */
    int P, Q, K;           /* GRAM: P x Q output, K rows; *_TAN: P = N_cap points,
                              Q output and K input features (padded to 64)        */
    int tiles;             /* *_TAN: tangent tiles that are split; GRAM: 0         */
    int sym;               /* GRAM: 1 = symmetric, upper-triangle tiles only      */
    int split;             /* 1: three split-BF16 products per entry              */
    int chunk;             /* GRAM: rows per chunk, a multiple of 64 in 64..K
                              rounded up to 64; *_TAN: tiles per chunk, 1..tiles  */
    int model_chunk;       /* the wave model's chunk length                       */
    float us;              /* measured time of chunk per launch (us), 0 when the
                              entry was set by kfac_pinn_set_tuning               */
    float model_us;        /* measured time of model_chunk per launch (us)        */
} kfac_tune_entry_t;

kfac_status_t kfac_pinn_set_autotune(kfac_handle_t h, int enable);

/* Copy up to cap entries of the handle's tuning table to out (host memory)
 * and the number of entries to *count (which may exceed cap).  out may be
 * NULL when cap is 0.  Errors: KFAC_BAD_ARG for a NULL handle or count, or
 * cap < 0. */
kfac_status_t kfac_pinn_get_tuning(kfac_handle_t h, kfac_tune_entry_t* out, int cap, int* count);

/* Replace the handle's tuning table by count entries from in (host memory),
 * e.g. a table read from another handle of the same configuration; count 0
 * clears it.  Every field but model_chunk, us and model_us is used.  An
 * entry whose chunk count would not fit the handle's partial-sum workspace
 * is ignored at launch time (the wave model decides).  Frees the handle's
 * graph.  Errors: KFAC_BAD_ARG for a NULL handle, count outside
 * 0..KFAC_TUNE_CAP, in NULL with count > 0, or an entry with an unknown
 * kind, P, Q or K below 1, sym or split not 0 or 1, or a chunk outside the
 * range its kind allows (GRAM: tiles 0 and chunk a multiple of 64 in 64..K
 * rounded up to 64; *_TAN: sym 0, tiles >= 1 and chunk in 1..tiles); the
 * table is then left unchanged. */
kfac_status_t kfac_pinn_set_tuning(kfac_handle_t h, const kfac_tune_entry_t* in, int count);

/* Curvature and gradient of one batch (App. B, Algorithm 1): forward
 * Laplacian on the interior points and plain forward pass on the boundary
 * points, residuals and loss (Eq. 1), one backward pass each for
 * g^{(l)} (Sec. 3.2), the loss gradient, the Kronecker factors (Eq. 8 or
 * KFAC-reduce; Eq. 3) and their exponential moving average (Sec. 3.4).
 * loss: 3 device doubles (L, L_Omega, L_boundary), may be NULL.  The gradient
 * and the factors stay in the handle.  1 <= N_int <= max_n_int,
 * 1 <= N_bdy <= max_n_bdy. */
kfac_status_t kfac_pinn_factors(kfac_handle_t h, void* stream, const double* theta,
                                const double* X_int, int N_int, const double* f,
                                const double* X_bdy, int N_bdy, const double* g,
                                double* loss);

/* Damped inverse of the Kronecker sum (Sec. 3.4; App. B): for every
 * layer, with A~ = A^ + lambda I (or sqrt(lambda) I), the simultaneous
 * diagonalisation V^T A~_Omega V = I, V^T A~_bdy V = diag(a) through an FP64
 * Cholesky of A~_Omega and an FP64 symmetric eigendecomposition of the
 * whitened A~_bdy; likewise for B.  The large matrix products of the
 * decomposition (the whitening with L^{-1}, the final V = L^{-T} U, the
 * divide-and-conquer updates) are FP64 products emulated on the BF16 tensor
 * cores by error-free splitting (8 slices of 7 bits, exact FP32 partial sums,
 * FP64 combination: rounding errors of the order of an FP64 product's).  A
 * factor that is not positive definite latches KFAC_NOT_PD.  Part of the work
 * runs on streams of the handle's own, forked from `stream` and joined back
 * into it: the call stays ordered with the rest of `stream` (and is captured
 * with it). */
kfac_status_t kfac_pinn_invert(kfac_handle_t h, void* stream);

/* direction = -(A~_Omega x B~_Omega + A~_bdy x B~_bdy)^{-1} grad per layer,
 * i.e. Delta = -V_B [(V_B^T G V_A) / (1 + b a^T)] V_A^T (Sec. 3.4).  grad and
 * direction are packed like theta (D doubles).  grad == NULL uses the
 * gradient of the last kfac_pinn_factors call; direction == NULL keeps the
 * result in the handle for kfac_pinn_update.  KFAC_NOT_READY before the first
 * kfac_pinn_invert. */
kfac_status_t kfac_pinn_precondition(kfac_handle_t h, void* stream, const double* grad,
                                     double* direction);

/* theta += delta with delta = lr (momentum * delta_prev + Delta) (Sec. 3.4,
 * fixed learning rate), using the handle's last preconditioned direction. */
kfac_status_t kfac_pinn_update(kfac_handle_t h, void* stream, double* theta);

/* One whole KFAC step: kfac_pinn_factors, kfac_pinn_invert,
 * kfac_pinn_precondition and the update rule cfg.update, in that order.  theta
 * is updated in place; loss (3 device doubles, may be NULL) is the loss at the
 * incoming theta.  LINE_SEARCH evaluates the 31 trial losses on the device
 * (each a forward Laplacian pass) and picks alpha* there (ties: the larger
 * alpha; non-finite losses never win; none finite: no update and
 * KFAC_NONFINITE latched).  AUTO forms the two residual Jacobian-vector
 * products J Delta and J delta_prev on the device (the Taylor pass in forward
 * mode) and solves the 2x2 system there (first step: alpha only, mu* = 0).
 * Neither synchronises the host. */
kfac_status_t kfac_pinn_step(kfac_handle_t h, void* stream, double* theta,
                             const double* X_int, int N_int, const double* f,
                             const double* X_bdy, int N_bdy, const double* g,
                             double* loss);

/* The same step with the batch in HOST memory (pinned memory gives
 * asynchronous copies): X_int_host, f_host, X_bdy_host, g_host are copied to
 * the handle's staging buffers on `stream`, the step runs, and the 3 loss
 * values are copied back to loss_host (may be NULL).  theta is a device
 * pointer (the parameters stay resident).  Synchronises `stream` before
 * returning, so loss_host is valid on return. */
kfac_status_t kfac_pinn_step_host(kfac_handle_t h, void* stream, double* theta,
                                  const double* X_int_host, int N_int, const double* f_host,
                                  const double* X_bdy_host, int N_bdy, const double* g_host,
                                  double* loss_host);

/* Copy the current EMA factor `which` (kfac_factor_t, undamped) of layer
 * `layer` (1..L) to dst (n x n row-major; n = h_{l-1}+1 for A, h_l for B). */
kfac_status_t kfac_pinn_get_factor(kfac_handle_t h, void* stream, int layer, int which, double* dst);

/* Overwrite the EMA factor `which` of layer `layer` with src (n x n). */
kfac_status_t kfac_pinn_set_factor(kfac_handle_t h, void* stream, int layer, int which,
                                   const double* src);

/* Copy the gradient of the last kfac_pinn_factors call (D doubles). */
kfac_status_t kfac_pinn_get_gradient(kfac_handle_t h, void* stream, double* dst);

/* Copy the last preconditioned direction Delta (D doubles). */
kfac_status_t kfac_pinn_get_direction(kfac_handle_t h, void* stream, double* dst);

/* Line search of the last kfac_pinn_step (Sec. 3.4): copy the trial losses
 * to dst, 31 x 3 device doubles, row k = (L, L_Omega, L_boundary) at
 * theta + 2^-k dhat on that step's batch.  KFAC_NOT_READY when the handle was
 * created with another update rule or has not stepped yet. */
kfac_status_t kfac_pinn_get_line_search_losses(kfac_handle_t h, void* stream, double* dst);

/* Coefficients of the last kfac_pinn_step's update delta = c0 Delta + c1 delta_prev:
 * dst = (c0, c1), 2 device doubles.  FIXED: (lr, lr momentum); LINE_SEARCH:
 * (alpha*, alpha* momentum); AUTO: (alpha*, mu*).  KFAC_NOT_READY before the first step. */
kfac_status_t kfac_pinn_get_update_coefficients(kfac_handle_t h, void* stream, double* dst);

/* Synchronise the handle's device, then read and clear the device status
 * word (first error latched since the last read). */
kfac_status_t kfac_pinn_sync_status(kfac_handle_t h, kfac_status_t* status);

/* Number of kernels this library launched on the handle since creation
 * (host-side counter; used to report launches per step). */
int64_t kfac_pinn_launch_count(kfac_handle_t h);

/* Kernel classes of the device timers. */
typedef enum {
    KFAC_KC_LAYER_GEMM = 0,   /* forward layer GEMMs of the Taylor pass       */
    KFAC_KC_ADJOINT_GEMM = 1, /* adjoint GEMMs (T^bar = Z^bar W)              */
    KFAC_KC_GRAM = 2,         /* factor Grams and weight-gradient reductions  */
    KFAC_KC_ELEMENTWISE = 3,  /* tanh Taylor rule, its adjoint, residuals     */
    KFAC_KC_EIG = 4,          /* Cholesky + generalized eigendecomposition    */
    KFAC_KC_PRECOND = 5,      /* preconditioning GEMMs and the update         */
    KFAC_KC_COUNT = 6
} kfac_kernel_class_t;

/* Enable (1) or disable (0) per-class device timers: while enabled, every
 * launch of a timed class is bracketed by CUDA events recorded on the
 * launching stream.  Enabling clears the accumulated timers. */
kfac_status_t kfac_pinn_timing_enable(kfac_handle_t h, int enable);

/* Synchronise the device and return, for one kernel class, the summed device
 * time of its recorded launches (ms), the number of launches, and their
 * summed algorithmic work (FLOPs for contractions, bytes for element-wise
 * kernels: 2 P Q K per GEMM; bytes read + written per element-wise pass).
 * Any pointer may be NULL.  The class's timers are cleared. */
kfac_status_t kfac_pinn_timing_read(kfac_handle_t h, int kernel_class, double* total_ms,
                                    int64_t* launches, double* work);

/* kfac_pinn_timing_read plus exec_work: the work as the hardware executed it
 * (tiles padded to the kernel's tile and feature multiples, and every
 * split-BF16 product: three tensor-core products per contraction where both
 * operands carry low halves), while `work` counts the method's contraction
 * once over the real sizes (2 P Q K per GEMM; n (n + 1) K per symmetric Gram
 * of K rows; element-wise kernels: bytes read + written).  exec_work may be
 * NULL.  The class's timers are cleared. */
kfac_status_t kfac_pinn_timing_read_ex(kfac_handle_t h, int kernel_class, double* total_ms,
                                       int64_t* launches, double* work, double* exec_work);

/* Failure detection without a fault (no counterpart in the paper).
 *
 * kfac_pinn_check_wait_timeout runs one of the library's bounded device waits
 * against a condition that nothing satisfies, with a limit of limit_ms
 * milliseconds instead of the 2 s its kernels use:
 *   kind 0: the group barrier of the cooperative eigensolver kernels (a group
 *           of two CTAs of which only one is launched);
 *   kind 1: the mbarrier wait of the tcgen05 engine (one expected arrival
 *           that never comes).
 * The wait gives up after limit_ms, the kernel latches KFAC_TIMEOUT in the
 * handle's status word (kfac_pinn_sync_status reads it) and returns, and the
 * context stays usable.  Synchronises `stream`.  Errors: KFAC_BAD_ARG (NULL
 * handle, kind not 0 or 1, limit_ms outside 1..10000).
 *
 * kfac_pinn_inject_alloc_failure makes the device allocation that comes after
 * n more successful ones fail as if the device were out of memory (n = 0: the
 * next one; -1: none; process-wide).  kfac_pinn_create then returns
 * KFAC_OOM and frees everything it had allocated.  Errors: KFAC_BAD_ARG for
 * n < -1. */
kfac_status_t kfac_pinn_check_wait_timeout(kfac_handle_t h, void* stream, int kind, int limit_ms);
kfac_status_t kfac_pinn_inject_alloc_failure(long long n);

/* Batched stepping of many independent problems (handles), each with its own
 * network, point counts and buffers.  The paper steps one problem at a time;
 * this serves many small PINNs together: the handles' steps are queued on
 * n_streams worker streams forked from and joined back into the caller's
 * stream, and from the second call on the whole batch is captured once into
 * a CUDA graph and replayed.
 *   - kfac_pinn_batch_create copies the handle array (the handles stay owned
 *     by the caller and must outlive the batch); all must be on the current
 *     device.  n_streams in 1..64.
 *   - kfac_pinn_batch_step: per-handle arrays (host arrays of device
 *     pointers and counts, count entries each) as in kfac_pinn_step; loss may
 *     be NULL or hold NULL entries.  Call 1 runs eagerly; call 2 captures and
 *     launches the graph; later calls replay it when every pointer and count
 *     equals those captured (write new batches into the same buffers), and
 *     re-capture otherwise.  use_graph = 0 always runs eagerly.
 *   - Same results as calling kfac_pinn_step on each handle in turn.  A handle
 *     with timing enabled is stepped eagerly (its timers need the host). */
typedef struct kfac_pinn_batch* kfac_batch_t;

kfac_status_t kfac_pinn_batch_create(const kfac_handle_t* handles, int count, int n_streams, kfac_batch_t* out);
kfac_status_t kfac_pinn_batch_destroy(kfac_batch_t b);
kfac_status_t kfac_pinn_batch_step(kfac_batch_t b, void* stream, double* const* theta,
                                   const double* const* X_int, const int* N_int, const double* const* f,
                                   const double* const* X_bdy, const int* N_bdy, const double* const* g,
                                   double* const* loss, int use_graph);

/* Grouped form of a batch (no counterpart in the paper: a serving pattern for many
 * small PINNs).  With enable = 1 the next captured batch step (a call with
 * use_graph = 1 from the second on) records every handle's step launch by
 * launch instead of running it, merges the launches of the same kernel
 * across handles into one grouped launch (each handle's launch keeps its own
 * grid and arguments, read from a member table in device memory: a block of
 * the grouped launch computes what the same block of the handle's own launch
 * computes) and solves the generalized eigenproblems of every factor pair of
 * every handle (Sec. 3.4) as one batched eigensolve.  The number of launches
 * of a batch step is then about that of one handle's step, whatever the
 * number of handles.  Results equal those of kfac_pinn_step on each handle.
 *   - Every handle must use a tensor-core precision (KFAC_MIXED_BF16 or
 *     KFAC_MIXED_SPLIT): KFAC_BAD_ARG otherwise.  enable = 0 returns to the
 *     stream form.  Switching drops the captured graph.
 *   - Eager calls (the first one, use_graph = 0, timing enabled) run the
 *     stream form.
 *   - A handle's own graph mode (kfac_pinn_set_graph) does not apply to its
 *     steps inside the batch.
 *
 * kfac_pinn_batch_launches writes the number of kernel launches of one
 * replayed batch step (the captured graph's kernels) to *per_step;
 * KFAC_NOT_READY before a graph has been captured. */
kfac_status_t kfac_pinn_batch_set_grouped(kfac_batch_t b, int enable);
kfac_status_t kfac_pinn_batch_launches(kfac_batch_t b, long long* per_step);

/* Allocation-free forward Laplacian.  The paper has no counterpart: this is
 * a service for callers that cannot allocate device memory while they run
 * (code inside another runtime's memory pool or fixed device-memory budget,
 * or a process that must not grow after start-up).  It computes the same u,
 * grad and lap as kfac_pinn_forward_laplacian on an FP64 handle built from
 * cfg (cfg->precision is ignored; FP64 throughout), without a handle and
 * without allocating anything: the per-layer Taylor matrices live in one
 * static 32 MiB scratch array in device memory that every GPU loading this
 * library holds until the process exits.
 *   - Inputs and outputs are caller-owned device pointers as in
 *     kfac_pinn_forward_laplacian; N >= 1.  cfg must pass the network checks
 *     of kfac_pinn_create (d, L, widths, operator); the other fields are
 *     ignored.  KFAC_OP_GENERAL returns KFAC_BAD_ARG: its tangent directions
 *     are set up on a handle. 
 *   - Capacity: d + sum over layers l of (2 if l < L else 1) * (d+2) * N * h_l
 *     doubles must not exceed 4,194,304 (32 MiB); larger requests return
 *     KFAC_BAD_ARG and queue nothing.
 *   - The first call on a device looks up the scratch array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture on the device.
 *   - Every call shares the scratch array: calls that overlap on the GPU
 *     (other streams or host threads) race and must be serialised by the
 *     caller.  Nothing needs clearing between calls: every scratch element a
 *     call reads is first written by the same call. */
kfac_status_t kfac_pinn_forward_laplacian_noalloc(const kfac_config_t* cfg, void* stream, const double* theta,
                                                  const double* X, int N,
                                                  double* u, double* grad, double* lap);

#ifdef __cplusplus
}
#endif
#endif /* KFAC_PINN_H */
