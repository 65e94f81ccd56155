// SIMT path in FP64 or FP32: forward Laplacian, residuals, adjoint, gradient
// and factors.
//
// Every stage runs in the handle's SIMT precision R (double for KFAC_FP64,
// float for KFAC_FP32); the residuals, the loss and everything downstream of
// the factors stay FP64.  The layer and adjoint GEMMs go through the tiled
// SIMT GEMM of gemm_simt.cuh in R; the weight gradient and the factor Grams,
// sums over all collocation points, accumulate in FP64 from R operands; the
// tanh Taylor rule and its adjoint are element-wise kernels that walk the S
// shared columns of one (point, feature) pair.
#include "kfac_internal.cuh"
#include "gemm_simt.cuh"
#include "group.cuh"

using namespace kfac;

namespace {

constexpr int EW_THREADS = 256;

template <class R>
R* act(void* p) { return static_cast<R*>(p); }

// --------------------------------------------------------------------------
// First layer (Sec. 3.1): the inputs are (x, v_1..v_d, 0), so the tangent
// columns of Z^{(1)} are W_1 v_i (Wt, h x d column-major: the columns of W_1
// for the coordinate directions v_i = e_i) and its Laplacian column is 0.
// Writes Z^{(1)} and, when a tanh follows, T^{(1)} by the rule of Eq. 6 with
// the tangent channels weighted by chw (App. C.3).
// --------------------------------------------------------------------------
template <class R>
__global__ void k_layer1_fwd(const double* __restrict__ W, const double* __restrict__ Wt,
                             const double* __restrict__ X, R* __restrict__ Z, R* __restrict__ T,
                             int N, int d, int h, int S, const double* __restrict__ chw, int has_act) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)N * h) return;
    int n = (int)(idx / h), j = (int)(idx % h);
    R a0 = (R)W[(long long)j + (long long)h * d];   // bias column
    for (int k = 0; k < d; k++) a0 = fma((R)W[j + (long long)h * k], (R)X[(long long)n * d + k], a0);
    const long long blk = (long long)N * h;
    const long long o = (long long)n * h + j;
    Z[o] = a0;
    if (S > 1) {
        for (int i = 0; i < d; i++) Z[(1 + i) * blk + o] = (R)Wt[j + (long long)h * i];
        Z[(S - 1) * blk + o] = R(0);
    }
    if (!has_act) return;
    R y = tanh(a0);
    R s1 = R(1) - y * y;
    R s2 = R(-2) * y * s1;
    T[o] = y;
    if (S > 1) {
        R sumsq = R(0);
        for (int i = 0; i < d; i++) {
            R w = (R)Wt[j + (long long)h * i];
            T[(1 + i) * blk + o] = s1 * w;
            sumsq = fma((R)chw[i] * w, w, sumsq);
        }
        T[(S - 1) * blk + o] = s2 * sumsq;
    }
}

// Tanh through the Taylor columns (Eq. 6; App. C.3 for weighted channels):
//   y_0 = tanh(a_0), y_i = s1 a_i, y_D = s1 a_D + s2 sum_i w_i a_i^2
// with s1 = 1 - y_0^2 and s2 = -2 y_0 s1; w = chw (1 for a Laplacian
// channel, 0 for a channel outside the operator, the operator's eigenvalues
// for a general one).
template <class R>
__global__ void k_act_fwd(const R* __restrict__ Z, R* __restrict__ T, int N, int S, int h,
                          const double* __restrict__ chw) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long blk = (long long)N * h;
    if (idx >= blk) return;
    R a0 = Z[idx];
    R y = tanh(a0);
    R s1 = R(1) - y * y;
    T[idx] = y;
    if (S == 1) return;
    R s2 = R(-2) * y * s1;
    R sumsq = R(0);
    for (int s = 1; s < S - 1; s++) {
        R a = Z[s * blk + idx];
        T[s * blk + idx] = s1 * a;
        sumsq = fma((R)chw[s - 1] * a, a, sumsq);
    }
    T[(S - 1) * blk + idx] = fma(s1, Z[(S - 1) * blk + idx], s2 * sumsq);
}

// Adjoint of k_act_fwd, in place on G (incoming ybar -> outgoing abar):
//   abar_D = s1 ybar_D
//   abar_i = s1 ybar_i + 2 s2 w_i a_i ybar_D
//   abar_0 = s1 ybar_0 + s2 sum_i a_i ybar_i + (s2 a_D + s3 sum_i w_i a_i^2) ybar_D
// with s3 = -2 s1 (1 - 3 y^2).
template <class R>
__global__ void k_act_bwd(const R* __restrict__ Z, R* __restrict__ G, int N, int S, int h,
                          const double* __restrict__ chw) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long blk = (long long)N * h;
    if (idx >= blk) return;
    R a0 = Z[idx];
    R y = tanh(a0);
    R s1 = R(1) - y * y;
    if (S == 1) { G[idx] = s1 * G[idx]; return; }
    R s2 = R(-2) * y * s1;
    R s3 = R(-2) * s1 * (R(1) - R(3) * y * y);
    R yd = G[(S - 1) * blk + idx];
    R y0 = G[idx];
    R cross = R(0), sumsq = R(0);
    for (int s = 1; s < S - 1; s++) {
        R a = Z[s * blk + idx];
        R yb = G[s * blk + idx];
        cross = fma(a, yb, cross);
        R ab = s1 * yb;
        const R wa = (R)chw[s - 1] * a;
        sumsq = fma(wa, a, sumsq);
        ab = fma(R(2) * s2 * wa, yd, ab);
        G[s * blk + idx] = ab;
    }
    R aD = Z[(S - 1) * blk + idx];
    G[idx] = s1 * y0 + s2 * cross + (s2 * aD + s3 * sumsq) * yd;
    G[(S - 1) * blk + idx] = s1 * yd;
}

// Forward-mode derivative of k_act_fwd, in place on D (incoming da -> outgoing dy):
//   dy_0 = s1 da_0
//   dy_i = s2 da_0 a_i + s1 da_i
//   dy_D = s2 da_0 a_D + s1 da_D + s3 da_0 sum_i w_i a_i^2 + 2 s2 sum_i w_i a_i da_i
template <class R>
__global__ void k_act_jvp(const R* __restrict__ Z, R* __restrict__ Dz, int N, int S, int h,
                          const double* __restrict__ chw) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long blk = (long long)N * h;
    if (idx >= blk) return;
    R y = tanh(Z[idx]);
    R s1 = R(1) - y * y;
    R da0 = Dz[idx];
    Dz[idx] = s1 * da0;
    if (S == 1) return;
    R s2 = R(-2) * y * s1;
    R s3 = R(-2) * s1 * (R(1) - R(3) * y * y);
    R sumsq = R(0), cross = R(0);
    for (int s = 1; s < S - 1; s++) {
        R a = Z[s * blk + idx];
        R da = Dz[s * blk + idx];
        Dz[s * blk + idx] = fma(s2 * da0, a, s1 * da);
        const R wa = (R)chw[s - 1] * a;
        sumsq = fma(wa, a, sumsq);
        cross = fma(wa, da, cross);
    }
    R aD = Z[(S - 1) * blk + idx];
    R daD = Dz[(S - 1) * blk + idx];
    Dz[(S - 1) * blk + idx] = s2 * da0 * aD + s1 * daD + s3 * da0 * sumsq + R(2) * s2 * cross;
}

// Directional derivative of the residuals: the residual rule applied to dZ^{(L)}
// (the data f, g do not depend on theta).
template <class R>
__global__ void k_residual_jvp(const R* __restrict__ dZL, double* __restrict__ jv, int N, int S,
                               int interior, double cT, double cD) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double v;
    if (!interior) {
        v = (double)dZL[n];
    } else {
        v = cD * (double)dZL[(long long)(S - 1) * N + n];
        if (cT != 0.0) v += cT * (double)dZL[N + n];
    }
    jv[n] = v;
}

// Residuals (Eq. 1): interior r = cT z_t + cD z_D - f (cT: coefficient of the
// time tangent, heat only; cD of the Laplacian column), boundary r = u - g.
// FP64 from here on.
template <class R>
__global__ void k_residual(const R* __restrict__ ZL, const double* __restrict__ target,
                           double* __restrict__ r, int N, int S, int interior, double cT, double cD) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double v;
    if (!interior) {
        v = (double)ZL[n] - target[n];
    } else {
        v = cD * (double)ZL[(long long)(S - 1) * N + n];
        if (cT != 0.0) v += cT * (double)ZL[N + n];
        v -= target[n];
    }
    r[n] = v;
}

// Seed of the backward pass, c = dr/dZ^{(L)} (one row per point).
template <class R>
__global__ void k_seed(R* __restrict__ ZbL, int N, int S, int interior, double cT, double cD) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)N * S) return;
    int s = (int)(idx / N);
    double c = 0.0;
    if (!interior) c = 1.0;
    else c = (s == S - 1) ? cD : (s == 1 ? cT : 0.0);
    ZbL[idx] = (R)c;
}

// loss[1] = sum r^2 / (2N), loss[2] = sum rb^2 / (2Nb), loss[0] = loss[1] + loss[2].
// r_sq: r already holds the per-point r_n^T W r_n of a general residual.
struct k_loss {
    static constexpr int THREADS = 1024;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const double* __restrict__ r, int N, const double* __restrict__ rb,
                               int Nb, double* __restrict__ loss, int* status, int r_sq) {
        __shared__ double sh[2][32];
        double a = 0.0, b = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) a = r_sq ? a + r[i] : fma(r[i], r[i], a);
        for (int i = threadIdx.x; i < Nb; i += blockDim.x) b = fma(rb[i], rb[i], b);
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        int w = threadIdx.x / 32, l = threadIdx.x % 32;
        if (l == 0) { sh[0][w] = a; sh[1][w] = b; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double A = 0.0, B = 0.0;
            for (int i = 0; i < (int)(blockDim.x / 32); i++) { A += sh[0][i]; B += sh[1][i]; }
            double li = A / (2.0 * N), lb = B / (2.0 * Nb);
            loss[0] = li + lb;
            loss[1] = li;
            loss[2] = lb;
            if (status && !isfinite(li + lb)) latch_status(status, KFAC_NONFINITE);
        }
    }
};

// out[p*osp + q*osq] = (accumulate ? out : 0) + scale * sum_z part[z][p][q],
// or the EMA  out = beta * out + (1 - beta) * scale * sum_z part  when ema.
__global__ void k_reduce_partials(const double* __restrict__ part, int splits, int P, int Q,
                                  double scale, double* __restrict__ out, long long osp,
                                  long long osq, int accumulate, int ema, double beta,
                                  int* status) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long PQ = (long long)P * Q;
    if (idx >= PQ) return;
    double v = 0.0;
    for (int z = 0; z < splits; z++) v += part[z * PQ + idx];
    v *= scale;
    int p = (int)(idx / Q), q = (int)(idx % Q);
    long long o = (long long)p * osp + (long long)q * osq;
    if (ema) v = beta * out[o] + (1.0 - beta) * v;
    else if (accumulate) v += out[o];
    if (!isfinite(v)) latch_status(status, KFAC_NONFINITE);
    out[o] = v;
}

// Per-point sums over the S shared columns (KFAC-reduce reading):
// out[n*ncols + q] = scale * sum_s R(s*N + n, q), summed in FP64.
template <class Rows, class R>
__global__ void k_colsum(Rows rows, int N, int S, int ncols, double scale, R* __restrict__ out) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)N * ncols) return;
    int n = (int)(idx / ncols), q = (int)(idx % ncols);
    double v = 0.0;
    for (int s = 0; s < S; s++) v += (double)rows(s * N + n, q);
    out[idx] = (R)(scale * v);
}

// out = scale * (A^T B) over K rows (the sums over collocation points of the
// gradient and the Kronecker factors), split-K partial sums reduced in a fixed
// order.  The tiles accumulate in FP64 for either storage precision: the
// product of two FP32 operands is exact in FP64, so in FP32 storage these
// sums carry no rounding beyond the operands' own (the preconditioned update
// amplifies gradient errors in the factors' small-eigenvalue directions by up
// to ~1e3-1e4 at lambda = 1e-3).
template <class LA, class LB>
kfac_status_t reduce_gemm(kfac_pinn_handle* h, cudaStream_t s, int P, int Q, int K, LA la, LB lb,
                          double scale, double* out, long long osp, long long osq, int accumulate,
                          int ema, double beta) {
    int splits = choose_splits(P, Q, K, h->sm_count);
    long long cap = (long long)(h->part_elems / ((size_t)P * Q));
    if (cap < 1) return KFAC_BAD_ARG;
    if (splits > cap) splits = (int)cap;
    int kchunk = (K + splits - 1) / splits;
    kchunk = ((kchunk + GK - 1) / GK) * GK;
    if (kchunk < GK) kchunk = GK;
    splits = (K + kchunk - 1) / kchunk;
    timer_begin(h, KFAC_KC_GRAM, s);
    if (cudaSuccess != launch_dgemm<LA, LB, EpPartial, double>(s, P, Q, K, splits, la, lb, EpPartial{h->part, P, Q}))
        return KFAC_CUDA_ERROR;
    timer_end(h, KFAC_KC_GRAM, s, 2.0 * P * Q * (double)K);
    h->launches++;
    long long PQ = (long long)P * Q;
    k_reduce_partials<<<ceil_div_u(PQ, EW_THREADS), EW_THREADS, 0, s>>>(
        h->part, splits, P, Q, scale, out, osp, osq, accumulate, ema, beta, h->status);
    KFAC_LAUNCH_CHECK(h);
    return KFAC_OK;
}

// Tangent inputs of layer 1 for directions v_m = Q e_m: W_1 Q (h_1 x d,
// column-major, written to dst), or W_1 itself for the coordinate directions.
const double* tangent_inputs(kfac_pinn_handle* h, cudaStream_t s, const double* W1, double* dst) {
    if (!h->opQ) return W1;
    const int h1 = h->dims[1], d = h->dims[0];
    if (dgemm_strided(h, s, h1, d, d, W1, 1, h1, h->opQ, d, 1, dst, 1, h1, 1.0, 0.0) != KFAC_OK) return nullptr;
    return dst;
}

template <class R>
kfac_status_t forward_t(kfac_pinn_handle* h, cudaStream_t s, const double* theta, const double* X, int N,
                        PassBuffers& pb, int S) {
    const int L = h->cfg.L, d = h->dims[0];
    {
        int h1 = h->dims[1];
        long long cnt = (long long)N * h1;
        const double* Wt = tangent_inputs(h, s, theta + h->woff[0], h->w1q);
        if (!Wt) return KFAC_CUDA_ERROR;
        k_layer1_fwd<R><<<ceil_div_u(cnt, EW_THREADS), EW_THREADS, 0, s>>>(
            theta + h->woff[0], Wt, X, act<R>(pb.Z[0]), act<R>(pb.T[0]), N, d, h1, S, h->chw64, L > 1);
        KFAC_LAUNCH_CHECK(h);
    }
    for (int l = 2; l <= L; l++) {
        int hin = h->dims[l - 1], hout = h->dims[l];
        const double* W = theta + h->woff[l - 1];
        Strided<true, R> A{act<R>(pb.T[l - 2]), hin, 1};
        Strided<true> B{W, hout, 1};   // B(k, j) = W~[j, k] = W[j + hout*k]
        EpStore<R> ep{act<R>(pb.Z[l - 1]), hout, 1, 1.0, 0.0, W + (long long)hout * hin, 1, N};
        timer_begin(h, KFAC_KC_LAYER_GEMM, s);
        if (cudaSuccess != launch_dgemm<decltype(A), decltype(B), EpStore<R>, R>(s, S * N, hout, hin, 1, A, B, ep))
            return KFAC_CUDA_ERROR;
        timer_end(h, KFAC_KC_LAYER_GEMM, s, 2.0 * S * N * (double)hout * hin);
        h->launches++;
        if (l < L) {
            long long cnt = (long long)N * hout;
            timer_begin(h, KFAC_KC_ELEMENTWISE, s);
            k_act_fwd<R><<<ceil_div_u(cnt, EW_THREADS), EW_THREADS, 0, s>>>(
                act<R>(pb.Z[l - 1]), act<R>(pb.T[l - 1]), N, S, hout, h->chw64);
            timer_end(h, KFAC_KC_ELEMENTWISE, s, 2.0 * sizeof(R) * S * (double)cnt);
            KFAC_LAUNCH_CHECK(h);
        }
    }
    return KFAC_OK;
}

template <class R>
kfac_status_t residual_and_seed_t(kfac_pinn_handle* h, cudaStream_t s, PassBuffers& pb, int N, int S,
                                  const double* target, bool interior) {
    const int L = h->cfg.L;
    k_residual<R><<<ceil_div_u(N, EW_THREADS), EW_THREADS, 0, s>>>(act<R>(pb.Z[L - 1]), target, pb.r, N, S,
                                                                   interior, h->cT, h->cD);
    KFAC_LAUNCH_CHECK(h);
    k_seed<R><<<ceil_div_u((long long)N * S, EW_THREADS), EW_THREADS, 0, s>>>(act<R>(pb.Zb[L - 1]), N, S,
                                                                               interior, h->cT, h->cD);
    KFAC_LAUNCH_CHECK(h);
    return KFAC_OK;
}

template <class R>
kfac_status_t backward_t(kfac_pinn_handle* h, cudaStream_t s, const double* theta, PassBuffers& pb, int N,
                         int S) {
    const int L = h->cfg.L;
    for (int l = L; l >= 2; l--) {
        int hin = h->dims[l - 1], hout = h->dims[l];
        const double* W = theta + h->woff[l - 1];
        // Tbar = Zbar_l W_l (bias column dropped):  (S*N x hout)(hout x hin)
        Strided<true, R> A{act<R>(pb.Zb[l - 1]), hout, 1};
        Strided<false> B{W, 1, hout};  // B(i, q) = W~[i, q] = W[i + hout*q]
        EpStore<R> ep{act<R>(pb.Zb[l - 2]), hin, 1, 1.0, 0.0, nullptr, 0, 0};
        timer_begin(h, KFAC_KC_ADJOINT_GEMM, s);
        if (cudaSuccess != launch_dgemm<decltype(A), decltype(B), EpStore<R>, R>(s, S * N, hin, hout, 1, A, B, ep))
            return KFAC_CUDA_ERROR;
        timer_end(h, KFAC_KC_ADJOINT_GEMM, s, 2.0 * S * N * (double)hin * hout);
        h->launches++;
        long long cnt = (long long)N * hin;
        timer_begin(h, KFAC_KC_ELEMENTWISE, s);
        k_act_bwd<R><<<ceil_div_u(cnt, EW_THREADS), EW_THREADS, 0, s>>>(act<R>(pb.Z[l - 2]), act<R>(pb.Zb[l - 2]),
                                                                        N, S, hin, h->chw64);
        timer_end(h, KFAC_KC_ELEMENTWISE, s, 3.0 * sizeof(R) * S * (double)cnt);
        KFAC_LAUNCH_CHECK(h);
    }
    return KFAC_OK;
}

// general: the interior adjoint was seeded with W r_n (a general residual), so
// its rows enter the gradient unweighted, and B_Omega was formed beforehand.
template <class R, class RowsI, class RowsB>
kfac_status_t layer_grad_and_factors(kfac_pinn_handle* h, cudaStream_t s, int l, RowsI in_i,
                                     RowsB in_b, int N, int Nb, bool general) {
    const int S = h->S;
    const int hout = h->dims[l], nin = h->dims[l - 1] + 1;
    const double beta = h->cfg.beta;
    double* gW = h->grad + h->woff[l - 1];
    kfac_status_t st;
    // Weight gradient: (1/N) sum_rows r_n g_row T^_row^T  +  (1/Nb) sum ...
    {
        Transposed<WeightedRows<R>> A{WeightedRows<R>{act<R>(h->in.Zb[l - 1]), hout, N, general ? nullptr : h->in.r}};
        st = reduce_gemm(h, s, hout, nin, S * N, A, in_i, 1.0 / N, gW, 1, hout, 0, 0, 0.0);
        if (st != KFAC_OK) return st;
        Transposed<WeightedRows<R>> Ab{WeightedRows<R>{act<R>(h->bd.Zb[l - 1]), hout, Nb, h->bd.r}};
        st = reduce_gemm(h, s, hout, nin, Nb, Ab, in_b, 1.0 / Nb, gW, 1, hout, 1, 0, 0.0);
        if (st != KFAC_OK) return st;
    }
    // Interior factors.
    if (h->cfg.variant == KFAC_EXPAND) {
        st = reduce_gemm(h, s, nin, nin, S * N, Transposed<RowsI>{in_i}, in_i, 1.0 / ((double)N * S),
                            h->fac[KFAC_A_INT][l - 1], nin, 1, 0, 1, beta);
        if (st != KFAC_OK) return st;
        if (!general) {
            WeightedRows<R> G{act<R>(h->in.Zb[l - 1]), hout, N, nullptr};
            st = reduce_gemm(h, s, hout, hout, S * N, Transposed<WeightedRows<R>>{G}, G, 1.0 / N,
                                h->fac[KFAC_B_INT][l - 1], hout, 1, 0, 1, beta);
            if (st != KFAC_OK) return st;
        }
    } else {
        // KFAC-reduce: abar_n = (1/S) sum_s T^_{n,s}, gbar_n = sum_s g_{n,s}.
        R* ra = act<R>(h->in.red_a);
        R* rg = act<R>(h->in.red_g);
        k_colsum<<<ceil_div_u((long long)N * nin, EW_THREADS), EW_THREADS, 0, s>>>(in_i, N, S, nin, 1.0 / S, ra);
        KFAC_LAUNCH_CHECK(h);
        WeightedRows<R> G{act<R>(h->in.Zb[l - 1]), hout, N, nullptr};
        k_colsum<<<ceil_div_u((long long)N * hout, EW_THREADS), EW_THREADS, 0, s>>>(G, N, S, hout, 1.0, rg);
        KFAC_LAUNCH_CHECK(h);
        Strided<true, R> Ra{ra, nin, 1};
        Strided<true, R> Rg{rg, hout, 1};
        st = reduce_gemm(h, s, nin, nin, N, Strided<false, R>{ra, 1, nin}, Ra, 1.0 / N,
                            h->fac[KFAC_A_INT][l - 1], nin, 1, 0, 1, beta);
        if (st != KFAC_OK) return st;
        st = reduce_gemm(h, s, hout, hout, N, Strided<false, R>{rg, 1, hout}, Rg, 1.0 / N,
                            h->fac[KFAC_B_INT][l - 1], hout, 1, 0, 1, beta);
        if (st != KFAC_OK) return st;
    }
    // Boundary factors (classic KFAC, S = 1).
    st = reduce_gemm(h, s, nin, nin, Nb, Transposed<RowsB>{in_b}, in_b, 1.0 / Nb,
                        h->fac[KFAC_A_BDY][l - 1], nin, 1, 0, 1, beta);
    if (st != KFAC_OK) return st;
    WeightedRows<R> Gb{act<R>(h->bd.Zb[l - 1]), hout, Nb, nullptr};
    st = reduce_gemm(h, s, hout, hout, Nb, Transposed<WeightedRows<R>>{Gb}, Gb, 1.0 / Nb,
                        h->fac[KFAC_B_BDY][l - 1], hout, 1, 0, 1, beta);
    return st;
}

template <class R>
kfac_status_t grad_and_factors_t(kfac_pinn_handle* h, cudaStream_t s, const double* X_int, int N_int,
                                 const double* X_bdy, int N_bdy, bool general = false) {
    const int L = h->cfg.L, d = h->dims[0];
    for (int l = 1; l <= L; l++) {
        kfac_status_t st;
        if (l == 1) {
            st = layer_grad_and_factors<R>(h, s, 1, InputRows{X_int, d, N_int, h->opQ},
                                           InputRows{X_bdy, d, N_bdy, h->opQ}, N_int, N_bdy, general);
        } else {
            int hin = h->dims[l - 1];
            st = layer_grad_and_factors<R>(h, s, l, ActRows<R>{act<R>(h->in.T[l - 2]), hin, N_int},
                                           ActRows<R>{act<R>(h->bd.T[l - 2]), hin, N_bdy}, N_int, N_bdy, general);
        }
        if (st != KFAC_OK) return st;
    }
    return KFAC_OK;
}

// Output seed of the reverse pass through the Taylor forward: for a scalar
// phi(u, grad u, lap u), Zbar^{(L)}_{n,s} = dphi/dZ^{(L)}_{n,s} with the
// Taylor rows ordered (value, d tangents, Laplacian).  NULL inputs are zero.
// With tangent directions v_m = Q e_m the gradient is Q times the tangent
// outputs, so its upstream gradient maps to Q^T dgrad on the tangent rows.
template <class R>
__global__ void k_seed_upstream(R* __restrict__ ZbL, int N, int S, const double* __restrict__ Q,
                                const double* __restrict__ du, const double* __restrict__ dgrad,
                                const double* __restrict__ dlap) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)N * S) return;
    int s = (int)(idx / N), n = (int)(idx % N);
    const int d = S - 2;
    double c = 0.0;
    if (s == 0) c = du ? du[n] : 0.0;
    else if (s == S - 1) c = dlap ? dlap[n] : 0.0;
    else if (dgrad && !Q) c = dgrad[(long long)n * d + (s - 1)];
    else if (dgrad)
        for (int i = 0; i < d; i++) c = fma(Q[(long long)i * d + (s - 1)], dgrad[(long long)n * d + i], c);
    ZbL[idx] = (R)c;
}

template <class R>
kfac_status_t forward_laplacian_backward_t(kfac_pinn_handle* h, cudaStream_t s, const double* theta,
                                           const double* X, int N, const double* du, const double* dgrad,
                                           const double* dlap, double* dtheta, double* dX, bool accumulate,
                                           bool reuse_forward) {
    const int L = h->cfg.L, d = h->dims[0], S = h->S;
    kfac_status_t st;
    // the Taylor activations are recomputed unless the caller holds them from the
    // forward pass on the same inputs (stored mode)
    if (!reuse_forward && (st = forward_t<R>(h, s, theta, X, N, h->in, S))) return st;
    k_seed_upstream<R><<<ceil_div_u((long long)N * S, EW_THREADS), EW_THREADS, 0, s>>>(
        act<R>(h->in.Zb[L - 1]), N, S, h->opQ, du, dgrad, dlap);
    KFAC_LAUNCH_CHECK(h);
    if ((st = backward_t<R>(h, s, theta, h->in, N, S))) return st;
    // dphi/dW~_l = sum over rows (n, s) of g^{(l)}_{n,s} T^^{(l-1)T}_{n,s} (Sec. 3.2)
    for (int l = 1; l <= L; l++) {
        const int hout = h->dims[l], nin = h->dims[l - 1] + 1;
        Transposed<WeightedRows<R>> A{WeightedRows<R>{act<R>(h->in.Zb[l - 1]), hout, N, nullptr}};
        double* gW = dtheta + h->woff[l - 1];
        if (l == 1)
            st = reduce_gemm(h, s, hout, nin, S * N, A, InputRows{X, d, N, h->opQ}, 1.0, gW, 1, hout,
                                accumulate, 0, 0.0);
        else
            st = reduce_gemm(h, s, hout, nin, S * N, A, ActRows<R>{act<R>(h->in.T[l - 2]), nin - 1, N}, 1.0,
                                gW, 1, hout, accumulate, 0, 0.0);
        if (st) return st;
    }
    // dphi/dx_n = W_1^T g^{(1)}_{n,0}: x enters the value column of layer 1 only
    // (the tangent inputs e_i and the zero Laplacian input are constants).
    if (dX) {
        const int h1 = h->dims[1];
        Strided<true, R> A{act<R>(h->in.Zb[0]), h1, 1};
        Strided<false> B{theta, 1, h1};   // B(j, i) = W_1[j, i] = theta[j + h1 * i]
        EpStore<double> ep{dX, d, 1, 1.0, 0.0, nullptr, 0, 0};
        if (cudaSuccess != launch_dgemm<decltype(A), decltype(B), EpStore<double>, R>(s, N, d, h1, 1, A, B, ep))
            return KFAC_CUDA_ERROR;
        h->launches++;
    }
    return KFAC_OK;
}

// J_theta r . v for one pass whose forward activations (Z, T) at theta are in
// pb: the Taylor pass differentiated in the direction v (Sec. 3.1-3.2),
//   dZ^{(1)} = dW~_1 T^^{(0)},  dZ^{(l)} = dW~_l T^^{(l-1)} + W_l dT^{(l-1)},
// with dT from the linearised tanh rule.  Overwrites pb.Zb; jv: N doubles.
template <class R>
kfac_status_t jvp_t(kfac_pinn_handle* h, cudaStream_t s, const double* theta, const double* v, const double* X,
                    int N, PassBuffers& pb, int S, bool interior, double* jv) {
    const int L = h->cfg.L, d = h->dims[0];
    {
        const int h1 = h->dims[1];
        long long cnt = (long long)N * h1;
        const double* Vt = tangent_inputs(h, s, v + h->woff[0], h->w1q2);
        if (!Vt) return KFAC_CUDA_ERROR;
        k_layer1_fwd<R><<<ceil_div_u(cnt, EW_THREADS), EW_THREADS, 0, s>>>(v + h->woff[0], Vt, X, act<R>(pb.Zb[0]),
                                                                           nullptr, N, d, h1, S, h->chw64, 0);
        KFAC_LAUNCH_CHECK(h);
        if (L > 1) {
            k_act_jvp<R><<<ceil_div_u(cnt, EW_THREADS), EW_THREADS, 0, s>>>(act<R>(pb.Z[0]), act<R>(pb.Zb[0]), N, S,
                                                                            h1, h->chw64);
            KFAC_LAUNCH_CHECK(h);
        }
    }
    for (int l = 2; l <= L; l++) {
        const int hin = h->dims[l - 1], hout = h->dims[l];
        const double* W = theta + h->woff[l - 1];
        const double* V = v + h->woff[l - 1];
        // dZ = T dW^T (+ db on the value rows)
        {
            Strided<true, R> A{act<R>(pb.T[l - 2]), hin, 1};
            Strided<true> B{V, hout, 1};
            EpStore<R> ep{act<R>(pb.Zb[l - 1]), hout, 1, 1.0, 0.0, V + (long long)hout * hin, 1, N};
            timer_begin(h, KFAC_KC_LAYER_GEMM, s);
            if (cudaSuccess != launch_dgemm<decltype(A), decltype(B), EpStore<R>, R>(s, S * N, hout, hin, 1, A, B, ep))
                return KFAC_CUDA_ERROR;
            timer_end(h, KFAC_KC_LAYER_GEMM, s, 2.0 * S * N * (double)hout * hin);
            h->launches++;
        }
        // dZ += dT W^T
        {
            Strided<true, R> A{act<R>(pb.Zb[l - 2]), hin, 1};
            Strided<true> B{W, hout, 1};
            EpStore<R> ep{act<R>(pb.Zb[l - 1]), hout, 1, 1.0, 1.0, nullptr, 0, 0};
            timer_begin(h, KFAC_KC_LAYER_GEMM, s);
            if (cudaSuccess != launch_dgemm<decltype(A), decltype(B), EpStore<R>, R>(s, S * N, hout, hin, 1, A, B, ep))
                return KFAC_CUDA_ERROR;
            timer_end(h, KFAC_KC_LAYER_GEMM, s, 2.0 * S * N * (double)hout * hin);
            h->launches++;
        }
        if (l < L) {
            long long cnt = (long long)N * hout;
            k_act_jvp<R><<<ceil_div_u(cnt, EW_THREADS), EW_THREADS, 0, s>>>(act<R>(pb.Z[l - 1]), act<R>(pb.Zb[l - 1]),
                                                                            N, S, hout, h->chw64);
            KFAC_LAUNCH_CHECK(h);
        }
    }
    k_residual_jvp<R><<<ceil_div_u(N, EW_THREADS), EW_THREADS, 0, s>>>(act<R>(pb.Zb[L - 1]), jv, N, S, interior,
                                                                       h->cT, h->cD);
    KFAC_LAUNCH_CHECK(h);
    return KFAC_OK;
}

// u, grad u and the operator column; with tangent directions v_m = Q e_m the
// gradient is grad u = sum_m Q[:, m] (directional derivative along v_m).
template <class R>
__global__ void k_extract(const R* __restrict__ ZL, int N, int S, int d, const double* __restrict__ Q,
                          double* u, double* grad, double* lap) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    if (u) u[n] = (double)ZL[n];
    if (grad) {
        if (!Q) {
            for (int i = 0; i < d; i++) grad[(long long)n * d + i] = (double)ZL[(long long)(1 + i) * N + n];
        } else {
            for (int i = 0; i < d; i++) {
                double acc = 0.0;
                for (int m = 0; m < d; m++)
                    acc = fma(Q[(long long)i * d + m], (double)ZL[(long long)(1 + m) * N + n], acc);
                grad[(long long)n * d + i] = acc;
            }
        }
    }
    if (lap) lap[n] = (double)ZL[(long long)(S - 1) * N + n];
}

// --------------------------------------------------------------------------
// General interior residual (Sec. 3.3): with z_n = Z^{(L)}_n (S outputs, in the
// column-block layout ZL[s * N + n]) and the coefficients b (M x S), W, its
// Cholesky factor L_W (M x M) and Q (M x S x S) one after another in coef,
//   r_{n,k} = b_k . z_n + 1/2 z_n^T Q_k z_n - f_{n,k},
//   J_{n,k,s} = dr_{n,k} / dz_{n,s} = b[k,s] + sum_t Q[k,s,t] z_{n,t}.
// --------------------------------------------------------------------------
struct ResCoef {
    const double* b;
    const double* W;
    const double* Lw;
    const double* Q;     // nullptr: linear
    int M, S;
};

// r (N x M) and the per-point r_n^T W r_n (rq, N); one thread per point.
template <class R>
__global__ void k_residual_general(const R* __restrict__ ZL, const double* __restrict__ f, ResCoef c, int N,
                                   double* __restrict__ r, double* __restrict__ rq) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double rk[KFAC_MAX_RESIDUALS];
    for (int k = 0; k < c.M; k++) {
        double v = -f[(long long)n * c.M + k];
        for (int s2 = 0; s2 < c.S; s2++) {
            const double zs = (double)ZL[(long long)s2 * N + n];
            v = fma(c.b[k * c.S + s2], zs, v);
            if (c.Q) {
                const double* q = c.Q + ((long long)k * c.S + s2) * c.S;
                double qz = 0.0;
                for (int t = 0; t < c.S; t++) qz = fma(q[t], (double)ZL[(long long)t * N + n], qz);
                v = fma(0.5 * zs, qz, v);
            }
        }
        rk[k] = v;
        r[(long long)n * c.M + k] = v;
    }
    double acc = 0.0;
    for (int k = 0; k < c.M; k++)
        for (int j = 0; j < c.M; j++) acc = fma(rk[k] * c.W[k * c.M + j], rk[j], acc);
    rq[n] = acc;
}

// Seed of one interior adjoint pass, Zbar^{(L)}_{n,s} = sum_k w_{n,k} J_{n,k,s}
// with w_n = L_W[:, mode] (the mode-th term of the outer-product rewrite of
// Lambda = W, Sec. 3.3) or, for mode = -1, w_n = W r_n (the loss gradient).
template <class R>
__global__ void k_seed_general(const R* __restrict__ ZL, const double* __restrict__ r, ResCoef c, int N, int mode,
                               R* __restrict__ ZbL) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)N * c.S) return;
    const int s2 = (int)(idx / N), n = (int)(idx % N);
    double acc = 0.0;
    for (int k = 0; k < c.M; k++) {
        double w;
        if (mode >= 0) {
            w = c.Lw[k * c.M + mode];
        } else {
            w = 0.0;
            for (int j = 0; j < c.M; j++) w = fma(c.W[k * c.M + j], r[(long long)n * c.M + j], w);
        }
        if (w == 0.0) continue;
        double J = c.b[k * c.S + s2];
        if (c.Q) {
            const double* q = c.Q + ((long long)k * c.S + s2) * c.S;
            for (int t = 0; t < c.S; t++) J = fma(q[t], (double)ZL[(long long)t * N + n], J);
        }
        acc = fma(w, J, acc);
    }
    ZbL[idx] = (R)acc;
}

ResCoef res_coef(const kfac_pinn_handle* h) {
    ResCoef c;
    c.M = h->res_M;
    c.S = h->S;
    c.b = h->res_coef;
    c.W = c.b + (size_t)c.M * c.S;
    c.Lw = c.W + (size_t)c.M * c.M;
    c.Q = h->res_has_Q ? c.Lw + (size_t)c.M * c.M : nullptr;
    return c;
}

template <class R>
kfac_status_t residual_general_t(kfac_pinn_handle* h, cudaStream_t s, int N, const double* f) {
    const int L = h->cfg.L;
    k_residual_general<R><<<ceil_div_u(N, EW_THREADS), EW_THREADS, 0, s>>>(act<R>(h->in.Z[L - 1]), f, res_coef(h),
                                                                           N, h->res_r, h->in.r);
    KFAC_LAUNCH_CHECK(h);
    return KFAC_OK;
}

// After both forward passes and the boundary adjoint: B_Omega of every layer
// from M seeded interior adjoint passes (Eq. 10 in the outer-product form,
// accumulated into the EMA), then the gradient pass and, with it, the
// gradient, A_Omega, A_bdy and B_bdy of every layer.
template <class R>
kfac_status_t backward_and_factors_general_t(kfac_pinn_handle* h, cudaStream_t s, const double* theta,
                                             const double* X_int, int N_int, const double* X_bdy, int N_bdy) {
    const int L = h->cfg.L, S = h->S, M = h->res_M;
    const double beta = h->cfg.beta;
    const ResCoef c = res_coef(h);
    const unsigned sg = ceil_div_u((long long)N_int * S, EW_THREADS);
    kfac_status_t st;
    for (int m = 0; m < M; m++) {
        k_seed_general<R><<<sg, EW_THREADS, 0, s>>>(act<R>(h->in.Z[L - 1]), h->res_r, c, N_int, m,
                                                    act<R>(h->in.Zb[L - 1]));
        KFAC_LAUNCH_CHECK(h);
        if ((st = backward_t<R>(h, s, theta, h->in, N_int, S))) return st;
        for (int l = 1; l <= L; l++) {
            const int hout = h->dims[l];
            WeightedRows<R> G{act<R>(h->in.Zb[l - 1]), hout, N_int, nullptr};
            // first term: the EMA step; the others add (1 - beta) / N of their Gram
            st = reduce_gemm(h, s, hout, hout, S * N_int, Transposed<WeightedRows<R>>{G}, G,
                             m == 0 ? 1.0 / N_int : (1.0 - beta) / N_int, h->fac[KFAC_B_INT][l - 1], hout, 1,
                             m == 0 ? 0 : 1, m == 0 ? 1 : 0, beta);
            if (st) return st;
        }
    }
    k_seed_general<R><<<sg, EW_THREADS, 0, s>>>(act<R>(h->in.Z[L - 1]), h->res_r, c, N_int, -1,
                                                act<R>(h->in.Zb[L - 1]));
    KFAC_LAUNCH_CHECK(h);
    if ((st = backward_t<R>(h, s, theta, h->in, N_int, S))) return st;
    return grad_and_factors_t<R>(h, s, X_int, N_int, X_bdy, N_bdy, true);
}

inline bool fp32_storage(const kfac_pinn_handle* h) { return h->cfg.precision == KFAC_FP32; }

}  // namespace

// --------------------------------------------------------------------------
// Library-internal entry points of the SIMT path (FP64 or FP32 by the handle)
// --------------------------------------------------------------------------
size_t simt_elem_bytes(const kfac_pinn_handle* h) { return fp32_storage(h) ? sizeof(float) : sizeof(double); }

kfac_status_t simt_forward(kfac_pinn_handle* h, cudaStream_t s, const double* theta, const double* X, int N,
                           PassBuffers& pb, int S) {
    return fp32_storage(h) ? forward_t<float>(h, s, theta, X, N, pb, S) : forward_t<double>(h, s, theta, X, N, pb, S);
}

kfac_status_t simt_residual_and_seed(kfac_pinn_handle* h, cudaStream_t s, PassBuffers& pb, int N, int S,
                                     const double* target, bool interior) {
    return fp32_storage(h) ? residual_and_seed_t<float>(h, s, pb, N, S, target, interior)
                           : residual_and_seed_t<double>(h, s, pb, N, S, target, interior);
}

kfac_status_t simt_backward(kfac_pinn_handle* h, cudaStream_t s, const double* theta, PassBuffers& pb, int N, int S) {
    return fp32_storage(h) ? backward_t<float>(h, s, theta, pb, N, S) : backward_t<double>(h, s, theta, pb, N, S);
}

kfac_status_t simt_grad_and_factors(kfac_pinn_handle* h, cudaStream_t s, const double* X_int, int N_int,
                                    const double* X_bdy, int N_bdy) {
    return fp32_storage(h) ? grad_and_factors_t<float>(h, s, X_int, N_int, X_bdy, N_bdy)
                           : grad_and_factors_t<double>(h, s, X_int, N_int, X_bdy, N_bdy);
}

kfac_status_t fp64_loss(kfac_pinn_handle* h, cudaStream_t s, int N_int, int N_bdy, double* loss_out) {
    KFAC_TRY(KL<k_loss>(h, s, 1, 0, h->in.r, N_int, h->bd.r, N_bdy, h->loss, h->status, h->res_M > 0));
    if (loss_out && loss_out != h->loss) return group_copy(h, s, loss_out, h->loss, 3 * sizeof(double));
    return KFAC_OK;
}

// Loss of the residuals in h->in.r / h->bd.r written to dst (3 doubles); a
// non-finite value is recorded, not latched (line-search trials may diverge).
kfac_status_t fp64_loss_to(kfac_pinn_handle* h, cudaStream_t s, int N_int, int N_bdy, double* dst) {
    KFAC_TRY(KL<k_loss>(h, s, 1, 0, h->in.r, N_int, h->bd.r, N_bdy, dst, nullptr, h->res_M > 0));
    return KFAC_OK;
}

kfac_status_t simt_residual_general(kfac_pinn_handle* h, cudaStream_t s, int N, const double* f) {
    return fp32_storage(h) ? residual_general_t<float>(h, s, N, f) : residual_general_t<double>(h, s, N, f);
}

kfac_status_t simt_backward_and_factors_general(kfac_pinn_handle* h, cudaStream_t s, const double* theta,
                                                const double* X_int, int N_int, const double*, const double* X_bdy,
                                                int N_bdy) {
    return fp32_storage(h) ? backward_and_factors_general_t<float>(h, s, theta, X_int, N_int, X_bdy, N_bdy)
                           : backward_and_factors_general_t<double>(h, s, theta, X_int, N_int, X_bdy, N_bdy);
}

kfac_status_t simt_eval_loss(kfac_pinn_handle* h, cudaStream_t s, const double* theta, const double* X_int,
                             int N_int, const double* f, const double* X_bdy, int N_bdy, const double* g,
                             double* dst) {
    kfac_status_t st;
    if ((st = simt_forward(h, s, theta, X_int, N_int, h->in, h->S))) return st;
    if (h->res_M > 0) st = simt_residual_general(h, s, N_int, f);
    else st = simt_residual_and_seed(h, s, h->in, N_int, h->S, f, true);
    if (st) return st;
    if ((st = simt_forward(h, s, theta, X_bdy, N_bdy, h->bd, 1))) return st;
    if ((st = simt_residual_and_seed(h, s, h->bd, N_bdy, 1, g, false))) return st;
    return fp64_loss_to(h, s, N_int, N_bdy, dst);
}

kfac_status_t simt_forward_laplacian_backward(kfac_pinn_handle* h, cudaStream_t s, const double* theta,
                                              const double* X, int N, const double* du, const double* dgrad,
                                              const double* dlap, double* dtheta, double* dX, bool accumulate,
                                              bool reuse_forward) {
    return fp32_storage(h)
               ? forward_laplacian_backward_t<float>(h, s, theta, X, N, du, dgrad, dlap, dtheta, dX, accumulate,
                                                     reuse_forward)
               : forward_laplacian_backward_t<double>(h, s, theta, X, N, du, dgrad, dlap, dtheta, dX, accumulate,
                                                      reuse_forward);
}

kfac_status_t simt_jvp(kfac_pinn_handle* h, cudaStream_t s, const double* theta, const double* v, const double* X,
                       int N, PassBuffers& pb, int S, bool interior, double* jv) {
    return fp32_storage(h) ? jvp_t<float>(h, s, theta, v, X, N, pb, S, interior, jv)
                           : jvp_t<double>(h, s, theta, v, X, N, pb, S, interior, jv);
}

kfac_status_t simt_extract_outputs(kfac_pinn_handle* h, cudaStream_t s, PassBuffers& pb, int N, int S, double* u,
                                   double* grad, double* lap) {
    const int L = h->cfg.L;
    if (fp32_storage(h))
        k_extract<float><<<ceil_div_u(N, EW_THREADS), EW_THREADS, 0, s>>>(act<float>(pb.Z[L - 1]), N, S, h->dims[0],
                                                                          h->opQ, u, grad, lap);
    else
        k_extract<double><<<ceil_div_u(N, EW_THREADS), EW_THREADS, 0, s>>>(act<double>(pb.Z[L - 1]), N, S,
                                                                           h->dims[0], h->opQ, u, grad, lap);
    KFAC_LAUNCH_CHECK(h);
    return KFAC_OK;
}

// Generic strided FP64 GEMM used by the linear-algebra code.
kfac_status_t dgemm_strided(kfac_pinn_handle* h, cudaStream_t s, int P, int Q, int K,
                            const double* A, long long a_sp, long long a_sk,
                            const double* B, long long b_sk, long long b_sq,
                            double* C, long long c_sp, long long c_sq, double alpha, double beta, bool fp32) {
    EpStore<double> ep{C, c_sp, c_sq, alpha, beta, nullptr, 0, 0};
    using E = EpStore<double>;
    cudaError_t e;
    bool akf = (a_sk == 1), bqf = (b_sq == 1);
    if (fp32) {
        if (akf && bqf)
            e = launch_dgemm<Strided<true>, Strided<true>, E, float>(
                s, P, Q, K, 1, Strided<true>{A, a_sp, a_sk}, Strided<true>{B, b_sk, b_sq}, ep);
        else if (akf)
            e = launch_dgemm<Strided<true>, Strided<false>, E, float>(
                s, P, Q, K, 1, Strided<true>{A, a_sp, a_sk}, Strided<false>{B, b_sk, b_sq}, ep);
        else if (bqf)
            e = launch_dgemm<Strided<false>, Strided<true>, E, float>(
                s, P, Q, K, 1, Strided<false>{A, a_sp, a_sk}, Strided<true>{B, b_sk, b_sq}, ep);
        else
            e = launch_dgemm<Strided<false>, Strided<false>, E, float>(
                s, P, Q, K, 1, Strided<false>{A, a_sp, a_sk}, Strided<false>{B, b_sk, b_sq}, ep);
    } else {
        if (akf && bqf) e = launch_dgemm(s, P, Q, K, 1, Strided<true>{A, a_sp, a_sk}, Strided<true>{B, b_sk, b_sq}, ep);
        else if (akf) e = launch_dgemm(s, P, Q, K, 1, Strided<true>{A, a_sp, a_sk}, Strided<false>{B, b_sk, b_sq}, ep);
        else if (bqf) e = launch_dgemm(s, P, Q, K, 1, Strided<false>{A, a_sp, a_sk}, Strided<true>{B, b_sk, b_sq}, ep);
        else e = launch_dgemm(s, P, Q, K, 1, Strided<false>{A, a_sp, a_sk}, Strided<false>{B, b_sk, b_sq}, ep);
    }
    h->launches++;
    return e == cudaSuccess ? KFAC_OK : KFAC_CUDA_ERROR;
}
