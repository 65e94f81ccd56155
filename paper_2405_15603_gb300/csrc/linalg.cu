// Damped Kronecker-sum preconditioning and the parameter update (Sec. 3.4).
//
// With V_A, a and V_B, b from the simultaneous diagonalisation of the damped
// factor pairs (eig.cu: V^T A~_Omega V = I, V^T A~_bdy V = diag(a)),
//     (A~_Omega (x) B~_Omega + A~_bdy (x) B~_bdy)^{-1} vec G
//         = vec( V_B [ (V_B^T G V_A) / (1 + b a^T) ] V_A^T ),
// which is exact because vec(B X A) = (A^T (x) B) vec X (Sec. 2).
#include "kfac_internal.cuh"
#include "group.cuh"
#include "tc_path.cuh"

namespace {

struct k_div_kron {
    static constexpr int THREADS = 256;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, double* Y, int nb, int na, const double* wb, const double* wa) {
        long long idx = (long long)vb.x * blockDim.x + threadIdx.x;
        if (idx >= (long long)nb * na) return;
        int p = (int)(idx / na), q = (int)(idx % na);
        Y[idx] /= (1.0 + wb[p] * wa[q]);
    }
};

// delta = lr (mu delta_prev + Delta); theta += delta (Sec. 3.4, fixed learning rate).
struct k_update {
    static constexpr int THREADS = 256;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, double* theta, const double* dir, double* delta_prev, long long D,
                               double lr, double mom, double* coef) {
        long long i = (long long)vb.x * blockDim.x + threadIdx.x;
        if (i == 0) {
            coef[0] = lr;
            coef[1] = lr * mom;
        }
        if (i >= D) return;
        double dlt = lr * (mom * delta_prev[i] + dir[i]);
        delta_prev[i] = dlt;
        theta[i] += dlt;
    }
};

// Line search over the grid alpha_k = 2^-k, k = 0..LS_GRID-1 (Sec. 3.4).
constexpr int LS_GRID = 31;

// dhat = mu delta_prev + Delta (delta_prev is zero before the first step).
struct k_dhat {
    static constexpr int THREADS = 256;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const double* dir, const double* delta_prev, double* dhat,
                               long long D, double mom) {
        long long i = (long long)vb.x * blockDim.x + threadIdx.x;
        if (i >= D) return;
        dhat[i] = mom * delta_prev[i] + dir[i];
    }
};

struct k_trial {
    static constexpr int THREADS = 256;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const double* theta, const double* dhat, double* trial,
                               long long D, double alpha) {
        long long i = (long long)vb.x * blockDim.x + threadIdx.x;
        if (i >= D) return;
        trial[i] = theta[i] + alpha * dhat[i];
    }
};

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
struct k_ls_apply {
    static constexpr int THREADS = 256;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, double* theta, const double* dhat, double* delta_prev, long long D,
                               const double* ls_loss, int* status, double mom, double* coef) {
        __shared__ int best;
        if (threadIdx.x == 0) {
            best = ls_argmin(ls_loss);
            if (best < 0 && vb.x == 0) latch_status(status, KFAC_NONFINITE);
        }
        __syncthreads();
        const double alpha = best < 0 ? 0.0 : ldexp(1.0, -best);
        if (vb.x == 0 && threadIdx.x == 0) {
            coef[0] = alpha;
            coef[1] = alpha * mom;
        }
        if (best < 0) return;       // no finite trial: theta and delta_prev stay as they are
        for (long long i = (long long)vb.x * blockDim.x + threadIdx.x; i < D;
             i += (long long)vg.x * blockDim.x) {
            double dlt = alpha * dhat[i];
            delta_prev[i] = dlt;
            theta[i] += dlt;
        }
    }
};

// KFAC*: (alpha*, mu*) = argmin of the quadratic model
//   m(alpha Delta + mu delta) = L + (alpha Delta + mu delta)^T g
//                              + 1/2 (alpha Delta + mu delta)^T (G + lambda I) (alpha Delta + mu delta)
// (Sec. 3.4), with v^T G w = (1/N) sum_n (J_n v)(J_n w) + (1/N_b) sum_b (J_b v)(J_b w)
// (Eq. 2) from the residual JVPs.  Eleven sums, reduced in a fixed order.
constexpr int KS_BLOCKS = 256;
constexpr int KS_Q = 11;

__device__ double ks_block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x / 32); w++) t += sh[w];
    return t;
}

struct k_ks_dots {
    static constexpr int THREADS = 256;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const double* __restrict__ Dl, const double* __restrict__ dl,
                               const double* __restrict__ g, long long D, const double* __restrict__ jDi,
                               const double* __restrict__ jdi, int Ni, const double* __restrict__ jDb,
                               const double* __restrict__ jdb, int Nb, int have_prev, double* part) {
        __shared__ double sh[8];
        double acc[KS_Q];
    #pragma unroll
        for (int q = 0; q < KS_Q; q++) acc[q] = 0.0;
        const long long stride = (long long)vg.x * blockDim.x;
        const long long i0 = (long long)vb.x * blockDim.x + threadIdx.x;
        for (long long i = i0; i < D; i += stride) {
            const double a = Dl[i], b = have_prev ? dl[i] : 0.0, gi = g[i];
            acc[0] = fma(a, a, acc[0]);
            acc[1] = fma(a, b, acc[1]);
            acc[2] = fma(b, b, acc[2]);
            acc[3] = fma(a, gi, acc[3]);
            acc[4] = fma(b, gi, acc[4]);
        }
        for (long long i = i0; i < Ni; i += stride) {
            const double a = jDi[i], b = have_prev ? jdi[i] : 0.0;
            acc[5] = fma(a, a, acc[5]);
            acc[6] = fma(a, b, acc[6]);
            acc[7] = fma(b, b, acc[7]);
        }
        for (long long i = i0; i < Nb; i += stride) {
            const double a = jDb[i], b = have_prev ? jdb[i] : 0.0;
            acc[8] = fma(a, a, acc[8]);
            acc[9] = fma(a, b, acc[9]);
            acc[10] = fma(b, b, acc[10]);
        }
    #pragma unroll
        for (int q = 0; q < KS_Q; q++) {
            double t = ks_block_sum(acc[q], sh);
            if (threadIdx.x == 0) part[(long long)vb.x * KS_Q + q] = t;
        }
    }
};

struct k_ks_solve {
    static constexpr int THREADS = 32;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const double* __restrict__ part, int nblocks, int Ni, int Nb,
                               double lam, int have_prev, double* coef, int* status) {
        __shared__ double tot[KS_Q];
        if (threadIdx.x < KS_Q) {
            double t = 0.0;
            for (int b = 0; b < nblocks; b++) t += part[(long long)b * KS_Q + threadIdx.x];
            tot[threadIdx.x] = t;
        }
        __syncthreads();
        if (threadIdx.x != 0) return;
        const double a11 = tot[5] / Ni + tot[8] / Nb + lam * tot[0];
        const double b1 = tot[3];
        double alpha, mu = 0.0, a12 = 0.0, a22 = 0.0, b2 = 0.0;
        if (have_prev && tot[2] > 0.0) {
            a12 = tot[6] / Ni + tot[9] / Nb + lam * tot[1];
            a22 = tot[7] / Ni + tot[10] / Nb + lam * tot[2];
            b2 = tot[4];
            const double det = a11 * a22 - a12 * a12;
            alpha = -(a22 * b1 - a12 * b2) / det;
            mu = -(a11 * b2 - a12 * b1) / det;
        } else {
            alpha = -b1 / a11;
        }
        double skip = 0.0;
        if (!(a11 > 0.0) || !isfinite(alpha) || !isfinite(mu)) {
            latch_status(status, KFAC_NONFINITE);
            alpha = 0.0;
            mu = 0.0;
            skip = 1.0;
        }
        coef[7] = skip;
        coef[0] = alpha;
        coef[1] = mu;
        coef[2] = a11;
        coef[3] = a12;
        coef[4] = a22;
        coef[5] = b1;
        coef[6] = b2;
    }
};

// delta = alpha* Delta + mu* delta_prev; theta += delta.
struct k_ks_apply {
    static constexpr int THREADS = 256;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, double* theta, const double* __restrict__ Dl, double* delta_prev,
                               long long D, const double* __restrict__ coef) {
        long long i = (long long)vb.x * blockDim.x + threadIdx.x;
        if (i >= D || coef[7] != 0.0) return;       // a non-finite model leaves theta unchanged
        const double dlt = coef[0] * Dl[i] + coef[1] * delta_prev[i];
        delta_prev[i] = dlt;
        theta[i] += dlt;
    }
};

// Batched FP32 GEMM of the mixed path's preconditioning: one launch runs the
// same stage for every layer (C = alpha op(A) op(B), operands read as FP64
// through strides and rounded to FP32, FP32 accumulation, FP64 result;
// optionally divided by 1 + dr[p] dc[q]).  64 x 64 tiles, 16-deep k slices,
// 256 threads with a 4 x 4 block of consecutive rows and columns each (vector
// shared-memory loads); the tiles of all layers form one grid.
struct PGemm {
    const double* A;
    long long a_sp, a_sk;
    const double* B;
    long long b_sk, b_sq;
    double* C;
    long long c_sp, c_sq;
    const double* dr;
    const double* dc;
    int P, Q, K, tiles_q, tile0;
    double alpha;
};
struct PBatch {
    PGemm g[KFAC_MAX_LAYERS];
    int n;
};

struct k_pgemm_f32 {
    static constexpr int THREADS = 256;
    __device__ __noinline__ static void run(uint3 vb, uint3 vg, const PBatch& b) {
        __shared__ __align__(16) float As[16][68];
        __shared__ __align__(16) float Bs[16][68];
        int gi = 0;
        while (gi + 1 < b.n && (int)vb.x >= b.g[gi + 1].tile0) gi++;
        const PGemm& g = b.g[gi];
        const int t = (int)vb.x - g.tile0;
        const int p0 = (t / g.tiles_q) * 64, q0 = (t % g.tiles_q) * 64;
        const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
        const bool akf = g.a_sk == 1, bqf = g.b_sq == 1;
        float acc[4][4];
    #pragma unroll
        for (int i = 0; i < 4; i++)
    #pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] = 0.f;
        for (int k0 = 0; k0 < g.K; k0 += 16) {
    #pragma unroll
            for (int i = 0; i < 4; i++) {
                const int e = tid + 256 * i;
                const int kk = akf ? e % 16 : e / 64, pp = akf ? e / 16 : e % 64;
                const int pr = p0 + pp, k = k0 + kk;
                As[kk][pp] = (pr < g.P && k < g.K) ? (float)g.A[(long long)pr * g.a_sp + (long long)k * g.a_sk] : 0.f;
                const int qq = bqf ? e % 64 : e / 16, kb = bqf ? e / 64 : e % 16;
                const int q = q0 + qq, kq = k0 + kb;
                Bs[kb][qq] = (q < g.Q && kq < g.K) ? (float)g.B[(long long)kq * g.b_sk + (long long)q * g.b_sq] : 0.f;
            }
            __syncthreads();
    #pragma unroll
            for (int kk = 0; kk < 16; kk++) {
                const float4 a4 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
                const float4 b4 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
                const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
    #pragma unroll
                for (int i = 0; i < 4; i++)
    #pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
            __syncthreads();
        }
    #pragma unroll
        for (int i = 0; i < 4; i++) {
            const int pr = p0 + ty * 4 + i;
            if (pr >= g.P) continue;
    #pragma unroll
            for (int j = 0; j < 4; j++) {
                const int q = q0 + tx * 4 + j;
                if (q >= g.Q) continue;
                float v = (float)g.alpha * acc[i][j];
                if (g.dr) v /= 1.f + (float)(g.dr[pr] * g.dc[q]);
                g.C[(long long)pr * g.c_sp + (long long)q * g.c_sq] = (double)v;
            }
        }
    }
};

// One stage over all layers: the stage's GEMM of layer l has the shape
// (P, Q, K) = (nb, na, K_l) and strides from `desc`.
template <class F>
kfac_status_t pgemm_stage(kfac_pinn_handle* h, cudaStream_t s, F desc) {
    PBatch b;
    memset(&b, 0, sizeof(b));
    int tiles = 0;
    for (int l = 1; l <= h->cfg.L; l++) {
        PGemm g = desc(l);
        g.tiles_q = (g.Q + 63) / 64;
        g.tile0 = tiles;
        tiles += ((g.P + 63) / 64) * g.tiles_q;
        b.g[b.n++] = g;
    }
    KFAC_TRY(KL<k_pgemm_f32>(h, s, tiles, 0, b));
    return KFAC_OK;
}

kfac_status_t precondition_impl(kfac_pinn_handle* h, cudaStream_t s, const double* grad, double* dir) {
    // FP32 products on the tensor-core precisions (whose 16-bit gradients
    // dominate the update's error); FP64 on the SIMT precisions
    if (is_mixed(h)) {
        // the four products of every layer as four batched launches; the
        // layers' scratch matrices X1 and Y are laid out one after another
        auto X1 = [&](int l) { return h->tmp + 2 * (size_t)h->woff[l - 1]; };
        auto Yb = [&](int l) {
            return h->tmp + 2 * (size_t)h->woff[l - 1] + (size_t)h->dims[l] * (h->dims[l - 1] + 1);
        };
        kfac_status_t st;
        // X1 = V_B^T G
        st = pgemm_stage(h, s, [&](int l) {
            const int na = h->dims[l - 1] + 1, nb = h->dims[l];
            PGemm g = {};
            g.A = h->VB[l - 1]; g.a_sp = 1; g.a_sk = nb;
            g.B = grad + h->woff[l - 1]; g.b_sk = 1; g.b_sq = nb;
            g.C = X1(l); g.c_sp = na; g.c_sq = 1;
            g.P = nb; g.Q = na; g.K = nb; g.alpha = 1.0;
            return g;
        });
        if (st) return st;
        // Y = (X1 V_A) / (1 + b a^T)
        st = pgemm_stage(h, s, [&](int l) {
            const int na = h->dims[l - 1] + 1, nb = h->dims[l];
            PGemm g = {};
            g.A = X1(l); g.a_sp = na; g.a_sk = 1;
            g.B = h->VA[l - 1]; g.b_sk = na; g.b_sq = 1;
            g.C = Yb(l); g.c_sp = na; g.c_sq = 1;
            g.dr = h->wb[l - 1]; g.dc = h->wa[l - 1];
            g.P = nb; g.Q = na; g.K = na; g.alpha = 1.0;
            return g;
        });
        if (st) return st;
        // X1 = V_B Y
        st = pgemm_stage(h, s, [&](int l) {
            const int na = h->dims[l - 1] + 1, nb = h->dims[l];
            PGemm g = {};
            g.A = h->VB[l - 1]; g.a_sp = nb; g.a_sk = 1;
            g.B = Yb(l); g.b_sk = na; g.b_sq = 1;
            g.C = X1(l); g.c_sp = na; g.c_sq = 1;
            g.P = nb; g.Q = na; g.K = nb; g.alpha = 1.0;
            return g;
        });
        if (st) return st;
        // Delta = -X1 V_A^T, stored column-stacked like theta
        return pgemm_stage(h, s, [&](int l) {
            const int na = h->dims[l - 1] + 1, nb = h->dims[l];
            PGemm g = {};
            g.A = X1(l); g.a_sp = na; g.a_sk = 1;
            g.B = h->VA[l - 1]; g.b_sk = 1; g.b_sq = na;
            g.C = dir + h->woff[l - 1]; g.c_sp = 1; g.c_sq = nb;
            g.P = nb; g.Q = na; g.K = na; g.alpha = -1.0;
            return g;
        });
    }
    // FP64 handles: FP64 products, one GEMM at a time
    const bool f32 = false;
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
        KFAC_TRY(KL<k_div_kron>(h, s, ceil_div_u((long long)nb * na, 256), 0, Y, nb, na, h->wb[l - 1], h->wa[l - 1]));
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
    if (group_recording()) {      // a grouped batch step solves every member's pairs at once
        group_record_marker();
        return KFAC_OK;
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
    KFAC_TRY(KL<k_update>(h, s, ceil_div_u(h->D, 256), 0, theta, h->dir, h->delta_prev, h->D, h->cfg.lr,
                          h->cfg.momentum, h->coef));
    return KFAC_OK;
}

kfac_status_t linalg_line_search_update(kfac_pinn_handle* h, cudaStream_t s, double* theta, const double* X_int,
                                        int N_int, const double* f, const double* X_bdy, int N_bdy,
                                        const double* g) {
    const unsigned blocks = ceil_div_u(h->D, 256);
    KFAC_TRY(KL<k_dhat>(h, s, blocks, 0, h->dir, h->delta_prev, h->dhat, h->D, h->cfg.momentum));
    const bool mixed = (is_mixed(h));
    for (int k = 0; k < LS_GRID; k++) {
        KFAC_TRY(KL<k_trial>(h, s, blocks, 0, theta, h->dhat, h->trial, h->D, ldexp(1.0, -k)));
        double* dst = h->ls_loss + 3 * k;
        kfac_status_t st = mixed ? tc_eval_loss(h, s, h->trial, X_int, N_int, f, X_bdy, N_bdy, g, dst)
                                 : simt_eval_loss(h, s, h->trial, X_int, N_int, f, X_bdy, N_bdy, g, dst);
        if (st) return st;
    }
    unsigned ab = blocks < (unsigned)(4 * h->sm_count) ? blocks : (unsigned)(4 * h->sm_count);
    KFAC_TRY(KL<k_ls_apply>(h, s, ab, 0, theta, h->dhat, h->delta_prev, h->D, h->ls_loss, h->status, h->cfg.momentum,
                            h->coef));
    return KFAC_OK;
}

size_t linalg_auto_part_elems() { return (size_t)KS_BLOCKS * KS_Q; }

kfac_status_t linalg_auto_update(kfac_pinn_handle* h, cudaStream_t s, double* theta, const double* X_int,
                                 int N_int, const double* X_bdy, int N_bdy) {
    const bool mixed = (is_mixed(h));
    double* jDi = h->ks_jv;
    double* jDb = jDi + h->cfg.max_n_int;
    double* jdi = jDb + h->cfg.max_n_bdy;
    double* jdb = jdi + h->cfg.max_n_int;
    const int have_prev = h->t > 0;
    kfac_status_t st;
    if (mixed) {
        // J v from the step's stored Taylor activations and adjoints, on the tensor cores
        if ((st = tc_residual_jvp(h, s, h->dir, N_int, N_bdy, jDi, jDb))) return st;
        if (have_prev && (st = tc_residual_jvp(h, s, h->delta_prev, N_int, N_bdy, jdi, jdb))) return st;
    } else {
        if ((st = simt_jvp(h, s, theta, h->dir, X_int, N_int, h->in, h->S, true, jDi))) return st;
        if ((st = simt_jvp(h, s, theta, h->dir, X_bdy, N_bdy, h->bd, 1, false, jDb))) return st;
        if (have_prev) {
            if ((st = simt_jvp(h, s, theta, h->delta_prev, X_int, N_int, h->in, h->S, true, jdi))) return st;
            if ((st = simt_jvp(h, s, theta, h->delta_prev, X_bdy, N_bdy, h->bd, 1, false, jdb))) return st;
        }
    }
    KFAC_TRY(KL<k_ks_dots>(h, s, KS_BLOCKS, 0, h->dir, h->delta_prev, h->grad, h->D, jDi, jdi, N_int, jDb, jdb, N_bdy,
                           have_prev, h->ks_part));
    KFAC_TRY(KL<k_ks_solve>(h, s, 1, 0, h->ks_part, KS_BLOCKS, N_int, N_bdy, h->cfg.lambda, have_prev, h->coef,
                            h->status));
    KFAC_TRY(KL<k_ks_apply>(h, s, ceil_div_u(h->D, 256), 0, theta, h->dir, h->delta_prev, h->D, h->coef));
    return KFAC_OK;
}
