// FP64 damped Kronecker-sum inverse, preconditioning and update (Sec. 3.4).
//
// For every layer the two factor pairs (A~_Omega, A~_bdy) and (B~_Omega,
// B~_bdy) are diagonalised simultaneously:
//     V^T P V = I,   V^T Q V = diag(w)        (P = A~_Omega, Q = A~_bdy)
// through P = L L^T (Cholesky), M = L^{-1} Q L^{-T}, M = U diag(w) U^T
// (Householder tridiagonalisation + implicit QL), V = L^{-T} U.  Then
//     (A~_Omega (x) B~_Omega + A~_bdy (x) B~_bdy)^{-1} vec G
//         = vec( V_B [ (V_B^T G V_A) / (1 + w_B w_A^T) ] V_A^T ),
// which is exact because vec(B X A) = (A^T (x) B) vec X (Sec. 2).
//
// One CTA owns one (P, Q) problem; all problems of all layers run in one
// launch.  Errors (a P that is not positive definite, a QL iteration that
// does not converge) are latched in the handle's status word.
#include "kfac_internal.cuh"

namespace {

constexpr int LA_THREADS = 1024;
constexpr int QL_MAXIT = 64;

struct EigProblem {
    const double* P;   // n x n, symmetric (EMA factor, undamped)
    const double* Q;
    double* V;         // out: n x n row-major
    double* w;         // out: n
    double* Lw;        // workspace n x n (Cholesky factor)
    double* Mw;        // workspace n x n
    double* Zw;        // workspace n x n
    double* vec;       // workspace 3n (d, e, tau)
    int n;
};

struct EigBatch {
    EigProblem p[2 * KFAC_MAX_LAYERS];
    int count;
    double eps;        // damping added to every factor
};

__device__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x / 32, l = threadIdx.x % 32;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x / 32); i++) t += sh[i];
        sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

__global__ void __launch_bounds__(LA_THREADS) k_gen_eig(EigBatch batch, int* status) {
    __shared__ double sh[40];
    __shared__ double rc[1024], rs[1024];       // rotations of one QL sweep
    __shared__ int s_lo, s_hi, s_done, s_fail;
    const EigProblem pr = batch.p[blockIdx.x];
    const int n = pr.n;
    const int tid = threadIdx.x, nt = blockDim.x;
    double* Lm = pr.Lw;
    double* M = pr.Mw;
    double* Z = pr.Zw;
    double* dd = pr.vec;
    double* ee = pr.vec + n;
    double* tau = pr.vec + 2 * n;

    // ---- 1. damped copies: L <- P + eps I, M <- Q + eps I ------------------
    for (long long i = tid; i < (long long)n * n; i += nt) {
        int r = (int)(i / n), c = (int)(i % n);
        double e = (r == c) ? batch.eps : 0.0;
        Lm[i] = pr.P[i] + e;
        M[i] = pr.Q[i] + e;
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();

    // ---- 2. Cholesky P = L L^T (right-looking, lower triangle) --------------
    for (int k = 0; k < n; k++) {
        if (tid == 0) {
            double a = Lm[(long long)k * n + k];
            if (!(a > 0.0) || !isfinite(a)) s_fail = 1;
            Lm[(long long)k * n + k] = sqrt(fmax(a, 0.0));
        }
        __syncthreads();
        if (s_fail) break;
        double dk = Lm[(long long)k * n + k];
        for (int i = k + 1 + tid; i < n; i += nt) Lm[(long long)i * n + k] /= dk;
        __syncthreads();
        // trailing update of the lower triangle: L[i][j] -= L[i][k] L[j][k], k < j <= i
        int m = n - k - 1;
        for (long long t = tid; t < (long long)m * m; t += nt) {
            int ii = (int)(t / m), jj = (int)(t % m);
            if (jj > ii) continue;
            int i = k + 1 + ii, j = k + 1 + jj;
            Lm[(long long)i * n + j] -= Lm[(long long)i * n + k] * Lm[(long long)j * n + k];
        }
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) latch_status(status, KFAC_NOT_PD);
        for (long long i = tid; i < (long long)n * n; i += nt) pr.V[i] = 0.0;
        for (int i = tid; i < n; i += nt) pr.w[i] = 0.0;
        return;
    }

    // ---- 3. whitening M <- L^{-1} Q L^{-T} ---------------------------------
    // Z <- L^{-1} Q  (forward substitution, one column per thread)
    for (int c = tid; c < n; c += nt) {
        for (int i = 0; i < n; i++) {
            double v = M[(long long)i * n + c];
            for (int j = 0; j < i; j++) v -= Lm[(long long)i * n + j] * Z[(long long)j * n + c];
            Z[(long long)i * n + c] = v / Lm[(long long)i * n + i];
        }
    }
    __syncthreads();
    // M <- L^{-1} Z^T  (= L^{-1} Q L^{-T} because Q is symmetric)
    for (int c = tid; c < n; c += nt) {
        for (int i = 0; i < n; i++) {
            double v = Z[(long long)c * n + i];
            for (int j = 0; j < i; j++) v -= Lm[(long long)i * n + j] * M[(long long)j * n + c];
            M[(long long)i * n + c] = v / Lm[(long long)i * n + i];
        }
    }
    __syncthreads();
    for (long long t = tid; t < (long long)n * n; t += nt) {
        int r = (int)(t / n), c = (int)(t % n);
        if (r < c) {
            double a = 0.5 * (M[(long long)r * n + c] + M[(long long)c * n + r]);
            M[(long long)r * n + c] = a;
            M[(long long)c * n + r] = a;
        }
    }
    __syncthreads();

    // ---- 4. Householder tridiagonalisation of M (full symmetric storage) -----
    // Step k zeroes M[k+2.., k] with H_k = I - tau_k v v^T acting on rows and
    // columns k+1..n-1, v_0 = 1; v_i (i >= 1) is kept in M[k+1+i][k].
    for (int k = 0; k + 2 < n; k++) {
        const int m = n - k - 1;
        const int b = k + 1;                       // first row/col of the trailing block
        double x0 = M[(long long)b * n + k];
        double part = 0.0;
        for (int i = 1 + tid; i < m; i += nt) {
            double x = M[(long long)(b + i) * n + k];
            part = fma(x, x, part);
        }
        double sigma = block_sum(part, sh);
        double t_k = 0.0, beta = x0, scale = 0.0;
        if (sigma > 0.0) {
            double mu = sqrt(x0 * x0 + sigma);
            beta = (x0 <= 0.0) ? mu : -mu;
            t_k = (beta - x0) / beta;
            scale = 1.0 / (x0 - beta);
        }
        // v_i stored in place (i >= 1)
        for (int i = 1 + tid; i < m; i += nt) M[(long long)(b + i) * n + k] *= scale;
        if (tid == 0) { tau[k] = t_k; ee[k] = beta; }
        __syncthreads();
        if (t_k != 0.0) {
            // p_j = tau sum_i M[b+i][b+j] v_i    (one column j per thread; dd as scratch)
            for (int j = tid; j < m; j += nt) {
                double acc = M[(long long)b * n + (b + j)];       // v_0 = 1
                for (int i = 1; i < m; i++) acc = fma(M[(long long)(b + i) * n + (b + j)], M[(long long)(b + i) * n + k], acc);
                dd[j] = t_k * acc;
            }
            __syncthreads();
            double kp = 0.0;
            for (int j = tid; j < m; j += nt) {
                double vj = (j == 0) ? 1.0 : M[(long long)(b + j) * n + k];
                kp = fma(dd[j], vj, kp);
            }
            double K = 0.5 * t_k * block_sum(kp, sh);
            // w = p - K v   (in dd)
            for (int j = tid; j < m; j += nt) {
                double vj = (j == 0) ? 1.0 : M[(long long)(b + j) * n + k];
                dd[j] = dd[j] - K * vj;
            }
            __syncthreads();
            // trailing block -= v w^T + w v^T
            for (int j = tid; j < m; j += nt) {
                double vj = (j == 0) ? 1.0 : M[(long long)(b + j) * n + k];
                double wj = dd[j];
                for (int i = 0; i < m; i++) {
                    double vi = (i == 0) ? 1.0 : M[(long long)(b + i) * n + k];
                    M[(long long)(b + i) * n + (b + j)] -= vi * wj + dd[i] * vj;
                }
            }
            __syncthreads();
        }
    }
    // diagonal and sub-diagonal of the tridiagonal matrix
    __syncthreads();
    for (int i = tid; i < n; i += nt) dd[i] = M[(long long)i * n + i];
    if (tid == 0 && n >= 2) ee[n - 2] = M[(long long)(n - 1) * n + (n - 2)];
    __syncthreads();
    // shift: ee[k] for k <= n-3 holds beta_k = T[k+1][k]; we want e[i] = T[i+1][i]
    // (already so: beta_k couples rows k and k+1).

    // ---- 5. Z <- H_0 H_1 .. H_{n-3}  (explicit orthogonal factor) -----------
    for (long long t = tid; t < (long long)n * n; t += nt) {
        int r = (int)(t / n), c = (int)(t % n);
        Z[t] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int k = n - 3; k >= 0; k--) {
        double t_k = tau[k];
        if (t_k == 0.0) continue;
        const int b = k + 1, m = n - k - 1;
        for (int c = tid; c < n; c += nt) {
            double dot = Z[(long long)b * n + c];
            for (int i = 1; i < m; i++) dot = fma(M[(long long)(b + i) * n + k], Z[(long long)(b + i) * n + c], dot);
            dot *= t_k;
            Z[(long long)b * n + c] -= dot;
            for (int i = 1; i < m; i++) Z[(long long)(b + i) * n + c] -= dot * M[(long long)(b + i) * n + k];
        }
        __syncthreads();
    }

    // ---- 6. implicit QL with Wilkinson shifts on (dd, ee) -------------------
    // Thread 0 runs the scalar recurrence one sweep at a time and records the
    // plane rotations; all threads then apply the sweep to the rows of Z.
    int l = 0, iter = 0;            // thread-0 state
    if (tid == 0) { if (n >= 1) ee[n - 1] = 0.0; }
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            s_done = 1;
            while (l < n) {
                int m = l;
                for (; m < n - 1; m++) {
                    double sc = fabs(dd[m]) + fabs(dd[m + 1]);
                    if (fabs(ee[m]) <= 2.2204460492503131e-16 * sc) break;
                }
                if (m == l) { l++; iter = 0; continue; }
                if (iter++ >= QL_MAXIT) { latch_status(status, KFAC_NONFINITE); l++; iter = 0; continue; }
                double g = (dd[l + 1] - dd[l]) / (2.0 * ee[l]);
                double r = hypot(g, 1.0);
                g = dd[m] - dd[l] + ee[l] / (g + copysign(r, g));
                double s = 1.0, c = 1.0, p = 0.0;
                int i = m - 1;
                bool early = false;
                for (; i >= l; i--) {
                    double f = s * ee[i], bb = c * ee[i];
                    r = hypot(f, g);
                    ee[i + 1] = r;
                    if (r == 0.0) { dd[i + 1] -= p; ee[m] = 0.0; early = true; break; }
                    s = f / r;
                    c = g / r;
                    g = dd[i + 1] - p;
                    r = (dd[i] - g) * s + 2.0 * c * bb;
                    p = s * r;
                    dd[i + 1] = g + p;
                    g = c * r - bb;
                    rc[i] = c;
                    rs[i] = s;
                }
                if (!early) { dd[l] -= p; ee[l] = g; ee[m] = 0.0; }
                s_lo = early ? i + 1 : l;
                s_hi = m - 1;
                s_done = 0;
                break;
            }
        }
        __syncthreads();
        if (s_done) break;
        const int lo = s_lo, hi = s_hi;
        for (int row = tid; row < n; row += nt) {
            double* zr = Z + (long long)row * n;
            double carry = zr[hi + 1];
            for (int i = hi; i >= lo; i--) {
                double c = rc[i], s = rs[i];
                double zi = zr[i];
                zr[i + 1] = s * zi + c * carry;
                carry = c * zi - s * carry;
            }
            zr[lo] = carry;
        }
        __syncthreads();
    }

    // ---- 7. V = L^{-T} Z  (back substitution, one column per thread) --------
    for (int c = tid; c < n; c += nt) {
        for (int i = n - 1; i >= 0; i--) {
            double v = Z[(long long)i * n + c];
            for (int j = i + 1; j < n; j++) v -= Lm[(long long)j * n + i] * pr.V[(long long)j * n + c];
            pr.V[(long long)i * n + c] = v / Lm[(long long)i * n + i];
        }
    }
    for (int i = tid; i < n; i += nt) {
        pr.w[i] = dd[i];
        if (!isfinite(dd[i])) latch_status(status, KFAC_NONFINITE);
    }
}

__global__ void k_div_kron(double* Y, int nb, int na, const double* wb, const double* wa) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nb * na) return;
    int p = (int)(idx / na), q = (int)(idx % na);
    Y[idx] /= (1.0 + wb[p] * wa[q]);
}

__global__ void k_update(double* theta, const double* dir, double* delta_prev, long long D, double lr,
                         double mom) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    double dlt = lr * (mom * delta_prev[i] + dir[i]);
    delta_prev[i] = dlt;
    theta[i] += dlt;
}

}  // namespace

kfac_status_t linalg_precondition_impl(kfac_pinn_handle* h, cudaStream_t s, const double* grad, double* dir);

size_t linalg_workspace_elems(const kfac_pinn_handle* h) {
    size_t tot = 0;
    for (int l = 1; l <= h->cfg.L; l++) {
        size_t na = h->dims[l - 1] + 1, nb = h->dims[l];
        tot += 3 * na * na + 3 * na + 3 * nb * nb + 3 * nb;
    }
    return tot;
}

kfac_status_t linalg_invert(kfac_pinn_handle* h, cudaStream_t s) {
    EigBatch batch;
    batch.count = 0;
    batch.eps = h->cfg.damping_sqrt ? sqrt(h->cfg.lambda) : h->cfg.lambda;
    double* ws = h->lin;
    for (int l = 1; l <= h->cfg.L; l++) {
        for (int which = 0; which < 2; which++) {
            int n = which == 0 ? h->dims[l - 1] + 1 : h->dims[l];
            EigProblem& p = batch.p[batch.count++];
            p.n = n;
            p.P = h->fac[which == 0 ? KFAC_A_INT : KFAC_B_INT][l - 1];
            p.Q = h->fac[which == 0 ? KFAC_A_BDY : KFAC_B_BDY][l - 1];
            p.V = which == 0 ? h->VA[l - 1] : h->VB[l - 1];
            p.w = which == 0 ? h->wa[l - 1] : h->wb[l - 1];
            p.Lw = ws; ws += (size_t)n * n;
            p.Mw = ws; ws += (size_t)n * n;
            p.Zw = ws; ws += (size_t)n * n;
            p.vec = ws; ws += 3 * (size_t)n;
        }
    }
    double work = 0.0;
    for (int i = 0; i < batch.count; i++) work += 10.0 * (double)batch.p[i].n * batch.p[i].n * batch.p[i].n;
    timer_begin(h, KFAC_KC_EIG, s);
    k_gen_eig<<<batch.count, LA_THREADS, 0, s>>>(batch, h->status);
    timer_end(h, KFAC_KC_EIG, s, work);
    KFAC_LAUNCH_CHECK(h);
    return KFAC_OK;
}

kfac_status_t linalg_precondition(kfac_pinn_handle* h, cudaStream_t s, const double* grad, double* dir) {
    double work = 0.0;
    for (int l = 1; l <= h->cfg.L; l++) {
        double na = h->dims[l - 1] + 1, nb = h->dims[l];
        work += 4.0 * (nb * nb * na + nb * na * na);
    }
    timer_begin(h, KFAC_KC_PRECOND, s);
    kfac_status_t r = linalg_precondition_impl(h, s, grad, dir);
    timer_end(h, KFAC_KC_PRECOND, s, work);
    return r;
}

kfac_status_t linalg_precondition_impl(kfac_pinn_handle* h, cudaStream_t s, const double* grad, double* dir) {
    for (int l = 1; l <= h->cfg.L; l++) {
        const int na = h->dims[l - 1] + 1, nb = h->dims[l];
        const double* G = grad + h->woff[l - 1];
        double* X1 = h->tmp;
        double* Y = h->tmp + (size_t)nb * na;
        const double* VA = h->VA[l - 1];
        const double* VB = h->VB[l - 1];
        kfac_status_t st;
        // X1 = V_B^T G      (nb x na, row-major)
        st = dgemm_strided(h, s, nb, na, nb, VB, 1, nb, G, 1, nb, X1, na, 1, 1.0, 0.0);
        if (st) return st;
        // Y = X1 V_A
        st = dgemm_strided(h, s, nb, na, na, X1, na, 1, VA, na, 1, Y, na, 1, 1.0, 0.0);
        if (st) return st;
        k_div_kron<<<ceil_div_u((long long)nb * na, 256), 256, 0, s>>>(Y, nb, na, h->wb[l - 1], h->wa[l - 1]);
        KFAC_LAUNCH_CHECK(h);
        // X1 = V_B Y
        st = dgemm_strided(h, s, nb, na, nb, VB, nb, 1, Y, na, 1, X1, na, 1, 1.0, 0.0);
        if (st) return st;
        // Delta = -X1 V_A^T, stored column-stacked like theta
        st = dgemm_strided(h, s, nb, na, na, X1, na, 1, VA, 1, na, dir + h->woff[l - 1], 1, nb, -1.0, 0.0);
        if (st) return st;
    }
    return KFAC_OK;
}

kfac_status_t linalg_update(kfac_pinn_handle* h, cudaStream_t s, double* theta) {
    k_update<<<ceil_div_u(h->D, 256), 256, 0, s>>>(theta, h->dir, h->delta_prev, h->D, h->cfg.lr,
                                                   h->cfg.momentum);
    KFAC_LAUNCH_CHECK(h);
    return KFAC_OK;
}
