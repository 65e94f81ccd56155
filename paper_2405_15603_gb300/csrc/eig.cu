// Batched FP64 simultaneous diagonalisation of the damped factor pairs
// (Sec. 3.4, "eigen-decomposing all Kronecker factors"):
//     V^T P V = I,  V^T Q V = diag(w),   P = A~_Omega, Q = A~_bdy   (and B)
// for every layer at once, each stage spread over the whole GPU:
//   1. Cholesky P = L L^T                       (one cluster per problem, as in 3;
//                                                 blocked diag / panel / trailing
//                                                 kernels for the largest factors)
//   2. M = L^{-1} Q L^{-T}                      (L^{-1} by column-parallel FP64
//                                                 solves, the two products on the
//                                                 tensor cores by error-free FP64
//                                                 emulation, ozaki.cu)
//   3. Householder tridiagonalisation of M      (one thread-block cluster per
//      problem with the triangle in distributed shared memory; for factors
//      too large for it, one cooperative kernel where each problem owns a
//      group of CTAs that sync through bounded global barriers)
//   4. divide and conquer on the tridiagonal T  (Cuppen's rank-one tearing,
//      deflation, secular equation by a safeguarded rational iteration, eigenvectors via the
//      Gu-Eisenstat recomputed z, block GEMMs per merge level, the large ones
//      on the tensor cores, ozaki.cu)
//   5. the reflectors' product Q_H = H_0 H_1 ... (column-parallel, applied to
//      I) and W = L^{-T} Q_H, beside step 4 on a stream of the group's own
//   6. V = W U = L^{-T} Q_H U                    (tensor cores, ozaki.cu)
// The factor pairs form one group per cluster size of steps 1 and 3, whose
// kernel sequences run on streams of their own at once.
// Errors (a P that is not positive definite, a barrier that gave up) are
// latched in the handle's status word; the problem's V and w are then zero.
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <vector>
#include <algorithm>
#include <map>
#include <cooperative_groups.h>

#include "kfac_internal.cuh"
#include "ozaki.cuh"

namespace {

constexpr int NB = 64;        // Cholesky / TRSM block
constexpr int CB_MAX = 32;    // widest TRSM column strip
// Column-strip widths of the triangular solves and the back-transformation:
// one CTA per strip, sequential down the strip, so the strips are the
// parallelism.  Narrower strips for larger factors keep the jobs' FP64 work
// about equal (n^2 x width) and make the largest factors' strips outnumber the
// SMs several times over (a 769 factor: 97 strips of 8 columns), so that the
// last wave of equal jobs leaves few SMs idle.
constexpr int STRIP_NARROW_FROM = 640;   // factors this large get 8-column strips
constexpr int STRIP_MEDIUM_FROM = 320;   // these 16, the smaller ones 32
inline int strip_width(int n) { return n >= STRIP_NARROW_FROM ? 8 : (n >= STRIP_MEDIUM_FROM ? 16 : 32); }
constexpr int KFAC_MAX_WIDTH_PLUS_ONE = 1024;   // widths <= 1023 and d + 1 <= 1024 (create checks)
constexpr double DEPS = 2.220446049250313e-16;
// Block GEMMs of the divide and conquer with a contraction this long or longer
// run on the tensor cores (ozaki.cu); shorter ones stay on the FP64 cores.
constexpr int OZ_MIN_K = 128;

struct Prob {
    int n;
    const double* P;
    const double* Q;
    double* V;
    double* w;
    double *L, *M, *Qa, *Qb, *R, *R2, *H;  // n x n row-major (H: Householder vectors, one per row)
    double* Ld;                            // inverses of the 64 x 64 diagonal blocks of L (n x 64)
    double* Li;                            // L^{-1}, n x n row-major (zero above the diagonal)
    double *d, *e, *tau, *D, *pbuf, *pbuf2;  // n
    double *Ds, *zs, *dK, *zK, *tauR, *zh, *rc, *rs, *val; // n (per-merge scratch at offset a)
    int *perm, *defl, *Kidx, *org, *rj, *ri, *col;          // n
    int *mk, *mnrot, *mflip;               // per merge (indexed by block start a)
    double* mrh;
    int final_buf;                         // 0: Qa, 1: Qb holds the D&C result
    double eps;                            // damping added to both factors' diagonals
    int* status;                           // status word of the problem's handle
};

struct Merge {
    int prob, a, s1, s2;
    int r0;      // prefix sum of the merge sizes within the level
};

// merge owning global row index t of a level (binary search on r0)
__device__ int find_merge(const Merge* mg, int n_merges, int t) {
    int lo = 0, hi = n_merges - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (mg[mid].r0 <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct Gd {   // one block GEMM of a merge: C = A B, A (M x K), B (K x N), all row stride ld
    const double* A;
    const double* B;
    double* C;
    int ld, M, N, K, tile0;
};

struct Copy {
    const double* src;
    double* dst;
    int ld, m;
};

struct Level {
    Merge* merges;     // device
    int n_merges;
    int max_m;
    Gd* gemms;         // device: the block GEMMs below OZ_MIN_K (FP64 CUDA cores)
    int n_gemms, n_tiles;
    OzPlan* oz;        // the others, on the tensor cores by error-free splitting (ozaki.cu)
    Copy* copies;      // device
    int n_copies, max_copy;
    int roots;         // sum of m over merges
};

struct EigState {
    int np;
    std::vector<Prob> host;
    Prob* dev;                  // device copy of host[]
    double* ws;                 // all double workspaces
    int* iws;                   // all int workspaces
    int* fail;                  // per problem
    unsigned* bar;              // per problem: count, generation
    int* abort_flag;
    int* cta_prob;              // cooperative tridiagonalisation: problem of each CTA
    int* cta_rank;
    int* group;                 // group size per problem
    int n_cta;
    void* trsm_jobs;            // TrsmJob list, largest work first (also the back-transform's)
    void* trsm_jobs_upper;      // the same jobs ordered by their work in the upper-triangle solve (mode 1)
    void* trsm_jobs_inv;        // ... and in the inverse (mode 3)
    OzPlan* oz_inv1;            // T = L21 X11 of the split inverses (tensor cores, ozaki.cu)
    OzPlan* oz_inv2;            // X21 = -X22 T
    OzPlan* oz_red1;            // Qa = L^{-1} M
    OzPlan* oz_red2;            // M = Qa L^{-T}
    OzPlan* oz_w;               // W = L^{-T} Q_H (Q_H = the reflectors' product, formed in L; W into H)
    OzPlan* oz_v;               // V = W U
    cudaStream_t aux;           // Q_H and W beside the divide and conquer
    cudaEvent_t ev_fork, ev_join;
    int n_trsm_jobs;
    size_t bt_smem;             // back-transform shared memory for the widest job
    std::vector<Level> levels;
    int nmax;
    // cluster tridiagonalisation (used when every problem's triangle fits)
    int trc_cl;                 // CTAs per cluster; 0: the cooperative kernel instead
    int trc_lds, trc_rmax;
    size_t trc_smem;
    int* clu_prob;              // problem of each cluster, largest first
};

// The factor pairs form one group per cluster size of the tridiagonalisation
// (the size follows from n alone: trc_cluster_size), each group one sequence
// of batched kernels, the groups on streams of their own: the largest
// problems' latency-bound stages hold only part of the GPU, and the smaller
// problems fill the idle SMs meanwhile.
constexpr int MAX_GROUPS = 6;    // cluster sizes 16, 8, 4, 2, 1 and the cooperative kernel

struct EigAll {
    EigState* g[MAX_GROUPS];
    int ng;
    cudaStream_t side[MAX_GROUPS - 1];   // groups 1.. run on these, forked from the caller's stream
    cudaEvent_t fork, join[MAX_GROUPS - 1];
};

EigAll* EA(kfac_pinn_handle* h) { return (EigAll*)h->eig; }

// --------------------------------------------------------------------------
// Small helpers
// --------------------------------------------------------------------------
__device__ double block_reduce_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x / 32); i++) t += sh[i];
        sh[32] = t;
    }
    __syncthreads();
    double r = sh[32];
    __syncthreads();
    return r;
}

__device__ double block_reduce_max(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x / 32); i++) t = fmax(t, sh[i]);
        sh[32] = t;
    }
    __syncthreads();
    double r = sh[32];
    __syncthreads();
    return r;
}

// --------------------------------------------------------------------------
// 0. damped copies
// --------------------------------------------------------------------------
__global__ void k_damp(Prob* pr, int* fail) {
    const Prob p = pr[blockIdx.y];
    const int n = p.n;
    if (threadIdx.x == 0 && blockIdx.x == 0) fail[blockIdx.y] = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)n * n;
         i += (long long)gridDim.x * blockDim.x) {
        int r = (int)(i / n), c = (int)(i % n);
        double e = (r == c) ? p.eps : 0.0;
        p.L[i] = p.P[i] + e;
        p.M[i] = p.Q[i] + e;
    }
}

// --------------------------------------------------------------------------
// 1. blocked Cholesky (lower), block k0
// --------------------------------------------------------------------------
__global__ void k_chol_diag(Prob* pr, int k0, int* fail) {
    __shared__ double A[NB][NB + 1];
    __shared__ int bad;
    const Prob p = pr[blockIdx.x];
    const int n = p.n;
    if (k0 >= n || fail[blockIdx.x]) return;
    const int nb = min(NB, n - k0);
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        int r = t / nb, c = t % nb;
        A[r][c] = p.L[(long long)(k0 + r) * n + k0 + c];
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < nb; j++) {
        if (threadIdx.x == 0) {
            double a = A[j][j];
            if (!(a > 0.0) || !isfinite(a)) bad = 1;
            A[j][j] = sqrt(fmax(a, 0.0));
        }
        __syncthreads();
        if (bad) break;
        const double djj = A[j][j];
        for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) A[i][j] /= djj;
        __syncthreads();
        const int m = nb - j - 1;
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            int i = j + 1 + t / m, c = j + 1 + t % m;
            if (c <= i) A[i][c] -= A[i][j] * A[c][j];
        }
        __syncthreads();
    }
    if (bad) {
        if (threadIdx.x == 0) {
            fail[blockIdx.x] = 1;
            latch_status(p.status, KFAC_NOT_PD);
        }
        return;
    }
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        int r = t / nb, c = t % nb;
        if (c <= r) p.L[(long long)(k0 + r) * n + k0 + c] = A[r][c];
    }
}

// rows below the diagonal block: X = A L_kk^{-T}.  The 64 x 64 row block is
// solved column by column in shared memory (right-looking): after column j
// is final, its contribution is removed from the later columns.
__global__ void __launch_bounds__(256) k_chol_panel(Prob* pr, int k0, int* fail) {
    __shared__ double Lk[NB][NB + 1];
    __shared__ double Xs[NB][NB + 1];
    const Prob p = pr[blockIdx.y];
    const int n = p.n;
    if (k0 >= n || fail[blockIdx.y]) return;
    const int nb = min(NB, n - k0);
    const int r0 = k0 + nb + blockIdx.x * NB;
    if (r0 >= n) return;
    const int rows = min(NB, n - r0);
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        int r = t / NB, c = t % NB;
        Lk[r][c] = (r < nb && c <= r) ? p.L[(long long)(k0 + r) * n + k0 + c] : 0.0;
        Xs[r][c] = (r < rows && c < nb) ? p.L[(long long)(r0 + r) * n + k0 + c] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < nb; j++) {
        const double ljj = Lk[j][j];
        for (int r = threadIdx.x; r < rows; r += blockDim.x) Xs[r][j] /= ljj;
        __syncthreads();
        for (int t = threadIdx.x; t < rows * NB; t += blockDim.x) {
            int r = t / NB, c = t % NB;
            if (c > j && c < nb) Xs[r][c] -= Xs[r][j] * Lk[c][j];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < rows * nb; t += blockDim.x) {
        int r = t / nb, c = t % nb;
        p.L[(long long)(r0 + r) * n + k0 + c] = Xs[r][c];
    }
}

// trailing update of the lower triangle: A_ij -= L_i L_j^T over the panel
__global__ void __launch_bounds__(256) k_chol_update(Prob* pr, int k0, int* fail) {
    __shared__ double As[16][NB + 1];
    __shared__ double Bs[16][NB + 1];
    const Prob p = pr[blockIdx.y];
    const int n = p.n;
    if (k0 >= n || fail[blockIdx.y]) return;
    const int nb = min(NB, n - k0);
    const int t0 = k0 + nb;
    if (t0 >= n) return;
    const int nt = (n - t0 + NB - 1) / NB;
    int t = blockIdx.x;
    if (t >= nt * (nt + 1) / 2) return;
    int bi = 0;
    while ((bi + 1) * (bi + 2) / 2 <= t) bi++;
    int bj = t - bi * (bi + 1) / 2;
    const int i0 = t0 + bi * NB, j0 = t0 + bj * NB;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int kc = 0; kc < nb; kc += 16) {
        __syncthreads();
        for (int q = threadIdx.x; q < NB * 16; q += blockDim.x) {
            int r = q / 16, c = q % 16;
            As[c][r] = (i0 + r < n && kc + c < nb) ? p.L[(long long)(i0 + r) * n + k0 + kc + c] : 0.0;
            Bs[c][r] = (j0 + r < n && kc + c < nb) ? p.L[(long long)(j0 + r) * n + k0 + kc + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int r = i0 + ty + 16 * i, c = j0 + tx + 16 * j;
            if (r < n && c < n && c <= r) p.L[(long long)r * n + c] -= acc[i][j];
        }
}

// --------------------------------------------------------------------------
// 2/6. column-parallel triangular solves with L
//   mode 0: X = L^{-1} B,   B = M (row-major),   X -> Qa
//   mode 1: X = L^{-1} B^T, B = Qa,              X -> M   (X is symmetric: only
//           rows 0..c of column c, the upper triangle, which k_symmetrize
//           copies to the lower one; a third of the solve's work)
//   mode 2: X = L^{-T} B,   B = final D&C buffer, X -> V
//   mode 3: X = L^{-1},     B = I,               X -> Li  (each column from the
//           block of its diagonal down: a third of a full solve's work)
// The eigensolver uses mode 3 and forms the products with L^{-1} on the
// tensor cores (ozaki.cu); modes 0-2 solve with L on the FP64 cores.
// --------------------------------------------------------------------------
// One column strip [c0, c0 + CB) of a triangular solve with NB x NB blocks.
template <int CB>
__device__ void trsm_strip(const Prob& p, int c0, int mode, bool failed, double* sm, int r_end) {
    constexpr int TRSM_RG = 256 / CB;      // row groups of the 256 threads
    double* Lb = sm;                       // NB x (NB+1)
    double* Xk = Lb + NB * (NB + 1);       // NB x (CB+1)
    double* acc = Xk + NB * (CB + 1);      // NB x (CB+1)
    const int n = p.n;
    const double* B;
    double* X;
    if (mode == 0) { B = p.M; X = p.Qa; }
    else if (mode == 1) { B = p.Qa; X = p.M; }
    else if (mode == 2) { B = p.final_buf ? p.Qb : p.Qa; X = p.V; }
    else { B = nullptr; X = p.Li; }
    const int ncb = min(CB, n - c0);
    const int nblk = (n + NB - 1) / NB;
    if (failed) {
        if (mode >= 2)
            for (int t = threadIdx.x; t < n * ncb; t += blockDim.x) X[(long long)(t / ncb) * n + c0 + t % ncb] = 0.0;
        return;
    }
    const bool upper = (mode == 2);
    // mode 1: the row blocks down to the strip's last column; mode 3 (the
    // inverse, right-hand side I): from the block of the strip's first column,
    // the rows above it being zero
    const int nrun = (mode == 1) ? min(nblk, (c0 + ncb - 1) / NB + 1)
                                 : (mode == 3 ? min(nblk, (r_end + NB - 1) / NB) : nblk);
    const int s0 = (mode == 3) ? c0 / NB : 0;
    for (int s = s0; s < nrun; s++) {
        const int ib = upper ? nblk - 1 - s : s;
        const int r0 = ib * NB, rows = min(NB, n - r0);
        for (int t = threadIdx.x; t < NB * CB; t += blockDim.x) {
            int r = t / CB, c = t % CB;
            double v = 0.0;
            if (r < rows && c < ncb) {
                if (mode == 3) v = (r0 + r == c0 + c) ? 1.0 : 0.0;
                else v = (mode == 1) ? B[(long long)(c0 + c) * n + r0 + r] : B[(long long)(r0 + r) * n + c0 + c];
            }
            acc[r * (CB + 1) + c] = v;
        }
        // subtract the solved blocks
        for (int kk = s0; kk < s; kk++) {
            const int kb = upper ? nblk - 1 - kk : kk;
            const int k0 = kb * NB, kr = min(NB, n - k0);
            __syncthreads();
            for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
                int r = t / NB, m = t % NB;
                double v = 0.0;
                if (r < rows && m < kr)
                    v = upper ? p.L[(long long)(k0 + m) * n + r0 + r] : p.L[(long long)(r0 + r) * n + k0 + m];
                Lb[r * (NB + 1) + m] = v;
            }
            for (int t = threadIdx.x; t < NB * CB; t += blockDim.x) {
                int m = t / CB, c = t % CB;
                Xk[m * (CB + 1) + c] = (m < kr && c < ncb) ? X[(long long)(k0 + m) * n + c0 + c] : 0.0;
            }
            __syncthreads();
            // acc[r][c] -= sum_m Lb[r][m] Xk[m][c]; NB / TRSM_RG outputs per thread
            const int c = threadIdx.x % CB, rg = threadIdx.x / CB;
            double v[NB / TRSM_RG];
#pragma unroll
            for (int i = 0; i < NB / TRSM_RG; i++) v[i] = 0.0;
#pragma unroll 4
            for (int m = 0; m < NB; m++) {
                const double x = Xk[m * (CB + 1) + c];
#pragma unroll
                for (int i = 0; i < NB / TRSM_RG; i++) v[i] = fma(Lb[(rg + TRSM_RG * i) * (NB + 1) + m], x, v[i]);
            }
#pragma unroll
            for (int i = 0; i < NB / TRSM_RG; i++) acc[(rg + TRSM_RG * i) * (CB + 1) + c] -= v[i];
        }
        // diagonal block: X_i = L_ii^{-1} acc (lower) or L_ii^{-T} acc (upper),
        // with the block inverse precomputed by k_diag_inv
        __syncthreads();
        for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
            int r = t / NB, m = t % NB;
            Lb[r * (NB + 1) + m] = (r < rows && m < rows) ? p.Ld[(long long)(r0 + r) * NB + m] : 0.0;
        }
        __syncthreads();
        {
            const int c = threadIdx.x % CB, rg = threadIdx.x / CB;
            double v[NB / TRSM_RG];
#pragma unroll
            for (int i = 0; i < NB / TRSM_RG; i++) v[i] = 0.0;
#pragma unroll 4
            for (int m = 0; m < NB; m++) {
                const double x = acc[m * (CB + 1) + c];
#pragma unroll
                for (int i = 0; i < NB / TRSM_RG; i++) {
                    const int r = rg + TRSM_RG * i;
                    v[i] = fma(upper ? Lb[m * (NB + 1) + r] : Lb[r * (NB + 1) + m], x, v[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < NB / TRSM_RG; i++) Xk[(rg + TRSM_RG * i) * (CB + 1) + c] = v[i];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < NB * CB; t += blockDim.x) {
            int r = t / CB, c = t % CB;
            if (r < rows && c < ncb) X[(long long)(r0 + r) * n + c0 + c] = Xk[r * (CB + 1) + c];
        }
        __syncthreads();
    }
}

// One CTA per job (problem, first column, strip width); the widths make the
// jobs' FP64 work about equal (16 columns of the largest factors, 32 of the
// others) and the list is sorted by work, largest first.
struct TrsmJob {
    int prob, c0, cb;
    int r_end;       // mode 3: rows solved end here (the first diagonal block of a split inverse)
};

// Factors from this size get L^{-1} as [X11 0; X21 X22]: the diagonal blocks
// by strip solves, X21 = -X22 (L21 X11) by two emulated products.
constexpr int INV_SPLIT_FROM = 256;
inline int inv_split(int n) { return n >= INV_SPLIT_FROM ? (n / 2 + NB - 1) / NB * NB : 0; }

__global__ void __launch_bounds__(256, 2) k_trsm(Prob* pr, const TrsmJob* jobs, int mode, int* fail) {
    extern __shared__ double sm[];
    const TrsmJob jb = jobs[blockIdx.x];
    const Prob p = pr[jb.prob];
    if (jb.c0 >= p.n) return;
    const bool failed = fail[jb.prob] != 0;
    if (jb.cb == 8) trsm_strip<8>(p, jb.c0, mode, failed, sm, jb.r_end);
    else if (jb.cb == 16) trsm_strip<16>(p, jb.c0, mode, failed, sm, jb.r_end);
    else trsm_strip<32>(p, jb.c0, mode, failed, sm, jb.r_end);
}

// Inverse of every 64 x 64 diagonal block of L (lower triangular), one CTA
// per block: column c of the inverse by forward substitution on e_c.
__global__ void __launch_bounds__(256) k_diag_inv(Prob* pr, int* fail) {
    extern __shared__ double dsm[];                       // 2 x NB x (NB+1), dynamic
    double (*Ls)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(dsm);
    double (*Xs)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(dsm + NB * (NB + 1));
    const Prob p = pr[blockIdx.y];
    const int n = p.n;
    const int r0 = blockIdx.x * NB;
    if (r0 >= n || fail[blockIdx.y]) return;
    const int rows = min(NB, n - r0);
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        int r = t / NB, c = t % NB;
        Ls[r][c] = (r < rows && c <= r) ? p.L[(long long)(r0 + r) * n + r0 + c] : 0.0;
        Xs[r][c] = (r == c && r < rows) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < rows; j++) {          // right-looking on all 64 columns at once
        const double ljj = Ls[j][j];
        for (int c = threadIdx.x; c < NB; c += blockDim.x) Xs[j][c] /= ljj;
        __syncthreads();
        for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
            int r = t / NB, c = t % NB;
            if (r > j && r < rows) Xs[r][c] -= Ls[r][j] * Xs[j][c];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        int r = t / NB, c = t % NB;
        if (r < rows) p.Ld[(long long)(r0 + r) * NB + c] = (c < rows) ? Xs[r][c] : 0.0;
    }
}

// The lower triangle of M = L^{-1} Q L^{-T} from its upper one (the only one
// the second solve computes).
__global__ void k_symmetrize(Prob* pr, int* fail) {
    const Prob p = pr[blockIdx.y];
    const int n = p.n;
    if (fail[blockIdx.y]) return;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)n * n;
         t += (long long)gridDim.x * blockDim.x) {
        int r = (int)(t / n), c = (int)(t % n);
        if (r > c) p.M[(long long)r * n + c] = p.M[(long long)c * n + r];
    }
}

// --------------------------------------------------------------------------
// 3. Householder tridiagonalisation, cooperative
// --------------------------------------------------------------------------
// Bounded wait of the g CTAs of a group: false (and the abort flag set) when
// the others have not all arrived within limit_ns of globaltimer, or when
// another CTA has aborted.
constexpr uint64_t GROUP_WAIT_LIMIT_NS = 2000000000ull;   // 2 s
__device__ bool group_barrier(unsigned* bar, int g, int* abort_flag, uint64_t limit_ns = GROUP_WAIT_LIMIT_NS) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned* vgen = bar + 1;
        unsigned gen = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == (unsigned)(g - 1)) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            uint64_t t0;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            for (unsigned it = 0;; it++) {
                if (*vgen != gen) break;
                if (*(volatile int*)abort_flag) { ok = 0; break; }
                if ((it & 63u) == 0) {
                    uint64_t t1;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
                    if (t1 - t0 > limit_ns) { ok = 0; atomicExch(abort_flag, 1); break; }
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Waits (bounded, thread 0) until the pivot row `k` has been published.
__device__ bool wait_row(const unsigned* ready, unsigned k, int* abort_flag) {
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        const volatile unsigned* vr = ready;
        uint64_t t0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        for (unsigned it = 0; *vr < k; it++) {
            if (*(volatile int*)abort_flag) { ok = 0; break; }
            if ((it & 63u) == 0) {
                uint64_t t1;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
                if (t1 - t0 > 2000000000ull) { ok = 0; atomicExch(abort_flag, 1); break; }
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Householder tridiagonalisation of M (full symmetric storage), one problem
// per CTA group.  Row r belongs to CTA (r mod g) for the whole reduction, and
// within it to warp ((r div g) mod nwarps), so the matrix-vector product and
// the rank-2 update of a row are done by the same threads.  Per column k:
// read the published pivot row k, form the reflector (redundantly in every
// CTA), p = tau M v on owned rows, one group barrier to exchange p, then the
// rank-2 update of owned rows; the owner of row k+1 updates it first and
// publishes it through a counter, which replaces a second barrier.
__global__ void __launch_bounds__(512) k_tridiag(Prob* pr, const int* cta_prob, const int* cta_rank,
                                                 const int* group, unsigned* bars, int* abort_flag, int* fail) {
    __shared__ double v[1024];
    __shared__ double w[1024];
    __shared__ double sh[40];
    const int pi = cta_prob[blockIdx.x];
    const int rank = cta_rank[blockIdx.x];
    const int g = group[pi];
    const Prob p = pr[pi];
    const int n = p.n;
    unsigned* bar = bars + 3 * pi;
    unsigned* ready = bar + 2;
    double* M = p.M;
    if (fail[pi]) return;   // uniform over the group
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nwarps = blockDim.x / 32;
    bool alive = true;
    for (int k = 0; k + 2 < n && alive; k++) {
        const int b = k + 1, m = n - b;
        double* pb = (k & 1) ? p.pbuf2 : p.pbuf;
        if (k > 0 && !wait_row(ready, (unsigned)k, abort_flag)) { alive = false; break; }
        // reflector from the published row k (= column k)
        const double* rowk = M + (long long)k * n + b;
        double part = 0.0;
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            double x = __ldcg(rowk + i);
            w[i] = x;
            if (i >= 1) part = fma(x, x, part);
        }
        const double sigma = block_reduce_sum(part, sh);
        const double x0 = w[0];
        double tk = 0.0, beta = x0, scale = 0.0;
        if (sigma > 0.0) {
            double mu = sqrt(x0 * x0 + sigma);
            beta = (x0 <= 0.0) ? mu : -mu;
            tk = (beta - x0) / beta;
            scale = 1.0 / (x0 - beta);
        }
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            const double vi = (i == 0) ? 1.0 : w[i] * scale;
            v[i] = vi;
            if (rank == 0) p.H[(long long)k * n + b + i] = vi;   // reflector k for the back-transformation
        }
        __syncthreads();
        if (tk == 0.0) {
            if (rank == 0 && threadIdx.x == 0) { p.tau[k] = 0.0; p.e[k] = beta; }
            if (rank == b % g && threadIdx.x == 0) {    // row b is unchanged: publish it as is
                __threadfence();
                atomicExch(ready, (unsigned)b);
            }
            continue;     // every CTA of the group skips the same step
        }
        // p_r = tau sum_j M[r][b+j] v_j for owned rows r >= b
        for (int t = warp;; t += nwarps) {
            const int r = rank + g * t;
            if (r >= n) break;
            if (r < b) continue;
            const double* row = M + (long long)r * n + b;
            double acc = 0.0;
            for (int j = lane; j < m; j += 32) acc = fma(row[j], v[j], acc);
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) pb[r - b] = tk * acc;
        }
        if (!group_barrier(bar, g, abort_flag)) { alive = false; break; }
        double kp = 0.0;
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            double pj = __ldcg(pb + j);
            w[j] = pj;
            kp = fma(pj, v[j], kp);
        }
        const double K = 0.5 * tk * block_reduce_sum(kp, sh);
        for (int j = threadIdx.x; j < m; j += blockDim.x) w[j] -= K * v[j];
        __syncthreads();
        // the next pivot row first (all threads of its owner), then publish it
        if (rank == b % g) {
            double* row = M + (long long)b * n + b;
            const double v0 = v[0], w0 = w[0];
            for (int j = threadIdx.x; j < m; j += blockDim.x) row[j] = fma(-v0, w[j], fma(-w0, v[j], row[j]));
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicExch(ready, (unsigned)b);
        }
        // rank-2 update of the other owned rows
        for (int t = warp;; t += nwarps) {
            const int r = rank + g * t;
            if (r >= n) break;
            if (r <= b) continue;
            double* row = M + (long long)r * n + b;
            const double vi = v[r - b], wi = w[r - b];
            for (int j = lane; j < m; j += 32) row[j] = fma(-vi, w[j], fma(-wi, v[j], row[j]));
        }
        if (rank == 0 && threadIdx.x == 0) { p.tau[k] = tk; p.e[k] = beta; }
        __syncthreads();
    }
    // every update must be in place before the diagonal is read
    if (alive && !group_barrier(bar, g, abort_flag)) alive = false;
    if (!alive) {
        if (threadIdx.x == 0) latch_status(p.status, KFAC_TIMEOUT);
        return;
    }
    if (rank == 0) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) p.d[i] = __ldcg(M + (long long)i * n + i);
        if (threadIdx.x == 0 && n >= 2) p.e[n - 2] = __ldcg(M + (long long)(n - 1) * n + (n - 2));
    }
}

// The same reduction with the lower triangle of M held in the distributed
// shared memory of one thread-block cluster per problem (CL = 1..16 CTAs).  CTA
// c of the cluster owns rows r = c + CL*t, t = 0, 1, ..., each stored as its
// columns 0..r, packed one row after another.  Per column k (b = k + 1):
//   - gather the pivot column x = M[b.., k] from its owners and form the
//     reflector (the same arithmetic in every CTA, so every CTA takes the
//     same decisions);
//   - M v over the owned rows, from M x and the column M e_0: column sums for
//     the transposed part and the diagonal, warp dots for the strictly lower
//     part (every stored element is used twice, so the symmetric matrix costs
//     half the FP64 operations of a full one);
//   - each CTA sums its slice of M v over the cluster's partials (fixed
//     order), and every CTA assembles w = tau M v - K v from the slices;
//   - rank-2 update of the owned rows, column b first: the next pivot column
//     is sent, the cluster barrier arrived at, and the rest of the update runs
//     while the barrier completes.
// Every exchange is a store into the consumer's shared memory before a
// barrier (no remote loads wait on the critical path).
// Three cluster barriers per column and no global-memory synchronisation;
// the cluster's barriers are hardware barriers that every CTA reaches in the
// same order (all control flow is uniform over the cluster).
constexpr int TRC_THREADS = 512;
constexpr int TRC_CL = 16;    // most CTAs per cluster (a non-portable cluster size)
constexpr int TRC_RED = TRC_THREADS + 8;   // reduction scratch: one slot per thread + scalars
constexpr int TRC_TK = TRC_THREADS, TRC_SCALE = TRC_THREADS + 1, TRC_K = TRC_THREADS + 3;

// Warp 0's sum of the per-thread partials sh[0..TRC_THREADS) (written and
// synchronised by the caller); every lane of warp 0 gets the same total.  The
// FP64 pipe is the scarce unit on this part, so the other warps issue no FP64
// adds for a reduction, and the dependency chain is kept short (four
// independent chains, then a butterfly).
__device__ __forceinline__ double trc_warp0_sum(const double* sh) {
    const int l = threadIdx.x % 32;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
    for (int u = 0; u < TRC_THREADS / 32; u += 4) {
        a0 += sh[l + 32 * u];
        a1 += sh[l + 32 * (u + 1)];
        a2 += sh[l + 32 * (u + 2)];
        a3 += sh[l + 32 * (u + 3)];
    }
    double t = (a0 + a1) + (a2 + a3);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

__host__ __device__ inline long long trc_off(int t, int c, int cl) {
    return (long long)t * (c + 1) + (long long)cl * t * (t - 1) / 2;
}

// Cholesky P = L L^T of the damped factor (in place in p.L, lower triangle)
// in one thread-block cluster per problem, with the same row ownership and
// packed storage as the tridiagonalisation.  Right-looking, one column per
// step: every CTA holds the pivot column (sent by its owners before the
// barrier), forms L_kk and the scaled column, updates column k+1 of its rows
// first and sends it, arrives at the cluster barrier, then runs the rest of
// the rank-1 update while the barrier completes.  One cluster barrier per
// column.  A pivot that is not positive and finite stops every CTA of the
// cluster at the same column (they all see the same pushed value) and marks
// the problem failed.
template <int CL>
__global__ void __launch_bounds__(TRC_THREADS, 1) k_chol_cluster(Prob* pr, const int* clu_prob, int lds, int nmax,
                                                                 int* fail) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double trc_sm[];
    const int c = (int)cl.block_rank();
    const int pi = clu_prob[blockIdx.x / CL];
    const Prob p = pr[pi];
    const int n = p.n;
    const int tid = threadIdx.x, T = blockDim.x;
    const int warp = tid / 32, lane = tid % 32, nwarps = T / 32;
    const int sp = warp & 3, slot = warp >> 2;
    const int snake = (slot & 1) ? 3 - sp : sp;   // rows to warps evenly over the SM sub-partitions
    double* As = trc_sm;              // owned rows, packed
    double* colb = As + lds;          // pivot columns by global row, two buffers (pushed by the owners)
    double* lb = colb + 2 * nmax;     // scaled column L[k+1.., k], by i = r - k - 1
    double* red = lb + nmax;          // per-column scalars
    const int R = c < n ? (n - c + CL - 1) / CL : 0;

    for (int t = warp; t < R; t += nwarps) {
        const int r = c + CL * t;
        const long long o = trc_off(t, c, CL);
        for (int j = lane; j <= r; j += 32) As[o + j] = p.L[(long long)r * n + j];
    }
    __syncthreads();
    for (int t = tid; t < R; t += T) {     // column 0, to every CTA
        const int r = c + CL * t;
        const double val = As[trc_off(t, c, CL)];
#pragma unroll
        for (int d = 0; d < CL; d++) cl.map_shared_rank(colb, d)[r] = val;
    }
    cl.sync();

    bool ok = true;
    for (int k = 0; k < n; k++) {
        const double* col = colb + (k & 1) * nmax;
        double* nxt = colb + ((k + 1) & 1) * nmax;
        const int m = n - k - 1;
        if (tid == 0) {
            const double a = col[k];
            const bool good = a > 0.0 && isfinite(a);
            const double lkk = sqrt(good ? a : 1.0);
            red[0] = lkk;
            red[1] = 1.0 / lkk;
            red[2] = good ? 1.0 : 0.0;
        }
        __syncthreads();
        if (red[2] == 0.0) { ok = false; break; }      // uniform over the cluster
        const double lkk = red[0], rinv = red[1];
        for (int i = tid; i < m; i += T) lb[i] = col[k + 1 + i] * rinv;
        __syncthreads();
        // column k of the owned rows, then column k + 1 updated and sent
        for (int t = tid; t < R; t += T) {
            const int r = c + CL * t;
            if (r < k) continue;
            double* row = As + trc_off(t, c, CL);
            if (r == k) { row[k] = lkk; continue; }
            const double lr = lb[r - k - 1];
            row[k] = lr;
            const double a = fma(-lr, lb[0], row[k + 1]);
            row[k + 1] = a;
#pragma unroll
            for (int d = 0; d < CL; d++) cl.map_shared_rank(nxt, d)[r] = a;
        }
        __cluster_barrier_arrive();
        for (int t = 4 * slot + snake; t < R; t += nwarps) {
            const int r = c + CL * t;
            if (r <= k + 1) continue;
            double* row = As + trc_off(t, c, CL);
            const double lr = lb[r - k - 1];
            for (int j = k + 2 + lane; j <= r; j += 32) row[j] = fma(-lr, lb[j - k - 1], row[j]);
        }
        __syncthreads();
        __cluster_barrier_wait();
    }
    if (!ok) {
        if (c == 0 && tid == 0) {
            fail[pi] = 1;
            latch_status(p.status, KFAC_NOT_PD);
        }
        return;
    }
    for (int t = warp; t < R; t += nwarps) {
        const int r = c + CL * t;
        const long long o = trc_off(t, c, CL);
        for (int j = lane; j <= r; j += 32) p.L[(long long)r * n + j] = As[o + j];
    }
}

template <int CL>
__global__ void __launch_bounds__(TRC_THREADS, 1) k_tridiag_cluster(Prob* pr, const int* clu_prob, int lds, int nmax,
                                                                    int rmax, int* fail) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ double trc_sm[];
    const int c = (int)cl.block_rank();
    const int pi = clu_prob[blockIdx.x / CL];
    if (fail[pi]) return;   // uniform over the cluster, before any barrier
    const Prob p = pr[pi];
    const int n = p.n;
    const int tid = threadIdx.x, T = blockDim.x;
    const int warp = tid / 32, lane = tid % 32, nwarps = T / 32;
    double* As = trc_sm;              // owned rows, packed
    double* xb = As + lds;            // pivot column by global row (pushed by its owners)
    double* v = xb + nmax;            // reflector, by i = j - b
    double* w = v + nmax;             // tau M v - K v, by i
    double* pp = w + nmax;            // this CTA's partial of M x, by i
    double* pf = pp + nmax;           // tau M v, by i (pushed by the slice owners)
    double* ppin = pf + nmax;         // the cluster's partials of this CTA's slice, [source][entry]
    double* kpin = ppin + CL * rmax;  // the slices' (tau M v)^T v (pushed)
    double* rd = kpin + CL;           // strictly-lower row dots, by local row
    double* red = rd + rmax;          // reductions and the per-column scalars
    const int R = c < n ? (n - c + CL - 1) / CL : 0;

    for (int t = warp; t < R; t += nwarps) {
        const int r = c + CL * t;
        const long long o = trc_off(t, c, CL);
        for (int j = lane; j <= r; j += 32) As[o + j] = p.M[(long long)r * n + j];
    }
    __syncthreads();
    for (int t = tid; t < R; t += T) {     // the first pivot column, to every CTA
        const int r = c + CL * t;
        if (r < 1) continue;
        const double val = As[trc_off(t, c, CL)];
#pragma unroll
        for (int d = 0; d < CL; d++) cl.map_shared_rank(xb, d)[r] = val;
    }
    cl.sync();

    for (int k = 0; k + 2 < n; k++) {
        const int b = k + 1, m = n - b;
        // x = M[b.., k] is in xb[b..n)
        double part = 0.0;
        for (int r = b + 1 + tid; r < n; r += T) part = fma(xb[r], xb[r], part);
        red[tid] = part;
        __syncthreads();
        // Warp 0 forms the reflector's scalars while every warp computes M x
        // over the owned rows: v = s x + (1 - s x_0) e_0 (s = 1/(x_0 - beta)),
        // so M v = s (M x) + (1 - s x_0) M e_0 is assembled afterwards and the
        // latency of the square root and division hides behind the FP64 work.
        if (warp == 0) {
            const double sigma = trc_warp0_sum(red);
            if (lane == 0) {
                const double x0 = xb[b];
                double tk = 0.0, beta = x0, scale = 0.0;
                if (sigma > 0.0) {
                    const double mu = sqrt(x0 * x0 + sigma);
                    beta = (x0 <= 0.0) ? mu : -mu;
                    tk = (beta - x0) / beta;
                    scale = 1.0 / (x0 - beta);
                }
                red[TRC_TK] = tk;
                red[TRC_SCALE] = scale;
                if (c == 0) { p.tau[k] = tk; p.e[k] = beta; }
            }
        }
        // transposed part and diagonal of M x, one thread per column j.  The
        // work of a column falls with j; 32-column chunks go to the warps in a
        // snake order over the four SM sub-partitions (warp w runs on
        // sub-partition w mod 4), so every sub-partition's FP64 pipe gets the
        // same share.
        const int sp = warp & 3, slot = warp >> 2;
        const int snake = (slot & 1) ? 3 - sp : sp;
        for (int q = 4 * slot + snake; 32 * q < m; q += 16) {
            const int j = b + 32 * q + lane;
            if (j >= n) break;
            double acc = 0.0;
            int t0 = j < c ? 0 : (j - c) / CL + 1;
            if (j >= c && (j - c) % CL == 0) acc = As[trc_off(t0 - 1, c, CL) + j] * xb[j];
            long long o = trc_off(t0, c, CL);
            for (int t = t0; t < R; t++) {
                const int r = c + CL * t;
                acc = fma(As[o + j], xb[r], acc);
                o += r + 1;
            }
            pp[j - b] = acc;
        }
        // strictly lower part of the owned rows r > b: four rows per warp,
        // eight lanes per row, one three-step butterfly for all four; the
        // groups (whose work grows with the row) in the same snake order
        {
            const int g = lane >> 3, gl = lane & 7;
            for (int t4 = 4 * (4 * slot + snake); t4 < R; t4 += 4 * nwarps) {
                const int t = t4 + g;
                const int r = c + CL * t;
                double acc = 0.0;
                if (t < R && r > b) {
                    const double* row = As + trc_off(t, c, CL);
                    for (int j = b + gl; j < r; j += 8) acc = fma(row[j], xb[j], acc);
                }
                acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                acc += __shfl_xor_sync(0xffffffffu, acc, 2);
                acc += __shfl_xor_sync(0xffffffffu, acc, 4);
                if (gl == 0 && t < R) rd[t] = acc;
            }
        }
        __syncthreads();
        const double tk = red[TRC_TK], scale = red[TRC_SCALE];
        const bool act = tk != 0.0;      // uniform: every CTA computed the same tk
        const double coef = fma(-scale, xb[b], 1.0);
        const int S = (m + CL - 1) / CL;  // slice length of the cluster reduction
        // this CTA's partial of M v, pushed to the owner of each entry's slice
        for (int i = tid; i < m; i += T) {
            const int r = b + i;
            double a = pp[i], e0 = 0.0;
            if (r % CL == c) {
                const int t = r / CL;
                if (r > b) a += rd[t];
                e0 = As[trc_off(t, c, CL) + b];
            }
            const int dst = i / S;
            cl.map_shared_rank(ppin, dst)[c * rmax + (i - dst * S)] = fma(scale, a, coef * e0);
            const double vi = (i == 0) ? 1.0 : xb[r] * scale;
            v[i] = vi;
            if (c == 0) p.H[(long long)k * n + b + i] = vi;   // reflector k for the back-transformation
        }
        cl.sync();
        // this CTA's slice of tau M v, summed over the partials in a fixed
        // order and pushed to every CTA with the slice's share of (tau M v)^T v
        if (act && warp == 0) {
            const int lo = c * S, hi = min(m, lo + S);
            double kpart = 0.0;
            for (int i = lo + lane; i < hi; i += 32) {
                double y[CL];
#pragma unroll
                for (int u = 0; u < CL; u++) y[u] = ppin[u * rmax + (i - lo)];
#pragma unroll
                for (int h2 = CL / 2; h2 > 0; h2 >>= 1)
#pragma unroll
                    for (int u = 0; u < h2; u++) y[u] += y[u + h2];
                const double pv = tk * y[0];
#pragma unroll
                for (int d = 0; d < CL; d++) cl.map_shared_rank(pf, d)[i] = pv;
                kpart = fma(pv, v[i], kpart);
            }
            for (int o = 16; o > 0; o >>= 1) kpart += __shfl_xor_sync(0xffffffffu, kpart, o);
            if (lane < CL) cl.map_shared_rank(kpin, lane)[c] = kpart;
        }
        cl.sync();
        if (act) {
            if (warp == 0) {   // K = tau (tau M v)^T v / 2 (the same tree in every CTA)
                double ks = lane < CL ? kpin[lane] : 0.0;
                for (int o = 16; o > 0; o >>= 1) ks += __shfl_xor_sync(0xffffffffu, ks, o);
                if (lane == 0) red[TRC_K] = 0.5 * tk * ks;
            }
            __syncthreads();
            const double K = red[TRC_K];
            for (int i = tid; i < m; i += T) w[i] = fma(-K, v[i], pf[i]);
            __syncthreads();
        }
        // column b of the owned rows first, pushed to every CTA as the next pivot column
        for (int t = tid; t < R; t += T) {
            const int r = c + CL * t;
            if (r < b) continue;
            double* a = As + trc_off(t, c, CL) + b;
            double val = *a;
            if (act) {
                val = fma(-v[r - b], w[0], fma(-w[r - b], v[0], val));
                *a = val;
            }
            if (r > b) {
#pragma unroll
                for (int d = 0; d < CL; d++) cl.map_shared_rank(xb, d)[r] = val;
            }
        }
        __cluster_barrier_arrive();
        if (act) {
            // the rest of the update, one warp per row; the rows (whose work
            // grows with t) go to the warps in the snake order, so every SM
            // sub-partition gets the same share of the FP64 work
            for (int t = 4 * slot + snake; t < R; t += nwarps) {
                const int r = c + CL * t;
                if (r <= b) continue;
                double* row = As + trc_off(t, c, CL);
                const double vr = v[r - b], wr = w[r - b];
                for (int j = b + 1 + lane; j <= r; j += 32) row[j] = fma(-vr, w[j - b], fma(-wr, v[j - b], row[j]));
            }
        }
        __syncthreads();
        __cluster_barrier_wait();
    }
    for (int t = tid; t < R; t += T) {
        const int r = c + CL * t;
        p.d[r] = As[trc_off(t, c, CL) + r];
    }
    if (tid == 0 && n >= 2 && (n - 1) % CL == c)
        p.e[n - 2] = As[trc_off((n - 1 - c) / CL, c, CL) + n - 2];
}

// --------------------------------------------------------------------------
// 4. divide and conquer on (d, e)
// --------------------------------------------------------------------------
// Rank-one tearing of every coupling and Q = I.
__global__ void k_dc_init(Prob* pr, int* fail) {
    const Prob p = pr[blockIdx.y];
    const int n = p.n;
    if (fail[blockIdx.y]) return;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)n * n;
         t += (long long)gridDim.x * blockDim.x) {
        int r = (int)(t / n), c = (int)(t % n);
        p.Qa[t] = (r == c) ? 1.0 : 0.0;
        if (c == 0) {
            double v = p.d[r];
            if (r > 0) v -= p.e[r - 1];
            if (r < n - 1) v -= p.e[r];
            p.D[r] = v;
        }
    }
}

// Per merge: z, sign flip, merge-sort of the two sorted halves, normalisation,
// deflation (small z components; nearly equal poles via plane rotations).
__global__ void __launch_bounds__(256) k_dc_prepare(Prob* pr, const Merge* merges, int level_parity, int* fail) {
    __shared__ double sh[40];
    const Merge mg = merges[blockIdx.x];
    const Prob p = pr[mg.prob];
    if (fail[mg.prob]) return;
    const int n = p.n, a = mg.a, s1 = mg.s1, s2 = mg.s2, m = s1 + s2;
    const double* Q = level_parity ? p.Qb : p.Qa;
    const double rho = p.e[a + s1 - 1];
    const bool flip = rho < 0.0;
    double* Ds = p.Ds + a;
    double* zs = p.zs + a;
    int* perm = p.perm + a;
    double dmax = 0.0, zz = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const bool h1 = i < s1;
        const double Di = flip ? -p.D[a + i] : p.D[a + i];
        const double zi = h1 ? Q[(long long)(a + s1 - 1) * n + a + i] : Q[(long long)(a + s1) * n + a + i];
        // own position (halves are ascending in D, descending after the flip)
        const int loc = h1 ? i : i - s1;
        const int sz = h1 ? s1 : s2, osz = h1 ? s2 : s1, obase = h1 ? s1 : 0;
        const int own = flip ? sz - 1 - loc : loc;
        // rank in the other half: # elements with key < Di (ties: half 1 first)
        int lo = 0, hi = osz;
        while (lo < hi) {
            int mid = (lo + hi) / 2;
            int oidx = obase + (flip ? osz - 1 - mid : mid);
            double ok = flip ? -p.D[a + oidx] : p.D[a + oidx];
            bool less = h1 ? (ok < Di) : (ok <= Di);
            if (less) lo = mid + 1; else hi = mid;
        }
        const int pos = own + lo;
        perm[pos] = i;
        Ds[pos] = Di;
        zs[pos] = zi;
        dmax = fmax(dmax, fabs(Di));
        zz = fma(zi, zi, zz);
    }
    const double zn2 = block_reduce_sum(zz, sh);
    dmax = block_reduce_max(dmax, sh);
    const double zn = sqrt(zn2);
    const double rh = fabs(rho) * zn2;
    const double rzn = 1.0 / zn;
    for (int i = threadIdx.x; i < m; i += blockDim.x) zs[i] *= rzn;
    __syncthreads();
    const double tol = 8.0 * DEPS * fmax(dmax, rh);
    // Speculative parallel deflation: the magnitude test per entry, then the
    // pair test of every surviving entry against the previous survivor on the
    // unmodified values.  When no pair deflates, that is exactly what the
    // serial scan below computes (its values only change at a pair deflation),
    // so the survivors are compacted in parallel; otherwise the serial scan
    // runs.  Each thread takes four consecutive entries (m <= 1024).
    if (m <= 4 * (int)blockDim.x) {
        __shared__ int wsh[32];
        const int i0 = 4 * threadIdx.x;
        bool small[4];
        int mylast = -1, mycnt = 0;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int i = i0 + u;
            small[u] = (i >= m) || (rh * fabs(zs[i]) <= tol);
            if (!small[u]) { mylast = i; mycnt++; }
        }
        // exclusive max-scan of the last survivor over the threads
        const int lane = threadIdx.x % 32, wid = threadIdx.x / 32, nw = blockDim.x / 32;
        int incl = mylast;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl = max(incl, y);
        }
        if (lane == 31) wsh[wid] = incl;
        __syncthreads();
        int before = -1;
        for (int w = 0; w < wid; w++) before = max(before, wsh[w]);
        const int up = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane > 0) before = max(before, up);
        __syncthreads();
        bool pair = false;
        int last = before;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int i = i0 + u;
            if (small[u]) continue;
            if (last >= 0) {
                const int j = last;
                const double r2 = fma(zs[j], zs[j], zs[i] * zs[i]);
                if (fabs(zs[i] * zs[j] * (Ds[i] - Ds[j])) <= tol * r2) pair = true;
            }
            last = i;
        }
        if (!__syncthreads_or(pair ? 1 : 0)) {
            // exclusive sum-scan of the survivor counts: the compaction
            int incs = mycnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incs, o);
                if (lane >= o) incs += y;
            }
            if (lane == 31) wsh[wid] = incs;
            __syncthreads();
            int base = 0, total = 0;
            for (int w = 0; w < nw; w++) {
                if (w < wid) base += wsh[w];
                total += wsh[w];
            }
            int kpos = base + incs - mycnt;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int i = i0 + u;
                if (i >= m) break;
                p.defl[a + i] = small[u] ? 1 : 0;
                if (!small[u]) {
                    p.Kidx[a + kpos] = i;
                    p.dK[a + kpos] = Ds[i];
                    p.zK[a + kpos] = zs[i];
                    kpos++;
                }
            }
            if (threadIdx.x == 0) {
                p.mk[a] = total;
                p.mnrot[a] = 0;
                p.mflip[a] = flip ? 1 : 0;
                p.mrh[a] = rh;
            }
            return;
        }
    }
    if (threadIdx.x == 0) {
        int* defl = p.defl + a;
        int nrot = 0, last = -1;
        for (int i = 0; i < m; i++) {
            defl[i] = 0;
            if (rh * fabs(zs[i]) <= tol) { defl[i] = 1; continue; }
            if (last >= 0) {
                const int j = last;
                // |c s (D_i - D_j)| <= tol with c = z_i / r, s = -z_j / r,
                // r^2 = z_i^2 + z_j^2, tested without a division (this loop is
                // serial, and FP64 division is a long sequence on this part);
                // c and s are formed only when the rotation is applied
                const double r2 = fma(zs[j], zs[j], zs[i] * zs[i]);
                if (fabs(zs[i] * zs[j] * (Ds[i] - Ds[j])) <= tol * r2) {
                    const double rr = hypot(zs[j], zs[i]);
                    const double c = zs[i] / rr, s = -zs[j] / rr;
                    const double dj = Ds[j], di = Ds[i];
                    Ds[j] = c * c * dj + s * s * di;
                    Ds[i] = s * s * dj + c * c * di;
                    zs[i] = rr;
                    zs[j] = 0.0;
                    defl[j] = 1;
                    p.rj[a + nrot] = j;
                    p.ri[a + nrot] = i;
                    p.rc[a + nrot] = c;
                    p.rs[a + nrot] = s;
                    nrot++;
                }
            }
            last = i;
        }
        int k = 0;
        for (int i = 0; i < m; i++)
            if (!defl[i]) {
                p.Kidx[a + k] = i;
                p.dK[a + k] = Ds[i];
                p.zK[a + k] = zs[i];
                k++;
            }
        p.mk[a] = k;
        p.mnrot[a] = nrot;
        p.mflip[a] = flip ? 1 : 0;
        p.mrh[a] = rh;
    }
}

// Secular equation 1 + rh sum_t zK_t^2 / (dK_t - lambda) = 0, one warp per
// root; lambda_j = dK[org] + tau with tau measured from the nearer pole, so
// that the differences d_i - lambda_j stay accurate.
__global__ void k_dc_roots(Prob* pr, const Merge* merges, int n_merges, int* fail) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    // locate (merge, j): merges are ordered, sizes known
    const int last = n_merges - 1;
    if (gw >= merges[last].r0 + merges[last].s1 + merges[last].s2) return;
    const int mi = find_merge(merges, n_merges, gw);
    const Merge mg = merges[mi];
    const int j = gw - mg.r0;
    const Prob p = pr[mg.prob];
    if (fail[mg.prob]) return;
    const int a = mg.a;
    const int k = p.mk[a];
    if (j >= k) return;
    const double rh = p.mrh[a];
    const double* dK = p.dK + a;
    const double* zK = p.zK + a;
    auto f = [&](int o, double t) {
        double s = 0.0;
        const double dO = dK[o];
        for (int q = lane; q < k; q += 32) {
            double del = (dK[q] - dO) - t;
            s += zK[q] * zK[q] / del;
        }
        for (int o2 = 16; o2 > 0; o2 >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o2);
        return 1.0 + rh * s;
    };
    int o;
    double lo, hi;
    if (j < k - 1) {
        const double gap = dK[j + 1] - dK[j];
        if (f(j, 0.5 * gap) > 0.0) { o = j; lo = 0.0; hi = 0.5 * gap; }
        else { o = j + 1; lo = -0.5 * gap; hi = 0.0; }
    } else {
        double zz = 0.0;
        for (int q = lane; q < k; q += 32) zz += zK[q] * zK[q];
        for (int o2 = 16; o2 > 0; o2 >>= 1) zz += __shfl_xor_sync(0xffffffffu, zz, o2);
        o = j; lo = 0.0; hi = rh * zz * (1.0 + 8.0 * DEPS) + 4.0 * DEPS * fabs(dK[j]);
    }
    // Safeguarded rational iteration: psi (poles <= d_j) and phi (poles >=
    // d_{j+1}) are each modelled by a constant plus one pole, matched in value
    // and slope at the iterate; the model's root in (lo, hi) is the next
    // iterate (bisection when it falls outside the bracket).
    const double dO = dK[o];
    const double dj = dK[j] - dO;
    const bool has_up = (j < k - 1);
    const double dj1 = has_up ? dK[j + 1] - dO : 0.0;
    double t = 0.5 * (lo + hi);
    {
        // Warm start in FP32 (a reciprocal is one instruction there, a long
        // FP64 sequence on this part): the same two-pole iteration on an FP32
        // copy of the bracket, to about 1e-6 relative.  Only its end point is
        // used, clamped into the FP64 bracket; the FP64 iteration below, whose
        // bracket moves on FP64 signs only, decides the root.
        float l32 = (float)lo, h32 = (float)hi, t32 = (float)t;
        const float dj32 = (float)dj, dj132 = (float)dj1, rh32 = (float)rh;
        for (int it = 0; it < 16; it++) {
            float psi = 0.f, dpsi = 0.f, phi = 0.f, dphi = 0.f;
            for (int q = lane; q < k; q += 32) {
                const float r = 1.0f / ((float)(dK[q] - dO) - t32);
                const float z = (float)zK[q];
                const float tq = z * z * r, dq = tq * r;
                if (q <= j) { psi += tq; dpsi += dq; } else { phi += tq; dphi += dq; }
            }
            for (int o2 = 16; o2 > 0; o2 >>= 1) {
                psi += __shfl_xor_sync(0xffffffffu, psi, o2);
                dpsi += __shfl_xor_sync(0xffffffffu, dpsi, o2);
                phi += __shfl_xor_sync(0xffffffffu, phi, o2);
                dphi += __shfl_xor_sync(0xffffffffu, dphi, o2);
            }
            psi *= rh32; dpsi *= rh32; phi *= rh32; dphi *= rh32;
            const float fv = 1.f + psi + phi;
            if (fv > 0.f) h32 = t32; else l32 = t32;
            const float a1 = dj32 - t32;
            const float q1 = dpsi * a1 * a1;
            const float p1 = psi - q1 / a1;
            float tn = 0.5f * (l32 + h32);
            if (!has_up) {
                const float c = 1.f + p1;
                if (c != 0.f) tn = dj32 + q1 / c;
            } else {
                const float a2 = dj132 - t32;
                const float q2 = dphi * a2 * a2;
                const float p2 = phi - q2 / a2;
                const float c = 1.f + p1 + p2;
                const float B = -(c * (dj32 + dj132) + q1 + q2);
                const float C = c * dj32 * dj132 + q1 * dj132 + q2 * dj32;
                if (c == 0.f) {
                    if (B != 0.f) tn = -C / B;
                } else {
                    const float sq = sqrtf(fmaxf(B * B - 4.f * c * C, 0.f));
                    const float r1 = (-B - copysignf(sq, B)) / (2.f * c);
                    const float r2 = (r1 != 0.f) ? C / (c * r1) : r1;
                    if (r1 > l32 && r1 < h32) tn = r1;
                    else if (r2 > l32 && r2 < h32) tn = r2;
                }
            }
            if (!(tn > l32 && tn < h32)) tn = 0.5f * (l32 + h32);
            const bool done = fabsf(tn - t32) <= 1e-6f * fabsf(tn);
            t32 = tn;
            if (done) break;
        }
        if ((double)t32 > lo && (double)t32 < hi) t = (double)t32;
    }
    for (int it = 0; it < 80; it++) {
        double psi = 0.0, dpsi = 0.0, phi = 0.0, dphi = 0.0, ab = 0.0;
        for (int q = lane; q < k; q += 32) {
            // one reciprocal instead of two divisions (FP64 division is a long
            // instruction sequence on this part)
            const double rdel = 1.0 / ((dK[q] - dO) - t);
            const double z2 = zK[q] * zK[q];
            const double tq = z2 * rdel;
            const double dq = tq * rdel;
            if (q <= j) { psi += tq; dpsi += dq; } else { phi += tq; dphi += dq; }
            ab += fabs(tq);
        }
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            psi += __shfl_xor_sync(0xffffffffu, psi, o2);
            dpsi += __shfl_xor_sync(0xffffffffu, dpsi, o2);
            phi += __shfl_xor_sync(0xffffffffu, phi, o2);
            dphi += __shfl_xor_sync(0xffffffffu, dphi, o2);
            ab += __shfl_xor_sync(0xffffffffu, ab, o2);
        }
        psi *= rh; dpsi *= rh; phi *= rh; dphi *= rh; ab *= rh;
        const double fv = 1.0 + psi + phi;
        if (fabs(fv) <= 8.0 * DEPS * (1.0 + ab)) break;
        if (fv > 0.0) hi = t; else lo = t;
        if (hi - lo <= 2.0 * DEPS * fmax(fabs(lo), fabs(hi))) break;
        const double a1 = dj - t;
        const double q1 = dpsi * a1 * a1;
        const double p1 = psi - q1 / a1;
        double tn;
        if (!has_up) {
            const double c = 1.0 + p1;
            tn = (c != 0.0) ? dj + q1 / c : 0.5 * (lo + hi);
        } else {
            const double a2 = dj1 - t;
            const double q2 = dphi * a2 * a2;
            const double p2 = phi - q2 / a2;
            const double c = 1.0 + p1 + p2;
            // c (dj - x)(dj1 - x) + q1 (dj1 - x) + q2 (dj - x) = 0
            const double B = -(c * (dj + dj1) + q1 + q2);
            const double C = c * dj * dj1 + q1 * dj1 + q2 * dj;
            tn = 0.5 * (lo + hi);
            if (c == 0.0) {
                if (B != 0.0) tn = -C / B;
            } else {
                const double sq = sqrt(fmax(B * B - 4.0 * c * C, 0.0));
                const double r1 = (-B - copysign(sq, B)) / (2.0 * c);
                const double r2 = (r1 != 0.0) ? C / (c * r1) : r1;
                if (r1 > lo && r1 < hi) tn = r1;
                else if (r2 > lo && r2 < hi) tn = r2;
            }
        }
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        t = tn;
    }
    if (lane == 0) {
        p.org[a + j] = o;
        p.tauR[a + j] = t;
    }
}

// Gu-Eisenstat: zhat_i^2 = prod_j (lambda_j - d_i) / (rh prod_{j != i} (d_j - d_i)).
// Gu-Eisenstat: |zhat_i|^2 = (lambda_i - d_i) / rh * prod_{q != i} (lambda_q - d_i) / (d_q - d_i).
// One warp per root: each lane multiplies its share of the factors, then the
// lanes' products are multiplied by a butterfly.
__global__ void k_dc_zhat(Prob* pr, const Merge* merges, int n_merges, int* fail) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x % 32;
    const int last = n_merges - 1;
    if (gw >= merges[last].r0 + merges[last].s1 + merges[last].s2) return;
    const int mi = find_merge(merges, n_merges, gw);
    const Merge mg = merges[mi];
    const int i = gw - mg.r0;
    const Prob p = pr[mg.prob];
    if (fail[mg.prob]) return;
    const int a = mg.a;
    const int k = p.mk[a];
    if (i >= k) return;     // uniform over the warp
    const double rh = p.mrh[a];
    const double* dK = p.dK + a;
    const double* tauR = p.tauR + a;
    const int* org = p.org + a;
    const double di = dK[i];
    // the ratio (lambda_q - d_i) / (d_q - d_i) is O(1) by interlacing, while
    // numerators and denominators alone can be tiny: one division per four
    // factors keeps every intermediate far inside the FP64 range
    double prod = 1.0, num = 1.0, den = 1.0;
    int cnt = 0;
    for (int q = lane; q < k; q += 32) {
        if (q == i) continue;
        num *= -((di - dK[org[q]]) - tauR[q]);
        den *= dK[q] - di;
        if (++cnt == 4) {
            prod *= num / den;
            num = den = 1.0;
            cnt = 0;
        }
    }
    prod *= num / den;
    for (int o = 16; o > 0; o >>= 1) prod *= __shfl_xor_sync(0xffffffffu, prod, o);
    if (lane != 0) return;
    prod *= -((di - dK[org[i]]) - tauR[i]) / rh;    // (lambda_i - d_i) / rh
    const double z = sqrt(fmax(prod, 0.0));
    p.zh[a + i] = (p.zK[a + i] < 0.0) ? -z : z;
}

// Eigenvalue order of the merged block: roots and deflated poles ranked by
// value; writes the new eigenvalues and the output column of each pair.
__global__ void __launch_bounds__(256) k_dc_order(Prob* pr, const Merge* merges, int* fail) {
    const Merge mg = merges[blockIdx.x];
    const Prob p = pr[mg.prob];
    if (fail[mg.prob]) return;
    const int a = mg.a, m = mg.s1 + mg.s2;
    const int k = p.mk[a];
    const bool flip = p.mflip[a] != 0;
    // candidate list: entries 0..k-1 roots, k..m-1 deflated poles (in sorted-basis order)
    double* val = p.val + a;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        double v;
        if (t < k) v = p.dK[a + p.org[a + t]] + p.tauR[a + t];
        else {
            // the (t-k)-th deflated position
            int cnt = -1, pos = 0;
            for (pos = 0; pos < m; pos++)
                if (p.defl[a + pos] && ++cnt == t - k) break;
            v = p.Ds[a + pos];
            val[t] = v;
            p.Kidx[a + t] = pos;                     // deflated positions follow the roots
            continue;
        }
        val[t] = v;
    }
    __syncthreads();
    // ranks by order-preserving 64-bit integer keys of the values (integer
    // compares run on the ALUs, not the scarce FP64 pipe); -0 and +0 tie
    long long* key = reinterpret_cast<long long*>(p.pbuf2 + a);   // scratch of m doubles, free during the merges
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        const double v = val[t] == 0.0 ? 0.0 : val[t];
        const long long b = __double_as_longlong(v);
        key[t] = b >= 0 ? b : (long long)(0x8000000000000000ull ^ ~(unsigned long long)b);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        const double v = val[t];
        const long long kv = key[t];
        int r = 0;
        for (int q = 0; q < m; q++) {
            const long long u = key[q];
            r += (u < kv || (u == kv && q < t)) ? 1 : 0;
        }
        const int c = flip ? m - 1 - r : r;
        p.col[a + t] = c;
        p.D[a + c] = flip ? -v : v;
    }
}

// Reduced eigenvectors u_j = zhat / (d - lambda_j), normalised, written into
// the sorted-basis matrix R (rows = sorted positions, columns = output order);
// deflated pairs are unit columns.  Grid: (column blocks of 32, merges).
__global__ void __launch_bounds__(256) k_dc_fillU(Prob* pr, const Merge* merges, int* fail) {
    const Merge mg = merges[blockIdx.y];
    const Prob p = pr[mg.prob];
    if (fail[mg.prob]) return;
    const int n = p.n, a = mg.a, m = mg.s1 + mg.s2;
    const int k = p.mk[a];
    const int t0 = blockIdx.x * 32;
    if (t0 >= m) return;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    double* R = p.R;
    for (int tt = warp; tt < 32; tt += blockDim.x / 32) {
        const int t = t0 + tt;
        if (t >= m) break;
        const int c = p.col[a + t];
        if (t >= k) {   // deflated: unit vector at its sorted position
            const int pos = p.Kidx[a + t];
            for (int r = lane; r < m; r += 32) R[(long long)(a + r) * n + a + c] = (r == pos) ? 1.0 : 0.0;
            continue;
        }
        const int o = p.org[a + t];
        const double dO = p.dK[a + o], tt_ = p.tauR[a + t];
        for (int r = lane; r < m; r += 32) R[(long long)(a + r) * n + a + c] = 0.0;
        __syncwarp();
        // unnormalised entries first (one division each), then the scaling
        double ss = 0.0;
        for (int q = lane; q < k; q += 32) {
            const double u = p.zh[a + q] / ((p.dK[a + q] - dO) - tt_);
            R[(long long)(a + p.Kidx[a + q]) * n + a + c] = u;
            ss = fma(u, u, ss);
        }
        for (int o2 = 16; o2 > 0; o2 >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o2);
        const double inv = 1.0 / sqrt(ss);
        for (int q = lane; q < k; q += 32) R[(long long)(a + p.Kidx[a + q]) * n + a + c] *= inv;
    }
}

// Undo the deflation rotations (reverse order, on rows of R) and scatter rows
// to the block's original index order: R2[perm[pos]][c] = R[pos][c].
// Deflation rotations on the columns of R, then R2[perm[pos]] = R[pos]; the
// columns are independent, so each CTA takes a chunk of 64 of them.
constexpr int RS_COLS = 64;
__global__ void __launch_bounds__(256) k_dc_rotate_scatter(Prob* pr, const Merge* merges, int* fail) {
    const Merge mg = merges[blockIdx.y];
    const Prob p = pr[mg.prob];
    if (fail[mg.prob]) return;
    const int n = p.n, a = mg.a, m = mg.s1 + mg.s2;
    const int c0 = blockIdx.x * RS_COLS;
    if (c0 >= m) return;
    const int nc = min(RS_COLS, m - c0);
    const int nrot = p.mnrot[a];
    double* R = p.R;
    if (threadIdx.x < nc) {
        const int col = c0 + threadIdx.x;
        for (int t = nrot - 1; t >= 0; t--) {
            const int j = p.rj[a + t], i = p.ri[a + t];
            const double c = p.rc[a + t], s = p.rs[a + t];
            const double uj = R[(long long)(a + j) * n + a + col], ui = R[(long long)(a + i) * n + a + col];
            R[(long long)(a + j) * n + a + col] = c * uj - s * ui;
            R[(long long)(a + i) * n + a + col] = s * uj + c * ui;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m * RS_COLS; t += blockDim.x) {
        const int pos = t / RS_COLS, cc = t % RS_COLS;
        if (cc >= nc) continue;
        const int col = c0 + cc;
        p.R2[(long long)(a + p.perm[a + pos]) * n + a + col] = R[(long long)(a + pos) * n + a + col];
    }
}

// Batched block GEMMs of one level: C = A B (FP64, 64 x 64 tiles).
__global__ void __launch_bounds__(256) k_dc_gemm(const Gd* gd, int n_gd, const int* fail_dummy) {
    __shared__ double As[16][65];
    __shared__ double Bs[16][65];
    const int t = blockIdx.x;
    int gi = 0, hi = n_gd - 1;
    while (gi < hi) {
        int mid = (gi + hi + 1) / 2;
        if (gd[mid].tile0 <= t) gi = mid; else hi = mid - 1;
    }
    const Gd g = gd[gi];
    const int lt = t - g.tile0;
    const int ntn = (g.N + 63) / 64;
    const int i0 = (lt / ntn) * 64, j0 = (lt % ntn) * 64;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < g.K; k0 += 16) {
        for (int q = threadIdx.x; q < 64 * 16; q += blockDim.x) {
            int r = q / 16, kk = q % 16;
            As[kk][r] = (i0 + r < g.M && k0 + kk < g.K) ? g.A[(long long)(i0 + r) * g.ld + k0 + kk] : 0.0;
            int kk2 = q / 64, c = q % 64;
            Bs[kk2][c] = (k0 + kk2 < g.K && j0 + c < g.N) ? g.B[(long long)(k0 + kk2) * g.ld + j0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; kk++) {
            double av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; i++) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int r = i0 + ty + 16 * i, c = j0 + tx + 16 * j;
            if (r < g.M && c < g.N) g.C[(long long)r * g.ld + c] = acc[i][j];
        }
}

__global__ void k_dc_copy(const Copy* cp, int n_cp) {
    const Copy c = cp[blockIdx.y];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < c.m * c.m; t += gridDim.x * blockDim.x) {
        int r = t / c.m, q = t % c.m;
        c.dst[(long long)r * c.ld + q] = c.src[(long long)r * c.ld + q];
    }
}

// --------------------------------------------------------------------------
// 5. back-transformation: U <- H_0 H_1 .. H_{n-3} U, columns in parallel
// --------------------------------------------------------------------------
// Shared memory of k_backtransform for a strip of W columns of an n x n U:
// the strip (n x W), two reflector buffers (2n), the dot partials (8 x W) and
// the reflector coefficients (W).
inline size_t bt_smem_bytes(int n, int W) {
    return sizeof(double) * ((size_t)n * W + 2 * (size_t)n + 9 * (size_t)W);
}
// the most any job can ask for: the widest strip of each width class at the
// largest factor of that class
inline size_t bt_smem_max() {
    return std::max(bt_smem_bytes(KFAC_MAX_WIDTH_PLUS_ONE, 8),
                    std::max(bt_smem_bytes(STRIP_NARROW_FROM - 1, 16), bt_smem_bytes(STRIP_MEDIUM_FROM - 1, 32)));
}

// U <- H_0 H_1 .. H_{n-3} U on a strip of W columns held in shared memory.
// Per reflector: the column dots over 256 / W row groups, folded to one
// partial per warp, summed by warp 0 only (FP64 adds are the scarce
// resource), then the rank-1 update.  The next reflector is loaded into
// registers while the current one is applied (two buffers).
template <int W>
__device__ void bt_strip(const Prob& p, int c0, double* sm, bool form) {
    constexpr int RG = 256 / W;                  // row groups
    const int n = p.n;
    double* Us = sm;                             // n x W
    double* vb = Us + (size_t)n * W;             // two reflectors of n
    double* part = vb + 2 * (size_t)n;           // 8 x W
    double* tot = part + 8 * W;                  // W
    // form: Q_H = H_0 H_1 ... applied to I, into L (free once L^{-1} is formed)
    double* U = form ? p.L : (p.final_buf ? p.Qb : p.Qa);
    const int cl = threadIdx.x % W, rg = threadIdx.x / W;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int c = c0 + cl;
    for (int i = rg; i < n; i += RG)
        Us[i * W + cl] = (c < n) ? (form ? (i == c ? 1.0 : 0.0) : U[(long long)i * n + c]) : 0.0;
    // H_k acts on rows > k, so on e_c only when c > k: starting from I, the
    // reflectors above the strip's last column leave it as it is
    const int k_top = form ? min(n - 3, min(c0 + W, n) - 2) : n - 3;
    // reflector k occupies H[k][k+1 .. n); at most 4 values per thread (n <= 1024)
    auto fetch = [&](int k, double* r4) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int i = threadIdx.x + 256 * u;
            r4[u] = (k >= 0 && i < n - k - 1) ? __ldcg(p.H + (long long)k * n + k + 1 + i) : 0.0;
        }
    };
    double nx[4];
    fetch(k_top, nx);
    for (int k = k_top; k >= 0; k--) {
        const int b = k + 1, m = n - b;
        double* v = vb + (k & 1) * n;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int i = threadIdx.x + 256 * u;
            if (i < m) v[i] = nx[u];
        }
        fetch(k - 1, nx);
        const double tk = p.tau[k];
        __syncthreads();
        if (tk == 0.0) continue;                  // uniform
        double dot = 0.0;
        for (int i = rg; i < m; i += RG) dot = fma(v[i], Us[(b + i) * W + cl], dot);
        // lanes l, l + W, .. of a warp hold the same column: fold them
        if (W <= 16) dot += __shfl_xor_sync(0xffffffffu, dot, 16);
        if (W <= 8) dot += __shfl_xor_sync(0xffffffffu, dot, 8);
        if (lane < W) part[warp * W + lane] = dot;
        __syncthreads();
        if (warp == 0 && lane < W) {
            double t = 0.0;
#pragma unroll
            for (int q = 0; q < 8; q++) t += part[q * W + lane];
            tot[lane] = t * tk;
        }
        __syncthreads();
        const double tt = tot[cl];
        for (int i = rg; i < m; i += RG) Us[(b + i) * W + cl] -= tt * v[i];
    }
    __syncthreads();
    if (c < n)
        for (int i = rg; i < n; i += RG) U[(long long)i * n + c] = Us[i * W + cl];
}

// One CTA per back-transformation job (problem, first column, strip width):
// the widths make the jobs' work about equal, the list is sorted largest
// first.  form: the reflectors' product Q_H itself (applied to I) into L.
__global__ void __launch_bounds__(256) k_backtransform(Prob* pr, const TrsmJob* jobs, int* fail, int form) {
    extern __shared__ double bt_sm[];
    const TrsmJob jb = jobs[blockIdx.x];
    const Prob p = pr[jb.prob];
    if (fail[jb.prob] || jb.c0 >= p.n) return;
    if (jb.cb == 8) bt_strip<8>(p, jb.c0, bt_sm, form != 0);
    else if (jb.cb == 16) bt_strip<16>(p, jb.c0, bt_sm, form != 0);
    else bt_strip<32>(p, jb.c0, bt_sm, form != 0);
}

__global__ void k_write_w(Prob* pr, int* fail) {
    const Prob p = pr[blockIdx.x];
    if (fail[blockIdx.x])      // a failed problem's V and w are zero
        for (long long i = threadIdx.x; i < (long long)p.n * p.n; i += blockDim.x) p.V[i] = 0.0;
    for (int i = threadIdx.x; i < p.n; i += blockDim.x) {
        double v = fail[blockIdx.x] ? 0.0 : p.D[i];
        if (!isfinite(v)) latch_status(p.status, KFAC_NONFINITE);
        p.w[i] = v;
    }
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
template <class T>
kfac_status_t dal(T** p, size_t n) {
    void* v = nullptr;
    kfac_status_t st = kfac_device_alloc(&v, (n == 0 ? 1 : n) * sizeof(T));
    *p = (T*)v;
    return st;
}

int ceil_log2(int n) {
    int l = 0;
    while ((1 << l) < n) l++;
    return l;
}

}  // namespace

static int pair_n(const kfac_pinn_handle* h, int l, int which) { return which == 0 ? h->dims[l - 1] + 1 : h->dims[l]; }

// Packed triangle length of the CTA that stores the most of an n-problem in a
// cluster of CL CTAs, and the cluster kernels' shared memory per CTA.
static int trc_lds(int n, int CL) {
    int lds = 0;
    for (int c = 0; c < CL && c < n; c++) lds = std::max(lds, (int)trc_off((n - c + CL - 1) / CL, c, CL));
    return lds;
}

static size_t trc_smem_bytes(int lds, int nmax, int CL) {
    const int rmax = (nmax + CL - 1) / CL;
    return sizeof(double) * ((size_t)lds + 5 * (size_t)nmax + (size_t)(CL + 1) * rmax + CL + TRC_RED);
}

// Cluster size of a problem of size n: the largest power of two up to 16 that
// leaves every CTA at least 16K of the triangle's n^2 / 2 elements (per
// column, a CTA's FP64 work then outweighs the latency of the cluster
// barriers, so small problems take few SMs and many of them run side by
// side), raised until the triangle fits in the cluster's shared memory (0: it
// does not fit in 16 CTAs).
static int trc_cluster_size(int n, size_t smem_optin) {
    int cl = 1;
    while (2 * cl <= TRC_CL && 2.0 * cl * 32768.0 <= (double)n * n) cl *= 2;
    while (cl <= TRC_CL && trc_smem_bytes(trc_lds(n, cl), n, cl) > smem_optin) cl *= 2;
    return cl <= TRC_CL ? cl : 0;
}

// f(std::integral_constant<int, CL>) for the cluster sizes the kernels are
// built for.
template <class F>
static cudaError_t with_cluster_size(int cl, F&& f) {
    switch (cl) {
        case 1: return f(std::integral_constant<int, 1>{});
        case 2: return f(std::integral_constant<int, 2>{});
        case 4: return f(std::integral_constant<int, 4>{});
        case 8: return f(std::integral_constant<int, 8>{});
        case 16: return f(std::integral_constant<int, 16>{});
        default: return cudaErrorInvalidValue;
    }
}

static cudaError_t trc_cluster_attributes(int cl, int optin) {
    return with_cluster_size(cl, [&](auto c) {
        constexpr int C = decltype(c)::value;
        cudaFuncSetAttribute(k_tridiag_cluster<C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(k_tridiag_cluster<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        cudaFuncSetAttribute(k_chol_cluster<C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        return cudaFuncSetAttribute(k_chol_cluster<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    });
}

static cudaLaunchConfig_t trc_config(cudaLaunchAttribute* attr, int cl, int np, size_t smem, cudaStream_t s) {
    attr->id = cudaLaunchAttributeClusterDimension;
    attr->val.clusterDim.x = cl;
    attr->val.clusterDim.y = 1;
    attr->val.clusterDim.z = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cl * np);
    lc.blockDim = dim3(TRC_THREADS);
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return lc;
}

static cudaError_t trc_max_clusters(int cl, int np, size_t smem, int* clusters) {
    cudaLaunchAttribute attr;
    const cudaLaunchConfig_t lc = trc_config(&attr, cl, np, smem, nullptr);
    return with_cluster_size(cl, [&](auto c) {
        return cudaOccupancyMaxActiveClusters(clusters, k_tridiag_cluster<decltype(c)::value>, &lc);
    });
}

static kfac_status_t group_schedule(kfac_pinn_handle* h0, EigState* es);

// One group of factor pairs (layer, 0: A / 1: B) of one handle solved by one
// sequence of batched kernels: the problems' workspaces, then the schedule.
static kfac_status_t group_alloc(kfac_pinn_handle* h, EigState* es, const std::vector<std::pair<int, int>>& pairs) {
    es->np = 0;
    size_t dtot = 0, itot = 0;
    std::vector<int> ns;
    for (const auto& pw : pairs) ns.push_back(pair_n(h, pw.first, pw.second));
    for (int n : ns) {
        dtot += 8 * (size_t)n * n + (size_t)n * NB + 20 * (size_t)n;
        itot += 12 * (size_t)n;
    }
    kfac_status_t st;
    if ((st = dal(&es->ws, dtot))) return st;
    if ((st = dal(&es->iws, itot))) return st;
    double* dp = es->ws;
    int* ip = es->iws;
    es->host.assign(pairs.size(), Prob());
    const double eps = h->cfg.damping_sqrt ? sqrt(h->cfg.lambda) : h->cfg.lambda;
    for (const auto& pw : pairs) {
        {
            const int l = pw.first, which = pw.second;
            Prob& p = es->host[es->np++];
            memset(&p, 0, sizeof(p));
            p.eps = eps;
            p.status = h->status;
            const int n = which == 0 ? h->dims[l - 1] + 1 : h->dims[l];
            p.n = n;
            p.P = h->fac[which == 0 ? KFAC_A_INT : KFAC_B_INT][l - 1];
            p.Q = h->fac[which == 0 ? KFAC_A_BDY : KFAC_B_BDY][l - 1];
            p.V = which == 0 ? h->VA[l - 1] : h->VB[l - 1];
            p.w = which == 0 ? h->wa[l - 1] : h->wb[l - 1];
            size_t nn = (size_t)n * n;
            p.L = dp; dp += nn;
            p.M = dp; dp += nn;
            p.Qa = dp; dp += nn;
            p.Qb = dp; dp += nn;
            p.R = dp; dp += nn;
            p.R2 = dp; dp += nn;
            p.H = dp; dp += nn;
            p.Li = dp; dp += nn;
            p.Ld = dp; dp += (size_t)n * NB;
            double** dv[] = {&p.d, &p.e, &p.tau, &p.D, &p.pbuf, &p.Ds, &p.zs, &p.dK, &p.zK, &p.tauR, &p.zh,
                             &p.rc, &p.rs, &p.val, &p.mrh};
            for (double** q : dv) { *q = dp; dp += n; }
            p.pbuf2 = dp;
            dp += 5 * (size_t)n;
            int** iv[] = {&p.perm, &p.defl, &p.Kidx, &p.org, &p.rj, &p.ri, &p.col, &p.mk, &p.mnrot, &p.mflip};
            for (int** q : iv) { *q = ip; ip += n; }
            ip += 2 * (size_t)n;
            // the number of merge levels fixes which buffer holds the result
            p.final_buf = ceil_log2(n) & 1;
        }
    }
    // L^{-1} is written from each column's diagonal block down: the blocks
    // above stay zero
    for (const Prob& p : es->host)
        if (cudaMemset(p.Li, 0, sizeof(double) * (size_t)p.n * p.n) != cudaSuccess) return KFAC_CUDA_ERROR;
    return group_schedule(h, es);
}

// The device copy of the problem list es->host and every schedule of the
// kernel sequence (cooperative groups, triangular-solve jobs, clusters, merge
// levels).  h0 supplies the device and the SM budget.
static kfac_status_t group_schedule(kfac_pinn_handle* h0, EigState* es) {
    kfac_pinn_handle* h = h0;
    kfac_status_t st;
    es->np = (int)es->host.size();
    es->nmax = 0;
    for (const Prob& p : es->host) es->nmax = std::max(es->nmax, p.n);
    if ((st = dal(&es->dev, (size_t)es->np))) return st;
    if (cudaMemcpy(es->dev, es->host.data(), sizeof(Prob) * es->np, cudaMemcpyHostToDevice) != cudaSuccess)
        return KFAC_CUDA_ERROR;
    if ((st = dal(&es->fail, (size_t)es->np))) return st;
    if ((st = dal(&es->bar, 3 * (size_t)es->np))) return st;
    if ((st = dal(&es->abort_flag, 1))) return st;
    cudaMemset(es->fail, 0, sizeof(int) * es->np);

    bool coop_fits = false;
    // cooperative tridiagonalisation: CTAs per problem ~ n^3, two CTAs per SM
    // (one CTA's synchronisation stalls overlap the other's FP64 work)
    {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tridiag, 512, 0);
        const int sms = h->cfg.eig_sm_budget > 0 ? std::min(h->cfg.eig_sm_budget, h->sm_count) : h->sm_count;
        int budget = sms * std::max(1, std::min(per_sm, 2));
        std::vector<double> wgt(es->np);
        double tot = 0.0;
        int need = 0;
        for (int i = 0; i < es->np; i++) {
            double n = es->host[i].n;
            wgt[i] = n > 2 ? n * n * n : 0.0;
            tot += wgt[i];
        }
        std::vector<int> g(es->np, 1);
        for (int i = 0; i < es->np; i++) need += 1;
        int spare = std::max(0, budget - need);
        for (int i = 0; i < es->np; i++) {
            if (tot > 0) g[i] += (int)floor(spare * wgt[i] / tot);
            int cap = std::max(1, es->host[i].n / 8);
            g[i] = std::min(g[i], cap);
        }
        std::vector<int> cp, cr;
        for (int i = 0; i < es->np; i++)
            for (int r = 0; r < g[i]; r++) { cp.push_back(i); cr.push_back(r); }
        es->n_cta = (int)cp.size();
        if ((st = dal(&es->cta_prob, cp.size()))) return st;
        if ((st = dal(&es->cta_rank, cr.size()))) return st;
        if ((st = dal(&es->group, (size_t)es->np))) return st;
        cudaMemcpy(es->cta_prob, cp.data(), sizeof(int) * cp.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(es->cta_rank, cr.data(), sizeof(int) * cr.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(es->group, g.data(), sizeof(int) * g.size(), cudaMemcpyHostToDevice);
        // (needed only when the cluster kernel below cannot take the problems)
        coop_fits = per_sm * h->sm_count >= es->n_cta;
    }

    // triangular-solve jobs of about equal work, largest first
    {
        std::vector<TrsmJob> jobs;
        for (int i = 0; i < es->np; i++) {
            const int n = es->host[i].n;
            const int cb = strip_width(n);
            for (int c0 = 0; c0 < n; c0 += cb) jobs.push_back(TrsmJob{i, c0, cb, n});
        }
        std::stable_sort(jobs.begin(), jobs.end(), [&](const TrsmJob& x, const TrsmJob& y) {
            const double wx = (double)es->host[x.prob].n * es->host[x.prob].n * x.cb;
            const double wy = (double)es->host[y.prob].n * es->host[y.prob].n * y.cb;
            return wx > wy;
        });
        es->n_trsm_jobs = (int)jobs.size();
        es->bt_smem = 0;
        for (const TrsmJob& j : jobs) es->bt_smem = std::max(es->bt_smem, bt_smem_bytes(es->host[j.prob].n, j.cb));
        kfac_status_t ast = kfac_device_alloc(&es->trsm_jobs, sizeof(TrsmJob) * jobs.size());
        if (ast != KFAC_OK) return ast;
        cudaMemcpy(es->trsm_jobs, jobs.data(), sizeof(TrsmJob) * jobs.size(), cudaMemcpyHostToDevice);
        // the upper-triangle solve of a strip runs down to its last column
        auto upper_work = [&](const TrsmJob& j) {
            const double e = std::min(es->host[j.prob].n, j.c0 + j.cb);
            return e * e * j.cb;
        };
        std::stable_sort(jobs.begin(), jobs.end(),
                         [&](const TrsmJob& x, const TrsmJob& y) { return upper_work(x) > upper_work(y); });
        if ((ast = kfac_device_alloc(&es->trsm_jobs_upper, sizeof(TrsmJob) * jobs.size())) != KFAC_OK) return ast;
        cudaMemcpy(es->trsm_jobs_upper, jobs.data(), sizeof(TrsmJob) * jobs.size(), cudaMemcpyHostToDevice);
        // the inverse's strip runs from the block of its first column down, in a
        // split inverse down to the end of the strip's diagonal block
        for (TrsmJob& j : jobs) {
            const int n1 = inv_split(es->host[j.prob].n);
            j.r_end = (n1 > 0 && j.c0 < n1) ? n1 : es->host[j.prob].n;
        }
        auto inv_work = [&](const TrsmJob& j) {
            const double e = j.r_end - (j.c0 / NB) * NB;
            return e * e * j.cb;
        };
        std::stable_sort(jobs.begin(), jobs.end(),
                         [&](const TrsmJob& x, const TrsmJob& y) { return inv_work(x) > inv_work(y); });
        if ((ast = kfac_device_alloc(&es->trsm_jobs_inv, sizeof(TrsmJob) * jobs.size())) != KFAC_OK) return ast;
        cudaMemcpy(es->trsm_jobs_inv, jobs.data(), sizeof(TrsmJob) * jobs.size(), cudaMemcpyHostToDevice);
    }

    // cluster tridiagonalisation: one cluster per problem when the problems'
    // lower triangles fit in the cluster's shared memory (the group's
    // problems share one cluster size)
    es->trc_cl = 0;
    es->clu_prob = nullptr;
    {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
        const int CL = trc_cluster_size(es->nmax, (size_t)optin);
        int lds = 0, rmax = 0;
        size_t smem = 0;
        if (CL > 0) {
            for (const Prob& p : es->host) lds = std::max(lds, trc_lds(p.n, CL));
            rmax = (es->nmax + CL - 1) / CL;
            smem = trc_smem_bytes(lds, es->nmax, CL);
        }
        int clusters = 0;
        if (CL > 0 && trc_cluster_attributes(CL, optin) == cudaSuccess &&
            trc_max_clusters(CL, es->np, smem, &clusters) == cudaSuccess && clusters >= 1) {
            std::vector<int> order(es->np);
            for (int i = 0; i < es->np; i++) order[i] = i;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return es->host[x].n > es->host[y].n; });
            if ((st = dal(&es->clu_prob, order.size()))) return st;
            cudaMemcpy(es->clu_prob, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice);
            es->trc_cl = CL;
            es->trc_lds = lds;
            es->trc_rmax = rmax;
            es->trc_smem = smem;
        }
        cudaGetLastError();   // a refused configuration only selects the cooperative kernel
    }
    if (es->trc_cl == 0 && !coop_fits) return KFAC_BAD_ARG;

    // divide-and-conquer schedules, one per merge level
    for (int s = 1; s < es->nmax; s *= 2) {
        std::vector<Merge> mg;
        std::vector<Gd> gd;
        std::vector<Copy> cp;
        const int parity = (int)es->levels.size() & 1;     // input buffer of this level
        int tiles = 0, roots = 0, max_m = 0, max_copy = 0;
        for (int i = 0; i < es->np; i++) {
            const Prob& p = es->host[i];
            const int n = p.n;
            if (s >= n) continue;          // this problem is done
            double* Qin = parity ? p.Qb : p.Qa;
            double* Qout = parity ? p.Qa : p.Qb;
            for (int a = 0; a < n; a += 2 * s) {
                const int s1 = std::min(s, n - a), s2 = std::min(s, n - a - s1);
                if (s2 <= 0) {
                    Copy c;
                    c.src = Qin + (size_t)a * n + a;
                    c.dst = Qout + (size_t)a * n + a;
                    c.ld = n;
                    c.m = s1;
                    cp.push_back(c);
                    max_copy = std::max(max_copy, s1);
                    continue;
                }
                Merge m;
                m.prob = i; m.a = a; m.s1 = s1; m.s2 = s2; m.r0 = roots;
                mg.push_back(m);
                roots += s1 + s2;
                max_m = std::max(max_m, s1 + s2);
                // Qout[a..a+s1, a..a+m] = Qin[a..a+s1, a..a+s1] R2[a..a+s1, a..a+m]
                Gd g1;
                g1.A = Qin + (size_t)a * n + a;
                g1.B = p.R2 + (size_t)a * n + a;
                g1.C = Qout + (size_t)a * n + a;
                g1.ld = n; g1.M = s1; g1.N = s1 + s2; g1.K = s1; g1.tile0 = tiles;
                tiles += ((s1 + 63) / 64) * ((s1 + s2 + 63) / 64);
                gd.push_back(g1);
                Gd g2;
                g2.A = Qin + (size_t)(a + s1) * n + a + s1;
                g2.B = p.R2 + (size_t)(a + s1) * n + a;
                g2.C = Qout + (size_t)(a + s1) * n + a;
                g2.ld = n; g2.M = s2; g2.N = s1 + s2; g2.K = s2; g2.tile0 = tiles;
                tiles += ((s2 + 63) / 64) * ((s1 + s2 + 63) / 64);
                gd.push_back(g2);
            }
        }
        // the block GEMMs with a contraction of at least OZ_MIN_K run as
        // error-free FP64 emulations on the tensor cores, the rest here
        std::vector<OzGemm> big;
        {
            std::vector<Gd> small;
            int t2 = 0;
            for (Gd g : gd) {
                if (g.K >= OZ_MIN_K) {
                    big.push_back(OzGemm{g.A, g.ld, g.B, g.ld, g.C, g.ld, g.M, g.N, g.K});
                    continue;
                }
                g.tile0 = t2;
                t2 += ((g.M + 63) / 64) * ((g.N + 63) / 64);
                small.push_back(g);
            }
            gd.swap(small);
            tiles = t2;
        }
        Level lv;
        memset(&lv, 0, sizeof(lv));
        if (!big.empty() && (st = oz_plan_create(big, es->host[0].status, &lv.oz))) {
            oz_plan_free(lv.oz);
            return st;
        }
        lv.n_merges = (int)mg.size();
        lv.n_gemms = (int)gd.size();
        lv.n_tiles = tiles;
        lv.n_copies = (int)cp.size();
        lv.max_copy = max_copy;
        lv.roots = roots;
        lv.max_m = max_m;
        if ((st = dal(&lv.merges, mg.size()))) return st;
        if ((st = dal(&lv.gemms, gd.size()))) return st;
        if ((st = dal(&lv.copies, cp.size()))) return st;
        if (!mg.empty()) cudaMemcpy(lv.merges, mg.data(), sizeof(Merge) * mg.size(), cudaMemcpyHostToDevice);
        if (!gd.empty()) cudaMemcpy(lv.gemms, gd.data(), sizeof(Gd) * gd.size(), cudaMemcpyHostToDevice);
        if (!cp.empty()) cudaMemcpy(lv.copies, cp.data(), sizeof(Copy) * cp.size(), cudaMemcpyHostToDevice);
        es->levels.push_back(lv);
    }
    // the products with L^{-1} on the tensor cores
    {
        std::vector<OzGemm> r1, r2, wq, vv, i1, i2;
        for (const Prob& p : es->host) {
            const int n = p.n;
            const int n1 = inv_split(n), n2 = n - n1;
            if (n1 > 0) {          // T = L21 X11 (into Qa, n2 x n1), X21 = -X22 T
                OzGemm t;
                t.A = p.L + (size_t)n1 * n; t.lda = n;
                t.B = p.Li; t.ldb = n;
                t.C = p.Qa; t.ldc = n1;
                t.M = n2; t.N = n1; t.K = n1;
                i1.push_back(t);
                OzGemm x;
                x.A = p.Li + (size_t)n1 * n + n1; x.lda = n;
                x.B = p.Qa; x.ldb = n1;
                x.C = p.Li + (size_t)n1 * n; x.ldc = n;
                x.M = n2; x.N = n1; x.K = n2;
                x.alpha = -1.0;
                i2.push_back(x);
            }
            OzGemm g;
            g.M = g.N = g.K = n;
            g.lda = g.ldb = g.ldc = n;
            g.A = p.Li; g.B = p.M; g.C = p.Qa; g.ta = false; g.tb = false;      // Qa = L^{-1} M
            r1.push_back(g);
            g.A = p.Qa; g.B = p.Li; g.C = p.M; g.ta = false; g.tb = true;       // M = Qa L^{-T}
            r2.push_back(g);
            g.A = p.Li; g.B = p.L; g.C = p.H; g.ta = true; g.tb = false;        // W = L^{-T} Q_H
            wq.push_back(g);
            g.A = p.H; g.B = p.final_buf ? p.Qb : p.Qa; g.C = p.V; g.ta = false; // V = W U
            vv.push_back(g);
        }
        int* status = es->host[0].status;
        if (!i1.empty()) {
            if ((st = oz_plan_create(i1, status, &es->oz_inv1))) return st;
            if ((st = oz_plan_create(i2, status, &es->oz_inv2))) return st;
        }
        if ((st = oz_plan_create(r1, status, &es->oz_red1))) return st;
        if ((st = oz_plan_create(r2, status, &es->oz_red2))) return st;
        if ((st = oz_plan_create(wq, status, &es->oz_w))) return st;
        if ((st = oz_plan_create(vv, status, &es->oz_v))) return st;
        if (cudaStreamCreateWithFlags(&es->aux, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&es->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&es->ev_join, cudaEventDisableTiming) != cudaSuccess)
            return KFAC_CUDA_ERROR;
    }
    cudaFuncSetAttribute(k_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(double) * (NB * (NB + 1) + 2 * NB * (CB_MAX + 1)));
    cudaFuncSetAttribute(k_diag_inv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(double) * 2 * NB * (NB + 1));
    // The attribute belongs to the kernel, not to this handle: set it for the
    // largest factor any handle can have (h_l + 1 <= 1024), so that handles of
    // different sizes can be created in any order.
    static_assert(KFAC_MAX_WIDTH_PLUS_ONE == 1024, "factor size bound");
    if (es->bt_smem > bt_smem_max()) return KFAC_BAD_ARG;
    cudaFuncSetAttribute(k_backtransform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt_smem_max());
    return cudaGetLastError() == cudaSuccess ? KFAC_OK : KFAC_CUDA_ERROR;
}

static kfac_status_t eigall_free_streams(EigAll* ea);

static void group_free(EigState* es) {
    if (!es) return;
    cudaFree(es->ws);
    cudaFree(es->iws);
    cudaFree(es->dev);
    cudaFree(es->fail);
    cudaFree(es->bar);
    cudaFree(es->abort_flag);
    cudaFree(es->cta_prob);
    cudaFree(es->cta_rank);
    cudaFree(es->group);
    cudaFree(es->clu_prob);
    cudaFree(es->trsm_jobs);
    cudaFree(es->trsm_jobs_upper);
    cudaFree(es->trsm_jobs_inv);
    oz_plan_free(es->oz_red1);
    oz_plan_free(es->oz_red2);
    oz_plan_free(es->oz_inv1);
    oz_plan_free(es->oz_inv2);
    oz_plan_free(es->oz_w);
    oz_plan_free(es->oz_v);
    if (es->aux) {
        cudaStreamSynchronize(es->aux);
        cudaStreamDestroy(es->aux);
    }
    if (es->ev_fork) cudaEventDestroy(es->ev_fork);
    if (es->ev_join) cudaEventDestroy(es->ev_join);
    for (auto& lv : es->levels) {
        oz_plan_free(lv.oz);
        cudaFree(lv.merges);
        cudaFree(lv.gemms);
        cudaFree(lv.copies);
    }
    delete es;
}

static kfac_status_t group_run(kfac_pinn_handle* h, EigState* es, cudaStream_t s) {
    const int np = es->np;
    Prob* pr = es->dev;
    const int nmax = es->nmax;
    const int nblk = (nmax + NB - 1) / NB;

    k_damp<<<dim3(64, np), 256, 0, s>>>(pr, es->fail);
    KFAC_LAUNCH_CHECK(h);
    // 1. Cholesky: one cluster per problem, or the blocked kernels
    if (es->trc_cl > 0) {
        cudaLaunchAttribute attr;
        const cudaLaunchConfig_t lc =
            trc_config(&attr, es->trc_cl, np, sizeof(double) * ((size_t)es->trc_lds + 3 * (size_t)nmax + 8), s);
        KFAC_CUDA_TRY(with_cluster_size(es->trc_cl, [&](auto c) {
            return cudaLaunchKernelEx(&lc, k_chol_cluster<decltype(c)::value>, (Prob*)pr, (const int*)es->clu_prob,
                                      es->trc_lds, nmax, (int*)es->fail);
        }));
        h->launches++;
    }
    for (int kb = 0; es->trc_cl == 0 && kb < nblk; kb++) {
        const int k0 = kb * NB;
        k_chol_diag<<<np, 256, 0, s>>>(pr, k0, es->fail);
        KFAC_LAUNCH_CHECK(h);
        const int rows = nmax - k0 - NB;
        if (rows <= 0) continue;
        const int rb = (rows + NB - 1) / NB;
        k_chol_panel<<<dim3(rb, np), 256, 0, s>>>(pr, k0, es->fail);
        KFAC_LAUNCH_CHECK(h);
        k_chol_update<<<dim3(rb * (rb + 1) / 2, np), 256, 0, s>>>(pr, k0, es->fail);
        KFAC_LAUNCH_CHECK(h);
    }
    // 2. whitening
    k_diag_inv<<<dim3(nblk, np), 256, 2 * NB * (NB + 1) * sizeof(double), s>>>(pr, es->fail);
    KFAC_LAUNCH_CHECK(h);
    const int smem_trsm = (int)sizeof(double) * (NB * (NB + 1) + 2 * NB * (CB_MAX + 1));
    // L^{-1} on the FP64 cores, then M = L^{-1} Q L^{-T} on the tensor cores
    k_trsm<<<es->n_trsm_jobs, 256, smem_trsm, s>>>(pr, (const TrsmJob*)es->trsm_jobs_inv, 3, es->fail);
    KFAC_LAUNCH_CHECK(h);
    if (es->oz_inv1) {
        KFAC_TRY(oz_run(h, es->oz_inv1, s));
        KFAC_TRY(oz_run(h, es->oz_inv2, s));
    }
    KFAC_TRY(oz_run(h, es->oz_red1, s));
    KFAC_TRY(oz_run(h, es->oz_red2, s));
    k_symmetrize<<<dim3(64, np), 256, 0, s>>>(pr, es->fail);
    KFAC_LAUNCH_CHECK(h);
    // 3. tridiagonalisation: one cluster per problem, or cooperative groups of CTAs
    if (es->trc_cl > 0) {
        cudaLaunchAttribute attr;
        const cudaLaunchConfig_t lc = trc_config(&attr, es->trc_cl, np, es->trc_smem, s);
        KFAC_CUDA_TRY(with_cluster_size(es->trc_cl, [&](auto c) {
            return cudaLaunchKernelEx(&lc, k_tridiag_cluster<decltype(c)::value>, (Prob*)pr,
                                      (const int*)es->clu_prob, es->trc_lds, es->nmax, es->trc_rmax, (int*)es->fail);
        }));
        h->launches++;
    } else {
        KFAC_CUDA_TRY(cudaMemsetAsync(es->bar, 0, sizeof(unsigned) * 3 * np, s));
        KFAC_CUDA_TRY(cudaMemsetAsync(es->abort_flag, 0, sizeof(int), s));
        // cooperative launch (every CTA co-resident), in the form stream capture accepts
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeCooperative;
        attr.val.cooperative = 1;
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(es->n_cta);
        lc.blockDim = dim3(512);
        lc.dynamicSmemBytes = 0;
        lc.stream = s;
        lc.attrs = &attr;
        lc.numAttrs = 1;
        KFAC_CUDA_TRY(cudaLaunchKernelEx(&lc, k_tridiag, (Prob*)pr, (const int*)es->cta_prob,
                                         (const int*)es->cta_rank, (const int*)es->group, (unsigned*)es->bar,
                                         (int*)es->abort_flag, (int*)es->fail));
        h->launches++;
    }
    // 5a. beside the divide and conquer (on the group's own stream): the
    // reflectors' product Q_H (in L) and W = L^{-T} Q_H (in H), so that the
    // back-transformation and V = L^{-T} Q_H U become one product afterwards
    KFAC_CUDA_TRY(cudaEventRecord(es->ev_fork, s));
    KFAC_CUDA_TRY(cudaStreamWaitEvent(es->aux, es->ev_fork, 0));
    k_backtransform<<<es->n_trsm_jobs, 256, es->bt_smem, es->aux>>>(pr, (const TrsmJob*)es->trsm_jobs_upper,
                                                                    es->fail, 1);
    kfac_status_t st_aux = cudaGetLastError() == cudaSuccess ? KFAC_OK : KFAC_CUDA_ERROR;
    h->launches++;
    if (st_aux == KFAC_OK) st_aux = oz_run(h, es->oz_w, es->aux);
    // the join is recorded even after an error so that s never runs ahead of aux
    KFAC_CUDA_TRY(cudaEventRecord(es->ev_join, es->aux));
    if (st_aux) {
        KFAC_CUDA_TRY(cudaStreamWaitEvent(s, es->ev_join, 0));
        return st_aux;
    }
    // 4. divide and conquer
    k_dc_init<<<dim3(64, np), 256, 0, s>>>(pr, es->fail);
    KFAC_LAUNCH_CHECK(h);
    for (size_t li = 0; li < es->levels.size(); li++) {
        const Level& lv = es->levels[li];
        const int parity = (int)li & 1;
        if (lv.n_merges > 0) {
            k_dc_prepare<<<lv.n_merges, 256, 0, s>>>(pr, lv.merges, parity, es->fail);
            KFAC_LAUNCH_CHECK(h);
            k_dc_roots<<<ceil_div_u((long long)lv.roots * 32, 256), 256, 0, s>>>(pr, lv.merges, lv.n_merges,
                                                                                es->fail);
            KFAC_LAUNCH_CHECK(h);
            k_dc_zhat<<<ceil_div_u((long long)lv.roots * 32, 256), 256, 0, s>>>(pr, lv.merges, lv.n_merges, es->fail);
            KFAC_LAUNCH_CHECK(h);
            k_dc_order<<<lv.n_merges, 256, 0, s>>>(pr, lv.merges, es->fail);
            KFAC_LAUNCH_CHECK(h);
            k_dc_fillU<<<dim3((lv.max_m + 31) / 32, lv.n_merges), 256, 0, s>>>(pr, lv.merges, es->fail);
            KFAC_LAUNCH_CHECK(h);
            k_dc_rotate_scatter<<<dim3((lv.max_m + RS_COLS - 1) / RS_COLS, lv.n_merges), 256, 0, s>>>(
                pr, lv.merges, es->fail);
            KFAC_LAUNCH_CHECK(h);
            if (lv.oz) KFAC_TRY(oz_run(h, lv.oz, s));
            if (lv.n_tiles > 0) {
                k_dc_gemm<<<lv.n_tiles, 256, 0, s>>>(lv.gemms, lv.n_gemms, es->fail);
                KFAC_LAUNCH_CHECK(h);
            }
        }
        if (lv.n_copies > 0) {
            k_dc_copy<<<dim3(ceil_div_u((long long)lv.max_copy * lv.max_copy, 256), lv.n_copies), 256, 0, s>>>(
                lv.copies, lv.n_copies);
            KFAC_LAUNCH_CHECK(h);
        }
    }
    // 5b, 6. V = L^{-T} Q_H U = W U
    KFAC_CUDA_TRY(cudaStreamWaitEvent(s, es->ev_join, 0));
    KFAC_TRY(oz_run(h, es->oz_v, s));
    k_write_w<<<np, 256, 0, s>>>(pr, es->fail);
    KFAC_LAUNCH_CHECK(h);
    return KFAC_OK;
}

// Self-check of the group barrier's bound: a group of two CTAs of which only
// this one is launched, so the barrier cannot complete and must give up after
// limit_ns (kfac_pinn_check_wait_timeout).
__global__ void k_check_group_barrier(unsigned* bar, int* abort_flag, int* status, uint64_t limit_ns) {
    if (!group_barrier(bar, 2, abort_flag, limit_ns) && threadIdx.x == 0) latch_status(status, KFAC_TIMEOUT);
}

kfac_status_t eig_check_wait(kfac_pinn_handle* h, cudaStream_t s, uint64_t limit_ns) {
    void* scratch = nullptr;     // barrier counter, generation and abort flag
    kfac_status_t st = kfac_device_alloc(&scratch, 4 * sizeof(unsigned));
    if (st) return st;
    cudaError_t e = cudaMemsetAsync(scratch, 0, 4 * sizeof(unsigned), s);
    if (e == cudaSuccess) {
        unsigned* bar = (unsigned*)scratch;
        k_check_group_barrier<<<1, 128, 0, s>>>(bar, (int*)(bar + 2), h->status, limit_ns);
        h->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(scratch);
    if (e != cudaSuccess) {
        kfac_record_cuda_error(e);
        return KFAC_CUDA_ERROR;
    }
    return KFAC_OK;
}

// Factor pairs of size at least 3/4 of the largest form the first group, the
// rest the second (run on a stream of the handle's own, forked from and joined
// back into the caller's stream; both are captured when the step is).
// Class of a factor pair: its cluster size, 0 for the cooperative kernel.
static int pair_class(int n, const kfac_pinn_handle* h) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    return trc_cluster_size(n, (size_t)optin);
}

// The order of the groups: the largest cluster size first (it runs on the
// caller's stream), the cooperative class last.
static int class_rank(int cl) { return cl == 0 ? 99 : -cl; }

static kfac_status_t eigall_streams(EigAll* ea) {
    if (ea->ng < 2) return KFAC_OK;
    if (cudaEventCreateWithFlags(&ea->fork, cudaEventDisableTiming) != cudaSuccess) return KFAC_CUDA_ERROR;
    for (int i = 0; i + 1 < ea->ng; i++)
        if (cudaStreamCreateWithFlags(&ea->side[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ea->join[i], cudaEventDisableTiming) != cudaSuccess)
            return KFAC_CUDA_ERROR;
    return KFAC_OK;
}

kfac_status_t eig_alloc(kfac_pinn_handle* h) {
    EigAll* ea = new EigAll();
    memset(ea, 0, sizeof(*ea));
    h->eig = ea;
    std::map<int, std::vector<std::pair<int, int>>> byclass;   // class rank -> (layer, which)
    for (int l = 1; l <= h->cfg.L; l++)
        for (int w = 0; w < 2; w++) byclass[class_rank(pair_class(pair_n(h, l, w), h))].push_back({l, w});
    kfac_status_t st;
    for (auto& kv : byclass) {
        EigState* es = new EigState();
        ea->g[ea->ng++] = es;
        if ((st = group_alloc(h, es, kv.second))) return st;
    }
    return eigall_streams(ea);
}

static void eigall_free(EigAll* ea) {
    if (!ea) return;
    eigall_free_streams(ea);
    for (int i = 0; i < MAX_GROUPS; i++) group_free(ea->g[i]);
    delete ea;
}

void eig_free(kfac_pinn_handle* h) {
    eigall_free(EA(h));
    h->eig = nullptr;
}

static kfac_status_t eigall_free_streams(EigAll* ea) {
    for (int i = 0; i + 1 < MAX_GROUPS; i++) {
        if (ea->side[i]) {
            cudaStreamSynchronize(ea->side[i]);
            cudaStreamDestroy(ea->side[i]);
        }
        if (ea->join[i]) cudaEventDestroy(ea->join[i]);
        ea->side[i] = nullptr;
        ea->join[i] = nullptr;
    }
    if (ea->fork) cudaEventDestroy(ea->fork);
    ea->fork = nullptr;
    return KFAC_OK;
}

// Group 0 on s, groups 1.. on the side streams, forked from s and joined back
// into it (captured with s when s is capturing).
static kfac_status_t eigall_run(kfac_pinn_handle* h, EigAll* ea, cudaStream_t s) {
    if (ea->ng == 1) return group_run(h, ea->g[0], s);
    bool coop = false;
    for (int i = 0; i < ea->ng; i++) coop = coop || ea->g[i]->trc_cl == 0;
    if (coop) {
        // a cooperative tridiagonalisation needs all its CTAs resident at
        // once: nothing runs beside it
        for (int i = ea->ng - 1; i >= 0; i--) KFAC_TRY(group_run(h, ea->g[i], s));
        return KFAC_OK;
    }
    KFAC_CUDA_TRY(cudaEventRecord(ea->fork, s));
    kfac_status_t st = KFAC_OK;
    for (int i = 1; i < ea->ng; i++) {
        KFAC_CUDA_TRY(cudaStreamWaitEvent(ea->side[i - 1], ea->fork, 0));
        if (st == KFAC_OK) st = group_run(h, ea->g[i], ea->side[i - 1]);
        // the joins are recorded even after an error so that s never runs ahead of a side stream
        KFAC_CUDA_TRY(cudaEventRecord(ea->join[i - 1], ea->side[i - 1]));
    }
    if (st == KFAC_OK) st = group_run(h, ea->g[0], s);
    for (int i = 1; i < ea->ng; i++) KFAC_CUDA_TRY(cudaStreamWaitEvent(s, ea->join[i - 1], 0));
    return st;
}

kfac_status_t eig_run(kfac_pinn_handle* h, cudaStream_t s) { return eigall_run(h, EA(h), s); }

// The eigensolves of many handles at once over the problems' own workspaces:
// every factor pair of every handle, one group per cluster size as for a
// single handle (a problem is solved by the same kernels with the same cluster
// size as in its own handle's eigensolve).  Dealing a size's problems over
// several groups on more streams was measured 2 % faster for the 64-problem
// batch at twice the launches, and is not done.
kfac_status_t eig_batch_alloc(kfac_pinn_handle* const* hs, int count, void** out) {
    *out = nullptr;
    if (count < 1) return KFAC_BAD_ARG;
    std::map<int, std::vector<Prob>> byclass;
    for (int i = 0; i < count; i++) {
        EigAll* ea = EA(hs[i]);
        if (!ea) return KFAC_BAD_ARG;
        for (int g = 0; g < ea->ng; g++)
            for (const Prob& p : ea->g[g]->host) byclass[class_rank(pair_class(p.n, hs[0]))].push_back(p);
    }
    if ((int)byclass.size() > MAX_GROUPS) return KFAC_BAD_ARG;
    EigAll* ea = new EigAll();
    memset(ea, 0, sizeof(*ea));
    *out = ea;
    kfac_status_t st;
    for (auto& kv : byclass) {
        EigState* es = new EigState();
        ea->g[ea->ng++] = es;
        es->host = kv.second;
        if ((st = group_schedule(hs[0], es))) return st;
    }
    return eigall_streams(ea);
}

kfac_status_t eig_batch_run(kfac_pinn_handle* h0, void* eb, cudaStream_t s) {
    return eigall_run(h0, (EigAll*)eb, s);
}

void eig_batch_free(void* eb) { eigall_free((EigAll*)eb); }
