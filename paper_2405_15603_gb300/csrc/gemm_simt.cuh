// Tiled SIMT GEMM with operand accessors (the FP64 and FP32 SIMT paths and
// the linear algebra).
//
// C(p, q) = sum_k A(p, k) B(k, q).  The operands are read through small
// accessor structs so that one kernel serves the layer GEMMs, the adjoint
// GEMMs, the factor Grams (with the implicit bias column of T^) and the
// weight gradient (with per-row residual weights).  64 x 64 output tile,
// 16-deep k slices staged in shared memory, 256 threads with a 4 x 4
// register block each; the grid's z dimension splits k (split-K partials).
//
// Each accessor declares which index is contiguous in memory so that the
// tile loads are coalesced:  A accessors set kfast (consecutive k adjacent),
// B accessors set qfast (consecutive q adjacent).
#pragma once
#include "kfac_internal.cuh"

namespace kfac {

constexpr int GT = 64;     // output tile edge
constexpr int GK = 16;     // k slice
constexpr int GTHREADS = 256;

// Plain strided operand: X[i * si + j * sj] (T: the storage type)
template <bool FAST_SECOND, class T = double>
struct Strided {
    const T* X;
    long long si, sj;
    static constexpr bool kfast = FAST_SECOND;   // as A(p, k): second index fast
    static constexpr bool qfast = FAST_SECOND;   // as B(k, q): second index fast
    KFAC_DEV T operator()(int i, int j) const { return X[(long long)i * si + (long long)j * sj]; }
};

// Rows of an activation block with the implicit bias column:
// element (row, q) = T[row*h + q] for q < h, and for q == h the bias entry,
// 1 on the value rows (row < N) and 0 elsewhere (the appended row of T^).
template <class T = double>
struct ActRows {
    const T* X;
    int h, N;
    static constexpr bool qfast = true;
    KFAC_DEV T operator()(int row, int q) const {
        if (q < h) return X[(long long)row * h + q];
        return row < N ? T(1) : T(0);
    }
};

// The input matrix T^{(0)} of the first layer, never stored: per point the
// columns (x, v_1..v_d, 0) with bias row (1, 0, .., 0) (Sec. 3.1; v_m = e_m,
// or the coefficient matrix's eigenvectors for a general operator), in the
// column-block-major row order of the activations.
struct InputRows {
    const double* X;
    int d, N;
    const double* Q;    // tangent directions v_m = Q e_m (d x d row-major), nullptr: e_m
    static constexpr bool qfast = true;
    KFAC_DEV double operator()(int row, int q) const {
        int s = row / N, n = row - s * N;
        if (s == 0) return q < d ? X[(long long)n * d + q] : 1.0;
        if (s <= d) {
            if (q >= d) return 0.0;
            return Q ? Q[(long long)q * d + (s - 1)] : (q == s - 1 ? 1.0 : 0.0);
        }
        return 0.0;
    }
};

// Adjoint rows scaled by a per-point weight w[row % N] (w == nullptr: 1).
template <class T = double>
struct WeightedRows {
    const T* G;
    int h, N;
    const double* w;
    static constexpr bool qfast = true;
    KFAC_DEV T operator()(int row, int i) const {
        T v = G[(long long)row * h + i];
        if (w) v *= (T)w[row % N];
        return v;
    }
};

// A(p, k) = R(k, p): contraction over the rows of R (Gram / weight gradient).
template <class R>
struct Transposed {
    R r;
    static constexpr bool kfast = !R::qfast;
    KFAC_DEV auto operator()(int p, int k) const { return r(k, p); }
};

// Epilogue writing split-K partials: part[z][p][q]
struct EpPartial {
    double* part;
    int P, Q;
    KFAC_DEV void operator()(int p, int q, int z, double v) const {
        part[((long long)z * P + p) * Q + q] = v;
    }
};

// Epilogue: C[p*sp + q*sq] = alpha * v + beta * C  (+ bias[q] on rows p < bias_rows)
template <class T = double>
struct EpStore {
    T* C;
    long long sp, sq;
    double alpha, beta;
    const double* bias;
    long long bias_stride;
    int bias_rows;
    KFAC_DEV void operator()(int p, int q, int, double v) const {
        long long o = (long long)p * sp + (long long)q * sq;
        double r = alpha * v;
        if (beta != 0.0) r += beta * (double)C[o];
        if (bias && p < bias_rows) r += bias[(long long)q * bias_stride];
        C[o] = (T)r;
    }
};

// Acc is the arithmetic type of the tile (double, or float where the caller
// accepts FP32 products: the FP32 path and the FP32 preconditioning); operands
// are read through their accessors and converted.
template <class Acc, class LA, class LB, class EP>
__global__ void __launch_bounds__(GTHREADS)
dgemm_tile_kernel(int P, int Q, int K, int kchunk, LA la, LB lb, EP ep) {
    __shared__ Acc As[GK][GT + 1];
    __shared__ Acc Bs[GK][GT + 1];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int p0 = blockIdx.y * GT, q0 = blockIdx.x * GT;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    Acc acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = Acc(0);

    for (int k0 = kbeg; k0 < kend; k0 += GK) {
#pragma unroll
        for (int i = 0; i < (GT * GK) / GTHREADS; i++) {
            int e = tid + GTHREADS * i;
            int pp, kk;
            if (LA::kfast) { kk = e % GK; pp = e / GK; } else { pp = e % GT; kk = e / GT; }
            int p = p0 + pp, k = k0 + kk;
            As[kk][pp] = (p < P && k < kend) ? Acc(la(p, k)) : Acc(0);
        }
#pragma unroll
        for (int i = 0; i < (GT * GK) / GTHREADS; i++) {
            int e = tid + GTHREADS * i;
            int qq, kk;
            if (LB::qfast) { qq = e % GT; kk = e / GT; } else { kk = e % GK; qq = e / GK; }
            int q = q0 + qq, k = k0 + kk;
            Bs[kk][qq] = (q < Q && k < kend) ? Acc(lb(k, q)) : Acc(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; kk++) {
            Acc a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int p = p0 + ty + 16 * i, q = q0 + tx + 16 * j;
            if (p < P && q < Q) ep(p, q, blockIdx.z, (double)acc[i][j]);
        }
}

// Launch with an explicit number of k splits (>= 1).
template <class LA, class LB, class EP, class Acc = double>
inline cudaError_t launch_dgemm(cudaStream_t s, int P, int Q, int K, int splits, LA la, LB lb, EP ep) {
    if (P <= 0 || Q <= 0) return cudaSuccess;
    if (splits < 1) splits = 1;
    int kchunk = (K + splits - 1) / splits;
    kchunk = ((kchunk + GK - 1) / GK) * GK;
    if (kchunk < GK) kchunk = GK;
    splits = (K + kchunk - 1) / kchunk;
    if (splits < 1) splits = 1;
    dim3 grid(ceil_div_u(Q, GT), ceil_div_u(P, GT), splits);
    dgemm_tile_kernel<Acc><<<grid, GTHREADS, 0, s>>>(P, Q, K, kchunk, la, lb, ep);
    return cudaGetLastError();
}

// Number of k splits so that the grid fills the GPU about `waves` times,
// each split covering at least `min_k` of the contraction.
inline int choose_splits(int P, int Q, int K, int sm_count, int waves = 2, int min_k = 512) {
    long long tiles = (long long)ceil_div_u(P, GT) * ceil_div_u(Q, GT);
    long long want = ((long long)sm_count * waves + tiles - 1) / tiles;
    long long maxs = (K + min_k - 1) / min_k;
    if (want > maxs) want = maxs;
    if (want < 1) want = 1;
    return (int)want;
}

}  // namespace kfac
